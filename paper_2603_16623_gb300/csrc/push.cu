// push.cu -- the beam push between two wake solves.
//
// The wake of a slice acts on the beam particles of that slice; after a
// full solve every beam particle has its E_z, W_r = E_r - B_theta and
// B_theta.  Between solves the beam moves over a time step dt in these
// fields (Sec. V: the paper's code uses the Boris method or fourth-order
// Runge-Kutta; this is the Boris method), in normalised units: time
// 1/omega_p, lengths 1/k_p, momenta u = p/(m c), fields m c omega_p/e, and
// beam particles of electron mass with charge q = -1 or +1.  The fields
// are axisymmetric: at (x, y), r = |(x, y)|, E = (E_r x/r, E_r y/r, E_z),
// B = (-B_theta y/r, B_theta x/r, 0) (zero transverse parts on the axis).
// One step per particle, h = q dt / 2:
//   u- = u + h E;  t = h B / gamma(u-);  s = 2 t / (1 + t.t)
//   u+ = u- + (u- + u- x t) x s;  u' = u+ + h E
//   x' = x + dt u'_xy / gamma(u');  xi' = xi + dt (1 - u'_z / gamma(u'))
// (xi = c t - z grows towards the back of the co-moving window), and the
// radius the next solve bins by, r' = |(x', y')|.  1 - u_z/gamma is taken
// as (1 + u_x^2 + u_y^2) / (gamma (gamma + u_z)), the same number without
// the cancellation of two nearly equal terms at gamma >> 1.
//
// Two arithmetics.  FP64 wakes push in FP64 throughout.  Mixed wakes (FP32
// fields) keep the phase space in FP64 but take every increment in FP32:
// this GPU runs FP64 (conversions included) at about 1/64 of the FP32 rate,
// and a push in FP64 is bound by that, ~20x slower than its HBM traffic.
// The mixed push does six FP64 additions (state += increment) and one for
// r; its float <-> double conversions are done on the bit fields with
// integer instructions.  Increments carry FP32 rounding (~1e-7 relative to
// themselves); the state keeps FP64 resolution.
#include <cuda_runtime.h>
#include <stdint.h>

#include "push.h"

namespace gbwake {

namespace {

// double -> float, truncating the fraction; |d| below the float normal
// range gives +-0, above it (or NaN) +-inf
__device__ __forceinline__ float f64_to_f32(double d) {
    const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
    const uint32_t sign = hi & 0x80000000u;
    const int32_t e = (int32_t)((hi >> 20) & 0x7ffu) - 1023 + 127;
    uint32_t f = sign | ((uint32_t)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    f = e <= 0 ? sign : f;
    f = e >= 255 ? (sign | 0x7f800000u) : f;
    return __uint_as_float(f);
}

// float -> double, exact for normal floats, +-inf and NaN; subnormal floats
// give +-0
__device__ __forceinline__ double f32_to_f64(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t sign = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    const uint32_t ed = e == 255u ? 2047u : e + 896u;
    const uint32_t hi = e == 0u ? sign : (sign | (ed << 20) | (m >> 3));
    const uint32_t lo = e == 0u ? 0u : (m << 29);
    return __hiloint2double((int)hi, (int)lo);
}

// d = hi + lo to ~2^-47 relative: hi its leading 24 significant bits, lo the
// next 23 (both 0 where |d| < 2^-80)
__device__ __forceinline__ void f64_split(double d, float& hi, float& lo) {
    hi = f64_to_f32(d);
    const uint32_t dh = (uint32_t)__double2hiint(d), dl = (uint32_t)__double2loint(d);
    const int32_t E = (int32_t)((dh >> 20) & 0x7ffu) - 1023;
    // the 29 fraction bits below hi's, top 23 of them: (dl & 2^29-1) >> 6
    const float rest = __uint_as_float(0x4b000000u | ((dl & 0x1fffffffu) >> 6)) - 8388608.0f;
    const int32_t se = E + 81;  // exponent field of 2^(E - 46)
    const float scale = (se >= 1 && se <= 254) ? __uint_as_float((uint32_t)se << 23) : 0.0f;
    const float mag = rest * scale;
    lo = (dh & 0x80000000u) ? -mag : mag;
}

// |(X, Y)| of two doubles to ~1e-14 relative, in float-float arithmetic
// (one Newton step on the float square root) and one FP64 addition
__device__ __forceinline__ double radius_ff(double X, double Y) {
    float hx, lx, hy, ly;
    f64_split(X, hx, lx);
    f64_split(Y, hy, ly);
    const float p1 = hx * hx, e1 = fmaf(hx, hx, -p1);
    const float p2 = hy * hy, e2 = fmaf(hy, hy, -p2);
    const float S = p1 + p2, bb = S - p1;
    const float err = (p1 - (S - bb)) + (p2 - bb);  // S + err = p1 + p2 exactly
    const float S_lo = err + e1 + e2 + 2.0f * (hx * lx + hy * ly);
    const float sr = sqrtf(S);
    const float d = fmaf(-sr, sr, S) + S_lo;
    const float corr = sr > 0.0f ? d * (0.5f / sr) : 0.0f;
    return f32_to_f64(sr) + f32_to_f64(corr);
}

// FP64 push of particle k
__device__ __forceinline__ void push_particle(const PushWake<double>& W, int64_t k, double h, double dt) {
    const int32_t p = W.inv[k];
    const double ez = p >= 0 ? W.ez[p] : 0.0;
    const double wr = p >= 0 ? W.wr[p] : 0.0;
    const double bt = p >= 0 ? W.bt[p] : 0.0;
    const double x = W.x[k], y = W.y[k];
    const double rr = hypot(x, y);
    const double ir = rr > 0.0 ? 1.0 / rr : 0.0;
    const double c = x * ir, sn = y * ir;
    const double er = wr + bt;
    const double ex = h * er * c, ey = h * er * sn, ezh = h * ez;  // h E
    const double bx = -h * bt * sn, by = h * bt * c;              // h B, B_z = 0
    const double mx = W.ux[k] + ex, my = W.uy[k] + ey, mz = W.uz[k] + ezh;
    const double igm = 1.0 / sqrt(1.0 + mx * mx + my * my + mz * mz);
    const double tx = bx * igm, ty = by * igm;  // t_z = 0
    const double f = 2.0 / (1.0 + tx * tx + ty * ty);
    const double sx = f * tx, sy = f * ty;
    // u' = u- + u- x t, u+ = u- + u' x s (t_z = s_z = 0)
    const double px = mx - mz * ty, py = my + mz * tx, pz = mz + (mx * ty - my * tx);
    const double nx = mx - pz * sy + ex, ny = my + pz * sx + ey, nz = mz + (px * sy - py * sx) + ezh;
    const double tp = 1.0 + nx * nx + ny * ny;
    const double g = sqrt(tp + nz * nz);
    const double ig = 1.0 / g;
    const double xn = x + dt * nx * ig, yn = y + dt * ny * ig;
    W.x[k] = xn;
    W.y[k] = yn;
    W.xi[k] = W.xi[k] + dt * tp * ig / (g + nz);
    W.ux[k] = nx;
    W.uy[k] = ny;
    W.uz[k] = nz;
    W.r[k] = hypot(xn, yn);
}

// mixed push of particle k: FP32 increments onto the FP64 state
__device__ __forceinline__ void push_particle(const PushWake<float>& W, int64_t k, double hd, double dt) {
    const float h = (float)hd;
    const float dtf = (float)dt;
    const int32_t p = W.inv[k];
    const float ez = p >= 0 ? W.ez[p] : 0.0f;
    const float wr = p >= 0 ? W.wr[p] : 0.0f;
    const float bt = p >= 0 ? W.bt[p] : 0.0f;
    const double X = W.x[k], Y = W.y[k], XI = W.xi[k], UX = W.ux[k], UY = W.uy[k], UZ = W.uz[k];
    const float x = f64_to_f32(X), y = f64_to_f32(Y);
    const float ux = f64_to_f32(UX), uy = f64_to_f32(UY), uz = f64_to_f32(UZ);
    const float r2 = x * x + y * y;
    const float ir = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
    const float c = x * ir, sn = y * ir;
    const float er = wr + bt;
    const float ex = h * er * c, ey = h * er * sn, ezh = h * ez;  // h E
    const float bx = -h * bt * sn, by = h * bt * c;              // h B, B_z = 0
    const float mx = ux + ex, my = uy + ey, mz = uz + ezh;
    const float igm = rsqrtf(1.0f + mx * mx + my * my + mz * mz);
    const float tx = bx * igm, ty = by * igm;  // t_z = 0
    const float f = 2.0f / (1.0f + tx * tx + ty * ty);
    const float sx = f * tx, sy = f * ty;
    const float px = mx - mz * ty, py = my + mz * tx, pz = mz + (mx * ty - my * tx);
    // whole momentum change: h E + u' x s + h E
    const float dux = 2.0f * ex - pz * sy, duy = 2.0f * ey + pz * sx, duz = 2.0f * ezh + (px * sy - py * sx);
    const float nx = ux + dux, ny = uy + duy, nz = uz + duz;
    const float tp = 1.0f + nx * nx + ny * ny;
    const float g = sqrtf(tp + nz * nz);
    const float ig = 1.0f / g;
    const float dx = dtf * nx * ig, dy = dtf * ny * ig;
    const float dxi = dtf * tp * ig / (g + nz);
    const double Xn = X + f32_to_f64(dx), Yn = Y + f32_to_f64(dy);
    W.x[k] = Xn;
    W.y[k] = Yn;
    W.xi[k] = XI + f32_to_f64(dxi);
    W.ux[k] = UX + f32_to_f64(dux);
    W.uy[k] = UY + f32_to_f64(duy);
    W.uz[k] = UZ + f32_to_f64(duz);
    W.r[k] = radius_ff(Xn, Yn);
}

constexpr int kPushThreads = 256;

template <class R>
__global__ void __launch_bounds__(kPushThreads) beam_push_kernel(const PushWake<R>* __restrict__ wakes,
                                                                 const PushItem* __restrict__ items, double dt) {
    const PushItem it = items[blockIdx.x];
    const PushWake<R> W = wakes[it.wake];
    const double h = 0.5 * it.q * dt;
    for (int64_t k = it.begin + threadIdx.x; k < it.end; k += kPushThreads) push_particle(W, k, h, dt);
}

__global__ void beam_radius_kernel(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                                   double* __restrict__ r) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        r[k] = hypot(x[k], y[k]);
}

}  // namespace

int64_t push_item_size(int64_t total) {
    // Small items: CTAs start in item order, so the resident ones (3 per SM
    // at 80 registers) cover ~1M particles, i.e. a few wakes, whose fields
    // (12 B per particle, gathered in random order through the sorted
    // position) then stay in L2 until every sector of them has been used.
    // Larger items spread the gathers over more wakes than L2 holds and turn
    // each 4-byte gather into a 32-byte DRAM sector.
    const int64_t per = (total + 152 * 8 - 1) / (152 * 8);
    int64_t c = (per + kPushThreads - 1) / kPushThreads * kPushThreads;
    if (c > 8 * kPushThreads) c = 8 * kPushThreads;
    return c < kPushThreads ? kPushThreads : c;
}

template <class R>
cudaError_t launch_beam_push(const PushWake<R>* wakes, const PushItem* items, int32_t n_items, double dt,
                             cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    beam_push_kernel<R><<<n_items, kPushThreads, 0, st>>>(wakes, items, dt);
    return cudaGetLastError();
}

cudaError_t launch_beam_radius(int64_t n, const double* x, const double* y, double* r, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    beam_radius_kernel<<<(int)g, 256, 0, st>>>(n, x, y, r);
    return cudaGetLastError();
}

template cudaError_t launch_beam_push<float>(const PushWake<float>*, const PushItem*, int32_t, double, cudaStream_t);
template cudaError_t launch_beam_push<double>(const PushWake<double>*, const PushItem*, int32_t, double,
                                              cudaStream_t);

}  // namespace gbwake
