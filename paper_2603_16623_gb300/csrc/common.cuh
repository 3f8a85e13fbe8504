// common.cuh -- device utilities of the wake solver: float-float arithmetic,
// the two precision policies, and block-wide scans for associative (not
// necessarily commutative) operators in either direction.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gbwake {

// control words of a wake (device ints): next slice, status, failing
// slice, ring-state buffer, AB2 history present; CTL_T_BEGIN and CTL_T_END
// (two words each) the device time (globaltimer ns) at which the last march
// launch began and finished marching the wake
enum { CTL_NEXT = 0, CTL_STATUS = 1, CTL_FAIL = 2, CTL_BUF = 3, CTL_PREV = 4, CTL_T_BEGIN = 8, CTL_T_END = 10,
       CTL_N = 16 };
// the wake status codes the kernels write into CTL_STATUS (the values of
// include/wake.h's WAKE_EINVAL, WAKE_ENONFINITE, WAKE_ETIMEOUT)
enum { WAKE_STATUS_INVALID = 1, WAKE_STATUS_NONFINITE = 4, WAKE_STATUS_TIMEOUT = 5 };

// ---------------------------------------------------------------------------
// float-float ("ff"): an unevaluated sum hi + lo of two floats (~48-bit
// significand).  Knuth's TwoSum and the FMA-based exact product; nothing here
// multiplies and adds in one expression except through fmaf.
// ---------------------------------------------------------------------------
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {  // |a| >= |b|
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = ff_two_sum(a.hi, b.hi);
    ff t = ff_two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = ff_fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return ff_fast_two_sum(s.hi, s.lo);
}
// Accumulation add ("sloppy" float-float add): the error stays ~2^-46 of
// |a| + |b|; used where a running sum meets one more term.
__device__ __forceinline__ ff ff_acc(ff a, ff b) {
    ff s = ff_two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return ff_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    ff s = ff_two_sum(a.hi, b);
    s.lo = __fadd_rn(s.lo, a.lo);
    return ff_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    float p = __fmul_rn(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ float ff_to_f(ff a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ ff ff_from_d(double d) {
    float h = (float)d;
    return {h, (float)(d - (double)h)};
}

// ---------------------------------------------------------------------------
// precision policies
//   PrecF64   : everything in double (the plain path)
//   PrecMixed : state, pushes and field evaluation in float; radial prefix
//               sums, psi and d_rho psi assembled in float-float
// ---------------------------------------------------------------------------
struct PrecF64 {
    using R = double;
    using A = double;
};
struct PrecMixed {
    using R = float;
    using A = ff;
};

// accumulator helpers, overloaded on the accumulator type
__device__ __forceinline__ double acc_zero(double) { return 0.0; }
__device__ __forceinline__ ff acc_zero(ff) { return {0.f, 0.f}; }
__device__ __forceinline__ double acc_add(double a, double b) { return a + b; }
__device__ __forceinline__ int64_t acc_add(int64_t a, int64_t b) { return a + b; }
// accumulations and scans of float-float values use the accumulation add
// (its error stays ~2^-46 of the operands' magnitudes)
__device__ __forceinline__ ff acc_add(ff a, ff b) { return ff_acc(a, b); }
__device__ __forceinline__ double acc_sub(double a, double b) { return a - b; }
__device__ __forceinline__ ff acc_sub(ff a, ff b) { return ff_sub(a, b); }
__device__ __forceinline__ double acc_add_r(double a, double b) { return a + b; }
__device__ __forceinline__ ff acc_add_r(ff a, float b) { return ff_add_f(a, b); }
__device__ __forceinline__ double acc_mul_r(double a, double b) { return a * b; }
__device__ __forceinline__ ff acc_mul_r(ff a, float b) { return ff_mul_f(a, b); }
__device__ __forceinline__ double acc_to_r(double a) { return a; }
__device__ __forceinline__ float acc_to_r(ff a) { return ff_to_f(a); }
__device__ __forceinline__ double acc_from_d(double d, double) { return d; }
__device__ __forceinline__ ff acc_from_d(double d, ff) { return ff_from_d(d); }
// exact square of a real as an accumulator
__device__ __forceinline__ double acc_sq(double x) { return x * x; }
__device__ __forceinline__ ff acc_sq(float x) { return ff_two_prod(x, x); }

__device__ __forceinline__ double real_log(double x) { return log(x); }
__device__ __forceinline__ float real_log(float x) { return logf(x); }
__device__ __forceinline__ bool real_finite(double x) { return isfinite(x); }
__device__ __forceinline__ bool real_finite(float x) { return isfinite(x); }

// ---------------------------------------------------------------------------
// shuffles for the scanned types
// ---------------------------------------------------------------------------
__device__ __forceinline__ double shfl_up_t(double v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_dn_t(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ int64_t shfl_up_t(int64_t v, int o) {
    return (int64_t)__shfl_up_sync(0xffffffffu, (long long)v, o);
}
__device__ __forceinline__ int64_t shfl_dn_t(int64_t v, int o) {
    return (int64_t)__shfl_down_sync(0xffffffffu, (long long)v, o);
}
__device__ __forceinline__ float shfl_up_t(float v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float shfl_dn_t(float v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ ff shfl_up_t(ff v, int o) { return {shfl_up_t(v.hi, o), shfl_up_t(v.lo, o)}; }
__device__ __forceinline__ ff shfl_dn_t(ff v, int o) { return {shfl_dn_t(v.hi, o), shfl_dn_t(v.lo, o)}; }
__device__ __forceinline__ double shfl_idx_t(double v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ float shfl_idx_t(float v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ int64_t shfl_idx_t(int64_t v, int l) {
    return (int64_t)__shfl_sync(0xffffffffu, (long long)v, l);
}
__device__ __forceinline__ ff shfl_idx_t(ff v, int l) { return {shfl_idx_t(v.hi, l), shfl_idx_t(v.lo, l)}; }

template <class T>
struct Pair {
    T x, y;
};
template <class T>
__device__ __forceinline__ Pair<T> shfl_up_t(Pair<T> v, int o) { return {shfl_up_t(v.x, o), shfl_up_t(v.y, o)}; }
template <class T>
__device__ __forceinline__ Pair<T> shfl_dn_t(Pair<T> v, int o) { return {shfl_dn_t(v.x, o), shfl_dn_t(v.y, o)}; }
template <class T>
__device__ __forceinline__ Pair<T> shfl_idx_t(Pair<T> v, int l) { return {shfl_idx_t(v.x, l), shfl_idx_t(v.y, l)}; }

// two accumulators and an integer count scanned together
template <class T>
struct Trip {
    T x, y;
    int64_t c;
};
template <class T>
__device__ __forceinline__ Trip<T> shfl_up_t(Trip<T> v, int o) {
    return {shfl_up_t(v.x, o), shfl_up_t(v.y, o), shfl_up_t(v.c, o)};
}
template <class T>
__device__ __forceinline__ Trip<T> shfl_dn_t(Trip<T> v, int o) {
    return {shfl_dn_t(v.x, o), shfl_dn_t(v.y, o), shfl_dn_t(v.c, o)};
}
template <class T>
__device__ __forceinline__ Trip<T> shfl_idx_t(Trip<T> v, int l) {
    return {shfl_idx_t(v.x, l), shfl_idx_t(v.y, l), shfl_idx_t(v.c, l)};
}

// 2x2 matrix and the affine map x -> M x + c
template <class R>
struct Mat2 {
    R m00, m01, m10, m11;
};
template <class R>
struct Aff2 {
    R m00, m01, m10, m11, c0, c1;
};
template <class R>
__device__ __forceinline__ Mat2<R> shfl_up_t(Mat2<R> v, int o) {
    return {shfl_up_t(v.m00, o), shfl_up_t(v.m01, o), shfl_up_t(v.m10, o), shfl_up_t(v.m11, o)};
}
template <class R>
__device__ __forceinline__ Mat2<R> shfl_dn_t(Mat2<R> v, int o) {
    return {shfl_dn_t(v.m00, o), shfl_dn_t(v.m01, o), shfl_dn_t(v.m10, o), shfl_dn_t(v.m11, o)};
}
template <class R>
__device__ __forceinline__ Mat2<R> shfl_idx_t(Mat2<R> v, int l) {
    return {shfl_idx_t(v.m00, l), shfl_idx_t(v.m01, l), shfl_idx_t(v.m10, l), shfl_idx_t(v.m11, l)};
}
template <class R>
__device__ __forceinline__ Aff2<R> shfl_up_t(Aff2<R> v, int o) {
    return {shfl_up_t(v.m00, o), shfl_up_t(v.m01, o), shfl_up_t(v.m10, o),
            shfl_up_t(v.m11, o), shfl_up_t(v.c0, o), shfl_up_t(v.c1, o)};
}
template <class R>
__device__ __forceinline__ Aff2<R> shfl_dn_t(Aff2<R> v, int o) {
    return {shfl_dn_t(v.m00, o), shfl_dn_t(v.m01, o), shfl_dn_t(v.m10, o),
            shfl_dn_t(v.m11, o), shfl_dn_t(v.c0, o), shfl_dn_t(v.c1, o)};
}

// ---------------------------------------------------------------------------
// operators: op(a, b) = "a, then b" where a covers the earlier elements of
// the scan order
// ---------------------------------------------------------------------------
struct OpAdd {
    template <class T>
    __device__ __forceinline__ T operator()(T a, T b) const { return acc_add(a, b); }
};
struct OpAddPair {
    template <class T>
    __device__ __forceinline__ Pair<T> operator()(Pair<T> a, Pair<T> b) const {
        return {acc_add(a.x, b.x), acc_add(a.y, b.y)};
    }
};
struct OpAddTrip {
    template <class T>
    __device__ __forceinline__ Trip<T> operator()(Trip<T> a, Trip<T> b) const {
        return {acc_add(a.x, b.x), acc_add(a.y, b.y), a.c + b.c};
    }
};
// matrix product, later element on the left: result = b * a
struct OpMatLeft {
    template <class R>
    __device__ __forceinline__ Mat2<R> operator()(Mat2<R> a, Mat2<R> b) const {
        return {b.m00 * a.m00 + b.m01 * a.m10, b.m00 * a.m01 + b.m01 * a.m11,
                b.m10 * a.m00 + b.m11 * a.m10, b.m10 * a.m01 + b.m11 * a.m11};
    }
};
// composition of affine maps, a applied first: x -> Mb (Ma x + ca) + cb
struct OpAffThen {
    template <class R>
    __device__ __forceinline__ Aff2<R> operator()(Aff2<R> a, Aff2<R> b) const {
        return {b.m00 * a.m00 + b.m01 * a.m10, b.m00 * a.m01 + b.m01 * a.m11,
                b.m10 * a.m00 + b.m11 * a.m10, b.m10 * a.m01 + b.m11 * a.m11,
                b.m00 * a.c0 + b.m01 * a.c1 + b.c0, b.m10 * a.c0 + b.m11 * a.c1 + b.c1};
    }
};

// ---------------------------------------------------------------------------
// block-wide exclusive scan.  REV = false: thread order 0, 1, ...;
// REV = true: the scan runs from the last thread down.  blockDim.x must be a
// multiple of 32 (<= 1024).  sbuf must hold 33 values of T in shared memory.
// Returns the exclusive fold of the earlier threads' values; `total` gets the
// fold over the whole block.  Contains barriers: every thread must call.
// ---------------------------------------------------------------------------
template <bool REV, class T, class Op>
__device__ __forceinline__ T warp_incl_scan(T v, Op op) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        T o = REV ? shfl_dn_t(v, off) : shfl_up_t(v, off);
        bool take = REV ? (lane + off < 32) : (lane >= off);
        if (take) v = op(o, v);
    }
    return v;
}

template <bool REV, class T, class Op>
__device__ T block_excl_scan(T v, Op op, T ident, T* sbuf, T& total) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    T inc = warp_incl_scan<REV>(v, op);
    T lex = REV ? shfl_dn_t(inc, 1) : shfl_up_t(inc, 1);
    if (REV ? (lane == 31) : (lane == 0)) lex = ident;
    if (REV ? (lane == 0) : (lane == 31)) sbuf[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T wv = lane < nw ? sbuf[lane] : ident;
        T winc = warp_incl_scan<REV>(wv, op);
        T wex = REV ? shfl_dn_t(winc, 1) : shfl_up_t(winc, 1);
        if (REV ? (lane == 31) : (lane == 0)) wex = ident;
        __syncwarp();
        if (lane < nw) sbuf[lane] = wex;
        if (lane == (REV ? 0 : 31)) sbuf[32] = winc;
    }
    __syncthreads();
    T res = op(sbuf[warp], lex);
    total = sbuf[32];
    __syncthreads();
    return res;
}

// One pass of two sums in opposite directions: fx scanned from thread 0 up,
// ry from the last thread down (same barriers as one scan).  Returns the
// exclusive forward sum of fx and the exclusive reverse (suffix) sum of ry;
// totals in tx, ty.  sbuf holds 33 Pair<T>.
template <class T>
__device__ Pair<T> block_excl_scan_fwd_rev(T fx, T ry, T zero, Pair<T>* sbuf, T& tx, T& ty) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    T ix = warp_incl_scan<false>(fx, OpAdd());
    T iy = warp_incl_scan<true>(ry, OpAdd());
    T ex = shfl_up_t(ix, 1), ey = shfl_dn_t(iy, 1);
    if (lane == 0) ex = zero;
    if (lane == 31) ey = zero;
    if (lane == 31) sbuf[warp].x = ix;
    if (lane == 0) sbuf[warp].y = iy;
    __syncthreads();
    if (warp == 0) {
        T wx = lane < nw ? sbuf[lane].x : zero;
        T wy = lane < nw ? sbuf[lane].y : zero;
        T sx = warp_incl_scan<false>(wx, OpAdd());
        T sy = warp_incl_scan<true>(wy, OpAdd());
        T qx = shfl_up_t(sx, 1), qy = shfl_dn_t(sy, 1);
        if (lane == 0) qx = zero;
        if (lane == 31) qy = zero;
        __syncwarp();
        if (lane < nw) {
            sbuf[lane].x = qx;
            sbuf[lane].y = qy;
        }
        if (lane == 31) sbuf[32].x = sx;
        if (lane == 0) sbuf[32].y = sy;
    }
    __syncthreads();
    Pair<T> res = {acc_add(sbuf[warp].x, ex), acc_add(sbuf[warp].y, ey)};
    tx = sbuf[32].x;
    ty = sbuf[32].y;
    __syncthreads();
    return res;
}

// Forward product scan of mf and reverse product scan of mr in one pass
// (op: later element on the left).  sbuf holds 33 Pair<Mat2<R>>.  With
// TOT, tf and tr receive the block's forward and reverse products.
template <bool TOT, class R>
__device__ __forceinline__ void block_excl_scan_mat_fwd_rev_t(Mat2<R> mf, Mat2<R> mr, Pair<Mat2<R>>* sbuf,
                                                              Mat2<R>& ef, Mat2<R>& er, Mat2<R>& tf, Mat2<R>& tr) {
    const Mat2<R> I2 = {1, 0, 0, 1};
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    Mat2<R> ix = warp_incl_scan<false>(mf, OpMatLeft());
    Mat2<R> iy = warp_incl_scan<true>(mr, OpMatLeft());
    Mat2<R> ex = shfl_up_t(ix, 1), ey = shfl_dn_t(iy, 1);
    if (lane == 0) ex = I2;
    if (lane == 31) ey = I2;
    if (lane == 31) sbuf[warp].x = ix;
    if (lane == 0) sbuf[warp].y = iy;
    __syncthreads();
    if (warp == 0) {
        Mat2<R> wx = lane < nw ? sbuf[lane].x : I2;
        Mat2<R> wy = lane < nw ? sbuf[lane].y : I2;
        Mat2<R> sx = warp_incl_scan<false>(wx, OpMatLeft());
        Mat2<R> sy = warp_incl_scan<true>(wy, OpMatLeft());
        Mat2<R> qx = shfl_up_t(sx, 1), qy = shfl_dn_t(sy, 1);
        if (lane == 0) qx = I2;
        if (lane == 31) qy = I2;
        __syncwarp();
        if (lane < nw) {
            sbuf[lane].x = qx;
            sbuf[lane].y = qy;
        }
        if (lane == 31) sbuf[32].x = sx;
        if (lane == 0) sbuf[32].y = sy;
    }
    __syncthreads();
    ef = OpMatLeft()(sbuf[warp].x, ex);
    er = OpMatLeft()(sbuf[warp].y, ey);
    if (TOT) {
        tf = sbuf[32].x;
        tr = sbuf[32].y;
    }
    __syncthreads();
}

template <class R>
__device__ void block_excl_scan_mat_fwd_rev(Mat2<R> mf, Mat2<R> mr, Pair<Mat2<R>>* sbuf, Mat2<R>& ef,
                                            Mat2<R>& er) {
    Mat2<R> tf, tr;
    block_excl_scan_mat_fwd_rev_t<false>(mf, mr, sbuf, ef, er, tf, tr);
}

// One-barrier forms of the three block scans above, with the same
// arithmetic in the same order (bitwise the same results): every warp scans
// the warp totals itself instead of warp 0 scanning them between two more
// barriers.  sbuf needs nw (not 33) values; every warp reads it after the
// one barrier, so it must not be written again before a later barrier:
// consecutive calls without a barrier between them alternate two buffers.
template <bool REV, class T, class Op>
__device__ __forceinline__ T block_excl_scan1(T v, Op op, T ident, T* sbuf, T& total) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    T inc = warp_incl_scan<REV>(v, op);
    T lex = REV ? shfl_dn_t(inc, 1) : shfl_up_t(inc, 1);
    if (REV ? (lane == 31) : (lane == 0)) lex = ident;
    if (REV ? (lane == 0) : (lane == 31)) sbuf[warp] = inc;
    __syncthreads();
    T wv = lane < nw ? sbuf[lane] : ident;
    T winc = warp_incl_scan<REV>(wv, op);
    T wex = REV ? shfl_dn_t(winc, 1) : shfl_up_t(winc, 1);
    if (REV ? (lane == 31) : (lane == 0)) wex = ident;
    total = shfl_idx_t(winc, REV ? 0 : 31);
    return op(shfl_idx_t(wex, warp), lex);
}

template <class T>
__device__ __forceinline__ Pair<T> block_excl_scan_fwd_rev1(T fx, T ry, T zero, Pair<T>* sbuf, T& tx, T& ty) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    T ix = warp_incl_scan<false>(fx, OpAdd());
    T iy = warp_incl_scan<true>(ry, OpAdd());
    T ex = shfl_up_t(ix, 1), ey = shfl_dn_t(iy, 1);
    if (lane == 0) ex = zero;
    if (lane == 31) ey = zero;
    if (lane == 31) sbuf[warp].x = ix;
    if (lane == 0) sbuf[warp].y = iy;
    __syncthreads();
    T wx = lane < nw ? sbuf[lane].x : zero;
    T wy = lane < nw ? sbuf[lane].y : zero;
    T sx = warp_incl_scan<false>(wx, OpAdd());
    T sy = warp_incl_scan<true>(wy, OpAdd());
    T qx = shfl_up_t(sx, 1), qy = shfl_dn_t(sy, 1);
    if (lane == 0) qx = zero;
    if (lane == 31) qy = zero;
    tx = shfl_idx_t(sx, 31);
    ty = shfl_idx_t(sy, 0);
    return {acc_add(shfl_idx_t(qx, warp), ex), acc_add(shfl_idx_t(qy, warp), ey)};
}

template <bool TOT, class R>
__device__ __forceinline__ void block_excl_scan_mat_fwd_rev1(Mat2<R> mf, Mat2<R> mr, Pair<Mat2<R>>* sbuf,
                                                             Mat2<R>& ef, Mat2<R>& er, Mat2<R>& tf, Mat2<R>& tr) {
    const Mat2<R> I2 = {1, 0, 0, 1};
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    Mat2<R> ix = warp_incl_scan<false>(mf, OpMatLeft());
    Mat2<R> iy = warp_incl_scan<true>(mr, OpMatLeft());
    Mat2<R> ex = shfl_up_t(ix, 1), ey = shfl_dn_t(iy, 1);
    if (lane == 0) ex = I2;
    if (lane == 31) ey = I2;
    if (lane == 31) sbuf[warp].x = ix;
    if (lane == 0) sbuf[warp].y = iy;
    __syncthreads();
    Mat2<R> wx = lane < nw ? sbuf[lane].x : I2;
    Mat2<R> wy = lane < nw ? sbuf[lane].y : I2;
    Mat2<R> sx = warp_incl_scan<false>(wx, OpMatLeft());
    Mat2<R> sy = warp_incl_scan<true>(wy, OpMatLeft());
    Mat2<R> qx = shfl_up_t(sx, 1), qy = shfl_dn_t(sy, 1);
    if (lane == 0) qx = I2;
    if (lane == 31) qy = I2;
    ef = OpMatLeft()(shfl_idx_t(qx, warp), ex);
    er = OpMatLeft()(shfl_idx_t(qy, warp), ey);
    if (TOT) {
        tf = shfl_idx_t(sx, 31);
        tr = shfl_idx_t(sy, 0);
    }
}

// first index i in [0, n) with a[i] >= x (n if none)
template <class R>
__device__ __forceinline__ int lower_bound_dev(const R* a, int n, R x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

}  // namespace gbwake
