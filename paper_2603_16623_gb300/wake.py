"""Python binding of libwake.so (include/wake.h): argument marshalling only.

The functions keep the C names (wake_init, wake_step_slices, wake_fields_at,
wake_get_beam_fields, wake_run, wake_batch_run, ...); `Wake` wraps a handle.
Every step of the solve runs in the library's CUDA kernels: if the library
cannot be loaded (not built, no CUDA runtime) the import of the handle-level
API raises -- there is no CPU fallback.

Host arrays are numpy; device arrays are torch CUDA tensors (their
data_ptr() is passed with device_ptrs=1).  Outputs are float64 for
precision "fp64" and float32 for "mixed".
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Iterable, List, Optional, Sequence

import numpy as np

from . import build as _build

WAKE_OK, WAKE_EINVAL, WAKE_ENOMEM, WAKE_ECUDA, WAKE_ENONFINITE, WAKE_ETIMEOUT, WAKE_EBUSY = range(7)
WAKE_FP64, WAKE_MIXED = 0, 1
WAKE_DUMP_RING_R, WAKE_DUMP_RING_FIELDS, WAKE_INIT_ASYNC, WAKE_TEST_STALL_STAGE, WAKE_NO_STAGE = 1, 2, 4, 8, 16
WAKE_STATIC_MAX_QUERIES = 65536  # queries per wake_fields_at_static call
PRECISION = {"fp64": WAKE_FP64, "mixed": WAKE_MIXED}
_STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENONFINITE", 5: "ETIMEOUT", 6: "EBUSY"}


class WakeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_dp = C.POINTER(C.c_double)


class wake_plasma_desc(C.Structure):
    _fields_ = [("n_rings", C.c_int32), ("r_edges", _dp), ("density", C.c_double), ("ion_charge", C.c_double),
                ("ion_mass", C.c_double), ("cell_density", _dp)]


class wake_beam_desc(C.Structure):
    _fields_ = [("n", C.c_int64), ("xi", _dp), ("r", _dp), ("w", _dp), ("q", C.c_double)]


class wake_config(C.Structure):
    _fields_ = [("dxi", C.c_double), ("n_steps", C.c_int32), ("precision", C.c_int32),
                ("flags", C.c_int32), ("block_threads", C.c_int32), ("rings_per_thread", C.c_int32),
                ("cluster_ctas", C.c_int32), ("integrator", C.c_int32), ("grid_nr", C.c_int32),
                ("grid_rmax", C.c_double)]


_vp = C.c_void_p
_SIGS = {
    "wake_init": ([C.POINTER(wake_config), C.POINTER(wake_plasma_desc), C.POINTER(wake_beam_desc), C.c_int32,
                   _vp, C.POINTER(_vp)], C.c_int),
    "wake_reset": ([_vp, C.POINTER(wake_beam_desc), C.c_int32], C.c_int),
    "wake_step_slices": ([_vp, C.c_int32], C.c_int),
    "wake_fields_at": ([_vp, C.c_int64, _vp, _vp, _vp, _vp, _vp, C.c_int32], C.c_int),
    "wake_get_beam_fields": ([_vp, _vp, _vp, _vp, _vp, C.c_int32], C.c_int),
    "wake_run": ([_vp, _vp, _vp, _vp], C.c_int),
    "wake_batch_run": ([C.c_int32, C.POINTER(_vp)], C.c_int),
    "wake_batch_reset": ([C.c_int32, C.POINTER(_vp), C.c_void_p, C.c_void_p], C.c_int),
    "wake_batch_step": ([C.c_int32, C.POINTER(_vp), C.c_int32, C.c_int64], C.c_int),
    "wake_batch_progress": ([C.c_int32, C.POINTER(_vp), C.c_void_p, C.c_void_p], C.c_int),
    "wake_get_device_bytes": ([_vp, C.POINTER(C.c_int64)], C.c_int),
    "wake_get_march_times": ([_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)], C.c_int),
    "wake_batch_get_beam_fields": ([C.c_int32, C.POINTER(_vp), C.c_void_p, C.c_void_p, C.c_int32], C.c_int),
    "wake_set_beam_phase_space": ([_vp, _vp, _vp, _vp, _vp, _vp], C.c_int),
    "wake_get_beam_phase_space": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], C.c_int),
    "wake_push_beam": ([_vp, C.c_double], C.c_int),
    "wake_batch_push_beam": ([C.c_int32, C.POINTER(_vp), C.c_double], C.c_int),
    "wake_batch_reset_run": ([C.c_int32, C.POINTER(_vp)], C.c_int),
    "wake_batch_solve": ([C.c_int32, C.POINTER(_vp), C.c_void_p, C.c_void_p], C.c_int),
    "wake_get_progress": ([_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)], C.c_int),
    "wake_get_ring_state": ([_vp, _vp, _vp, _vp, _vp], C.c_int),
    "wake_set_ring_state": ([_vp, C.c_int32, _vp, _vp, _vp, _vp], C.c_int),
    "wake_get_ring_dumps": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], C.c_int),
    "wake_get_launch_config": ([_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)], C.c_int),
    "wake_fields_at_static": ([_vp, C.c_int64, _vp, _vp, _vp, _vp, _vp], C.c_int),
    "wake_destroy": ([_vp], None),
    "wake_last_error": ([], C.c_char_p),
    "wake_max_rings": ([C.c_int32], C.c_int32),
    "wake_launch_shape": ([C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int32),
                           C.POINTER(C.c_int32), C.POINTER(C.c_int32)], C.c_int),
    "wake_launch_shape_latency": ([C.c_int32, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int32)], C.c_int),
    "wake_gm_launch_shape": ([C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int32),
                              C.POINTER(C.c_int32), C.POINTER(C.c_int32)], C.c_int),
    "wake_set_latency_shape_ms": ([C.c_double], C.c_int),
    "wake_get_latency_shape_ms": ([], C.c_double),
    "wake_max_slice_particles": ([C.c_int32], C.c_int64),
    "wake_measure_peaks": ([C.c_void_p], C.c_int),
    "wake_debug_bounds_violations": ([], C.c_int64),
}


class wake_peaks(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("fp32_tflops", "fp64_tflops", "mufu_lg2_tops", "smem_tbs",
                                          "fma_latency_cycles", "syncthreads_cycles", "syncthreads_ns",
                                          "cluster_barrier_cycles", "cluster_barrier_ns", "sm_clock_mhz")] + \
        [("sms", C.c_int32)]


def measure_peaks() -> Dict[str, float]:
    """On-chip peaks of the current GPU by the library's microbenchmarks
    (include/wake_peaks.h): FP32/FP64 FMA TFLOP/s, lg2 rate, shared-memory
    TB/s, FMA and barrier latencies, the SM clock seen meanwhile."""
    out = wake_peaks()
    rc = load().wake_measure_peaks(C.byref(out))
    if rc != 0:
        raise WakeError(WAKE_ECUDA, f"wake_measure_peaks failed ({rc})")
    return {k: getattr(out, k) for k, _ in wake_peaks._fields_}

_lib = None


def _bounds_check() -> bool:
    return os.environ.get("GBWAKE_BOUNDS_CHECK", "") == "1"


def lib_path() -> str:
    return _build.lib_for(_bounds_check())


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load libwake.so (building it first if needed; the bounds-checking
    debug build when GBWAKE_BOUNDS_CHECK=1).  Raises if it cannot be loaded:
    the solver has no other implementation."""
    global _lib
    if _lib is None:
        bc = _bounds_check()
        path = _build.lib_for(bc)
        if not os.path.exists(path) or not _build.up_to_date(bc):
            if not build_if_missing:
                raise OSError(f"{path} is missing; run python -m paper_2603_16623_gb300.build")
            _build.build(bounds_check=bc)
        lib = C.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _check(status: int):
    if status != WAKE_OK:
        msg = load().wake_last_error()
        raise WakeError(status, msg.decode() if msg else "")


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


class Wake:
    """One wake solve on the GPU (a wake_handle)."""

    def __init__(self, edges, beams: Sequence = (), dxi: float = 0.01, n_steps: int = 1000,
                 precision: str = "mixed", density: float = 1.0, flags: int = 0,
                 block_threads: int = 0, stream=None, rings_per_thread: int = 0, cluster_ctas: int = 0,
                 ions=None, cell_density=None, integrator: str = "ab2", grid_nr: int = 0,
                 grid_rmax: float = 0.0):
        """ions: None (immobile ion column) or (Z, M) for mobile ions (M =
        inf: ion rings that never move); the wake then has 2 x cells rings
        (electrons, then ions) in every per-ring array.  cell_density: a
        radial density profile, one value per cell (needs ions).  integrator:
        "ab2" or "rk4".  grid_nr > 0: beam fields through adaptive beam
        grids of grid_nr radial cells per beam; grid_rmax > 0 fixes their
        extent (the regular intermediate grid)."""
        lib = load()
        self.precision = precision
        self.dtype = np.float64 if precision == "fp64" else np.float32
        self.edges = _f64(edges)
        self.n_cells = self.edges.shape[0] - 1
        self.n_rings = self.n_cells if ions is None else 2 * self.n_cells
        self.n_steps = int(n_steps)
        self._keep = [self.edges]
        # beams: numpy arrays, or pinned float64 torch CPU tensors (uploaded
        # asynchronously: the caller keeps them alive until the stream has
        # passed wake_init's copies)
        descs, keep = _beam_descs(beams)
        self._keep += keep
        self.n_beam = int(sum(d.n for d in descs[:len(beams)]))
        cfg = wake_config(float(dxi), self.n_steps, PRECISION[precision], int(flags), int(block_threads),
                          int(rings_per_thread), int(cluster_ctas), {"ab2": 0, "rk4": 1}[integrator], int(grid_nr),
                          float(grid_rmax))
        z, m = (0.0, 0.0) if ions is None else (float(ions[0]), float(ions[1]))
        prof = None if cell_density is None else _f64(cell_density)
        self._keep.append(prof)
        plasma = wake_plasma_desc(self.n_cells, _dptr(self.edges), float(density), z, m,
                                  _dptr(prof) if prof is not None else None)
        if stream is None:
            stream = _default_stream()
        self.stream = stream
        h = _vp()
        _check(lib.wake_init(C.byref(cfg), C.byref(plasma), descs, len(beams), stream, C.byref(h)))
        self.handle = h
        self._keep = None

    @classmethod
    def from_workload(cls, wake, **kw) -> "Wake":
        kw.setdefault("ions", getattr(wake, "ions", None))
        kw.setdefault("cell_density", getattr(wake, "cell_density", None))
        kw.setdefault("integrator", getattr(wake, "integrator", "ab2"))
        kw.setdefault("grid_nr", getattr(wake, "grid_nr", 0))
        kw.setdefault("grid_rmax", getattr(wake, "grid_rmax", 0.0))
        return cls(wake.edges, wake.beams, wake.dxi, wake.n_steps, density=wake.density, **kw)

    def close(self):
        if getattr(self, "handle", None):
            load().wake_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, beams: Optional[Sequence] = None):
        """Back to slice 0 (a0/a1 redone on the device).  beams: None to keep
        the device-resident beams, else a sequence of objects with xi, r, w, q
        (numpy arrays, or pinned torch CPU tensors for asynchronous upload)."""
        if beams is None:
            _check(load().wake_reset(self.handle, None, 0))
            return
        descs, keep = _beam_descs(beams)
        _check(load().wake_reset(self.handle, descs, len(beams)))
        self._reset_keep = keep

    def step_slices(self, n: int):
        _check(load().wake_step_slices(self.handle, int(n)))

    def progress(self):
        nxt, st, fl = C.c_int32(), C.c_int32(), C.c_int32()
        _check(load().wake_get_progress(self.handle, C.byref(nxt), C.byref(st), C.byref(fl)))
        return nxt.value, st.value, fl.value

    def fields_at(self, r) -> Dict[str, np.ndarray]:
        """Fields at the current slice at host radii r (numpy)."""
        r = _f64(r)
        n = r.shape[0]
        out = {k: np.zeros(n, dtype=self.dtype) for k in ("ez", "wr", "bt", "psi")}
        _check(load().wake_fields_at(self.handle, n, r.ctypes.data, out["ez"].ctypes.data, out["wr"].ctypes.data,
                                     out["bt"].ctypes.data, out["psi"].ctypes.data, 0))
        return out

    def fields_at_static(self, r) -> Dict[str, np.ndarray]:
        """fields_at through the entry point that allocates nothing (its
        scratch is a static device array of the library): host radii r,
        at most WAKE_STATIC_MAX_QUERIES of them."""
        r = _f64(r)
        n = r.shape[0]
        out = {k: np.zeros(n, dtype=self.dtype) for k in ("ez", "wr", "bt", "psi")}
        _check(load().wake_fields_at_static(self.handle, n, r.ctypes.data, out["ez"].ctypes.data,
                                            out["wr"].ctypes.data, out["bt"].ctypes.data, out["psi"].ctypes.data))
        return out

    def fields_at_device(self, r_dev, outs: Dict[str, object]):
        """Device variant: r_dev a float64 CUDA tensor, outs torch tensors."""
        ptr = lambda k: outs[k].data_ptr() if k in outs and outs[k] is not None else None
        _check(load().wake_fields_at(self.handle, r_dev.numel(), r_dev.data_ptr(), ptr("ez"), ptr("wr"),
                                     ptr("bt"), ptr("psi"), 1))

    def beam_fields(self, which: Iterable[str] = ("ez", "wr", "bt", "psi")) -> Dict[str, np.ndarray]:
        which = list(which)
        out = {k: np.zeros(self.n_beam, dtype=self.dtype) for k in which}
        p = [out[k].ctypes.data if k in out else None for k in ("ez", "wr", "bt", "psi")]
        _check(load().wake_get_beam_fields(self.handle, *p, 0))
        return out

    def beam_fields_device(self, outs: Dict[str, object]):
        p = [outs[k].data_ptr() if k in outs and outs[k] is not None else None for k in ("ez", "wr", "bt", "psi")]
        _check(load().wake_get_beam_fields(self.handle, *p, 1))

    def run(self, ring_r: bool = False):
        """Rest of the window; returns (status, ez, wr, ring_r or None)."""
        ez = np.zeros(self.n_beam, dtype=self.dtype)
        wr = np.zeros(self.n_beam, dtype=self.dtype)
        rr = np.zeros((self.n_steps, self.n_rings), dtype=self.dtype) if ring_r else None
        st = load().wake_run(self.handle, ez.ctypes.data, wr.ctypes.data, rr.ctypes.data if rr is not None else None)
        if st not in (WAKE_OK, WAKE_ENONFINITE):
            _check(st)
        return st, ez, wr, rr

    def ring_state(self, history: bool = False):
        """(rho, u_r) by ring index as float64; with history=True also the AB2
        history (f_rho, f_u)."""
        arrs = [np.zeros(self.n_rings) for _ in range(4)]
        _check(load().wake_get_ring_state(self.handle, *[a.ctypes.data for a in arrs]))
        return tuple(arrs) if history else (arrs[0], arrs[1])

    def set_ring_state(self, slice_: int, rho, ur, f_rho=None, f_ur=None):
        """Restore a checkpoint: continue from slice_ with this ring state."""
        rho, ur = _f64(rho), _f64(ur)
        fr = _f64(f_rho) if f_rho is not None else None
        fu = _f64(f_ur) if f_ur is not None else None
        _check(load().wake_set_ring_state(self.handle, int(slice_), rho.ctypes.data, ur.ctypes.data,
                                          fr.ctypes.data if fr is not None else None,
                                          fu.ctypes.data if fu is not None else None))

    def set_beam_phase_space(self, x, y, ux, uy, uz):
        """Full phase space of the beam particles (concatenated order) for
        push_beam; the binning radius becomes |(x, y)|."""
        arrs = [_f64(a) for a in (x, y, ux, uy, uz)]
        _check(load().wake_set_beam_phase_space(self.handle, *[a.ctypes.data for a in arrs]))

    def beam_phase_space(self) -> Dict[str, np.ndarray]:
        """x, y, xi, r, ux, uy, uz of the beam particles (float64)."""
        keys = ("x", "y", "xi", "r", "ux", "uy", "uz")
        out = {k: np.zeros(self.n_beam) for k in keys}
        _check(load().wake_get_beam_phase_space(self.handle, *[out[k].ctypes.data for k in keys]))
        return out

    def push_beam(self, dt: float):
        """One Boris step dt of the beam in the fields of the last march
        (asynchronous); reset() then bins the moved beam."""
        _check(load().wake_push_beam(self.handle, float(dt)))

    def device_bytes(self) -> int:
        b = C.c_int64()
        _check(load().wake_get_device_bytes(self.handle, C.byref(b)))
        return int(b.value)

    def march_times(self):
        """(begin, end) device time in ns of the last march launch on this
        wake (the GPU's global timer)."""
        t0, t1 = C.c_int64(), C.c_int64()
        _check(load().wake_get_march_times(self.handle, C.byref(t0), C.byref(t1)))
        return t0.value, t1.value

    def launch_config(self):
        """(threads per block, rings per thread, blocks per wake)."""
        t, k, c = C.c_int32(), C.c_int32(), C.c_int32()
        _check(load().wake_get_launch_config(self.handle, C.byref(t), C.byref(k), C.byref(c)))
        return t.value, k.value, c.value

    def ring_dumps(self, which=("r", "ur", "psi", "dpsidr", "dpsidz", "bp", "bb")) -> Dict[str, np.ndarray]:
        keys = ("r", "ur", "psi", "dpsidr", "dpsidz", "bp", "bb")
        out = {k: np.zeros((self.n_steps, self.n_rings), dtype=self.dtype) for k in which}
        p = [out[k].ctypes.data if k in out else None for k in keys]
        _check(load().wake_get_ring_dumps(self.handle, *p))
        return out


def _beam_descs(beams):
    """wake_beam_desc array for beams given as numpy arrays (kept alive by the
    returned list) or pinned torch CPU tensors."""
    descs = (wake_beam_desc * max(1, len(beams)))()
    keep = []
    for i, b in enumerate(beams):
        ptrs = []
        n = 0
        for a in (b.xi, b.r, b.w):
            if hasattr(a, "data_ptr"):
                ptrs.append(C.cast(C.c_void_p(a.data_ptr()), _dp))
                n = a.numel()
            else:
                a = _f64(a)
                keep.append(a)
                ptrs.append(_dptr(a))
                n = a.shape[0]
        descs[i] = wake_beam_desc(n, ptrs[0], ptrs[1], ptrs[2], float(b.q))
    return descs, keep


def wake_batch_reset(wakes: List[Wake], beams: Optional[Sequence] = None):
    """reset() of many wakes at once, their preparations running concurrently.
    beams: None, or one entry per wake (None or a beam sequence as in reset)."""
    n = len(wakes)
    arr = (_vp * max(1, n))(*[w.handle for w in wakes])
    if beams is None:
        _check(load().wake_batch_reset(n, arr, None, None))
        return
    dps = (C.POINTER(wake_beam_desc) * max(1, n))()
    counts = (C.c_int32 * max(1, n))()
    keep = []
    for i, bs in enumerate(beams):
        if bs is None:
            continue
        descs, k = _beam_descs(bs)
        keep += [descs, k]
        dps[i] = C.cast(descs, C.POINTER(wake_beam_desc))
        counts[i] = len(bs)
    _check(load().wake_batch_reset(n, arr, dps, counts))
    for w in wakes:
        w._reset_keep = keep


def wake_batch_step(wakes: List[Wake], max_slices: int, time_budget_ns: int = 0):
    """Advance every wake by up to max_slices slices (and, with a budget, for
    about time_budget_ns on the device); asynchronous."""
    arr = (_vp * max(1, len(wakes)))(*[w.handle for w in wakes])
    _check(load().wake_batch_step(len(wakes), arr, int(max_slices), int(time_budget_ns)))


def wake_batch_progress(wakes: List[Wake]):
    """(next_slice, status) int32 arrays of the wakes, one synchronisation."""
    n = len(wakes)
    arr = (_vp * max(1, n))(*[w.handle for w in wakes])
    nxt = np.zeros(max(1, n), dtype=np.int32)
    st = np.zeros(max(1, n), dtype=np.int32)
    _check(load().wake_batch_progress(n, arr, nxt.ctypes.data, st.ctypes.data))
    return nxt[:n], st[:n]


def wake_batch_get_beam_fields(wakes: List[Wake], ez: Sequence, wr: Sequence):
    """E_z and W_r of every wake's beam particles into host arrays (numpy or
    pinned torch tensors; None to skip), one synchronisation."""
    n = len(wakes)
    ptr = lambda a: (a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data) if a is not None else None
    arr = (_vp * max(1, n))(*[w.handle for w in wakes])
    pez = (_vp * max(1, n))(*[ptr(a) for a in ez])
    pwr = (_vp * max(1, n))(*[ptr(a) for a in wr])
    _check(load().wake_batch_get_beam_fields(n, arr, pez, pwr, 0))


def wake_batch_push_beam(wakes: List[Wake], dt: float):
    """push_beam of many wakes at once (asynchronous)."""
    arr = (_vp * max(1, len(wakes)))(*[w.handle for w in wakes])
    _check(load().wake_batch_push_beam(len(wakes), arr, float(dt)))


def wake_batch_run(wakes: List[Wake]):
    """All wakes' remaining slices in one persistent launch."""
    arr = (_vp * len(wakes))(*[w.handle for w in wakes])
    _check(load().wake_batch_run(len(wakes), arr))


def wake_batch_reset_run(wakes: List[Wake]):
    """wake_batch_reset (device-resident beams) + wake_batch_run as one
    pipelined submission: each launch shape's march starts once its own
    wakes are prepared."""
    arr = (_vp * len(wakes))(*[w.handle for w in wakes])
    _check(load().wake_batch_reset_run(len(wakes), arr))


def wake_batch_solve(wakes: List[Wake], beams: Optional[Sequence] = None):
    """Upload (beams: None, or one entry per wake, None or a beam sequence
    as in reset; pinned torch tensors overlap), prepare and march every
    wake's whole window in one pipelined submission that never waits for
    the device."""
    n = len(wakes)
    arr = (_vp * max(1, n))(*[w.handle for w in wakes])
    if beams is None:
        _check(load().wake_batch_solve(n, arr, None, None))
        return
    dps = (C.POINTER(wake_beam_desc) * max(1, n))()
    counts = (C.c_int32 * max(1, n))()
    keep = []
    for i, bs in enumerate(beams):
        if bs is None:
            continue
        descs, k = _beam_descs(bs)
        keep += [descs, k]
        dps[i] = C.cast(descs, C.POINTER(wake_beam_desc))
        counts[i] = len(bs)
    _check(load().wake_batch_solve(n, arr, dps, counts))
    for w in wakes:
        w._reset_keep = keep


def wake_max_rings(precision: str = "mixed") -> int:
    return int(load().wake_max_rings(PRECISION[precision]))


def wake_launch_shape(n_rings: int, rings_per_thread: int = 0, cluster_ctas: int = 0, precision: str = "mixed",
                      n_steps: int = 0):
    """(threads per CTA, rings per thread, CTAs per wake) that wake_init
    gives the on-chip march for these fields, computed on the host; (0, 0,
    0) when the wake runs on a one-CTA march.  n_steps 0: the batch shape;
    else an automatic-shape wake long enough (latency_shape_ms()) gets the
    latency shape.  WakeError for a shape wake_init would refuse."""
    t, k, c = C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().wake_launch_shape(PRECISION[precision], int(n_rings), int(n_steps), int(rings_per_thread),
                                    int(cluster_ctas), C.byref(t), C.byref(k), C.byref(c)))
    return t.value, k.value, c.value


def wake_launch_shape_latency(n_rings: int, precision: str = "mixed"):
    """(threads per CTA, rings per thread, CTAs per wake) of the latency
    shape: 2 rings per thread, the shortest time per slice, which wake_init
    gives automatic-shape wakes whose predicted march time reaches
    latency_shape_ms()."""
    t, k, c = C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().wake_launch_shape_latency(PRECISION[precision], int(n_rings), C.byref(t), C.byref(k), C.byref(c)))
    return t.value, k.value, c.value


GM_MARCHES = {"ions": 1, "rk4": 2, "grid": 3}


def wake_gm_launch_shape(n_cells: int, march: str = "ions", block_threads: int = 0, cluster_ctas: int = 0):
    """(threads per block, rings per thread, blocks per wake) that wake_init
    gives a wake of the two-species march ("ions": n_cells per species), the
    RK4 march or a beam-grid wake, computed on the host."""
    t, k, c = C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().wake_gm_launch_shape(GM_MARCHES[march], int(n_cells), int(block_threads), int(cluster_ctas),
                                       C.byref(t), C.byref(k), C.byref(c)))
    return t.value, k.value, c.value


def set_latency_shape_ms(ms: float) -> None:
    """Wakes created afterwards whose predicted march time on the batch
    shape is at least ms milliseconds take the latency shape (0: all;
    math.inf: none)."""
    _check(load().wake_set_latency_shape_ms(float(ms)))


def latency_shape_ms() -> float:
    return float(load().wake_get_latency_shape_ms())


def debug_bounds_violations() -> int:
    """Out-of-range shared-memory positions and DSMEM ranks met since the
    last call (bounds-checking debug build); -1 in the normal build."""
    return int(load().wake_debug_bounds_violations())


def wake_max_slice_particles(precision: str = "mixed") -> int:
    return int(load().wake_max_slice_particles(PRECISION[precision]))
