"""ctypes wrapper of the C oracle (wake_oracle.c).

TEST INFRASTRUCTURE ONLY.  The oracle is plain sequential FP64 C that follows
Sec. II-III and App. A of the paper step by step; this module only marshals
numpy arrays in and out of it and builds it with gcc on first use.

The environment variable ORACLE_LIB, when set, names another build of the
same source to load instead (the planted-mistake tests load altered copies
through it).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Dict, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wake_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class _Problem(C.Structure):
    _fields_ = [("n_rings", C.c_int32), ("edges", _dp), ("density", C.c_double),
                ("n_beam", C.c_int64), ("beam_xi", _dp), ("beam_r", _dp), ("beam_qw", _dp),
                ("dxi", C.c_double), ("n_steps", C.c_int32), ("cell_density", _dp), ("integrator", C.c_int32),
                ("grid_nr", C.c_int32), ("beam_species", _ip), ("n_species", C.c_int32),
                ("grid_rmax", C.c_double), ("init_r", _dp), ("init_ur", _dp), ("init_fr", _dp),
                ("init_fu", _dp)]


_RING_DUMPS = ["ring_r", "ring_ur", "ring_psi", "ring_dpsidr", "ring_dpsidz", "ring_bp",
               "ring_bb", "ring_psibar", "ring_gamma", "ring_uz", "ring_frprev", "ring_fuprev"]


class _Outputs(C.Structure):
    _fields_ = ([(k, _dp) for k in ["ez", "wr", "bt", "psi"]]
                + [(k, _dp) for k in _RING_DUMPS]
                + [("final_r", _dp), ("final_ur", _dp), ("status", C.c_int32),
                   ("fail_slice", C.c_int32), ("slices_run", C.c_int32),
                   ("n_snap", C.c_int32), ("snap_slice", _ip), ("snap", _dp)])

_SNAP_FIELDS = ["r", "ur", "psi", "dpsidr", "dpsidz", "bp", "bb", "frprev", "fuprev"]


_SLICE_RING = ["psi", "dpsidr", "dpsidz", "psibar", "gamma", "uz", "bb", "A", "B", "C", "bp"]
_SLICE_Q = ["q_ez", "q_wr", "q_bt", "q_psi", "q_bp", "q_bb", "q_dpsidr", "q_dpsidz"]


class _SliceOut(C.Structure):
    _fields_ = ([(k, _dp) for k in _SLICE_RING] + [("a", _dp), ("b", _dp), ("order", _ip),
                                                     ("nq", C.c_int64), ("rq", _dp)]
                + [(k, _dp) for k in _SLICE_Q])


def lib_path() -> str:
    return _LIB


GCC_FLAGS = ["-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB)
             or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC),
                                             os.path.getmtime(os.path.join(_HERE, "wake_oracle.h"))))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *GCC_FLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = C.CDLL(os.environ.get("ORACLE_LIB") or build())
        lib.orc_run.argtypes = [C.POINTER(_Problem), C.c_int32, C.POINTER(_Outputs)]
        lib.orc_run.restype = C.c_int
        lib.orc_run_ions.argtypes = [C.POINTER(_Problem), C.c_double, C.c_double, C.c_int32,
                                     C.POINTER(_Outputs)]
        lib.orc_run_ions.restype = C.c_int
        lib.orc_slice_fields.argtypes = [C.c_int32, _dp, _dp, _dp, _dp, C.c_double, C.c_double,
                                         C.c_int64, _dp, _dp, C.c_double, C.POINTER(_SliceOut)]
        lib.orc_slice_fields.restype = C.c_int
        lib.orc_bp_shooting.argtypes = [C.c_int32, _dp, _dp, _dp, _dp, _dp, _dp]
        lib.orc_bp_shooting.restype = C.c_int
        lib.orc_bp_solve.argtypes = [C.c_int32, _dp, _dp, _dp, _dp, _dp, _dp]
        lib.orc_bp_solve.restype = C.c_int
        lib.orc_ring_init.argtypes = [C.c_int32, _dp, C.c_double, _dp, _dp, _dp, _dp]
        lib.orc_ring_init.restype = None
        _lib_handle = lib
    return _lib_handle


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def ring_init(edges, density: float = 1.0):
    """Cell centres, widths, weights and self weights of the rings."""
    edges = _f64(edges)
    n = edges.shape[0] - 1
    rho0, drho, w, wh = (np.empty(n) for _ in range(4))
    _lib().orc_ring_init(n, _ptr(edges), density, _ptr(rho0), _ptr(drho), _ptr(w), _ptr(wh))
    return rho0, drho, w, wh


def bp_shooting(rho, A, B, Cc):
    rho, A, B, Cc = (_f64(x) for x in (rho, A, B, Cc))
    n = rho.shape[0]
    a = np.empty(n + 1)
    b = np.empty(n + 1)
    rc = _lib().orc_bp_shooting(n, _ptr(rho), _ptr(A), _ptr(B), _ptr(Cc), _ptr(a), _ptr(b))
    if rc:
        raise RuntimeError(f"orc_bp_shooting failed ({rc})")
    return a, b


def bp_solve(rho, A, B, Cc):
    rho, A, B, Cc = (_f64(x) for x in (rho, A, B, Cc))
    n = rho.shape[0]
    a = np.empty(n + 1)
    b = np.empty(n + 1)
    rc = _lib().orc_bp_solve(n, _ptr(rho), _ptr(A), _ptr(B), _ptr(Cc), _ptr(a), _ptr(b))
    if rc:
        raise RuntimeError(f"orc_bp_solve failed ({rc})")
    return a, b


def slice_fields(rho, ur, w, wh, density: float, rho_max: float, beam_r=(), beam_qw=(),
                 dxi: float = 1.0, rq=None) -> Dict[str, np.ndarray]:
    """Fields of one slice for the ring state (rho, ur) indexed by ring id.

    Returns per-ring fields by id, per-region a, b (radius order), the radius
    order, and fields at the query radii rq (keys q_*)."""
    rho, ur, w, wh = (_f64(x) for x in (rho, ur, w, wh))
    beam_r, beam_qw = _f64(beam_r), _f64(beam_qw)
    n = rho.shape[0]
    out = _SliceOut()
    res: Dict[str, np.ndarray] = {}
    for k in _SLICE_RING:
        res[k] = np.empty(n)
        setattr(out, k, _ptr(res[k]))
    res["a"] = np.empty(n + 1)
    res["b"] = np.empty(n + 1)
    out.a, out.b = _ptr(res["a"]), _ptr(res["b"])
    res["order"] = np.empty(n, dtype=np.int32)
    out.order = res["order"].ctypes.data_as(_ip)
    if rq is not None:
        rq = _f64(rq)
        res["rq"] = rq
        out.nq = rq.shape[0]
        out.rq = _ptr(rq)
        for k in _SLICE_Q:
            res[k] = np.empty(rq.shape[0])
            setattr(out, k, _ptr(res[k]))
    else:
        out.nq = 0
    rc = _lib().orc_slice_fields(n, _ptr(rho), _ptr(ur), _ptr(w), _ptr(wh), density, rho_max,
                                 beam_r.shape[0], _ptr(beam_r), _ptr(beam_qw), dxi, C.byref(out))
    res["status"] = rc
    if rc not in (0, 4):
        raise RuntimeError(f"orc_slice_fields failed ({rc})")
    return res


@dataclass
class OracleResult:
    status: int
    fail_slice: int
    slices_run: int
    beam: Dict[str, np.ndarray]
    rings: Dict[str, np.ndarray]
    final_r: np.ndarray
    final_ur: np.ndarray
    snapshots: Dict[int, Dict[str, np.ndarray]] = None


def run(edges, beam_xi, beam_r, beam_qw, dxi: float, n_steps: int, density: float = 1.0,
        max_slices: int = 0, beam_fields: Sequence[str] = ("ez", "wr", "bt", "psi"),
        ring_dumps: Sequence[str] = (), ions: Optional[Tuple[float, float]] = None,
        cell_density=None, integrator: str = "ab2", grid_nr: int = 0, beam_species=None,
        grid_rmax: float = 0.0, init_state=None, snapshots: Sequence[int] = ()) -> OracleResult:
    """March the whole window (or its first max_slices slices).

    beam_fields: subset of ez, wr, bt, psi (per particle, caller order).
    ring_dumps: subset of r, ur, psi, dpsidr, dpsidz, bp, bb, psibar, gamma, uz,
    frprev, fuprev
    ([slices, rings] by ring id, values at the start of each slice).
    ions: (Z, M) for mobile ions as a second ring species (orc_run_ions;
    M = inf: ion rings that never move); ring dumps and final state then have
    2 N columns, ions after electrons.  cell_density: the density of each
    cell (a radial profile), with ions only.  integrator: "ab2" or "rk4"
    (electron-only march).  grid_nr > 0: beam fields through adaptive beam
    grids of grid_nr radial cells per species (beam_species: each
    particle's species index; None: one species); grid_rmax > 0: grids of
    that fixed extent (the regular intermediate grid).  init_state: None
    (rings at rest at their cell centres), or (rho, u_r) or (rho, u_r,
    f_rho, f_u) by ring id, the starting state (f_*: the AB2 history; without
    it the first step is forward Euler); electron-only runs.  snapshots:
    slices at which to keep every ring dump (r, ur, psi, dpsidr, dpsidz, bp,
    bb, frprev, fuprev by ring id), returned as {slice: {name: array}} for
    the slices the run reached; electron-only runs."""
    edges = _f64(edges)
    bxi, br, bqw = _f64(beam_xi), _f64(beam_r), _f64(beam_qw)
    n_e = edges.shape[0] - 1
    n = n_e if ions is None else 2 * n_e
    nb = bxi.shape[0]
    cd = None if cell_density is None else _f64(cell_density)
    sp = None if beam_species is None else np.ascontiguousarray(beam_species, dtype=np.int32)
    n_sp = 1 if sp is None or sp.shape[0] == 0 else int(sp.max()) + 1
    init = [None] * 4
    if init_state is not None:
        if ions is not None:
            raise ValueError("init_state applies to electron-only runs")
        init[: len(init_state)] = [_f64(a) for a in init_state]
        assert all(a is None or a.shape == (n,) for a in init)
    prob = _Problem(n_e, _ptr(edges), density, nb, _ptr(bxi), _ptr(br), _ptr(bqw), dxi, n_steps, _ptr(cd),
                    {"ab2": 0, "rk4": 1}[integrator], int(grid_nr),
                    None if sp is None else sp.ctypes.data_as(_ip), n_sp, float(grid_rmax),
                    *(_ptr(a) for a in init))
    out = _Outputs()
    beam = {}
    for k in beam_fields:
        beam[k] = np.empty(nb)
        setattr(out, k, _ptr(beam[k]))
    nrun = n_steps if max_slices <= 0 else min(max_slices, n_steps)
    rings = {}
    for k in ring_dumps:
        rings[k] = np.zeros((nrun, n))
        setattr(out, "ring_" + k, _ptr(rings[k]))
    final_r = np.empty(n)
    final_ur = np.empty(n)
    out.final_r, out.final_ur = _ptr(final_r), _ptr(final_ur)
    snap_sl = np.ascontiguousarray(sorted(set(int(v) for v in snapshots)), dtype=np.int32)
    snap = np.zeros((snap_sl.shape[0], len(_SNAP_FIELDS), n))
    if snap_sl.shape[0]:
        if ions is not None:
            raise ValueError("snapshots apply to electron-only runs")
        out.n_snap = snap_sl.shape[0]
        out.snap_slice = snap_sl.ctypes.data_as(_ip)
        out.snap = _ptr(snap)
    if ions is None:
        rc = _lib().orc_run(C.byref(prob), max_slices, C.byref(out))
    else:
        rc = _lib().orc_run_ions(C.byref(prob), float(ions[0]), float(ions[1]), max_slices, C.byref(out))
    if rc:
        raise RuntimeError(f"orc_run failed ({rc})")
    snaps = {int(sl): dict(zip(_SNAP_FIELDS, snap[j])) for j, sl in enumerate(snap_sl) if sl < out.slices_run}
    return OracleResult(out.status, out.fail_slice, out.slices_run, beam, rings, final_r, final_ur, snaps)


def run_wake(wake, **kw) -> OracleResult:
    """Run a workloads.Wake (beams concatenated in order, charge folded into
    the weight)."""
    if wake.beams:
        xi = np.concatenate([b.xi for b in wake.beams])
        r = np.concatenate([b.r for b in wake.beams])
        qw = np.concatenate([b.q * b.w for b in wake.beams])
    else:
        xi = r = qw = np.zeros(0)
    kw.setdefault("ions", getattr(wake, "ions", None))
    kw.setdefault("cell_density", getattr(wake, "cell_density", None))
    kw.setdefault("integrator", getattr(wake, "integrator", "ab2"))
    kw.setdefault("grid_nr", getattr(wake, "grid_nr", 0))
    kw.setdefault("grid_rmax", getattr(wake, "grid_rmax", 0.0))
    if wake.beams:
        kw.setdefault("beam_species", np.concatenate([np.full(b.n, i, dtype=np.int32)
                                                      for i, b in enumerate(wake.beams)]))
    return run(wake.edges, xi, r, qw, wake.dxi, wake.n_steps, density=wake.density, **kw)
