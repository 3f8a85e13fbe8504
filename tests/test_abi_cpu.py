"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, and exports every entry point include/wake.h declares; the
product package never imports the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2603_16623_gb300 import build as wbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wake_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib_path = wbuild.build()
    lib = ctypes.CDLL(lib_path)
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            names += _declared(os.path.join(ROOT, "include", h))
    assert len(names) >= 13
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_limits_are_queryable_without_a_gpu():
    from paper_2603_16623_gb300 import wake
    assert wake.wake_max_rings("mixed") >= 8192
    assert wake.wake_max_slice_particles("fp64") >= 8192


def test_product_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_2603_16623_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", src, re.M), f
                assert "wake_oracle" not in src and "liboracle" not in src, f


@pytest.mark.parametrize("precision,n,k,cl,why", [
    ("mixed", 1000, 5, 0, "rings_per_thread"),
    ("mixed", 1000, 4, 17, "cluster_ctas"),
    ("fp64", 1000, 4, 0, "WAKE_MIXED only"),
    ("mixed", 100, 4, 4, "empty"),
    ("mixed", 8192, 4, 2, "do not fit"),
    ("mixed", 70000, 4, 16, "n_rings"),
])
def test_launch_shape_is_validated_on_the_host(precision, n, k, cl, why):
    """Invalid (rings per thread, CTAs per wake) choices fail in wake_init
    with EINVAL before any device work."""
    from paper_2603_16623_gb300 import wake as wm
    lib = wm.load()
    edges = np.linspace(0.0, 5.0, n + 1)
    cfg = wm.wake_config(0.01, 10, wm.PRECISION[precision], 0, 0, k, cl)
    plasma = wm.wake_plasma_desc(n, edges.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1.0)
    h = ctypes.c_void_p()
    st = lib.wake_init(ctypes.byref(cfg), ctypes.byref(plasma), None, 0, None, ctypes.byref(h))
    assert st == wm.WAKE_EINVAL
    assert not h.value
    assert why in lib.wake_last_error().decode()


@pytest.mark.parametrize("precision,n,k,cl,why", [
    ("mixed", 1000, 5, 0, "rings_per_thread"),
    ("mixed", 1000, 4, 17, "cluster_ctas"),
    ("fp64", 1000, 4, 0, "WAKE_MIXED only"),
    ("mixed", 100, 4, 4, "empty"),
    ("mixed", 8192, 4, 2, "do not fit"),
    ("mixed", 70000, 0, 0, "n_rings"),
    ("fp64", 9000, 0, 0, "n_rings"),
])
def test_the_shape_query_refuses_what_wake_init_refuses(precision, n, k, cl, why):
    """wake_launch_shape (host-only) gives EINVAL with the same reason for
    the shapes wake_init refuses."""
    from paper_2603_16623_gb300 import wake as wm
    wm.load()
    with pytest.raises(wm.WakeError, match=re.escape(why)):
        wm.wake_launch_shape(n, k, cl, precision)


def test_the_shape_query_gives_the_automatic_and_explicit_shapes():
    """The automatic on-chip shapes (one CTA up to 2048 rings, then
    clusters of up to 1024, then 2048 rings per CTA, then 8 rings per
    thread) and explicit ones, computed on the host; FP64 wakes run on the
    one-CTA march (all zeros)."""
    from paper_2603_16623_gb300 import wake as wm
    wm.load()
    assert wm.wake_launch_shape(200) == (128, 2, 1)
    assert wm.wake_launch_shape(1024) == (512, 2, 1)
    assert wm.wake_launch_shape(1025) == (288, 4, 1)
    assert wm.wake_launch_shape(2048) == (512, 4, 1)
    assert wm.wake_launch_shape(2049) == (192, 4, 3)
    assert wm.wake_launch_shape(16384) == (256, 4, 16)
    assert wm.wake_launch_shape(16385) == (480, 4, 9)
    assert wm.wake_launch_shape(65536) == (512, 8, 16)
    assert wm.wake_launch_shape(3000, 8, 0) == (384, 8, 1)
    assert wm.wake_launch_shape(3000, 4, 3) == (256, 4, 3)
    assert wm.wake_launch_shape(3000, 2, 3) == (512, 2, 3)
    assert wm.wake_launch_shape(1000, 2, 1) == (512, 2, 1)
    assert wm.wake_launch_shape(4000, precision="fp64") == (0, 0, 0)
    for n in range(1, 65537, 997):
        t, k, c = wm.wake_launch_shape(n)
        assert 32 <= t <= 512 and t % 32 == 0 and k in (2, 4, 8) and 1 <= c <= 16
        assert t * k * c >= n and (c == 1 or t * k * (c - 1) < n)


def test_the_normal_build_has_no_bounds_checks():
    """wake_debug_bounds_violations answers -1 (no checks compiled in)
    without touching a device; the checking build is a separate library."""
    from paper_2603_16623_gb300 import build, wake as wm
    wm.load()
    if os.environ.get("GBWAKE_BOUNDS_CHECK", "") != "1":
        assert wm.debug_bounds_violations() == -1
    assert build.lib_for(True) != build.lib_for(False)


def test_the_latency_shape_query():
    """The latency shapes (2 rings per thread: one CTA up to 1024 rings,
    clusters of CTAs of <= 512 rings up to 8192, of <= 1024 rings up to
    16,384, then the batch shape); every CTA holds rings and none more than
    its threads x 2; an explicit request for the same shape gives it."""
    from paper_2603_16623_gb300 import wake as wm
    wm.load()
    assert wm.wake_launch_shape_latency(200) == (128, 2, 1)
    assert wm.wake_launch_shape_latency(1024) == (512, 2, 1)
    assert wm.wake_launch_shape_latency(1025) == (192, 2, 3)
    assert wm.wake_launch_shape_latency(6587) == (256, 2, 13)
    assert wm.wake_launch_shape_latency(8192) == (256, 2, 16)
    assert wm.wake_launch_shape_latency(8193) == (480, 2, 9)
    assert wm.wake_launch_shape_latency(16384) == (512, 2, 16)
    assert wm.wake_launch_shape_latency(16385) == wm.wake_launch_shape(16385)
    assert wm.wake_launch_shape_latency(65536) == (512, 8, 16)
    assert wm.wake_launch_shape_latency(4000, precision="fp64") == (0, 0, 0)
    for n in range(1, 16385, 37):
        t, k, c = wm.wake_launch_shape_latency(n)
        assert k == 2 and 32 <= t <= 512 and t % 32 == 0 and 1 <= c <= 16
        assert t * k * c >= n and (c == 1 or t * k * (c - 1) < n)
        assert wm.wake_launch_shape(n, k, c) == (t, k, c)
    for bad in (0, 65537):
        with pytest.raises(wm.WakeError):
            wm.wake_launch_shape_latency(bad)


def test_long_wakes_get_the_latency_shape():
    """An automatic-shape wake whose predicted march time on the batch shape
    reaches the threshold (off by default) gets the latency shape; a short
    one, n_steps 0 and explicit shapes keep theirs; the threshold is
    validated and applies to what is created afterwards."""
    import math
    from paper_2603_16623_gb300 import wake as wm
    wm.load()
    assert wm.latency_shape_ms() == math.inf
    assert wm.wake_launch_shape(6587, n_steps=10 ** 6) == (256, 4, 7)
    wm.set_latency_shape_ms(100.0)
    batch = wm.wake_launch_shape(6587)
    assert batch == (256, 4, 7)
    assert wm.wake_launch_shape(6587, n_steps=5664) == wm.wake_launch_shape_latency(6587)  # ~206 ms predicted
    assert wm.wake_launch_shape(6587, n_steps=1000) == batch  # ~36 ms
    assert wm.wake_launch_shape(6587, 4, 7, n_steps=5664) == batch
    assert wm.wake_launch_shape(1500, n_steps=4000) == (384, 4, 1)  # ~75 ms
    assert wm.wake_launch_shape(1500, n_steps=6000) == wm.wake_launch_shape_latency(1500)  # ~113 ms
    assert wm.wake_launch_shape(4000, n_steps=10 ** 6, precision="fp64") == (0, 0, 0)
    with pytest.raises(wm.WakeError):
        wm.wake_launch_shape(6587, n_steps=-1)
    for bad in (-0.1, float("nan")):
        with pytest.raises(wm.WakeError):
            wm.set_latency_shape_ms(bad)
    try:
        wm.set_latency_shape_ms(math.inf)
        assert wm.wake_launch_shape(6587, n_steps=10 ** 6) == batch
        wm.set_latency_shape_ms(0.0)
        assert wm.wake_launch_shape(3000, n_steps=1) == wm.wake_launch_shape_latency(3000)
    finally:
        wm.set_latency_shape_ms(math.inf)


@pytest.mark.parametrize("case,why", [
    ({"ion_charge": -1.0, "ion_mass": 10.0}, "ion_charge > 0"),
    ({"ion_charge": 1.0, "ion_mass": 0.0}, "ion_charge > 0"),
    ({"ion_charge": 1.0, "ion_mass": float("nan")}, "ion_charge > 0"),
    ({"ion_charge": 1.0, "ion_mass": 100.0, "k": 4}, "with mobile ions rings_per_thread must be 0"),
    ({"ion_charge": 1.0, "ion_mass": 100.0, "cl": 9}, "cluster_ctas in [0, 8]"),
    ({"ion_charge": 1.0, "ion_mass": 100.0, "cl": -1, "precision": "fp64"}, "cluster_ctas in [0, 8]"),
    ({"ion_charge": 1.0, "ion_mass": 100.0, "n": 4097}, "with mobile ions"),
    ({"profile": 1.0}, "needs ion rings"),
    ({"ion_charge": 1.0, "ion_mass": 100.0, "profile": -1.0}, "cell_density[7]"),
    ({"integrator": 7}, "unknown integrator"),
    ({"integrator": 1, "ion_charge": 1.0, "ion_mass": 100.0}, "RK4 runs electron-only"),
    ({"integrator": 1, "cl": 9}, "RK4 runs electron-only"),
    ({"integrator": 1, "k": 4}, "RK4 runs electron-only"),
    ({"integrator": 1, "n": 16385}, "RK4 wakes have at most 16384 rings"),
    ({"grid_nr": 2000, "precision": "fp64"}, "grid_nr must be"),
    ({"grid_nr": 16, "ion_charge": 1.0, "ion_mass": 100.0}, "beam grids run WAKE_AB2"),
    ({"grid_nr": 16, "precision": "fp64", "integrator": 1}, "beam grids run WAKE_AB2"),
    ({"grid_nr": 16, "cl": 9}, "beam-grid wakes take rings_per_thread 0"),
    ({"grid_nr": 16, "k": 4, "precision": "fp64"}, "beam-grid wakes take rings_per_thread 0"),
    ({"grid_nr": 16, "n": 16385}, "beam-grid wakes have at most 16384 rings"),
    ({"grid_rmax": 2.0}, "grid_rmax must be"),
    ({"grid_nr": 16, "grid_rmax": -1.0}, "grid_rmax must be"),
])
def test_model_options_are_validated_on_the_host(case, why):
    """Mobile ions, density profiles, the RK4 integrator and beam grids: bad
    combinations fail in wake_init with EINVAL before any device work."""
    from paper_2603_16623_gb300 import wake as wm
    lib = wm.load()
    n = case.get("n", 100)
    edges = np.linspace(0.0, 5.0, n + 1)
    prof = None
    if "profile" in case:
        prof = np.full(n, 1.0)
        prof[7] = case["profile"]
    cfg = wm.wake_config(0.01, 10, wm.PRECISION[case.get("precision", "mixed")], 0, 0, case.get("k", 0),
                         case.get("cl", 0), case.get("integrator", 0), case.get("grid_nr", 0),
                         case.get("grid_rmax", 0.0))
    dp = ctypes.POINTER(ctypes.c_double)
    plasma = wm.wake_plasma_desc(n, edges.ctypes.data_as(dp), 1.0, case.get("ion_charge", 0.0),
                                 case.get("ion_mass", 0.0), prof.ctypes.data_as(dp) if prof is not None else None)
    h = ctypes.c_void_p()
    st = lib.wake_init(ctypes.byref(cfg), ctypes.byref(plasma), None, 0, None, ctypes.byref(h))
    assert st == wm.WAKE_EINVAL
    assert not h.value
    assert why in lib.wake_last_error().decode()


def test_a_beam_beyond_a_fixed_grid_is_refused_on_the_host():
    from paper_2603_16623_gb300 import wake as wm
    lib = wm.load()
    n = 50
    edges = np.linspace(0.0, 5.0, n + 1)
    xi, r, w = np.array([0.1, 0.2]), np.array([0.3, 2.5]), np.array([1e-3, 1e-3])
    dp = ctypes.POINTER(ctypes.c_double)
    beam = wm.wake_beam_desc(2, xi.ctypes.data_as(dp), r.ctypes.data_as(dp), w.ctypes.data_as(dp), -1.0)
    cfg = wm.wake_config(0.01, 10, wm.PRECISION["fp64"], 0, 0, 0, 0, 0, 8, 2.0)
    plasma = wm.wake_plasma_desc(n, edges.ctypes.data_as(dp), 1.0)
    h = ctypes.c_void_p()
    st = lib.wake_init(ctypes.byref(cfg), ctypes.byref(plasma), ctypes.byref(beam), 1, None, ctypes.byref(h))
    assert st == wm.WAKE_EINVAL and not h.value
    assert "beyond grid_rmax" in lib.wake_last_error().decode()


def test_global_memory_march_shapes_on_the_host():
    """wake_gm_launch_shape: the blocks per wake wake_init gives the
    two-species, RK4 and beam-grid marches -- the fewest blocks (at most 8)
    that hold at most 2 rings of each species, 2 rings and 4 rings per
    thread -- and the rings per thread wake_get_launch_config reports."""
    from paper_2603_16623_gb300 import wake as wm
    cases = {("ions", 1024): (512, 4, 1), ("ions", 1025): (512, 3, 2), ("ions", 2048): (512, 4, 2),
             ("ions", 3993): (512, 4, 4), ("ions", 4096): (512, 4, 4), ("rk4", 1024): (512, 2, 1),
             ("rk4", 1025): (512, 2, 2), ("rk4", 7905): (512, 2, 8), ("rk4", 16384): (512, 4, 8),
             ("grid", 1024): (256, 4, 1), ("grid", 1025): (256, 3, 2), ("grid", 8192): (256, 4, 8)}
    for (march, n), shape in cases.items():
        assert wm.wake_gm_launch_shape(n, march) == shape, (march, n)
    # explicit shapes: a block size alone keeps the automatic blocks for it
    assert wm.wake_gm_launch_shape(4096, "ions", 512, 1) == (512, 16, 1)
    assert wm.wake_gm_launch_shape(300, "ions", 64, 8) == (64, 2, 8)
    assert wm.wake_gm_launch_shape(3000, "rk4", 256, 0) == (256, 2, 6)
    assert wm.wake_gm_launch_shape(300, "grid", 96, 3) == (96, 2, 3)
    for args in ((0, "ions"), (4097, "ions"), (16385, "rk4"), (100, "grid", 48), (100, "grid", 0, 9),
                 (100, "rk4", 0, -1), (100, "ions", 1024)):
        with pytest.raises(wm.WakeError):
            wm.wake_gm_launch_shape(*args)
    lib = wm.load()
    t = ctypes.c_int32()
    assert lib.wake_gm_launch_shape(7, 100, 0, 0, ctypes.byref(t), None, None) == wm.WAKE_EINVAL
