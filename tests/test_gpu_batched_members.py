"""The batched workload (256 independent wakes, log-uniform 500-8000 rings,
n_b0 up to 20) compared with the FP64 oracle member by member, on the
stratified sample of tests/batched_members.py (32 members: every ring-count
class, the strongest drivers, the longest windows), run as one batch the way
the benchmark runs the workload.

Per member:
- where it stops: the march stops at the first slice whose psibar <= 0 or a
  non-finite field (the guard; the paper requires psibar > 0).  Every member
  must end with the oracle's status in FP64, at the oracle's slice where
  that lies before slice 2000, within 1 % of it beyond (two FP64 codes that
  differ only in summation order part after ~1000 slices of a chaotic
  wake, which moves a breakdown that deep by a slice or two).  The mixed
  path's trajectories part from the oracle's sooner, so its stop slices
  are reported as a distribution and bounded loosely;
- the first 300 slices whole: ring radii at every slice and E_z, W_r on
  every beam particle of those slices, FP64 within 1e-10; the mixed path
  over the laminar part of those slices (before any two rings of the
  oracle's wake cross; past that the flow is multi-stream and chaotic, and
  FP32 rounding is amplified by hundreds within a few hundred slices, so
  those slices are checked one at a time below): E_z within 1e-5, W_r
  within 1e-4 (W_r = -d_rho psi at a particle is S(x) - n x^2 / 2 over x,
  two nearly equal FP32 terms where the wake is still weak), radii within
  2e-5 (31 of the 32 members stay within 1e-5; the strongest narrow driver,
  member 251 with n_b0 = 19.6 and sigma_r = 0.28, reaches 1.4e-5 at slice
  298 as its first rings converge to cross);
  Beam particles within rounding of a ring are left out of the mixed
  comparison (both sides of the ring are correct);
- one-step parity at three slices spread over the member's run after slice
  300 (before it the fields are still small next to the sums they cancel
  from): the oracle's ring state with its AB2 history loaded through the
  checkpoint entry, one slice solved, the ring fields, the next state and
  the fields on the slice's beam particles compared (tolerances of the
  one-step tests of test_gpu_parity.py, with psi and beam W_r at 1e-4 for
  the mixed path: see ONE_STEP_MIXED; rings tied within 5e-7 of a
  neighbour, which either order sorts correctly, are left out, at most 2 %).
"""
import numpy as np
import pytest

import batched_members as BM
from paper_2603_16623_gb300 import workloads as W
from test_gpu_parity import FP64_TOL, MIXED_FIELD_TOL, MIXED_TOL, unambiguous

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sample():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2603_16623_gb300 import wake
    wake.load()
    ks = BM.stratified_sample()
    return ks, BM.oracle_members(ks)


def _wm():
    from paper_2603_16623_gb300 import wake
    return wake


def _batch(ks, precision, window=None, flags=0):
    wm = _wm()
    wakes = [W.batched_wake(k) for k in ks]
    if window:
        wakes = [W.Wake(w.name, w.edges, w.beams, w.dxi, min(window, w.n_steps)) for w in wakes]
    gs = [wm.Wake.from_workload(wk, precision=precision, flags=flags) for wk in wakes]
    wm.wake_batch_run(gs)
    return wakes, gs


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_members_stop_where_the_oracle_stops(sample, precision):
    ks, ref = sample
    wakes, gs = _batch(ks, precision)
    rows = []
    for k, g in zip(ks, gs):
        nxt, st, fail = g.progress()
        r = ref[k]
        rows.append((k, r["status"], r["fail_slice"], st, fail, nxt))
        g.close()
    stopped = [row for row in rows if row[1] != 0]
    print(f"\n{precision}: {len(stopped)} of {len(rows)} members stop at the guard in the oracle")
    if precision == "fp64":
        bad = [row for row in rows if row[3] != row[1]
               or (row[1] != 0 and row[2] < 2000 and row[4] != row[2])
               or (row[1] != 0 and abs(row[4] - row[2]) > 0.01 * row[2])]
        print("fp64 stop slices differing from the oracle's:", [row for row in rows if row[4] != row[2]])
        assert not bad, bad
        return
    diffs = np.array([row[4] - row[2] for row in rows if row[1] == row[3] == 4])
    same_status = sum(row[1] == row[3] for row in rows)
    print(f"mixed: same status {same_status}/{len(rows)}; stop slice - oracle's: "
          f"{np.percentile(diffs, [0, 25, 50, 75, 100]) if diffs.size else []}")
    for row in rows:
        print("  member %3d oracle (status %d, stop %5d)  mixed (status %d, stop %5d)" % row[:5])
    # the same members break down, mostly at the same slice
    assert same_status >= 0.9 * len(rows), rows
    assert diffs.size == 0 or np.median(np.abs(diffs)) <= 2, diffs


def _laminar_slices(ring_r):
    """Slices before the first one at which two rings of the oracle's wake
    have crossed (their radius order differs from the cells' order)."""
    crossed = np.nonzero(np.any(np.diff(ring_r, axis=1) <= 0.0, axis=1))[0]
    return int(crossed[0]) if crossed.size else ring_r.shape[0]


TOL_WINDOW = {"fp64": {"r": FP64_TOL, "ez": FP64_TOL, "wr": FP64_TOL},
              "mixed": {"r": 2e-5, "ez": MIXED_TOL, "wr": 1e-4}}
# mixed one-step bounds that differ from test_gpu_parity.py's: psi late in
# a long window (rings far from their initial cells, where ln rho = ln rho0
# + log1p(d) carries log1p's FP32 rounding into S ln rho and the prefix of
# w ln rho, against a psi that has decayed behind the driver; measured up
# to 6.3e-5 after slice 1400) and W_r on beam particles (the cancellation
# of S(x) - n x^2 / 2 at the driver's head; measured 1.6e-5)
ONE_STEP_MIXED = dict(MIXED_FIELD_TOL, psi=1e-4, beam_wr=1e-4)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_members_match_over_their_first_slices(sample, precision):
    wm = _wm()
    ks, ref = sample
    wakes, gs = _batch(ks, precision, window=BM.WINDOW, flags=wm.WAKE_DUMP_RING_R)
    worst = {}
    bad = []
    for k, wk, g in zip(ks, wakes, gs):
        r = ref[k]
        nxt, st, fail = g.progress()
        assert st == r["head_status"], (k, st, r["head_status"])
        n_ok = nxt if st == 0 else fail + 1
        if precision == "mixed":
            n_ok = min(n_ok, _laminar_slices(r["head_r"]))
        got_r = g.ring_dumps(which=("r",))["r"][:n_ok]
        ref_r = r["head_r"][:n_ok]
        e = {"r": BM.nerr(got_r, ref_r)}
        bf = g.beam_fields(which=("ez", "wr"))
        xi = np.concatenate([b.xi for b in wk.beams])
        sl = np.floor(xi / wk.dxi + 0.5)
        m = (sl >= 0) & (sl < n_ok)
        if precision == "mixed":
            m &= unambiguous(W.Wake(wk.name, wk.edges, wk.beams, wk.dxi, n_ok), ref_r, got_r)
        for f in ("ez", "wr"):
            e[f] = BM.nerr(bf[f][m], r["head_beam"][f][m])
        print(f"  member {k:3d} slices {n_ok:3d}: " + " ".join(f"{f} {v:.2e}" for f, v in e.items()))
        for f, v in e.items():
            worst[f] = max(worst.get(f, 0.0), v)
            if not v < TOL_WINDOW[precision][f]:
                bad.append((k, f, v))
        g.close()
    print(f"{precision}: worst over {len(ks)} members, first {BM.WINDOW} slices: {worst}")
    assert not bad, bad


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_members_one_step_parity_along_their_run(sample, precision):
    wm = _wm()
    ks, ref = sample
    worst, bad = {}, []
    for k in ks:
        r = ref[k]
        wk = W.batched_wake(k)
        snaps, picks = r["snapshots"], r["picks"]
        assert len(picks) >= 1, (k, r["status"], r["fail_slice"])
        xi = np.concatenate([b.xi for b in wk.beams])
        sl = np.floor(xi / wk.dxi + 0.5)
        ref_beam = {f: np.zeros(xi.shape[0]) for f in ("ez", "wr", "bt")}
        for f in ref_beam:
            ref_beam[f][r["beam_idx"]] = r["beam"][f]
        for s in picks:
            S, S1 = snaps[s], snaps[s + 1]
            g = wm.Wake.from_workload(wk, precision=precision, flags=wm.WAKE_DUMP_RING_FIELDS)
            g.set_ring_state(s, S["r"], S["ur"], S["frprev"], S["fuprev"])
            g.step_slices(1)
            assert g.progress()[:2] == (s + 1, 0), (k, s, g.progress())
            d = g.ring_dumps()
            rho, ur = g.ring_state()
            keep = np.ones(wk.n_rings, dtype=bool)
            if precision == "mixed":
                order = np.argsort(S["r"], kind="stable")
                rs = S["r"][order]
                close = np.diff(rs) <= 5e-7 * rs[1:]
                tied = np.zeros(wk.n_rings, dtype=bool)
                tied[order[1:][close]] = True
                tied[order[:-1][close]] = True
                assert tied.mean() < 0.02, (k, s, tied.sum())
                keep = ~tied
            e = {f: BM.nerr(d[f][s][keep], S[f][keep]) for f in ("psi", "dpsidr", "dpsidz", "bp", "bb")}
            e["r"] = BM.nerr(rho[keep], S1["r"][keep])
            e["ur"] = BM.nerr(ur[keep], S1["ur"][keep])
            m = sl == s
            if m.any():
                bf = g.beam_fields()
                if precision == "mixed":
                    rr = np.zeros((s + 1, wk.n_rings))
                    rg = np.zeros((s + 1, wk.n_rings))
                    rr[s], rg[s] = S["r"], d["r"][s]
                    m &= unambiguous(W.Wake(wk.name, wk.edges, wk.beams, wk.dxi, s + 1), rr, rg)
                for f in ("ez", "wr", "bt"):
                    e["beam_" + f] = BM.nerr(bf[f][m], ref_beam[f][m])
            g.close()
            print(f"  member {k:3d} slice {s:4d}: " + " ".join(f"{f} {v:.2e}" for f, v in e.items()))
            for f, v in e.items():
                worst[f] = max(worst.get(f, 0.0), v)
                tol = FP64_TOL if precision == "fp64" else ONE_STEP_MIXED.get(f, MIXED_TOL)
                if f == "ur":
                    tol = max(tol, 1e-14)
                if f == "beam_bt" and precision == "mixed":
                    tol = 5e-5
                if not v < tol:
                    bad.append((k, s, f, v))
    print(f"\n{precision}: one-step worst over {len(ks)} members x 3 slices: {worst}")
    assert not bad, bad
