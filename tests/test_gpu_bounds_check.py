"""The bounds-checking debug build (compiled with -DWAKE_BOUNDS_CHECK, loaded
when GBWAKE_BOUNDS_CHECK=1): the on-chip marches check every swizzled
shared-memory position and every DSMEM peer rank they use.  On small parity
cases -- one CTA with rings crossing (2 and 4 rings per thread), clusters with
rings crossing CTA boundaries (2, 4 and 8 rings per thread), slices denser
than the beam stage -- no index is out of range, and the results are bitwise
those of the normal build.  Each build runs in a subprocess of its own (the
package loads one library per process)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import hashlib, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2603_16623_gb300 import wake as wm, workloads as W

axis = W.Wake("axis", W.edges_uniform(300, 5.0), [W.gaussian_beam(60_000, 5.0, 0.15, 0.5, 2.0, seed=21)], 0.01, 400)
cross = W.Wake("cross", W.edges_uniform(4915, 6.0), [W.gaussian_beam(40_000, 2.0, 1.0, 0.6, 2.4, seed=4915)], 0.01,
               300)
dense = W.Wake("dense", W.edges_uniform(200, 5.0), [W.gaussian_beam(400_000, 5.0, 0.2, 0.3, 1.2, seed=12)], 0.01, 300)
cases = [(axis, (4, 1)), (axis, (2, 1)), (cross, (0, 0)), (cross, (2, 5)), (cross, (8, 2)), (dense, (4, 1))]
out = {"violations_before": wm.debug_bounds_violations(), "runs": []}
for wk, (k, cl) in cases:
    g = wm.Wake.from_workload(wk, precision="mixed", rings_per_thread=k, cluster_ctas=cl)
    st, _, _, _ = g.run()
    h = hashlib.sha256()
    for a in g.ring_state(history=True):
        h.update(np.ascontiguousarray(a).tobytes())
    for key, a in sorted(g.beam_fields().items()):
        h.update(np.ascontiguousarray(a).tobytes())
    out["runs"].append({"case": wk.name, "launch": list(g.launch_config()), "status": int(st),
                        "progress": list(g.progress()), "digest": h.hexdigest()})
    g.close()
out["violations"] = wm.debug_bounds_violations()
print(json.dumps(out))
"""


def _run(bounds_check: bool):
    env = dict(os.environ, GBWAKE_BOUNDS_CHECK="1" if bounds_check else "0")
    res = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], capture_output=True, text=True, env=env, timeout=1200)
    assert res.returncode == 0, res.stderr[-3000:]
    return json.loads(res.stdout.strip().splitlines()[-1])


def test_no_index_out_of_range_and_the_same_results_as_the_normal_build():
    checked = _run(True)
    normal = _run(False)
    assert normal["violations"] == -1  # the normal build has no checks
    assert checked["violations_before"] == 0
    assert checked["violations"] == 0
    assert [r["launch"][1:] for r in checked["runs"]] == [[4, 1], [2, 1], [4, 5], [2, 5], [8, 2], [4, 1]]
    for a, b in zip(checked["runs"], normal["runs"]):
        assert a["status"] == b["status"] == 0, (a, b)
        assert a["progress"] == b["progress"]
        assert a["digest"] == b["digest"], a["case"]
