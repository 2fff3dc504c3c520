"""The NMC_TRACE build on the GPU: the fused kernel's stage counters are filled for every stage a
solve passes through, the build's results match the release build's, and the release build reports
the call unsupported.

The trace library is loaded in a child process (NMC_TRACE=1 selects it), so that the two builds never
share a process; the child prints its results as JSON.
"""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
from paper_2601_00976_gb300 import nmc
from gpu_helpers import make_case, to_device
res = {"lib": nmc.LIB_PATH}
edges, g, tables, inp = make_case(32, 1.0, 2, 4, "perturbed", 512, seed=9)
ctx = nmc.Context(edges, 2, 4, tables)
t = to_device(inp)
for name, kw in (("fp64", dict(tol_inner=1e-12, tol_outer=1e-12)), ("mixed", dict(precision=nmc.MIXED, tol_inner=1e-10, tol_outer=1e-9))):
    if nmc.LIB_PATH.endswith("_lib_trace/libnmc.so"):
        ctx.trace_read(clear=True)
    o = ctx.collision_solve(nmc.default_params(**kw), t["rho"], t["T"], t["Ye"], t["D"], t["I"], t["dt"], t["scale"])
    torch.cuda.synchronize()
    res[name + "_J"] = o["J"].cpu().numpy().ravel()[::29].tolist()
    res[name + "_inner"] = int(o["n_inner"].sum().item())
    if nmc.LIB_PATH.endswith("_lib_trace/libnmc.so"):
        res[name + "_trace"] = ctx.trace_read(clear=True)
    else:
        try:
            ctx.trace_read()
            res["unsupported"] = False
        except nmc.NmcError:
            res["unsupported"] = True
ctx.close()
print(json.dumps(res))
"""


def _run(trace):
    env = dict(os.environ)
    env.pop("NMC_TRACE", None)
    env.pop("NMC_DEBUG", None)
    if trace:
        env["NMC_TRACE"] = "1"
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_trace_build_counts_every_stage_and_matches_release():
    from paper_2601_00976_gb300 import _build, trace
    _build.build(trace=True)
    tr, rel = _run(True), _run(False)
    assert tr["lib"].endswith("_lib_trace/libnmc.so") and rel["lib"].endswith("_lib/libnmc.so")
    assert rel["unsupported"]
    for name in ("fp64", "mixed"):
        c = tr[name + "_trace"]
        assert len(c) == 16 and all(x == 0 for x in c[len(trace.STAGES):]), c
        # every stage of a solve is passed through (the queue counter too: each block takes one past the end)
        assert all(x > 0 for x in c[:len(trace.STAGES)]), (name, c)
        assert tr[name + "_inner"] == rel[name + "_inner"]
        a, b = np.asarray(tr[name + "_J"]), np.asarray(rel[name + "_J"])
        # the counters add clock reads, not arithmetic; two compilations may still round differently
        err = np.abs(a - b) / np.maximum(np.abs(b), 1e-4 * np.max(np.abs(b)))
        assert np.max(err) <= 1e-10, (name, float(np.max(err)))
