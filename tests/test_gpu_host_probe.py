"""collision_solve_host (host buffers, copies pipelined against the solve) against collision_solve,
and the FMA-pipe peak probe, through the C ABI.

The host path runs the same fused kernel on chunks of the batch, so every node's result is the one
collision_solve gives (each node is solved independently): outputs are compared bit for bit, with a
ragged last chunk, with and without opacity scale factors, from page-locked and pageable memory.
"""

import numpy as np
import pytest
import torch

from paper_2601_00976_gb300 import nmc
from gpu_helpers import make_case, to_device

pytestmark = pytest.mark.gpu


def _host_inputs(inp, pin, scale=True):
    h = {k: torch.tensor(np.ascontiguousarray(v)) for k, v in inp.items() if scale or k != "scale"}
    return {k: v.pin_memory() for k, v in h.items()} if pin else h


@pytest.mark.parametrize("precision,chunk,pin,scale", [(nmc.FP64, 700, True, True), (nmc.MIXED, 0, True, True),
                                                       (nmc.FP64, 1024, False, False)])
def test_host_path_matches_device_path(precision, chunk, pin, scale):
    N = 3000
    edges, g, tables, inp = make_case(16, 1.875, 2, 4, "profile", N, seed=41)
    if scale:
        inp["scale"] = np.random.default_rng(3).uniform(0.5, 2.0, size=(N, 4))
    ctx = nmc.Context(edges, 2, 4, tables)
    prm = nmc.default_params(precision=precision)
    t = to_device(inp)
    ref = ctx.collision_solve(prm, t["rho"], t["T"], t["Ye"], t["D"], t["I"], t["dt"], t["scale"] if scale else None)
    torch.cuda.synchronize()
    h = _host_inputs(inp, pin, scale)
    out = ctx.host_outputs(N) if pin else {k: torch.empty(v.shape, dtype=v.dtype) for k, v in ref.items()}
    for _ in range(2):   # twice: the second call reuses the context's staging
        for v in out.values():
            v.fill_(0)
        ctx.collision_solve_host(prm, h, out, chunk=chunk)
        for k in ref:
            assert torch.equal(out[k], ref[k].cpu()), k
    ctx.close()


def test_host_path_rejects_device_tensors_and_bad_sizes():
    edges, g, tables, inp = make_case(16, 1.875, 2, 4, "profile", 8, seed=42)
    ctx = nmc.Context(edges, 2, 4, tables)
    prm = nmc.default_params()
    with pytest.raises(ValueError):
        ctx.collision_solve_host(prm, to_device(inp), ctx.host_outputs(8))
    import ctypes
    L = nmc.load_library()
    rc = L.collision_solve_host(ctx._h, ctypes.byref(prm), 8, *([None] * 15), 0, None)
    assert rc == nmc.NMC_EINVAL
    rc = L.collision_solve_host(ctx._h, ctypes.byref(prm), 0, *([None] * 15), 0, None)
    assert rc == nmc.NMC_OK
    ctx.close()


def test_fma_probe_rates_are_plausible():
    """The probe's flop count and timing give FP64 and FP32 FMA rates of the GB300's order (nominal
    dense: FP64 ~1.2 TFLOP/s, FP32 ~80 TFLOP/s at the boost clock)."""
    rates = {}
    for name, prec, iters, dt in (("fp64", nmc.FP64, 2000, torch.float64), ("fp32", nmc.MIXED, 100000, torch.float32)):
        sink = torch.zeros(1, dtype=dt, device="cuda")
        nmc.fma_probe(prec, iters, sink)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fl = nmc.fma_probe(prec, iters, sink)
        e1.record()
        e1.synchronize()
        rates[name] = fl / (e0.elapsed_time(e1) * 1e-3) / 1e12
    assert 0.3 <= rates["fp64"] <= 5.0, rates
    assert 20.0 <= rates["fp32"] <= 200.0, rates
    with pytest.raises(nmc.NmcError):
        nmc.fma_probe(nmc.FP64, 0, torch.zeros(1, dtype=torch.float64, device="cuda"))


def test_smem_probe_rates_are_plausible():
    """Lane-consecutive 4-byte loads move 128 bytes per warp load at about one warp load per SM cycle
    (152 SMs at up to 2.07 GHz: ~40 TB/s); the broadcasts cost at least as much per load as one
    wavefront, and a 16-byte load of consecutive words four wavefronts."""
    sink = torch.zeros(1, dtype=torch.float32, device="cuda")
    ms = {}
    for mode in range(5):
        nmc.smem_probe(mode, 50, sink)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        loads = nmc.smem_probe(mode, 200, sink)
        e1.record()
        e1.synchronize()
        ms[mode] = e0.elapsed_time(e1) / loads
    gbs = 128.0 / (ms[nmc.SMEM_B32_CONSECUTIVE] * 1e-3) / 1e9
    assert 10e3 <= gbs <= 60e3, gbs
    rel = {m: ms[m] / ms[nmc.SMEM_B32_CONSECUTIVE] for m in ms}
    assert all(r >= 0.8 for r in rel.values()), rel
    assert 3.0 <= rel[nmc.SMEM_B128_CONSECUTIVE] <= 5.0, rel
    with pytest.raises(nmc.NmcError):
        nmc.smem_probe(7, 10, sink)
