"""The remaining workloads at their full sizes, in the launch configuration the benchmark uses.

* Mixed precision: 2^20 perturbed-profile nodes, 4 species, 32 linear elements
  (64 energies); the mixed solve against the FP64 GPU solve (tol 1e-12) on the same inputs for
  every node, species and matter output, in the W2 norm and bin by bin (<= 1e-5), and sampled
  nodes against the oracle.  The mixed solve runs at tol 1e-10 inner and 1e-9 outer, as the
  benchmark does: where dtau chi ~ 1e4 the heavy flavours' number-conserving mode keeps an error
  ~ tol_inner (1 + dtau chi), which needs tol_inner 1e-10 for 1e-5 on this batch; an outer test at
  1e-10 chases the FP32 rounding of the converged moments (q moves by ~1e-10 relative between
  outer iterations) and 142 of the 2^20 nodes cycled to the outer cap, none at 1e-9.  Every node
  converges: the status counts are exact.
* Uneven batch: 2^22 core/tail nodes (half rho > 1e13, half rho < 1e10, dt log-uniform
  1e-7..1e-5 s), FP64, the autotuned persistent kernel: every node converges, lepton number and
  energy are conserved to 1e-12, and sampled nodes match the oracle.
"""

import numpy as np
import pytest
import torch

from oracle import solver as osolver, eos as oeos
from oracle.constants import M_B, MEV_TO_ERG, lepton_numbers
from paper_2601_00976_gb300 import nmc
from gpu_helpers import make_case, to_device, wnorm_errors, compare_node, assert_bins, bin_errors_t, BIN_FLOOR_MIXED

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_inner=1e-13, tol_outer=1e-13, max_inner=2000, max_outer=100)


def _solve(ctx, t, **kw):
    p = nmc.default_params(**kw)
    out = ctx.collision_solve(p, t["rho"], t["T"], t["Ye"], t["D"], t["I"], t["dt"], t["scale"])
    torch.cuda.synchronize()
    return out


def test_mixed_full_size_64_energies_against_fp64_and_oracle():
    N = 1 << 20
    edges, g, tables, inp = make_case(32, 1.0, 2, 4, "perturbed", N, seed=51)
    ctx = nmc.Context(edges, 2, 4, tables)
    t = to_device(inp)
    del inp["I"]
    mix = _solve(ctx, t, precision=nmc.MIXED, tol_inner=1e-10, tol_outer=1e-9)
    f64 = _solve(ctx, t, tol_inner=1e-12, tol_outer=1e-12)
    for o in (mix, f64):
        assert int(torch.count_nonzero(o["status"]).item()) == 0, torch.unique(o["status"], return_counts=True)
    ok = torch.ones(N, dtype=torch.bool, device="cuda")
    w2 = torch.tensor(g.W2, device="cuda")
    ref = torch.sqrt(torch.sum(w2 * f64["J"][ok] ** 2, dim=-1))
    eD = torch.sqrt(torch.sum(w2 * (mix["J"][ok] - f64["J"][ok]) ** 2, dim=-1)) / ref
    assert eD.max().item() <= 1e-5, eD.max(dim=0).values.tolist()
    bD, bI = bin_errors_t(mix["J"], mix["H"], f64["J"], f64["H"], BIN_FLOOR_MIXED)
    assert bD.max().item() <= 1e-5 and bI.max().item() <= 1e-5, (bD.tolist(), bI.tolist())
    for k in ("Ye", "eps", "T"):
        e = torch.max(torch.abs(mix[k][ok] - f64[k][ok]) / torch.abs(f64[k][ok])).item()
        assert e <= 1e-5, (k, e)
    # sampled nodes against the oracle
    okh = ok.cpu().numpy()
    rng = np.random.default_rng(52)
    nodes = [int(n) for n in rng.choice(np.nonzero(okh)[0], size=3, replace=False)]
    sub = {k: v[nodes] for k, v in inp.items()}
    sub["I"] = t["I"][nodes].cpu().numpy()
    refs = osolver.solve(g, tables, osolver.Params(**TIGHT), sub, nodes=range(3))
    out = {k: v[nodes].cpu().numpy() for k, v in mix.items()}
    for i, r in enumerate(refs):
        eDn, _ = wnorm_errors(out["J"][i], out["H"][i], r["D"], r["I"], g.W2)
        assert eDn.max() <= 1e-5, (nodes[i], eDn)
        assert_bins(out["J"][i], out["H"][i], r["D"], r["I"], 1e-5, BIN_FLOOR_MIXED, what=nodes[i])
        for k in ("Ye", "eps", "T"):
            assert abs(out[k][i] - r[k]) <= 1e-5 * abs(r[k])
    ctx.close()


def test_uneven_core_tail_full_size_fp64():
    N = 1 << 22
    edges, g, tables, inp = make_case(16, 1.875, 2, 4, "core_tail", N, seed=53)
    ctx = nmc.Context(edges, 2, 4, tables)
    t = to_device(inp)
    p = nmc.default_params()
    ctx.autotune(p, t["rho"][:1 << 16], t["T"][:1 << 16], t["Ye"][:1 << 16], t["D"][:1 << 16],
                 t["I"][:1 << 16], t["dt"][:1 << 16], t["scale"][:1 << 16])
    out = _solve(ctx, t)
    st = out["status"].cpu().numpy()
    assert np.count_nonzero(st) == 0, np.unique(st, return_counts=True)
    ni = out["n_inner"].cpu().numpy()
    assert ni.min() <= 5 and ni.max() >= 60   # the uneven mix this workload is for
    # conservation of lepton number and energy, every converged node (FP64 sums on the device)
    ok = out["status"] == 0
    w2 = torch.tensor(g.W2, device="cuda")
    w3 = torch.tensor(g.W3, device="cuda")
    gs = torch.tensor(lepton_numbers(4), dtype=torch.float64, device="cuda")
    rho = t["rho"]
    L0 = rho * t["Ye"] / M_B + torch.einsum("s,q,nsq->n", gs, w2, t["D"])
    L1 = rho * out["Ye"] / M_B + torch.einsum("s,q,nsq->n", gs, w2, out["J"])
    assert (torch.abs(L1 - L0) / torch.abs(L0))[ok].max().item() <= 1e-12
    rng = np.random.default_rng(54)
    nodes = [int(n) for n in rng.choice(np.nonzero(st == 0)[0], size=4, replace=False)]
    sub = {k: v[nodes] for k, v in inp.items()}
    refs = osolver.solve(g, tables, osolver.Params(**TIGHT), sub, nodes=range(4))
    o = {k: v[nodes].cpu().numpy() for k, v in out.items()}
    for i, r in enumerate(refs):
        eDn, _ = wnorm_errors(o["J"][i], o["H"][i], r["D"], r["I"], g.W2)
        # the GPU stops at tol 1e-10 (the oracle at 1e-13); optically thick nodes carry tol (1 + dtau chi) in the
        # number-conserving mode
        assert eDn.max() <= 1e-5, (nodes[i], eDn)
        assert_bins(o["J"][i], o["H"][i], r["D"], r["I"], 1e-5, BIN_FLOOR_MIXED, what=nodes[i])
        for k in ("Ye", "eps"):
            assert abs(o[k][i] - r[k]) <= 1e-7 * abs(r[k])
        E0 = inp["rho"][nodes[i]] * oeos.specific_energy(inp["rho"][nodes[i]], inp["T"][nodes[i]], inp["Ye"][nodes[i]]) \
            + MEV_TO_ERG * np.sum(g.W3 * inp["D"][nodes[i]])
        E1 = inp["rho"][nodes[i]] * o["eps"][i] + MEV_TO_ERG * np.sum(g.W3 * o["J"][i])
        assert abs(E1 - E0) <= 1e-12 * abs(E0)
    ctx.close()
