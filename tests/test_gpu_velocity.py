"""GPU parity of the O(v/c) solve (collision_solve_v) against the oracle (oracle/velocity.py).

* Node by node against the oracle at tol 1e-13 on both sides: D and I per species in the W2 norm
  and bin by bin (the FP64 floor of gpu_helpers), v, Ye, eps and T to 1e-10 (FP64 path), over the collapse profile with an infall velocity field
  and over isotropic random velocities up to 0.3 c.
* At the benchmark's size (2^16 profile nodes): momentum, total energy and lepton number are
  conserved to 1e-12 on every node.
* Degenerate cases: dt = 0 returns the inputs; v* = 0 with the velocity frozen is the v = 0 solve;
  |v*| >= 1 is a bad input; mixed precision and deep Anderson memories are rejected.
"""

import numpy as np
import pytest
import torch

from oracle.constants import C_LIGHT, MEV_TO_ERG, M_B, lepton_numbers
from oracle import velocity as ovel
from paper_2601_00976_gb300 import nmc, synthetic
from gpu_helpers import make_case, to_device, wnorm_errors, assert_bins, bin_errors_t, BIN_FLOOR_FP64
import oracle_pool

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_inner=1e-13, tol_outer=1e-13, max_inner=3000, max_outer=300)


def _solve_v(ctx, t, v, freeze=False, **kw):
    p = nmc.default_params(**kw)
    out = ctx.collision_solve_v(p, t["rho"], t["T"], t["Ye"], v, t["D"], t["I"], t["dt"], t["scale"],
                                freeze_velocity=freeze)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("kind,vkind,N", [("profile", "profile", 12), ("random", "random", 8)])
def test_velocity_solve_matches_oracle(kind, vkind, N):
    case = (16, 1.875, 2, 4, 0)
    edges, g, tables, inp = make_case(*case[:4], kind, N, seed=61)
    v = synthetic.make_velocities(vkind, N, seed=62, vmax=0.3 if vkind == "random" else 0.15)
    ctx = nmc.Context(edges, 2, 4, tables)
    t = to_device(inp)
    vt = torch.tensor(v, dtype=torch.float64, device="cuda")
    out = {k: x.cpu().numpy() for k, x in _solve_v(ctx, t, vt, **TIGHT).items()}
    tasks = [dict(case=case, params=TIGHT,
                  x=dict(rho=float(inp["rho"][n]), T=float(inp["T"][n]), Ye=float(inp["Ye"][n]), v=v[n],
                         D=inp["D"][n], I=inp["I"][n], dt=float(inp["dt"][n]), scale=inp["scale"][n]))
             for n in range(N)]
    refs = oracle_pool.run(tasks, oracle_pool.node_velocity)
    for n, r in enumerate(refs):
        assert int(out["status"][n]) == int(r["status"]), (n, out["status"][n], r["status"])
        eD, eI = wnorm_errors(out["J"][n], out["H"][n], r["D"], r["I"], g.W2)
        assert np.all(eD <= 1e-10) and np.all(eI <= 1e-10), (n, eD, eI)
        assert_bins(out["J"][n], out["H"][n], r["D"], r["I"], 1e-10, BIN_FLOOR_FP64, what=n)
        assert np.max(np.abs(out["v"][n] - r["v"])) <= 1e-12, (n, out["v"][n], r["v"])
        for key in ("Ye", "eps", "T"):
            assert abs(out[key][n] - r[key]) <= 1e-10 * abs(r[key]), (n, key, out[key][n], r[key])


def test_conservation_at_full_size():
    N = 1 << 16
    edges, g, tables, inp = make_case(16, 1.875, 2, 4, "profile", N, seed=63)
    v = synthetic.make_velocities("profile", N, seed=64)
    ctx = nmc.Context(edges, 2, 4, tables)
    t = to_device(inp)
    vt = torch.tensor(v, dtype=torch.float64, device="cuda")
    out = _solve_v(ctx, t, vt)
    ok = out["status"] == 0
    assert int(torch.count_nonzero(out["status"]).item()) == 0, torch.unique(out["status"], return_counts=True)
    W2 = torch.tensor(g.W2, device="cuda")
    W3 = torch.tensor(g.W3, device="cuda")
    gs = torch.tensor(lepton_numbers(4), dtype=torch.float64, device="cuda")
    rho = t["rho"]

    def totals(D, I, vv, eps_f, Ye):
        # Eqs. eulerianMomentumLG, eulerianEnergyLG, eulerianNumberLG with K from the closure
        k = torch.tensor(ovel.eddington_tensor(D.cpu().numpy(), I.cpu().numpy()), device="cuda")
        K = k * D[..., None, None]
        vI = torch.einsum("nsqi,ni->nsq", I, vv)
        F = torch.einsum("q,nsqj->nj", W3, I + D[..., None] * vv[:, None, None, :]
                         + torch.einsum("nk,nsqjk->nsqj", vv, K))
        E = torch.einsum("q,nsq->n", W3, D + 2 * vI)
        N_ = torch.einsum("s,q,nsq->n", gs, W2, D + vI)
        return (rho[:, None] * vv * C_LIGHT ** 2 + F * MEV_TO_ERG, rho * eps_f + E * MEV_TO_ERG,
                rho * Ye / M_B + N_)

    from oracle import eos as oeos
    eps0 = torch.tensor([oeos.specific_energy(float(r), float(T), float(y))
                         for r, T, y in zip(inp["rho"], inp["T"], inp["Ye"])], dtype=torch.float64, device="cuda")
    P0, E0, L0 = totals(t["D"], t["I"], vt, eps0 + 0.5 * (vt * vt).sum(1) * C_LIGHT ** 2, t["Ye"])
    eps_f1 = out["eps"] + 0.5 * (out["v"] * out["v"]).sum(1) * C_LIGHT ** 2
    P1, E1, L1 = totals(out["J"], out["H"], out["v"], eps_f1, out["Ye"])
    eP = (torch.abs(P1 - P0).max(1).values / torch.abs(P0).max(1).values)[ok]
    eE = (torch.abs(E1 - E0) / torch.abs(E0))[ok]
    eL = (torch.abs(L1 - L0) / torch.abs(L0))[ok]
    assert eP.max().item() <= 1e-12 and eE.max().item() <= 1e-12 and eL.max().item() <= 1e-12, \
        (eP.max().item(), eE.max().item(), eL.max().item())


def test_degenerate_cases():
    N = 256
    edges, g, tables, inp = make_case(16, 1.875, 2, 4, "profile", N, seed=65)
    ctx = nmc.Context(edges, 2, 4, tables)
    t = to_device(inp)
    v = torch.tensor(synthetic.make_velocities("profile", N, seed=66), dtype=torch.float64, device="cuda")
    # no time step, no exchange
    t0 = dict(t)
    t0["dt"] = torch.zeros_like(t["dt"])
    o = _solve_v(ctx, t0, v, **TIGHT)
    assert torch.all(o["status"] == 0)
    assert torch.max(torch.abs(o["J"] - t["D"])).item() <= 1e-12
    assert torch.max(torch.abs(o["H"] - t["I"])).item() <= 1e-12
    assert torch.max(torch.abs(o["v"] - v)).item() <= 1e-15
    assert torch.max(torch.abs(o["Ye"] - t["Ye"]) / t["Ye"]).item() <= 1e-13
    # v* = 0 with the velocity frozen: the v = 0 solve
    z = torch.zeros_like(v)
    o = _solve_v(ctx, t, z, freeze=True, **TIGHT)
    p = nmc.default_params(**TIGHT)
    r = ctx.collision_solve(p, t["rho"], t["T"], t["Ye"], t["D"], t["I"], t["dt"], t["scale"])
    torch.cuda.synchronize()
    assert torch.equal(o["status"], r["status"])
    assert torch.all(o["v"] == 0)
    ref = torch.sqrt(torch.sum(torch.tensor(g.W2, device="cuda") * r["J"] ** 2, dim=-1))
    eD = torch.sqrt(torch.sum(torch.tensor(g.W2, device="cuda") * (o["J"] - r["J"]) ** 2, dim=-1)) / ref
    assert eD.max().item() <= 1e-11
    bD, bI = bin_errors_t(o["J"], o["H"], r["J"], r["H"], BIN_FLOOR_FP64)
    assert bD.max().item() <= 1e-10 and bI.max().item() <= 1e-10, (bD.tolist(), bI.tolist())
    for k in ("Ye", "eps", "T"):
        assert (torch.abs(o[k] - r[k]) / torch.abs(r[k])).max().item() <= 1e-11, k
    # |v*| >= 1: bad input, outputs = inputs
    vb = v.clone()
    vb[3] = torch.tensor([0.8, 0.7, 0.0])
    o = _solve_v(ctx, t, vb)
    assert int(o["status"][3]) == nmc.BAD_INPUT
    assert torch.equal(o["J"][3], t["D"][3]) and torch.equal(o["v"][3], vb[3])
    assert int(o["status"][4]) & nmc.BAD_INPUT == 0
    # rejected configurations
    with pytest.raises(RuntimeError):
        _solve_v(ctx, t, v, precision=nmc.MIXED)
    with pytest.raises(RuntimeError):
        _solve_v(ctx, t, v, m_inner=5)
