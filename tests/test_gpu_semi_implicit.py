"""GPU parity of the semi-implicit variant (Sec. 3.5: opacities evaluated once, at the old
state) against the CPU oracle, through the C ABI.

* FP64, fused and plain modes: <= 1e-10 against the oracle's semi-implicit solve (both at
  tol 1e-13), status bits equal.
* EmAb + Iso with coupled matter: the closed-form relaxation with the OLD state's opacities.
* Mixed precision against the FP64 semi-implicit solve: <= 1e-5.
* O(v/c): <= 1e-10 and velocities to 1e-12 against the oracle.
* collision_adjoint refuses it (it differentiates the fully implicit solve).
"""

import numpy as np
import pytest
import torch

from oracle import solver as osolver, opacities as oop
from oracle.constants import C_LIGHT
from paper_2601_00976_gb300 import nmc, synthetic
from gpu_helpers import (make_case, to_device, gpu_solve, compare_node, wnorm_errors, assert_bins, bin_errors,
                         BIN_FLOOR_FP64, BIN_FLOOR_MIXED)
import oracle_pool

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_inner=1e-13, tol_outer=1e-13, max_inner=2000, max_outer=100)
PARITY = 1e-10
SEMI = dict(semi_implicit=1, **TIGHT)


@pytest.fixture(scope="module")
def case():
    edges, g, tables, inp = make_case(16, 1.875, 2, 4, "profile", 16, seed=71)
    ctx = nmc.Context(edges, 2, 4, tables)
    ref = osolver.solve(g, tables, osolver.Params(semi_implicit=True, **TIGHT), inp, nodes=range(16))
    yield g, tables, inp, ctx, ref
    ctx.close()


@pytest.mark.parametrize("mode", [nmc.MODE_FUSED, nmc.MODE_PLAIN])
def test_semi_implicit_matches_oracle(case, mode):
    g, tables, inp, ctx, ref = case
    out = gpu_solve(ctx, inp, mode=mode, **SEMI)
    for n, r in enumerate(ref):
        compare_node(out, n, r, g.W2, PARITY)
        assert out["n_outer"][n] <= 3, (n, out["n_outer"][n])   # v = 0: the opacities never move


def test_closed_form_at_the_old_state():
    N = 32
    edges, g, tables, inp = make_case(16, 1.875, 2, 2, "profile", N, seed=72)
    ctx = nmc.Context(edges, 2, 2, tables)
    mask = nmc.PROC_EMAB | nmc.PROC_ISO
    out = gpu_solve(ctx, inp, proc_mask=mask, **SEMI)
    moved = 0
    for n in range(N):
        o = oop.compute_opacities(g, tables, inp["rho"][n], inp["T"][n], inp["Ye"][n], (1, 1, 1, 1), mask,
                                  1e-30, 1 - 1e-6)
        x = C_LIGHT * inp["dt"][n] * o["chi_ab"]
        D = (inp["D"][n] + x * o["deq"]) / (1 + x)
        I = inp["I"][n] / (1 + C_LIGHT * inp["dt"][n] * (o["chi_ab"] + o["sig"]))[..., None]
        assert out["status"][n] == 0
        eD, eI = wnorm_errors(out["J"][n], out["H"][n], D, I, g.W2)
        assert np.all(eD <= 1e-12) and np.all(eI <= 1e-12), (n, eD, eI)
        assert_bins(out["J"][n], out["H"][n], D, I, 1e-12, BIN_FLOOR_FP64, what=n)
        moved += abs(out["T"][n] - inp["T"][n]) > 1e-6 * inp["T"][n]
    assert moved > N // 2      # the matter state did change; the opacities stayed at the old one
    ctx.close()


def test_mixed_semi_implicit_against_fp64():
    N = 4096
    edges, g, tables, inp = make_case(16, 1.875, 2, 4, "profile", N, seed=73)
    ctx = nmc.Context(edges, 2, 4, tables)
    ref = gpu_solve(ctx, inp, semi_implicit=1, tol_inner=1e-12, tol_outer=1e-12)
    out = gpu_solve(ctx, inp, semi_implicit=1, precision=nmc.MIXED, tol_inner=1e-9, tol_outer=1e-9)
    assert np.count_nonzero(ref["status"]) == 0, np.unique(ref["status"], return_counts=True)
    assert np.count_nonzero(out["status"]) == 0, np.unique(out["status"], return_counts=True)
    worst = 0.0
    for n in range(N):
        eD, eI = wnorm_errors(out["J"][n], out["H"][n], ref["J"][n], ref["H"][n], g.W2)
        errs = [eD.max()] + [abs(out[k][n] - ref[k][n]) / abs(ref[k][n]) for k in ("Ye", "eps", "T")]
        worst = max(worst, max(errs))
    assert worst <= 1e-5, worst
    bD, bI = bin_errors(out["J"], out["H"], ref["J"], ref["H"], BIN_FLOOR_MIXED)
    assert bD.max() <= 1e-5 and bI.max() <= 1e-5, (bD.max(), bI.max())
    ctx.close()


def test_velocity_semi_implicit_matches_oracle():
    N = 8
    case = (16, 1.875, 2, 4, 0)
    edges, g, tables, inp = make_case(*case[:4], "profile", N, seed=74)
    v = synthetic.make_velocities("profile", N, seed=75)
    ctx = nmc.Context(edges, 2, 4, tables)
    t = to_device(inp)
    vt = torch.tensor(v, dtype=torch.float64, device="cuda")
    p = nmc.default_params(**SEMI)
    out = ctx.collision_solve_v(p, t["rho"], t["T"], t["Ye"], vt, t["D"], t["I"], t["dt"], t["scale"])
    torch.cuda.synchronize()
    out = {k: x.cpu().numpy() for k, x in out.items()}
    params = dict(semi_implicit=True, **TIGHT)
    tasks = [dict(case=case, params=params,
                  x=dict(rho=float(inp["rho"][n]), T=float(inp["T"][n]), Ye=float(inp["Ye"][n]), v=v[n],
                         D=inp["D"][n], I=inp["I"][n], dt=float(inp["dt"][n]), scale=inp["scale"][n]))
             for n in range(N)]
    refs = oracle_pool.run(tasks, oracle_pool.node_velocity)
    for n, r in enumerate(refs):
        assert int(out["status"][n]) == int(r["status"]), (n, out["status"][n], r["status"])
        eD, eI = wnorm_errors(out["J"][n], out["H"][n], r["D"], r["I"], g.W2)
        assert np.all(eD <= PARITY) and np.all(eI <= PARITY), (n, eD, eI)
        assert_bins(out["J"][n], out["H"][n], r["D"], r["I"], PARITY, BIN_FLOOR_FP64, what=n)
        assert np.max(np.abs(out["v"][n] - r["v"])) <= 1e-12, (n, out["v"][n], r["v"])
        for key in ("Ye", "eps", "T"):
            assert abs(out[key][n] - r[key]) <= PARITY * abs(r[key]), (n, key, out[key][n], r[key])
    ctx.close()


def test_adjoint_refuses_semi_implicit(case):
    g, tables, inp, ctx, ref = case
    t = to_device(inp)
    p = nmc.default_params(**SEMI)
    with pytest.raises(Exception, match="fully implicit"):
        ctx.collision_adjoint(p, t["rho"], t["T"], t["Ye"], t["D"], t["I"], t["dt"], t["scale"], t["D"],
                              gJ=torch.ones_like(t["D"]))
