"""Pins of the O(v/c) oracle (oracle/velocity.py), each against something other than itself.

* Minerbo's closure at its limits (diffusion psi = 1/3, free streaming psi = 1) and the
  Eddington tensor's defining properties (trace 1, psi along n, isotropic without a flux).
* With v* = 0 and the velocity frozen it is the v = 0 solve (the deleptonization setting).
* Momentum, total energy and lepton number are conserved to rounding at v != 0.
* With dtau = 0 nothing exchanges: the outputs are the inputs.
* The converged moments satisfy the unrelaxed implicit equations (Eqs. implicitNumberNodal and
  implicitNumberFluxNodal, written out here without lambda): the lambda-form of
  Eq. implicitMomentsNodal, its v terms and the conserved old moments are all pinned by it.
* An independent damped-Newton root solve on a tiny node agrees with the nested iteration.
"""

import math
import numpy as np
import pytest

from oracle import solver, velocity as vel, eos
from oracle.constants import C_LIGHT, MEV_TO_ERG, M_B, lepton_numbers
from oracle.opacities import compute_opacities
from paper_2601_00976_gb300 import synthetic

TIGHT = dict(tol_inner=1e-13, tol_outer=1e-13, max_inner=3000, max_outer=300)


def test_minerbo_closure_limits_and_tensor_properties():
    assert vel.eddington_factor(0.0) == pytest.approx(1.0 / 3.0, abs=1e-16)
    assert vel.eddington_factor(1.0) == pytest.approx(1.0, abs=1e-15)
    h = np.linspace(0.0, 1.0, 101)
    assert np.all(np.diff(vel.eddington_factor(h)) > 0)       # more forward-peaked, larger psi
    rng = np.random.default_rng(3)
    D = rng.uniform(0.1, 1.0, size=50)
    I = rng.normal(size=(50, 3))
    I *= (rng.uniform(0, 1, size=(50, 1)) * D[:, None] / np.linalg.norm(I, axis=1, keepdims=True))
    k = vel.eddington_tensor(D, I)
    assert np.allclose(np.trace(k, axis1=1, axis2=2), 1.0, atol=1e-15)
    assert np.allclose(k, np.swapaxes(k, 1, 2), atol=0)
    n = I / np.linalg.norm(I, axis=1, keepdims=True)
    psi = vel.eddington_factor(np.linalg.norm(I, axis=1) / D)
    assert np.allclose(np.einsum("ni,nij,nj->n", n, k, n), psi, atol=1e-15)
    assert np.allclose(vel.eddington_tensor(1.0, np.zeros(3)), np.eye(3) / 3.0, atol=1e-16)


def _case(grid, n, seed=40):
    t = synthetic.make_tables(grid.eps, 2, seed=6)
    inp = synthetic.make_inputs("profile", 4, grid.eps, 2, seed=seed)
    a = {k: inp[k][n] for k in ("rho", "T", "Ye", "D", "I", "dt", "scale")}
    return t, a


@pytest.mark.parametrize("n", [0, 3])
def test_frozen_zero_velocity_is_the_v0_solve(grid_tiny, n):
    t, a = _case(grid_tiny, n)
    P = solver.Params(**TIGHT)
    r0 = solver.solve_node(grid_tiny, t, P, a["rho"], a["T"], a["Ye"], a["D"], a["I"], a["dt"], a["scale"])
    r1 = vel.solve_node(grid_tiny, t, P, a["rho"], a["T"], a["Ye"], np.zeros(3), a["D"], a["I"], a["dt"],
                        a["scale"], freeze_velocity=True)
    assert r1["n_inner"] == r0["n_inner"] and r1["n_outer"] == r0["n_outer"]
    assert np.max(np.abs(r1["D"] - r0["D"])) <= 1e-14
    assert np.max(np.abs(r1["I"] - r0["I"])) <= 1e-14 * max(1.0, np.max(np.abs(r0["I"])))
    assert r1["Ye"] == pytest.approx(r0["Ye"], rel=1e-14)
    assert r1["eps"] == pytest.approx(r0["eps"], rel=1e-14)
    assert np.all(r1["v"] == 0.0)


@pytest.mark.parametrize("n", [0, 1, 3])
def test_momentum_energy_lepton_number_conserved(grid_tiny, n):
    t, a = _case(grid_tiny, n)
    v = np.array([0.05, -0.02, 0.08])
    rho = a["rho"]
    r = vel.solve_node(grid_tiny, t, solver.Params(**TIGHT), rho, a["T"], a["Ye"], v, a["D"], a["I"], a["dt"],
                       a["scale"])
    assert r["status"] == 0
    gs = np.asarray(lepton_numbers(2))
    W2, W3 = grid_tiny.W2, grid_tiny.W3

    def totals(D, I, vv, eps_f, Ye):
        # written out from Eqs. eulerianMomentumLG, eulerianEnergyLG, eulerianNumberLG and
        # Eq. eddingtonTensor (K = k D)
        K = vel.eddington_tensor(D, I) * D[..., None, None]
        F = np.einsum("q,sqj->j", W3, I + D[..., None] * vv + np.einsum("k,sqjk->sqj", vv, K))
        E = np.sum(W3 * (D + 2 * np.einsum("sqi,i->sq", I, vv)))
        N = np.sum(gs[:, None] * W2 * (D + np.einsum("sqi,i->sq", I, vv)))
        return (rho * vv * C_LIGHT ** 2 + F * MEV_TO_ERG, rho * eps_f + E * MEV_TO_ERG, rho * Ye / M_B + N)

    eps_f0 = eos.specific_energy(rho, a["T"], a["Ye"]) + 0.5 * (v @ v) * C_LIGHT ** 2
    P0, E0, L0 = totals(a["D"], a["I"], v, eps_f0, a["Ye"])
    P1, E1, L1 = totals(r["D"], r["I"], r["v"], r["eps_f"], r["Ye"])
    assert np.max(np.abs(P1 - P0)) <= 1e-12 * np.max(np.abs(P0))
    assert abs(E1 - E0) <= 1e-12 * abs(E0)
    assert abs(L1 - L0) <= 1e-12 * abs(L0)
    assert np.max(np.abs(r["v"] - v)) > 1e-8     # momentum did move
    assert r["eps"] == pytest.approx(r["eps_f"] - 0.5 * (r["v"] @ r["v"]) * C_LIGHT ** 2, rel=1e-15)


def test_no_exchange_without_time_step(grid_tiny):
    t, a = _case(grid_tiny, 1)
    v = np.array([-0.1, 0.03, 0.0])
    r = vel.solve_node(grid_tiny, t, solver.Params(**TIGHT), a["rho"], a["T"], a["Ye"], v, a["D"], a["I"], 0.0,
                       a["scale"])
    assert np.max(np.abs(r["D"] - a["D"])) <= 1e-13
    assert np.max(np.abs(r["I"] - a["I"])) <= 1e-13
    assert np.max(np.abs(r["v"] - v)) <= 1e-15
    assert r["Ye"] == pytest.approx(a["Ye"], rel=1e-14)
    assert r["T"] == pytest.approx(a["T"], rel=1e-12)


def unrelaxed_residuals(grid, t, a, v_star, r, at=None):
    """Residuals of Eqs. implicitNumberNodal and implicitNumberFluxNodal at the returned state,
    relative to the size of their terms: (D + v.I) - N* - dtau (eta - chi D) and
    (I_j + v^i K_ij) - G*_j + dtau kappa I_j, with the opacities at the matter state `at` = (T, Ye),
    by default the returned one."""
    W2 = grid.W2
    dtau = C_LIGHT * a["dt"]
    D, I, v = r["D"], r["I"], r["v"]
    T_op, Ye_op = (r["T"], r["Ye"]) if at is None else at
    op = compute_opacities(grid, t, a["rho"], T_op, Ye_op, a["scale"], solver.ALL_PROCESSES, 1e-30, 1 - 1e-6)
    en, cn, ep, cp = solver.compute_rates(D, op, W2)
    eta = op["chi_ab"] * op["deq"] + en + ep
    chi = op["chi_ab"] + cn + cp
    kap = chi + op["sig"]
    Ks = vel.eddington_tensor(a["D"], a["I"]) * a["D"][..., None, None]
    Ns = a["D"] + a["I"] @ v_star
    Gs = a["I"] + np.einsum("i,sqij->sqj", v_star, Ks)
    K = vel.eddington_tensor(D, I) * D[..., None, None]
    rN = (D + I @ v) - Ns - dtau * (eta - chi * D)
    sN = np.abs(D) + np.abs(I @ v) + np.abs(Ns) + dtau * (np.abs(eta) + np.abs(chi * D))
    vK = np.einsum("i,sqij->sqj", v, K)
    rG = (I + vK) - Gs + dtau * kap[..., None] * I
    sG = np.abs(I) + np.abs(vK) + np.abs(Gs) + dtau * np.abs(kap[..., None] * I)

    # per species in the W2-weighted norm of Algorithm 2, relative to the norm of the terms
    def rel(r, s):
        w = W2.reshape((1, -1) + (1,) * (r.ndim - 2))
        return np.max(np.sqrt(np.sum(w * r * r, axis=tuple(range(1, r.ndim))))
                      / np.sqrt(np.sum(w * s * s, axis=tuple(range(1, s.ndim)))))
    return rel(rN, sN), rel(rG, sG)


@pytest.mark.parametrize("n,frozen", [(0, False), (3, False), (1, True)])
def test_converged_state_solves_the_unrelaxed_equations(grid_tiny, n, frozen):
    t, a = _case(grid_tiny, n)
    v = np.array([0.12, -0.05, 0.02])
    P = solver.Params(frozen_matter=frozen, **TIGHT)
    r = vel.solve_node(grid_tiny, t, P, a["rho"], a["T"], a["Ye"], v, a["D"], a["I"], a["dt"], a["scale"])
    assert r["status"] == 0
    eN, eG = unrelaxed_residuals(grid_tiny, t, a, v, r)
    # with coupled matter the moments were converged at the last matter iterate, which differs from
    # the returned (exactly conserving) state by the outer tolerance
    bar = 1e-11
    assert eN <= bar and eG <= bar, (eN, eG)


def test_newton_root_agrees_with_nested_iteration():
    from oracle import grid as ogrid
    edges, _ = ogrid.geometric_edges(2, 30.0)
    g = ogrid.EnergyGrid(edges, 2)
    t = synthetic.make_tables(g.eps, 2, seed=8)
    inp = synthetic.make_inputs("profile", 2, g.eps, 2, seed=9)
    v = np.array([0.08, 0.03, -0.04])
    args = (g, t, solver.Params(**TIGHT), float(inp["rho"][1]), float(inp["T"][1]), float(inp["Ye"][1]), v,
            inp["D"][1], inp["I"][1], float(inp["dt"][1]))
    r = vel.solve_node(*args)
    rn = vel.newton_solve_node(*args)
    assert r["status"] == 0 and rn["residual"] < 1e-12
    assert np.max(np.abs(r["D"] - rn["D"])) <= 1e-11 * max(1.0, np.max(np.abs(rn["D"])))
    assert np.max(np.abs(r["I"] - rn["I"])) <= 1e-11 * max(1.0, np.max(np.abs(rn["I"])))
    assert np.max(np.abs(r["v"] - rn["v"])) <= 1e-12
    assert r["Ye"] == pytest.approx(rn["Ye"], rel=1e-11)
    assert r["eps_f"] == pytest.approx(rn["eps_f"], rel=1e-11)


# ---- each pin above catches a plausible mistake planted in the oracle (CPU, monkeypatch) ----

def _solve_and_residual(grid, frozen=True):
    t, a = _case(grid, 0)
    v = np.array([0.12, -0.05, 0.02])
    P = solver.Params(frozen_matter=frozen, **TIGHT)
    r = vel.solve_node(grid, t, P, a["rho"], a["T"], a["Ye"], v, a["D"], a["I"], a["dt"], a["scale"])
    return max(unrelaxed_residuals(grid, t, a, v, r))


def test_mistake_lambda_missing_from_denominator_is_caught(grid_tiny, monkeypatch):
    assert _solve_and_residual(grid_tiny) <= 1e-11

    def mutated(M, U_star, op, W2, dtau, v):
        v = np.asarray(v, dtype=float)
        D, I = M[:, :, 0], M[:, :, 1:]
        en, cn, ep, cp = solver.compute_rates(D, op, W2)
        eta = op["chi_ab"] * op["deq"] + en + ep
        chi = op["chi_ab"] + cn + cp
        kap = chi + op["sig"]
        lam = 1.0 / (1.0 + math.sqrt(float(v @ v)))
        Q = np.empty_like(M)
        Q[:, :, 0] = ((1.0 - lam) * D + lam * (U_star[0] - I @ v + dtau * eta)) / (1.0 + dtau * chi)
        vK = np.einsum("i,...ij->...j", v, vel.rank2(M))
        Q[:, :, 1:] = ((1.0 - lam) * I + lam * (U_star[1] - vK)) / (1.0 + dtau * kap)[:, :, None]
        return Q
    monkeypatch.setattr(vel, "moment_map", mutated)
    assert _solve_and_residual(grid_tiny) > 1e-4


def test_mistake_old_flux_without_rank2_term_is_caught(grid_tiny, monkeypatch):
    assert _solve_and_residual(grid_tiny) <= 1e-11
    monkeypatch.setattr(vel, "conserved", lambda M, v: (M[..., 0] + M[..., 1:] @ np.asarray(v), M[..., 1:].copy()))
    assert _solve_and_residual(grid_tiny) > 1e-4


def test_mistake_momentum_update_sign_is_caught(grid_tiny, monkeypatch):
    t, a = _case(grid_tiny, 3)
    v = np.array([0.05, -0.02, 0.08])
    rho = a["rho"]

    def momentum_error():
        r = vel.solve_node(grid_tiny, t, solver.Params(**TIGHT), rho, a["T"], a["Ye"], v, a["D"], a["I"],
                           a["dt"], a["scale"])
        gs_ = lepton_numbers(2)
        F0 = vel.eulerian_sums(np.concatenate([a["D"][..., None], a["I"]], axis=2), v, grid_tiny, gs_)[0]
        F1 = vel.eulerian_sums(np.concatenate([r["D"][..., None], r["I"]], axis=2), r["v"], grid_tiny, gs_)[0]
        P0 = rho * v * C_LIGHT ** 2 + F0 * MEV_TO_ERG
        P1 = rho * r["v"] * C_LIGHT ** 2 + F1 * MEV_TO_ERG
        return np.max(np.abs(P1 - P0)) / np.max(np.abs(P0))

    assert momentum_error() <= 1e-12
    real = vel.final_matter_state

    def flipped(M, rho_, y_star, S_star, grid, g, freeze_velocity=False):
        y = real(M, rho_, y_star, S_star, grid, g, freeze_velocity)
        y[:3] = 2.0 * y_star[:3] - y[:3]      # momentum exchanged with the wrong sign
        return y
    monkeypatch.setattr(vel, "final_matter_state", flipped)
    assert momentum_error() > 1e-6
