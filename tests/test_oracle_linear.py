"""Pins of the linear-order (Phi_1) NES and pair corrections in the O(v/c) oracle.

* Conservation at arbitrary moments: the NES linear terms change no species' number
  (sum_q W2 cD_s = 0) and the pair terms change no N_s - N_sbar, which holds only with the
  in-out invariance of the Phi_1 kernels (Eqs. inOutInvarianceNES, inOutInvariancePair).
* Limits: Phi_1 = 0 reproduces the isotropic-kernel solve exactly; isotropic radiation (I = 0,
  v = 0) never feels Phi_1.
* The converged state solves the unrelaxed equations with the linear terms written out here from
  Eqs. zerothMomentCollisionTerm_NES/Pair and firstMomentCollisionTerm_NES/Pair.
* An independent Newton root solve agrees on a tiny node.
* A planted mistake (the partner species' flux in the NES products) breaks the conservation pin.
"""

import numpy as np
import pytest

from oracle import solver, velocity as vel, opacities as op_
from oracle.constants import C_LIGHT
from oracle.opacities import compute_opacities
from paper_2601_00976_gb300 import synthetic

TIGHT = dict(tol_inner=1e-13, tol_outer=1e-13, max_inner=3000, max_outer=300)


def _ops(grid, mask, seed=6):
    t = synthetic.make_tables(grid.eps, 4, seed=seed, linear=True)
    return t, compute_opacities(grid, t, 3e12, 9.0, 0.3, (1, 1, 1, 1), mask, 1e-30, 1 - 1e-6)


def _moments(ne, seed):
    rng = np.random.default_rng(seed)
    D = rng.uniform(0.05, 0.9, size=(4, ne))
    I = rng.normal(size=(4, ne, 3)) * 0.3 * D[..., None]
    return np.concatenate([D[..., None], I], axis=2)


def test_linear_terms_conserve_number(grid_tiny):
    M = _moments(grid_tiny.ne, 1)
    W2 = grid_tiny.W2
    _, o = _ops(grid_tiny, op_.NES)
    cD, _ = vel.linear_corrections(M, o, W2)
    scale = np.sum(W2 * np.abs(cD), axis=1)
    assert np.all(scale > 0)
    assert np.all(np.abs(np.sum(W2 * cD, axis=1)) <= 1e-13 * scale)
    _, o = _ops(grid_tiny, op_.PAIR)
    cD, _ = vel.linear_corrections(M, o, W2)
    for s in (0, 2):
        d = np.sum(W2 * cD[s]) - np.sum(W2 * cD[s + 1])
        assert abs(d) <= 1e-13 * (np.sum(W2 * np.abs(cD[s])) + np.sum(W2 * np.abs(cD[s + 1]))), s


def test_mistake_partner_flux_in_nes_is_caught(grid_tiny, monkeypatch):
    """NES built from the partner species' flux (a plausible index slip) breaks number conservation."""
    M = _moments(grid_tiny.ne, 2)
    W2 = grid_tiny.W2
    _, o = _ops(grid_tiny, op_.NES)
    real = vel.linear_corrections

    def mutated(M_, op, W2_):
        Mp = M_.copy()
        Mp[:, :, 1:] = M_[[1, 0, 3, 2], :, 1:]        # partner's I in the <Phi_1 I> products
        cD, cI = real(Mp, op, W2_)
        # ... dotted with the species' own I, as the number term is
        A = np.stack([op["phi1_in"][s] @ (W2_[:, None] * Mp[s, :, 1:]) - op["phi1_out"][s] @ (W2_[:, None] * Mp[s, :, 1:])
                      for s in range(4)])
        return -np.sum(A * M_[:, :, 1:], axis=-1), cI
    monkeypatch.setattr(vel, "linear_corrections", mutated)
    cD, _ = vel.linear_corrections(M, o, W2)
    assert np.max(np.abs(np.sum(W2 * cD, axis=1)) / np.sum(W2 * np.abs(cD), axis=1)) > 1e-3


def _node(grid, n, linear, zero_phi1=False):
    t = synthetic.make_tables(grid.eps, 2, seed=6, linear=linear)
    if zero_phi1:
        t["nes1"] = np.zeros_like(t["nes1"])
        t["pair1"] = np.zeros_like(t["pair1"])
    inp = synthetic.make_inputs("profile", 4, grid.eps, 2, seed=40)
    return t, {k: inp[k][n] for k in ("rho", "T", "Ye", "D", "I", "dt", "scale")}


def test_limits(grid_tiny):
    P = solver.Params(**TIGHT)
    v = np.array([0.1, 0.0, 0.05])
    t0, a = _node(grid_tiny, 1, False)
    tz, _ = _node(grid_tiny, 1, True, zero_phi1=True)
    r0 = vel.solve_node(grid_tiny, t0, P, a["rho"], a["T"], a["Ye"], v, a["D"], a["I"], a["dt"], a["scale"])
    rz = vel.solve_node(grid_tiny, tz, P, a["rho"], a["T"], a["Ye"], v, a["D"], a["I"], a["dt"], a["scale"])
    assert np.array_equal(r0["D"], rz["D"]) and np.array_equal(r0["I"], rz["I"]) and r0["Ye"] == rz["Ye"]
    # isotropic radiation at rest: the linear terms are quadratic/linear in I and vanish
    t1, _ = _node(grid_tiny, 1, True)
    I0 = np.zeros_like(a["I"])
    ra = vel.solve_node(grid_tiny, t0, P, a["rho"], a["T"], a["Ye"], np.zeros(3), a["D"], I0, a["dt"], a["scale"])
    rb = vel.solve_node(grid_tiny, t1, P, a["rho"], a["T"], a["Ye"], np.zeros(3), a["D"], I0, a["dt"], a["scale"])
    assert np.array_equal(ra["D"], rb["D"]) and np.all(rb["I"] == 0.0)


def _written_out_linear(D, I, o, W2):
    """Eqs. zerothMomentCollisionTerm_NES/Pair and firstMomentCollisionTerm_NES/Pair, linear parts."""
    ns = D.shape[0]
    cD = np.zeros_like(D)
    cI = np.zeros_like(I)
    for s in range(ns):
        sb = s ^ 1
        k = vel.eddington_tensor(D[s], I[s])
        for q in range(D.shape[1]):
            Kq = k[q] * D[s, q]
            Ai = sum(o["phi1_in"][s][q, j] * W2[j] * I[s, j] for j in range(D.shape[1]))
            Ao = sum(o["phi1_out"][s][q, j] * W2[j] * I[s, j] for j in range(D.shape[1]))
            Pp = sum(o["phi1_pro"][s][q, j] * W2[j] * I[sb, j] for j in range(D.shape[1]))
            Pa = sum(o["phi1_ann"][s][q, j] * W2[j] * I[sb, j] for j in range(D.shape[1]))
            cD[s, q] = -(Ai - Ao) @ I[s, q] + (Pp - Pa) @ I[s, q]
            gK = np.eye(3) - 3.0 * Kq
            cI[s, q] = (gK @ Ai) / 3.0 + Kq @ Ao - (gK @ Pp) / 3.0 - Kq @ Pa
    return cD, cI


@pytest.mark.parametrize("n", [0, 3])
def test_converged_state_solves_unrelaxed_equations_with_linear_terms(grid_tiny, n):
    t, a = _node(grid_tiny, n, True)
    v = np.array([0.12, -0.05, 0.02])
    P = solver.Params(frozen_matter=True, **TIGHT)
    r = vel.solve_node(grid_tiny, t, P, a["rho"], a["T"], a["Ye"], v, a["D"], a["I"], a["dt"], a["scale"])
    assert r["status"] == 0
    W2 = grid_tiny.W2
    dtau = C_LIGHT * a["dt"]
    D, I = r["D"], r["I"]
    o = compute_opacities(grid_tiny, t, a["rho"], a["T"], a["Ye"], a["scale"], solver.ALL_PROCESSES, 1e-30, 1 - 1e-6)
    en, cn, ep, cp = solver.compute_rates(D, o, W2)
    eta = o["chi_ab"] * o["deq"] + en + ep
    chi = o["chi_ab"] + cn + cp
    kap = chi + o["sig"]
    cD, cI = _written_out_linear(D, I, o, W2)
    Ks = vel.eddington_tensor(a["D"], a["I"]) * a["D"][..., None, None]
    Ns = a["D"] + a["I"] @ v
    Gs = a["I"] + np.einsum("i,sqij->sqj", v, Ks)
    K = vel.eddington_tensor(D, I) * D[..., None, None]
    vK = np.einsum("i,sqij->sqj", v, K)
    rN = (D + I @ v) - Ns - dtau * (eta - chi * D + cD)
    rG = (I + vK) - Gs + dtau * kap[..., None] * I - dtau * cI
    sN = np.abs(D) + np.abs(Ns) + dtau * (np.abs(eta) + np.abs(chi * D) + np.abs(cD))
    sG = np.abs(I) + np.abs(Gs) + dtau * (np.abs(kap[..., None] * I) + np.abs(cI))
    w = W2[None, :]
    eN = np.max(np.sqrt(np.sum(w * rN ** 2, axis=1)) / np.sqrt(np.sum(w * sN ** 2, axis=1)))
    eG = np.max(np.sqrt(np.sum(w[..., None] * rG ** 2, axis=(1, 2))) / np.sqrt(np.sum(w[..., None] * sG ** 2, axis=(1, 2))))
    assert eN <= 1e-12 and eG <= 1e-12, (eN, eG)


def test_newton_agrees_with_linear_terms():
    from oracle import grid as ogrid
    edges, _ = ogrid.geometric_edges(2, 30.0)
    g = ogrid.EnergyGrid(edges, 2)
    t = synthetic.make_tables(g.eps, 2, seed=8, linear=True)
    inp = synthetic.make_inputs("profile", 2, g.eps, 2, seed=9)
    v = np.array([0.08, 0.03, -0.04])
    args = (g, t, solver.Params(**TIGHT), float(inp["rho"][1]), float(inp["T"][1]), float(inp["Ye"][1]), v,
            inp["D"][1], inp["I"][1], float(inp["dt"][1]))
    r = vel.solve_node(*args)
    rn = vel.newton_solve_node(*args)
    assert r["status"] == 0 and rn["residual"] < 1e-12
    assert np.max(np.abs(r["D"] - rn["D"])) <= 1e-11 * max(1.0, np.max(np.abs(rn["D"])))
    assert np.max(np.abs(r["I"] - rn["I"])) <= 1e-11 * max(1.0, np.max(np.abs(rn["I"])))
    assert r["Ye"] == pytest.approx(rn["Ye"], rel=1e-11)
