"""Pins of the oracle's nested fixed-point solve (Algorithm 1).

* Anderson least squares: the weights satisfy the optimality (KKT) conditions
  of the constrained problem; memory 1 is Picard iteration;
* closed-form relaxation: with emission/absorption and isoenergetic
  scattering only and frozen matter, D = (D* + dtau chi D^Eq)/(1 + dtau chi)
  and I = I*/(1 + dtau (chi + sigma)) (Eq. implicitMomentsNodal at v = 0);
* dtau -> infinity: every species relaxes to the local Fermi--Dirac
  equilibrium of the final matter state (paper, relaxation problem);
* conservation of total lepton number n_e + N_nu and total energy
  rho eps + E_nu (Eq. collision_invariants), NES number conservation and pair
  conservation of N_s - N_sbar;
* an independent damped Newton solve of R_M = 0, R_y = 0 agrees with the
  nested Anderson iteration on tiny nodes;
* heavy flavours with identical data evolve identically (paper: nu_mu and
  nu_tau results are identical).
"""

import math

import numpy as np
import pytest

from oracle import solver, eos, opacities as op_
from oracle.constants import C_LIGHT, M_B, MEV_TO_ERG, lepton_numbers
from paper_2601_00976_gb300 import synthetic


def test_anderson_kkt():
    rng = np.random.default_rng(0)
    for m in (2, 3, 4):
        F = [rng.normal(size=20) for _ in range(m)]
        a = solver.anderson_weights(F)
        assert abs(np.sum(a) - 1.0) < 1e-14
        A = np.stack(F, axis=1)
        grad = A.T @ (A @ a)          # = lambda * 1 at the constrained optimum
        assert np.allclose(grad, grad[0], rtol=1e-9, atol=1e-12)
        # no feasible perturbation lowers the objective
        for _ in range(20):
            d = rng.normal(size=m)
            d -= d.mean()
            assert np.linalg.norm(A @ (a + 1e-3 * d)) >= np.linalg.norm(A @ a) - 1e-12
    assert np.array_equal(solver.anderson_weights([rng.normal(size=5)]), [1.0])


def test_convergence_checks():
    W2 = np.array([1.0, 4.0])
    dM = np.zeros((1, 2, 4))
    dM[0, 1, 2] = 1e-3          # I^2 change at node 1: weighted norm sqrt(4e-6) = 2e-3
    assert solver.check_inner(dM, np.array([1.0]), W2, 2.1e-3, 0.0)
    assert not solver.check_inner(dM, np.array([1.0]), W2, 1.9e-3, 0.0)
    assert solver.check_outer(np.array([1e-9, 1e-11]), np.array([1.0, 0.01]), 1e-9)
    assert not solver.check_outer(np.array([1e-9, 1e-10]), np.array([1.0, 0.01]), 1e-9)


def _inputs(grid, ns, kind="profile", N=4, seed=3):
    return synthetic.make_inputs(kind, N, grid.eps, ns, seed=seed)


def test_relaxation_closed_form(grid_c0):
    """EmAb + Iso, frozen matter: one inner update gives the closed form."""
    t = synthetic.make_tables(grid_c0.eps, 2, seed=0)
    inp = _inputs(grid_c0, 2, "uniform", N=6)
    p = solver.Params(proc_mask=op_.EMAB | op_.ISO, frozen_matter=True)
    for n in range(6):
        r = solver.solve_node(grid_c0, t, p, inp["rho"][n], inp["T"][n], inp["Ye"][n],
                              inp["D"][n], inp["I"][n], inp["dt"][n])
        o = op_.compute_opacities(grid_c0, t, inp["rho"][n], inp["T"][n], inp["Ye"][n],
                                  (1, 1, 1, 1), op_.EMAB | op_.ISO, 1e-30, 1 - 1e-6)
        x = C_LIGHT * inp["dt"][n] * o["chi_ab"]
        D = (inp["D"][n] + x * o["deq"]) / (1 + x)
        I = inp["I"][n] / (1 + C_LIGHT * inp["dt"][n] * (o["chi_ab"] + o["sig"]))[..., None]
        assert np.allclose(r["D"], D, rtol=1e-14, atol=1e-300)
        assert np.allclose(r["I"], I, rtol=1e-14, atol=1e-300)
        assert r["n_inner"] <= 2 and r["status"] == 0
        assert r["Ye"] == inp["Ye"][n] and r["T"] == inp["T"][n]


def _totals(grid, rho, Ye, eps, D):
    g = lepton_numbers(D.shape[0])
    N = np.sum(np.asarray(g)[:, None] * grid.W2[None, :] * D)
    E = np.sum(grid.W3[None, :] * D)
    lepton = rho * Ye / M_B + N
    energy = rho * eps + E * MEV_TO_ERG
    return lepton, energy


def test_coupled_emab_matches_closed_form_at_converged_state(grid_c1):
    t = synthetic.make_tables(grid_c1.eps, 2, seed=0)
    inp = _inputs(grid_c1, 2, N=3)
    p = solver.Params(proc_mask=op_.EMAB | op_.ISO, tol_inner=1e-13, tol_outer=1e-13)
    for n in range(3):
        r = solver.solve_node(grid_c1, t, p, inp["rho"][n], inp["T"][n], inp["Ye"][n],
                              inp["D"][n], inp["I"][n], inp["dt"][n])
        assert r["status"] == 0
        o = op_.compute_opacities(grid_c1, t, inp["rho"][n], r["T"], r["Ye"], (1, 1, 1, 1),
                                  op_.EMAB | op_.ISO, 1e-30, 1 - 1e-6)
        x = C_LIGHT * inp["dt"][n] * o["chi_ab"]
        D = (inp["D"][n] + x * o["deq"]) / (1 + x)
        wn = np.sqrt(np.sum(grid_c1.W2 * D ** 2, axis=1))
        err = np.sqrt(np.sum(grid_c1.W2 * (r["D"] - D) ** 2, axis=1)) / wn
        assert np.all(err < 1e-10), err


@pytest.mark.parametrize("final_q", [True, False])
def test_conservation_all_processes(grid_c1, tables_c1_4, final_q):
    inp = _inputs(grid_c1, 4, N=3, seed=7)
    tol = 1e-10
    p = solver.Params(tol_inner=tol, tol_outer=tol, final_q=final_q)
    for n in range(3):
        rho = inp["rho"][n]
        r = solver.solve_node(grid_c1, tables_c1_4, p, rho, inp["T"][n], inp["Ye"][n],
                              inp["D"][n], inp["I"][n], inp["dt"][n])
        assert r["status"] == 0
        eps0 = eos.specific_energy(rho, inp["T"][n], inp["Ye"][n])
        L0, E0 = _totals(grid_c1, rho, inp["Ye"][n], eps0, inp["D"][n])
        L1, E1 = _totals(grid_c1, rho, r["Ye"], r["eps"], r["D"])
        bound = 1e-12 if final_q else 20 * tol
        assert abs(L1 - L0) <= bound * abs(L0)
        assert abs(E1 - E0) <= bound * abs(E0)
        # the temperature returned is the EoS temperature of the returned state
        assert eos.specific_energy(rho, r["T"], r["Ye"]) == pytest.approx(r["eps"], rel=1e-12)


def test_nes_only_conserves_species_number(grid_c1, tables_c1_4):
    inp = _inputs(grid_c1, 4, N=2, seed=8)
    # a single number-conserving process is a stiff fixed-point problem: allow many iterations
    p = solver.Params(proc_mask=op_.NES, frozen_matter=True, tol_inner=1e-14, max_inner=1000)
    for n, (rho, T, Ye) in enumerate([(1e13, 15.0, 0.3), (3e12, 10.0, 0.32)]):
        r = solver.solve_node(grid_c1, tables_c1_4, p, rho, T, Ye, inp["D"][n], inp["I"][n], 1e-6)
        assert r["status"] == 0
        N0 = np.sum(grid_c1.W2 * inp["D"][n], axis=1)
        N1 = np.sum(grid_c1.W2 * r["D"], axis=1)
        # Algorithm 2 bounds the last step, not the error; for a single
        # number-conserving process the contraction is close to one, so the
        # error is the step divided by (1 - contraction): allow 1e-9.
        assert np.allclose(N1, N0, rtol=1e-9, atol=0.0)
        change = np.sqrt(np.sum(grid_c1.W2 * (r["D"] - inp["D"][n]) ** 2, axis=1))
        assert np.all(change > 1e-3 * np.sqrt(np.sum(grid_c1.W2 * inp["D"][n] ** 2, axis=1)))


def test_pair_only_conserves_lepton_difference(grid_c1, tables_c1_4):
    inp = _inputs(grid_c1, 4, N=2, seed=9)
    p = solver.Params(proc_mask=op_.PAIR, frozen_matter=True, tol_inner=1e-12, max_inner=1000)
    for n, (rho, T, Ye) in enumerate([(1e13, 15.0, 0.3), (3e12, 10.0, 0.32)]):
        r = solver.solve_node(grid_c1, tables_c1_4, p, rho, T, Ye, inp["D"][n], inp["I"][n], 1e-6)
        assert r["status"] == 0
        N0 = np.sum(grid_c1.W2 * inp["D"][n], axis=1)
        N1 = np.sum(grid_c1.W2 * r["D"], axis=1)
        for s in (0, 2):
            assert (N1[s] - N1[s + 1]) == pytest.approx(N0[s] - N0[s + 1], rel=1e-9, abs=1e-9 * N0[s])
            assert abs((N1[s] - N1[s + 1]) - (N0[s] - N0[s + 1])) <= 1e-9 * (N0[s] + N0[s + 1])
        assert abs(N1[0] - N0[0]) > 1e-6 * N0[0]


def test_long_step_reaches_equilibrium(grid_c1, tables_c1_4):
    """dtau -> infinity: D -> D^Eq(T_out, mu(rho, T_out, Ye_out)) for every species."""
    g = grid_c1
    inp = _inputs(g, 4, N=1, seed=10)
    rho, T0, Ye0 = 1e13, 15.0, 0.3
    p = solver.Params(tol_inner=1e-12, tol_outer=1e-12, max_inner=400)
    r = solver.solve_node(g, tables_c1_4, p, rho, T0, Ye0, inp["D"][0], inp["I"][0], 1.0)
    assert r["status"] & (solver.NOT_CONVERGED_OUTER | solver.NONFINITE | solver.EOS_FAIL) == 0
    o = op_.compute_opacities(g, tables_c1_4, rho, r["T"], r["Ye"], (1, 1, 1, 1), 15, 1e-30, 1 - 1e-6)
    for s in range(4):
        wn = math.sqrt(np.sum(g.W2 * o["deq"][s] ** 2))
        err = math.sqrt(np.sum(g.W2 * (r["D"][s] - o["deq"][s]) ** 2)) / wn
        assert err < 1e-6, (s, err)
    assert np.max(np.abs(r["I"])) < 1e-6 * np.max(np.abs(inp["I"][0]))
    eps0 = eos.specific_energy(rho, T0, Ye0)
    L0, E0 = _totals(g, rho, Ye0, eps0, inp["D"][0])
    L1, E1 = _totals(g, rho, r["Ye"], r["eps"], r["D"])
    assert abs(L1 - L0) <= 1e-12 * L0 and abs(E1 - E0) <= 1e-12 * E0


def test_newton_agrees_with_nested_anderson(grid_tiny):
    g = grid_tiny
    t = synthetic.make_tables(g.eps, 2, seed=4)
    inp = synthetic.make_inputs("profile", 3, g.eps, 2, seed=12)
    p = solver.Params(tol_inner=1e-14, tol_outer=1e-14, max_inner=300, max_outer=200)
    for n in range(2):
        args = (inp["rho"][n], inp["T"][n], inp["Ye"][n], inp["D"][n], inp["I"][n], inp["dt"][n])
        a = solver.solve_node(g, t, p, *args)
        b = solver.newton_solve_node(g, t, p, *args)
        assert b["residual"] < 1e-12
        wn = np.sqrt(np.sum(g.W2 * b["D"] ** 2, axis=1))
        err = np.sqrt(np.sum(g.W2 * (a["D"] - b["D"]) ** 2, axis=1)) / wn
        assert np.all(err < 1e-11), err
        assert a["Ye"] == pytest.approx(b["Ye"], rel=1e-12)
        assert a["eps"] == pytest.approx(b["eps"], rel=1e-12)
        assert a["T"] == pytest.approx(b["T"], rel=1e-11)


def test_picard_and_anderson_reach_same_fixed_point(grid_tiny):
    g = grid_tiny
    t = synthetic.make_tables(g.eps, 2, seed=4)
    inp = synthetic.make_inputs("profile", 2, g.eps, 2, seed=13)
    args = (inp["rho"][0], inp["T"][0], inp["Ye"][0], inp["D"][0], inp["I"][0], inp["dt"][0])
    a = solver.solve_node(g, t, solver.Params(tol_inner=1e-13, tol_outer=1e-13, M_inner=3, M_outer=3,
                                              max_inner=1000, max_outer=1000), *args)
    b = solver.solve_node(g, t, solver.Params(tol_inner=1e-13, tol_outer=1e-13, M_inner=1, M_outer=1,
                                              max_inner=5000, max_outer=1000), *args)
    assert a["status"] == 0 and b["status"] == 0
    assert a["n_inner"] <= b["n_inner"]
    wn = np.sqrt(np.sum(g.W2 * b["D"] ** 2, axis=1))
    assert np.all(np.sqrt(np.sum(g.W2 * (a["D"] - b["D"]) ** 2, axis=1)) < 1e-10 * wn)
    assert a["Ye"] == pytest.approx(b["Ye"], rel=1e-11)


def test_iteration_cap_sets_status(grid_c1, tables_c1_4):
    inp = _inputs(grid_c1, 4, N=1, seed=3)
    # an inner loop stopped at its cap ends the node before the matter update
    p = solver.Params(max_inner=1, max_outer=1)
    r = solver.solve_node(grid_c1, tables_c1_4, p, 5e13, 20.0, 0.3, inp["D"][0], inp["I"][0], 1e-6)
    assert r["status"] == solver.NOT_CONVERGED_INNER
    assert r["n_outer"] == 1 and r["n_inner"] == 1
    p = solver.Params(max_inner=1, max_outer=5)
    r = solver.solve_node(grid_c1, tables_c1_4, p, 5e13, 20.0, 0.3, inp["D"][0], inp["I"][0], 1e-6)
    assert r["status"] == solver.NOT_CONVERGED_INNER and r["n_outer"] == 1
    # converging inner loops with too few outer iterations
    p = solver.Params(max_outer=1)
    r = solver.solve_node(grid_c1, tables_c1_4, p, 5e13, 20.0, 0.3, inp["D"][0], inp["I"][0], 1e-6)
    assert r["status"] == solver.NOT_CONVERGED_OUTER and r["n_outer"] == 1


def test_heavy_flavours_with_identical_data_evolve_identically(grid_tiny):
    g = grid_tiny
    t = synthetic.make_tables(g.eps, 6, seed=5)
    for key in ("emab", "iso", "nes"):
        t[key][4] = t[key][2]
        t[key][5] = t[key][3]
    t["pair"][2] = t["pair"][1]
    inp = synthetic.make_inputs("profile", 2, g.eps, 6, seed=14)
    inp["D"][:, 4] = inp["D"][:, 2]
    inp["D"][:, 5] = inp["D"][:, 3]
    inp["I"][:, 4] = inp["I"][:, 2]
    inp["I"][:, 5] = inp["I"][:, 3]
    p = solver.Params()
    for n in range(2):
        r = solver.solve_node(g, t, p, inp["rho"][n], inp["T"][n], inp["Ye"][n],
                              inp["D"][n], inp["I"][n], inp["dt"][n])
        assert r["status"] == 0
        assert np.array_equal(r["D"][4], r["D"][2]) and np.array_equal(r["D"][5], r["D"][3])
        assert np.array_equal(r["I"][4], r["I"][2])
