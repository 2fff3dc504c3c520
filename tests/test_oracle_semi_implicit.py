"""Pins of the oracle's semi-implicit variant of Algorithm 1 (Sec. 3.5: ComputeOpacities is
bypassed after the first outer iteration, so every opacity stays at the old state y*).

* EmAb + Iso with coupled matter: the returned moments are the closed-form relaxation
  D = (D* + dtau chi D^Eq)/(1 + dtau chi), I = I*/(1 + dtau (chi + sigma)) with chi, sigma and
  D^Eq at the OLD state (T*, Ye*), while the fully implicit solve misses that form by far
  more than its tolerance: the pin separates the two variants.
* Lepton number and energy are still conserved to rounding (y_out = q(M_out)).
* At v = 0 the moment map depends on the matter state only through the opacities, so the
  semi-implicit moments are the frozen-matter moments and the outer loop settles at k = 2.
* Lagging the opacities is a first-order change of the time discretisation: with
  dtau chi << 1 the gap to the fully implicit solve falls as dt^2 (ratio ~16 per factor 4).
* O(v/c): at v* = 0 with the velocity frozen it is the v = 0 semi-implicit solve; at v != 0
  the converged state solves the unrelaxed implicit equations with the old-state opacities
  and conserves momentum, energy and lepton number.
"""

import numpy as np
import pytest

from oracle import solver, velocity as vel, eos, opacities as op_
from oracle.constants import C_LIGHT, M_B, MEV_TO_ERG, lepton_numbers
from paper_2601_00976_gb300 import synthetic
from test_oracle_velocity import TIGHT, _case, unrelaxed_residuals

EMAB_ISO = op_.EMAB | op_.ISO


def _wrel(grid, x, ref):
    """Per species W2-weighted relative difference."""
    return np.sqrt(np.sum(grid.W2 * (x - ref) ** 2, axis=1)) / np.sqrt(np.sum(grid.W2 * ref ** 2, axis=1))


def _closed_form(grid, t, rho, T, Ye, D_star, I_star, dt):
    o = op_.compute_opacities(grid, t, rho, T, Ye, (1, 1, 1, 1), EMAB_ISO, 1e-30, 1 - 1e-6)
    x = C_LIGHT * dt * o["chi_ab"]
    D = (D_star + x * o["deq"]) / (1 + x)
    I = I_star / (1 + C_LIGHT * dt * (o["chi_ab"] + o["sig"]))[..., None]
    return D, I


def test_emab_iso_closed_form_at_the_old_state(grid_c1):
    t = synthetic.make_tables(grid_c1.eps, 2, seed=0)
    inp = synthetic.make_inputs("profile", 3, grid_c1.eps, 2, seed=3)
    for n in range(3):
        a = [inp[k][n] for k in ("rho", "T", "Ye", "D", "I", "dt")]
        semi = solver.solve_node(grid_c1, t, solver.Params(proc_mask=EMAB_ISO, tol_inner=1e-13, tol_outer=1e-13,
                                                           semi_implicit=True), *a)
        full = solver.solve_node(grid_c1, t, solver.Params(proc_mask=EMAB_ISO, tol_inner=1e-13, tol_outer=1e-13), *a)
        assert semi["status"] == 0 and full["status"] == 0
        D, I = _closed_form(grid_c1, t, *a)
        assert np.all(_wrel(grid_c1, semi["D"], D) < 1e-13)
        assert np.max(np.abs(semi["I"] - I)) <= 1e-13 * np.max(np.abs(I))
        # matter did change, and the fully implicit solve is not this closed form
        assert abs(semi["T"] - a[1]) > 1e-6 * a[1]
        assert np.max(_wrel(grid_c1, full["D"], D)) > 1e-7


def test_conservation_and_frozen_matter_moments(grid_c1, tables_c1_4):
    inp = synthetic.make_inputs("profile", 3, grid_c1.eps, 4, seed=7)
    g = np.asarray(lepton_numbers(4))
    for n in range(3):
        rho, T, Ye, D0, I0, dt = (inp[k][n] for k in ("rho", "T", "Ye", "D", "I", "dt"))
        r = solver.solve_node(grid_c1, tables_c1_4, solver.Params(tol_inner=1e-12, tol_outer=1e-12,
                                                                 semi_implicit=True), rho, T, Ye, D0, I0, dt)
        fz = solver.solve_node(grid_c1, tables_c1_4, solver.Params(tol_inner=1e-12, tol_outer=1e-12,
                                                                 frozen_matter=True), rho, T, Ye, D0, I0, dt)
        assert r["status"] == 0 and fz["status"] == 0
        assert r["n_outer"] <= 3
        assert np.all(_wrel(grid_c1, r["D"], fz["D"]) < 1e-10)
        eps0 = eos.specific_energy(rho, T, Ye)
        L0 = rho * Ye / M_B + np.sum(g[:, None] * grid_c1.W2 * D0)
        L1 = rho * r["Ye"] / M_B + np.sum(g[:, None] * grid_c1.W2 * r["D"])
        E0 = rho * eps0 + np.sum(grid_c1.W3 * D0) * MEV_TO_ERG
        E1 = rho * r["eps"] + np.sum(grid_c1.W3 * r["D"]) * MEV_TO_ERG
        assert abs(L1 - L0) <= 1e-12 * abs(L0)
        assert abs(E1 - E0) <= 1e-12 * abs(E0)
        assert eos.specific_energy(rho, r["T"], r["Ye"]) == pytest.approx(r["eps"], rel=1e-12)


def test_gap_to_fully_implicit_is_second_order_in_dt(grid_c1, tables_c1_4):
    inp = synthetic.make_inputs("profile", 3, grid_c1.eps, 4, seed=3)
    n = 2     # a low-density node: dtau chi << 1, where lagging the opacities costs O(dt^2)
    rho, T, Ye, D0, I0, dt0 = (inp[k][n] for k in ("rho", "T", "Ye", "D", "I", "dt"))
    gaps = []
    for f in (0.25, 0.0625, 1.0 / 64.0):
        rs = [solver.solve_node(grid_c1, tables_c1_4, solver.Params(tol_inner=1e-13, tol_outer=1e-13,
                                                                    semi_implicit=s), rho, T, Ye, D0, I0, dt0 * f)
              for s in (True, False)]
        assert all(r["status"] == 0 for r in rs)
        gaps.append(np.sqrt(np.sum(grid_c1.W2 * (rs[0]["D"] - rs[1]["D"]) ** 2))
                    / np.sqrt(np.sum(grid_c1.W2 * rs[1]["D"] ** 2)))
    for g0, g1 in zip(gaps, gaps[1:]):
        assert 13.0 < g0 / g1 < 19.0, gaps


def test_velocity_semi_implicit(grid_tiny):
    t, a = _case(grid_tiny, 0)
    P = solver.Params(semi_implicit=True, **TIGHT)
    args = (a["rho"], a["T"], a["Ye"])
    r0 = solver.solve_node(grid_tiny, t, P, *args, a["D"], a["I"], a["dt"], a["scale"])
    r1 = vel.solve_node(grid_tiny, t, P, *args, np.zeros(3), a["D"], a["I"], a["dt"], a["scale"],
                        freeze_velocity=True)
    assert r1["n_outer"] == r0["n_outer"] and r1["n_inner"] == r0["n_inner"]
    assert np.max(np.abs(r1["D"] - r0["D"])) <= 1e-14
    assert r1["Ye"] == pytest.approx(r0["Ye"], rel=1e-14)

    v = np.array([0.12, -0.05, 0.02])
    r = vel.solve_node(grid_tiny, t, P, *args, v, a["D"], a["I"], a["dt"], a["scale"])
    assert r["status"] == 0 and np.max(np.abs(r["v"] - v)) > 1e-8
    eN, eG = unrelaxed_residuals(grid_tiny, t, a, v, r, at=(a["T"], a["Ye"]))
    assert eN <= 1e-11 and eG <= 1e-11, (eN, eG)
    # with the fully implicit opacities the same residuals are not small: the old state is used
    eN_full, _ = unrelaxed_residuals(grid_tiny, t, a, v, r)
    assert eN_full > 1e3 * eN
