"""Each pin must catch a plausible mistake.

Every test plants one mistake in the oracle (CPU only, via monkeypatch) and
shows that the corresponding pin's check fails on the mutated oracle while it
holds on the real one.
"""

import numpy as np
import pytest

from oracle import solver, opacities as op_, equilibrium as eq, eos, grid as ogrid
from oracle.constants import M_B, MEV_TO_ERG, C_LIGHT, lepton_numbers
from paper_2601_00976_gb300 import synthetic


def _nes_conservation_error(g, t):
    o = op_.compute_opacities(g, t, 3e12, 10.0, 0.3, (1, 1, 1, 1), op_.NES, 1e-30, 1 - 1e-6)
    D = np.random.default_rng(1).uniform(0, 1, size=(4, g.ne))
    en, cn, _, _ = solver.compute_rates(D, o, g.W2)
    c = en - cn * D
    return max(abs(np.sum(g.W2 * c[s])) / np.sum(g.W2 * np.abs(cn[s] * D[s])) for s in range(4))


def test_nes_transpose_mistake_is_caught(grid_c1, tables_c1_4, monkeypatch):
    assert _nes_conservation_error(grid_c1, tables_c1_4) < 1e-13
    real = op_.nes_kernels

    def no_transpose(lower, deq):
        out, _ = real(lower, deq)
        return out, out.copy()          # Phi_In = Phi_Out instead of its transpose
    monkeypatch.setattr(op_, "nes_kernels", no_transpose)
    assert _nes_conservation_error(grid_c1, tables_c1_4) > 1e-3


def _pair_difference_error(g, t):
    o = op_.compute_opacities(g, t, 3e12, 10.0, 0.3, (1, 1, 1, 1), op_.PAIR, 1e-30, 1 - 1e-6)
    D = np.random.default_rng(2).uniform(0, 1, size=(4, g.ne))
    _, _, ep, cp = solver.compute_rates(D, o, g.W2)
    c = ep - cp * D
    return abs(np.sum(g.W2 * c[0]) - np.sum(g.W2 * c[1])) / np.sum(g.W2 * np.abs(c[0]))


def test_pair_transpose_mistake_is_caught(grid_c1, tables_c1_4, monkeypatch):
    assert _pair_difference_error(grid_c1, tables_c1_4) < 1e-13
    real = op_.pair_kernels
    monkeypatch.setattr(op_, "pair_kernels",
                        lambda ann, ds, dsb, particle: real(ann, ds, dsb, True))   # no transpose
    assert _pair_difference_error(grid_c1, tables_c1_4) > 1e-3


def _conservation_errors(g, t):
    inp = synthetic.make_inputs("profile", 1, g.eps, 4, seed=21)
    rho = 5e12
    r = solver.solve_node(g, t, solver.Params(), rho, 12.0, 0.32, inp["D"][0], inp["I"][0], 1e-6)
    gs = np.asarray(lepton_numbers(4))
    L = lambda Ye, D: rho * Ye / M_B + np.sum(gs[:, None] * g.W2 * D)            # noqa: E731
    E = lambda e, D: rho * e + MEV_TO_ERG * np.sum(g.W3 * D)                      # noqa: E731
    eps0 = eos.specific_energy(rho, 12.0, 0.32)
    return (abs(L(r["Ye"], r["D"]) - L(0.32, inp["D"][0])) / L(0.32, inp["D"][0]),
            abs(E(r["eps"], r["D"]) - E(eps0, inp["D"][0])) / E(eps0, inp["D"][0]))


def test_matter_update_mistakes_are_caught(grid_c1, tables_c1_4, monkeypatch):
    dl, de = _conservation_errors(grid_c1, tables_c1_4)
    assert dl < 1e-12 and de < 1e-12

    real = solver.neutrino_energy_number

    def w2_for_energy(D, grid, g):
        E, N = real(D, grid, g)
        return float(np.sum(grid.W2[None, :] * D)), N      # W2 where W3 belongs
    monkeypatch.setattr(solver, "neutrino_energy_number", w2_for_energy)
    dl, de = _conservation_errors(grid_c1, tables_c1_4)
    assert de > 1e-6
    monkeypatch.undo()

    def wrong_sign(D, rho, y_star, EN_star, grid, g):
        E, N = solver.neutrino_energy_number(D, grid, g)
        return np.array([y_star[0] - (E - EN_star[0]) * MEV_TO_ERG / rho,
                         y_star[1] + M_B * (N - EN_star[1]) / rho])
    monkeypatch.setattr(solver, "matter_map", wrong_sign)
    dl, de = _conservation_errors(grid_c1, tables_c1_4)
    assert dl > 1e-6


def test_flux_opacity_mistake_is_caught(grid_c0, monkeypatch):
    """Using chi instead of kappa = chi + sigma in the I update breaks the closed form."""
    t = synthetic.make_tables(grid_c0.eps, 2, seed=0)
    inp = synthetic.make_inputs("uniform", 1, grid_c0.eps, 2, seed=4)
    p = solver.Params(proc_mask=op_.EMAB | op_.ISO, frozen_matter=True)

    def closed_form_error():
        r = solver.solve_node(grid_c0, t, p, inp["rho"][0], inp["T"][0], inp["Ye"][0],
                              inp["D"][0], inp["I"][0], inp["dt"][0])
        o = op_.compute_opacities(grid_c0, t, inp["rho"][0], inp["T"][0], inp["Ye"][0],
                                  (1, 1, 1, 1), op_.EMAB | op_.ISO, 1e-30, 1 - 1e-6)
        I = inp["I"][0] / (1 + C_LIGHT * inp["dt"][0] * (o["chi_ab"] + o["sig"]))[..., None]
        return np.max(np.abs(r["I"] - I) / np.abs(I))
    assert closed_form_error() < 1e-14
    real = solver.moment_map

    def no_sigma(M, M_star, op, W2, dtau):
        op2 = dict(op)
        op2["sig"] = np.zeros_like(op["sig"])
        return real(M, M_star, op2, W2, dtau)
    monkeypatch.setattr(solver, "moment_map", no_sigma)
    assert closed_form_error() > 1e-3


def test_projection_weight_mistake_is_caught(monkeypatch):
    """Dropping the eps^2 weight of the projection breaks the cell-average pin."""
    from scipy.integrate import quad
    T, mu = 7.6, 3.5
    a, b = 20.0, 40.0
    f = lambda e: eq.fermi_dirac(e, mu, T)   # noqa: E731
    num, _ = quad(lambda x: f(x) * x * x, a, b, epsabs=0, epsrel=1e-13)
    exact = num / ((b ** 3 - a ** 3) / 3)
    _, avg = eq.project_element(a, b, 2, f)
    assert avg == pytest.approx(exact, rel=1e-12)
    real_rule = eq.lg_rule

    def unweighted(a_, b_, nq, ff):
        xi, _ = real_rule(nq)
        xg, wg = real_rule(eq.NQUAD)
        c, h = 0.5 * (a_ + b_), b_ - a_
        eg = c + h * xg
        lg = ogrid.lagrange_basis(xi, xg)
        wt = wg * h                         # eps^2 missing
        coef = np.linalg.solve((lg * wt) @ lg.T, lg @ (wt * ff(eg)))
        return coef, np.sum(wt * ff(eg)) / np.sum(wt)
    monkeypatch.setattr(eq, "project_element", unweighted)
    _, avg = eq.project_element(a, b, 2, f)
    assert abs(avg - exact) > 1e-3 * exact


def test_limiter_removed_is_caught(monkeypatch):
    edges, _ = ogrid.geometric_edges(16, 1.875)
    g = ogrid.EnergyGrid(edges, 3)
    lim = eq.equilibrium_distribution(g, 3.5, 7.6, 1e-30, 1 - 1e-6)
    assert lim.min() > 0
    monkeypatch.setattr(eq, "limit_element", lambda coef, avg, nq, dmin, dmax: coef)
    raw = eq.equilibrium_distribution(g, 3.5, 7.6, 1e-30, 1 - 1e-6)
    ends = ogrid.lagrange_basis(g.xi, np.array([-0.5, 0.5]))
    vals = np.concatenate([raw] + [raw[3 * e:3 * e + 3] @ ends for e in range(g.n_elem)])
    assert vals.min() < 0.0


def test_anderson_constraint_mistake_is_caught(monkeypatch):
    rng = np.random.default_rng(6)
    F = [rng.normal(size=10) for _ in range(3)]
    real = solver.anderson_weights(F)
    assert abs(real.sum() - 1) < 1e-14

    def unconstrained(Fl):
        A = np.stack([x.ravel() for x in Fl[:-1]], axis=1)
        gamma, *_ = np.linalg.lstsq(A, -Fl[-1].ravel(), rcond=None)
        return np.concatenate([gamma, [1.0]])     # forgets the differences
    w = unconstrained(F)
    assert abs(w.sum() - 1) > 1e-6
