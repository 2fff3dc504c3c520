"""Pins of the oracle's table interpolation, kernel construction and rates.

* interpolation is exact at table nodes and exact everywhere for data that
  is exactly log-multilinear (EmAb/Iso) or bilinear (kernels) in the axes;
* detailed balance: with the exact Fermi--Dirac distribution in place of the
  projected one, the NES factor is exp(-(eps - eps')/T) and the pair factor is
  exp(-(eps + eps')/T) (paper, text after Eqs. detailedBalanceNES and
  detailedBalancePair);
* in-out invariance holds for NES and pair kernels;
* NES and pair collision terms vanish at equilibrium, NES conserves the number
  of each species and pair processes conserve N_s - N_sbar.
"""

import math

import numpy as np
import pytest

from oracle import opacities as op_
from oracle import solver
from oracle import eos
from oracle.equilibrium import fermi_dirac
from paper_2601_00976_gb300 import synthetic


def _linear_table(grid, ns, coef):
    """Tables whose ln-values are exactly linear in (log10 rho, log10 T, Ye, ln E)."""
    t = synthetic.make_tables(grid.eps, ns, seed=1)
    lr = np.linspace(*t["lrho"])
    lt = np.linspace(*t["lT"])
    ye = np.linspace(*t["ye"])
    lE = np.log(t["energies"])
    a, b, c, d, e = coef
    for s in range(ns):
        t["emab"][s] = (a + s + b * lr[None, None, :, None] + c * lt[None, :, None, None]
                        + d * ye[:, None, None, None] + e * lE[None, None, None, :])
    return t


def test_opacity_interp_exact_for_log_linear(grid_c1):
    coef = (-3.0, 1.0, 0.7, -2.0, 2.0)
    t = _linear_table(grid_c1, 2, coef)
    rng = np.random.default_rng(5)
    for _ in range(20):
        rho = 10 ** rng.uniform(8.5, 14.5)
        T = 10 ** rng.uniform(math.log10(0.6), math.log10(50.0))
        Ye = rng.uniform(0.06, 0.59)
        vals, clamped = op_.interpolate_opacity(t["emab"], t, rho, T, Ye)
        assert not clamped
        for s in range(2):
            exact = np.exp(coef[0] + s + coef[1] * math.log10(rho) + coef[2] * math.log10(T)
                           + coef[3] * Ye + coef[4] * np.log(t["energies"]))
            assert np.allclose(vals[s], exact, rtol=1e-12)
            E = rng.uniform(t["energies"][0], t["energies"][-1])
            v = op_.opacity_at(t, 0, s, rho, T, Ye, E)
            ex = math.exp(coef[0] + s + coef[1] * math.log10(rho) + coef[2] * math.log10(T)
                          + coef[3] * Ye + coef[4] * math.log(E))
            assert v == pytest.approx(ex, rel=1e-12)


def test_opacity_interp_exact_at_nodes(grid_c1, tables_c1_4):
    t = tables_c1_4
    lr = np.linspace(*t["lrho"])
    lt = np.linspace(*t["lT"])
    ye = np.linspace(*t["ye"])
    for (i, j, k) in [(0, 0, 0), (5, 7, 3), (31, 31, 15), (12, 20, 9)]:
        vals, _ = op_.interpolate_opacity(t["iso"], t, 10 ** lr[i], 10 ** lt[j], ye[k])
        assert np.allclose(np.log(vals), t["iso"][:, k, j, i, :], rtol=1e-12, atol=1e-12)


def test_table_clamp_flag(grid_c1, tables_c1_4):
    _, clamped = op_.interpolate_opacity(tables_c1_4["emab"], tables_c1_4, 1e16, 10.0, 0.3)
    assert clamped
    _, clamped = op_.interpolate_opacity(tables_c1_4["emab"], tables_c1_4, 1e12, 10.0, 0.3)
    assert not clamped


def test_kernel_interp_exact_for_bilinear(grid_tiny):
    t = synthetic.make_tables(grid_tiny.eps, 2, seed=2)
    lt = np.linspace(*t["klT"])
    et = np.linspace(*t["keta"])
    base = np.random.default_rng(0).uniform(1, 2, size=(grid_tiny.ne, grid_tiny.ne))
    # f = base * (1 + 0.3 log10T) * (2 + 0.01 eta): bilinear in (log10 T, eta)
    t["nes"][0] = ((1 + 0.3 * lt)[:, None, None, None] * (2 + 0.01 * et)[None, :, None, None]
                   * base[None, None])
    T, eta = 7.3, 13.7
    v, _ = op_.interpolate_kernel(t["nes"], t, T, eta)
    assert np.allclose(v[0], (1 + 0.3 * math.log10(T)) * (2 + 0.01 * eta) * base, rtol=1e-13)


def test_nes_detailed_balance_and_invariance(grid_c1, tables_c1_4):
    g = grid_c1
    T, mu = 9.0, 12.0
    f = fermi_dirac(g.eps, mu, T)               # exact FD at the nodes
    lower = tables_c1_4["nes"][0, 10, 6]
    out, inn = op_.nes_kernels(lower, f)
    assert np.array_equal(inn, out.T)           # Eq. inOutInvarianceNES
    E, Ep = np.meshgrid(g.eps, g.eps, indexing="ij")
    ratio = inn / out
    expected = np.exp(-(E - Ep) / T)            # paper: factor reduces to exp(-(eps - eps')/T)
    assert np.allclose(ratio, expected, rtol=1e-10)
    # lower triangle is the table itself
    assert np.array_equal(np.tril(out), np.tril(lower))


def test_pair_detailed_balance_and_invariance(grid_c1, tables_c1_4):
    g = grid_c1
    T, mu = 9.0, 12.0
    f = fermi_dirac(g.eps, mu, T)
    fb = fermi_dirac(g.eps, -mu, T)
    ann = tables_c1_4["pair"][0, 10, 6]
    pro_s, ann_s = op_.pair_kernels(ann, f, fb, True)
    pro_b, ann_b = op_.pair_kernels(ann, fb, f, False)
    assert np.array_equal(ann_b, ann_s.T)       # Eq. inOutInvariancePair (Ann)
    assert np.allclose(pro_b, pro_s.T, rtol=1e-14)  # Eq. inOutInvariancePair (Pro)
    E, Ep = np.meshgrid(g.eps, g.eps, indexing="ij")
    assert np.allclose(pro_s / ann_s, np.exp(-(E + Ep) / T), rtol=1e-10)


def _opac(grid, tables, mask, rho=3e12, T=10.0, Ye=0.3):
    return op_.compute_opacities(grid, tables, rho, T, Ye, (1, 1, 1, 1), mask, 1e-30, 1 - 1e-6)


def _collision(D, op, W2):
    en, cn, ep, cp = solver.compute_rates(D, op, W2)
    return (en - cn * D), (ep - cp * D)


def test_nes_and_pair_vanish_at_equilibrium(grid_c1, tables_c1_4):
    o = _opac(grid_c1, tables_c1_4, op_.NES | op_.PAIR)
    cn, cp = _collision(o["deq"], o, grid_c1.W2)
    en, chn, ep, chp = solver.compute_rates(o["deq"], o, grid_c1.W2)
    assert np.max(np.abs(cn) / np.maximum(chn * o["deq"], 1e-300)) < 1e-12
    assert np.max(np.abs(cp) / np.maximum(chp * o["deq"], 1e-300)) < 1e-12


def test_nes_conserves_number_pair_conserves_lepton_difference(grid_c1, tables_c1_4):
    o = _opac(grid_c1, tables_c1_4, op_.NES | op_.PAIR)
    rng = np.random.default_rng(11)
    D = rng.uniform(0, 1, size=(4, grid_c1.ne))
    cn, cp = _collision(D, o, grid_c1.W2)
    W2 = grid_c1.W2
    scale = np.sum(W2 * np.abs(solver.compute_rates(D, o, W2)[1] * D), axis=1)
    for s in range(4):
        assert abs(np.sum(W2 * cn[s])) <= 1e-13 * scale[s]
    for p in (0, 2):
        diff = np.sum(W2 * cp[p]) - np.sum(W2 * cp[p + 1])
        assert abs(diff) <= 1e-13 * np.sum(W2 * np.abs(cp[p]))
    # and pair production/annihilation does not conserve N_s alone
    assert abs(np.sum(W2 * cp[0])) > 1e-6 * np.sum(W2 * np.abs(cp[0]))


def test_emab_emissivity_detailed_balance(grid_c1, tables_c1_4):
    """EmAb alone: eta - chi D vanishes at D = D^Eq (Eq. emissivityEmAbNodal)."""
    o = _opac(grid_c1, tables_c1_4, op_.EMAB)
    M = np.zeros((4, grid_c1.ne, 4))
    M[:, :, 0] = o["deq"]
    Q = solver.moment_map(M, M, o, grid_c1.W2, 1e7)
    assert np.allclose(Q[:, :, 0], o["deq"], rtol=1e-13)


def test_scale_factors_and_mask(grid_c1, tables_c1_4):
    a = op_.compute_opacities(grid_c1, tables_c1_4, 1e12, 8.0, 0.3, (1, 1, 1, 1), 15, 1e-30, 1 - 1e-6)
    b = op_.compute_opacities(grid_c1, tables_c1_4, 1e12, 8.0, 0.3, (2, 3, 0.5, 4), 15, 1e-30, 1 - 1e-6)
    assert np.allclose(b["chi_ab"], 2 * a["chi_ab"])
    assert np.allclose(b["sig"], 3 * a["sig"])
    assert np.allclose(b["phi_out"], 0.5 * a["phi_out"])
    assert np.allclose(b["phi_pro"], 4 * a["phi_pro"])
    c = op_.compute_opacities(grid_c1, tables_c1_4, 1e12, 8.0, 0.3, (1, 1, 1, 1), op_.EMAB, 1e-30, 1 - 1e-6)
    assert np.all(c["sig"] == 0) and np.all(c["phi_out"] == 0) and np.all(c["phi_ann"] == 0)


def test_eta_index_uses_electron_degeneracy(grid_c1, tables_c1_4):
    rho, T, Ye = 1e13, 12.0, 0.3
    o = _opac(grid_c1, tables_c1_4, 15, rho, T, Ye)
    mu_e = eos.electron_chemical_potential(rho, T, Ye)
    assert o["eta_e"] == pytest.approx(mu_e / T)
    lower, _ = op_.interpolate_kernel(tables_c1_4["nes"], tables_c1_4, T, mu_e / T)
    assert np.allclose(np.tril(o["phi_out"][1]), np.tril(lower[1]))
