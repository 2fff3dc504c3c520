"""Pins of the oracle's energy grid, quadrature and equation of state.

Each check compares the oracle with something fixed independently of it: the
values printed in the paper's Table energyGrids, exact polynomial integrals,
and the defining Fermi--Dirac / Bose--Einstein integrals evaluated by adaptive
quadrature.
"""

import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import grid as ogrid
from oracle import eos
from oracle.constants import HC, HBARC, M_B
from conftest import read_golden


@pytest.mark.parametrize("row", read_golden("energy_grids.txt"))
def test_geometric_grid_matches_table(row):
    """Zoom factor and outer width of Table energyGrids from (N, de1, 300 MeV)."""
    name, n, alpha, de1, den = row[0], int(row[1]), float(row[2]), float(row[3]), float(row[4])
    edges, a = ogrid.geometric_edges(n, de1, 300.0)
    assert abs(a - alpha) <= 1e-12 * alpha, name
    assert abs(edges[-1] - 300.0) < 1e-9
    widths = np.diff(edges)
    assert abs(widths[0] - de1) < 1e-12
    # table prints the outer width to 3 significant figures
    assert float(f"{widths[-1]:.3g}") == pytest.approx(den, rel=1e-12), (name, widths[-1])


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_lg_rule_exactness(n):
    """N-point LG on (-1/2, 1/2) with unit weight sum integrates degree <= 2N-1 exactly."""
    xi, w = ogrid.lg_rule(n)
    assert abs(np.sum(w) - 1.0) < 1e-15
    assert np.all(np.abs(xi) < 0.5)
    for d in range(2 * n):
        exact = (0.5 ** (d + 1) - (-0.5) ** (d + 1)) / (d + 1)
        assert abs(np.sum(w * xi ** d) - exact) < 1e-15
    # and fails at degree 2N
    d = 2 * n
    exact = (0.5 ** (d + 1) - (-0.5) ** (d + 1)) / (d + 1)
    assert abs(np.sum(w * xi ** d) - exact) > 1e-8


def test_lagrange_basis_delta():
    xi, _ = ogrid.lg_rule(3)
    B = ogrid.lagrange_basis(xi, xi)
    assert np.allclose(B, np.eye(3), atol=1e-15)
    # partition of unity anywhere
    x = np.linspace(-0.5, 0.5, 7)
    assert np.allclose(ogrid.lagrange_basis(xi, x).sum(axis=0), 1.0, atol=1e-14)


def test_energy_weights_integrate_moments(grid_c1):
    """sum W2 = 4 pi/h^3 int eps^2 and sum W3 = 4 pi/h^3 int eps^3 exactly for k = 1."""
    g = grid_c1
    emax = g.edges[-1]
    assert np.sum(g.W2) == pytest.approx(4 * math.pi / HC ** 3 * emax ** 3 / 3, rel=1e-13)
    assert np.sum(g.W3) == pytest.approx(4 * math.pi / HC ** 3 * emax ** 4 / 4, rel=1e-13)
    # global index q = (e-1) N + q_eps: nodes increase and stay inside their element
    assert np.all(np.diff(g.eps) > 0)
    for q in range(g.ne):
        e = g.elem[q]
        assert g.edges[e] < g.eps[q] < g.edges[e + 1]
        assert e == q // g.nq


def _fd(x):
    return 1.0 / (math.exp(x) + 1.0) if x < 700 else 0.0


def _net_number_integral(mu, T):
    """(1/(pi^2 (hbar c)^3)) int eps^2 [f(eps-mu) - f(eps+mu)] d eps (two spin states)."""
    f = lambda e: e * e * (_fd((e - mu) / T) - _fd((e + mu) / T))  # noqa: E731
    v, _ = quad(f, 0.0, mu + 60.0 * T, limit=400, epsabs=0, epsrel=1e-12)
    return v / (math.pi ** 2 * HBARC ** 3)


def _energy_integral(mu, T):
    f = lambda e: e ** 3 * (_fd((e - mu) / T) + _fd((e + mu) / T))  # noqa: E731
    v, _ = quad(f, 0.0, abs(mu) + 60.0 * T, limit=400, epsabs=0, epsrel=1e-12)
    return v / (math.pi ** 2 * HBARC ** 3)


@pytest.mark.parametrize("mu,T", [(0.3, 5.0), (10.0, 3.0), (50.0, 20.0), (150.0, 15.0)])
def test_electron_gas_closed_forms(mu, T):
    """Closed forms of the massless e+e- gas against the Fermi--Dirac integrals."""
    n_closed = eos.electron_number_density(mu, T)
    assert n_closed == pytest.approx(_net_number_integral(mu, T), rel=1e-9)
    ue = (7 * math.pi ** 2 * T ** 4 / 60 + 0.5 * T * T * mu * mu + mu ** 4 / (4 * math.pi ** 2)) / HBARC ** 3
    assert ue == pytest.approx(_energy_integral(mu, T), rel=1e-9)


def test_photon_energy_density():
    T = 7.0
    f = lambda e: e ** 3 / math.expm1(e / T)  # noqa: E731
    v, _ = quad(f, 0.0, 80 * T, epsabs=0, epsrel=1e-12)
    u_int = v / (math.pi ** 2 * HBARC ** 3)
    rho, Ye = 1e10, 0.3
    u_total = eos.energy_density(rho, T, Ye)
    mu = eos.electron_chemical_potential(rho, T, Ye)
    ue = (7 * math.pi ** 2 * T ** 4 / 60 + 0.5 * T * T * mu * mu + mu ** 4 / (4 * math.pi ** 2)) / HBARC ** 3
    un = 1.5 * T * rho / M_B
    assert u_total - ue - un == pytest.approx(u_int, rel=1e-9)


@pytest.mark.parametrize("rho,T,Ye", [(1e9, 1.0, 0.5), (1e12, 7.6, 0.135), (3e14, 40.0, 0.25), (1e11, 0.6, 0.45)])
def test_chemical_potential_root(rho, T, Ye):
    """mu_e solves n_e(mu, T) = rho Ye / m_B."""
    mu = eos.electron_chemical_potential(rho, T, Ye)
    assert eos.electron_number_density(mu, T) == pytest.approx(rho * Ye / M_B, rel=1e-12)


def test_degenerate_limit():
    """T -> 0: mu_e -> hbar c (3 pi^2 n_e)^(1/3)."""
    rho, Ye = 1e13, 0.3
    ne = rho * Ye / M_B
    mu0 = HBARC * (3 * math.pi ** 2 * ne) ** (1 / 3)
    assert eos.electron_chemical_potential(rho, 1e-3, Ye) == pytest.approx(mu0, rel=1e-8)


@pytest.mark.parametrize("rho,T,Ye", [(1e9, 1.2, 0.49), (1e12, 7.6, 0.135), (2e14, 35.0, 0.26), (5e10, 3.0, 0.4)])
def test_temperature_inversion(rho, T, Ye):
    eps = eos.specific_energy(rho, T, Ye)
    T2, ok = eos.temperature(rho, eps, Ye)
    assert ok
    assert T2 == pytest.approx(T, rel=1e-13)
    # monotone in T
    assert eos.specific_energy(rho, 1.01 * T, Ye) > eps > eos.specific_energy(rho, 0.99 * T, Ye)


def test_temperature_out_of_range_flags():
    T, ok = eos.temperature(1e10, -1.0, 0.3)
    assert not ok


def test_neutrino_chemical_potentials():
    rho, T, Ye = 1e12, 7.6, 0.135
    mu_e, eta, mus = eos.chemical_potentials(rho, T, Ye, 4)
    assert eta == pytest.approx(mu_e / T)
    assert mus[1] == -mus[0] and mus[2] == 0.0 and mus[3] == 0.0
    # symmetric matter with zero mass splitting gives mu_nue = mu_e - 1.2933 at Ye = 1/2
    mu_e2, _, mus2 = eos.chemical_potentials(rho, T, 0.5, 2)
    assert mus2[0] == pytest.approx(mu_e2 - 1.2933, rel=1e-14)
