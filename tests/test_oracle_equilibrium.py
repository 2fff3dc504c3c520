"""Pins of the oracle's equilibrium distribution D^Eq (Eq. fermiDiracProjection).

* a polynomial of degree <= k is reproduced exactly by the projection;
* the eps^2-weighted cell average equals the adaptive-quadrature integral of
  f^Eq eps^2, with and without the limiter;
* RMS error against the exact distribution converges at order k+1 on the
  paper's Grids A-F at the low-density state of Fig. FermiDiracDG;
* for k = 2 the unlimited projection goes negative in the last elements of
  Grid C while the limited one stays within bounds at the nodes and element
  interfaces (paper: Fig. FermiDiracDG discussion).
"""

import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import grid as ogrid
from oracle import equilibrium as eq
from conftest import read_golden


DMIN, DMAX = 1e-30, 1.0 - 1e-6


@pytest.mark.parametrize("nq", [1, 2, 3])
def test_projection_reproduces_polynomials(nq):
    rng = np.random.default_rng(3)
    c = rng.uniform(-1, 1, size=nq)
    f = lambda e: sum(c[j] * (e / 50.0) ** j for j in range(nq))  # noqa: E731
    coef, avg = eq.project_element(10.0, 60.0, nq, f)
    xi, _ = ogrid.lg_rule(nq)
    nodes = 35.0 + 50.0 * xi
    assert np.allclose(coef, f(nodes), atol=1e-13)


@pytest.mark.parametrize("T,mu,label", [(float(r[0]), float(r[1]), r[2]) for r in read_golden("fd_states.txt")])
@pytest.mark.parametrize("nq", [1, 2, 3])
def test_cell_average_preserved(T, mu, label, nq):
    edges, _ = ogrid.geometric_edges(16, 1.875)
    g = ogrid.EnergyGrid(edges, nq)
    f = lambda e: eq.fermi_dirac(e, mu, T)  # noqa: E731
    for limit in (False, True):
        deq = eq.equilibrium_distribution(g, mu, T, DMIN, DMAX, limit=limit)
        for e in range(g.n_elem):
            a, b = edges[e], edges[e + 1]
            num, _ = quad(lambda x: f(x) * x * x, a, b, epsabs=0, epsrel=1e-13, limit=200)
            den = (b ** 3 - a ** 3) / 3
            exact = num / den
            # eps^2-weighted average of the projected polynomial (exact quadrature)
            xg, wg = ogrid.lg_rule(8)
            x = 0.5 * (a + b) + (b - a) * xg
            p = eq.element_polynomial(g, deq, x)
            avg = np.sum(wg * p * x * x) * (b - a) / den
            if DMIN <= exact <= DMAX:
                assert avg == pytest.approx(exact, rel=1e-10, abs=1e-300), (label, e, limit)


@pytest.mark.parametrize("nq", [1, 2, 3])
def test_convergence_order_grids_a_to_f(nq):
    """RMS error at T = 7.6, mu = 3.5 MeV falls at order k+1 over Grids A-F."""
    T, mu = 7.6, 3.5
    rows = read_golden("energy_grids.txt")
    n_el, errs = [], []
    x = np.linspace(0.0, 300.0, 6001)[1:-1]
    for r in rows:
        edges, _ = ogrid.geometric_edges(int(r[1]), float(r[3]))
        g = ogrid.EnergyGrid(edges, nq)
        deq = eq.equilibrium_distribution(g, mu, T, DMIN, DMAX)
        err = eq.element_polynomial(g, deq, x) - eq.fermi_dirac(x, mu, T)
        n_el.append(int(r[1]))
        errs.append(math.sqrt(np.mean(err ** 2)))
    slope = -np.polyfit(np.log(n_el), np.log(errs), 1)[0]
    assert nq - 0.15 <= slope <= nq + 0.25, (nq, slope, errs)
    assert np.all(np.diff(errs) < 0)


def test_limiter_keeps_bounds_and_k2_undershoot():
    T, mu = 7.6, 3.5
    edges, _ = ogrid.geometric_edges(16, 1.875)
    g = ogrid.EnergyGrid(edges, 3)
    raw = eq.equilibrium_distribution(g, mu, T, DMIN, DMAX, limit=False)
    lim = eq.equilibrium_distribution(g, mu, T, DMIN, DMAX, limit=True)
    # unlimited quadratic goes negative somewhere in the last few elements
    x = np.linspace(edges[-5], 300.0, 4000)[1:-1]
    assert np.min(eq.element_polynomial(g, raw, x)) < 0.0
    # limited: within bounds at LG nodes and element interfaces, up to the
    # rounding of avg + theta (v - avg), i.e. a few ulps of the element's values
    ends = ogrid.lagrange_basis(g.xi, np.array([-0.5, 0.5]))
    for e in range(g.n_elem):
        nodal = lim[3 * e:3 * e + 3]
        v = np.concatenate([nodal, nodal @ ends])
        slack = 4e-16 * np.max(np.abs(v))
        assert np.all(v >= DMIN - slack) and np.all(v <= DMAX + slack), e


@pytest.mark.parametrize("nq", [2, 3])
def test_limited_nodal_values_strictly_inside_bounds(nq):
    """At the LG nodes the limited values lie in [D_min, D_max] exactly (no rounding slack), so that
    a = D^Eq / (1 - D^Eq) is finite and positive, over states with steep Fermi--Dirac tails on the
    coarse and fine grids; without the final clip, the quadratic case rounds some limited nodes to zero
    or below."""
    worst = 1.0
    for n_elem, de1 in ((16, 1.875), (32, 1.0)):
        edges, _ = ogrid.geometric_edges(n_elem, de1)
        g = ogrid.EnergyGrid(edges, nq)
        for T in (0.5, 1.3, 2.7, 8.0, 18.0, 33.0):
            for mu in (-20.0, 0.0, 5.0, 40.0, 110.0):
                d = eq.equilibrium_distribution(g, mu, T, DMIN, DMAX)
                assert np.all(d >= DMIN) and np.all(d <= DMAX), (n_elem, nq, T, mu, d.min(), d.max())
                a = d / (1.0 - d)
                assert np.all(np.isfinite(a)) and np.all(a > 0.0)
                worst = min(worst, float(np.min(d)))
    assert worst >= DMIN


def test_limiter_upper_bound_degenerate():
    """Degenerate state (T = 15, mu = 113): values capped at D_max, averages kept."""
    T, mu = 15.0, 113.0
    edges, _ = ogrid.geometric_edges(16, 1.875)
    g = ogrid.EnergyGrid(edges, 2)
    dmax = 1.0 - 1e-3
    lim = eq.equilibrium_distribution(g, mu, T, DMIN, dmax)
    assert np.max(lim) <= dmax
    f = eq.fermi_dirac(g.eps, mu, T)
    assert np.max(np.abs(lim - f)) < 1e-2


def test_fermi_dirac_values():
    assert eq.fermi_dirac(10.0, 10.0, 3.0) == 0.5
    assert eq.fermi_dirac(1e4, 0.0, 1.0) == 0.0
    x = np.array([1.0, 5.0, 20.0])
    assert np.allclose(eq.fermi_dirac(x, 3.0, 2.0) + eq.fermi_dirac(6.0 - x, 3.0, 2.0), 1.0)
