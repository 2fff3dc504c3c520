"""Approximate equilibrium distribution D^Eq (oracle).

Sec. 3.5.1, Eq. fermiDiracProjection and the paragraph after it:

1. For each energy element K_e and each Lagrange basis function ell_q find the
   polynomial D~ of degree k with
       int_K D~ ell_q eps^2 d eps = int_K f^Eq ell_q eps^2 d eps   for all q,
   i.e. the eps^2-weighted L2 projection of the Fermi--Dirac distribution
   f^Eq = 1 / (exp((eps - mu)/T) + 1)  (Eq. FermiDiracDistribution).
2. Apply a bound-enforcing limiter (Zhang & Shu) that keeps D in
   [D_min, D_max] at the LG nodes and the two element interfaces without
   changing the eps^2-weighted cell average.
3. Nodal values [D^Eq]_q are the limited polynomial at the LG nodes.

Readings of points the paper leaves open:
* both integrals use an NQUAD-point Gauss--Legendre rule per element
  (NQUAD = 16); the mass matrix integrand is a polynomial of degree 2k+2, so
  it is integrated exactly;
* when the cell average itself lies outside [D_min, D_max] no limiter can keep
  it, and the element is set to the clamped cell average (constant);
* the limited nodal values are clipped to [D_min, D_max]: in exact arithmetic
  the limiter puts the extreme check point on the bound, but the rounding of
  avg + theta (D~ - avg) is of the order of the cell average's last digit and
  can leave that point just outside, below zero where the cell average is far
  above D_min (quadratic elements on a steep Fermi--Dirac tail); the clip
  restores the property the limiter states (NaN passes through).
"""

import numpy as np
from scipy.special import expit

from .grid import lg_rule, lagrange_basis

NQUAD = 16


def fermi_dirac(eps, mu, T):
    """f^Eq = 1 / (exp((eps - mu)/T) + 1)  (Eq. FermiDiracDistribution)."""
    return expit(-(np.asarray(eps, dtype=np.float64) - mu) / T)


def project_element(a, b, nq, f):
    """Unlimited eps^2-weighted L2 projection of f on [a, b] onto degree nq-1.

    Returns (nodal coefficients at the LG nodes, eps^2-weighted average of f).
    """
    xi, _ = lg_rule(nq)
    xg, wg = lg_rule(NQUAD)
    c, h = 0.5 * (a + b), b - a
    eg = c + h * xg                       # quadrature points in energy
    lg = lagrange_basis(xi, xg)           # ell_p at quadrature points, (nq, NQUAD)
    wt = wg * eg ** 2 * h                 # eps^2 d eps weights
    mass = (lg * wt) @ lg.T               # M_pq = int ell_p ell_q eps^2
    fg = f(eg)
    rhs = lg @ (wt * fg)                  # r_q = int f ell_q eps^2
    coef = np.linalg.solve(mass, rhs)
    avg = np.sum(wt * fg) / np.sum(wt)
    return coef, avg


def limit_element(coef, avg, nq, dmin, dmax):
    """Zhang--Shu bound-enforcing limiter on one element.

    The limited polynomial is avg + theta (D~ - avg) with the largest
    theta in [0, 1] that keeps the values at the LG nodes and at the element
    interfaces inside [dmin, dmax].
    """
    if avg < dmin or avg > dmax:
        return np.full(nq, min(max(avg, dmin), dmax))
    xi, _ = lg_rule(nq)
    ends = lagrange_basis(xi, np.array([-0.5, 0.5]))      # (nq, 2)
    pts = np.concatenate([coef, coef @ ends])
    vmin, vmax = pts.min(), pts.max()
    theta = 1.0
    if vmin < dmin:
        theta = min(theta, (avg - dmin) / (avg - vmin))
    if vmax > dmax:
        theta = min(theta, (dmax - avg) / (vmax - avg))
    return np.minimum(np.maximum(avg + theta * (coef - avg), dmin), dmax)


def equilibrium_distribution(grid, mu, T, dmin, dmax, limit=True):
    """[D^Eq]_q on every node of `grid` for chemical potential mu and temperature T."""
    out = np.empty(grid.ne)
    f = lambda e: fermi_dirac(e, mu, T)  # noqa: E731
    for e in range(grid.n_elem):
        coef, avg = project_element(grid.edges[e], grid.edges[e + 1], grid.nq, f)
        if limit:
            coef = limit_element(coef, avg, grid.nq, dmin, dmax)
        out[e * grid.nq:(e + 1) * grid.nq] = coef
    return out


def element_polynomial(grid, nodal, x_energy):
    """Evaluate the piecewise polynomial with nodal values `nodal` at energies x."""
    x_energy = np.asarray(x_energy, dtype=np.float64)
    out = np.empty_like(x_energy)
    e_idx = np.clip(np.searchsorted(grid.edges, x_energy, side="right") - 1, 0, grid.n_elem - 1)
    for e in range(grid.n_elem):
        m = e_idx == e
        if not np.any(m):
            continue
        xi = (x_energy[m] - grid.center[e]) / grid.width[e]
        basis = lagrange_basis(grid.xi, xi)
        out[m] = nodal[e * grid.nq:(e + 1) * grid.nq] @ basis
    return out
