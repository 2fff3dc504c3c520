"""Energy grid, Legendre--Gauss rule and energy integration weights (oracle).

* Geometric energy grids: Sec. 3.5 (Neutrino--matter coupling), text before
  Table energyGrids: Delta eps_{e+1} = alpha * Delta eps_e on [0, 300] MeV.
* Legendre--Gauss nodes and weights on the reference interval (-1/2, 1/2),
  weights normalised to sum to one: Sec. 3.2 (nodal DG, Eq. lagrangePolynomial
  and the quadrature paragraph after Fig. SpectralElements).
* Global energy index q = (e-1) N + q_eps and the weights
  W2_q = 4 pi w_q eps_q^2 Delta eps_e / h^3, W3_q = W2_q eps_q:
  Eq. energy_integration_weights and the paragraph after it.
"""

import math
import numpy as np

from .constants import HC


def geometric_alpha(n_elem, de1, emax=300.0):
    """Zoom factor alpha with de1 * (1 + alpha + ... + alpha^(n-1)) = emax.

    The left side increases monotonically with alpha, so plain bisection on
    [1, 4] finds the unique root.
    """
    def total(a):
        return de1 * sum(a ** i for i in range(n_elem))

    lo, hi = 1.0, 4.0
    if total(lo) > emax:
        raise ValueError("de1 * n_elem exceeds emax")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if total(mid) < emax:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def geometric_edges(n_elem, de1, emax=300.0):
    """Element interfaces eps_{1/2} = 0 < ... < eps_{N+1/2} for a geometric grid."""
    alpha = geometric_alpha(n_elem, de1, emax)
    widths = np.array([de1 * alpha ** i for i in range(n_elem)], dtype=np.float64)
    edges = np.concatenate([[0.0], np.cumsum(widths)])
    return edges, alpha


def lg_rule(n):
    """N-point Legendre--Gauss nodes on (-1/2, 1/2) and weights summing to 1."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * x, 0.5 * w


def lagrange_basis(nodes, x):
    """Values ell_p(x) of the Lagrange polynomials on `nodes` (Eq. lagrangePolynomial).

    Returns an array of shape (len(nodes),) + shape(x).
    """
    x = np.asarray(x, dtype=np.float64)
    out = []
    for p, xp in enumerate(nodes):
        v = np.ones_like(x)
        for q, xq in enumerate(nodes):
            if q != p:
                v = v * (x - xq) / (xp - xq)
        out.append(v)
    return np.array(out)


class EnergyGrid:
    """Nodal energy grid of one spatial point.

    edges : element interfaces (MeV), length n_elem + 1
    nq    : nodes per element, N = k + 1
    """

    def __init__(self, edges, nq):
        self.edges = np.asarray(edges, dtype=np.float64)
        self.n_elem = len(self.edges) - 1
        self.nq = int(nq)
        self.xi, self.w = lg_rule(self.nq)
        self.center = 0.5 * (self.edges[:-1] + self.edges[1:])
        self.width = self.edges[1:] - self.edges[:-1]
        ne = self.n_elem * self.nq
        self.ne = ne
        self.eps = np.empty(ne)
        self.elem = np.empty(ne, dtype=np.int64)
        self.wq = np.empty(ne)
        for e in range(self.n_elem):
            for qe in range(self.nq):
                q = e * self.nq + qe            # global index q = (e-1)N + q_eps
                self.eps[q] = self.center[e] + self.width[e] * self.xi[qe]
                self.elem[q] = e
                self.wq[q] = self.w[qe]
        # W^(2)_q = 4 pi w eps^2 Delta eps / h^3  [cm^-3]
        self.W2 = 4.0 * math.pi * self.wq * self.eps ** 2 * self.width[self.elem] / HC ** 3
        # W^(3)_q = W^(2)_q eps_q  [MeV cm^-3]
        self.W3 = self.W2 * self.eps
