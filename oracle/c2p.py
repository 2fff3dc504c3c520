"""Conserved-to-primitive moment recovery (oracle), Sec. 3.4 "Primitive Moments Recovery".

TEST INFRASTRUCTURE ONLY (see the package docstring).

For given conserved moments U = (N, G_j) and fluid three-velocity v, the
primitive moments M = (D, I_j) solve U = A(M, v) M (Eq. conservedToPrimitive):
N = D + v^i I_i and G_j = I_j + v^i K_ij(M).  Written as the fixed-point map
of Eq. c2p_FP,

    g(M) = (1 - lam) M + lam (N - v^i I_i, G_j - v^i K_ij(M)),   lam = 1 / (1 + |v|),

the sequence M^[k+1] = g(M^[k]) of Eq. c2p_sequence starts from M^[0] = U and
stops when ||M^[k+1] - M^[k]|| <= tol ||U|| (Euclidean norms; tol = 1e-8 by
default), with Anderson acceleration of the sequence.

Readings (each also listed in the design notes):

* every (species, energy) bin is its own four-unknown problem (the closure
  couples nothing across bins), solved with the closure and metric of the
  O(v/c) collision solve (Minerbo, flat metric, oracle/velocity.py);
* the Anderson step is that of the collision solve's inner loop: memory M,
  constraint sum alpha = 1 eliminated, least squares by numpy's lstsq, mixed
  iterate sum alpha_j g(M_j); the stopping test compares successive iterates.
"""

import math
import numpy as np

from .velocity import rank2
from .solver import anderson_weights


def c2p_map(M, U, v):
    """g(M) of Eq. c2p_FP for one bin: M, U of shape (4,), v of shape (3,)."""
    v = np.asarray(v, dtype=float)
    lam = 1.0 / (1.0 + math.sqrt(float(v @ v)))
    K = rank2(M)
    target = np.empty(4)
    target[0] = U[0] - M[1:] @ v
    target[1:] = U[1:] - v @ K
    return (1.0 - lam) * M + lam * target


def recover(U, v, tol=1e-8, memory=3, max_iter=100):
    """(M, iterations, converged) for one bin."""
    U = np.asarray(U, dtype=float)
    M = U.copy()
    ref = tol * float(np.linalg.norm(U))
    Gh, Fh = [], []
    for k in range(1, max_iter + 1):
        g = c2p_map(M, U, v)
        Gh.append(g)
        Fh.append(g - M)
        Gh, Fh = Gh[-memory:], Fh[-memory:]
        alpha = anderson_weights(Fh)
        M_new = sum(a * gj for a, gj in zip(alpha, Gh))
        done = float(np.linalg.norm(M_new - M)) <= ref
        M = M_new
        if done:
            return M, k, True
    return M, max_iter, False


def recover_all(N, G, v, tol=1e-8, memory=3, max_iter=100):
    """Recovery over a batch: N (n, ns, ne), G (n, ns, ne, 3), v (n, 3).

    Returns D, I, iterations (n, ns, ne) and converged (n, ns, ne)."""
    n, ns, ne = N.shape
    D = np.empty_like(N)
    I = np.empty_like(G)
    it = np.empty((n, ns, ne), dtype=np.int64)
    ok = np.empty((n, ns, ne), dtype=bool)
    for a in range(n):
        for s in range(ns):
            for q in range(ne):
                U = np.concatenate([[N[a, s, q]], G[a, s, q]])
                M, k, c = recover(U, v[a], tol, memory, max_iter)
                D[a, s, q], I[a, s, q] = M[0], M[1:]
                it[a, s, q], ok[a, s, q] = k, c
    return D, I, it, ok
