"""Pins of the conserved-to-primitive recovery oracle (oracle/c2p.py), against things other than itself.

* Round trip: from realizable primitive moments M and |v| <= 0.35, conserved moments written out
  here from Eq. conservedToPrimitive (N = D + v.I, G_j = I_j + v^i K_ij with Minerbo's closure)
  are recovered to 1e-12.
* v = 0: the conserved moments are the primitive ones, recovered in one step.
* An independent Newton solve of U = A(M, v) M agrees.
* Picard (memory 1) and Anderson reach the same moments; the paper's contraction statement
  (|v| < sqrt(2) - 1) holds: Picard converges on every sampled bin.
* A planted sign mistake in the map is caught by the round trip.
"""

import numpy as np
import pytest

from oracle import c2p, velocity as vel


def _samples(n, vmax, seed):
    rng = np.random.default_rng(seed)
    D = rng.uniform(1e-3, 0.999, size=n)
    h = rng.uniform(0.0, 0.95, size=n)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    I = (D * h)[:, None] * d
    vd = rng.normal(size=(n, 3))
    vd /= np.linalg.norm(vd, axis=1, keepdims=True)
    v = vd * rng.uniform(0.0, vmax, size=(n, 1))
    return D, I, v


def _conserved(D, I, v):
    """Eq. conservedToPrimitive written out: N = D + v.I, G_j = I_j + v^i k_ij D."""
    k = vel.eddington_tensor(D, I)
    N = D + np.sum(I * v, axis=-1)
    G = I + np.einsum("ni,nij->nj", v, k) * D[:, None]
    return N, G


def test_round_trip_recovers_primitive_moments():
    D, I, v = _samples(300, 0.35, 1)
    N, G = _conserved(D, I, v)
    for a in range(len(D)):
        M, k, ok = c2p.recover(np.r_[N[a], G[a]], v[a], tol=1e-14, max_iter=200)
        assert ok
        assert np.max(np.abs(M - np.r_[D[a], I[a]])) <= 1e-12 * max(D[a], 1e-300), (a, M, D[a], I[a])


def test_zero_velocity_is_the_identity():
    D, I, _ = _samples(20, 0.0, 2)
    for a in range(len(D)):
        U = np.r_[D[a], I[a]]
        M, k, ok = c2p.recover(U, np.zeros(3))
        assert ok and k == 1 and np.array_equal(M, U)


def test_newton_solve_agrees():
    D, I, v = _samples(20, 0.3, 3)
    N, G = _conserved(D, I, v)
    for a in range(len(D)):
        U = np.r_[N[a], G[a]]

        def residual(M):
            k = vel.eddington_tensor(M[0], M[1:])
            return U - np.r_[M[0] + M[1:] @ v[a], M[1:] + (v[a] @ k) * M[0]]
        M = U.copy()
        for _ in range(50):
            J = np.empty((4, 4))
            for j in range(4):
                h = 1e-7 * max(abs(M[j]), 1e-8)
                e = np.zeros(4)
                e[j] = h
                J[:, j] = (residual(M + e) - residual(M - e)) / (2 * h)
            dM = np.linalg.solve(J, -residual(M))
            M = M + dM
            if np.linalg.norm(dM) <= 1e-15 * np.linalg.norm(M):
                break
        Mc, _, ok = c2p.recover(U, v[a], tol=1e-14, max_iter=200)
        assert ok and np.max(np.abs(Mc - M)) <= 1e-12 * np.linalg.norm(M)


def test_picard_and_anderson_reach_the_same_moments_and_picard_contracts():
    D, I, v = _samples(100, 0.4, 4)     # |v| < sqrt(2) - 1
    N, G = _conserved(D, I, v)
    n_aa, n_pi = 0, 0
    for a in range(len(D)):
        U = np.r_[N[a], G[a]]
        Ma, ka, oka = c2p.recover(U, v[a], tol=1e-13, memory=3, max_iter=500)
        Mp, kp, okp = c2p.recover(U, v[a], tol=1e-13, memory=1, max_iter=500)
        assert oka and okp
        assert np.max(np.abs(Ma - Mp)) <= 1e-11 * np.linalg.norm(U)
        n_aa += ka
        n_pi += kp
    assert n_aa < n_pi


def test_sign_mistake_is_caught(monkeypatch):
    D, I, v = _samples(10, 0.3, 5)
    N, G = _conserved(D, I, v)
    real = c2p.c2p_map

    def flipped(M, U, vv):
        return real(M, U, -np.asarray(vv))          # v^i I_i and v^i K_ij with the wrong sign
    monkeypatch.setattr(c2p, "c2p_map", flipped)
    errs = []
    for a in range(len(D)):
        M, _, _ = c2p.recover(np.r_[N[a], G[a]], v[a], tol=1e-14, max_iter=200)
        errs.append(np.max(np.abs(M - np.r_[D[a], I[a]])) / D[a])
    assert max(errs) > 1e-3
