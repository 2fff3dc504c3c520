"""Host logic of the relaxation driver (paper_2601_00976_gb300/relaxation.py), CPU only.

* The step schedule of Sec. 6.1: 1e-4 ms growing by 1.04 per step, capped at 10 ms, ending exactly
  at 100 ms (271 steps).
* The initial moments of f0 = 0.99 exp(-((eps - 2T)/sigma)^2 / 2) H(mu - mu0): by direct quadrature
  of (1/2) int f0 {1, mu} dmu over mu in [-1, 1] (the moments' definition), for mu0 = 0 (the paper's,
  flux factor 1/2) and another mu0.
"""

import math
import numpy as np
import pytest

from paper_2601_00976_gb300 import relaxation


def test_schedule_of_the_paper():
    s = relaxation.schedule()
    assert len(s) == 271
    assert s[0] == pytest.approx(1e-7, rel=1e-15)
    assert all(b == pytest.approx(min(1.04 * a, 1e-2), rel=1e-12) for a, b in zip(s[:-2], s[1:-1]))
    assert math.fsum(s) == pytest.approx(0.1, rel=1e-13)
    assert max(s) <= 1e-2
    capped = relaxation.schedule(dt0=1e-3, growth=1.5, dt_max=2e-3, t_end=0.01)
    assert max(capped) == pytest.approx(2e-3) and math.fsum(capped) == pytest.approx(0.01)


@pytest.mark.parametrize("mu0", [0.0, -0.3])
def test_initial_moments_by_quadrature(mu0):
    e = np.linspace(1.0, 60.0, 17)
    T, sigma = 7.6, 10.0
    D, I = relaxation.initial_moments(e, 3, T, sigma=sigma, mu0=mu0)
    x, w = np.polynomial.legendre.leggauss(64)          # on [-1, 1]
    for q, eq in enumerate(e):
        fE = 0.99 * math.exp(-0.5 * ((eq - 2 * T) / sigma) ** 2)
        # H(mu - mu0): integrate over [mu0, 1] with a mapped rule (the step makes [-1, 1] rules inexact)
        mu = 0.5 * (1 - mu0) * x + 0.5 * (1 + mu0)
        wm = 0.5 * (1 - mu0) * w
        assert D[:, q] == pytest.approx(0.5 * fE * np.sum(wm), rel=1e-14)
        assert I[:, q, 0] == pytest.approx(0.5 * fE * np.sum(wm * mu), rel=1e-13)
    assert np.all(I[..., 1:] == 0.0)
    if mu0 == 0.0:
        assert np.allclose(I[..., 0] / D, 0.5, rtol=1e-15)
