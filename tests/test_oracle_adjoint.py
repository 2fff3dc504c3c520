"""Pin of the oracle's IFT gradient: central finite differences of full solves.

The gradient of L = gD . D_out + gYe Ye_out + geps eps_out with respect to the
step's inputs, from the implicit-function theorem on the converged solve, must
match central differences (h = 1e-6 relative) of Algorithm 1 itself, run to
tol 1e-14 so that the solver tolerance does not swamp the difference quotient.
"""

import numpy as np
import pytest

from oracle import solver, adjoint
from paper_2601_00976_gb300 import synthetic

TIGHT = solver.Params(tol_inner=1e-14, tol_outer=1e-14, max_inner=3000, max_outer=300)


def _loss(g, t, n, inp, gD, gYe, geps, D_star=None, Ye=None, T=None, scale=None):
    r = solver.solve_node(g, t, TIGHT, inp["rho"][n], inp["T"][n] if T is None else T,
                          inp["Ye"][n] if Ye is None else Ye,
                          inp["D"][n] if D_star is None else D_star, inp["I"][n], inp["dt"][n],
                          inp["scale"][n] if scale is None else scale)
    assert r["status"] == 0
    return float(np.sum(gD * r["D"]) + gYe * r["Ye"] + geps * r["eps"]), r


@pytest.mark.parametrize("n", [0, 1])
def test_ift_gradient_matches_finite_differences(grid_tiny, n):
    g = grid_tiny
    t = synthetic.make_tables(g.eps, 2, seed=6)
    inp = synthetic.make_inputs("profile", 2, g.eps, 2, seed=40)
    rng = np.random.default_rng(41 + n)
    gD = rng.normal(size=(2, g.ne))
    gYe, geps = rng.normal(), rng.normal() / inp["T"][n] * 1e-18
    L0, r = _loss(g, t, n, inp, gD, gYe, geps)
    grad = adjoint.gradient(g, t, TIGHT, inp["rho"][n], inp["T"][n], inp["Ye"][n], inp["D"][n], inp["dt"][n],
                            inp["scale"][n], r["D"], gD, gYe, geps)
    fd = {}
    h = 1e-6
    for key, base in (("Ye", inp["Ye"][n]), ("T", inp["T"][n])):
        Lu, _ = _loss(g, t, n, inp, gD, gYe, geps, **{key: base * (1 + h)})
        Ld, _ = _loss(g, t, n, inp, gD, gYe, geps, **{key: base * (1 - h)})
        fd[key] = (Lu - Ld) / (2 * h * base)
    fd_scale = np.empty(4)
    for k in range(4):
        su, sd = inp["scale"][n].copy(), inp["scale"][n].copy()
        su[k] *= 1 + h
        sd[k] *= 1 - h
        fd_scale[k] = (_loss(g, t, n, inp, gD, gYe, geps, scale=su)[0]
                       - _loss(g, t, n, inp, gD, gYe, geps, scale=sd)[0]) / (2 * h * inp["scale"][n][k])
    fd_D = {}
    for (s, q) in [(0, 0), (0, 5), (1, 3), (1, 7)]:
        Du, Dd = inp["D"][n].copy(), inp["D"][n].copy()
        dh = h * max(abs(Du[s, q]), 1e-8)
        Du[s, q] += dh
        Dd[s, q] -= dh
        fd_D[(s, q)] = (_loss(g, t, n, inp, gD, gYe, geps, D_star=Du)[0]
                        - _loss(g, t, n, inp, gD, gYe, geps, D_star=Dd)[0]) / (2 * dh)
    assert grad["Ye"] == pytest.approx(fd["Ye"], rel=1e-6, abs=1e-9 * abs(fd["Ye"]) + 1e-12)
    assert grad["T"] == pytest.approx(fd["T"], rel=1e-6)
    scale_ref = np.max(np.abs(fd_scale))
    assert np.max(np.abs(grad["scale"] - fd_scale)) <= 1e-6 * scale_ref, (grad["scale"], fd_scale)
    d_ref = np.max(np.abs(list(fd_D.values())))
    for (s, q), v in fd_D.items():
        assert abs(grad["D_star"][s, q] - v) <= 1e-6 * d_ref, ((s, q), grad["D_star"][s, q], v)
    assert np.all(grad["I_star"] == 0.0)
