"""Pin of the oracle's IFT gradient: central finite differences of full solves.

The gradient of L = gD . D_out + gYe Ye_out + geps eps_out + gT T_out + gH . H_out
with respect to the step's inputs, from the implicit-function theorem on the
converged solve, must match fourth-order central differences (h = 1e-5 relative) of
Algorithm 1 itself, run to tol 1e-14 so that the solver tolerance does not
swamp the difference quotient.  Coupled and frozen matter are both checked.
"""

import numpy as np
import pytest

from oracle import solver, adjoint, eos
from paper_2601_00976_gb300 import synthetic

TIGHT = dict(tol_inner=1e-14, tol_outer=1e-14, max_inner=3000, max_outer=300)


class _Case:
    def __init__(self, grid, n, frozen, seed):
        self.g = grid
        self.params = solver.Params(frozen_matter=frozen, **TIGHT)
        self.t = synthetic.make_tables(grid.eps, 2, seed=6)
        self.inp = synthetic.make_inputs("profile", 2, grid.eps, 2, seed=40)
        self.n = n
        rng = np.random.default_rng(seed)
        ne = grid.ne
        self.gD = rng.normal(size=(2, ne))
        self.gYe = rng.normal()
        self.geps = rng.normal() * 1e-18
        self.gT = rng.normal()
        self.gH = rng.normal(size=(2, ne, 3))

    def loss(self, **over):
        i, n = self.inp, self.n
        args = dict(rho=i["rho"][n], T=i["T"][n], Ye=i["Ye"][n], D=i["D"][n], I=i["I"][n], scale=i["scale"][n])
        args.update(over)
        r = solver.solve_node(self.g, self.t, self.params, args["rho"], args["T"], args["Ye"], args["D"],
                              args["I"], i["dt"][n], args["scale"])
        assert r["status"] == 0
        L = (np.sum(self.gD * r["D"]) + self.gYe * r["Ye"] + self.geps * r["eps"] + self.gT * r["T"]
             + np.sum(self.gH * r["I"]))
        return float(L), r


@pytest.mark.parametrize("n,frozen", [(0, 0), (1, 0), (1, 1)])
def test_ift_gradient_matches_finite_differences(grid_tiny, n, frozen):
    c = _Case(grid_tiny, n, frozen, seed=41 + n + 7 * frozen)
    i = c.inp
    _, r = c.loss()
    grad = adjoint.gradient(c.g, c.t, c.params, i["rho"][n], i["T"][n], i["Ye"][n], i["D"][n], i["I"][n],
                            i["dt"][n], i["scale"][n], r["D"], gD=c.gD, gYe=c.gYe, geps=c.geps, gT=c.gT, gH=c.gH)
    h = 1e-5
    # fourth-order central differences of full solves; steps in D* scaled per entry by the change that
    # moves the matter state by O(1) relative (the solve is smooth on that scale)
    eps_star = eos.specific_energy(i["rho"][n], i["T"][n], i["Ye"][n])
    sD = adjoint.natural_scale(c.g, c.params, i["rho"][n], eps_star, i["Ye"][n], 2)

    def central(key, base, idx=None, step=None):
        def L(t):
            if idx is None:
                return c.loss(**{key: base + t})[0]
            v = base.copy()
            v[idx] += t
            return c.loss(**{key: v})[0]
        d = step if step is not None else h * abs(base if idx is None else base[idx])
        return (8 * (L(d) - L(-d)) - (L(2 * d) - L(-2 * d))) / (12 * d)

    fd_Ye = central("Ye", i["Ye"][n])
    fd_T = central("T", i["T"][n])
    assert grad["Ye"] == pytest.approx(fd_Ye, rel=1e-6, abs=1e-6 * abs(fd_T) * i["T"][n] / i["Ye"][n])
    assert grad["T"] == pytest.approx(fd_T, rel=1e-6)
    fd_scale = np.array([central("scale", i["scale"][n], k, h * max(i["scale"][n][k], 1e-3)) for k in range(4)])
    assert np.max(np.abs(grad["scale"] - fd_scale)) <= 1e-6 * np.max(np.abs(fd_scale)), (grad["scale"], fd_scale)
    fd_D = {sq: central("D", i["D"][n], sq, h * sD[sq]) for sq in [(0, 0), (0, 5), (1, 3), (1, 7)]}
    d_ref = max(abs(v) for v in fd_D.values())
    for sq, v in fd_D.items():
        assert abs(grad["D_star"][sq] - v) <= 1e-6 * abs(v) + 1e-9 * d_ref, (sq, grad["D_star"][sq], v)
    hI = h * np.max(np.abs(i["I"][n]))
    fd_I = {sqc: central("I", i["I"][n], sqc, hI) for sqc in [(0, 1, 0), (0, 6, 2), (1, 2, 1), (1, 7, 0)]}
    i_ref = max(abs(v) for v in fd_I.values())
    for sqc, v in fd_I.items():
        assert abs(grad["I_star"][sqc] - v) <= 1e-6 * abs(v) + 1e-9 * i_ref, (sqc, grad["I_star"][sqc], v)


def test_gradient_without_first_moment_cotangent_ignores_I_star(grid_tiny):
    """With gH = 0 the outputs that remain do not depend on I* at v = 0."""
    c = _Case(grid_tiny, 0, 0, seed=3)
    i = c.inp
    _, r = c.loss()
    grad = adjoint.gradient(c.g, c.t, c.params, i["rho"][0], i["T"][0], i["Ye"][0], i["D"][0], i["I"][0],
                            i["dt"][0], i["scale"][0], r["D"], gD=c.gD, gYe=c.gYe, geps=c.geps)
    assert np.all(grad["I_star"] == 0.0)
    assert grad["scale"][1] == 0.0   # isoenergetic scattering enters only H


@pytest.mark.parametrize("n,frozen", [(0, 0), (1, 1)])
def test_scale_partials_closed_form_match_differences(grid_tiny, n, frozen):
    """The closed-form derivatives of G = D - Q_D and of H with respect to the four scale factors,
    against fourth-order central differences of the oracle's own map at the converged D (each rate is
    linear in its factor, so the map is smooth in s_k on the scale of s_k itself)."""
    c = _Case(grid_tiny, n, frozen, seed=5)
    i = c.inp
    _, r = c.loss()
    p0 = (i["D"][n], i["I"][n], float(i["Ye"][n]), float(i["T"][n]), np.array(i["scale"][n], dtype=float),
          float(i["dt"][n]))
    state = adjoint._matter(c.g, c.t, c.params, i["rho"][n], p0, r["D"])
    dG, dH = adjoint.scale_partials(c.g, c.t, c.params, i["rho"][n], p0, r["D"], state)
    for k in range(4):
        def f(t):
            sc = p0[4].copy()
            sc[k] += t
            p = p0[:4] + (sc, p0[5])
            st = adjoint._matter(c.g, c.t, c.params, i["rho"][n], p, r["D"])
            G, _, _, _, H = adjoint._outputs(c.g, c.t, c.params, i["rho"][n], p, r["D"], st)
            return G, H
        h = 1e-3 * max(p0[4][k], 1e-3)
        (Gp, Hp), (Gm, Hm), (Gp2, Hp2), (Gm2, Hm2) = f(h), f(-h), f(2 * h), f(-2 * h)
        fdG = (8 * (Gp - Gm) - (Gp2 - Gm2)) / (12 * h)
        fdH = (8 * (Hp - Hm) - (Hp2 - Hm2)) / (12 * h)
        # per species: the difference quotient resolves entries down to ~1e-9 of the species' largest
        refG = np.max(np.abs(dG[k]), axis=1, keepdims=True) + 1e-300
        refH = np.max(np.abs(dH[k]), axis=(1, 2), keepdims=True)[..., 0] + 1e-300
        assert np.all(np.abs(dG[k] - fdG) <= 1e-7 * refG + 1e-9 * np.max(refG)), (k, np.max(np.abs(dG[k] - fdG) / refG))
        assert np.all(np.abs(dH[k] - fdH) <= 1e-7 * refH[..., None] + 1e-9 * np.max(refH)), k
    # Iso does not enter Q_D; EmAb, NES and pair do
    assert np.all(dG[1] == 0.0) and np.any(dG[0] != 0.0) and np.any(dG[2] != 0.0) and np.any(dG[3] != 0.0)
