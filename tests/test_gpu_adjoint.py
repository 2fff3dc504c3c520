"""GPU collision_adjoint: parity with the oracle's IFT gradient, finite
differences of GPU forward solves, the autograd Function, and edge cases.

Parity with the oracle: collision_adjoint takes the converged moments as an
input, so it is given the oracle's own converged D (and T) for the compared
nodes, and both sides differentiate the same root at the same point.  The
bar is 1e-6 relative for every gradient group (per node, relative to the
group's largest entry, plus 1e-5 per entry on the entries that carry it),
with no allowance for the forward solve: the oracle forms every derivative
by fourth-order central differences, the GPU forms dQ/dD analytically and
dQ/dy by second-order differences with 1e-6 steps, so both sit ~1e-9 from
the exact gradient.
"""

import numpy as np
import pytest
import torch

from paper_2601_00976_gb300 import nmc
from paper_2601_00976_gb300.autograd import CollisionSolve
from oracle import eos as oeos, adjoint as oadjoint
from gpu_helpers import make_case, to_device
import oracle_pool

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_inner=1e-13, tol_outer=1e-13, max_inner=2000, max_outer=100)
ORACLE_TIGHT = dict(tol_inner=1e-13, tol_outer=1e-13, max_inner=2000, max_outer=100)
GRAD_TOL = 1e-6
OK_STATUS = (0, nmc.TABLE_CLAMP)


def _forward(ctx, t, **params):
    p = nmc.default_params(**params)
    return p, ctx.collision_solve(p, t["rho"], t["T"], t["Ye"], t["D"], t["I"], t["dt"], t["scale"])


def _adjoint(ctx, p, t, fw, ct):
    d = {k: torch.tensor(np.ascontiguousarray(v), dtype=torch.float64, device=t["rho"].device)
         for k, v in ct.items()}
    g = ctx.collision_adjoint(p, t["rho"], t["T"], t["Ye"], t["D"], t["I"], t["dt"], t["scale"], fw["J"],
                              fw["T"], gJ=d["gD"], gH=d["gH"], gYe=d["gYe"], geps=d["geps"], gT=d["gT"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in g.items()}


def _at_oracle_root(t, nodes, res):
    """The nodes' inputs, with J_out and T_out set to the oracle's converged D and T (res: oracle
    (solve, gradient) pairs), so that the GPU adjoint differentiates at the oracle's point."""
    idx = torch.tensor(nodes, device=t["rho"].device)
    sub = {k: v[idx].contiguous() for k, v in t.items()}
    fw = dict(J=torch.tensor(np.stack([r["D"] for r, _ in res]), dtype=torch.float64, device=t["rho"].device),
              T=torch.tensor([r["T"] for r, _ in res], dtype=torch.float64, device=t["rho"].device))
    return sub, fw


def _assert_group(a, b, what, n):
    """a (GPU) against b (oracle) for one gradient group of node n."""
    a, b = (np.asarray(x, dtype=float) for x in (a, b))
    ref = np.max(np.abs(b))
    err = np.abs(a - b)
    assert np.all(err <= GRAD_TOL * ref + 1e-300), (what, n, np.max(err) / max(ref, 1e-300))
    big = np.abs(b) >= 1e-3 * ref
    assert np.all(err[big] <= 1e-5 * np.abs(b[big])), (what, n)


def _compare(gg, i, r_or, g_or, n=None):
    """GPU gradients of row i against the oracle's gradient of node n (default i)."""
    n = i if n is None else n
    assert int(gg["status"][i]) in OK_STATUS, (n, gg["status"][i])
    _assert_group(gg["J"][i], g_or["D_star"], "D*", n)
    _assert_group(gg["H"][i], g_or["I_star"], "I*", n)
    _assert_group(gg["scale"][i], g_or["scale"], "scale", n)
    sT = r_or["T"] / r_or["Ye"]
    _assert_group([gg["Ye"][i], gg["T"][i] * sT], [g_or["Ye"], g_or["T"] * sT], "Ye,T", n)
    assert abs(gg["T"][i] - g_or["T"]) <= 1e-5 * abs(g_or["T"])


def _oracle_parity(ctx, p, t, ct, nodes, res):
    """GPU adjoint at the oracle's converged point of each node, against the oracle's gradient."""
    sub, fw = _at_oracle_root(t, nodes, res)
    gg = _adjoint(ctx, p, sub, fw, {k: v[nodes] for k, v in ct.items()})
    for i, (n, (r, go)) in enumerate(zip(nodes, res)):
        assert r["status"] == 0
        _compare(gg, i, r, go, n)


def _oracle_tasks(case, inp, nodes, ct, params):
    return [dict(case=case, x=oracle_pool.node_slice(inp, n), params=params, cot=oracle_pool.node_slice(ct, n))
            for n in nodes]


@pytest.mark.parametrize("frozen", [0, 1])
def test_adjoint_matches_oracle_gradient_small_grid(frozen):
    """2 species, 4 linear elements (8 energies), all processes, 12 profile nodes."""
    case = (4, 20.0, 2, 2, 6)
    edges, g, tables, inp = make_case(4, 20.0, 2, 2, "profile", 12, seed=40 + frozen, table_seed=6)
    ctx = nmc.Context(edges, 2, 2, tables)
    t = to_device(inp)
    p = nmc.default_params(frozen_matter=frozen, **TIGHT)
    ct = oracle_pool.cotangents(np.random.default_rng(5 + frozen), 12, 2, g.ne)
    res = oracle_pool.run(_oracle_tasks(case, inp, range(12), ct, dict(frozen_matter=frozen, **ORACLE_TIGHT)))
    _oracle_parity(ctx, p, t, ct, list(range(12)), res)
    ctx.close()


def test_adjoint_matches_oracle_gradient_four_species_grid_c():
    """The adjoint workload's shape: 4 species, 16 linear elements (32 energies), 6 profile nodes
    spanning the density range, compared with the oracle's gradient node by node."""
    N = 64
    case = (16, 1.875, 2, 4, 0)
    edges, g, tables, inp = make_case(16, 1.875, 2, 4, "profile", N, seed=11, table_seed=0)
    ctx = nmc.Context(edges, 2, 4, tables)
    t = to_device(inp)
    p = nmc.default_params(**TIGHT)
    ct = oracle_pool.cotangents(np.random.default_rng(17), N, 4, g.ne)
    order = np.argsort(inp["rho"])
    nodes = [int(order[i]) for i in np.linspace(0, N - 1, 6).astype(int)]
    res = oracle_pool.run(_oracle_tasks(case, inp, nodes, ct, ORACLE_TIGHT))
    _oracle_parity(ctx, p, t, ct, nodes, res)
    ctx.close()


def _near_table_face(tables, rho, T, Ye, margin=2e-3):
    """True where the state sits within `margin` cell widths of a face of a table cell (the
    tables are piecewise linear, so a difference quotient across a face is no derivative)."""
    near = np.zeros(len(rho), dtype=bool)
    eta = np.array([oeos.chemical_potentials(r, tt, y, 2)[1] for r, tt, y in zip(rho, T, Ye)])
    for v, ax in ((np.log10(T), tables["lT"]), (Ye, tables["ye"]), (np.log10(T), tables["klT"]),
                  (eta, tables["keta"]), (np.log10(rho), tables["lrho"])):
        x = (v - ax[0]) / (ax[1] - ax[0]) * (ax[2] - 1)
        near |= np.abs(x - np.round(x)) < margin
    return near


def test_adjoint_matches_finite_differences_of_gpu_solves():
    """256 profile nodes of the adjoint workload's shape: <grad, v> against a fourth-order central
    difference of L along v, for v in D*, I*, Ye*, T* and each scale factor; L sums every output.

    Steps: 1e-5 relative in Ye* and T*, 1e-5 of each entry's natural scale in D*, 1e-3 in I* (the
    outputs are linear in it) and in the scale factors (the solve is a smooth function of them on
    the scale of s itself).  Bar: |fd - ad| <= 1e-6 * S + F, with S the sum of |terms| of <grad, v>
    and F = 1e-11 |L|_1 / h, the rounding of forward solves converged to 1e-13 (a difference
    quotient cannot resolve less).  Nodes within 2e-3 cell widths of a table face (the tables are
    piecewise linear there) or with a flagged status are left out and counted.  A forward solve's
    error grows with cond(dG/dD) along the lepton-number mode of optically thick nodes, so a
    difference quotient there can miss the bar without the gradient being wrong: every node over
    the bar is re-checked against the oracle's gradient at the oracle's converged point, at the
    strict 1e-6 bar; at most 10% of the nodes may need it."""
    N = 256
    edges, g, tables, inp = make_case(16, 1.875, 2, 4, "profile", N, seed=23, table_seed=0)
    ctx = nmc.Context(edges, 2, 4, tables)
    t = to_device(inp)
    p, fw = _forward(ctx, t, **TIGHT)
    ct = oracle_pool.cotangents(np.random.default_rng(29), N, 4, g.ne)
    gg = _adjoint(ctx, p, t, fw, ct)
    rng = np.random.default_rng(31)
    eps_star = np.array([oeos.specific_energy(r, tt, y) for r, tt, y in zip(inp["rho"], inp["T"], inp["Ye"])])
    sD = np.stack([oadjoint.natural_scale(g, p, inp["rho"][n], eps_star[n], inp["Ye"][n], 4) for n in range(N)])
    vD = rng.normal(size=inp["D"].shape) * sD
    vI = rng.normal(size=inp["I"].shape) * np.max(np.abs(inp["I"]), axis=(1, 2, 3))[:, None, None, None]
    dirs = [("D", "D", vD, 1e-5, np.sum(gg["J"] * vD, axis=(1, 2)), np.sum(np.abs(gg["J"] * vD), axis=(1, 2))),
            ("I", "I", vI, 1e-3, np.sum(gg["H"] * vI, axis=(1, 2, 3)),
             np.sum(np.abs(gg["H"] * vI), axis=(1, 2, 3))),
            ("Ye", "Ye", inp["Ye"], 1e-5, gg["Ye"] * inp["Ye"], np.abs(gg["Ye"] * inp["Ye"])),
            ("T", "T", inp["T"], 1e-5, gg["T"] * inp["T"], np.abs(gg["T"] * inp["T"]))]
    for k in range(4):
        v = np.zeros_like(inp["scale"])
        v[:, k] = np.maximum(inp["scale"][:, k], 1e-3)
        dirs.append((f"s{k}", "scale", v, 1e-3, gg["scale"][:, k] * v[:, k], np.abs(gg["scale"][:, k] * v[:, k])))
    near = _near_table_face(tables, inp["rho"], fw["T"].cpu().numpy(), fw["Ye"].cpu().numpy())

    def loss(out):
        o = {k: v.cpu().numpy() for k, v in out.items()}
        terms = [np.sum(ct["gD"] * o["J"], axis=(1, 2)), np.sum(ct["gH"] * o["H"], axis=(1, 2, 3)),
                 ct["gYe"] * o["Ye"], ct["geps"] * o["eps"], ct["gT"] * o["T"]]
        return sum(terms), sum(np.abs(x) for x in terms), o["status"]

    _, Lmag, _ = loss(fw)
    report = []
    over = []
    for name, key, v, h, ad, S in dirs:
        Ls, ok = {}, np.isin(gg["status"], OK_STATUS) & ~near
        for m in (-2, -1, 1, 2):
            pert = dict(inp)
            pert[key] = inp[key] + m * h * v
            _, out = _forward(ctx, to_device(pert), **TIGHT)
            Ls[m], _, st = loss(out)
            ok &= np.isin(st, OK_STATUS)
        fd = (8 * (Ls[1] - Ls[-1]) - (Ls[2] - Ls[-2])) / (12 * h)
        F = 1e-11 * Lmag / h
        err = np.abs(fd - ad)
        bad = ok & (err > GRAD_TOL * S + F)
        rel = err / np.maximum(S, 1e-300)
        report.append(f"{name}: checked {ok.sum()} max rel {np.max(rel[ok]):.2e} "
                      f"median rel {np.median(rel[ok]):.2e} floor-bound {np.sum(ok & (GRAD_TOL * S < F))} "
                      f"over {bad.sum()}")
        assert ok.sum() >= 0.9 * N, (name, ok.sum())
        over += [(name, int(i), err[i], GRAD_TOL * S[i] + F[i], h) for i in np.nonzero(bad)[0]]
    nodes = sorted({o[1] for o in over})
    report.append(f"left out: {int(np.count_nonzero(near))} near a table face; "
                  f"re-checked against the oracle's gradient: {len(nodes)}")
    print("\n".join(report))
    assert len(nodes) <= 0.1 * N, (len(nodes), report)
    if nodes:
        for name, i, e, bar, h in over:
            print(f"{name} node {i}: rho {inp['rho'][i]:.3g} err {e:.3g} bar {bar:.3g}")
        res = oracle_pool.run(_oracle_tasks((16, 1.875, 2, 4, 0), inp, nodes, ct, ORACLE_TIGHT))
        _oracle_parity(ctx, p, t, ct, nodes, res)
    ctx.close()


def test_autograd_function_matches_adjoint_and_flows_to_inputs():
    N = 8
    edges, g, tables, inp = make_case(4, 20.0, 2, 2, "profile", N, seed=3, table_seed=6)
    ctx = nmc.Context(edges, 2, 2, tables)
    t = to_device(inp)
    p = nmc.default_params(**TIGHT)
    leaves = {k: t[k].clone().requires_grad_(True) for k in ("T", "Ye", "D", "I", "scale")}
    J, H, Ye, eps, T, n_outer, n_inner, status = CollisionSolve.apply(
        ctx, p, t["rho"], leaves["T"], leaves["Ye"], leaves["D"], leaves["I"], t["dt"], leaves["scale"])
    assert not status.requires_grad and not n_inner.requires_grad
    ct = oracle_pool.cotangents(np.random.default_rng(2), N, 2, g.ne)
    d = {k: torch.tensor(v, dtype=torch.float64, device=J.device) for k, v in ct.items()}
    L = (d["gD"] * J).sum() + (d["gH"] * H).sum() + (d["gYe"] * Ye).sum() + (d["geps"] * eps).sum() \
        + (d["gT"] * T).sum()
    L.backward()
    fw = dict(J=J.detach(), T=T.detach())
    gg = _adjoint(ctx, p, t, fw, ct)
    for k_leaf, k_adj in (("T", "T"), ("Ye", "Ye"), ("D", "J"), ("I", "H"), ("scale", "scale")):
        assert np.array_equal(leaves[k_leaf].grad.cpu().numpy(), gg[k_adj]), k_leaf
    # an output left out of the loss contributes nothing (its cotangent is passed as NULL)
    for v in leaves.values():
        v.grad = None
    J, H, Ye, eps, T, *_ = CollisionSolve.apply(
        ctx, p, t["rho"], leaves["T"], leaves["Ye"], leaves["D"], leaves["I"], t["dt"], leaves["scale"])
    (d["gYe"] * Ye).sum().backward()
    ct0 = dict(ct, gD=np.zeros_like(ct["gD"]), gH=np.zeros_like(ct["gH"]), geps=np.zeros_like(ct["geps"]),
               gT=np.zeros_like(ct["gT"]))
    g0 = _adjoint(ctx, p, t, dict(J=J.detach(), T=T.detach()), ct0)
    assert np.allclose(leaves["Ye"].grad.cpu().numpy(), g0["Ye"], rtol=1e-14, atol=0)
    assert np.all(leaves["I"].grad.cpu().numpy() == 0.0)
    ctx.close()


def test_adjoint_edge_cases():
    N = 6
    edges, g, tables, inp = make_case(4, 20.0, 2, 2, "profile", N, seed=9, table_seed=6)
    ctx = nmc.Context(edges, 2, 2, tables)
    bad = {k: v.copy() for k, v in inp.items()}
    bad["Ye"][2] = 1.5   # outside (0, 1): the node is skipped by both calls
    t = to_device(bad)
    p, fw = _forward(ctx, t, **TIGHT)
    ct = oracle_pool.cotangents(np.random.default_rng(4), N, 2, g.ne)
    gg = _adjoint(ctx, p, t, fw, ct)
    assert gg["status"][2] & nmc.BAD_INPUT
    assert np.all(gg["J"][2] == 0) and gg["Ye"][2] == 0 and gg["T"][2] == 0 and np.all(gg["H"][2] == 0)
    good = [n for n in range(N) if n != 2]
    t_good = to_device({k: v[good] for k, v in inp.items()})
    p, fw_good = _forward(ctx, t_good, **TIGHT)
    g_good = _adjoint(ctx, p, t_good, fw_good, {k: v[good] for k, v in ct.items()})
    for i, n in enumerate(good):   # a bad neighbour does not change the other nodes' gradients
        assert np.array_equal(gg["J"][n], g_good["J"][i]) and gg["Ye"][n] == g_good["Ye"][i]
    # n = 0 is a no-op; a first-moment cotangent without I* is an argument error
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    e3 = torch.empty((0, 2, g.ne), dtype=torch.float64, device="cuda")
    out = ctx.collision_adjoint(p, e, e, e, e3, None, e, None, e3)
    assert out["J"].shape == (0, 2, g.ne)
    with pytest.raises(nmc.NmcError):
        ctx.collision_adjoint(p, t_good["rho"], t_good["T"], t_good["Ye"], t_good["D"], None, t_good["dt"],
                              None, fw_good["J"], gH=torch.ones_like(t_good["I"]))
    ctx.close()


def test_adjoint_full_size_sampled_against_oracle():
    """2^18 nodes of the adjoint workload (4 species, 16 x 2 energies, profile) at the benchmark's
    tolerance: every node converged, every gradient finite with a clean status, and 4 sampled nodes
    against the oracle's gradient at the oracle's converged point."""
    N = 1 << 18
    case = (16, 1.875, 2, 4, 0)
    edges, g, tables, inp = make_case(16, 1.875, 2, 4, "profile", N, seed=5, table_seed=0)
    ctx = nmc.Context(edges, 2, 4, tables)
    t = to_device(inp)
    p, fw = _forward(ctx, t, tol_inner=1e-10, tol_outer=1e-10)
    ct = oracle_pool.cotangents(np.random.default_rng(8), N, 4, g.ne)
    gg = _adjoint(ctx, p, t, fw, ct)
    st_fw = fw["status"].cpu().numpy()
    assert np.count_nonzero(st_fw) == 0, np.unique(st_fw, return_counts=True)
    assert np.count_nonzero(gg["status"]) == 0, np.unique(gg["status"], return_counts=True)
    for k in ("J", "H", "Ye", "T", "scale"):
        assert np.all(np.isfinite(gg[k])), k
    rng = np.random.default_rng(12)
    nodes = [int(n) for n in rng.choice(N, size=4, replace=False)]
    res = oracle_pool.run(_oracle_tasks(case, inp, nodes, ct, ORACLE_TIGHT))
    _oracle_parity(ctx, p, t, ct, nodes, res)
    ctx.close()
