"""Helpers shared by the GPU parity tests (no solver arithmetic here)."""

import numpy as np
import torch

from paper_2601_00976_gb300 import nmc, synthetic
from oracle import grid as ogrid


def make_case(n_elem, de1, nq, ns, kind, N, seed=0, table_seed=0):
    edges, _ = ogrid.geometric_edges(n_elem, de1)
    g = ogrid.EnergyGrid(edges, nq)
    tables = synthetic.make_tables(g.eps, ns, seed=table_seed)
    inp = synthetic.make_inputs(kind, N, g.eps, ns, seed=seed)
    return edges, g, tables, inp


def to_device(inp):
    dev = torch.device("cuda", 0)
    return {k: torch.tensor(np.ascontiguousarray(v), dtype=torch.float64, device=dev) for k, v in inp.items()}


def gpu_solve(ctx, inp, **params):
    t = to_device(inp)
    p = nmc.default_params(**params)
    out = ctx.collision_solve(p, t["rho"], t["T"], t["Ye"], t["D"], t["I"], t["dt"], t["scale"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def wnorm_errors(D, I, ref_D, ref_I, W2, floor=1e-300):
    """Per-species W2-norm errors of D and I relative to ||D_ref||_W2."""
    ref = np.sqrt(np.sum(W2 * ref_D ** 2, axis=-1))
    ref = np.maximum(ref, floor)
    eD = np.sqrt(np.sum(W2 * (D - ref_D) ** 2, axis=-1)) / ref
    eI = np.sqrt(np.sum(W2[:, None] * (I - ref_I) ** 2, axis=(-2, -1))) / ref
    return eD, eI


def compare_node(out, n, r, W2, tol):
    """Assert GPU node n matches oracle result r within relative tolerance tol."""
    eD, eI = wnorm_errors(out["J"][n], out["H"][n], r["D"], r["I"], W2)
    assert np.all(eD <= tol), (n, eD)
    assert np.all(eI <= tol), (n, eI)
    for key, rk in (("Ye", "Ye"), ("eps", "eps"), ("T", "T")):
        assert abs(out[key][n] - r[rk]) <= tol * abs(r[rk]), (n, key, out[key][n], r[rk])
    assert int(out["status"][n]) == int(r["status"]), (n, out["status"][n], r["status"])
