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


# Per-bin comparison floor, as a fraction of the species' largest |D_ref|.  Algorithm 2 stops on
# W2-weighted norms of the whole spectrum, so a bin many orders of magnitude below its species' peak
# is not held to the solve's tolerance by either side, and the exchange sums that set it carry
# rounding relative to their largest terms; below the floor a bin is compared in absolute terms,
# tol * floor * max_q |D_ref|.  Bins within four orders of magnitude of the peak keep their full
# relative bar.
BIN_FLOOR_FP64 = 1e-4
BIN_FLOOR_MIXED = 1e-4


def bin_errors(D, I, ref_D, ref_I, floor):
    """Element-wise relative errors of D (..., ns, ne) and I (..., ns, ne, 3): |x - x_ref| over
    max(|x_ref|, floor * max_q |D_ref|) per species (I's components share their bin's D scale floor)."""
    D, I, ref_D, ref_I = (np.asarray(x, dtype=np.float64) for x in (D, I, ref_D, ref_I))
    fl = floor * np.max(np.abs(ref_D), axis=-1, keepdims=True)
    eD = np.abs(D - ref_D) / np.maximum(np.maximum(np.abs(ref_D), fl), 1e-300)
    eI = np.abs(I - ref_I) / np.maximum(np.maximum(np.abs(ref_I), fl[..., None]), 1e-300)
    return eD, eI


def assert_bins(D, I, ref_D, ref_I, tol, floor, what=""):
    """Every bin of D and every component of I within tol (bin_errors)."""
    eD, eI = bin_errors(D, I, ref_D, ref_I, floor)
    iD = np.unravel_index(np.argmax(eD), eD.shape)
    iI = np.unravel_index(np.argmax(eI), eI.shape)
    assert eD[iD] <= tol, (what, "D", iD, float(eD[iD]), float(np.asarray(ref_D)[iD]))
    assert eI[iI] <= tol, (what, "I", iI, float(eI[iI]), float(np.asarray(ref_I)[iI]))


def bin_errors_t(D, I, ref_D, ref_I, floor):
    """bin_errors on torch tensors (full-size batches stay on the device); returns the largest
    D and I errors per species over the batch."""
    import torch
    fl = floor * ref_D.abs().amax(dim=-1, keepdim=True)
    eD = (D - ref_D).abs() / torch.clamp(torch.maximum(ref_D.abs(), fl), min=1e-300)
    eI = (I - ref_I).abs() / torch.clamp(torch.maximum(ref_I.abs(), fl[..., None]), min=1e-300)
    return eD.amax(dim=(0, 2)), eI.amax(dim=(0, 2, 3))


def compare_node(out, n, r, W2, tol, floor=BIN_FLOOR_FP64):
    """Assert GPU node n matches oracle result r within relative tolerance tol: D and I per species in
    the W2 norm and bin by bin (bin_errors), Ye, eps and T pointwise, status bits exactly."""
    eD, eI = wnorm_errors(out["J"][n], out["H"][n], r["D"], r["I"], W2)
    assert np.all(eD <= tol), (n, eD)
    assert np.all(eI <= tol), (n, eI)
    assert_bins(out["J"][n], out["H"][n], r["D"], r["I"], tol, floor, what=n)
    for key, rk in (("Ye", "Ye"), ("eps", "eps"), ("T", "T")):
        assert abs(out[key][n] - r[rk]) <= tol * abs(r[rk]), (n, key, out[key][n], r[rk])
    assert int(out["status"][n]) == int(r["status"]), (n, out["status"][n], r["status"])
