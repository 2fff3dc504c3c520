"""Plain per-iteration mode (NMC_MODE_PLAIN) against the fused persistent kernel
and the oracle.

The two modes run the same algorithm with the same FP64 arithmetic and differ
only in how the work is scheduled (launch per phase and iteration over
compacted work lists, state in global memory, the batch in chunks), so their
results agree to rounding order: 1e-12 relative here, and the iteration
counts and status bits must match exactly.
"""

import numpy as np
import pytest

from oracle import solver as osolver
from paper_2601_00976_gb300 import nmc
from gpu_helpers import make_case, gpu_solve, compare_node, wnorm_errors, bin_errors, BIN_FLOOR_FP64

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_inner=1e-13, tol_outer=1e-13, max_inner=2000, max_outer=100)


def _agree(a, b, W2, tol):
    eD, eI = wnorm_errors(a["J"], a["H"], b["J"], b["H"], W2)
    assert eD.max() <= tol and eI.max() <= tol, (eD.max(), eI.max())
    # bin by bin at the FP64 parity bar (the two modes' rounding orders differ, and small bins carry
    # that rounding relative to the large terms of the exchange sums)
    bD, bI = bin_errors(a["J"], a["H"], b["J"], b["H"], BIN_FLOOR_FP64)
    assert bD.max() <= 1e-10 and bI.max() <= 1e-10, (bD.max(), bI.max())
    for k in ("Ye", "eps", "T"):
        assert np.max(np.abs(a[k] - b[k]) / np.abs(b[k])) <= tol, k


@pytest.mark.parametrize("kind,N,m", [("profile", 512, 3), ("core_tail", 384, 3), ("profile", 256, 5)])
def test_plain_matches_fused(kind, N, m):
    edges, g, tables, inp = make_case(16, 1.875, 2, 4, kind, N, seed=31)
    ctx = nmc.Context(edges, 2, 4, tables)
    fused = gpu_solve(ctx, inp, m_inner=m)
    plain = gpu_solve(ctx, inp, m_inner=m, mode=nmc.MODE_PLAIN)
    assert np.array_equal(fused["status"], plain["status"])
    assert np.array_equal(fused["n_inner"], plain["n_inner"])
    assert np.array_equal(fused["n_outer"], plain["n_outer"])
    _agree(plain, fused, g.W2, 1e-12)
    ctx.close()


def test_plain_against_oracle_and_chunks():
    """More nodes than one chunk (the chunk is set small), bad-input and frozen-matter nodes."""
    N = 40
    edges, g, tables, inp = make_case(8, 4.0, 2, 2, "profile", N, seed=32)
    inp["Ye"][7] = 1.5   # invalid: outputs = inputs, BAD_INPUT
    ctx = nmc.Context(edges, 2, 2, tables)
    ctx.set_plain_chunk(16)
    out = gpu_solve(ctx, inp, mode=nmc.MODE_PLAIN, **TIGHT)
    good = [n for n in range(N) if n != 7]
    ref = osolver.solve(g, tables, osolver.Params(**TIGHT), inp, nodes=good)
    assert out["status"][7] == nmc.BAD_INPUT and np.array_equal(out["J"][7], inp["D"][7])
    for n, r in zip(good, ref):
        compare_node(out, n, r, g.W2, 1e-10)
    frozen = gpu_solve(ctx, inp, mode=nmc.MODE_PLAIN, frozen_matter=1)
    fused = gpu_solve(ctx, inp, frozen_matter=1)
    assert np.array_equal(frozen["status"], fused["status"])
    _agree({k: v[np.arange(N) != 7] for k, v in frozen.items()},
           {k: v[np.arange(N) != 7] for k, v in fused.items()}, g.W2, 1e-12)
    ctx.close()


def test_plain_mixed_is_rejected():
    edges, g, tables, inp = make_case(8, 4.0, 2, 2, "profile", 4, seed=33)
    ctx = nmc.Context(edges, 2, 2, tables)
    with pytest.raises(nmc.NmcError):
        gpu_solve(ctx, inp, mode=nmc.MODE_PLAIN, precision=nmc.MIXED)
    ctx.close()
