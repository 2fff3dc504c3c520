"""collision_solve_noalloc against collision_solve, through the C ABI.

The no-allocation entry point serves callers that cannot allocate device
memory when they solve (their memory is owned by another allocator after
set-up).  It must give the same results as collision_solve; it is called twice
in a row because its static work counter keeps the previous call's value and
must be cleared by each call, and the second call must leave the device's free
memory unchanged.  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_2601_00976_gb300 import nmc
from gpu_helpers import make_case, to_device

pytestmark = pytest.mark.gpu


def _outputs(n, ns, ne):
    f64 = dict(dtype=torch.float64, device="cuda")
    i32 = dict(dtype=torch.int32, device="cuda")
    return dict(J=torch.empty((n, ns, ne), **f64), H=torch.empty((n, ns, ne, 3), **f64),
                Ye=torch.empty(n, **f64), eps=torch.empty(n, **f64), T=torch.empty(n, **f64),
                n_outer=torch.empty(n, **i32), n_inner=torch.empty(n, **i32), status=torch.empty(n, **i32))


def _call(lib_fn, ctx, prm, t, out):
    p = lambda x: ctypes.c_void_p(x.data_ptr())  # noqa: E731
    rc = lib_fn(ctx._h, ctypes.byref(prm), t["rho"].shape[0], p(t["rho"]), p(t["T"]), p(t["Ye"]), p(t["D"]),
                p(t["I"]), p(t["dt"]), p(t["scale"]), p(out["J"]), p(out["H"]), p(out["Ye"]), p(out["eps"]),
                p(out["T"]), p(out["n_outer"]), p(out["n_inner"]), p(out["status"]),
                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == nmc.NMC_OK, ctx.last_error()


@pytest.mark.parametrize("precision", [nmc.FP64, nmc.MIXED])
def test_noalloc_matches_collision_solve_twice(precision):
    N = 3000
    edges, g, tables, inp = make_case(16, 1.875, 2, 4, "profile", N, seed=31)
    ctx = nmc.Context(edges, 2, 4, tables)
    L = nmc.load_library()
    t = to_device(inp)
    kw = dict(precision=precision)
    if precision == nmc.MIXED:
        kw.update(tol_inner=1e-6, tol_outer=1e-7)
    prm = nmc.default_params(**kw)
    ref = _outputs(N, 4, ctx.ne)
    _call(L.collision_solve, ctx, prm, t, ref)
    for call in range(2):
        out = _outputs(N, 4, ctx.ne)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        _call(L.collision_solve_noalloc, ctx, prm, t, out)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if call == 1:   # after a warm-up call, a call takes no device memory (cudaMemGetInfo)
            assert free1 == free0, (free0, free1)
        for k in ("J", "H", "Ye", "eps", "T"):
            a, b = out[k].cpu().numpy(), ref[k].cpu().numpy()
            assert np.allclose(a, b, rtol=1e-10, atol=0.0), k
        for k in ("n_outer", "n_inner", "status"):
            assert torch.equal(out[k], ref[k]), k
    ctx.close()


def test_noalloc_rejects_oversized_and_bad_arguments():
    edges, g, tables, inp = make_case(16, 1.875, 2, 4, "profile", 4, seed=32)
    ctx = nmc.Context(edges, 2, 4, tables)
    L = nmc.load_library()
    prm = nmc.default_params()
    rc = L.collision_solve_noalloc(ctx._h, ctypes.byref(prm), (1 << 30) + 1, *([None] * 16))
    assert rc == nmc.NMC_EUNSUPPORTED and "2^30" in ctx.last_error()
    rc = L.collision_solve_noalloc(ctx._h, ctypes.byref(prm), 4, *([None] * 16))
    assert rc == nmc.NMC_EINVAL
    plain = nmc.default_params(mode=nmc.MODE_PLAIN)
    rc = L.collision_solve_noalloc(ctx._h, ctypes.byref(plain), 4, *([None] * 16))
    assert rc == nmc.NMC_EUNSUPPORTED
    ctx.close()
