"""Python binding of libnmc (ctypes).  Argument marshalling only: every step of
the collision solve runs in the library's CUDA kernels.

The names follow the C ABI in include/nmc.h: ``Context.collision_solve``,
``Context.collision_adjoint``, ``Context.opacity_interp``; ``Context`` wraps
``nmc_create``/``nmc_destroy``.  ``CollisionSolve`` (in
``paper_2601_00976_gb300.autograd``) is the torch.autograd.Function whose
backward calls ``collision_adjoint``.
PyTorch provides device memory and streams.  There is no CPU fallback: if the
shared library is missing or no CUDA device is present the calls raise.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# NMC_DEBUG=1 in the environment selects the bounds-checked build, NMC_TRACE=1 the stage-counter build
# (built by `python -m paper_2601_00976_gb300._build --debug` / `--trace`)
LIB_PATH = os.path.join(_HERE, "_lib_debug" if os.environ.get("NMC_DEBUG") == "1" else
                        ("_lib_trace" if os.environ.get("NMC_TRACE") == "1" else "_lib"), "libnmc.so")

NMC_OK, NMC_EINVAL, NMC_ECUDA, NMC_ENOMEM, NMC_EUNSUPPORTED = 0, 1, 2, 3, 4
NOT_CONVERGED_INNER, NOT_CONVERGED_OUTER, NONFINITE, EOS_FAIL, TABLE_CLAMP, BAD_INPUT = 1, 2, 4, 8, 16, 32
PROC_EMAB, PROC_ISO, PROC_NES, PROC_PAIR, PROC_ALL = 1, 2, 4, 8, 15
FP64, MIXED = 0, 1
MODE_FUSED, MODE_PLAIN = 0, 1

_c_double_p = ctypes.POINTER(ctypes.c_double)


class Grid(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int32), ("n_q", ctypes.c_int32), ("n_species", ctypes.c_int32),
                ("edges", _c_double_p)]


class Tables(ctypes.Structure):
    _fields_ = [("n_rho", ctypes.c_int32), ("n_t", ctypes.c_int32), ("n_ye", ctypes.c_int32),
                ("lrho_min", ctypes.c_double), ("lrho_max", ctypes.c_double),
                ("lt_min", ctypes.c_double), ("lt_max", ctypes.c_double),
                ("ye_min", ctypes.c_double), ("ye_max", ctypes.c_double),
                ("emab", _c_double_p), ("iso", _c_double_p),
                ("n_kt", ctypes.c_int32), ("n_eta", ctypes.c_int32),
                ("klt_min", ctypes.c_double), ("klt_max", ctypes.c_double),
                ("eta_min", ctypes.c_double), ("eta_max", ctypes.c_double),
                ("nes", _c_double_p), ("pair", _c_double_p),
                ("nes1", _c_double_p), ("pair1", _c_double_p)]


class Params(ctypes.Structure):
    _fields_ = [("tol_inner", ctypes.c_double), ("tol_outer", ctypes.c_double),
                ("m_inner", ctypes.c_int32), ("m_outer", ctypes.c_int32),
                ("max_inner", ctypes.c_int32), ("max_outer", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("proc_mask", ctypes.c_int32), ("frozen_matter", ctypes.c_int32),
                ("final_q", ctypes.c_int32), ("semi_implicit", ctypes.c_int32),
                ("d_min", ctypes.c_double), ("d_max", ctypes.c_double),
                ("norm_floor", ctypes.c_double)]


EXPORTS = ("nmc_default_params", "nmc_create", "nmc_destroy", "nmc_last_error", "nmc_energy_nodes",
           "nmc_grid_nodes", "nmc_geometric_edges", "collision_solve", "collision_solve_noalloc", "collision_solve_v", "conserved_to_primitive",
           "opacity_interp", "collision_adjoint", "nmc_set_plain_chunk", "nmc_autotune", "nmc_fma_probe", "collision_solve_host", "opacity_interp_mixed", "nmc_debug_word",
           "nmc_smem_probe", "nmc_trace_read")

_lib = None


def load_library(path=LIB_PATH):
    """Load libnmc.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.nmc_default_params.argtypes = [ctypes.POINTER(Params)]
    lib.nmc_default_params.restype = None
    lib.nmc_create.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Tables), ctypes.POINTER(vp)]
    lib.nmc_create.restype = ctypes.c_int
    lib.nmc_destroy.argtypes = [vp]
    lib.nmc_destroy.restype = None
    lib.nmc_last_error.argtypes = [vp]
    lib.nmc_last_error.restype = ctypes.c_char_p
    lib.nmc_energy_nodes.argtypes = [vp, _c_double_p, _c_double_p, _c_double_p, ctypes.POINTER(ctypes.c_int32)]
    lib.nmc_energy_nodes.restype = ctypes.c_int
    lib.nmc_grid_nodes.argtypes = [ctypes.POINTER(Grid), _c_double_p, _c_double_p, _c_double_p]
    lib.nmc_grid_nodes.restype = ctypes.c_int
    lib.nmc_geometric_edges.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, _c_double_p, _c_double_p]
    lib.nmc_geometric_edges.restype = ctypes.c_int
    lib.collision_solve.argtypes = [vp, ctypes.POINTER(Params), ctypes.c_int64] + [vp] * 16
    lib.collision_solve.restype = ctypes.c_int
    lib.collision_solve_noalloc.argtypes = [vp, ctypes.POINTER(Params), ctypes.c_int64] + [vp] * 16
    lib.collision_solve_noalloc.restype = ctypes.c_int
    lib.collision_solve_host.argtypes = [vp, ctypes.POINTER(Params), ctypes.c_int64] + [vp] * 15 + [ctypes.c_int64, vp]
    lib.collision_solve_host.restype = ctypes.c_int
    lib.collision_solve_v.argtypes = ([vp, ctypes.POINTER(Params), ctypes.c_int64] + [vp] * 8 +
                                      [ctypes.c_int32, ctypes.c_double] + [vp] * 10)
    lib.collision_solve_v.restype = ctypes.c_int
    lib.conserved_to_primitive.argtypes = ([vp, ctypes.c_int64, vp, vp, vp, ctypes.c_double, ctypes.c_int32,
                                            ctypes.c_int32] + [vp] * 5)
    lib.conserved_to_primitive.restype = ctypes.c_int
    lib.opacity_interp.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64] + [vp] * 6
    lib.opacity_interp.restype = ctypes.c_int
    lib.opacity_interp_mixed.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64] + [vp] * 6
    lib.opacity_interp_mixed.restype = ctypes.c_int
    lib.collision_adjoint.argtypes = [vp, ctypes.POINTER(Params), ctypes.c_int64] + [vp] * 20
    lib.collision_adjoint.restype = ctypes.c_int
    lib.nmc_autotune.argtypes = [vp, ctypes.POINTER(Params), ctypes.c_int64] + [vp] * 18
    lib.nmc_autotune.restype = ctypes.c_int
    lib.nmc_set_plain_chunk.argtypes = [vp, ctypes.c_int64]
    lib.nmc_set_plain_chunk.restype = ctypes.c_int
    lib.nmc_fma_probe.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp,
                                  ctypes.POINTER(ctypes.c_double), vp]
    lib.nmc_fma_probe.restype = ctypes.c_int
    lib.nmc_smem_probe.argtypes = [ctypes.c_int32, ctypes.c_int32, vp, ctypes.POINTER(ctypes.c_double), vp]
    lib.nmc_smem_probe.restype = ctypes.c_int
    lib.nmc_debug_word.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int32]
    lib.nmc_debug_word.restype = ctypes.c_int
    lib.nmc_trace_read.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int32]
    lib.nmc_trace_read.restype = ctypes.c_int
    _lib = lib
    return lib


def default_params(**overrides):
    p = Params()
    load_library().nmc_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def geometric_edges(n_elem, de1, emax=300.0):
    lib = load_library()
    edges = np.zeros(n_elem + 1)
    alpha = ctypes.c_double()
    rc = lib.nmc_geometric_edges(n_elem, de1, emax, edges.ctypes.data_as(_c_double_p), ctypes.byref(alpha))
    if rc != NMC_OK:
        raise ValueError(f"nmc_geometric_edges failed ({rc})")
    return edges, alpha.value


def grid_nodes(edges, n_q):
    """(eps, W2, W3) of the grid with element interfaces `edges` and n_q nodes per element."""
    lib = load_library()
    e = np.ascontiguousarray(edges, dtype=np.float64)
    ne = (len(e) - 1) * n_q
    eps, w2, w3 = np.zeros(ne), np.zeros(ne), np.zeros(ne)
    g = Grid(len(e) - 1, n_q, 2, e.ctypes.data_as(_c_double_p))
    rc = lib.nmc_grid_nodes(ctypes.byref(g), eps.ctypes.data_as(_c_double_p), w2.ctypes.data_as(_c_double_p),
                            w3.ctypes.data_as(_c_double_p))
    if rc != NMC_OK:
        raise ValueError(f"nmc_grid_nodes failed ({rc})")
    return eps, w2, w3


def fma_probe(precision, iters, sink, blocks_per_sm=0, stream=None):
    """Launch the FMA-pipe peak probe on `stream` (torch's current one by default); returns the
    launch's flop count.  sink: a one-element CUDA tensor of the precision's dtype."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    flops = ctypes.c_double()
    rc = load_library().nmc_fma_probe(int(precision), int(blocks_per_sm), int(iters),
                                      ctypes.c_void_p(sink.data_ptr()), ctypes.byref(flops),
                                      ctypes.c_void_p(s.cuda_stream))
    if rc != NMC_OK:
        raise NmcError(f"nmc_fma_probe failed with code {rc}")
    return flops.value


# nmc_smem_probe modes
SMEM_B32_CONSECUTIVE, SMEM_B32_BROADCAST, SMEM_B64_BROADCAST, SMEM_B128_BROADCAST, SMEM_B128_CONSECUTIVE = range(5)


def smem_probe(mode, iters, sink, stream=None):
    """Launch the shared-memory load probe on `stream` (torch's current one by default); returns the
    launch's warp-load count.  sink: a one-element float32 CUDA tensor."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    loads = ctypes.c_double()
    rc = load_library().nmc_smem_probe(int(mode), int(iters), ctypes.c_void_p(sink.data_ptr()), ctypes.byref(loads),
                                       ctypes.c_void_p(s.cuda_stream))
    if rc != NMC_OK:
        raise NmcError(f"nmc_smem_probe failed with code {rc}")
    return loads.value


def _dptr(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class NmcError(RuntimeError):
    pass


class Context:
    """A libnmc context: energy grid + tables resident on the current CUDA device."""

    def __init__(self, edges, n_q, n_species, tables):
        import torch  # noqa: F401  (initialises the CUDA runtime)
        self._lib = load_library()
        self._keep = [_dptr(edges)]
        g = Grid(len(edges) - 1, n_q, n_species, self._keep[0].ctypes.data_as(_c_double_p))
        arrs = {k: _dptr(tables[k]) for k in ("emab", "iso", "nes", "pair", "nes1", "pair1") if k in tables}
        self._keep += list(arrs.values())
        t = Tables()
        t.n_rho, t.n_t, t.n_ye = tables["lrho"][2], tables["lT"][2], tables["ye"][2]
        t.lrho_min, t.lrho_max = tables["lrho"][0], tables["lrho"][1]
        t.lt_min, t.lt_max = tables["lT"][0], tables["lT"][1]
        t.ye_min, t.ye_max = tables["ye"][0], tables["ye"][1]
        t.n_kt, t.n_eta = tables["klT"][2], tables["keta"][2]
        t.klt_min, t.klt_max = tables["klT"][0], tables["klT"][1]
        t.eta_min, t.eta_max = tables["keta"][0], tables["keta"][1]
        for k, v in arrs.items():
            setattr(t, k, v.ctypes.data_as(_c_double_p))
        h = ctypes.c_void_p()
        rc = self._lib.nmc_create(ctypes.byref(g), ctypes.byref(t), ctypes.byref(h))
        self._keep = None
        if rc != NMC_OK:
            raise NmcError(f"nmc_create failed with code {rc}")
        self._h = h
        self.n_species = n_species
        ne = ctypes.c_int32()
        self._lib.nmc_energy_nodes(self._h, None, None, None, ctypes.byref(ne))
        self.ne = ne.value
        self.energies = np.zeros(self.ne)
        self.w2 = np.zeros(self.ne)
        self.w3 = np.zeros(self.ne)
        self._lib.nmc_energy_nodes(self._h, self.energies.ctypes.data_as(_c_double_p),
                                   self.w2.ctypes.data_as(_c_double_p), self.w3.ctypes.data_as(_c_double_p), None)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.nmc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self):
        return self._lib.nmc_last_error(self._h).decode()

    def trace_read(self, clear=False):
        """The fused kernel's 16 stage counters (SM cycles of block time) of the NMC_TRACE build; raises
        NmcError in other builds."""
        c = (ctypes.c_uint64 * 16)()
        self._check(self._lib.nmc_trace_read(self._h, c, 1 if clear else 0), "nmc_trace_read")
        return [int(x) for x in c]

    def debug_word(self, clear=False):
        """The NMC_DEBUG build's bounds-check error word (0: no check failed); raises NmcError on a
        release build."""
        w = ctypes.c_uint32()
        self._check(self._lib.nmc_debug_word(self._h, ctypes.byref(w), 1 if clear else 0), "nmc_debug_word")
        return int(w.value)

    def _check(self, rc, what):
        if rc != NMC_OK:
            raise NmcError(f"{what} failed with code {rc}: {self.last_error()}")

    @staticmethod
    def _stream_handle(stream):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        return ctypes.c_void_p(s.cuda_stream)

    def collision_solve(self, params, rho, T, Ye, J, H, dt, scale=None, out=None, stream=None):
        """Run collision_solve on CUDA float64 tensors; returns a dict of output tensors.

        CPU tensors are accepted too: they are copied to the current device
        (non-blocking when pinned), solved there, and the outputs copied back.
        """
        import torch
        host = not rho.is_cuda
        if host:
            dev = torch.device("cuda", torch.cuda.current_device())
            rho, T, Ye, J, H, dt = (x.to(dev, non_blocking=True) for x in (rho, T, Ye, J, H, dt))
            if scale is not None:
                scale = scale.to(dev, non_blocking=True)
        ins = [rho, T, Ye, J, H, dt] + ([scale] if scale is not None else [])
        for x in ins:
            if x.dtype != torch.float64 or not x.is_contiguous() or not x.is_cuda:
                raise ValueError("inputs must be contiguous CUDA float64 tensors")
        n = rho.shape[0]
        ns, ne = self.n_species, self.ne
        if J.shape != (n, ns, ne) or H.shape != (n, ns, ne, 3):
            raise ValueError(f"J must be {(n, ns, ne)} and H {(n, ns, ne, 3)}")
        if out is None:
            f64 = dict(dtype=torch.float64, device=rho.device)
            out = dict(J=torch.empty_like(J), H=torch.empty_like(H), Ye=torch.empty(n, **f64),
                       eps=torch.empty(n, **f64), T=torch.empty(n, **f64),
                       n_outer=torch.empty(n, dtype=torch.int32, device=rho.device),
                       n_inner=torch.empty(n, dtype=torch.int32, device=rho.device),
                       status=torch.empty(n, dtype=torch.int32, device=rho.device))
        p = lambda x: ctypes.c_void_p(x.data_ptr()) if x is not None else None  # noqa: E731
        rc = self._lib.collision_solve(
            self._h, ctypes.byref(params), n, p(rho), p(T), p(Ye), p(J), p(H), p(dt), p(scale),
            p(out["J"]), p(out["H"]), p(out["Ye"]), p(out["eps"]), p(out["T"]),
            p(out["n_outer"]), p(out["n_inner"]), p(out["status"]), self._stream_handle(stream))
        self._check(rc, "collision_solve")
        if host:
            out = {k: v.to("cpu", non_blocking=False) for k, v in out.items()}
        return out

    def host_outputs(self, n):
        """Page-locked host tensors for the outputs of collision_solve_host on n nodes."""
        import torch
        ns, ne = self.n_species, self.ne
        f64 = dict(dtype=torch.float64, pin_memory=True)
        i32 = dict(dtype=torch.int32, pin_memory=True)
        return dict(J=torch.empty((n, ns, ne), **f64), H=torch.empty((n, ns, ne, 3), **f64),
                    Ye=torch.empty(n, **f64), eps=torch.empty(n, **f64), T=torch.empty(n, **f64),
                    n_outer=torch.empty(n, **i32), n_inner=torch.empty(n, **i32), status=torch.empty(n, **i32))

    def collision_solve_host(self, params, inp, out, chunk=0, stream=None, sync=True):
        """collision_solve_host on CPU tensors: inp holds rho, T, Ye, D (J), I (H), dt and optionally scale
        (contiguous float64, page-locked for overlapped copies); out is a dict like host_outputs(n).
        The copies and the solve are pipelined by the library; with sync the call waits for `stream`."""
        import torch
        x = [inp[k] for k in ("rho", "T", "Ye", "D", "I", "dt")] + [inp.get("scale")]
        for v in x + list(out.values()):
            if v is not None and (v.is_cuda or not v.is_contiguous()):
                raise ValueError("collision_solve_host takes contiguous CPU tensors")
        n = inp["rho"].shape[0]
        ns, ne = self.n_species, self.ne
        if inp["D"].shape != (n, ns, ne) or inp["I"].shape != (n, ns, ne, 3):
            raise ValueError(f"D must be {(n, ns, ne)} and I {(n, ns, ne, 3)}")
        p = lambda v: ctypes.c_void_p(v.data_ptr()) if v is not None else None  # noqa: E731
        s = self._stream_handle(stream)
        rc = self._lib.collision_solve_host(
            self._h, ctypes.byref(params), n, *[p(v) for v in x],
            p(out["J"]), p(out["H"]), p(out["Ye"]), p(out["eps"]), p(out["T"]),
            p(out["n_outer"]), p(out["n_inner"]), p(out["status"]), int(chunk), s)
        self._check(rc, "collision_solve_host")
        if sync:
            (stream if stream is not None else torch.cuda.current_stream()).synchronize()
        return out

    def collision_solve_v(self, params, rho, T, Ye, v, J, H, dt, scale=None, freeze_velocity=False,
                          v_floor=1e-6, out=None, stream=None):
        """Run collision_solve_v (the O(v/c) solve) on CUDA float64 tensors; v has shape (n, 3)
        in units of c.  Returns the outputs of collision_solve plus "v" (n, 3); "eps" is the
        specific internal energy."""
        import torch
        ins = [rho, T, Ye, v, J, H, dt] + ([scale] if scale is not None else [])
        for x in ins:
            if x.dtype != torch.float64 or not x.is_contiguous() or not x.is_cuda:
                raise ValueError("inputs must be contiguous CUDA float64 tensors")
        n = rho.shape[0]
        ns, ne = self.n_species, self.ne
        if J.shape != (n, ns, ne) or H.shape != (n, ns, ne, 3) or v.shape != (n, 3):
            raise ValueError(f"J must be {(n, ns, ne)}, H {(n, ns, ne, 3)} and v {(n, 3)}")
        if out is None:
            f64 = dict(dtype=torch.float64, device=rho.device)
            out = dict(J=torch.empty_like(J), H=torch.empty_like(H), v=torch.empty_like(v),
                       Ye=torch.empty(n, **f64), eps=torch.empty(n, **f64), T=torch.empty(n, **f64),
                       n_outer=torch.empty(n, dtype=torch.int32, device=rho.device),
                       n_inner=torch.empty(n, dtype=torch.int32, device=rho.device),
                       status=torch.empty(n, dtype=torch.int32, device=rho.device))
        p = lambda x: ctypes.c_void_p(x.data_ptr()) if x is not None else None  # noqa: E731
        rc = self._lib.collision_solve_v(
            self._h, ctypes.byref(params), n, p(rho), p(T), p(Ye), p(v), p(J), p(H), p(dt), p(scale),
            1 if freeze_velocity else 0, float(v_floor),
            p(out["J"]), p(out["H"]), p(out["v"]), p(out["Ye"]), p(out["eps"]), p(out["T"]),
            p(out["n_outer"]), p(out["n_inner"]), p(out["status"]), self._stream_handle(stream))
        self._check(rc, "collision_solve_v")
        return out

    def conserved_to_primitive(self, N, G, v, tol=1e-8, memory=3, max_iter=100, out=None, stream=None):
        """Run conserved_to_primitive on CUDA float64 tensors N (n, ns, ne), G (n, ns, ne, 3),
        v (n, 3); returns D, I, iters (per bin) and status (per node)."""
        import torch
        for x in (N, G, v):
            if x.dtype != torch.float64 or not x.is_contiguous() or not x.is_cuda:
                raise ValueError("inputs must be contiguous CUDA float64 tensors")
        n = N.shape[0]
        ns, ne = self.n_species, self.ne
        if N.shape != (n, ns, ne) or G.shape != (n, ns, ne, 3) or v.shape != (n, 3):
            raise ValueError(f"N must be {(n, ns, ne)}, G {(n, ns, ne, 3)} and v {(n, 3)}")
        if out is None:
            out = dict(D=torch.empty_like(N), I=torch.empty_like(G),
                       iters=torch.empty((n, ns, ne), dtype=torch.int32, device=N.device),
                       status=torch.empty(n, dtype=torch.int32, device=N.device))
        p = lambda x: ctypes.c_void_p(x.data_ptr()) if x is not None else None  # noqa: E731
        rc = self._lib.conserved_to_primitive(self._h, n, p(N), p(G), p(v), float(tol), int(memory), int(max_iter),
                                              p(out["D"]), p(out["I"]), p(out["iters"]), p(out["status"]),
                                              self._stream_handle(stream))
        self._check(rc, "conserved_to_primitive")
        return out

    def collision_adjoint(self, params, rho, T, Ye, J, H, dt, scale, J_out, T_out=None,
                          gJ=None, gH=None, gYe=None, geps=None, gT=None, out=None, stream=None):
        """Run collision_adjoint on CUDA float64 tensors.

        Inputs are the forward call's inputs and its converged J_out (T_out
        optional, the EoS starting guess) plus cotangents of the outputs (any
        may be None).  Returns a dict of input cotangents J, H, Ye, T, scale
        and the per-node status.
        """
        import torch
        for x in (rho, T, Ye, J, H, dt, scale, J_out, T_out, gJ, gH, gYe, geps, gT):
            if x is not None and (x.dtype != torch.float64 or not x.is_contiguous() or not x.is_cuda):
                raise ValueError("adjoint arguments must be contiguous CUDA float64 tensors")
        n = rho.shape[0]
        ns, ne = self.n_species, self.ne
        if J.shape != (n, ns, ne) or J_out.shape != (n, ns, ne) or (H is not None and H.shape != (n, ns, ne, 3)):
            raise ValueError(f"J, J_out must be {(n, ns, ne)} and H {(n, ns, ne, 3)}")
        if out is None:
            f64 = dict(dtype=torch.float64, device=rho.device)
            out = dict(J=torch.empty_like(J), H=torch.empty((n, ns, ne, 3), **f64), Ye=torch.empty(n, **f64),
                       T=torch.empty(n, **f64), scale=torch.empty((n, 4), **f64),
                       status=torch.empty(n, dtype=torch.int32, device=rho.device))
        p = lambda x: ctypes.c_void_p(x.data_ptr()) if x is not None else None  # noqa: E731
        rc = self._lib.collision_adjoint(
            self._h, ctypes.byref(params), n, p(rho), p(T), p(Ye), p(J), p(H), p(dt), p(scale),
            p(J_out), p(T_out), p(gJ), p(gH), p(gYe), p(geps), p(gT),
            p(out["J"]), p(out["H"]), p(out["Ye"]), p(out["T"]), p(out["scale"]), p(out["status"]),
            self._stream_handle(stream))
        self._check(rc, "collision_adjoint")
        return out

    def autotune(self, params, rho, T, Ye, J, H, dt, scale=None, stream=None):
        """Time the fused kernel's variants on this batch and keep the fastest for these parameters.

        Returns (blocks_per_sm, grid_percent, milliseconds) of the chosen variant.
        """
        import torch
        n = rho.shape[0]
        f64 = dict(dtype=torch.float64, device=rho.device)
        out = dict(J=torch.empty_like(J), H=torch.empty_like(H), Ye=torch.empty(n, **f64),
                   eps=torch.empty(n, **f64), T=torch.empty(n, **f64),
                   n_outer=torch.empty(n, dtype=torch.int32, device=rho.device),
                   n_inner=torch.empty(n, dtype=torch.int32, device=rho.device),
                   status=torch.empty(n, dtype=torch.int32, device=rho.device))
        chosen = (ctypes.c_int32 * 2)()
        ms = ctypes.c_float()
        p = lambda x: ctypes.c_void_p(x.data_ptr()) if x is not None else None  # noqa: E731
        rc = self._lib.nmc_autotune(
            self._h, ctypes.byref(params), n, p(rho), p(T), p(Ye), p(J), p(H), p(dt), p(scale),
            p(out["J"]), p(out["H"]), p(out["Ye"]), p(out["eps"]), p(out["T"]),
            p(out["n_outer"]), p(out["n_inner"]), p(out["status"]), ctypes.cast(chosen, ctypes.c_void_p),
            ctypes.cast(ctypes.pointer(ms), ctypes.c_void_p), self._stream_handle(stream))
        self._check(rc, "nmc_autotune")
        return int(chosen[0]), int(chosen[1]), float(ms.value)

    def set_plain_chunk(self, nodes):
        """Chunk size (nodes) of the plain per-iteration mode."""
        self._check(self._lib.nmc_set_plain_chunk(self._h, int(nodes)), "nmc_set_plain_chunk")

    def opacity_interp(self, which, species, rho, T, Ye, E, out=None, stream=None, mixed=False):
        """chi_EmAb (which = 0) or sigma_Iso (1) of `species` at points (rho, T, Ye, E): CUDA float64
        tensors of one length.  mixed=True runs opacity_interp_mixed (FP32 arithmetic)."""
        import torch
        for x in (rho, T, Ye, E):
            if x.dtype != torch.float64 or not x.is_contiguous() or not x.is_cuda or x.shape != rho.shape:
                raise ValueError("points must be contiguous CUDA float64 tensors of one length")
        if out is None:
            out = torch.empty_like(rho)
        p = lambda x: ctypes.c_void_p(x.data_ptr())  # noqa: E731
        fn = self._lib.opacity_interp_mixed if mixed else self._lib.opacity_interp
        rc = fn(self._h, which, species, rho.shape[0], p(rho), p(T), p(Ye), p(E), p(out), self._stream_handle(stream))
        self._check(rc, "opacity_interp_mixed" if mixed else "opacity_interp")
        return out
