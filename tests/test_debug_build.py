"""The NMC_DEBUG build (bounds checks that record a failed index in a device error word) builds,
exports the same entry points as the release build, and rejects inconsistent shapes on the host
before any launch.  No GPU is needed; tests/test_gpu_debug.py runs its kernels."""

import ctypes

import numpy as np
import pytest

from test_abi import declared_functions


@pytest.fixture(scope="module")
def dlib():
    from paper_2601_00976_gb300 import _build
    _build.build(debug=True)   # incremental: recompiles the units whose sources changed
    return ctypes.CDLL(_build.LIB_DEBUG)


def test_debug_library_exports_every_declared_symbol(dlib):
    for name in declared_functions():
        assert hasattr(dlib, name), name


def test_debug_word_needs_a_context(dlib):
    w = ctypes.c_uint32(7)
    dlib.nmc_debug_word.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int32]
    assert dlib.nmc_debug_word(None, ctypes.byref(w), 0) == 1   # NMC_EINVAL


@pytest.mark.parametrize("n_elem,n_q,ns,ok", [(0, 2, 4, False), (16, 4, 4, False), (16, 2, 3, False),
                                               (16, 2, 8, False), (65, 2, 4, False)])
def test_inconsistent_shapes_are_rejected_before_launch(dlib, n_elem, n_q, ns, ok):
    """Shapes the kernels cannot index are refused by nmc_create on the host: no element, more than 3
    nodes per element, an odd or too large species count, more than 128 energies."""
    from paper_2601_00976_gb300 import nmc
    edges = np.linspace(0.0, 300.0, max(n_elem, 1) + 1)
    g = nmc.Grid(n_elem, n_q, ns, edges.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    t = nmc.Tables()
    dlib.nmc_create.argtypes = [ctypes.POINTER(nmc.Grid), ctypes.POINTER(nmc.Tables), ctypes.POINTER(ctypes.c_void_p)]
    h = ctypes.c_void_p()
    rc = dlib.nmc_create(ctypes.byref(g), ctypes.byref(t), ctypes.byref(h))
    assert rc in (1, 4) and not h.value   # NMC_EINVAL or NMC_EUNSUPPORTED, no context
