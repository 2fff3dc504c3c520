"""The NMC_TRACE build (per-stage SM-cycle counters of the fused kernel) builds, exports the same
entry points as the release build, and rejects a missing context on the host.  No GPU is needed;
tests/test_gpu_trace.py runs it."""

import ctypes

import pytest

from test_abi import declared_functions


@pytest.fixture(scope="module")
def tlib():
    from paper_2601_00976_gb300 import _build
    _build.build(trace=True)   # incremental: recompiles the units whose sources changed
    return ctypes.CDLL(_build.LIB_TRACE)


def test_trace_library_exports_every_declared_symbol(tlib):
    for name in declared_functions():
        assert hasattr(tlib, name), name


def test_trace_read_needs_a_context(tlib):
    c = (ctypes.c_uint64 * 16)()
    tlib.nmc_trace_read.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
    assert tlib.nmc_trace_read(None, c, 0) == 1   # NMC_EINVAL


def test_stage_table_shares_sum_to_one():
    from paper_2601_00976_gb300 import trace
    counts = [5, 30, 1, 40, 2, 3, 10, 5, 3, 1, 0] + [0] * 5
    rows = trace.stage_table(counts, 10, 100)
    assert len(rows) == len(trace.STAGES)
    assert abs(sum(r[1] for r in rows) - 1.0) < 1e-12
    assert rows[3][0] == "contraction loop and map Q" and rows[3][2] == 4.0
