import numpy as np
import pytest

from oracle import grid as ogrid
from paper_2601_00976_gb300 import synthetic


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU; runs the CUDA path through the C-ABI")


@pytest.fixture(scope="session")
def grid_c1():
    """Grid C (16 elements) with linear elements: 32 energy nodes."""
    edges, _ = ogrid.geometric_edges(16, 1.875)
    return ogrid.EnergyGrid(edges, 2)


@pytest.fixture(scope="session")
def grid_c0():
    """Grid C with constant elements: 16 energy nodes."""
    edges, _ = ogrid.geometric_edges(16, 1.875)
    return ogrid.EnergyGrid(edges, 1)


@pytest.fixture(scope="session")
def grid_tiny():
    """Four geometric elements with linear elements: 8 energy nodes."""
    edges, _ = ogrid.geometric_edges(4, 20.0)
    return ogrid.EnergyGrid(edges, 2)


@pytest.fixture(scope="session")
def tables_c1_4(grid_c1):
    return synthetic.make_tables(grid_c1.eps, 4, seed=0)


def read_golden(name):
    rows = []
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows
