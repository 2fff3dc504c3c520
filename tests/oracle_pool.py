"""Oracle work for the GPU tests, run in worker processes started with `spawn`.

Each task carries one node's inputs and rebuilds the grid and the synthetic
tables from their seed, so nothing large crosses the process boundary; no
worker touches the GPU.
"""

import os
from concurrent.futures import ProcessPoolExecutor
import multiprocessing as mp

import numpy as np

from oracle import grid as ogrid, solver as osolver, adjoint as oadjoint, velocity as ovel
from paper_2601_00976_gb300 import synthetic

_TABLES = {}


def _grid_tables(n_elem, de1, nq, ns, table_seed, linear=False):
    key = (n_elem, de1, nq, ns, table_seed, linear)
    if key not in _TABLES:
        edges, _ = ogrid.geometric_edges(n_elem, de1)
        g = ogrid.EnergyGrid(edges, nq)
        _TABLES.clear()
        _TABLES[key] = (g, synthetic.make_tables(g.eps, ns, seed=table_seed, linear=linear))
    return _TABLES[key]


def node_gradient(task):
    """(oracle solve result, oracle IFT gradient) of one node.

    task: case = (n_elem, de1, nq, ns, table_seed), x = the node's inputs
    (rho, T, Ye, D, I, dt, scale), params (oracle Params fields), cot (cotangents).
    """
    g, tables = _grid_tables(*task["case"])
    x = task["x"]
    params = osolver.Params(**task["params"])
    r = osolver.solve_node(g, tables, params, x["rho"], x["T"], x["Ye"], x["D"], x["I"], x["dt"], x["scale"])
    ct = task["cot"]
    grad = oadjoint.gradient(g, tables, params, x["rho"], x["T"], x["Ye"], x["D"], x["I"], x["dt"], x["scale"],
                             r["D"], gD=ct["gD"], gYe=ct["gYe"], geps=ct["geps"], gT=ct["gT"], gH=ct["gH"])
    return r, grad


def node_condition(task):
    """Condition number of dG/dD at the oracle's own converged moments of one node."""
    g, tables = _grid_tables(*task["case"])
    x = task["x"]
    params = osolver.Params(**task["params"])
    r = osolver.solve_node(g, tables, params, x["rho"], x["T"], x["Ye"], x["D"], x["I"], x["dt"], x["scale"])
    return oadjoint.condition_number(g, tables, params, x["rho"], x["T"], x["Ye"], x["D"], x["I"], x["dt"],
                                     x["scale"], r["D"])


def node_velocity(task):
    """Oracle O(v/c) solve of one node; task as node_gradient's plus "v" and "freeze" in x."""
    g, tables = _grid_tables(*task["case"])
    x = task["x"]
    params = osolver.Params(**task["params"])
    return ovel.solve_node(g, tables, params, x["rho"], x["T"], x["Ye"], x["v"], x["D"], x["I"], x["dt"],
                           x["scale"], freeze_velocity=x.get("freeze", False))


def run(tasks, fn=node_gradient, workers=None):
    """fn over tasks in a spawn pool (sequential for one task)."""
    if len(tasks) == 1:
        return [fn(tasks[0])]
    workers = workers or max(1, min(len(tasks), (os.cpu_count() or 2) - 1))
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(fn, tasks))


def cotangents(rng, N, ns, ne):
    """Seeded cotangents of (J, H, Ye, eps, T) with O(1) contributions to the loss."""
    return dict(gD=rng.normal(size=(N, ns, ne)), gH=rng.normal(size=(N, ns, ne, 3)),
                gYe=rng.normal(size=N), geps=rng.normal(size=N) * 1e-19, gT=rng.normal(size=N))


def node_slice(d, n):
    """Node n of a dict of per-node arrays."""
    return {k: (v[n] if np.ndim(v) else v) for k, v in d.items()}
