"""Where the fused mixed kernel's time goes: runs the headline workload's first n nodes (perturbed
collapse profile, 4 species, Grid F 32 x 2 = 64 energies, mixed precision at tol 1e-10 / 1e-9) through
the NMC_TRACE build and prints the share of each stage of Algorithm 1 in the blocks' time.

    python -m paper_2601_00976_gb300._build --trace
    NMC_TRACE=1 python -m paper_2601_00976_gb300.trace --nodes 262144

The counters are thread 0's SM cycles between stage boundaries, summed over blocks (block time:
barrier waits and cycles the SM gives to other resident blocks included).
"""

import argparse
import os
import sys

STAGES = ("node set-up", "ComputeOpacities", "reference norms, first vectors", "contraction loop and map Q",
          "least-squares partial sums", "least-squares solve", "Anderson mixing, next vectors",
          "Algorithm 2 vote", "matter update", "final state, outputs", "next node from the queue")


def stage_table(counts, n_nodes, n_inner):
    """Rows (stage, share, cycles per node, cycles per inner iteration) from the 16 trace counters."""
    tot = float(sum(counts[:len(STAGES)])) or 1.0
    return [(name, counts[i] / tot, counts[i] / n_nodes, counts[i] / max(n_inner, 1)) for i, name in enumerate(STAGES)]


def main():
    if os.environ.get("NMC_TRACE") != "1":
        sys.exit("set NMC_TRACE=1 to load the stage-counter build")
    ap = argparse.ArgumentParser()
    ap.add_argument("--nodes", type=int, default=1 << 18)
    ap.add_argument("--seed", type=int, default=1234)
    args = ap.parse_args()
    import numpy as np
    import torch
    from paper_2601_00976_gb300 import nmc, synthetic
    edges, _ = nmc.geometric_edges(32, 1.0)
    eps, _, _ = nmc.grid_nodes(edges, 2)
    tables = synthetic.make_tables(eps, 4, seed=0)
    inp = synthetic.make_inputs("perturbed", args.nodes, eps, 4, seed=args.seed)
    ctx = nmc.Context(edges, 2, 4, tables)
    t = {k: torch.tensor(v, device="cuda") for k, v in inp.items()}
    p = nmc.default_params(tol_inner=1e-10, tol_outer=1e-9, m_inner=3, m_outer=3, precision=nmc.MIXED)
    args_t = (t["rho"], t["T"], t["Ye"], t["D"], t["I"], t["dt"], t["scale"])
    ctx.collision_solve(p, *args_t)       # warm-up (module load, clocks)
    torch.cuda.synchronize()
    ctx.trace_read(clear=True)
    out = ctx.collision_solve(p, *args_t)
    torch.cuda.synchronize()
    counts = ctx.trace_read(clear=True)
    n_inner = int(out["n_inner"].sum().item())
    print(f"{args.nodes} nodes, {n_inner / args.nodes:.2f} inner and {out['n_outer'].float().mean().item():.2f} "
          f"outer iterations per node, {int(torch.count_nonzero(out['status']).item())} flagged")
    print(f"{'stage':34s} {'share':>7s} {'cycles/node':>12s} {'cycles/inner':>13s}")
    for name, share, per_node, per_inner in stage_table(counts, args.nodes, n_inner):
        print(f"{name:34s} {100 * share:6.2f}% {per_node:12.0f} {per_inner:13.0f}")
    ctx.close()


if __name__ == "__main__":
    main()
