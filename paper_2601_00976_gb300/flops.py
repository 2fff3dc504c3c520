"""Algorithmic floating-point work of one collision solve (roofline numerator).

Counts the arithmetic Algorithm 1 requires, not what a kernel happens to
execute: an FMA is 2 flops; an add, multiply, divide, square root, exp or log is
1 flop.  Per node, with L = 4 ns ne unknowns and Anderson memory m:

inner iteration
  rates (Eqs. nesRatesNodal, pairRatesNodal): NES 2 mat-vecs and pair 2 mat-vecs
  per species, 2 ne^2 flops each                         -> 8 ns ne^2
  vectors, totals, map Q, residual, Gram row, mixing, Algorithm 2
                                                         -> (13 + 4 m) L
outer iteration (ComputeOpacities + matter update)
  EoS root find (about 6 Newton steps of ~100 flops)     -> 600
  Fermi-Dirac at 16 points per element (exp + 3)         -> 4 * 16 ns n_elem
  projection (2 (nq + 1) per point) and limiter          -> 2 (nq+1) 16 ns n_elem + 20 ns n_elem
  EmAb/Iso trilinear + exp (2 tables, 33 each)           -> 66 ns ne
  NES lower triangle bilinear (9), upper by detailed balance (2),
  pair bilinear (9)                                      -> 9 ns ne(ne+1)/2 + 2 ns ne(ne-1)/2 + 9 (ns/2) ne^2
  D/(1-D), norms, matter sums                            -> 11 ns ne
final: EoS root find 600, initial sums 4 ns ne.
"""


def inner_flops(ns, ne, m, nes=True, pair=True):
    L = 4 * ns * ne
    mv = (4 * ns * ne * ne if nes else 0) + (4 * ns * ne * ne if pair else 0)
    return mv + (13 + 4 * m) * L


def outer_flops(ns, ne, n_elem, nq, nes=True, pair=True):
    f = 600 + 4 * 16 * ns * n_elem + 2 * (nq + 1) * 16 * ns * n_elem + 20 * ns * n_elem
    f += 66 * ns * ne + 11 * ns * ne
    if nes:
        f += 9 * ns * ne * (ne + 1) // 2 + 2 * ns * ne * (ne - 1) // 2
    if pair:
        f += 9 * (ns // 2) * ne * ne
    return f


def node_flops(ns, ne, n_elem, nq, m, n_inner, n_outer, nes=True, pair=True):
    """Total flops of one node given its inner and outer iteration counts (arrays ok)."""
    return (n_inner * inner_flops(ns, ne, m, nes, pair) + n_outer * outer_flops(ns, ne, n_elem, nq, nes, pair)
            + 600 + 4 * ns * ne)


def mixed_fp64_flops(ns, ne, n_outer):
    """The part of node_flops that the mixed-precision path keeps in FP64 (the rest runs in FP32):
    per outer iteration the EoS root find (600) and the matter sums E_nu, N_nu (4 ns ne), and once the
    final EoS root find and the initial sums.  The inner least-squares solves are FP64 as well but
    are not part of node_flops's count (their Gram entries are, and those are FP32)."""
    return n_outer * (600 + 4 * ns * ne) + 600 + 4 * ns * ne


def adjoint_flops(ns, ne, n_elem, nq, with_h=True):
    """Algorithmic flops of one node's gradient by the adjoint kernel.

    five ComputeOpacities passes (the matter state and its four central-difference
    neighbours in eps and Ye), each with its EoS root find   -> 5 outer_flops
    five unit-scale rate evaluations (4 mat-vecs per species) and map values
                                                              -> 5 (8 ns ne^2 + 20 ns ne)
    dQ_D/dD rows from the kernel matrices (NES 8, pair 10 per entry) -> 18 ns ne^2
    dkappa/dD^T g_kappa (NES 3, pair 5 per entry, with an H cotangent) -> 8 ns ne^2
    per particle/antiparticle pair, Gaussian elimination of an n x n block with
    three right-hand sides and the back substitutions, n = 2 ne
                                                              -> (ns/2) (2/3 n^3 + 6 n^2)
    Woodbury update, reductions and outputs                   -> 30 ns ne
    """
    n2 = 2 * ne
    f = 5 * outer_flops(ns, ne, n_elem, nq) + 5 * (8 * ns * ne * ne + 20 * ns * ne)
    f += 18 * ns * ne * ne + (8 * ns * ne * ne if with_h else 0)
    f += (ns // 2) * (2 * n2 ** 3 // 3 + 6 * n2 * n2)
    return f + 30 * ns * ne


def velocity_node_flops(ns, ne, n_elem, nq, m, n_inner, n_outer):
    """Flops of one node of the O(v/c) solve: node_flops plus the velocity terms.

    per inner iteration and bin: the closure (|I|, h, Minerbo psi, the two
    coefficients of K: ~25), v.I and v^i K_ij (~11), the lambda-form map of
    D and I (~14)                                              -> 50 ns ne
    per outer iteration: the fifteen Eulerian terms per bin (~25) and the
    five-component matter update and least squares (~100)      -> 25 ns ne + 100
    once: the old state's conserved moments and Eulerian sums (~65 per bin)
    and the final momentum solve with its sums (~100)          -> 65 ns ne + 100
    """
    return (node_flops(ns, ne, n_elem, nq, m, n_inner, n_outer) + n_inner * 50 * ns * ne
            + n_outer * (25 * ns * ne + 100) + 65 * ns * ne + 100)


def c2p_bin_flops(iters):
    """Flops of one bin's conserved-to-primitive recovery with `iters` iterations.

    per iteration: the closure (|I|, h, Minerbo psi, K's two coefficients: ~25),
    v.I and the map of D and I (~20), the residual and the four-vector dot
    products of the eliminated normal equations (~40), the 2 x 2 solve (~15),
    the mixing and the stopping norm (~20)                        -> 120
    once: lambda and the reference norm                              -> 10
    """
    return 120 * iters + 10


def interp_point_flops():
    """Algorithmic flops of one opacity_interp point (tetralinear in log10 rho, log10 T, Ye, ln E).

    two log10 and one ln of the coordinates                   -> 3
    cell offsets and fractions on four axes (2 each, the
    energy fraction a division more)                          -> 9
    the complements 1 - t of three axes                       -> 3
    per corner of the (rho, T, Ye) cube: its weight (2),
    the linear blend of the two energy entries (3), the
    weighted accumulation (FMA, 2)                            -> 8 x 7
    exp of the interpolated logarithm                         -> 1
    """
    return 3 + 9 + 3 + 8 * 7 + 1
