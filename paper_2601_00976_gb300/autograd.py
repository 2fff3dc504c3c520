"""torch.autograd.Function around collision_solve / collision_adjoint.

``CollisionSolve.apply(ctx, params, rho, T, Ye, J, H, dt, scale)`` runs the
collision solve (Algorithm 1) and returns (J_out, H_out, Ye_out, eps_out,
T_out, n_outer, n_inner, status).  Its backward calls the library's adjoint
kernel, which differentiates the converged solve by the implicit-function
theorem, so gradients flow from every floating-point output to T, Ye, J, H and
the opacity scale factors.  rho and dt get no gradient.  Argument marshalling
only: the solve and its adjoint run in the library's CUDA kernels.
"""

import torch


class CollisionSolve(torch.autograd.Function):
    @staticmethod
    def forward(fctx, nctx, params, rho, T, Ye, J, H, dt, scale):
        out = nctx.collision_solve(params, rho, T, Ye, J, H, dt, scale)
        fctx.nctx = nctx
        fctx.params = params
        fctx.has_scale = scale is not None
        fctx.save_for_backward(rho, T, Ye, J, H, dt, scale if scale is not None else rho, out["J"], out["T"])
        fctx.set_materialize_grads(False)
        fctx.mark_non_differentiable(out["n_outer"], out["n_inner"], out["status"])
        return (out["J"], out["H"], out["Ye"], out["eps"], out["T"], out["n_outer"], out["n_inner"],
                out["status"])

    @staticmethod
    def backward(fctx, gJ, gH, gYe, geps, gT, *_):
        rho, T, Ye, J, H, dt, scale, J_out, T_out = fctx.saved_tensors
        if not fctx.has_scale:
            scale = None
        c = lambda g: None if g is None else g.contiguous()  # noqa: E731
        g = fctx.nctx.collision_adjoint(fctx.params, rho, T, Ye, J, H, dt, scale, J_out, T_out,
                                        gJ=c(gJ), gH=c(gH), gYe=c(gYe), geps=c(geps), gT=c(gT))
        need = fctx.needs_input_grad
        return (None, None, None,
                g["T"] if need[3] else None,
                g["Ye"] if need[4] else None,
                g["J"] if need[5] else None,
                g["H"] if need[6] else None,
                None,
                g["scale"] if (need[8] and fctx.has_scale) else None)


def collision_solve(nctx, params, rho, T, Ye, J, H, dt, scale=None):
    """Differentiable collision solve: (J_out, H_out, Ye_out, eps_out, T_out, n_outer, n_inner, status)."""
    return CollisionSolve.apply(nctx, params, rho, T, Ye, J, H, dt, scale)
