"""torch.autograd.Function over the library's forward run and hand-written
discrete adjoint (mx_rk_forward_record / mx_rk_backward): argument
marshalling only; both passes run in libmx."""
import torch


class RK4Run(torch.autograd.Function):
    """m_T = RK4^n(normalize(m0_raw)) with gradients to m0_raw and the Ms map.

    ``ms_map`` must be the (nz, ny, nx) float32 CUDA tensor set on the context;
    it is an input only so that autograd routes dJ/dMs to it.
    """

    @staticmethod
    def forward(fctx, m0_raw, ms_map, ctx, dt):
        fctx.ctx = ctx
        fctx.want_ms = ms_map is not None and ms_map.requires_grad
        return ctx.rk_forward_record(m0_raw.contiguous(), dt)

    @staticmethod
    def backward(fctx, lam):
        g_m0, g_ms = fctx.ctx.rk_backward(lam.contiguous(), want_ms=fctx.want_ms)
        return g_m0, g_ms, None, None


def rk4_run(ctx, m0_raw, dt, ms_map=None):
    return RK4Run.apply(m0_raw, ms_map, ctx, dt)
