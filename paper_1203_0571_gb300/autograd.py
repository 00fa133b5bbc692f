"""torch.autograd bridges of libfse: the chi^2 adjoint (fse_sersic_chi2_grad)
and the moment fixed point (fse_ellipticity / fse_centroid with
fse_moment_vjp).

    chi2 = sersic_chi2(params, pix, index, ctx)        # float64 [N]
    chi2.sum().backward()                              # params.grad, pix.grad

    theta = moment_shape(pix, index, ctx)              # float32 [N, 5]: x0, y0, e1, e2, sigma_w
    loss(theta).backward()                             # pix.grad

params is float32 [N, 7] = (x0, y0, e1, e2, I0, r_e, n) per stamp (Eq. 10 with
the ellipticity of Eq. A1); pix is the flat float32 pixel buffer indexed by
`index` (fse_stamp rows, see binding.make_index).  The forward launch computes
chi^2 (Eq. 11) only.  The backward launch computes the vector-Jacobian
product: the upstream gradient of each stamp times d chi^2/dp and, when the
pixels require a gradient, d chi^2/dI.  Both run in libfse's kernel; this
module only passes tensors through.
"""
from __future__ import annotations

import torch

from . import binding as B


class SersicChi2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, pix, index, fse, scale, inv_var):
        if pix.dtype != torch.float32 and pix.requires_grad:
            raise TypeError("pixel gradients need float32 pixels")
        chi2, _, _ = fse.chi2_grad(pix.detach(), index, params.detach(), scale=scale,
                                   inv_var=inv_var, want_dparams=False)
        ctx.save_for_backward(params.detach(), pix.detach(), index)
        ctx.fse, ctx.scale, ctx.inv_var = fse, scale, inv_var
        return chi2

    @staticmethod
    def backward(ctx, gchi2):
        params, pix, index = ctx.saved_tensors
        need_p, need_pix = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        _, dpar, dpix = ctx.fse.chi2_grad(pix, index, params, scale=ctx.scale, inv_var=ctx.inv_var,
                                          gout=gchi2, want_chi2=False, want_dparams=need_p,
                                          want_dpix=need_pix)
        return dpar, dpix, None, None, None, None


def sersic_chi2(params: torch.Tensor, pix: torch.Tensor, index: torch.Tensor, ctx: B.Context,
                scale: torch.Tensor | None = None, inv_var: torch.Tensor | None = None) -> torch.Tensor:
    """chi^2 per stamp with gradients to params and pixels through libfse."""
    return SersicChi2.apply(params, pix, index, ctx, scale, inv_var)


class MomentShape(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pix, index, fse, opts, ellip):
        if pix.dtype != torch.float32 and pix.requires_grad:
            raise TypeError("pixel gradients need float32 pixels")
        p = pix.detach()
        mom = fse.centroid(p, index, opts=opts)
        if ellip:
            fse.ellipticity(p, index, mom, opts=opts)
        r = mom.view(torch.float32).reshape(-1, 16)
        # x0, y0, e1, e2 are floats 0-3 of the record, sigma_w float 14
        theta = torch.cat([r[:, 0:4], r[:, 14:15]], dim=1).clone()
        if not ellip:
            theta[:, 2:4] = 0.0
        ctx.save_for_backward(p, index, mom)
        ctx.fse, ctx.ellip = fse, ellip
        ctx.mode = (B.FSE_MOM_ELLIP if ellip else 0) | \
            (B.FSE_MOM_SIGW_R50 if (opts or B.default_opts()).sigw_mode == 1 else 0)
        return theta

    @staticmethod
    def backward(ctx, gtheta):
        pix, index, mom = ctx.saved_tensors
        dpix = ctx.fse.moment_vjp(pix, index, mom, gtheta, mode=ctx.mode)
        return dpix, None, None, None, None


def moment_shape(pix: torch.Tensor, index: torch.Tensor, ctx: B.Context, opts=None,
                 ellip: bool = True) -> torch.Tensor:
    """The moment fixed point (x0, y0, e1, e2, sigma_w) of each stamp (Secs. 2-3;
    Sec. 2 alone with ellip=False), differentiable with respect to the pixels
    through the implicit-function theorem."""
    return MomentShape.apply(pix, index, ctx, opts, ellip)
