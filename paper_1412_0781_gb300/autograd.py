"""torch.autograd wrappers of the library's linear maps.

Coefficients are real tensors (n, P, 2) holding (Re, Im), so every map here
is real-linear and its backward is the transpose for the plain real inner
product, i.e. the adjoint for Re sum conj(u) v:

* ``Expand``      a = T* I                backward: T g (ffb_expand_adjoint)
* ``Filter``      a' = M (a - m) + m      backward: M g (ffb_filter, linear part;
                                           M = U diag(h) U^T is symmetric; the
                                           selected eigenvectors are constants)
* ``Synthesize``  I = T (W a)             backward: W T* g (ffb_weight(ffb_expand))

All arithmetic runs in libffb.so; these classes only route tensors.
"""
import torch


class Expand(torch.autograd.Function):
    @staticmethod
    def forward(ctx, images, plan):
        ctx.plan = plan
        return plan.expand(images.contiguous())

    @staticmethod
    def backward(ctx, grad):
        return ctx.plan.expand_adjoint(grad.contiguous()), None


class Filter(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coef, plan):
        ctx.plan = plan
        return plan.filter(coef.contiguous())

    @staticmethod
    def backward(ctx, grad):
        return ctx.plan.filter(grad.contiguous(), linear=True), None


class Synthesize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coef, plan):
        ctx.plan = plan
        return plan.synthesize(coef.contiguous())

    @staticmethod
    def backward(ctx, grad):
        return ctx.plan.weight(ctx.plan.expand(grad.contiguous())), None


def expand(images, plan):
    return Expand.apply(images, plan)


def steerable_filter(coef, plan):
    return Filter.apply(coef, plan)


def synthesize(coef, plan):
    return Synthesize.apply(coef, plan)


def denoise(images, plan):
    """Differentiable denoising with the plan's selected filter (ffb_select)."""
    return synthesize(steerable_filter(expand(images, plan), plan), plan)
