"""torch.autograd front end of the training path (Sec. 1, shifted reverse KL).

`flow_sample(flow, theta, ...)` returns (phi, log q) as differentiable functions
of the flat FP32 weight tensor `theta`; `phi4_action(...)` returns S(phi) as a
differentiable function of phi.  Their backward passes call the library's
reverse pass and action VJP, so a loss assembled in torch, e.g.

    phi, logq = flow_sample(flow, theta, B, seed=s, counter0=c)
    loss = (logq + phi4_action(nd, L, phi4, phi)).mean()
    loss.backward()          # theta.grad = dloss/dtheta from libgfflow kernels

gives the same gradient as Flow.train_step.  The fused train step remains the
fast path; this one lets torch optimisers and custom losses drive the flow.
"""
from __future__ import annotations

import torch
from torch.autograd.function import once_differentiable

from . import api


class _FlowSample(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, flow, B, seed, counter0, z):
        flow.set_weights(theta.detach().contiguous())
        phi, logq, ws = flow.forward_train(B, seed=seed, counter0=counter0, z=z)
        ctx.flow, ctx.B, ctx.ws, ctx.version = flow, B, ws, flow.weights_version
        return phi, logq

    @staticmethod
    @once_differentiable
    def backward(ctx, gphi, glogq):
        flow = ctx.flow
        if flow.weights_version != ctx.version:
            raise RuntimeError("the flow's weights changed between forward and backward")
        if ctx.ws is None:
            raise RuntimeError("backward through the same flow_sample twice")
        g = flow.backward(ctx.B, None if gphi is None else gphi.contiguous(),
                          None if glogq is None else glogq.contiguous(), ctx.ws)
        ctx.ws = None                         # the reverse pass overwrites the workspace
        return g, None, None, None, None, None


class _Phi4Action(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, nd, L, phi4):
        ctx.save_for_backward(phi)
        ctx.nd, ctx.L, ctx.phi4 = nd, L, phi4
        return api.phi4_action(nd, L, phi4, phi)

    @staticmethod
    @once_differentiable
    def backward(ctx, gS):
        (phi,) = ctx.saved_tensors
        return api.phi4_action_vjp(ctx.nd, ctx.L, ctx.phi4, phi, gS.contiguous()), None, None, None


def flow_sample(flow: "api.Flow", theta: torch.Tensor, B: int, seed: int = 0, counter0: int = 0,
                z: torch.Tensor | None = None):
    """(phi [B][V] FP32, log q [B] FP64), differentiable in theta [n_params] FP32."""
    if flow.precision != "fp32":
        raise ValueError("the training path runs on FP32 flows")
    return _FlowSample.apply(theta, flow, B, seed, counter0, z)


def phi4_action(nd: int, L: int, phi4, phi: torch.Tensor) -> torch.Tensor:
    """S(phi) [B] FP64, differentiable in the FP32 field phi."""
    return _Phi4Action.apply(phi, nd, L, phi4)


def reverse_kl_loss(flow: "api.Flow", theta: torch.Tensor, B: int, phi4, seed: int = 0,
                    counter0: int = 0, z: torch.Tensor | None = None) -> torch.Tensor:
    """(1/B) sum_b [log q(phi_b) + S(phi_b)] (the shifted reverse KL, ln Z omitted)."""
    phi, logq = flow_sample(flow, theta, B, seed=seed, counter0=counter0, z=z)
    return (logq + phi4_action(flow.shape.nd, flow.shape.L, phi4, phi)).mean()
