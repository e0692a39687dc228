"""torch.autograd integration: a fused dcp program as a differentiable function.

Forward runs the fused program (dcp_run); backward runs its reverse pass
(dcp_run_adjoint: one fused kernel per reverse step, states taped or
sqrt(T)-checkpointed within ``tape_budget_bytes``).  Torch only provides the
tensors and the stream.
"""
from __future__ import annotations

import torch


class DcpFunction(torch.autograd.Function):
    """``DcpFunction.apply(graph, tape_budget_bytes, *inputs)`` -> outputs."""

    @staticmethod
    def forward(ctx, graph, tape_budget_bytes, *inputs):
        inputs = [t.contiguous() for t in inputs]
        outs = graph.run(inputs)
        ctx.graph = graph
        ctx.budget = int(tape_budget_bytes)
        ctx.save_for_backward(*inputs)
        return outs[0] if len(outs) == 1 else tuple(outs)

    @staticmethod
    def backward(ctx, *grads):
        inputs = ctx.saved_tensors
        g = ctx.graph
        out_grads = []
        for v, gr in zip(g.outputs, grads):
            if gr is None:
                gr = torch.zeros(g.shape[v], dtype=inputs[0].dtype, device=inputs[0].device)
            out_grads.append(gr.contiguous())
        in_grads = g.adjoint(list(inputs), out_grads, tape_budget_bytes=ctx.budget)
        return (None, None, *in_grads)


def apply(graph, *inputs, tape_budget_bytes=1 << 62):
    """Differentiable call of a fused graph on CUDA tensors."""
    return DcpFunction.apply(graph, tape_budget_bytes, *inputs)
