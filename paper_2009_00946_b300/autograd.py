"""torch.autograd form of the differentiable FEWHA solve.

``FewhaSolve.apply(solver, n_iter, slopes, cn2, alpha, w)`` returns the layers
phi = W^T c_K of a cold-started K-step Alg. 2 solve for every frame of
``slopes`` ([B, S] or [S], device, the solver's dtype), as a function of the
Sec. 2.2 model parameters: the Cn^2 fractions gamma_l (``cn2``, [L]), the
regularisation weight alpha (0-d) and the sensor weights w_g = 1/sigma_g^2
([G]), all float64 tensors.  Gradients flow to the slopes and to the three
parameter tensors; the Jacobi preconditioner is a constant of the map.

Every step runs in libfewha's kernels (fewha_solve_taped_batch /
fewha_backward_batch): the frames of a batch are solved together, every kernel
of the operator chain taking all of them in one launch.  This module only
orders the solver's stream against torch's current stream, allocates the tape
(one for the batch, kept until backward) and sums the per-frame parameter
gradients.
"""

from __future__ import annotations

import numpy as np
import torch

from . import fewha


def _host_params(cn2, alpha, w):
    return (cn2.detach().double().cpu().numpy(), float(alpha.detach().double().cpu()),
            w.detach().double().cpu().numpy())


class FewhaSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver: fewha.Solver, n_iter: int, slopes, cn2, alpha, w):
        if not slopes.is_cuda or slopes.dtype != solver.torch_dtype:
            raise ValueError("slopes must be a device tensor of the solver's dtype")
        single = slopes.dim() == 1
        S2 = slopes.reshape(-1, solver.S).contiguous()
        params = _host_params(cn2, alpha, w)
        solver.set_params(*params)
        cur = torch.cuda.current_stream()
        solver.stream.wait_stream(cur)
        B = S2.shape[0]
        tape = torch.empty(solver.tape_bytes_batch(n_iter, B), dtype=torch.uint8, device=slopes.device)
        out = torch.empty(B, solver.N, dtype=solver.torch_dtype, device=slopes.device)
        solver.solve_taped_batch(S2, n_iter, tape, out)
        cur.wait_stream(solver.stream)
        solver.sync()   # BREAKDOWN / INPUT of the solve surface here
        ctx.solver, ctx.n_iter, ctx.params, ctx.tape, ctx.single = solver, n_iter, params, tape, single
        ctx.save_for_backward(S2)
        return out[0] if single else out

    @staticmethod
    def backward(ctx, phibar):
        solver = ctx.solver
        (S2,) = ctx.saved_tensors
        B = S2.shape[0]
        phibar = phibar.reshape(B, solver.N).to(solver.torch_dtype).contiguous()
        dev = S2.device
        solver.set_params(*ctx.params)   # the tape was recorded with these
        cur = torch.cuda.current_stream()
        solver.stream.wait_stream(cur)
        gg = torch.empty(B, solver.n_layers, dtype=torch.float64, device=dev)
        ga = torch.empty(B, dtype=torch.float64, device=dev)
        gw = torch.empty(B, solver.n_wfs, dtype=torch.float64, device=dev)
        gs = torch.empty_like(S2) if ctx.needs_input_grad[2] else None
        solver.backward_batch(S2, ctx.n_iter, ctx.tape, phibar, gg, ga, gw, gs)
        cur.wait_stream(solver.stream)
        ctx.tape = None
        g_slopes = None if gs is None else (gs[0] if ctx.single else gs)
        return None, None, g_slopes, gg.sum(0), ga.sum(), gw.sum(0)


def default_params(cfg: dict, dtype=torch.float64, device="cuda"):
    """(cn2, alpha, w) tensors of a configuration (w_g = 1/sigma_g^2)."""
    cn2 = torch.tensor([l["cn2"] for l in cfg["layers"]], dtype=dtype, device=device)
    alpha = torch.tensor(float(cfg["alpha"]), dtype=dtype, device=device)
    w = torch.tensor([1.0 / wf["sigma"] ** 2 for wf in cfg["wfs"]], dtype=dtype, device=device)
    return cn2, alpha, w


__all__ = ["FewhaSolve", "default_params", "np"]
