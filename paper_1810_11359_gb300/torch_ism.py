"""PyTorch front end: RIRs of a batch of rooms as a differentiable function of
the reflection coefficients and the source and receiver positions.

Forward: one ism_simulate_batch call (all rooms in one set of launches).
Backward: one ism_simulate_backward_batch call, the adjoint kernel of the
library (the chain rule through eq. (1)-(6)); nothing is recomputed in
PyTorch.  PyTorch supplies device memory and the current stream only.

    h = rir(L, beta, pos_src, pos_rcv, Tmax=0.4, fs=16000.0, Tw=32 / 16000)
    loss = ((h - target) ** 2).sum()
    loss.backward()          # beta.grad, pos_src.grad, pos_rcv.grad

Shapes: one room -- L [3], beta [6], pos_src [S, 3], pos_rcv [M, 3] ->
h [S, M, n_S]; B rooms -- L [B, 3], beta [B, 6], pos_src [B, S, 3],
pos_rcv [B, M, 3] -> h [B, S, M, n_S].  All rooms share Tmax, fs, Tdiff and
Tw.  The samples of a diffuse tail (k >= ceil(Tdiff fs)) carry no gradient.
A CUDA beta is read by the kernels in place (ism_job.beta_dev): a training
step then never waits for the GPU; a CPU beta is copied into the job structs
(and its gradient back to the host, which waits for the backward pass).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import ism


@dataclass
class _Spec:
    L: np.ndarray          # [B, 3] FP64
    nb_img: np.ndarray     # [B, 3] int
    Tmax: float
    fs: float
    Tdiff: float
    Tw: float
    c: float
    seed: int
    prec: str
    workspace: Optional[ism.Workspace]


def _jobs(spec: _Spec, beta, ps: torch.Tensor, pr: torch.Tensor, out: torch.Tensor):
    # beta: [B, 6] host array, or FP32 CUDA tensor read in place (ism_job.beta_dev)
    return ism.make_jobs_strided(spec.L, beta, ps, pr, spec.nb_img, spec.Tmax, spec.fs, out, Tdiff=spec.Tdiff,
                                 Tw=spec.Tw, c=spec.c, seed=spec.seed)


class _RoomsRIR(torch.autograd.Function):
    @staticmethod
    def forward(ctx, beta, pos_src, pos_rcv, spec: _Spec):
        B, S, M = pos_src.shape[0], pos_src.shape[1], pos_rcv.shape[1]
        n_S = ism.ism_rir_length(spec.Tmax, spec.fs)
        ps = pos_src.detach().float().contiguous()
        pr = pos_rcv.detach().float().contiguous()
        if beta.is_cuda:   # read in place by the kernels: no copy to the host, no synchronisation
            beta_k = beta.detach().to(device=ps.device, dtype=torch.float32).reshape(B, 6).contiguous()
        else:
            beta_k = beta.detach().double().numpy().reshape(B, 6)
        out = torch.empty((B, S, M, n_S), dtype=torch.float32, device=ps.device)
        ism.ism_simulate_batch(_jobs(spec, beta_k, ps, pr, out), prec=spec.prec, workspace=spec.workspace)
        ctx.spec = spec
        ctx.beta_k = beta_k
        ctx.beta_meta = (beta.dtype, beta.device)
        ctx.save_for_backward(ps, pr)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        ps, pr = ctx.saved_tensors
        spec = ctx.spec
        B, S, M = ps.shape[0], ps.shape[1], pr.shape[1]
        go = grad_out.float().contiguous()
        gb = torch.empty((B, 6), dtype=torch.float32, device=ps.device)
        gs = torch.empty((B, S, 3), dtype=torch.float32, device=ps.device)
        gr = torch.empty((B, M, 3), dtype=torch.float32, device=ps.device)
        gjobs = ism.make_grad_jobs_strided(_jobs(spec, ctx.beta_k, ps, pr, go), go, gb, gs, gr)
        ism.ism_simulate_backward_batch(gjobs, workspace=spec.workspace)
        dtype, device = ctx.beta_meta
        return gb.to(dtype=dtype, device=device), gs, gr, None


def rir(L, beta, pos_src, pos_rcv, Tmax: float, fs: float, Tw: float = 0.0, nb_img=None, Tdiff: float = 0.0,
        c: float = 343.0, seed: int = 0, prec: str = "fp32", workspace: Optional[ism.Workspace] = None):
    """RIRs [S, M, n_S] (one room) or [B, S, M, n_S] (B rooms), differentiable
    with respect to beta, pos_src and pos_rcv.  nb_img defaults to the images
    per axis that cover max(Tdiff, Tmax) if there is no tail, else Tdiff
    (ism_nb_img_from_t)."""
    single = torch.as_tensor(pos_src).dim() == 2
    Lh = np.asarray(L, dtype=np.float64).reshape(-1, 3)
    B = Lh.shape[0]
    beta_t = torch.as_tensor(beta) if not isinstance(beta, torch.Tensor) else beta
    ps = pos_src if isinstance(pos_src, torch.Tensor) else torch.as_tensor(np.asarray(pos_src, np.float32))
    pr = pos_rcv if isinstance(pos_rcv, torch.Tensor) else torch.as_tensor(np.asarray(pos_rcv, np.float32))
    if single:
        beta_t, ps, pr = beta_t.reshape(1, 6), ps.unsqueeze(0), pr.unsqueeze(0)
    if ps.device.type != "cuda" or pr.device.type != "cuda":
        raise ValueError("pos_src and pos_rcv must be CUDA tensors")
    if ps.shape[0] != B or pr.shape[0] != B or beta_t.shape[0] != B:
        raise ValueError("L, beta, pos_src and pos_rcv must describe the same number of rooms")
    T_img = Tdiff if (Tdiff and 0.0 < Tdiff < Tmax) else Tmax
    if nb_img is None:
        nb = np.array([ism.ism_nb_img_from_t(T_img, Lh[b], c, Tw if Tw else 4e-3) for b in range(B)], np.int32)
    else:
        nb = np.asarray(nb_img, np.int32).reshape(-1, 3)
        nb = np.repeat(nb, B, axis=0) if nb.shape[0] == 1 else nb
    spec = _Spec(L=Lh, nb_img=nb, Tmax=float(Tmax), fs=float(fs), Tdiff=float(Tdiff or 0.0), Tw=float(Tw or 0.0),
                 c=float(c), seed=int(seed), prec=prec, workspace=workspace)
    out = _RoomsRIR.apply(beta_t, ps, pr, spec)
    return out[0] if single else out
