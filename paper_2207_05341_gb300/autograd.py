"""torch.autograd bridge for the NN-QST likelihood of libqst.

``QstLikelihood.apply(theta, f, ctx)`` returns L(theta) = -sum_k f_k log p_k
(Sec. 3.1) for the 3-layer network, Chol_H state map (Sec. 3.2) and product
POVM (Sec. 3.3).  Forward and backward run in libqst's kernels through
``qst_loss_grad``: the forward pass already produces dL/dtheta with the
hand-written backward kernels (adjoint POVM chain, G T product, network
backward), and the probabilities q are recomputed inside the fused kernels,
never stored.  ``backward`` only scales that gradient by the incoming
gradient.  PyTorch is used for the tensors and the autograd graph; no
arithmetic of the method runs in PyTorch.
"""
from __future__ import annotations

import torch

from . import qst


class QstLikelihood(torch.autograd.Function):
    @staticmethod
    def forward(actx, theta: torch.Tensor, f: torch.Tensor, handle: int):
        if not theta.is_cuda or not f.is_cuda:
            raise ValueError("theta and f must be CUDA tensors")
        th = theta.detach().contiguous()
        dtheta = torch.empty_like(th)
        loss, _ = qst.qst_loss_grad(handle, th, f.detach().contiguous(), dtheta)
        actx.save_for_backward(dtheta)
        return torch.tensor(loss, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(actx, grad_out):
        (dtheta,) = actx.saved_tensors
        return dtheta * grad_out.to(dtheta.dtype), None, None


class NNQST(torch.nn.Module):
    """The paper's network as a module: theta is a Parameter, forward(f) returns the loss.

    Training with any torch optimizer goes through QstLikelihood; the fused
    in-library loop (qst_step / qst_reconstruct) does the same iteration with
    Rprop fused into the weight passes.
    """

    def __init__(self, N: int, theta0: torch.Tensor, precision: int = qst.QST_FP32, stream: int = 0):
        super().__init__()
        opt = qst.qst_default_options()
        opt.precision = precision
        self.N = N
        self.handle = qst.qst_init(N, opt=opt, stream=stream)
        if theta0.numel() != qst.qst_theta_size(N):
            raise ValueError("theta0 has the wrong size")
        self.theta = torch.nn.Parameter(theta0.detach().clone())

    def forward(self, f: torch.Tensor) -> torch.Tensor:
        return QstLikelihood.apply(self.theta, f, self.handle)

    def close(self):
        if self.handle:
            qst.qst_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
