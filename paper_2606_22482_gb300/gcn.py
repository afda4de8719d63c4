"""GCN forward on the hybrid SpMM (the paper's GNN workload, Section 8.6 / Table 3).

Each layer is H' = act(A_hat (H W)): the dense product H W is a plain library GEMM (cuBLAS
through torch.matmul, FP32 without TF32), the sparse product A_hat (H W) is one execution of a
plan made once for A_hat and reused by every layer and epoch, which is how the paper amortises
partitioning over a training run.
"""
from __future__ import annotations

import torch

from . import Plan


class GCN:
    """A stack of GCN layers sharing one SpMM plan of the normalised adjacency A_hat.

    ``weights``: list of (K_in x K_out) FP32 CUDA tensors; every K_out must equal the plan's K.
    The hidden layers apply ReLU, the last one none.
    """

    def __init__(self, plan: Plan, weights: list):
        self.plan = plan
        self.weights = weights
        for W in weights:
            if not W.is_cuda or W.dtype != torch.float32 or W.shape[1] != plan.K:
                raise ValueError("weights must be FP32 CUDA tensors with K_out equal to the plan's K")
        self._bufs = None

    def _buffers(self, m: int, dev):
        if self._bufs is None or self._bufs[0].shape[0] != m:
            K = self.plan.K
            self._bufs = [torch.empty((m, K), device=dev, dtype=torch.float32) for _ in range(3)]
        return self._bufs

    def forward(self, X: torch.Tensor, stream=None) -> torch.Tensor:
        """Run every layer on X (n x K_in, FP32 CUDA); returns the last layer's output (m x K)."""
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        try:
            XW, H0, H1 = self._buffers(X.shape[0], X.device)
            H = X
            out = None
            for li, W in enumerate(self.weights):
                torch.matmul(H, W, out=XW)
                out = H0 if li % 2 == 0 else H1
                self.plan.execute(XW, out, stream=stream)
                if li + 1 < len(self.weights):
                    torch.relu_(out)
                H = out
            return out
        finally:
            torch.backends.cuda.matmul.allow_tf32 = prev
