"""Differentiable projection y = A x (Sec. II: A x = b) for PyTorch.

`Projector` holds one acquisition (phantom grid + geometry) and applies A or
A^T through the C ABI: on an explicit CSR, or matrix-free in row chunks with
the paths recomputed each time (for systems larger than HBM).  `Project` is
the torch.autograd.Function: forward y = A x, backward g = A^T dL/dy.  No
arithmetic happens here; every product runs in libpct.
"""
from __future__ import annotations

import torch

from . import pct


class Projector:
    def __init__(self, workload: dict, csr: dict | None = None, chunk_rows: int = 10_000_000,
                 precision: int = pct.PREC_MIXED, device="cuda"):
        self.phantom = pct.Phantom(workload["phantom"])
        self.geo = pct.GeometryArgs(workload)
        self.n_rows = self.geo.n_rows
        self.n_cols = self.phantom.nvox
        self.csr = csr
        self.precision = precision
        self.chunk = max(1, min(int(chunk_rows), max(self.n_rows, 1)))
        self.workspace = None
        if csr is None:
            nbytes = pct.projector_workspace_size(self.phantom, self.geo, self.chunk, precision)
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.device = device

    def _chunks(self):
        if self.csr is not None:
            yield 0, self.n_rows
            return
        for r0 in range(0, self.n_rows, self.chunk):
            yield r0, min(self.chunk, self.n_rows - r0)

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        x = x.contiguous().float()
        y = torch.empty(self.n_rows, dtype=torch.float32, device=x.device)
        for r0, n in self._chunks():
            pct.forward(self.phantom, self.geo, self.csr, r0, n, x, y[r0:r0 + n], self.workspace,
                        precision=self.precision)
        return y

    def adjoint(self, r: torch.Tensor) -> torch.Tensor:
        r = r.contiguous().float()
        g = torch.zeros(self.n_cols, dtype=torch.float32, device=r.device)
        for r0, n in self._chunks():
            pct.adjoint(self.phantom, self.geo, self.csr, r0, n, r[r0:r0 + n], g, self.workspace,
                        precision=self.precision)
        return g


class Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, projector: Projector):
        ctx.projector = projector
        return projector.forward(x)

    @staticmethod
    def backward(ctx, gy):
        return ctx.projector.adjoint(gy), None


def project(x: torch.Tensor, projector: Projector) -> torch.Tensor:
    """y = A x with gradient A^T."""
    return Project.apply(x, projector)
