"""User-facing driver: tr(D^{-1}) of the Schwinger operator by MG-MLMC++.

    est = TraceEstimator(U_host, L, m0)          # uploads U, builds the hierarchy
    res = est.run(eps=1e-3, d=32, k=2)          # Algorithm 2 on the GPU

`U_host` is a numpy complex128 array [L, L, 2] (host); everything after the
upload runs in libmgmlmc's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api


class TraceEstimator:
    def __init__(self, U_host: np.ndarray, L: int, m0: float, ctx: api.Context | None = None,
                 pinned: bool = True, **mg_params):
        self.ctx = ctx or api.Context()
        t = torch.from_numpy(np.ascontiguousarray(U_host, dtype=np.complex128))
        if pinned:
            t = t.pin_memory()
        self.U = t.to("cuda", non_blocking=True)
        self.L, self.m0 = L, m0
        self.h2d_bytes = t.numel() * 16
        self.hier = api.mg_setup(self.ctx, self.U, L, m0, **mg_params)

    def run(self, eps: float = 1e-3, **kw) -> dict:
        return api.trace_estimate(self.ctx, self.hier, eps=eps, **kw)

    def close(self):
        self.hier.close()
