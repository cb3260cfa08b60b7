"""The McWeeny purification chain X <- 3X^2 - 2X^3 as one CUDA graph.

An eager pass runs every multiply and add once and fixes the storage of
each intermediate handle; the same sequence of calls is then captured with
``no_sync`` (no host synchronisation) into a ``torch.cuda.CUDAGraph``.  A
replay recomputes every pattern and value on the device into that storage;
if a recomputed size differs from the eager pass (new values that change
the filtered patterns), the handle's device status word is set and the
handle keeps its old contents -- ``status()`` reports it.
"""
from __future__ import annotations

import torch

from . import bsm


class McWeenyGraph:
    def __init__(self, X0: bsm.Matrix, steps: int, eps: float, prec: str = "fp64"):
        self.X0, self.steps, self.eps, self.prec = X0, steps, eps, prec
        self.X, self.X2, self.X3 = [X0], [], []
        for _ in range(steps):
            X = self.X[-1]
            X2 = bsm.multiply(1.0, X, X, eps=eps, prec=prec, build_stacks=False)
            X3 = bsm.multiply(1.0, X2, X, eps=eps, prec=prec, build_stacks=False)
            self.X.append(bsm.add(3.0, X2, -2.0, X3, eps=eps))
            self.X2.append(X2)
            self.X3.append(X3)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._issue()

    def _issue(self):
        for k in range(self.steps):
            X = self.X[k]
            bsm.multiply(1.0, X, X, Cm=self.X2[k], eps=self.eps, prec=self.prec, build_stacks=False, no_sync=True)
            bsm.multiply(1.0, self.X2[k], X, Cm=self.X3[k], eps=self.eps, prec=self.prec, build_stacks=False,
                         no_sync=True)
            bsm.add(3.0, self.X2[k], -2.0, self.X3[k], Z=self.X[k + 1], eps=self.eps, no_sync=True)

    def replay(self):
        self.graph.replay()

    @property
    def result(self) -> bsm.Matrix:
        return self.X[-1]

    def status(self) -> int:
        """OR of the device status words of every handle the graph writes."""
        s = 0
        for h in self.X2 + self.X3 + self.X[1:]:
            s |= bsm.bsm_get_status(h.h)
        return s
