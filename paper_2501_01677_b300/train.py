"""Densification-free parallel group training (Sec. 5.1: the building groups are
optimised independently and in parallel; 30k iterations per group).

A GroupTrainer holds the Gaussians of several sub-regions (groups) in one set of
parameter tensors, each group with its own views.  View slot j of the trainer is
the j-th view of every group; one iteration renders one slot -- one view per
group, all groups batched in one plan -- and applies Adam to every parameter.
Each slot's iteration is captured once as a CUDA graph (render step + one fused
multi-tensor Adam launch whose step count lives in device memory) and replayed
for every later iteration on that slot; the slots are visited in a fresh random
order every epoch (the per-iteration view sampling of 3DGS training).  All work
runs in libpgsag's kernels; the host only picks the slot and replays.
"""
from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import _lib as L
from . import raster

# 3DGS learning rates by parameter tensor (means, log-scales, quaternions,
# opacity logits, SH); the paper does not list its own
DEFAULT_LRS = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class GroupTrainer:
    """Training state of a set of groups.

    views_by_group[s] lists group s's views (objects with cam, mask, target);
    ranges[s] = (begin, end) of group s's Gaussians in P.  Groups may have
    different numbers of views: slot j uses view j mod len(views) of each group."""

    def __init__(self, P: raster.GaussianParams, views_by_group: Sequence[Sequence], ranges: Sequence[Tuple[int, int]],
                 lrs: Sequence[float] = DEFAULT_LRS, tile=(16, 16), persistent: bool = True, lpt: bool = False,
                 betas=(0.9, 0.999), eps: float = 1e-15, objective: str = "pg"):
        self.P = P
        self.lib = L.load()
        self.n_slots = max(len(v) for v in views_by_group)
        self.plans: List[raster.Plan] = []
        for j in range(self.n_slots):
            vs = [group[j % len(group)] for group in views_by_group]
            plan = raster.Plan([v.cam for v in vs], [v.mask for v in vs], [v.target for v in vs], P.n,
                               g_ranges=list(ranges), tile=tile)
            plan.set_objective(objective)
            plan.forward(P)  # sizes the duplicate capacity
            if persistent:
                plan.use_persistent_schedule(ctas_per_sm=0, lpt=lpt)
            self.plans.append(plan)
        self.grads = raster.new_param_grads(P)
        self.m = [torch.zeros_like(t) for t in P.tensors()]
        self.v = [torch.zeros_like(t) for t in P.tensors()]
        self.step_dev = torch.zeros(4, dtype=torch.int32, device=P.means.device)
        self.status = torch.zeros(1, dtype=torch.int32, device=P.means.device)
        self.betas, self.eps = betas, eps
        self.table = (L.PgsagAdamTensor * 5)()
        for k, (p, g, mm, vv, lr) in enumerate(zip(P.tensors(), self.grads, self.m, self.v, lrs)):
            self.table[k] = L.PgsagAdamTensor(p.data_ptr(), g.data_ptr(), mm.data_ptr(), vv.data_ptr(), p.numel(),
                                              float(lr), 0)
        self.loss_buf = [torch.zeros(3 * pl.n_views + 1, dtype=torch.float32, device=P.means.device)
                         for pl in self.plans]
        self.graphs: List[Optional[torch.cuda.CUDAGraph]] = [None] * self.n_slots
        self.iterations = 0

    # ------------------------------------------------------------------ one iteration
    def _adam(self, stream=None):
        s = raster._stream_ptr(stream)
        L.check(self.lib.pgsag_adam_multi(5, self.table, float(self.betas[0]), float(self.betas[1]), float(self.eps),
                                          _ptr(self.step_dev), _ptr(self.status), s), "pgsag_adam_multi")

    def _body(self, j: int, stream=None):
        self.plans[j].step(self.P, self.grads, loss_out=self.loss_buf[j], stream=stream)
        self._adam(stream)

    def iteration(self, j: int):
        """One training iteration on view slot j: the first one on a slot runs
        eagerly (on a side stream) and then captures the slot's graph; later ones
        replay it."""
        if self.graphs[j] is None:
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                self._body(j, side)
            torch.cuda.current_stream().wait_stream(side)
            torch.cuda.synchronize()
            self.plans[j].check_status()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                self._body(j)
            self.graphs[j] = graph
        else:
            self.graphs[j].replay()
        self.iterations += 1
        return self.loss_buf[j]

    def eager_iteration(self, j: int):
        """The same iteration without graphs (for checks)."""
        self._body(j)
        self.iterations += 1
        return self.loss_buf[j]

    def schedule(self, n_iters: int, seed: int = 0) -> List[int]:
        """Slot order: a fresh random permutation of the slots every epoch."""
        rng = np.random.default_rng(seed)
        order: List[int] = []
        while len(order) < n_iters:
            order.extend(int(x) for x in rng.permutation(self.n_slots))
        return order[:n_iters]

    def run(self, n_iters: int, seed: int = 0, record_losses: bool = True) -> torch.Tensor:
        """n_iters iterations; returns the total loss of each iteration (device
        float32 [n_iters], copied on the device after each iteration, no host
        synchronisation inside the loop)."""
        losses = torch.zeros(n_iters, dtype=torch.float32, device=self.P.means.device)
        for i, j in enumerate(self.schedule(n_iters, seed + self.iterations)):
            lb = self.iteration(j)
            if record_losses:
                losses[i:i + 1].copy_(lb[-1:])
        return losses

    # ------------------------------------------------------------------ checkpoints
    def state_dict(self) -> dict:
        """Parameters, Adam moments and step count (device tensors cloned to host)."""
        return {"params": [t.detach().cpu().clone() for t in self.P.tensors()],
                "m": [t.cpu().clone() for t in self.m], "v": [t.cpu().clone() for t in self.v],
                "step": self.step_dev.cpu().clone(), "iterations": self.iterations}

    def load_state_dict(self, sd: dict) -> None:
        """Restore into the existing device buffers (the captured graphs stay valid)."""
        with torch.no_grad():
            for dst, src in zip(self.P.tensors(), sd["params"]):
                dst.copy_(src)
            for dst, src in zip(self.m, sd["m"]):
                dst.copy_(src)
            for dst, src in zip(self.v, sd["v"]):
                dst.copy_(src)
            self.step_dev.copy_(sd["step"])
        self.iterations = int(sd["iterations"])

    def save(self, path: str) -> None:
        torch.save(self.state_dict(), path)

    def load(self, path: str) -> None:
        self.load_state_dict(torch.load(path, weights_only=True))

    def check_status(self):
        for pl in self.plans:
            pl.check_status()
        st = int(self.status.item())
        if st:
            raise L.PgsagError(f"device status {st} in the optimiser")

    def mask_pixels_per_iteration(self) -> float:
        return float(np.mean([pl.n_mask for pl in self.plans]))

    def launches_per_iteration(self) -> float:
        return float(np.mean([pl.kernel_launches_per_step() for pl in self.plans])) + 2
