"""Many slices of uneven sizes (Section 7 batches slices "to fill up the GPU memory").

Slices are grouped by size.  Each group runs as same-size batches of at most the plan's batch
capacity (one set of launches per transform and batch: radon_forward_batch /
radon_backproject_batch), and the whole multi-size sequence can be captured once in a CUDA graph
and replayed.  `tune()` picks, per plan, the slices per batched call and the theta-convolution
kernel by timing; neither changes results beyond FP32 rounding.
"""

from __future__ import annotations

import collections

import torch

from . import binding


class UnevenBatch:
    def __init__(self, sizes, n_angles_of=lambda n: n, n_det_of=lambda n: 3 * n // 2, interp_order: int = 3,
                 n_partitions: int = 3, max_batch: int = 16):
        self.sizes = [int(n) for n in sizes]
        self.groups = collections.OrderedDict()  # N -> list of slice indices
        for i, n in enumerate(self.sizes):
            self.groups.setdefault(n, []).append(i)
        self.plans, self.images, self.sinos, self.chunk = {}, {}, {}, {}
        for n, idx in self.groups.items():
            plan = binding.radon_plan_create(n, n_angles_of(n), n_det_of(n), interp_order, n_partitions)
            cap = min(len(idx), max_batch)
            while cap > 1:
                try:
                    binding.radon_plan_reserve_batch(plan, cap)
                    break
                except binding.RadonError:
                    cap //= 2
            self.plans[n] = plan
            self.chunk[n] = cap
            self.images[n] = torch.zeros((len(idx),) + plan.image_shape, device="cuda")
            self.sinos[n] = torch.zeros((len(idx),) + plan.sino_shape, device="cuda")
        self.graph = None

    # ---------------------------------------------------------------- data in / out
    def set_images(self, images):
        for n, idx in self.groups.items():
            for j, i in enumerate(idx):
                self.images[n][j].copy_(images[i])

    def set_sinograms(self, sinos):
        for n, idx in self.groups.items():
            for j, i in enumerate(idx):
                self.sinos[n][j].copy_(sinos[i])

    def image(self, i):
        n = self.sizes[i]
        return self.images[n][self.groups[n].index(i)]

    def sinogram(self, i):
        n = self.sizes[i]
        return self.sinos[n][self.groups[n].index(i)]

    # ---------------------------------------------------------------- transforms
    def forward(self):
        for n, plan in self.plans.items():
            c = self.chunk[n]
            for s in range(0, len(self.groups[n]), c):
                binding.radon_forward_batch(plan, self.images[n][s:s + c], self.sinos[n][s:s + c])

    def backproject(self):
        for n, plan in self.plans.items():
            c = self.chunk[n]
            for s in range(0, len(self.groups[n]), c):
                binding.radon_backproject_batch(plan, self.sinos[n][s:s + c], self.images[n][s:s + c])

    def capture(self, fn=None):
        """Capture fn (default: forward then backproject) in a CUDA graph; replay() runs it."""
        fn = fn or (lambda: (self.forward(), self.backproject()))
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            fn()
        torch.cuda.current_stream().wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            fn()
        return self.graph

    def replay(self):
        self.graph.replay()

    # ---------------------------------------------------------------- autotuning
    def _time_group(self, n, repeats):
        """Milliseconds of `repeats` passes of R then R# over group n with its current chunk."""
        self._run_group(n)
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record()
        for _ in range(repeats):
            self._run_group(n)
        stop.record()
        torch.cuda.synchronize()
        return start.elapsed_time(stop)

    def _run_group(self, n):
        plan, c = self.plans[n], self.chunk[n]
        for s in range(0, len(self.groups[n]), c):
            binding.radon_forward_batch(plan, self.images[n][s:s + c], self.sinos[n][s:s + c])
        for s in range(0, len(self.groups[n]), c):
            binding.radon_backproject_batch(plan, self.sinos[n][s:s + c], self.images[n][s:s + c])

    def tune(self, groups=(0, 1, 2, 4), chunks=(1, 2, 4, 8, 16), repeats: int = 2):
        """Per size group, choose the slices per batched call (up to the reserved capacity), then
        the theta-convolution kernel, by timing R then R# over the whole group.  Neither choice
        changes results beyond FP32 rounding of the theta kernel (chunking changes nothing).
        Uses (and overwrites) the group buffers: set the inputs afterwards.  Returns
        {N: (chunk, column group)}."""
        choice = {}
        for n, plan in self.plans.items():
            cap = self.chunk[n]
            best = None
            for c in sorted({min(c, cap) for c in chunks}):
                self.chunk[n] = c
                t = self._time_group(n, repeats)
                if best is None or t < best[0]:
                    best = (t, c)
            self.chunk[n] = best[1]
            best = None
            for g in groups:
                try:
                    binding.radon_plan_set_column_group(plan, g)
                except binding.RadonError:
                    continue
                t = self._time_group(n, repeats)
                if best is None or t < best[0]:
                    best = (t, g)
            binding.radon_plan_set_column_group(plan, best[1])
            choice[n] = (self.chunk[n], best[1])
        return choice
