"""Many slices of uneven sizes (Section 7 batches slices "to fill up the GPU memory").

Slices are grouped by size.  Each group runs as same-size batches of at most the plan's batch
capacity (one set of launches per transform and batch: radon_forward_batch /
radon_backproject_batch), and the whole multi-size sequence can be captured once in a CUDA graph
and replayed.  `tune()` picks, per size, the slices per batched call and the theta-convolution
kernel by timing (neither changes results beyond FP32 rounding) and, when several partition
counts M are offered, the fastest M.  M sets the log-polar lattice (Section 2: beta = pi / M, the
radial factor a_R, N_rho, n_theta), so a different M gives a different discretisation of the same
transforms, each as accurate as the method (the tests compare every M against the oracle at that
M); at M = 4 the angular FFT length is a power of two for N = n_angles in 256 ... 4096.
"""

from __future__ import annotations

import collections

import torch

from . import binding


class UnevenBatch:
    def __init__(self, sizes, n_angles_of=lambda n: n, n_det_of=lambda n: 3 * n // 2, interp_order: int = 3,
                 n_partitions=3, max_batch: int = 16):
        """``n_partitions``: M for every size, or a sequence of candidate M values from which
        ``tune()`` picks per size (the first one is used until then)."""
        self.sizes = [int(n) for n in sizes]
        self.groups = collections.OrderedDict()  # N -> list of slice indices
        for i, n in enumerate(self.sizes):
            self.groups.setdefault(n, []).append(i)
        self.partition_candidates = tuple(n_partitions) if hasattr(n_partitions, "__iter__") else (int(n_partitions),)
        self._geom = (n_angles_of, n_det_of, interp_order, max_batch)
        self.plans, self.images, self.sinos, self.chunk = {}, {}, {}, {}
        for n, idx in self.groups.items():
            plan = self._make_plan(n, self.partition_candidates[0])
            self.plans[n] = plan
            self.images[n] = torch.zeros((len(idx),) + plan.image_shape, device="cuda")
            self.sinos[n] = torch.zeros((len(idx),) + plan.sino_shape, device="cuda")
        self.graph = None

    def _make_plan(self, n, M):
        """Plan for size n with M partitions, batch capacity reserved (halved until it fits)."""
        n_angles_of, n_det_of, interp_order, max_batch = self._geom
        plan = binding.radon_plan_create(n, n_angles_of(n), n_det_of(n), interp_order, M)
        cap = min(len(self.groups[n]), max_batch)
        while cap > 1:
            try:
                binding.radon_plan_reserve_batch(plan, cap)
                break
            except binding.RadonError:
                cap //= 2
        self.chunk[n] = cap
        return plan

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
        """Per size group and candidate M, choose the slices per batched call (up to the reserved
        capacity), then the theta-convolution kernel, by timing R then R# over the whole group;
        then keep the fastest M.  Chunking changes nothing and the theta kernel only FP32
        rounding; M changes the discretisation (see the module docstring).  Uses (and
        overwrites) the group buffers: set the inputs afterwards, and capture after tuning.
        Returns {N: (chunk, column group, M)}."""
        choice = {}
        for n in self.plans:
            best_m = None
            for M in self.partition_candidates:
                plan = self.plans[n] if self.plans[n].info["n_partitions"] == M else self._make_plan(n, M)
                self.plans[n] = plan
                chunk, group, t = self._tune_plan(n, plan, groups, chunks, repeats)
                if best_m is None or t < best_m[0]:
                    best_m = (t, plan, chunk, group, M)
            _, plan, chunk, group, M = best_m
            self.plans[n] = plan
            self.chunk[n] = chunk
            binding.radon_plan_set_column_group(plan, group)
            choice[n] = (chunk, group, M)
        self.graph = None
        return choice

    def _tune_plan(self, n, plan, groups, chunks, repeats):
        cap = plan.max_batch if plan.max_batch > 1 else 1
        best = None
        for c in sorted({min(c, cap) for c in chunks}):
            self.chunk[n] = c
            t = self._time_group(n, repeats)
            if best is None or t < best[0]:
                best = (t, c)
        self.chunk[n] = best[1]
        best_g = None
        for g in groups:
            try:
                binding.radon_plan_set_column_group(plan, g)
            except binding.RadonError:
                continue
            t = self._time_group(n, repeats)
            if best_g is None or t < best_g[0]:
                best_g = (t, g)
        binding.radon_plan_set_column_group(plan, best_g[1])
        return self.chunk[n], best_g[1], best_g[0]
