"""Benchmark: log-polar Radon transform R + back-projection R# at N = 2048 on GB300.

One step = one forward transform R (image -> sinogram) plus one back-projection R#
(sinogram -> image) of the 2048 x 2048 / 2048-angle / 3072-bin workload, cubic B-splines,
M = 3 partitions, FP32, inputs resident in HBM.  The L2 cache is flushed (a 256 MB write)
before every timed step, outside the timed interval.  Under torchrun every rank runs the same
per-GPU work on its own slices (weak scaling, no collective in the data path).

``--impl reference`` times the FP64 CPU oracle (the reference arm of this build) on the host
cores, on a bounded sample of the same workload.

Prints one JSON line (rank 0).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Radon+back-projection samples/sec and % HBM roofline at N=2048, err vs FP64 oracle"
UNIT = "samples/s"
N, N_ANGLES, N_DET, INTERP, M = 2048, 2048, 3072, 3, 3
WORKLOAD = "radon_pair_N2048_A2048_D3072_cubic_M3"
L2_FLUSH_BYTES = 256 << 20


def _config():
    return {
        "workload": WORKLOAD,
        "N": N, "n_angles": N_ANGLES, "n_det": N_DET, "interp_order": INTERP, "n_partitions": M,
        "step": "one R (image->sinogram) + one R# (sinogram->image) of independent inputs",
        "phantom": "50 random ellipses, seed 2; sinogram i.i.d. N(0,1), seed 3",
        "l2": "flushed before each timed step (256 MB write, outside the timed interval)",
    }


def _samples_per_step():
    return N_ANGLES * N_DET + N * N


# ---------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------- roofline model

def stage_bytes(info):
    """Algorithmic DRAM bytes per launch of each stage (unique bytes a stage must move)."""
    n, na, nd, mm = info["N"], info["n_angles"], info["n_det"], info["n_partitions"]
    nh, nr = info["n_theta_half"], info["N_rho"]
    nc1 = nr // 2 + 1
    spec_in = mm * nh * nc1 * 8          # half spectrum of the sampled rows
    spec_out = mm * (nh + 4) * nc1 * 8   # kept rows after the theta convolution
    ylp = mm * (nh + 4) * nr * 4         # log-polar coefficients
    kern = (info["n_theta"] // 2 + 1) * nc1 * 8
    img = 4 * n * n
    sino = 4 * na * nd
    disc = 4 * math.pi / 4 * n * n       # coefficient pixels inside the disc (read once per launch)
    lp_rows = mm * nh * nr * 4           # sampled real log-polar rows
    return {
        "prefilter_image": 2 * img,
        "sample_fwd": disc + lp_rows,
        "rows_fwd": lp_rows + spec_in,
        "columns_fwd": spec_in + kern + spec_out,
        "rows_inv_fwd": spec_out + ylp,
        "gather_sino": ylp + sino,
        "prefilter_sino": 2 * sino,
        "rows_bp": sino + spec_in,
        "columns_bp": spec_in + kern + spec_out,
        "rows_inv_bp": spec_out + ylp,
        "gather_image": ylp + img,
    }


def sample_fwd_fine_samples(info) -> int:
    """Fine samples the forward sampling reads (cubic: 16 taps each): per partition m, angular row
    jj and sub-angle q, the rho indices whose 4 x 4 tap block lies inside the padded coefficient
    array and within 16 + 1.5 pixels of the disc (the rule the plan's sampling ranges follow)."""
    import numpy as np

    n, mm, nh, r, nr = info["N"], info["n_partitions"], info["n_theta_half"], info["r"], info["N_rho"]
    a_R, beta, d_phi, d_rho = info["a_R"], info["beta"], info["d_phi"], info["d_rho"]
    pad, margin = 3, 16
    S = n / (2.0 * a_R)
    P = n + 2.0 * pad
    lo_b, hi_b = 1.0 + 1e-3, P - 2.0 - 1e-3
    cz, Rd = pad + n / 2.0, n / 2.0 + margin + 1.5
    jj = np.arange(nh)[:, None]
    q = np.arange(r)[None, :]
    total = 0
    for m in range(mm):
        C0 = n / 2.0 - (1.0 - a_R) * math.cos(m * beta) * S + pad
        R0 = n / 2.0 - (1.0 - a_R) * math.sin(m * beta) * S + pad
        phi = (jj + nh // 2 - nh) * d_phi + (q - 0.5 * (r - 1)) * d_phi / r
        Cv, Rv = np.cos(phi + m * beta) * S, np.sin(phi + m * beta) * S
        tl = np.zeros_like(Cv)
        th = np.full_like(Cv, 1e300)
        for x0, v in ((C0, Cv), (R0, Rv)):
            with np.errstate(divide="ignore", invalid="ignore"):
                a, b = (lo_b - x0) / v, (hi_b - x0) / v
            ok = v != 0.0
            tl = np.where(ok, np.maximum(tl, np.minimum(a, b)), tl)
            th = np.where(ok, np.minimum(th, np.maximum(a, b)), np.where((x0 < lo_b) | (x0 > hi_b), -1.0, th))
        dx, dy = C0 - cz, R0 - cz
        A = Cv * Cv + Rv * Rv
        B = 2.0 * (dx * Cv + dy * Rv)
        Cq = dx * dx + dy * dy - Rd * Rd
        disc = B * B - 4.0 * A * Cq
        sq = np.sqrt(np.maximum(disc, 0.0))
        tl = np.maximum(tl, (-B - sq) / (2.0 * A))
        th = np.where(disc < 0.0, -1.0, np.minimum(th, (-B + sq) / (2.0 * A)))
        live = (th > tl) & (th > 0.0)
        with np.errstate(divide="ignore", invalid="ignore"):
            il = np.where(tl > 0.0, np.log(np.where(tl > 0.0, tl, 1.0)) / d_rho + nr - 1, -1.0)
            ih = np.log(np.where(th > 0.0, th, 1.0)) / d_rho + nr - 1
        ilo = np.maximum(0.0, np.ceil(il))
        ihi = np.minimum(nr - 1.0, np.floor(ih))
        cnt = np.where(live & (ihi >= ilo), ihi - ilo + 1, 0.0)
        total += int(cnt.sum())
    return total


def live_bin_count(n_det: int) -> int:
    """Detector bins with |s| < 1 (exact integer test 2 (2k - n_det)^2 < n_det^2)."""
    return sum(1 for k in range(n_det) if 2 * (2 * k - n_det) ** 2 < n_det * n_det)


def pair_bytes(info) -> dict:
    """Algorithmic bytes of one R and one R# with the log-polar convolution fused:
    B_R  = 4 N^2 + 4 n_angles n_det + 4 S_c + |K|
    B_R# = 4 n_angles n_live + 4 N^2 + 4 S_c + |K|
    where S_c = M n_theta_half (N_rho/2 + 1) 8 is the half spectrum of the kept theta rows (written
    and read twice per transform: between the rho pass and the theta pass, and between the theta
    pass and the inverse rho pass), |K| = (n_theta/2 + 1)(N_rho/2 + 1) 8 the kernel table read once,
    and n_live the detector bins with |s| < 1 (the only ones R# reads)."""
    n, na, nd, mm = info["N"], info["n_angles"], info["n_det"], info["n_partitions"]
    nh, nr, nt = info["n_theta_half"], info["N_rho"], info["n_theta"]
    S_c = mm * nh * (nr // 2 + 1) * 8
    K = (nt // 2 + 1) * (nr // 2 + 1) * 8
    B_R = 4 * n * n + 4 * na * nd + 4 * S_c + K
    B_B = 4 * na * live_bin_count(nd) + 4 * n * n + 4 * S_c + K
    return {"R": B_R, "R#": B_B, "pair": B_R + B_B, "S_c": S_c, "K": K}


def _event_ms(torch, fn, reps: int, flush=None) -> float:
    """Median CUDA-event time of fn() over reps runs on the current stream (L2 flushed before each)."""
    import statistics

    times = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


def closed_form_errors(rl, torch, plan) -> dict:
    """R of sampled Gaussians against their analytic Radon transform and R# of that analytic
    sinogram against its closed-form back-projection, through ``plan`` (sizes the oracle cannot
    finish in seconds)."""
    import numpy as np

    from oracle import direct, geometry
    from workloads import gaussian_image

    info = plan.info
    n, na, nd = info["N"], info["n_angles"], info["n_det"]
    geo = geometry.make_geometry(n, na, nd, info["n_partitions"], info["interp_order"])
    blobs = [(0.2, -0.1, 0.12, 1.0), (-0.3, 0.25, 0.08, -0.7), (0.05, 0.5, 0.1, 0.4)]
    th = np.arange(na) * geo.dtheta
    s = (np.arange(nd) - nd / 2) * geo.ds
    sino = direct.gaussian_radon(th[:, None], s[None, :], blobs)
    sino[:, ~geometry.live_bins(nd)] = 0.0
    x = (np.arange(n) - n / 2) * (2.0 / n)
    bp = np.zeros((n, n))
    for cx, cy, sg, w in blobs:
        bp += w * math.sqrt(2 * math.pi) * sg * direct.gaussian_bp(np.hypot(x[None, :] - cx, x[:, None] - cy), sg)
    bp[~geometry.disc_mask(n)] = 0.0
    f = torch.from_numpy(gaussian_image(n, blobs).astype(np.float32)).cuda()
    g = torch.from_numpy(sino.astype(np.float32)).cuda()
    Rf = torch.empty((na, nd), device="cuda")
    Bg = torch.empty((n, n), device="cuda")
    rl.radon_forward(plan, f, Rf)
    rl.radon_backproject(plan, g, Bg)
    torch.cuda.synchronize()
    return {"R": rel_l2(Rf.cpu().numpy(), sino), "R#": rel_l2(Bg.cpu().numpy(), bp),
            "reference": "closed forms: analytic Radon transform of 3 Gaussians and its back-projection "
                         "pi sqrt(2 pi) s e^-u I0(u)", "metric": "relative L2"}


def oracle_errors(rl, torch, plan, seed: int = 11) -> dict:
    """R of a seeded smooth image and R# of a seeded N(0, 1) sinogram through ``plan`` against the
    FP64 log-polar oracle on the same FP32 inputs (whole outputs)."""
    import numpy as np

    from oracle import geometry, logpolar
    from workloads import random_sinogram, smooth_random_image

    info = plan.info
    n, na, nd = info["N"], info["n_angles"], info["n_det"]
    geo = geometry.make_geometry(n, na, nd, info["n_partitions"], info["interp_order"])
    f = smooth_random_image(n, seed).astype(np.float32)
    g = random_sinogram(na, nd, seed + 1).astype(np.float32)
    Rf = torch.empty((na, nd), device="cuda")
    Bg = torch.empty((n, n), device="cuda")
    rl.radon_forward(plan, torch.from_numpy(f).cuda(), Rf)
    rl.radon_backproject(plan, torch.from_numpy(g).cuda(), Bg)
    torch.cuda.synchronize()
    return {"R": rel_l2(Rf.cpu().numpy(), logpolar.forward(f.astype(np.float64), geo)),
            "R#": rel_l2(Bg.cpu().numpy(), logpolar.backproject(g.astype(np.float64), geo)),
            "tolerance": 1e-5, "metric": "relative L2",
            "inputs": f"smooth random image (seed {seed}), N(0,1) sinogram (seed {seed + 1}), this plan's geometry"}


def bench_batched(rl, torch, flush, with_oracle: bool = True) -> dict:
    """96 slices of uneven N drawn from {256, 512, 1024, 2048, 4096} (seed 4), n_angles = N,
    n_det = 1.5 N: per-slice calls versus same-size batches replayed from one CUDA graph.  One
    pass = R of every image, then R# of every sinogram.  Inputs are seeded uniform images; the
    kernels' work does not depend on the values."""
    from paper_1506_00014_gb300.batch import UnevenBatch
    from workloads import slice_sizes

    sizes = slice_sizes(96, 4)
    ub = UnevenBatch(sizes, max_batch=16, n_partitions=(3, 4))
    gen = torch.Generator(device="cuda")
    for i, n in enumerate(sizes):
        gen.manual_seed(100 + i)
        ub.image(i).copy_(torch.rand((n, n), device="cuda", generator=gen))

    def per_slice():
        for n, idx in ub.groups.items():
            plan = ub.plans[n]
            for j in range(len(idx)):
                rl.radon_forward(plan, ub.images[n][j], ub.sinos[n][j])
        for n, idx in ub.groups.items():
            plan = ub.plans[n]
            for j in range(len(idx)):
                rl.radon_backproject(plan, ub.sinos[n][j], ub.images[n][j])

    per_slice()
    t_slice = _event_ms(torch, per_slice, 3, flush)
    choice = ub.tune()  # slices per batched call, theta kernel and partition count, per size group
    per_slice()
    t_slice_tuned = _event_ms(torch, per_slice, 3, flush)  # per-slice calls of the tuned plans
    ub.capture()
    ub.replay()
    t_graph = _event_ms(torch, ub.replay, 3, flush)
    samples = sum(n * n + n * (3 * n // 2) for n in sizes)

    # accuracy: fresh seeded inputs and one replay; the first slice of each size is compared with
    # per-slice calls of its plan (bit for bit) and with the FP64 oracle
    import numpy as np

    from oracle import geometry, logpolar

    for i, n in enumerate(sizes):
        gen.manual_seed(100 + i)
        ub.image(i).copy_(torch.rand((n, n), device="cuda", generator=gen))
    firsts = {n: idx[0] for n, idx in ub.groups.items()}
    f0 = {n: ub.image(i).clone() for n, i in firsts.items()}
    ub.replay()
    torch.cuda.synchronize()
    accuracy = {}
    for n, i in firsts.items():
        plan = ub.plans[n]
        s1 = torch.empty(plan.sino_shape, device="cuda")
        b1 = torch.empty(plan.image_shape, device="cuda")
        rl.radon_forward(plan, f0[n], s1)
        rl.radon_backproject(plan, ub.sinogram(i), b1)
        torch.cuda.synchronize()
        entry = {"slice": i, "batched_equals_per_slice": bool(torch.equal(s1, ub.sinogram(i)) and
                                                              torch.equal(b1, ub.image(i)))}
        if with_oracle and n <= 1024:
            geo = geometry.make_geometry(n, n, 3 * n // 2, plan.info["n_partitions"], 3)
            ref_s = logpolar.forward(f0[n].cpu().numpy().astype(np.float64), geo)
            ref_b = logpolar.backproject(ub.sinogram(i).cpu().numpy().astype(np.float64), geo)
            entry["err_vs_oracle"] = {"R": rel_l2(ub.sinogram(i).cpu().numpy(), ref_s),
                                      "R#": rel_l2(ub.image(i).cpu().numpy(), ref_b), "tolerance": 1e-5,
                                      "oracle": "FP64 log-polar oracle, this slice's inputs", "metric": "relative L2"}
        elif with_oracle:
            entry["err_vs_closed_form"] = closed_form_errors(rl, torch, plan)
        accuracy[str(n)] = entry
    return {
        "slices": len(sizes), "sizes": {str(n): len(v) for n, v in ub.groups.items()},
        "per_slice_ms": t_slice, "per_slice_tuned_plans_ms": t_slice_tuned, "batched_graph_ms": t_graph,
        "speedup": t_slice / t_graph,
        "baseline": "per_slice_ms: one call per slice and transform, M = 3, default theta kernel",
        "tuned": {str(n): {"slices_per_call": c, "column_group": g, "n_partitions": m}
                  for n, (c, g, m) in choice.items()},
        "batched_samples_per_s": samples / (t_graph / 1e3), "unit": UNIT,
        "accuracy": accuracy,
    }


def bench_least_squares(rl, torch, with_oracle: bool = True) -> dict:
    """64 slices, N = 1024, 720 angles, 1536 bins; data = analytic ellipse line integrals plus
    Gaussian noise at 1 % of the maximum (seeds 200 + i); 50 gradient steps of ||R f - g||^2:
    the per-slice eager loop versus the batched autograd loop (backward = R#) replayed from a CUDA
    graph."""
    import numpy as np

    from paper_1506_00014_gb300.recon import BatchedLeastSquares, LeastSquares, normal_operator_norm
    from workloads import ellipse_sinogram, random_ellipses

    n, na, nd, slices, steps = 1024, 720, 1536, 64, 50
    plan = rl.radon_plan_create(n, na, nd, 3, 3)
    g = []
    for sl in range(slices):
        s = ellipse_sinogram(random_ellipses(10, 200 + sl), na, nd)
        s = s + np.random.default_rng(200 + sl).normal(0.0, 0.01 * np.abs(s).max(), s.shape)
        g.append(s.astype(np.float32))
    g = torch.from_numpy(np.stack(g)).cuda()
    step = 1.0 / (2.0 * normal_operator_norm(plan))

    def per_slice():
        return [LeastSquares(plan, g[b], step=step).run(steps) for b in range(slices)]

    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    per_slice()  # warm-up
    torch.cuda.synchronize()
    t0.record()
    ref = per_slice()
    t1.record()
    torch.cuda.synchronize()
    t_slice = t0.elapsed_time(t1)
    rl.radon_plan_reserve_batch(plan, 16)
    bl = BatchedLeastSquares(plan, g, step=step, use_graph=True)  # autograd's gradient is 2 c_R R#(R f - g)
    torch.cuda.synchronize()
    t0.record()
    got = bl.run(steps)
    t1.record()
    torch.cuda.synchronize()
    t_batch = t0.elapsed_time(t1)
    ref = torch.stack(ref)
    diff = float((got - ref).norm() / ref.norm())
    loss0 = float((g * g).sum())
    out = {
        "slices": slices, "N": n, "n_angles": na, "n_det": nd, "steps": steps,
        "per_slice_eager_ms": t_slice, "batched_autograd_graph_ms": t_batch, "speedup": t_slice / t_batch,
        "rel_diff_batched_vs_per_slice": diff, "loss_ratio_final_over_initial": float(bl.losses().sum()) / loss0,
    }
    if with_oracle:
        out["err_vs_oracle"] = oracle_errors(rl, torch, plan)
    return out


def bench_fbp_large(rl, torch, flush, with_oracle: bool = True) -> dict:
    """FBP at N = 8192 with 8192 angles x 12288 bins, Shepp-Logan window, then R#.  The sinogram is
    the analytic line integrals of 200 random ellipses (seed 5) plus Gaussian noise with sigma =
    0.5 % of its maximum (seed 5).  Accuracy: against the phantom itself (closed form: 4 x 4
    sub-pixel coverage at 4096 seeded pixels of the disc), and against the direct oracle (the FP64
    filter of the same noisy sinogram, then the rectangle rule over the 8192 angles with cubic
    interpolation in s) at 256 of those pixels."""
    import numpy as np

    from workloads import ellipse_sinogram_torch, ellipse_values_at, random_ellipses

    n, na, nd = 8192, 8192, 12288
    ell = random_ellipses(200, 5)
    g64 = ellipse_sinogram_torch(ell, na, nd, "cuda")
    sigma = 0.005 * float(g64.abs().max())
    noise = torch.from_numpy(np.random.default_rng(5).standard_normal((na, nd), dtype=np.float32)).cuda()
    g = (g64 + sigma * noise.double()).float()
    g_clean = g64.float()
    del g64, noise
    plan = rl.radon_plan_create(n, na, nd, 3, 3)
    img = torch.empty((n, n), device="cuda")
    fn = lambda: rl.radon_fbp(plan, g, img, rl.RADON_FILTER_SHEPP_LOGAN)  # noqa: E731
    for _ in range(2):
        fn()
    t = _event_ms(torch, fn, 5, flush)
    fn()
    torch.cuda.synchronize()
    out = {"N": n, "n_angles": na, "n_det": nd, "filter": "shepp-logan", "ms_per_fbp": t,
           "output_pixels_per_s": n * n / (t / 1e3),
           "data": "analytic sinogram of 200 random ellipses (seed 5) + N(0, (0.005 max)^2) noise (seed 5)"}
    rng = np.random.default_rng(6)
    v = 2 * np.arange(n) - n
    ii, jj = np.nonzero((v[:, None] ** 2 + v[None, :] ** 2) < n * n)
    sel = rng.choice(ii.size, 4096, replace=False)
    rows, cols = ii[sel], jj[sel]
    got = img.cpu().numpy()[rows, cols].astype(np.float64)
    truth = ellipse_values_at(ell, n, rows, cols)
    rl.radon_fbp(plan, g_clean, img, rl.RADON_FILTER_SHEPP_LOGAN)
    torch.cuda.synchronize()
    got_clean = img.cpu().numpy()[rows, cols].astype(np.float64)
    out["err_vs_phantom"] = {
        "noisy": rel_l2(got, truth), "noise_free": rel_l2(got_clean, truth), "metric": "relative L2",
        "sample": "4096 disc pixels (seed 6)",
        "note": "reconstruction error against the phantom itself: the noisy figure is dominated by the 0.5 % noise "
                "that the ramp amplifies; the noise-free one (same FBP of the analytic sinogram) by the ellipse edges"}
    if with_oracle:
        from oracle import direct, fbp, geometry

        geo = geometry.make_geometry(n, na, nd, 3, 3)
        k = 256
        out["err_vs_direct_sampled"] = {"metric": "relative L2", "sample": f"{k} of the pixels above",
                                        "oracle": "FP64 Shepp-Logan filter of the same sinogram, then the rectangle "
                                                  "rule over the angles (a different discretisation of R#)"}
        for name, sino, vals in (("noise_free", g_clean, got_clean), ("noisy", g, got)):
            gh = sino.cpu().numpy().astype(np.float64)
            Wg = np.empty_like(gh)
            for a0 in range(0, na, 512):
                Wg[a0:a0 + 512] = fbp.filter_sinogram(gh[a0:a0 + 512], geo, "shepp-logan")
            ref = direct.backproject_direct(Wg, geo, pixels=(rows[:k], cols[:k]))
            out["err_vs_direct_sampled"][name] = rel_l2(vals[:k], ref)
    del plan
    return out


def bench_exact_transpose(rl, torch, flush) -> dict:
    """R^T (radon_transpose, the exact transpose of the discrete R) on the headline workload
    (N = 2048, 2048 angles x 3072 bins, cubic, M = 3) beside R and R# of the same plan, each
    timed alone; plus R^T's per-stage split from the profiling events (a separate pass)."""
    plan = rl.radon_plan_create(N, N_ANGLES, N_DET, INTERP, M)
    gen = torch.Generator(device="cuda").manual_seed(7)
    g = torch.randn((N_ANGLES, N_DET), device="cuda", generator=gen)
    f = torch.rand((N, N), device="cuda", generator=gen)
    img = torch.empty((N, N), device="cuda")
    sino = torch.empty((N_ANGLES, N_DET), device="cuda")
    calls = {"R": lambda: rl.radon_forward(plan, f, sino), "R#": lambda: rl.radon_backproject(plan, g, img),
             "R^T": lambda: rl.radon_transpose(plan, g, img)}
    out = {}
    for name, fn in calls.items():
        for _ in range(3):
            fn()
        out["ms_" + name] = _event_ms(torch, fn, 20, flush)
    rl.radon_profile_enable(plan, True)
    rl.radon_profile_read(plan)
    for _ in range(5):
        calls["R^T"]()
    stages = rl.radon_profile_read(plan)
    rl.radon_profile_enable(plan, False)
    out["stage_ms_R^T"] = {k: round(ms / n, 4) for k, (ms, n) in stages.items() if n}
    calls["R"]()
    calls["R^T"]()
    torch.cuda.synchronize()
    lhs = float((sino.double() * g.double()).sum())
    rhs = float((f.double() * img.double()).sum())
    out["dot_product_identity"] = {
        "abs_diff_over_norms": abs(lhs - rhs) / float(sino.double().norm() * g.double().norm()),
        "identity": "<R f, g> = <f, R^T g> (plain sums), this workload; parity with the oracle's transpose is "
                    "tested at smaller sizes"}
    return out


def bench_em_volume(rl, torch, n: int = 256, iters: int = 100, with_oracle: bool = True) -> dict:
    """100 EM iterations (Section 8) on an n x n x n volume: n slices, 1.5 n angles, n bins,
    M = 3 (the paper's EM timing setup), data = analytic line integrals of non-negative random
    ellipses (32 phantoms, seeds 300 + i, repeated over the slices); everything stays on the GPU
    between upload and result."""
    import numpy as np

    from paper_1506_00014_gb300.recon import em_batched
    from workloads import ellipse_sinogram, random_ellipses

    na, nd = 3 * n // 2, n
    plan = rl.radon_plan_create(n, na, nd, 3, 3)
    rl.radon_plan_reserve_batch(plan, 64)
    distinct = min(n, 32)  # phantoms generated on the host; slice i uses phantom i % distinct
    base = []
    for sl in range(distinct):
        ell = [type(e)(e.cx, e.cy, e.a, e.b, e.psi, abs(e.density)) for e in random_ellipses(10, 300 + sl)]
        base.append(torch.from_numpy(ellipse_sinogram(ell, na, nd).astype(np.float32)).cuda())
    g = torch.stack([base[i % distinct] for i in range(n)])
    em_batched(plan, g[:2], 2)  # warm-up
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record()
    f = em_batched(plan, g, iters)
    t1.record()
    torch.cuda.synchronize()
    s = torch.empty_like(g)
    for b0 in range(0, n, 64):
        rl.radon_forward_batch(plan, f[b0:b0 + 64].contiguous(), s[b0:b0 + 64])
    resid = float(torch.linalg.norm(s - g) / torch.linalg.norm(g))
    out = {"volume": f"{n}^3", "slices": n, "n_angles": na, "n_det": nd, "iterations": iters,
           "seconds": t0.elapsed_time(t1) / 1e3, "relative_data_residual": resid,
           "paper_gtx770_seconds": {"256": 88.0, "512": 690.0, "1024": 5400.0, "2048": 42000.0}.get(str(n))}
    if with_oracle:
        out["err_vs_oracle"] = oracle_errors(rl, torch, plan)
    return out


def bench_paper_table1(rl, torch, flush, with_oracle: bool = True) -> dict:
    """R# per slice on the paper's own back-projection workload (Table 1): N x N images from
    1.5 N angles x N bins, M = 3, slices batched (the paper batched slices to fill GPU memory);
    the forward R on the same shapes beside it (the paper reports R only inside the EM loop).
    Seeded N(0, 1) sinograms; the work does not depend on the values."""
    paper = {256: 1.6e-3, 512: 6.1e-3, 1024: 2.5e-2, 2048: 9.9e-2}  # seconds, GTX 770
    out = {}
    for n, batch in ((256, 32), (512, 16), (1024, 8), (2048, 4)):
        na, nd = 3 * n // 2, n
        plan = rl.radon_plan_create(n, na, nd, 3, 3)
        rl.radon_plan_reserve_batch(plan, batch)
        gen = torch.Generator(device="cuda").manual_seed(7)
        g = torch.randn((batch, na, nd), device="cuda", generator=gen)
        img = torch.empty((batch, n, n), device="cuda")
        fn = lambda: rl.radon_backproject_batch(plan, g, img)  # noqa: E731
        fwd = lambda: rl.radon_forward_batch(plan, img, g)  # noqa: E731
        for _ in range(2):
            fn()
            fwd()
        t = _event_ms(torch, fn, 5, flush) / batch
        t_fwd = _event_ms(torch, fwd, 5, flush) / batch
        out[str(n)] = {"n_angles": na, "n_det": nd, "batch": batch, "ms_per_slice": t,
                       "paper_gtx770_ms_per_slice": 1e3 * paper[n], "forward_ms_per_slice": t_fwd}
        if with_oracle:
            out[str(n)]["err_vs_oracle" if n <= 1024 else "err_vs_closed_form"] = (
                oracle_errors(rl, torch, plan) if n <= 1024 else closed_form_errors(rl, torch, plan))
        del plan, g, img
    return out


KERNEL_SOURCES = ("radon_kernels.cu", "radon_kernels.cuh", "radon_fft.cuh")
NCU_SUMMARY = os.path.join(ROOT, "profiles", "dram_traffic_radon_pair_N2048.txt")


def kernel_sources_sha() -> str:
    """sha256 (first 16 hex digits) over the CUDA sources of the transform kernels."""
    import hashlib

    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1506_00014_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_summary(path: str = NCU_SUMMARY) -> tuple[dict, str | None, str | None]:
    """Per stage (DRAM bytes per launch, L1/TEX %, issue %, binding unit) from a committed ncu
    summary, with the kernel-source hash and commit it was captured at.  The figures are returned
    only while the kernels are unchanged since that capture (same source hash); else {}."""
    out, sha, commit = {}, None, None
    try:
        with open(path) as fh:
            for line in fh:
                if line.startswith("# kernel_sources_sha256:"):
                    sha = line.split(":", 1)[1].strip()
                elif line.startswith("# commit:"):
                    commit = line.split(":", 1)[1].strip()
                elif line.strip() and not line.startswith("#"):
                    parts = line.split()
                    if len(parts) == 5:
                        out[parts[0]] = (float(parts[1]), float(parts[2]), float(parts[3]), parts[4])
    except OSError:
        return {}, None, None
    if sha is None or sha != kernel_sources_sha():
        return {}, sha, commit
    return out, sha, commit


def reduce_max(value: float, dist, device) -> float:
    """Max over ranks of a per-rank scalar (identity without a process group)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_step: int, steps: int, max_seconds: float) -> float:
    """Units all ranks processed per second of the slowest rank (weak scaling)."""
    return world * units_per_step * steps / max_seconds


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------- our arm

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1506_00014_gb300 as rl
    from paper_1506_00014_gb300 import build as _build
    from workloads import ellipse_image, random_ellipses, random_sinogram

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    if _build.needs_build() and rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()

    plan = rl.radon_plan_create(N, N_ANGLES, N_DET, INTERP, M)
    info = plan.info
    launches_per_step = rl.radon_plan_kernel_launches(plan, "forward") + rl.radon_plan_kernel_launches(plan, "backproject")
    f = ellipse_image(N, random_ellipses(50, 2 + 1000 * rank)).astype(np.float32)
    g = random_sinogram(N_ANGLES, N_DET, 3 + 1000 * rank).astype(np.float32)
    f_d = torch.from_numpy(f).to(dev)
    g_d = torch.from_numpy(g).to(dev)
    sino_d = torch.empty((N_ANGLES, N_DET), dtype=torch.float32, device=dev)
    img_d = torch.empty((N, N), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    # R and R# of a step are independent: R runs on the current stream with `plan`, R# on a second
    # stream with its own plan (a plan's scratch serves one transform at a time)
    plan_bp = rl.radon_plan_create(N, N_ANGLES, N_DET, INTERP, M)
    side = torch.cuda.Stream(dev)

    def step():
        side.wait_stream(stream)
        rl.radon_forward(plan, f_d, sino_d, stream)
        rl.radon_backproject(plan_bp, g_d, img_d, side)
        stream.wait_stream(side)

    def step_serial():
        rl.radon_forward(plan, f_d, sino_d, stream)
        rl.radon_backproject(plan, g_d, img_d, stream)

    def timed(fn, steps):
        """Per-step CUDA events on the launching stream around fn only; the L2 flush sits between."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            fn()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev)

    for _ in range(args.warmup):
        flush.zero_()
        step()
        step_serial()
    torch.cuda.synchronize()

    # timed region (headline): the concurrent step, no profiling events
    clocks = ClockSampler(dev.index)
    clocks.start()
    if world > 1:
        dist.barrier()
    total_ms = reduce_max(timed(step, args.steps), dist if world > 1 else None, dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(world, _samples_per_step(), args.steps, total_ms / 1e3)
    n_aux = max(1, min(args.steps, 50))
    serial_ms = reduce_max(timed(step_serial, n_aux), dist if world > 1 else None, dev) / n_aux

    # per-kernel times: a separate serial pass with an event after every kernel launch
    rl.radon_profile_enable(plan, True)
    rl.radon_profile_read(plan)
    timed(step_serial, n_aux)
    stage = rl.radon_profile_read(plan)
    rl.radon_profile_enable(plan, False)

    # roofline of the dominant stage
    nbytes = stage_bytes(info)
    dom = max(stage, key=lambda k: stage[k][0])
    dom_ms = stage[dom][0] / max(1, stage[dom][1])
    peak, peak_kind = _peaks()
    achieved = nbytes[dom] / (dom_ms / 1e3) / 1e9
    stage_ms = {k: round(v[0] / v[1], 4) for k, v in stage.items() if v[1]}  # stages the pair launched
    ncu, ncu_sha, ncu_commit = ncu_summary()
    summary = ncu.get(dom)
    traffic = summary[0] if summary else None
    pb = pair_bytes(info)
    l1_roofline = None
    if dom == "sample_fwd" and INTERP == 3:
        # the binding unit's own roofline: the tap bytes the L1 data path must deliver to registers
        # (fine samples x 16 taps x 4 B) against n_SM x 128 B per clock at the sampled SM clock
        fine = sample_fwd_fine_samples(info)
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0  # no samples: maximum clock
        l1_peak = n_sm * 128 * mhz * 1e6 / 1e9
        l1_ach = 64 * fine / (dom_ms / 1e3) / 1e9
        l1_roofline = {"fine_samples": fine, "bytes": 64 * fine, "n_sm": n_sm, "bytes_per_clock_per_sm": 128,
                       "sm_mhz": mhz, "achieved": l1_ach, "peak": l1_peak, "unit": "GB/s", "frac": l1_ach / l1_peak}

    # the linear-interpolation variant of the same workload (same timing rules, fewer steps)
    plan_lin = rl.radon_plan_create(N, N_ANGLES, N_DET, 1, M)
    for _ in range(3):
        flush.zero_()
        rl.radon_forward(plan_lin, f_d, sino_d, stream)
        rl.radon_backproject(plan_lin, g_d, img_d, stream)
    n_lin = max(1, min(args.steps, 50))
    ev_lin = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_lin)]
    torch.cuda.synchronize()
    for k in range(n_lin):
        flush.zero_()
        ev_lin[k][0].record(stream)
        rl.radon_forward(plan_lin, f_d, sino_d, stream)
        rl.radon_backproject(plan_lin, g_d, img_d, stream)
        ev_lin[k][1].record(stream)
    torch.cuda.synchronize()
    lin_ms = reduce_max(sum(a.elapsed_time(b) for a, b in ev_lin), dist if world > 1 else None, dev) / n_lin
    lin_out = (sino_d.cpu().numpy(), img_d.cpu().numpy())  # R f and R# g of the linear variant
    linear = {"interp_order": 1, "ms_per_step": lin_ms, "steps": n_lin,
              "value": whole_job_rate(world, _samples_per_step(), 1, lin_ms / 1e3), "unit": UNIT}
    del plan_lin

    # end to end through the host-buffer C ABI entry points (pinned host memory).  Two pipelines,
    # each an R thread and an R# thread with their own plans and streams, take alternate steps:
    # one step's host copies overlap the other step's kernels.  Each call blocks until its result
    # is in host memory (ctypes releases the GIL while it runs); a pipeline starts its next step
    # only after both calls of its previous step returned.
    from concurrent.futures import ThreadPoolExecutor

    h_f = torch.from_numpy(f).pin_memory()
    h_g = torch.from_numpy(g).pin_memory()
    lanes = []
    for li in range(2):
        lanes.append({
            "plan_r": plan if li == 0 else rl.radon_plan_create(N, N_ANGLES, N_DET, INTERP, M),
            "plan_b": plan_bp if li == 0 else rl.radon_plan_create(N, N_ANGLES, N_DET, INTERP, M),
            "st_r": stream if li == 0 else torch.cuda.Stream(dev),
            "st_b": torch.cuda.Stream(dev),
            "h_s": torch.empty((N_ANGLES, N_DET), dtype=torch.float32).pin_memory(),
            "h_i": torch.empty((N, N), dtype=torch.float32).pin_memory(),
        })
    pool = ThreadPoolExecutor(max_workers=4)

    def submit_pair(ln):
        return (pool.submit(rl.radon_forward_host, ln["plan_r"], h_f, ln["h_s"], ln["st_r"]),
                pool.submit(rl.radon_backproject_host, ln["plan_b"], h_g, ln["h_i"], ln["st_b"]))

    def run_host(n_steps, n_lanes):
        pending = [None] * n_lanes
        for k in range(n_steps):
            li = k % n_lanes
            if pending[li] is not None:
                for fut in pending[li]:
                    fut.result()
            pending[li] = submit_pair(lanes[li])
        for pend in pending:
            if pend is not None:
                for fut in pend:
                    fut.result()

    def pair_host_serial():
        rl.radon_forward_host(plan, h_f, lanes[0]["h_s"], stream)
        rl.radon_backproject_host(plan, h_g, lanes[0]["h_i"], stream)

    run_host(4, 2)
    run_host(2, 1)
    for _ in range(2):
        pair_host_serial()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    run_host(args.steps, 2)
    e2e_s = reduce_max(time.perf_counter() - t0, dist if world > 1 else None, dev)
    t0 = time.perf_counter()
    run_host(n_aux, 1)
    e2e_one_s = reduce_max(time.perf_counter() - t0, dist if world > 1 else None, dev)
    t0 = time.perf_counter()
    for _ in range(n_aux):
        pair_host_serial()
    e2e_serial_s = reduce_max(time.perf_counter() - t0, dist if world > 1 else None, dev)
    pool.shutdown()
    e2e_out = (lanes[0]["h_s"].numpy().copy(), lanes[0]["h_i"].numpy().copy(),
               lanes[1]["h_s"].numpy().copy(), lanes[1]["h_i"].numpy().copy())
    for ln in lanes[1:]:
        del ln["plan_r"], ln["plan_b"]
    e2e = {
        "value": whole_job_rate(world, _samples_per_step(), args.steps, e2e_s),
        "unit": UNIT,
        "h2d_bytes_per_step": 4 * (N * N + N_ANGLES * N_DET),
        "d2h_bytes_per_step": 4 * (N_ANGLES * N_DET + N * N),
        "api": "radon_forward_host and radon_backproject_host; two pipelines (an R thread and an R# thread "
               "each, own plans and streams) take alternate steps",
        "one_pipeline_value": whole_job_rate(world, _samples_per_step(), n_aux, e2e_one_s),
        "serial_value": whole_job_rate(world, _samples_per_step(), n_aux, e2e_serial_s),
        "pipelines_equal": bool(np.array_equal(e2e_out[0], e2e_out[2]) and np.array_equal(e2e_out[1], e2e_out[3])),
    }
    h_s, h_i = e2e_out[0], e2e_out[1]

    extras = {}
    if world == 1 and not args.no_extras:
        extras["batched"] = bench_batched(rl, torch, flush, with_oracle=not args.no_cpu_baseline)
        extras["least_squares"] = bench_least_squares(rl, torch, with_oracle=not args.no_cpu_baseline)
        extras["fbp_8192"] = bench_fbp_large(rl, torch, flush, with_oracle=not args.no_cpu_baseline)
        extras["exact_transpose"] = bench_exact_transpose(rl, torch, flush)
        extras["paper_table1_backprojection"] = bench_paper_table1(rl, torch, flush,
                                                                   with_oracle=not args.no_cpu_baseline)
        extras["em_volume_256"] = bench_em_volume(rl, torch, 256, with_oracle=not args.no_cpu_baseline)
        extras["em_volume_512"] = bench_em_volume(rl, torch, 512, with_oracle=not args.no_cpu_baseline)

    cpu = None
    err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, (ref_s, ref_i) = cpu_baseline(f, g)
        err = {"R": rel_l2(h_s, ref_s), "R#": rel_l2(h_i, ref_i), "tolerance": 1e-5,
               "oracle": "FP64 log-polar oracle (Algorithms 1 and 2, dense DFTs), same inputs", "metric": "relative L2"}
        from oracle import geometry as _geometry

        err["vs_direct_sampled"] = err_vs_direct(
            _geometry.make_geometry(N, N_ANGLES, N_DET, M, INTERP), f, g,
            {"cuda": (h_s, h_i), "logpolar_oracle": (ref_s, ref_i)})
        _, (lin_s, lin_i) = cpu_baseline(f, g, interp=1)
        linear["err_vs_oracle"] = {"R": rel_l2(lin_out[0], lin_s), "R#": rel_l2(lin_out[1], lin_i), "tolerance": 1e-5,
                                   "oracle": "FP64 log-polar oracle, linear interpolation, same inputs",
                                   "metric": "relative L2"}
        err["vs_direct_sampled"]["note"] = (
            "the method's discretisation against exact line integrals (R, ellipse phantom) and the "
            "rectangle rule over angles (R#, white-noise sinogram: the two angular discretisations "
            "differ at the noise level); compare the cuda and oracle entries")

    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": _config(),
        "execution": "R on one stream and R# on a second stream, one plan each; serial_ms_per_step: "
                     "both on one stream",
        "serial_ms_per_step": serial_ms,
        "roofline": {
            # the dominant kernel's algorithmic bytes against the measured HBM copy bandwidth; its
            # binding unit (from ncu) is L1/TEX or instruction issue, not DRAM
            "bound": summary[3] if summary else "l1tex", "kernel": dom, "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
            "algorithmic_bytes": nbytes[dom], "ms_per_launch": dom_ms,
            "traffic_source": (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch, captured at "
                               f"commit {ncu_commit} (kernel sources {ncu_sha}, unchanged since)") if summary else
                              f"null: the kernel sources ({kernel_sources_sha()}) changed since the last ncu capture",
            "binding_units_ncu": None if summary is None else {
                "l1tex_pct_of_peak": summary[1], "issue_pct_of_peak": summary[2],
                "note": "DRAM throughput is a few percent of peak; L1/TEX and issue bind this kernel"},
            "l1": l1_roofline,
            "pair": {
                "bytes": pb["pair"], "bytes_R": pb["R"], "bytes_R#": pb["R#"],
                "model": "B_R = 4N^2 + 4 n_angles n_det + 4 S_c + |K|, B_R# = 4 n_angles n_live + 4N^2 + 4 S_c + |K|, "
                         f"S_c = M n_theta_half (N_rho/2+1) 8 = {pb['S_c']}, |K| = (n_theta/2+1)(N_rho/2+1) 8 = {pb['K']}",
                "ms": ms_per_step, "achieved": pb["pair"] / (ms_per_step / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                "frac": pb["pair"] / (ms_per_step / 1e3) / 1e9 / peak,
            },
        },
        "cpu_baseline": cpu,
        "err_vs_oracle": err,
        "linear_variant": linear,
        **extras,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "stage_ms_per_launch": stage_ms,
        "pixel_angle_updates_per_s": world * N * N * N_ANGLES * args.steps / (total_ms / 1e3),
    }
    print(json.dumps(out), flush=True)


def cpu_baseline(f, g, partitions=None, interp=INTERP):
    """FP64 log-polar oracle on the host cores: R f and R# g of the same inputs, all partitions
    (partitions=None) or the listed ones; kernel tables and DFT matrices are set up outside the
    timed interval.  Returns (the cpu_baseline object, (R f, R# g))."""
    import numpy as np

    from oracle import geometry, kernels, logpolar

    geo = geometry.make_geometry(N, N_ANGLES, N_DET, M, interp)
    KR = kernels.multiplier(geo, "R")
    KB = kernels.multiplier(geo, "B")
    dft = logpolar._Dft(geo)
    t0 = time.perf_counter()
    rf = logpolar.forward(f.astype(np.float64), geo, K=KR, dft=dft, partitions=partitions)
    bg = logpolar.backproject(g.astype(np.float64), geo, K=KB, dft=dft, partitions=partitions)
    dt = time.perf_counter() - t0
    parts = list(range(M)) if partitions is None else list(partitions)
    frac = len(parts) / M
    sample = (f"R and R# of the whole N=2048 workload ({dt:.1f} s)" if frac == 1.0 else
              f"R and R# of the N=2048 workload restricted to partition(s) {parts} of {M} "
              f"({dt:.1f} s); value scaled by that fraction")
    info = {"value": frac * _samples_per_step() / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": sample}
    return info, (rf, bg)


def err_vs_direct(geo, f, g, results: dict, seed: int = 0, n_ang: int = 16, n_bins: int = 32,
                  n_pix: int = 512) -> dict:
    """Relative L2 distance of R f and R# g from the direct oracle (exact line integrals of the
    interpolated image; the rectangle rule over the measured angles for R#) on a seeded random
    sample of outputs: n_ang angles x n_bins live bins, and n_pix pixels inside the disc.
    ``results`` maps a name to (R f, R# g) full outputs; each gets its own distances, so the
    CUDA path can be read against the log-polar oracle's own discretisation difference."""
    import numpy as np

    from oracle import direct, geometry

    rng = np.random.default_rng(seed)
    ang = np.sort(rng.choice(geo.n_angles, n_ang, replace=False))
    live = np.nonzero(geometry.live_bins(geo.n_det))[0]
    det = np.sort(rng.choice(live, min(n_bins, live.size), replace=False))
    ii, jj = np.nonzero(geometry.disc_mask(geo.N))
    sel = rng.choice(ii.size, min(n_pix, ii.size), replace=False)
    Rd = direct.radon_direct(np.asarray(f, dtype=np.float64), geo, angle_idx=ang, det_idx=det)
    Bd = direct.backproject_direct(np.asarray(g, dtype=np.float64), geo, pixels=(ii[sel], jj[sel]))
    out = {"sample": f"{ang.size} angles x {det.size} live bins; {sel.size} pixels in the disc (seed {seed})"}
    for name, (rf, bg) in results.items():
        out[name] = {"R": rel_l2(np.asarray(rf)[np.ix_(ang, det)], Rd),
                     "R#": rel_l2(np.asarray(bg)[ii[sel], jj[sel]], Bd)}
    return out


def rel_l2(got, ref) -> float:
    import numpy as np

    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(np.asarray(got, dtype=np.float64) - ref) / np.linalg.norm(ref))


def run_reference(args):
    import numpy as np

    from workloads import ellipse_image, random_ellipses, random_sinogram

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    f = ellipse_image(N, random_ellipses(50, 2)).astype(np.float32)
    g = random_sinogram(N_ANGLES, N_DET, 3).astype(np.float32)
    vals = []
    last = None
    t_start = time.perf_counter()
    for _ in range(args.steps):  # bounded: stop after ~2 minutes of oracle time
        last, _ = cpu_baseline(f, g, partitions=(0,))
        vals.append(last["value"])
        if time.perf_counter() - t_start > 120.0:
            break
    value = statistics.median(vals)
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": len(vals), "warmup": 0, "ms_per_step": 1e3 * _samples_per_step() / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": last["sample"] if last else ""},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def run_once(transpose: bool = False):
    """One untimed R and R# (or, with ``transpose``, one exact transpose R^T) of the workload."""
    import numpy as np
    import torch

    import paper_1506_00014_gb300 as rl
    from workloads import ellipse_image, random_ellipses, random_sinogram

    plan = rl.radon_plan_create(N, N_ANGLES, N_DET, INTERP, M)
    f = torch.from_numpy(ellipse_image(N, random_ellipses(50, 2)).astype(np.float32)).cuda()
    g = torch.from_numpy(random_sinogram(N_ANGLES, N_DET, 3).astype(np.float32)).cuda()
    s = torch.empty((N_ANGLES, N_DET), dtype=torch.float32, device="cuda")
    i = torch.empty((N, N), dtype=torch.float32, device="cuda")
    if transpose:
        rl.radon_transpose(plan, g, i)
    else:
        rl.radon_forward(plan, f, s)
        rl.radon_backproject(plan, g, i)
    torch.cuda.synchronize()
    print(json.dumps({"once": WORKLOAD, "transpose": transpose, "sino_sum": float(s.double().sum()) if not transpose
                      else None, "img_sum": float(i.double().sum())}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched (96 uneven slices) and least-squares (64 slices) comparisons")
    ap.add_argument("--once", action="store_true",
                    help="one untimed R + R# on the workload (for profiler captures); prints a short line")
    ap.add_argument("--once-transpose", action="store_true",
                    help="one untimed exact transpose R^T on the workload (for profiler captures)")
    args = ap.parse_args()
    if args.once or args.once_transpose:
        run_once(transpose=args.once_transpose)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
