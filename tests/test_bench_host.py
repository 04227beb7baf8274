"""Host-side checks of bench.py's bookkeeping (no GPU): the byte model covers every profiling
stage the forward and back-projection launch, and the committed DRAM-traffic summary parses."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1506_00014_gb300 import binding  # noqa: E402


def _info():
    from oracle import geometry

    geo = geometry.make_geometry(bench.N, bench.N_ANGLES, bench.N_DET, bench.M, bench.INTERP)
    return {"N": bench.N, "n_angles": bench.N_ANGLES, "n_det": bench.N_DET, "n_partitions": bench.M,
            "n_theta_half": geo.n_th_h, "N_rho": geo.N_rho, "n_theta": 2 * geo.n_th_h}


def test_byte_model_covers_the_transform_stages():
    model = bench.stage_bytes(_info())
    # the FBP filter and the exact transpose are not part of the pair
    stages = set(binding.STAGE_NAMES) - {"sino_filter"} - set(binding.TRANSPOSE_STAGES)
    assert set(model) == stages
    assert all(v > 0 for v in model.values())


def test_ncu_summary_is_used_only_for_the_kernels_it_was_captured_from(tmp_path):
    rows = "sample_fwd 76370000 77.8 69.6 l1tex\ngather_sino 33660000 89.3 68.1 l1tex\n"
    good = tmp_path / "good.txt"
    good.write_text(f"# commit: abc1234\n# kernel_sources_sha256: {bench.kernel_sources_sha()}\n" + rows)
    out, sha, commit = bench.ncu_summary(str(good))
    assert commit == "abc1234" and sha == bench.kernel_sources_sha()
    assert out["sample_fwd"] == (76370000.0, 77.8, 69.6, "l1tex")
    assert set(out) <= set(binding.STAGE_NAMES)
    stale = tmp_path / "stale.txt"
    stale.write_text("# commit: abc1234\n# kernel_sources_sha256: 0000000000000000\n" + rows)
    assert bench.ncu_summary(str(stale))[0] == {}
    assert bench.ncu_summary(str(tmp_path / "missing.txt"))[0] == {}


def test_committed_ncu_summary_parses():
    out, sha, commit = bench.ncu_summary()
    assert sha is not None and commit is not None
    assert all(len(v) == 4 and v[0] > 0 for v in out.values())


def test_pair_byte_model_at_the_single_slice_workload():
    """B_R = 4N^2 + 4 n_angles n_det + 4 S_c + |K| ~ 198 MB and B_R# ~ 190 MB at N = 2048."""
    from oracle import geometry

    b = bench.pair_bytes(_info())
    assert abs(b["R"] / 198.1e6 - 1) < 0.01 and abs(b["R#"] / 190.7e6 - 1) < 0.01
    assert b["pair"] == b["R"] + b["R#"]
    assert bench.live_bin_count(bench.N_DET) == int(geometry.live_bins(bench.N_DET).sum())


def test_samples_per_step_counts_both_outputs():
    assert bench._samples_per_step() == bench.N_ANGLES * bench.N_DET + bench.N * bench.N


def test_direct_oracle_sampling_runs_and_reports_each_result():
    import numpy as np

    from oracle import geometry, logpolar
    from workloads import ellipse_image, random_ellipses, random_sinogram

    geo = geometry.make_geometry(64, 48, 96, 3, 3)
    f = ellipse_image(64, random_ellipses(10, 2))
    g = random_sinogram(48, 96, 3)
    rf, bg = logpolar.forward(f, geo), logpolar.backproject(g, geo)
    out = bench.err_vs_direct(geo, f, g, {"a": (rf, bg), "b": (rf.astype(np.float32), bg.astype(np.float32))},
                              n_ang=8, n_bins=16, n_pix=64)
    assert out["a"]["R"] < 0.05  # the method against exact line integrals of the same interpolant
    assert abs(out["a"]["R"] - out["b"]["R"]) < 1e-5 and abs(out["a"]["R#"] - out["b"]["R#"]) < 1e-5
    assert "8 angles x 16 live bins" in out["sample"]


def test_fine_sample_count_matches_a_per_sample_scan():
    """The forward sampling's fine-sample count (used for its L1 roofline) equals a direct scan of
    every (partition, angular row, sub-angle, rho index): the tap block inside the padded array and
    within 16 + 1.5 pixels of the disc."""
    import math

    import numpy as np

    geo = binding.radon_geometry(64, 48, 96, 3, 3)
    n, mm, nh, r, nr = geo["N"], geo["n_partitions"], geo["n_theta_half"], geo["r"], geo["N_rho"]
    S = n / (2.0 * geo["a_R"])
    P = n + 6.0
    lo_b, hi_b = 1.0 + 1e-3, P - 2.0 - 1e-3
    cz, Rd = 3 + n / 2.0, n / 2.0 + 17.5
    t = np.exp((np.arange(nr) - nr + 1) * geo["d_rho"])
    count = 0
    for m in range(mm):
        C0 = n / 2.0 - (1.0 - geo["a_R"]) * math.cos(m * geo["beta"]) * S + 3
        R0 = n / 2.0 - (1.0 - geo["a_R"]) * math.sin(m * geo["beta"]) * S + 3
        for jj in range(nh):
            for q in range(r):
                phi = (jj + nh // 2 - nh) * geo["d_phi"] + (q - 0.5 * (r - 1)) * geo["d_phi"] / r
                col = C0 + t * math.cos(phi + m * geo["beta"]) * S
                row = R0 + t * math.sin(phi + m * geo["beta"]) * S
                ok = (col >= lo_b) & (col <= hi_b) & (row >= lo_b) & (row <= hi_b)
                ok &= (col - cz) ** 2 + (row - cz) ** 2 <= Rd * Rd
                count += int(ok.sum())
    assert bench.sample_fwd_fine_samples(geo) == count
    assert count > 0
