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


def test_dram_traffic_summary_names_known_stages():
    traffic = bench._dram_traffic()
    assert traffic, "profiles/dram_traffic_radon_pair_N2048.txt is missing or empty"
    assert set(traffic) <= set(binding.STAGE_NAMES)
    assert all(v > 0 for v in traffic.values())


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
