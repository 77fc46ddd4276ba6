"""Host logic of bench.py's kernel report (CPU): the roofline of the kernel
with the most device time, its arithmetic against the measured peak, the
per-kernel table and the launch count of the library's own kernels."""
import bench


def _prof():
    # name: (launches, total device ms, algorithmic bytes) over 10 steps
    return {"sda_sum": (10, 11.0, 6.72e10), "shrink": (80, 7.3, 2.0e10), "final_mle": (10, 5.0, 1.1e10),
            "cufft_r2c": (10, 0.3, 0.0), "not_launched": (0, 0.0, 0.0)}


def test_roofline_of_the_kernel_with_most_device_time():
    roof, sda_roof, kern, launches = bench.kernel_report(_prof(), 10, None, None)
    peak, _ = bench.peaks()
    assert roof["kernel"] == "sda_sum" and roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    per_launch_s = 11.0 / 10 / 1000.0
    assert abs(roof["achieved"] - 6.72e9 / per_launch_s / 1e9) < 1e-6
    assert abs(roof["frac"] - roof["achieved"] / peak) < 1e-12 and roof["peak"] == peak
    assert roof["bytes_per_launch"] == 6.72e9 and roof["launches"] == 10
    assert roof["traffic"] is None or roof["traffic"] > 0
    assert sda_roof["kernel"] == "sda_sum" and abs(sda_roof["frac"] - roof["frac"]) < 1e-12
    # library kernels only (cuFFT excluded), per step figures, kernels never launched left out
    assert launches == 100
    assert "not_launched" not in kern
    assert kern["shrink"]["launches_per_step"] == 8 and abs(kern["shrink"]["ms_per_step"] - 0.73) < 1e-12
    assert abs(sum(v["share"] for v in kern.values()) - 1.0) < 1e-12
    assert "algorithmic_GBps" not in kern["cufft_r2c"]


def test_forced_dominant_kernel():
    roof, _, _, _ = bench.kernel_report(_prof(), 10, None, None, dominant="final_mle")
    assert roof["kernel"] == "final_mle" and roof["launches"] == 10
    assert abs(roof["achieved"] - 1.1e9 / (5.0 / 10 / 1000.0) / 1e9) < 1e-6


def test_fallback_peak_without_measured_file(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")


def test_headline_parity_host_logic(monkeypatch):
    """The parity block of the video bench: relative L2 of num / den / K and the
    max-abs of the group-0 residual against the oracle, pass / fail at the
    stated tolerances (small frames; the oracle computes both sides here, one
    of them perturbed)."""
    import numpy as np

    import oracle as O
    from paper_1909_04573_gb300 import synth
    monkeypatch.setattr(bench, "D_SDA", 4)
    fr = synth.frames(synth.Camera(H=32, W=48, C=3, camera_id=77), 8).numpy()
    onum, oden = O.fingerprint_accumulate(fr, 4)
    res0 = O.residual(O.sda_average(fr[:4], 4)[0])
    good = {"num": onum.astype(np.float32), "den": oden.astype(np.float32),
            "K": O.fingerprint_finalize(onum, oden).astype(np.float32), "res0": res0.astype(np.float32)}
    out = bench.headline_parity(good, fr, onum, oden)
    assert out["pass"] and out["num_rel_l2"] < 1e-6 and out["residual_max_abs"] < 1e-4
    bad = dict(good, res0=good["res0"] + 2e-3)             # a residual off by more than 1e-3
    out = bench.headline_parity(bad, fr, onum, oden)
    assert not out["pass"] and out["residual_max_abs"] > 1e-3
    bad = dict(good, num=good["num"] * (1 + 1e-4))          # sums off by 1e-4 relative
    out = bench.headline_parity(bad, fr, onum, oden)
    assert not out["pass"] and abs(out["num_rel_l2"] - 1e-4) < 1e-5


def test_group_sum_roofline_follows_the_fused_kernel():
    """With the group sums fused into the level-1 analysis the group-sum
    roofline is that kernel's (sda_dwt); with the separate kernels it is the
    sums kernel's (sda_sum)."""
    prof = {"sda_dwt": (10, 11.8, 7.345e10), "shrink": (80, 7.3, 2.0e10), "analysis_l1": (10, 2.8, 1.1e10)}
    roof, sda_roof, kern, _ = bench.kernel_report(prof, 10, None, None)
    assert roof["kernel"] == "sda_dwt" and sda_roof["kernel"] == "sda_dwt"
    assert abs(sda_roof["bytes_per_launch"] - 7.345e9) < 1.0
    assert abs(sda_roof["achieved"] - 7.345e9 / (11.8 / 10 / 1000.0) / 1e9) < 1e-6
    _, sda_roof, _, _ = bench.kernel_report(_prof(), 10, None, None)
    assert sda_roof["kernel"] == "sda_sum"
    _, sda_roof, _, _ = bench.kernel_report({"final_mle": (1, 1.0, 1e9)}, 1, None, None)
    assert sda_roof is None
