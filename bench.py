"""Throughput of SDA camera-fingerprint extraction on GB300.

Step = one pass of the whole path over the video-scale workload: 1000 RGB
1920x1080 uint8 frames of one synthetic camera (drifting scene), SDA groups of
50 (20 SDA frames, 60 channel denoises), MLE accumulation, finalize (grey,
zero-mean, DFT Wiener), then 10 same-camera and 10 foreign query frames each
denoised and matched by PCE.  The metric is frames/s into the fingerprint.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU (torchrun): every rank runs its own camera (independent problems,
no data-path collective): weak scaling.  --impl reference times the FP64 CPU
oracle (the only reference this path has) on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "frames/sec into fingerprint (1080p, SDA vs per-frame) and HBM GB/s % of peak"
UNIT = "frames/s"
H, W, C = 1080, 1920, 3
M_FRAMES, D_SDA, N_QUERY = 1000, 50, 10
WORKLOAD = "video-1080p-rgb-1000f-sda50"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-perframe", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="video config: time eager launches, not a CUDA graph")
    ap.add_argument("--sda-fusion", type=int, default=0,
                    help="video and batch configs: prnu_params.sda_fusion of the fingerprints (0: fused group sums + level-1 "
                         "analysis where it applies, -1: separate kernels, n >= 1: fused with n row strips)")
    ap.add_argument("--frames", type=int, default=M_FRAMES,
                    help="frames of the workload (default 1000; smaller values are for profiling captures)")
    ap.add_argument("--config", default="video", choices=["video", "precision", "depth", "batch", "grad"],
                    help="video: 1000 RGB 1920x1080 frames, SDA-50 (the headline); precision: 500 RGB 4032x3024 "
                         "frames, SDA-25, per storage type throughput and error against the FP64 oracle; depth: "
                         "SDA-depth study; batch: 32 cameras of mixed resolutions, frame counts and SDA groups; "
                         "grad: forward + adjoint of the chain on 256 grey 512x512 frames and 50 PCE ascent steps")
    ap.add_argument("--cameras", type=int, default=32, help="batch config: number of cameras")
    ap.add_argument("--chunk-gb", type=float, default=96.0, help="batch config: frame buffer per chunk (GiB)")
    ap.add_argument("--groups-per-pass", type=int, default=32, help="batch config: SDA groups per pass")
    ap.add_argument("--batch-path", default="both", choices=["persistent", "stage", "both"],
                    help="batch config: the persistent launch (value), the per-stage launches, or both (the "
                         "per-stage form reported beside the persistent one)")
    ap.add_argument("--slots", type=int, default=4, help="batch config: workspace slots of the persistent launch")
    ap.add_argument("--mode", default="weak", choices=["weak", "shard"],
                    help="weak: one camera per GPU (no exchange); shard: one camera's groups split over the GPUs, "
                         "num/den summed with one all-reduce (strong scaling)")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed SDA region with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Kernels bound by FP32 arithmetic issue rather than HBM, with their
# algorithmic FP32 operations per algorithmic byte the profiler records.
# shrink: per coefficient 8 bytes (read + write) and 41 operations: c^2 (1),
# nested horizontal sums (8), vertical sums of 3/5/7/9 terms (20), four
# 1/w^2 scalings (4), three minima (3), max(0, v - s0^2) (2), + s0^2 (1),
# c s0^2 / den (2).
ALU_OPS_PER_BYTE = {"shrink": 41.0 / 8.0}
FP32_LANES_PER_SM = 128

# profiler name -> kernel symbol in the ncu captures (profiles/)
NCU_NAME = {"shrink": "k_shrink_strip<0, float>", "sda_sum": "k_sda_sum<3, 1024, 0>",
            "sda_dwt": "k_sda_dwt<3, 2, float>",
            "analysis_l1": "k_analysis_stream<1, float, 32, 2>", "analysis": "k_analysis<0, float>",
            "synthesis": "k_synthesis_stream<0, float>", "final_mle": "k_final_async_w<0, 2>",
            "final_pce": "k_final_pce<1>", "pce_fft_rows": "k_rfft_rows_w<4>",
            "pce_fft_columns": "k_corr_columns_4s", "pce_fft_rows_inverse": "k_corr_rows_w<4>",
            "pce_outputs": "k_pce_outputs"}

def dram_traffic(kernel_symbol):
    """DRAM bytes per launch of a kernel from the committed ncu capture, or
    None when the capture is missing or the kernel source changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic_video-1080p-rgb-1000f-sda50.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split("\t")
        if len(parts) == 5 and parts[0] == kernel_symbol:
            src = os.path.join(ROOT, "paper_1909_04573_gb300", "csrc", parts[3])
            if not os.path.exists(src):
                return None
            sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
            return float(parts[2]) if sha == parts[4].strip() else None
    return None


# ------------------------------------------------------------------ clocks --
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def kernel_report(prof, steps, ck, dev, dominant=None):
    """Per-kernel table and rooflines from the library's event profile of
    `steps` steps: (roofline of the dominant kernel -- the one with the most
    device time, or `dominant` --, roofline of sda_sum, per-kernel table,
    launches of the library's own kernels)."""
    import torch
    own = {k: v for k, v in prof.items() if not k.startswith("cufft")}
    launches = sum(v[0] for v in own.values())
    total_dev = sum(v[1] for v in prof.values())
    hbm, peak_kind = peaks()
    kern = {}
    for k, (n, t, nbytes) in sorted(prof.items(), key=lambda kv: -kv[1][1]):
        if n == 0:
            continue
        e = {"launches_per_step": n / steps, "ms_per_step": t / steps,
             "share": t / total_dev if total_dev else None}
        if nbytes > 0 and t > 0:
            e["algorithmic_GBps"] = nbytes / (t / 1000.0) / 1e9
        kern[k] = e
    dom = dominant if dominant in own else max(own.items(), key=lambda kv: kv[1][1])[0]
    dom_n, dom_t, dom_b = own[dom]
    roof = None
    if dom_b > 0 and dom_n > 0:
        sec = dom_t / dom_n / 1000.0
        gbps = (dom_b / dom_n) / sec / 1e9
        sym = NCU_NAME.get(dom)
        traffic = dram_traffic(sym) if sym else None
        if dom in ALU_OPS_PER_BYTE:
            sm_mhz = (ck or {}).get("sm_mhz") or 2070.0
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            peak_tops = sms * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12
            ach = ALU_OPS_PER_BYTE[dom] * (dom_b / dom_n) / sec / 1e12
            roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak_tops, "unit": "TOP/s (FP32)",
                    "frac": ach / peak_tops,
                    "peak_kind": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_mhz:.0f} MHz",
                    "traffic": traffic, "bytes_per_launch": dom_b / dom_n, "launches": dom_n,
                    "ms_per_launch": dom_t / dom_n, "hbm_achieved_GBps": gbps, "hbm_frac": gbps / hbm}
        else:
            roof = {"kernel": dom, "bound": "hbm", "achieved": gbps, "peak": hbm, "unit": "GB/s",
                    "frac": gbps / hbm, "peak_kind": f"{peak_kind} copy bandwidth", "traffic": traffic,
                    "bytes_per_launch": dom_b / dom_n, "launches": dom_n, "ms_per_launch": dom_t / dom_n}
    sda_roof = None  # the group-sum kernel: fused with the level-1 analysis, or alone
    sk = next((k for k in ("sda_dwt", "sda_sum") if k in own and own[k][1] > 0), None)
    if sk:
        n_, t_, b_ = own[sk]
        g_ = (b_ / n_) / (t_ / n_ / 1000.0) / 1e9
        sda_roof = {"kernel": sk, "bound": "hbm", "achieved": g_, "peak": hbm, "unit": "GB/s",
                    "frac": g_ / hbm, "traffic": dram_traffic(NCU_NAME[sk]), "bytes_per_launch": b_ / n_}
    return roof, sda_roof, kern, launches


# ------------------------------------------------------------- CPU oracle --
def oracle_sample(frames_host, groups: int, sums: bool = False):
    """Time the FP64 oracle on `groups` SDA groups of the workload: SDA mean,
    per-channel residual, MLE sums.  Returns (seconds, frames, cores), and
    with sums=True also the oracle's (num, den) [C, H, W] float64."""
    import numpy as np

    import oracle as O
    O.build()
    t0 = time.perf_counter()
    num = np.zeros((C, H, W))
    den = np.zeros((C, H, W))
    O.fingerprint_accumulate(frames_host[: groups * D_SDA], D_SDA, num=num, den=den)
    t = time.perf_counter() - t0
    if sums:
        return t, groups * D_SDA, O.threads(), num, den
    return t, groups * D_SDA, O.threads()


# Tolerances of the FP32 path against the FP64 oracle (fingerprint relative
# L2, residual max-abs in 0..255 units); the MLE sums take the fingerprint's.
PARITY_TOL = {"num_rel_l2": 1e-5, "den_rel_l2": 1e-5, "K_rel_l2": 1e-5, "residual_max_abs": 1e-3}


def headline_parity(gpu, frames_host, onum, oden):
    """Compare the timed step's fingerprint sums with the oracle's on the same
    frames: num, den and K = num/den (no finalize flags) as relative L2, and
    the residual of the first SDA frame (group 0) as max-abs."""
    import numpy as np

    import oracle as O

    def rel(a, b):
        return float(np.linalg.norm(a.astype(np.float64) - b) / np.linalg.norm(b))

    oK = O.fingerprint_finalize(onum, oden, 0)
    I0 = O.sda_average(frames_host[:D_SDA], D_SDA)[0]
    ores = O.residual(I0)
    out = {"num_rel_l2": rel(gpu["num"], onum), "den_rel_l2": rel(gpu["den"], oden),
           "K_rel_l2": rel(gpu["K"], oK),
           "residual_max_abs": float(np.abs(gpu["res0"].astype(np.float64) - ores).max())}
    out["pass"] = all(out[k] <= PARITY_TOL[k] for k in PARITY_TOL)
    out["tolerance"] = dict(PARITY_TOL)
    out["sample"] = (f"the timed step's num/den ({len(frames_host)} frames, SDA-{D_SDA}, all groups), K = num/den, "
                     "and the residual of the group-0 SDA frame, against the FP64 oracle on the same uint8 frames")
    return out


def oracle_sample_1core(frames_host):
    """The same oracle on one core, over a fifth of a group (10 frames, the
    SDA mean and residual of those frames): seconds per frame."""
    import numpy as np

    import oracle as O
    O.set_threads(1)
    try:
        t0 = time.perf_counter()
        num = np.zeros((C, H, W))
        den = np.zeros((C, H, W))
        O.fingerprint_accumulate(frames_host[:10], 10, num=num, den=den)
        return (time.perf_counter() - t0) / 10
    finally:
        O.set_threads(None)


def reference_arm(args, rank):
    if rank != 0:
        return
    import torch

    from paper_1909_04573_gb300 import synth
    cam = synth.Camera(H=H, W=W, C=C, camera_id=0)
    fr = synth.frames(cam, D_SDA, device="cpu", drift_px=2.0).numpy()  # one SDA group
    for _ in range(args.warmup):
        oracle_sample(fr, 1)
    ts = []
    cores = 1
    for _ in range(args.steps):
        t, n, cores = oracle_sample(fr, 1)
        ts.append(t)
    ms = 1000.0 * sum(ts) / len(ts)
    value = D_SDA / (ms / 1000.0)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "frames": M_FRAMES, "H": H, "W": W, "C": C, "d": D_SDA,
                       "parallelism": "oracle on host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"1 SDA group of {D_SDA} frames (1080p RGB) per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    del torch
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- precision config --
def precision_config(args, rank, world, local):
    """500 RGB 4032x3024 frames (sigma_read 3), SDA groups of 25.  For each
    storage variant: step time of accumulate + finalize over all frames, and
    the error of the residual (one SDA frame), the fingerprint and the PCE of
    a same-camera query against the FP64 oracle on the first two groups."""
    import numpy as np
    import torch

    import __graft_entry__
    import oracle as O
    from paper_1909_04573_gb300 import prnu as P
    from paper_1909_04573_gb300 import synth

    torch.cuda.set_device(local)
    __graft_entry__.build()
    dev = torch.device("cuda", local)
    Hh, Ww, Cc, m, d = 3024, 4032, 3, args.frames if args.frames != M_FRAMES else 500, 25
    cam = synth.Camera(H=Hh, W=Ww, C=Cc, camera_id=rank, sigma_read=3.0)
    frames = synth.frames(cam, m, device=dev, drift_px=2.0)
    q = synth.frames(cam, 1, stream=1, device=dev)
    ctx = P.Context(local)
    qimg = ctx.sda_average(q, 1)
    # oracle on the first two groups
    sample = frames[: 2 * d].cpu().numpy()
    t0 = time.perf_counter()
    onum, oden = O.fingerprint_accumulate(sample, d)
    oK = O.fingerprint_finalize(onum, oden, O.TO_GRAY)[0]
    oimg = O.sda_average(sample[:d], d)[0]
    ores = O.residual(oimg)
    qh = qimg[0].cpu().numpy().astype(np.float64)
    oq = O.residual(qh)
    opce = O.pce_match(oK, O.to_gray(oq), O.to_gray(qh)).pce
    t_oracle = time.perf_counter() - t0
    frames16 = frames.to(torch.float16)
    variants = [("u8-f32", P.PRNU_FRAMES_U8, P.PRNU_DTYPE_F32, False),
                ("u8-f32-compensated", P.PRNU_FRAMES_U8, P.PRNU_DTYPE_F32, True),
                ("u8-f16", P.PRNU_FRAMES_U8, P.PRNU_DTYPE_F16, False),
                ("u8-bf16", P.PRNU_FRAMES_U8, P.PRNU_DTYPE_BF16, False),
                ("f16-f16", P.PRNU_FRAMES_F16, P.PRNU_DTYPE_F16, False)]
    out = {}
    for name, fdt, sdt, comp in variants:
        prm = P.default_params(dtype=sdt, frame_dtype=fdt, compensated=comp)
        src = frames16 if fdt == P.PRNU_FRAMES_F16 else frames
        shape = (2, Cc, Hh, Ww) if comp else (Cc, Hh, Ww)
        num = torch.zeros(shape, device=dev)
        den = torch.zeros_like(num)

        def step():
            num.zero_()
            den.zero_()
            ctx.fingerprint_accumulate(src, d, num, den, params=prm)
            ctx.fingerprint_finalize(num, den, P.PRNU_TO_GRAY, params=prm)

        for _ in range(max(1, args.warmup)):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        # errors on the two-group sample
        num.zero_()
        den.zero_()
        ctx.fingerprint_accumulate(src[: 2 * d], d, num, den, params=prm)
        K = ctx.fingerprint_finalize(num, den, P.PRNU_TO_GRAY, params=prm)
        res = ctx.denoise_residual(torch.as_tensor(oimg.astype(np.float32), device=dev), params=prm)
        wq = ctx.denoise_residual(qimg[0], params=prm)
        pce = ctx.pce_match(K[0], wq, qimg[0])[0]
        Kc = K[0].cpu().numpy()
        out[name] = {"frames_per_s": m / (ms / 1000.0), "ms_per_step": ms,
                     "residual_maxabs": float(np.abs(res.cpu().numpy() - ores).max()),
                     "fingerprint_relL2": float(np.linalg.norm(Kc - oK) / np.linalg.norm(oK)),
                     "pce_rel": abs(pce - opce) / abs(opce), "pce": pce}
    line = {"metric": "precision: error vs FP64 oracle and frames/s per storage type", "unit": "frames/s",
            "config": {"workload": f"precision-4032x3024-rgb-{m}f-sda25", "frames": m, "H": Hh, "W": Ww, "C": Cc,
                       "d": d, "sigma_read": 3.0, "error_sample": "first 2 SDA groups (50 frames) + 1 query"},
            "oracle_pce": opce, "oracle_seconds": t_oracle, "variants": out, "steps": args.steps}
    print(json.dumps(line), flush=True)
    ctx.close()


# ----------------------------------------------------------- depth study --
def depth_config(args, rank, world, local):
    """Synthetic analogue of the paper's SDA-depth experiment (Sec. IV-C): per
    camera 50 frames give fingerprints at d = 1, 2, 5, 10, 25, 50 (50 .. 1
    denoise calls); 8 queries per camera are matched block-wise (disjoint
    500 x 500 blocks, Sec. IV-A) against their own camera's fingerprint (true
    cases) and the next camera's (false cases); PCE threshold 60 (Sec. IV).
    Flat scenes (low-pass sigma 8 px) against textured ones (sigma 1.5 px)."""
    import numpy as np
    import torch

    import __graft_entry__
    from paper_1909_04573_gb300 import prnu as P
    from paper_1909_04573_gb300 import synth

    torch.cuda.set_device(local)
    __graft_entry__.build()
    dev = torch.device("cuda", local)
    ctx = P.Context(local)
    Hh = Ww = 1000
    Cc, n_cam, m, n_q, blk = 3, 4, 50, 8, 500
    depths = [1, 2, 5, 10, 25, 50]
    flags = P.PRNU_TO_GRAY | P.PRNU_ZERO_MEAN | P.PRNU_WIENER_DFT
    result = {}
    for label, sig in (("flat", 8.0), ("textured", 1.5)):
        cams = [synth.Camera(H=Hh, W=Ww, C=Cc, camera_id=700 + i, scene_sigma=sig) for i in range(n_cam)]
        frames = [synth.frames(c, m, device=dev) for c in cams]
        qimg = [ctx.sda_average(synth.frames(c, n_q, stream=1, device=dev), 1) for c in cams]
        qres = [ctx.denoise_residual_batch(q).clone() for q in qimg]
        rows = {}
        for d in depths:
            Ks = []
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for i in range(n_cam):
                num = torch.zeros((Cc, Hh, Ww), device=dev)
                den = torch.zeros_like(num)
                ctx.fingerprint_accumulate(frames[i], d, num, den)
                Ks.append(ctx.fingerprint_finalize(num, den, flags)[0].clone())
            e1.record()
            torch.cuda.synchronize()
            fe_ms = e0.elapsed_time(e1) / n_cam
            pos, neg = [], []
            for i in range(n_cam):
                for j, tgt in ((i, pos), ((i + 1) % n_cam, neg)):
                    Kb, Wb, Ib = [], [], []
                    for by in range(Hh // blk):
                        for bx in range(Ww // blk):
                            ys, xs = slice(by * blk, (by + 1) * blk), slice(bx * blk, (bx + 1) * blk)
                            for k in range(n_q):
                                Kb.append(Ks[i][ys, xs])
                                Wb.append(qres[j][k][:, ys, xs])
                                Ib.append(qimg[j][k][:, ys, xs])
                    res = ctx.pce_match_pairs(torch.stack(Kb), torch.stack(Wb), torch.stack(Ib))
                    tgt.extend(r[0] for r in res)
            pos, neg = np.array(pos), np.array(neg)
            rows[str(d)] = {"denoise_calls": (m + d - 1) // d, "fe_ms_per_camera": fe_ms,
                            "pce_mean_true": float(pos.mean()), "pce_median_true": float(np.median(pos)),
                            "tpr": float((pos > 60).mean()), "fpr": float((neg > 60).mean()),
                            "blocks_true": int(pos.size), "blocks_false": int(neg.size)}
        result[label] = rows
    line = {"metric": "SDA depth study: block-wise PCE / TPR at threshold 60 vs SDA depth",
            "config": {"workload": "depth-1000x1000-rgb-50f", "cameras": n_cam, "frames": m, "queries": n_q,
                       "block": blk, "depths": depths, "finalize": "grey, zero-mean, DFT Wiener"},
            "result": result}
    print(json.dumps(line), flush=True)
    ctx.close()


# ------------------------------------------------------ multi-camera batch --
def batch_config(args, rank, world, local):
    """32 synthetic cameras (own K each) with frame counts uniform in
    100..2000, resolutions from {1280x720, 1920x1080, 4032x3024} RGB and SDA
    group sizes uniform in 10..100 (ragged last groups): 32,282 frames, 453 GB.
    The frames do not fit in HBM, so they are produced chunk by chunk into one
    reusable buffer (generation is outside the timed region); each chunk is one
    multi-camera accumulate call, captured once in a CUDA graph and replayed.
    Then the 32 fingerprints are finalised (grey, zero-mean, DFT Wiener) and
    matched in a 32 x 32 PCE matrix on the common top-left 1280 x 720 window
    (one query frame per camera).  Every rank runs the whole batch (weak)."""
    import numpy as np
    import torch

    import __graft_entry__
    from paper_1909_04573_gb300 import batch as B
    from paper_1909_04573_gb300 import prnu as P
    from paper_1909_04573_gb300 import synth

    torch.cuda.set_device(local)
    __graft_entry__.build()
    dev = torch.device("cuda", local)
    ctx = P.Context(local)
    specs = synth.batch_cameras(args.cameras)
    ncam = len(specs)
    budget = int(args.chunk_gb * (1 << 30))
    fbytes = [c.H * c.W * c.C for c, _, _ in specs]
    chunks = B.plan_chunks([(fb, m, d) for fb, (_, m, d) in zip(fbytes, specs)], budget)
    total_frames = sum(m for _, m, _ in specs)
    total_bytes = sum(fb * m for fb, (_, m, _) in zip(fbytes, specs))
    buf = torch.empty(max(B._align(p.offset + (p.f1 - p.f0) * fbytes[p.cam]) for ch in chunks for p in ch),
                      dtype=torch.uint8, device=dev)
    nums = [torch.zeros((c.C, c.H, c.W), device=dev) for c, _, _ in specs]
    dens = [torch.zeros_like(n) for n in nums]
    prm = P.default_params(sda_fusion=args.sda_fusion)
    gpp = args.groups_per_pass

    def items_of(ch):
        out = []
        for p in ch:
            c, _, d = specs[p.cam]
            n = p.f1 - p.f0
            v = buf[p.offset: p.offset + n * fbytes[p.cam]].view(n, c.H, c.W, c.C)
            out.append((v, d, nums[p.cam], dens[p.cam]))
        return out

    chunk_items = [items_of(ch) for ch in chunks]
    chunk_cams = [ctx.cameras(it) for it in chunk_items]
    # queries: one frame per camera, cropped to the common top-left window
    Hq, Wq = min(c.H for c, _, _ in specs), min(c.W for c, _, _ in specs)
    qimg = torch.empty((ncam, 3, Hq, Wq), device=dev)
    for i, (c, _, _) in enumerate(specs):
        q = ctx.sda_average(synth.frames_fast(c, 1, stream=1, device=dev), 1)
        qimg[i].copy_(q[0, :, :Hq, :Wq])
    wq = torch.empty_like(qimg)
    Kc = torch.empty((ncam, Hq, Wq), device=dev)
    flags = P.PRNU_TO_GRAY | P.PRNU_ZERO_MEAN | P.PRNU_WIENER_DFT
    # autotuned level-1 analysis shapes, one per geometry (outside the timed region)
    tuned = {}
    for geo in sorted({(c.H, c.W) for c, _, _ in specs}):
        shape, t = ctx.autotune(geo[0], geo[1], 3, prm, images=8)
        tuned[f"{geo[1]}x{geo[0]}"] = {"strip_rows": shape[0], "warps": shape[1], "ms": t}
    need = max(P.prnu_workspace_size_multi(ctx.ctx, cc, prm, gpp) for cc in chunk_cams)
    for c, _, _ in specs:
        need = max(need, P.prnu_workspace_size(ctx.ctx, c.H, c.W, c.C, prm, 1))
    need = max(need, P.prnu_workspace_size(ctx.ctx, Hq, Wq, 3, prm, ncam))
    ws = ctx.workspace(need)
    gen_s = [0.0]

    def generate(ci):
        t0 = time.perf_counter()
        for p, it in zip(chunks[ci], chunk_items[ci]):
            synth.frames_fast(specs[p.cam][0], p.f1 - p.f0, device=dev, out=it[0], start=p.f0)
        torch.cuda.synchronize()
        gen_s[0] += time.perf_counter() - t0

    # the persistent path: one workspace per chunk, so that every chunk's queue
    # status can be read back after the timed steps
    paths = ["persistent", "stage"] if args.batch_path == "both" else [args.batch_path]
    pws = []
    if "persistent" in paths:
        for cc in chunk_cams:
            nb_ = P.prnu_workspace_size_persistent(ctx.ctx, cc, prm, args.slots)
            pws.append(torch.empty(nb_, dtype=torch.uint8, device=dev))

    def accumulate(ci, path, stream=None):
        st = stream if stream is not None else ctx._stream()
        if path == "persistent":
            P.prnu_fingerprint_accumulate_persistent(ctx.ctx, chunk_cams[ci], prm, args.slots, 2000.0,
                                                     pws[ci].data_ptr(), pws[ci].numel(), st)
        else:
            P.prnu_fingerprint_accumulate_multi(ctx.ctx, chunk_cams[ci], prm, ws.data_ptr(), ws.numel(), st)

    def queue_status():
        bad = []
        for ci, w in enumerate(pws):
            st_, info = P.prnu_persistent_status(ctx.ctx, w.data_ptr(), w.numel(), ctx._stream())
            if st_ != P.PRNU_OK:
                bad.append({"chunk": ci, "status": st_, "item_group_stage": info})
        return bad

    pce = np.zeros((ncam, ncam))

    def tail():
        for i, (c, _, _) in enumerate(specs):
            K = ctx.fingerprint_finalize(nums[i], dens[i], flags)
            Kc[i].copy_(K[0, :Hq, :Wq])
        ctx.denoise_residual_batch(qimg, out=wq)
        for i in range(ncam):
            pce[i] = [r[0] for r in ctx.pce_match_batch(Kc[i], wq, qimg)]

    graphs = {pth: [None] * len(chunks) for pth in paths}

    def run_step(path, use_graphs, times):
        for n_, d_ in zip(nums, dens):
            n_.zero_()
            d_.zero_()
        for ci in range(len(chunks)):
            generate(ci)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if use_graphs:
                graphs[path][ci].replay()
            else:
                accumulate(ci, path)
            e1.record()
            times.append((e0, e1))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        tail()
        e1.record()
        times.append((e0, e1))

    side = torch.cuda.Stream()
    results = {}
    for path in paths:
        # warm-up 1 (eager, also creates the cuFFT plans), then capture one graph per chunk
        run_step(path, False, [])
        for ci in range(len(chunks)):
            g = torch.cuda.CUDAGraph()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                with torch.cuda.graph(g, stream=side):
                    accumulate(ci, path, side.cuda_stream)
            torch.cuda.current_stream().wait_stream(side)
            graphs[path][ci] = g
        for _ in range(max(0, args.warmup - 1)):
            run_step(path, True, [])
        # per-kernel profile of one eager step (the graphs replay the same launches)
        P.prnu_profile_reset(ctx.ctx)
        P.prnu_profile_enable(ctx.ctx, True)
        run_step(path, False, [])
        torch.cuda.synchronize()
        P.prnu_profile_enable(ctx.ctx, False)
        prof = P.prnu_profile_read(ctx.ctx)
        P.prnu_profile_reset(ctx.ctx)
        # timed steps: graph replays; only the device time between generation gaps counts
        gen_s[0] = 0.0
        clocks = Clocks(local)
        clocks.start()
        times = []
        for _ in range(args.steps):
            run_step(path, True, times)
        torch.cuda.synchronize()
        ck = clocks.stop()
        total_ms = sum(a.elapsed_time(b) for a, b in times)
        tail_ms = sum(times[i][0].elapsed_time(times[i][1])
                      for i in range(len(chunks), len(times), len(chunks) + 1))
        bad = queue_status() if path == "persistent" else []
        results[path] = {"ms": total_ms / args.steps, "tail_ms": tail_ms / args.steps, "prof": prof, "ck": ck,
                         "pce": pce.copy(), "queue_failures": bad, "gen_s": gen_s[0] / args.steps}
        for gs_ in graphs[path]:
            del gs_
        graphs[path] = [None] * len(chunks)
        torch.cuda.synchronize()
    main = results[paths[0]]
    ms, tail_ms, prof, ck = main["ms"], main["tail_ms"], main["prof"], main["ck"]
    pce[:] = main["pce"]
    roof, sda_roof, kern, launches = kernel_report(prof, 1, ck, dev)
    hbm, _ = peaks()
    diag = np.diag(pce)
    off = pce[~np.eye(ncam, dtype=bool)]
    res = sorted({(c.W, c.H) for c, _, _ in specs})
    line = {"metric": "multi-camera batch: frames/sec into 32 fingerprints + 32x32 PCE matrix",
            "value": world * total_frames / (ms / 1000.0), "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded sensor model, whole-pixel drift; VISION/NYUAD-MMD absent)",
            "config": {"workload": f"batch-{ncam}cam-{total_frames}f", "cameras": ncam, "frames": total_frames,
                       "frame_GB": total_bytes / 1e9, "resolutions": [f"{w}x{h}" for w, h in res],
                       "chunks": len(chunks), "chunk_GB": args.chunk_gb, "groups_per_pass": gpp,
                       "groups": sum((m + d - 1) // d for _, m, d in specs), "cuda_graphs": len(chunks),
                       "pce_window": f"{Wq}x{Hq}", "parallelism": f"whole batch per GPU x {world}",
                       "l2": "inputs 453 GB > 129 MB L2 (no flush)"},
            "path": paths[0], "tail_ms_per_step": tail_ms, "generation_s_per_step_untimed": main["gen_s"],
            "frame_GBps": total_bytes / (ms / 1000.0) / 1e9,
            "frame_frac_of_peak": total_bytes / (ms / 1000.0) / 1e9 / hbm,
            "autotune": tuned, "roofline": roof, "roofline_sda_sum": sda_roof, "gpu_launches": int(launches),
            "kernels": kern,
            "pce_matrix": {"diag_min": float(diag.min()), "diag_median": float(np.median(diag)),
                           "offdiag_max": float(off.max()), "offdiag_max_abs": float(np.abs(off).max()),
                           "diag_above_60": int((diag > 60).sum()), "offdiag_above_60": int((off > 60).sum())}}
    if "persistent" in results:
        line["queue_failures"] = results["persistent"]["queue_failures"]
    if len(paths) == 2:
        o = results[paths[1]]
        line["per_stage"] = {"value": world * total_frames / (o["ms"] / 1000.0), "unit": "frames/s",
                             "ms_per_step": o["ms"], "tail_ms_per_step": o["tail_ms"],
                             "mode": "one launch per stage per pass (prnu_fingerprint_accumulate_multi), graph per chunk",
                             "pce_matrix_max_rel_diff": float(np.max(np.abs(o["pce"] - main["pce"]) /
                                                                     np.maximum(np.abs(main["pce"]), 1.0)))}
    if "persistent" in paths and rank == 0:
        line["parity"] = batch_parity_sample(ctx, chunks, chunk_items, specs, prm, args.slots)
    if ck:
        line["clocks"] = ck
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def batch_parity_sample(ctx, chunks, chunk_items, specs, prm, slots):
    """Per-camera parity of the persistent launch on the first chunk: the first
    SDA group of each of its camera parts (one part per resolution, at most
    four), run as one persistent call into fresh sums and compared with the FP64
    oracle on the same frames."""
    import numpy as np
    import torch

    import oracle as O
    O.build()
    picked, seen = [], set()
    for p, it in zip(chunks[0], chunk_items[0]):
        c, _, d = specs[p.cam]
        if (c.H, c.W) in seen or len(picked) == 4:
            continue
        seen.add((c.H, c.W))
        fr = it[0][: min(d, it[0].shape[0])]
        num = torch.zeros((c.C, c.H, c.W), device=fr.device)
        picked.append((fr, d, num, torch.zeros_like(num)))
    ctx.fingerprint_accumulate_persistent(picked, params=prm, slots=slots)
    out = []
    for fr, d, num, den in picked:
        onum, oden = O.fingerprint_accumulate(fr.cpu().numpy(), d)
        out.append({"geometry": f"{fr.shape[2]}x{fr.shape[1]}", "frames": int(fr.shape[0]),
                    "num_rel_l2": float(np.linalg.norm(num.cpu().numpy() - onum) / np.linalg.norm(onum)),
                    "den_rel_l2": float(np.linalg.norm(den.cpu().numpy() - oden) / np.linalg.norm(oden))})
    ok = all(r["num_rel_l2"] <= 1e-5 and r["den_rel_l2"] <= 1e-5 for r in out)
    return {"pass": ok, "tolerance": 1e-5, "cameras": out,
            "sample": "first SDA group of one camera part per resolution in the first chunk, one persistent call"}


# ------------------------------------------------------- differentiation --
def grad_config(args, rank, world, local):
    """256 grey 512x512 frames (independent scenes), SDA groups of 16 with
    learnable per-frame weights (init 1/16) and a learnable sigma0 (init 3).
    Step = forward (weighted SDA, residuals with checkpoint, MLE, PCE of 8
    held-out query frames) plus the adjoint of all of it; value = frames/s
    through forward + adjoint.  Then 50 Adam steps maximising the queries'
    mean PCE, with 8 further queries as an evaluation set; the FP64 oracle's
    gradient at the start is timed beside it (one evaluation, 2 queries)."""
    import numpy as np
    import torch

    import __graft_entry__
    from paper_1909_04573_gb300 import grad as G
    from paper_1909_04573_gb300 import prnu as P
    from paper_1909_04573_gb300 import synth

    torch.cuda.set_device(local)
    __graft_entry__.build()
    dev = torch.device("cuda", local)
    ctx = P.Context(local)
    m, Hh, Ww, d, nq = 256, 512, 512, 16, 8
    cam = synth.Camera(H=Hh, W=Ww, C=1, camera_id=900 + rank)
    frames = synth.frames(cam, m, device=dev)
    q_train = ctx.sda_average(synth.frames(cam, nq, stream=1, device=dev), 1)
    q_eval = ctx.sda_average(synth.frames(cam, nq, stream=2, device=dev), 1)
    w = torch.full((m,), 1.0 / d, device=dev, requires_grad=True)
    sig = torch.tensor(3.0, dtype=torch.float64, requires_grad=True)

    def step():
        w.grad = None
        sig.grad = None
        J = G.mean_pce(frames, w, d, sig, q_train, ctx)
        J.backward()
        return J

    for _ in range(args.warmup):
        step()
    P.prnu_profile_reset(ctx.ctx)
    P.prnu_profile_enable(ctx.ctx, True)
    clocks = Clocks(local)
    clocks.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record()
    for _ in range(args.steps):
        J0 = step()
    e1.record()
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) / args.steps * 1000.0
    ck = clocks.stop()
    P.prnu_profile_enable(ctx.ctx, False)
    prof = P.prnu_profile_read(ctx.ctx)
    P.prnu_profile_reset(ctx.ctx)
    ms = e0.elapsed_time(e1) / args.steps
    roof, _, kern, launches = kernel_report(prof, args.steps, ck, dev)
    g_w0, g_s0 = w.grad.detach().clone(), float(sig.grad)
    out = {"metric": "differentiation: frames/s through forward + adjoint (weighted SDA, residual, MLE, PCE)",
           "value": world * m / (ms / 1000.0), "unit": "frames/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "wall_ms_per_step": wall, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded sensor model)",
           "config": {"workload": "grad-512x512-gray-256f-sda16", "frames": m, "H": Hh, "W": Ww, "C": 1, "d": d,
                      "queries_train": nq, "queries_eval": nq, "l2": "inputs 67 MB < L2; residual and PCE "
                      "intermediates ~0.4 GB per step (no flush)"},
           "roofline": roof, "gpu_launches": int(launches), "kernels": kern,
           "grad_at_start": {"J": J0.item(), "g_sigma0": g_s0, "g_w_norm": float(g_w0.norm()),
                             "g_w_mean": float(g_w0.mean())}}
    if ck:
        out["clocks"] = ck
    # FP64 oracle gradient at the start (bounded: 2 queries), timed on the host
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle as O
        from oracle import grad as OG
        O.build()
        t0 = time.perf_counter()
        oJ, ogw, ogs = OG.objective_and_grad(frames.cpu().numpy(), d, np.full(m, 1.0 / d), 3.0,
                                             q_train[:2].double().cpu().numpy())
        t_or = time.perf_counter() - t0
        with torch.no_grad():
            w2 = torch.full((m,), 1.0 / d, device=dev, requires_grad=True)
            s2 = torch.tensor(3.0, dtype=torch.float64, requires_grad=True)
        J2 = G.mean_pce(frames, w2, d, s2, q_train[:2], ctx)
        J2.backward()
        gw2 = w2.grad.double().cpu().numpy()
        out["cpu_baseline"] = {"value": m / t_or, "unit": "frames/s", "cores": O.threads(), "kind": "oracle",
                               "sample": "one forward + adjoint of the whole workload with 2 queries",
                               "seconds": t_or}
        out["oracle_parity"] = {"J_rel": abs(J2.item() - oJ) / abs(oJ),
                                "g_w_relL2": float(np.linalg.norm(gw2 - ogw) / np.linalg.norm(ogw)),
                                "g_sigma0_rel": abs(float(s2.grad) - ogs) / abs(ogs)}
    # 50 ascent steps on the training queries' mean PCE
    opt = torch.optim.Adam([{"params": [w], "lr": 2e-3}, {"params": [sig], "lr": 5e-2}])
    with torch.no_grad():
        ev0 = G.mean_pce(frames, w, d, sig, q_eval, ctx).item()
    traj = []
    for it in range(50):
        opt.zero_grad()
        J = G.mean_pce(frames, w, d, sig, q_train, ctx)
        (-J).backward()
        opt.step()
        traj.append(J.item())
    with torch.no_grad():
        J_end = G.mean_pce(frames, w, d, sig, q_train, ctx).item()
        ev1 = G.mean_pce(frames, w, d, sig, q_eval, ctx).item()
    out["ascent"] = {"steps": 50, "optimizer": "Adam (lr 2e-3 weights, 5e-2 sigma0)",
                     "pce_train_start": traj[0], "pce_train_end": J_end, "pce_eval_start": ev0, "pce_eval_end": ev1,
                     "sigma0_end": float(sig.detach()), "w_min": float(w.detach().min()),
                     "w_max": float(w.detach().max()), "w_mean": float(w.detach().mean()), "trajectory_every_10": traj[::10]}
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()


# --------------------------------------------------------------- GPU arm ---
def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        reference_arm(args, rank)
        return
    if args.config == "precision":
        precision_config(args, rank, world, local)
        return
    if args.config == "depth":
        depth_config(args, rank, world, local)
        return
    if args.config == "batch":
        batch_config(args, rank, world, local)
        return
    if args.config == "grad":
        grad_config(args, rank, world, local)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_1909_04573_gb300 import prnu as P
    from paper_1909_04573_gb300 import synth

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    dev = torch.device("cuda", local)
    ctx = P.Context(local)

    m_frames = args.frames
    shard_mode = args.mode == "shard" and world > 1
    cam = synth.Camera(H=H, W=W, C=C, camera_id=0 if args.mode == "shard" else rank)
    frames = synth.frames(cam, m_frames, device=dev, drift_px=2.0)        # 6.22 GB resident at 1000 frames
    qf = torch.cat([synth.frames(cam, N_QUERY, stream=1, device=dev),
                    synth.frames(synth.foreign(cam), N_QUERY, stream=1, device=dev)])
    qimg = ctx.sda_average(qf, 1)                                         # [20, 3, H, W] float
    num = torch.zeros((C, H, W), dtype=torch.float32, device=dev)
    den = torch.zeros_like(num)
    flags = P.PRNU_TO_GRAY | P.PRNU_ZERO_MEAN | P.PRNU_WIENER_DFT
    # the step's PCE / NCC / peaks stay on the device (no synchronisation
    # inside a step); they are read back once after the timed region
    pout = (torch.empty(2 * N_QUERY, dtype=torch.float64, device=dev),
            torch.empty(2 * N_QUERY, dtype=torch.float64, device=dev),
            torch.empty((2 * N_QUERY, 2), dtype=torch.int32, device=dev))

    from paper_1909_04573_gb300 import shard

    prm = P.default_params(sda_fusion=args.sda_fusion)

    def step(d=D_SDA, images_per_pass=None):
        num.zero_()
        den.zero_()
        if shard_mode:
            shard.accumulate_sharded(
                lambda f, dd, a, b: ctx.fingerprint_accumulate(f, dd, a, b, params=prm,
                                                               images_per_pass=images_per_pass),
                frames, d, num, den, rank, world)
        else:
            ctx.fingerprint_accumulate(frames, d, num, den, params=prm, images_per_pass=images_per_pass)
        K = ctx.fingerprint_finalize(num, den, flags)
        ctx.pce_match_images_async(K[0], qimg, out=pout)

    # The queries' denoising does not involve K: on the single-GPU camera path
    # it runs on a side stream (own context and workspace) while the
    # fingerprint is extracted, and only the grey level-1 synthesis + PCE wait
    # for K.  Same kernels and results as step().
    qctx = P.Context(local)
    side = torch.cuda.Stream(device=dev)

    def step_forked():
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            qctx.pce_images_prepare(qimg)
        num.zero_()
        den.zero_()
        ctx.fingerprint_accumulate(frames, D_SDA, num, den, params=prm)
        K = ctx.fingerprint_finalize(num, den, flags)
        torch.cuda.current_stream().wait_stream(side)
        qctx.pce_images_finish_async(K[0], qimg, out=pout)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        if world > 1:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
            dist.barrier()
        return ms

    # ---- level-1 analysis launch shape for this geometry (outside the timed region)
    g_pass = (m_frames + D_SDA - 1) // D_SDA
    shape, t_shape = ctx.autotune(H, W, C, images=min(g_pass, 20))
    tuned = {f"{W}x{H}": {"strip_rows": shape[0], "warps": shape[1], "ms": t_shape}}
    qctx.autotune(H, W, C, images=min(g_pass, 20))

    # ---- SDA path, timed with per-kernel events on the launch stream.
    # Single-GPU camera path: the K timed steps are captured once in a CUDA
    # graph and the timed region is one replay of it (after one untimed
    # replay).  Events become event nodes of the graph and cost about 3 us
    # each, so the timed replay brackets only the roofline kernels; the
    # per-kernel table comes from a replay of a second capture of the same K
    # steps with every launch bracketed.  The sharded accumulate (collectives
    # across ranks) runs eagerly, every launch bracketed.
    use_graph = not shard_mode and not args.no_graph
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    eager_pce = pout[0].cpu().tolist()
    gs = torch.cuda.Stream(device=dev)

    def capture(timed_kernels, fn=step, profile=True):
        P.prnu_profile_reset(ctx.ctx)
        P.prnu_profile_select(ctx.ctx, timed_kernels)
        P.prnu_profile_enable(ctx.ctx, profile)
        g = torch.cuda.CUDAGraph()
        gs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(g, stream=gs):
            for _ in range(args.steps):
                fn()
        P.prnu_profile_enable(ctx.ctx, False)
        torch.cuda.synchronize()
        g.replay()                                  # untimed
        torch.cuda.synchronize()
        return g

    kern_all = None
    if use_graph:
        g_all = capture(None)
        timed(g_all.replay, 1, 0)
        prof_all = P.prnu_profile_read(ctx.ctx)
        del g_all
        torch.cuda.synchronize()
        _, _, kern_all, _ = kernel_report(prof_all, args.steps, None, dev)
        dominant = max((k for k in prof_all if not k.startswith("cufft")), key=lambda k: prof_all[k][1])
        graph = capture([dominant, "sda_sum"])
        body, n_body = graph.replay, 1
    else:
        P.prnu_profile_reset(ctx.ctx)
        P.prnu_profile_enable(ctx.ctx, True)
        body, n_body = step, args.steps
    clocks = Clocks(local)
    clocks.start()
    if args.profile_range:
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
    ms = timed(body, n_body, 0) * n_body / args.steps
    if args.profile_range:
        torch.cuda.profiler.stop()
    ck = clocks.stop()
    P.prnu_profile_enable(ctx.ctx, False)
    prof = P.prnu_profile_read(ctx.ctx)
    if use_graph:
        del graph, body
        torch.cuda.synchronize()
    P.prnu_profile_reset(ctx.ctx)
    P.prnu_profile_select(ctx.ctx, None)
    frames_per_step = m_frames if shard_mode else world * m_frames
    value = frames_per_step / (ms / 1000.0)
    pces = pout[0].cpu().tolist()
    assert np.allclose(pces, eager_pce, rtol=1e-9, atol=0.0), "graph replay changed the PCE"
    pos = [p for p in pces[:N_QUERY]]
    neg = [p for p in pces[N_QUERY:]]

    # the timed step's fingerprint sums, kept for the parity check against the
    # oracle (the later forms of the step reuse num / den)
    gpu_par = None
    if not shard_mode and not args.no_cpu and rank == 0 and world == 1:
        K0 = ctx.fingerprint_finalize(num, den, 0)
        res0 = ctx.denoise_residual(ctx.sda_average(frames[:D_SDA], D_SDA)[0])
        torch.cuda.synchronize()
        gpu_par = {"num": num.cpu().numpy(), "den": den.cpu().numpy(), "K": K0.cpu().numpy(),
                   "res0": res0.cpu().numpy()}
        del K0, res0

    roof, sda_roof, kern, launches = kernel_report(prof, args.steps, ck, dev)
    if kern_all is not None:
        kern = kern_all
    hbm, _ = peaks()
    step_bytes = m_frames * H * W * C
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if args.mode == "shard" else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded sensor model; VISION/NYUAD-MMD absent)",
            "config": {"workload": WORKLOAD if m_frames == M_FRAMES else f"video-1080p-rgb-{m_frames}f-sda50",
                       "frames": m_frames, "H": H, "W": W, "C": C, "d": D_SDA,
                       "queries": 2 * N_QUERY,
                       "parallelism": (f"1 camera sharded by SDA groups over {world} GPUs" if args.mode == "shard"
                                       else f"1 camera per GPU x {world}"),
                       "l2": "inputs 6.22 GB > 129 MB L2 (no flush)",
                       "launch": (f"one CUDA graph of {args.steps} steps, one replay timed; events around "
                                  f"{roof['kernel'] if roof else '?'} and sda_sum only (the kernel table is from "
                                  "a second capture with every launch timed)" if use_graph
                                  else "eager launches, every launch timed")},
            "frame_GBps": step_bytes / (ms / 1000.0) / 1e9,
            "frame_frac_of_peak": step_bytes / (ms / 1000.0) / 1e9 / hbm,
            "roofline": roof, "roofline_sda_sum": sda_roof, "gpu_launches": int(launches), "kernels": kern,
            "autotune": tuned,
            "pce": {"same_camera_min": min(pos), "foreign_max_abs": max(abs(x) for x in neg)}}
    if ck:
        line["clocks"] = ck

    # ---- the same step with the queries' denoising on a second stream while
    # the fingerprint is extracted (prepare / finish split); no profiler events
    if use_graph:
        g_fork = capture(None, fn=step_forked, profile=False)
        ms_fork = timed(g_fork.replay, 1, 0) / args.steps
        same = bool(np.allclose(pout[0].cpu().tolist(), pces, rtol=1e-9, atol=0.0))
        del g_fork
        torch.cuda.synchronize()
        P.prnu_profile_reset(ctx.ctx)
        line["queries_overlapped"] = {"value": frames_per_step / (ms_fork / 1000.0), "unit": UNIT,
                                      "ms_per_step": ms_fork, "same_pce": same,
                                      "mode": "queries denoised on a second stream during the extraction "
                                              "(prnu_pce_images_prepare / _finish_async), one graph replay"}

    # ---- extraction alone (accumulate + finalize of the fingerprint, no
    # queries): its frame bytes against the copy peak
    if use_graph:
        def extraction_ms(p):
            def extract():
                num.zero_()
                den.zero_()
                ctx.fingerprint_accumulate(frames, D_SDA, num, den, params=p)
                ctx.fingerprint_finalize(num, den, flags)
            g_ex = capture(None, fn=extract, profile=False)
            ms_ = timed(g_ex.replay, 1, 0) / args.steps
            del g_ex
            torch.cuda.synchronize()
            P.prnu_profile_reset(ctx.ctx)
            return ms_
        ms_ex = extraction_ms(prm)
        ex_gbps = step_bytes / (ms_ex / 1000.0) / 1e9
        line["extraction"] = {"value": frames_per_step / (ms_ex / 1000.0), "unit": UNIT, "ms_per_step": ms_ex,
                              "frame_GBps": ex_gbps, "frame_frac_of_peak": ex_gbps / hbm,
                              "sda_fusion": args.sda_fusion,
                              "mode": "accumulate (SDA-50 sums, denoise, MLE) + finalize (grey, zero-mean, DFT "
                                      "Wiener) of the step's fingerprint, without the queries; one graph replay"}
        # A/B: the same extraction with the other form of the group sums
        alt = P.PRNU_SDA_SEPARATE if args.sda_fusion != P.PRNU_SDA_SEPARATE else 0
        ms_alt = extraction_ms(P.default_params(sda_fusion=alt))
        line["extraction"]["other_sda_form"] = {"sda_fusion": alt, "ms_per_step": ms_alt,
                                                "value": frames_per_step / (ms_alt / 1000.0)}

    # ---- per-frame (ALL-FE) comparison: d = 1, 1000 denoise passes x 3 channels
    if not args.no_perframe:
        ms_pf = timed(lambda: step(d=1, images_per_pass=100), 2, 1)
        line["perframe"] = {"value": frames_per_step / (ms_pf / 1000.0), "unit": UNIT, "ms_per_step": ms_pf,
                            "sda_speedup": ms_pf / ms,
                            "paper_context": "Sec. V-B: SDA-50 29.3x and SDA-1200 52.1x faster than denoising "
                                             "every frame of a ~1200-frame Full HD video (1407 s), one Matlab "
                                             "thread on a Xeon E5-2687W v2, decoding and disk reads included"}

    # ---- end to end through the host-buffer entry point
    if not args.no_e2e:
        host = frames.cpu().pin_memory()
        qhost = qf.cpu().pin_memory()
        del frames
        torch.cuda.empty_cache()
        qdev = torch.empty_like(qf)
        # the queries do not need K until their PCE: their copy, conversion and
        # residuals run on a side stream (own context, own workspace) while the
        # fingerprint's frames stream over the host link

        qi_e2e = torch.empty_like(qimg)
        pout_host = tuple(torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in pout)

        def step_e2e():
            num.zero_()
            den.zero_()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                qdev.copy_(qhost, non_blocking=True)
                qi_e2e.copy_(qctx.sda_average(qdev, 1))
                qctx.pce_images_prepare(qi_e2e)
            ctx.fingerprint_accumulate_host(host, D_SDA, num, den, groups_per_pass=4)
            K = ctx.fingerprint_finalize(num, den, flags)
            torch.cuda.current_stream().wait_stream(side)
            qctx.pce_images_finish_async(K[0], qi_e2e, out=pout)
            for hst, dv in zip(pout_host, pout):
                hst.copy_(dv, non_blocking=True)

        ms_e2e = timed(step_e2e, 3, 1)
        # raw pinned H2D bandwidth of one 1 GiB copy, for context
        probe = torch.empty(1 << 30, dtype=torch.uint8, device=dev)
        src = host.view(-1)[: 1 << 30]
        probe.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        probe.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        h2d_gbps = (1 << 30) / (e0.elapsed_time(e1) / 1000.0) / 1e9
        del probe
        h2d = host.numel() + qhost.numel()
        d2h = sum(t.numel() * t.element_size() for t in pout)
        line["e2e"] = {"value": world * m_frames / (ms_e2e / 1000.0), "unit": UNIT, "ms_per_step": ms_e2e,
                       "mode": "one camera per GPU through the host-buffer entry point (page-locked frames read "
                               "in place); the queries' copy and denoising on a side stream during the frame "
                               "reads; PCE / NCC / peaks read back to pinned host memory every step",
                       "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                       "pinned_h2d_GBps": h2d_gbps}
        frames_host = host.numpy()
    else:
        frames_host = frames.cpu().numpy()

    # ---- CPU baseline: the FP64 oracle on a bounded sample, rank 0 at N = 1
    if rank == 0 and world == 1 and not args.no_cpu:
        groups = (m_frames + D_SDA - 1) // D_SDA
        t, n, cores, onum, oden = oracle_sample(frames_host, groups, sums=True)
        if gpu_par is not None:
            line["parity"] = headline_parity(gpu_par, frames_host, onum, oden)
        t1 = oracle_sample_1core(frames_host)
        line["cpu_baseline"] = {"value": n / t, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "value_1core": 1.0 / t1,
                                "sample": f"the whole SDA-{D_SDA} fingerprint of the step ({groups} groups, "
                                          f"{n} 1080p RGB frames): means, 3 residuals per group, MLE sums "
                                          "(not the queries' PCE); 1-core figure: a 10-frame group timed the same "
                                          "way",
                                "seconds": t}
    if rank == 0:
        print(json.dumps(line), flush=True)
    qctx.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    del np
    if "parity" in line and not line["parity"]["pass"]:
        sys.exit("parity against the FP64 oracle failed at the timed configuration: " +
                 json.dumps({k: v for k, v in line["parity"].items() if k != "sample"}))


if __name__ == "__main__":
    main()
