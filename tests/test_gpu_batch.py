"""Multi-camera batches (ragged frame counts, resolutions, SDA group sizes)
and CUDA-graph capture of the whole accumulate + finalize sequence (GPU)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1909_04573_gb300 import prnu as P
from paper_1909_04573_gb300 import synth

pytestmark = pytest.mark.gpu

SPECS = [  # (H, W, C, m, d): two geometries, ragged last groups, d = m, d = 1
    (64, 96, 3, 13, 4), (80, 112, 1, 30, 10), (64, 96, 3, 7, 7), (80, 112, 1, 25, 3), (64, 96, 3, 41, 6),
    (64, 96, 3, 5, 1),
]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04573_gb300 import build
    build.build()
    c = P.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def cams():
    out = []
    for i, (H, W, C, m, d) in enumerate(SPECS):
        fr = synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=300 + i), m, device="cuda", drift_px=1.0)
        out.append((fr, d))
    return out


def _zeros(fr):
    num = torch.zeros((fr.shape[3], fr.shape[1], fr.shape[2]), device="cuda")
    return num, torch.zeros_like(num)


def _rel(a, b):
    return float((a - b).norm() / b.norm())


@pytest.mark.parametrize("groups_per_pass", [64, 2])
def test_multi_camera_equals_single_calls(ctx, cams, groups_per_pass):
    items, refs = [], []
    for fr, d in cams:
        n, dd = _zeros(fr)
        items.append((fr, d, n, dd))
        rn, rd = _zeros(fr)
        ctx.fingerprint_accumulate(fr, d, rn, rd)
        refs.append((rn, rd))
    ctx.fingerprint_accumulate_multi(items, groups_per_pass=groups_per_pass)
    torch.cuda.synchronize()
    for (fr, d, n, dd), (rn, rd) in zip(items, refs):
        assert _rel(n, rn) <= 1e-6 and _rel(dd, rd) <= 1e-6


def test_multi_camera_matches_oracle(ctx, cams):
    fr, d = cams[4]
    n, dd = _zeros(fr)
    items = [(c[0], c[1], *_zeros(c[0])) for c in cams]
    items[4] = (fr, d, n, dd)
    ctx.fingerprint_accumulate_multi(items)
    onum, oden = O.fingerprint_accumulate(fr.cpu().numpy(), d)
    assert float(np.linalg.norm(n.cpu().numpy() - onum) / np.linalg.norm(onum)) <= 1e-5
    assert float(np.linalg.norm(dd.cpu().numpy() - oden) / np.linalg.norm(oden)) <= 1e-6


def test_cuda_graph_capture_and_replay(ctx, cams):
    items = [(fr, d, *_zeros(fr)) for fr, d in cams]
    flags = P.PRNU_ZERO_MEAN | P.PRNU_WIENER_DFT
    # eager reference (also creates the cuFFT plans the graph will use)
    ctx.fingerprint_accumulate_multi(items)
    eager = [ctx.fingerprint_finalize(n, dd, flags).clone() for _, _, n, dd in items]
    Ks = [torch.empty_like(e) for e in eager]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        cams_c = ctx.cameras(items)
        p = P.default_params()
        nbytes = P.prnu_workspace_size_multi(ctx.ctx, cams_c, p, 64)
        ws = ctx.workspace(max(nbytes, P.prnu_workspace_size(ctx.ctx, 80, 112, 3, p, 1)))
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=side):
            for _, _, n, dd in items:
                n.zero_()
                dd.zero_()
            P.prnu_fingerprint_accumulate_multi(ctx.ctx, cams_c, p, ws.data_ptr(), ws.numel(), side.cuda_stream)
            for (_, _, n, dd), K in zip(items, Ks):
                C, H, W = n.shape
                P.prnu_fingerprint_finalize(ctx.ctx, n.data_ptr(), dd.data_ptr(), H, W, C, flags, p, K.data_ptr(),
                                            ws.data_ptr(), ws.numel(), side.cuda_stream)
    for _ in range(2):
        for K in Ks:
            K.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for K, e in zip(Ks, eager):
            assert torch.isfinite(K).all()
            assert _rel(K, e) <= 1e-6


def test_batch_resolutions_full_size_match_oracle(ctx):
    """The three resolutions of the 32-camera workload at full size, with the
    bench's launch configuration (32 groups per pass, autotuned level-1
    shapes, accumulate captured in a CUDA graph and replayed), against the
    oracle; then the PCE of one camera on the common 1280x720 window."""
    specs = [(synth.Camera(H=720, W=1280, C=3, camera_id=2900), 23, 10),
             (synth.Camera(H=1080, W=1920, C=3, camera_id=2901), 25, 12),
             (synth.Camera(H=3024, W=4032, C=3, camera_id=2902), 12, 10)]
    prm = P.default_params()
    for c, _, _ in specs:
        ctx.autotune(c.H, c.W, 3, prm, images=2)
    items = []
    for c, m, d in specs:
        fr = synth.frames_fast(c, m, device="cuda")
        items.append((fr, d, *_zeros(fr)))
    cams_c = ctx.cameras(items)
    nbytes = P.prnu_workspace_size_multi(ctx.ctx, cams_c, prm, 32)
    ws = ctx.workspace(nbytes)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            P.prnu_fingerprint_accumulate_multi(ctx.ctx, cams_c, prm, ws.data_ptr(), ws.numel(), side.cuda_stream)
    torch.cuda.current_stream().wait_stream(side)
    g.replay()
    torch.cuda.synchronize()
    for fr, d, n, dd in items:
        onum, oden = O.fingerprint_accumulate(fr.cpu().numpy(), d)
        assert float(np.linalg.norm(n.cpu().numpy() - onum) / np.linalg.norm(onum)) <= 1e-5
        assert float(np.linalg.norm(dd.cpu().numpy() - oden) / np.linalg.norm(oden)) <= 1e-6
    # PCE of the 4032x3024 camera's fingerprint against its own query, top-left 1280x720
    c, _, _ = specs[2]
    fr, d, n, dd = items[2]
    K = ctx.fingerprint_finalize(n, dd, P.PRNU_TO_GRAY)[0, :720, :1280].contiguous()
    qf = synth.frames_fast(c, 1, stream=1, device="cuda")
    q = ctx.sda_average(qf, 1)[0, :, :720, :1280].contiguous()
    wq = ctx.denoise_residual(q)
    pce = ctx.pce_match(K, wq, q)[0]
    onum, oden = O.fingerprint_accumulate(fr.cpu().numpy(), d)
    oK = O.fingerprint_finalize(onum, oden, O.TO_GRAY)[0, :720, :1280]
    qh = O.sda_average(qf.cpu().numpy(), 1)[0][:, :720, :1280]
    opce = O.pce_match(oK, O.to_gray(O.residual(qh)), O.to_gray(qh)).pce
    assert opce > 60
    assert abs(pce - opce) <= 1e-3 * abs(opce)
