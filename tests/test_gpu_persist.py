"""The persistent multi-camera pipeline (one launch over a device work queue)
against the per-stage multi-camera path and the FP64 oracle, its CUDA-graph
capture, and its bounded device-side waits (GPU)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1909_04573_gb300 import prnu as P
from paper_1909_04573_gb300 import synth

pytestmark = pytest.mark.gpu

SPECS = [  # (H, W, C, m, d): two geometries (RGB and grey), ragged last groups, d = m, d = 1
    (64, 96, 3, 13, 4), (80, 112, 1, 30, 10), (64, 96, 3, 7, 7), (80, 112, 1, 25, 3), (64, 96, 3, 41, 6),
    (64, 96, 3, 5, 1), (37, 50, 3, 9, 2),
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
        fr = synth.frames(synth.Camera(H=H, W=W, C=C, camera_id=400 + i), m, device="cuda", drift_px=1.0)
        out.append((fr, d))
    return out


def _zeros(fr, comp=False):
    shape = (fr.shape[3], fr.shape[1], fr.shape[2])
    num = torch.zeros((2, *shape) if comp else shape, device="cuda")
    return num, torch.zeros_like(num)


def _rel(a, b):
    return float((a - b).norm() / b.norm())


@pytest.mark.parametrize("slots", [3, 5])
def test_persistent_equals_per_stage_multi_camera(ctx, cams, slots):
    items, refs = [], []
    for fr, d in cams:
        items.append((fr, d, *_zeros(fr)))
        refs.append((fr, d, *_zeros(fr)))
    ctx.fingerprint_accumulate_multi(refs)
    ctx.fingerprint_accumulate_persistent(items, slots=slots)
    torch.cuda.synchronize()
    for (_, _, n, dd), (_, _, rn, rd) in zip(items, refs):
        assert torch.isfinite(n).all()
        assert _rel(n, rn) <= 1e-6 and _rel(dd, rd) <= 1e-6


def test_persistent_matches_oracle(ctx, cams):
    items = [(fr, d, *_zeros(fr)) for fr, d in cams]
    ctx.fingerprint_accumulate_persistent(items)
    for fr, d, n, dd in items:
        onum, oden = O.fingerprint_accumulate(fr.cpu().numpy(), d)
        assert float(np.linalg.norm(n.cpu().numpy() - onum) / np.linalg.norm(onum)) <= 1e-5
        assert float(np.linalg.norm(dd.cpu().numpy() - oden) / np.linalg.norm(oden)) <= 1e-6
        K = ctx.fingerprint_finalize(n, dd).cpu().numpy()
        assert float(np.linalg.norm(K - O.fingerprint_finalize(onum, oden)) /
                     np.linalg.norm(O.fingerprint_finalize(onum, oden))) <= 1e-5


def test_persistent_compensated_and_other_windows(ctx, cams):
    # compensated num/den pairs, and a non-standard window set (generic shrink tile)
    for params, comp in ((P.default_params(compensated=True), True), (P.default_params(windows=(5, 9)), False)):
        items = [(fr, d, *_zeros(fr, comp)) for fr, d in cams[:4]]
        refs = [(fr, d, *_zeros(fr, comp)) for fr, d in cams[:4]]
        ctx.fingerprint_accumulate_multi(refs, params=params)
        ctx.fingerprint_accumulate_persistent(items, params=params)
        for (_, _, n, dd), (_, _, rn, rd) in zip(items, refs):
            if comp:
                n, dd, rn, rd = (t[0].double() + t[1] for t in (n, dd, rn, rd))
            assert _rel(n, rn) <= 1e-6 and _rel(dd, rd) <= 1e-6


def test_persistent_graph_capture_and_replay(ctx, cams):
    items = [(fr, d, *_zeros(fr)) for fr, d in cams]
    ctx.fingerprint_accumulate_persistent(items)  # eager (also sizes the workspace)
    torch.cuda.synchronize()
    eager = [(n.clone(), dd.clone()) for _, _, n, dd in items]
    prm = P.default_params()
    cams_c = ctx.cameras(items)
    nbytes = P.prnu_workspace_size_persistent(ctx.ctx, cams_c, prm, 4)
    ws = ctx.workspace(nbytes)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            for _, _, n, dd in items:
                n.zero_()
                dd.zero_()
            P.prnu_fingerprint_accumulate_persistent(ctx.ctx, cams_c, prm, 4, 2000.0, ws.data_ptr(), nbytes,
                                                     side.cuda_stream)
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):
        for _, _, n, dd in items:
            n.fill_(float("nan"))
        g.replay()
        st, _ = P.prnu_persistent_status(ctx.ctx, ws.data_ptr(), nbytes, torch.cuda.current_stream().cuda_stream)
        assert st == P.PRNU_OK
        for (_, _, n, dd), (en, ed) in zip(items, eager):
            assert _rel(n, en) <= 1e-6 and _rel(dd, ed) <= 1e-6


def test_bounded_wait_gives_up_and_the_context_stays_usable(ctx, cams):
    """A queue item whose dependency nothing satisfies: its wait gives up
    after the budget, the status reads PRNU_ETIMEOUT, and the next launch
    works."""
    ws = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    P.prnu_persistent_wait_probe(ctx.ctx, 50.0, ws.data_ptr(), ws.numel(), stream)
    st, info = P.prnu_persistent_status(ctx.ctx, ws.data_ptr(), ws.numel(), stream)
    assert st == P.PRNU_ETIMEOUT
    assert info[0] == 0 and info[1] == 0
    msg = P.lib().prnu_last_error(ctx.ctx).decode()
    assert "gave up" in msg
    # the GPU and the context still work: a regular persistent call succeeds
    items = [(fr, d, *_zeros(fr)) for fr, d in cams[:2]]
    refs = [(fr, d, *_zeros(fr)) for fr, d in cams[:2]]
    ctx.fingerprint_accumulate_persistent(items)
    ctx.fingerprint_accumulate_multi(refs)
    for (_, _, n, dd), (_, _, rn, rd) in zip(items, refs):
        assert _rel(n, rn) <= 1e-6


def test_persistent_rejects_what_it_does_not_take(ctx, cams):
    fr, d = cams[0]
    with pytest.raises(P.PrnuError) as e:
        ctx.fingerprint_accumulate_persistent([(fr, d, *_zeros(fr))], params=P.default_params(dtype=P.PRNU_DTYPE_F16))
    assert e.value.status == P.PRNU_EUNSUPPORTED
    with pytest.raises(P.PrnuError) as e:
        ctx.fingerprint_accumulate_persistent([(fr, d, *_zeros(fr))], slots=2)
    assert e.value.status == P.PRNU_EINVAL
    n, dd = _zeros(fr)
    with pytest.raises(P.PrnuError) as e:
        ctx.fingerprint_accumulate_persistent([(fr, d, n, dd), (fr, d, n, dd)])
    assert e.value.status == P.PRNU_EINVAL


def test_persistent_full_size_resolutions_match_oracle(ctx):
    """The three resolutions of the multi-camera workload at full size in one
    persistent launch (captured in a graph and replayed), against the oracle."""
    specs = [(synth.Camera(H=720, W=1280, C=3, camera_id=2910), 23, 10),
             (synth.Camera(H=1080, W=1920, C=3, camera_id=2911), 25, 12),
             (synth.Camera(H=3024, W=4032, C=3, camera_id=2912), 12, 10)]
    items = []
    for c, m, d in specs:
        fr = synth.frames_fast(c, m, device="cuda")
        items.append((fr, d, *_zeros(fr)))
    prm = P.default_params()
    cams_c = ctx.cameras(items)
    nbytes = P.prnu_workspace_size_persistent(ctx.ctx, cams_c, prm, 4)
    ws = ctx.workspace(nbytes)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            P.prnu_fingerprint_accumulate_persistent(ctx.ctx, cams_c, prm, 4, 2000.0, ws.data_ptr(), nbytes,
                                                     side.cuda_stream)
    torch.cuda.current_stream().wait_stream(side)
    g.replay()
    st, info = P.prnu_persistent_status(ctx.ctx, ws.data_ptr(), nbytes, torch.cuda.current_stream().cuda_stream)
    assert st == P.PRNU_OK, info
    for fr, d, n, dd in items:
        onum, oden = O.fingerprint_accumulate(fr.cpu().numpy(), d)
        assert float(np.linalg.norm(n.cpu().numpy() - onum) / np.linalg.norm(onum)) <= 1e-5
        assert float(np.linalg.norm(dd.cpu().numpy() - oden) / np.linalg.norm(oden)) <= 1e-6
