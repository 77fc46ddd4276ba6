"""prnu_pce_match_pairs against the FP64 oracle at the geometries it serves.

Two uses of the pairs entry point (each query against its own fingerprint
plane):
* a 4 x 4 slice of the multi-camera PCE matrix on the common top-left
  1280 x 720 window of RGB cameras;
* block-wise matching, Sec. IV-A: a 1000 x 1000 fingerprint split into four
  disjoint 500 x 500 blocks, each correlated with the same block of a query.

For each pair the CUDA PCE is compared with ``oracle.pce_match`` on the same
float32 inputs (fingerprint block, query residual, query image) within 0.1 %,
the peak position exactly where the correlation peak is unique (true pairs:
zero shift), and otherwise checked to be a valid maximiser of the oracle's
correlation within float32 rounding.  The whole chain is also compared with
the oracle's own fingerprint and residuals (PCE within 0.1 %).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1909_04573_gb300 import prnu as P
from paper_1909_04573_gb300 import synth

pytestmark = pytest.mark.gpu

PCE_TOL = 1e-3
FLAGS = P.PRNU_TO_GRAY | P.PRNU_ZERO_MEAN | P.PRNU_WIENER_DFT


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04573_gb300 import build
    build.build()
    c = P.Context(0)
    yield c
    c.close()


def _pce_tol(ref, true_pair):
    """0.1 % of the PCE; for an unrelated pair, whose C(0) sits at the noise
    level of the correlation (|PCE| ~ 1), the float32 rounding of C(0) is
    ~3e-4 of it at a megapixel, so the bound gets an absolute floor."""
    return PCE_TOL * abs(ref) if true_pair else PCE_TOL * max(abs(ref), 1.0) + 1e-3


def _check_pairs(K, Wq, Iq, got, true_pair):
    """K [n, H, W]; Wq, Iq [n, C, H, W] (float32 numpy, the CUDA inputs);
    got = [(pce, ncc, peak)]; true_pair[i]: same camera."""
    for i, (pce, ncc, peak) in enumerate(got):
        X = O.to_gray(Wq[i].astype(np.float64))
        I = O.to_gray(Iq[i].astype(np.float64))
        r = O.pce_match(K[i].astype(np.float64), X, I)
        assert abs(pce - r.pce) <= _pce_tol(r.pce, true_pair[i]), (i, pce, r.pce)
        assert abs(ncc - r.ncc) <= 1e-4 * abs(r.ncc) + 2e-6, (i, ncc, r.ncc)
        if true_pair[i]:
            assert r.pce > 60 and pce > 60
            assert peak == r.peak == (0, 0)
        else:
            assert abs(pce) < 60 and abs(r.pce) < 60
            # the maximum of a noise correlation may be a near tie: the CUDA
            # peak must be a maximiser of the oracle's correlation to within
            # float32 rounding of the correlation values
            Xc = X - X.mean()
            Y = K[i].astype(np.float64) * I
            Cr = O.cross_correlation(Xc, Y - Y.mean())
            slack = 1e-5 * float(np.sqrt(np.mean(Cr ** 2))) * np.sqrt(Cr.size)
            assert Cr[peak] >= Cr.max() - slack, (i, peak, r.peak)


def test_pce_matrix_slice_on_1280x720_windows(ctx):
    """Rows of the 32 x 32 matrix of the multi-camera workload: 4 fingerprints
    (cameras of 1280x720, 1920x1080 and 4032x3024 RGB) against 4 queries, all
    cropped to the common top-left 1280 x 720 window."""
    Hq, Wq = 720, 1280
    specs = [(720, 1280), (1080, 1920), (3024, 4032), (720, 1280)]
    cams = [synth.Camera(H=h, W=w, C=3, camera_id=3100 + i) for i, (h, w) in enumerate(specs)]
    Ks, Kos, qs, qres, qres_o = [], [], [], [], []
    for c in cams:
        fr = synth.frames_fast(c, 8, device="cuda")
        num = torch.zeros((3, c.H, c.W), device="cuda")
        den = torch.zeros_like(num)
        ctx.fingerprint_accumulate(fr, 4, num, den)
        K = ctx.fingerprint_finalize(num, den, FLAGS)[0, :Hq, :Wq].contiguous()
        Ks.append(K)
        if (c.H, c.W) == (Hq, Wq):  # the oracle's fingerprint of the window-sized cameras
            onum, oden = O.fingerprint_accumulate(fr.cpu().numpy(), 4)
            Kos.append(O.fingerprint_finalize(onum, oden, O.TO_GRAY | O.ZERO_MEAN | O.WIENER_DFT)[0])
        else:
            Kos.append(None)
        qf = synth.frames_fast(c, 1, stream=1, device="cuda")
        q = ctx.sda_average(qf, 1)[0, :, :Hq, :Wq].contiguous()
        qs.append(q)
        qres.append(ctx.denoise_residual(q).clone())
        qres_o.append(O.residual(q.cpu().numpy().astype(np.float64)))
    n = len(cams)
    # pairs (i, j): fingerprint i against query j, as one pairs call
    Kp = torch.stack([Ks[i] for i in range(n) for j in range(n)])
    Wp = torch.stack([qres[j] for i in range(n) for j in range(n)])
    Ip = torch.stack([qs[j] for i in range(n) for j in range(n)])
    got = ctx.pce_match_pairs(Kp, Wp, Ip)
    true_pair = [i == j for i in range(n) for j in range(n)]
    _check_pairs(Kp.cpu().numpy(), Wp.cpu().numpy(), Ip.cpu().numpy(), got, true_pair)
    # the whole chain against the oracle's own fingerprints and residuals
    # (the CUDA fingerprint of cameras larger than the window is built from
    # the whole frame, the oracle's from the window: compare the window camera)
    for i in (0, 3):
        for j in range(n):
            r = O.pce_match(Kos[i], O.to_gray(qres_o[j]), O.to_gray(qs[j].cpu().numpy().astype(np.float64)))
            pce = got[i * n + j][0]
            assert abs(pce - r.pce) <= _pce_tol(r.pce, i == j), (i, j, pce, r.pce)


def test_blockwise_500x500_pce(ctx):
    """Sec. IV-A: one 1000 x 1000 fingerprint split into four disjoint
    500 x 500 blocks, each matched against the same block of a same-camera
    query and of a foreign query (eight pairs in one call)."""
    H = W = 1000
    blk = 500
    cam = synth.Camera(H=H, W=W, C=3, camera_id=3200)
    fr = synth.frames(cam, 8, device="cuda")
    num = torch.zeros((3, H, W), device="cuda")
    den = torch.zeros_like(num)
    ctx.fingerprint_accumulate(fr, 4, num, den)
    K = ctx.fingerprint_finalize(num, den, FLAGS)[0]
    onum, oden = O.fingerprint_accumulate(fr.cpu().numpy(), 4)
    oK = O.fingerprint_finalize(onum, oden, O.TO_GRAY | O.ZERO_MEAN | O.WIENER_DFT)[0]
    qf = torch.cat([synth.frames(cam, 1, stream=1, device="cuda"),
                    synth.frames(synth.foreign(cam), 1, stream=1, device="cuda")])
    q = ctx.sda_average(qf, 1)
    wq = ctx.denoise_residual_batch(q)
    Kb, Wb, Ib, true_pair, ref = [], [], [], [], []
    for qi in range(2):
        qh = q[qi].cpu().numpy().astype(np.float64)
        wo = O.residual(qh)
        for by in range(H // blk):
            for bx in range(W // blk):
                ys, xs = slice(by * blk, (by + 1) * blk), slice(bx * blk, (bx + 1) * blk)
                Kb.append(K[ys, xs])
                Wb.append(wq[qi][:, ys, xs])
                Ib.append(q[qi][:, ys, xs])
                true_pair.append(qi == 0)
                ref.append(O.pce_match(oK[ys, xs], O.to_gray(wo[:, ys, xs]), O.to_gray(qh[:, ys, xs])).pce)
    Kb, Wb, Ib = (torch.stack(t).contiguous() for t in (Kb, Wb, Ib))
    got = ctx.pce_match_pairs(Kb, Wb, Ib)
    _check_pairs(Kb.cpu().numpy(), Wb.cpu().numpy(), Ib.cpu().numpy(), got, true_pair)
    for (pce, _, _), r, t in zip(got, ref, true_pair):   # the whole chain against the oracle's own
        assert abs(pce - r) <= _pce_tol(r, t), (pce, r)
