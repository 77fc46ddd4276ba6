"""The seeded generator follows the stated sensor-model recipe (CPU): scene
mean 128 / std 40 after a Gaussian low-pass, K ~ N(0, 0.005^2) i.i.d. and
fixed per camera, read noise N(0, sigma_read^2), deterministic seeding with
independent streams, and a drifting scene that stays correlated from frame
to frame."""
import dataclasses

import numpy as np
import torch

from paper_1909_04573_gb300 import synth


def _cam(**kw):
    base = dict(H=128, W=160, C=1, camera_id=5)
    base.update(kw)
    return synth.Camera(**base)


def test_scene_statistics_and_smoothness():
    cam = _cam(k_std=0.0, sigma_read=0.0)
    f = synth.frames(cam, 3).numpy()[..., 0].astype(np.float64)
    for s in f:
        assert abs(s.mean() - 128.0) < 1.0 and abs(s.std() - 40.0) < 1.0
        # sigma = 8 px Gaussian low-pass: neighbours are almost equal
        r = np.corrcoef(s[:, :-1].ravel(), s[:, 1:].ravel())[0, 1]
        assert r > 0.98
    # independent scenes per frame without drift
    assert abs(np.corrcoef(f[0].ravel(), f[1].ravel())[0, 1]) < 0.3


def test_prnu_distribution_and_identity():
    cam = _cam(H=256, W=256)
    K = synth.k_true(cam).numpy()
    assert abs(K.std() - 0.005) < 0.0001 and abs(K.mean()) < 0.0001
    np.testing.assert_array_equal(K, synth.k_true(cam).numpy())
    Kf = synth.k_true(synth.foreign(cam)).numpy()
    assert abs(np.corrcoef(K.ravel(), Kf.ravel())[0, 1]) < 0.02


def test_read_noise_level():
    # same seeds with and without read noise: the frames differ by the noise
    # (plus rounding) only
    cam = _cam()
    quiet = dataclasses.replace(cam, sigma_read=0.0)
    a = synth.frames(cam, 2).numpy().astype(np.float64)
    b = synth.frames(quiet, 2).numpy().astype(np.float64)
    sd = (a - b).std()
    assert 1.9 < sd < 2.2


def test_seeding_streams_and_chunks():
    cam = _cam(C=3, H=48, W=64)
    a = synth.frames(cam, 4, drift_px=2.0)
    assert torch.equal(a, synth.frames(cam, 4, drift_px=2.0))
    assert not torch.equal(a, synth.frames(cam, 4, stream=1, drift_px=2.0))
    # a chunk starting at frame 2 reproduces frames 2..3
    assert torch.equal(a[2:], synth.frames(cam, 2, drift_px=2.0, start=2))


def test_drifting_scene_stays_correlated():
    cam = _cam(k_std=0.0, sigma_read=0.0)
    f = synth.frames(cam, 6, drift_px=2.0).numpy()[..., 0].astype(np.float64)
    for j in range(5):
        assert np.corrcoef(f[j].ravel(), f[j + 1].ravel())[0, 1] > 0.9
