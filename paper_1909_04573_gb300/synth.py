"""Seeded synthetic cameras and frames (the stand-in for the paper's datasets).

The paper's experiments use the VISION and NYUAD-MMD datasets, which are not
available; frames here follow the sensor model of Sec. III-A, Eq. (1):

    I = I0 + I0 K + psi

* I0, the scene, per frame and channel: white N(0,1) noise, periodic Gaussian
  low-pass with standard deviation ``scene_sigma`` px (applied in the Fourier
  domain), standardised to mean 128 and standard deviation 40.
* K, the PRNU of one camera: N(0, k_std^2) i.i.d. per pixel and channel.
* psi: read noise N(0, sigma_read^2), then rounding and clipping to uint8.
* With ``drift_px > 0`` a frame sequence shares one scene per channel that
  drifts by a random-walk translation, each step uniform in
  [-drift_px, drift_px] along each axis, applied as an exact Fourier shift of
  the periodic scene (a video with a slowly panning view).

This module contains only input generation: none of the extraction method's
arithmetic.  Both the CUDA path and the oracle consume the same uint8 bytes.
Random draws come from torch generators seeded by (camera, stream, index), so a
given device and seed always give the same bytes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

BASE_SEED = 1909_04573


@dataclass(frozen=True)
class Camera:
    """One synthetic camera: its id selects its PRNU K."""
    H: int
    W: int
    C: int = 1
    camera_id: int = 0
    k_std: float = 0.005
    scene_sigma: float = 8.0
    scene_mean: float = 128.0
    scene_std: float = 40.0
    sigma_read: float = 2.0


def _gen(device, *key: int) -> torch.Generator:
    s = BASE_SEED
    for k in key:
        s = (s * 1_000_003 + int(k) + 0x9E3779B9) % (2 ** 62)
    g = torch.Generator(device=device)
    g.manual_seed(s)
    return g


def k_true(cam: Camera, device="cpu") -> torch.Tensor:
    """PRNU K of the camera: float32 [C, H, W] ~ N(0, k_std^2)."""
    g = _gen(device, 1, cam.camera_id)
    return torch.randn((cam.C, cam.H, cam.W), generator=g, device=device, dtype=torch.float32) * cam.k_std


def _lowpass_spectrum(cam: Camera, g: torch.Generator, device) -> torch.Tensor:
    """rfft2 of a standardised low-passed white field, float64 -> complex128."""
    H, W = cam.H, cam.W
    white = torch.randn((H, W), generator=g, device=device, dtype=torch.float64)
    fy = torch.fft.fftfreq(H, device=device, dtype=torch.float64)[:, None]
    fx = torch.fft.rfftfreq(W, device=device, dtype=torch.float64)[None, :]
    gain = torch.exp(-2.0 * math.pi ** 2 * cam.scene_sigma ** 2 * (fx * fx + fy * fy))
    spec = torch.fft.rfft2(white) * gain
    field = torch.fft.irfft2(spec, s=(H, W))
    mu, sd = field.mean(), field.std(unbiased=False)
    field = (field - mu) / sd * cam.scene_std + cam.scene_mean
    return torch.fft.rfft2(field)


def _shifted(spec: torch.Tensor, H: int, W: int, dy: float, dx: float) -> torch.Tensor:
    fy = torch.fft.fftfreq(H, device=spec.device, dtype=torch.float64)[:, None]
    fx = torch.fft.rfftfreq(W, device=spec.device, dtype=torch.float64)[None, :]
    phase = torch.exp(-2j * math.pi * (fy * dy + fx * dx))
    return torch.fft.irfft2(spec * phase, s=(H, W))


def frames(cam: Camera, m: int, stream: int = 0, device="cpu", drift_px: float = 0.0,
           out: torch.Tensor | None = None, start: int = 0) -> torch.Tensor:
    """m uint8 frames [m, H, W, C] of the camera.

    ``stream`` separates independent sets of frames of one camera (for example
    the fingerprint set and the query set).  With drift_px == 0 every frame has
    its own scene; otherwise one scene per channel drifts by a random walk.
    ``start`` generates frames start..start+m-1 of the stream (for chunking).
    """
    H, W, C = cam.H, cam.W, cam.C
    if out is None:
        out = torch.empty((m, H, W, C), dtype=torch.uint8, device=device)
    K = k_true(cam, device).to(torch.float64)
    base = None
    offsets = None
    if drift_px > 0:
        gb = _gen(device, 2, cam.camera_id, stream)
        base = [_lowpass_spectrum(cam, gb, device) for _ in range(C)]
        n_steps = start + m
        steps = (torch.rand((n_steps, 2), generator=_gen("cpu", 3, cam.camera_id, stream),
                            dtype=torch.float64) * 2.0 - 1.0) * drift_px
        offsets = torch.cumsum(steps, dim=0)
    for j in range(m):
        idx = start + j
        gf = _gen(device, 4, cam.camera_id, stream, idx)
        for c in range(C):
            if base is None:
                scene = torch.fft.irfft2(_lowpass_spectrum(cam, gf, device), s=(H, W))
            else:
                dy, dx = float(offsets[idx, 0]), float(offsets[idx, 1])
                scene = _shifted(base[c], H, W, dy, dx)
            noise = torch.randn((H, W), generator=gf, device=device, dtype=torch.float64) * cam.sigma_read
            val = scene * (1.0 + K[c]) + noise
            out[j, :, :, c] = torch.clamp(torch.round(val), 0, 255).to(torch.uint8)
    return out


def foreign(cam: Camera, offset: int = 1000) -> Camera:
    """A camera of the same geometry with an independent K."""
    return Camera(H=cam.H, W=cam.W, C=cam.C, camera_id=cam.camera_id + offset, k_std=cam.k_std,
                  scene_sigma=cam.scene_sigma, scene_mean=cam.scene_mean, scene_std=cam.scene_std,
                  sigma_read=cam.sigma_read)
