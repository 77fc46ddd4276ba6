"""Seeded synthetic cameras and frames (the stand-in for the paper's datasets).

The paper's experiments use the VISION and NYUAD-MMD datasets, which are not
available; frames here follow the sensor model of Sec. II-A, Eq. (1):

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


def frames_fast(cam: Camera, m: int, stream: int = 0, device="cpu", drift_px: int = 2,
                out: torch.Tensor | None = None, start: int = 0) -> torch.Tensor:
    """m uint8 frames [m, H, W, C] for large batches: the same sensor model as
    ``frames`` with a drifting scene, but the drift is a random walk of whole
    pixels (steps uniform in {-drift_px .. drift_px} per axis), so a frame's
    scene is an index roll of the camera's base scene instead of a Fourier
    shift, and the read noise is drawn in float32.  Frames start..start+m-1 of
    the stream; each frame's noise comes from its own seeded generator, so
    chunked generation gives the same bytes."""
    H, W, C = cam.H, cam.W, cam.C
    if out is None:
        out = torch.empty((m, H, W, C), dtype=torch.uint8, device=device)
    gain = 1.0 + k_true(cam, device)                                  # [C, H, W] float32
    gb = _gen(device, 7, cam.camera_id, stream)
    base = torch.stack([torch.fft.irfft2(_lowpass_spectrum(cam, gb, device), s=(H, W)) for _ in range(C)])
    base = base.to(torch.float32)
    steps = torch.randint(-drift_px, drift_px + 1, (start + m, 2), generator=_gen("cpu", 8, cam.camera_id, stream))
    offsets = torch.cumsum(steps, dim=0)
    for j in range(m):
        idx = start + j
        v = torch.randn((C, H, W), generator=_gen(device, 9, cam.camera_id, stream, idx), device=device,
                        dtype=torch.float32)
        v.mul_(cam.sigma_read)
        v.addcmul_(torch.roll(base, shifts=(int(offsets[idx, 0]), int(offsets[idx, 1])), dims=(1, 2)), gain)
        v.round_().clamp_(0, 255)
        out[j].copy_(v.permute(1, 2, 0))
    return out


BATCH_RESOLUTIONS = ((720, 1280), (1080, 1920), (3024, 4032))


def batch_cameras(n: int = 32, seed: int = 2, m_range=(100, 2000), d_range=(10, 100),
                  resolutions=BATCH_RESOLUTIONS, C: int = 3):
    """A seeded multi-camera workload: n cameras (camera_id 2000 + i, each with
    its own K), each with a resolution drawn from ``resolutions``, a frame
    count uniform in m_range and an SDA group size uniform in d_range (both
    inclusive).  Returns [(Camera, m, d)]."""
    g = torch.Generator()
    g.manual_seed(BASE_SEED + seed)
    out = []
    for i in range(n):
        r = int(torch.randint(len(resolutions), (1,), generator=g))
        m = int(torch.randint(m_range[0], m_range[1] + 1, (1,), generator=g))
        d = int(torch.randint(d_range[0], d_range[1] + 1, (1,), generator=g))
        H, W = resolutions[r]
        out.append((Camera(H=H, W=W, C=C, camera_id=2000 + i), m, d))
    return out
