"""torch.autograd bindings of the differentiable chain (marshalling only:
every forward and adjoint step runs in libprnu's kernels).

  S = sda_weighted(frames, w, d)        Sec. III-B with free per-frame weights
  W = residual(S, sigma0)               Sec. II-A, noise-form wavelet denoiser
  K = mle(W, S, gray=True)              Sec. III-A
  p = pce(K, Wq, Iq)                    Sec. IV (one value per query)

sigma0 is a 0-d CPU tensor (its value is a kernel parameter); frames are
uint8 [m, H, W, C] device tensors.  The residual keeps its detail
coefficients as the checkpoint for its adjoint.
"""
from __future__ import annotations

import ctypes

import torch

from . import prnu as P


def _stream(t):
    return torch.cuda.current_stream(t.device).cuda_stream


def _params(sigma0: float, levels: int = 4):
    return P.default_params(levels=levels, sigma0=float(sigma0))


class _SDAWeighted(torch.autograd.Function):
    @staticmethod
    def forward(fctx, frames, weights, d, ctx):
        frames4 = frames if frames.dim() == 4 else frames.unsqueeze(-1)
        m, H, W, C = frames4.shape
        fr = frames4.contiguous()
        w = weights.detach().to(torch.float32).contiguous()
        S = torch.empty(((m + d - 1) // d, C, H, W), dtype=torch.float32, device=frames.device)
        P.call("prnu_sda_weighted", ctx.ctx, fr.data_ptr(), m, H, W, C, H * W * C, W * C, d, w.data_ptr(),
               S.data_ptr(), _stream(S))
        fctx.save_for_backward(fr)
        fctx.d, fctx.ctx = d, ctx
        return S

    @staticmethod
    def backward(fctx, gS):
        (fr,) = fctx.saved_tensors
        m, H, W, C = fr.shape
        ctx = fctx.ctx
        gw = torch.empty(m, dtype=torch.float32, device=fr.device)
        ws = ctx.workspace(m * min(H, 64) * 8)
        P.call("prnu_sda_weighted_backward", ctx.ctx, fr.data_ptr(), m, H, W, C, H * W * C, W * C, fctx.d,
               gS.contiguous().data_ptr(), gw.data_ptr(), ws.data_ptr(), ws.numel(), _stream(gw))
        return None, gw, None, None


class _Residual(torch.autograd.Function):
    @staticmethod
    def forward(fctx, img, sigma0, ctx, levels):
        n, C, H, W = img.shape
        prm = _params(sigma0.item(), levels)
        wsb, ckb = P.prnu_workspace_size_grad(ctx.ctx, H, W, C, prm, n)
        img = img.contiguous()
        out = torch.empty_like(img)
        ckpt = torch.empty(ckb // 4, dtype=torch.float32, device=img.device)
        ws = ctx.workspace(wsb)
        P.call("prnu_denoise_residual_ckpt", ctx.ctx, img.data_ptr(), n, H, W, C, ctypes.byref(prm), out.data_ptr(),
               ckpt.data_ptr(), ws.data_ptr(), ws.numel(), _stream(img))
        fctx.save_for_backward(ckpt)
        fctx.prm, fctx.ctx, fctx.shape, fctx.sig = prm, ctx, (n, C, H, W), sigma0
        return out

    @staticmethod
    def backward(fctx, gW):
        (ckpt,) = fctx.saved_tensors
        n, C, H, W = fctx.shape
        ctx = fctx.ctx
        g_img = torch.zeros((n, C, H, W), dtype=torch.float32, device=ckpt.device)
        g_sig = torch.zeros(1, dtype=torch.float64, device=ckpt.device)
        wsb, _ = P.prnu_workspace_size_grad(ctx.ctx, H, W, C, fctx.prm, n)
        ws = ctx.workspace(wsb)
        P.call("prnu_denoise_residual_backward", ctx.ctx, ckpt.data_ptr(), n, H, W, C, ctypes.byref(fctx.prm),
               gW.contiguous().data_ptr(), g_img.data_ptr(), g_sig.data_ptr(), ws.data_ptr(), ws.numel(),
               _stream(g_img))
        gs = g_sig.to(device=fctx.sig.device, dtype=fctx.sig.dtype).reshape(fctx.sig.shape)
        return g_img, gs, None, None


class _MLE(torch.autograd.Function):
    @staticmethod
    def forward(fctx, Wr, S, gray, ctx):
        n, C, H, W = S.shape
        Wr, S = Wr.contiguous(), S.contiguous()
        num = torch.empty((C, H, W), dtype=torch.float32, device=S.device)
        den = torch.empty_like(num)
        K = torch.empty((H, W) if gray else (C, H, W), dtype=torch.float32, device=S.device)
        P.call("prnu_mle_images", ctx.ctx, Wr.data_ptr(), S.data_ptr(), n, H, W, C, int(gray), num.data_ptr(),
               den.data_ptr(), K.data_ptr(), _stream(S))
        fctx.save_for_backward(Wr, S, num, den)
        fctx.gray, fctx.ctx = gray, ctx
        return K

    @staticmethod
    def backward(fctx, gK):
        Wr, S, num, den = fctx.saved_tensors
        n, C, H, W = S.shape
        gW, gS = torch.empty_like(Wr), torch.empty_like(S)
        P.call("prnu_mle_images_backward", fctx.ctx.ctx, Wr.data_ptr(), S.data_ptr(), n, H, W, C, int(fctx.gray),
               num.data_ptr(), den.data_ptr(), gK.contiguous().data_ptr(), gW.data_ptr(), gS.data_ptr(), _stream(S))
        return gW, gS, None, None


class _PCE(torch.autograd.Function):
    @staticmethod
    def forward(fctx, K, Wq, Iq, nbhd, ctx):
        n, C, H, W = Wq.shape
        per_query = K.dim() == 3
        Kc, Wq, Iq = K.contiguous(), Wq.contiguous(), Iq.contiguous()
        res = (ctx.pce_match_pairs if per_query else ctx.pce_match_batch)(Kc, Wq, Iq, nbhd)
        fctx.save_for_backward(Kc, Wq, Iq)
        fctx.nbhd, fctx.ctx, fctx.per_query = nbhd, ctx, per_query
        return torch.tensor([r[0] for r in res], dtype=torch.float64, device=Wq.device)

    @staticmethod
    def backward(fctx, g):
        K, Wq, Iq = fctx.saved_tensors
        n, C, H, W = Wq.shape
        ctx = fctx.ctx
        gK, gWq = torch.empty_like(K), torch.empty_like(Wq)
        nb = P.prnu_workspace_size_pce_backward(ctx.ctx, H, W, n)
        ws = ctx.workspace(nb)
        g = g.to(torch.float64).contiguous()
        P.call("prnu_pce_backward", ctx.ctx, K.data_ptr(), int(fctx.per_query), Wq.data_ptr(), Iq.data_ptr(), n, H, W,
               C, fctx.nbhd, g.data_ptr(), gK.data_ptr(), gWq.data_ptr(), ws.data_ptr(), ws.numel(), _stream(Wq))
        return gK, gWq, None, None, None


def sda_weighted(frames, weights, d: int, ctx):
    return _SDAWeighted.apply(frames, weights, d, ctx)


def residual(img, sigma0, ctx, levels: int = 4):
    """img float32 [n, C, H, W] -> W [n, C, H, W]; sigma0 a 0-d CPU tensor."""
    return _Residual.apply(img, sigma0, ctx, levels)


def mle(Wr, S, ctx, gray: bool = True):
    return _MLE.apply(Wr, S, gray, ctx)


def pce(K, Wq, Iq, ctx, nbhd: int = 11):
    return _PCE.apply(K, Wq, Iq, nbhd, ctx)


def mean_pce(frames, weights, d: int, sigma0, qimgs, ctx, levels: int = 4, nbhd: int = 11):
    """The whole chain: mean PCE of the queries qimgs [nq, C, H, W] against the
    fingerprint of `frames` with SDA weights `weights` and denoiser sigma0."""
    S = sda_weighted(frames, weights, d, ctx)
    K = mle(residual(S, sigma0, ctx, levels), S, ctx, gray=True)
    return pce(K, residual(qimgs, sigma0, ctx, levels), qimgs, ctx, nbhd).mean()
