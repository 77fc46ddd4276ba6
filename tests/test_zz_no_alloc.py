"""prnu_denoise_residual_static: the allocation-free entry point.

Callers that cannot allocate device memory when they need a residual (inside
a CUDA stream capture, in a plug-in whose host owns all allocations, in a
service with a fixed footprint) use this entry point, whose scratch is a fixed
64 MiB device array of the library.  The test calls it through the C ABI two
times in a row per case, on different images, and checks each output against
the regular prnu_denoise_residual (which takes a caller workspace).  Both run
the same kernels with the same launch shapes in the same context, so the
outputs must be bit-identical: any difference would mean the shared scratch
leaks one call's contents into the next.  This file is collected last so that
a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_static_scratch_matches_workspace_entry_point_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04573_gb300 import build
    from paper_1909_04573_gb300 import prnu as P
    build.build()
    ctx = P.prnu_create(0)
    try:
        stream = torch.cuda.current_stream().cuda_stream
        rng = np.random.default_rng(2024)
        # a grey full-HD frame, a ragged RGB one, and full-HD RGB with float16
        # subbands (its intermediates fit the 64 MiB only at 16-bit storage)
        cases = [(1, 1080, 1920, P.PRNU_DTYPE_F32), (3, 300, 500, P.PRNU_DTYPE_F32),
                 (3, 1080, 1920, P.PRNU_DTYPE_F16)]
        for C, H, W, dt in cases:
            params = P.default_params(dtype=dt)
            n = P.prnu_workspace_size(ctx, H, W, C, params, 1)
            ws = torch.empty(n, dtype=torch.uint8, device="cuda")
            for _ in range(2):
                img = torch.as_tensor(rng.uniform(0, 255, size=(C, H, W)).astype(np.float32)).cuda()
                got = torch.full_like(img, float("nan"))
                ref = torch.empty_like(img)
                P.prnu_denoise_residual_static(ctx, img.data_ptr(), H, W, C, params, got.data_ptr(), stream)
                P.prnu_denoise_residual(ctx, img.data_ptr(), H, W, C, params, ref.data_ptr(), ws.data_ptr(), n,
                                        stream)
                torch.cuda.synchronize()
                assert torch.isfinite(got).all()
                assert torch.equal(got, ref), f"{C}x{H}x{W} dtype {dt}: max diff {float((got - ref).abs().max())}"
        # beyond the static scratch: a clear error, nothing launched
        params = P.default_params()
        img = torch.zeros((3, 1080, 1920), dtype=torch.float32, device="cuda")
        out = torch.zeros_like(img)
        with pytest.raises(P.PrnuError) as e:
            P.prnu_denoise_residual_static(ctx, img.data_ptr(), 1080, 1920, 3, params, out.data_ptr(), stream)
        assert e.value.status == P.PRNU_ENOSPC and "static scratch" in str(e.value)
        # invalid input is rejected before anything is resolved or launched
        with pytest.raises(P.PrnuError) as e:
            P.prnu_denoise_residual_static(ctx, img.data_ptr(), 1080, 1920, 2, params, out.data_ptr(), stream)
        assert e.value.status == P.PRNU_EINVAL
        with pytest.raises(P.PrnuError) as e:
            P.prnu_denoise_residual_static(ctx, img.data_ptr(), 64, 64, 1, params, img.data_ptr(), stream)
        assert e.value.status == P.PRNU_EINVAL
    finally:
        torch.cuda.synchronize()
        P.prnu_destroy(ctx)
