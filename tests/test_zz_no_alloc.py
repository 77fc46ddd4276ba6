"""prnu_denoise_residual_static: the allocation-free entry point.

Callers that cannot allocate device memory when they need a residual (inside
a CUDA stream capture, in a plug-in whose host owns all allocations, in a
service with a fixed footprint) use this entry point, whose scratch is a fixed
64 MiB device array of the library.  The test calls it through the C ABI twice
in a row on different images and checks each output against the regular
prnu_denoise_residual (which takes a caller workspace) at the residual
tolerance of the parity tests.  This file is collected last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

RES_TOL = 1e-3


def test_static_scratch_matches_workspace_entry_point_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04573_gb300 import build
    from paper_1909_04573_gb300 import prnu as P
    build.build()
    ctx = P.prnu_create(0)
    try:
        params = P.default_params()
        stream = torch.cuda.current_stream().cuda_stream
        rng = np.random.default_rng(2024)
        shapes = [(1, 1080, 1920), (3, 300, 500)]  # a grey full-HD frame, then a ragged RGB one
        for C, H, W in shapes:
            img = torch.as_tensor(rng.uniform(0, 255, size=(C, H, W)).astype(np.float32)).cuda()
            got = torch.full_like(img, float("nan"))
            ref = torch.empty_like(img)
            P.prnu_denoise_residual_static(ctx, img.data_ptr(), H, W, C, params, got.data_ptr(), stream)
            n = P.prnu_workspace_size(ctx, H, W, C, params, 1)
            ws = torch.empty(n, dtype=torch.uint8, device="cuda")
            P.prnu_denoise_residual(ctx, img.data_ptr(), H, W, C, params, ref.data_ptr(), ws.data_ptr(), n,
                                    stream)
            torch.cuda.synchronize()
            assert torch.isfinite(got).all()
            assert float((got - ref).abs().max()) <= RES_TOL
        # beyond the static scratch: a clear error, nothing launched
        img = torch.zeros((3, 1080, 1920), dtype=torch.float32, device="cuda")
        with pytest.raises(P.PrnuError) as e:
            P.prnu_denoise_residual_static(ctx, img.data_ptr(), 1080, 1920, 3, params, img.data_ptr(), stream)
        assert e.value.status == P.PRNU_ENOSPC and "static scratch" in str(e.value)
    finally:
        torch.cuda.synchronize()
        P.prnu_destroy(ctx)
