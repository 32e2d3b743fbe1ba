"""mot_apply_Z0_static: the Z0 product for callers that cannot allocate device
memory when they call in (allocation-free pools or budgets, real-time loops
that cannot take cudaMalloc's device synchronisation).  Its scratch is the
library's file-scope device array, so the call allocates nothing; this checks
it against mot_apply_Z0, which uses allocated scratch, on two calls in a row
(the array keeps the previous call's contents), with the parity tolerances used
elsewhere (FP64 1e-10, FP32 1e-5 relative L2); that the device's free memory
is the same before and after a call; and that the largest request the array
holds is accepted while one more right-hand side is refused before any GPU work.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import paper_2607_28309_b300 as mot
from paper_2607_28309_b300 import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(torch.linalg.vector_norm((a - b).double()) / torch.linalg.vector_norm(b.double()))


def test_static_scratch_product_matches_allocating_product():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2607_28309_b300 import build

    build.build()
    ctx = mot.mot_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        N, alpha = (24, 20, 18), 8.0
        eps = synthetic.block_eps(N, 4, 1.5, 6.0, 33)
        prob = mot.mot_problem_create(ctx, N, 10e-9, eps, alpha)
        try:
            nv = int(np.prod(N))
            gen = torch.Generator(device="cuda").manual_seed(5)
            for dtype, tdt, tol in ((mot.MOT_F64, torch.float64, 1e-10), (mot.MOT_F32, torch.float32, 1e-5),
                                    (mot.MOT_F64DF, torch.float64, 1e-10)):
                for nrhs in (1, 3):
                    x = torch.randn(nrhs, 3, nv, device="cuda", dtype=tdt, generator=gen)
                    ref = torch.empty_like(x)
                    mot.mot_apply_Z0(prob, x, ref, nrhs, dtype)
                    for _ in range(2):  # two calls in a row share the static scratch
                        y = torch.full_like(x, float("nan"))
                        torch.cuda.synchronize()
                        free0 = torch.cuda.mem_get_info()[0]
                        mot.mot_apply_Z0_static(prob, x, y, nrhs, dtype)
                        torch.cuda.synchronize()
                        assert torch.cuda.mem_get_info()[0] == free0
                        assert torch.isfinite(y).all()
                        assert _rel(y, ref) <= tol
            # pointers off the 16-byte grid are refused before any device work
            x = torch.zeros(3 * nv + 1, device="cuda", dtype=torch.float32)
            y = torch.zeros_like(x)
            for f in (mot.mot_apply_Z0, mot.mot_apply_Z0_static):
                with pytest.raises(mot.MotError) as e:
                    f(prob, x[1:].data_ptr(), y[1:].data_ptr(), 1, mot.MOT_F32)
                assert e.value.status == mot.MOT_EINVAL
            # the largest request the array holds (the bound stated in the header) is
            # accepted; one more right-hand side is refused with MOT_EINVAL
            info = mot.mot_problem_info_get(prob)
            H0, c = info.M0[0] // 2 + 1, 16

            def need(b):
                rows = b * 3 * N[2] * N[1] * H0 * c
                return (rows + 255) // 256 * 256 + b * 3 * N[2] * info.M0[1] * H0 * c

            big = 1
            while need(big + 1) <= mot.MOT_STATIC_SCRATCH_BYTES:
                big += 1
            x = torch.zeros(big + 1, 3, nv, device="cuda", dtype=torch.float64)
            y = torch.zeros_like(x)
            mot.mot_apply_Z0_static(prob, x[:big], y[:big], big, mot.MOT_F64)
            torch.cuda.synchronize()
            assert float(y[:big].abs().max()) == 0.0
            with pytest.raises(mot.MotError) as e:
                mot.mot_apply_Z0_static(prob, x, y, big + 1, mot.MOT_F64)
            assert e.value.status == mot.MOT_EINVAL
        finally:
            mot.mot_problem_destroy(prob)
    finally:
        mot.mot_ctx_destroy(ctx)
