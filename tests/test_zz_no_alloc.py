"""fst_project_noalloc: the projection entry point for callers that cannot allocate
device memory when they project (graph capture, a memory manager that owns the GPU).
It must give the same results as fst_project, call after call, using only the
library's fixed scratch array.  Collected last on purpose (file name)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1611_04950_gb300 import fst as F  # noqa: E402
from paper_1611_04950_gb300 import workloads  # noqa: E402


def _stream():
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("N,W,eps,dtype", [(65536, 1 / 8, 1e-4, torch.float32),     # four-step path (scratch)
                                           (4096, 1 / 16, 1e-6, torch.float32),      # single-CTA path
                                           (20000, 0.05, 1e-6, torch.complex64),
                                           (9000, 0.2, 1e-8, torch.float64)])
def test_noalloc_matches_fst_project_twice(N, W, eps, dtype):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    assert F.fst_noalloc_scratch_bytes() == 128 << 20
    plan = F.Plan(N, W, eps=eps)
    y = workloads.gaussian(9, N, seed=N, complex_=dtype.is_complex).to(dtype).cuda()
    code = F._dtype_code(dtype)
    ref = plan.project(y)
    outs = []
    for _ in range(2):
        out = torch.full_like(y, float("nan"))
        F.fst_project_noalloc(plan.h, y.data_ptr(), out.data_ptr(), y.shape[0], N, code, _stream())
        outs.append(out)
    torch.cuda.synchronize()
    tol = 1e-12 if dtype in (torch.float64, torch.complex128) else 1e-5
    ynrm = torch.linalg.vector_norm(y, dim=1)
    for out in outs:
        assert torch.isfinite(torch.view_as_real(out) if out.is_complex() else out).all()
        err = torch.linalg.vector_norm(out - ref, dim=1) / ynrm
        assert torch.all(err <= tol), err
