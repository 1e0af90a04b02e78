"""fst_project_noalloc: the projection entry point for callers that cannot allocate
device memory when they project (a process whose memory manager owns all device
memory after start-up, or a service that must not stall on the allocator).  It must
give the same results as fst_project, call after call, using only the library's
fixed scratch array, and refuse work whose scratch does not fit in that array.
Collected last on purpose (file name)."""
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


def test_noalloc_rejects_scratch_beyond_the_array():
    # FP64, N = 2^21 + 1: FFT length 2^23, one pair's intermediate alone is 128 MiB, so the
    # call must fail with FST_EINVAL before launching anything (the output stays untouched)
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    N = (1 << 21) + 1
    plan = F.Plan(N, 0.01, eps=1e-3)
    y = workloads.gaussian(1, N, seed=3).cuda()
    out = torch.full_like(y, 5.0)
    with pytest.raises(F.FSTError) as ei:
        F.fst_project_noalloc(plan.h, y.data_ptr(), out.data_ptr(), 1, N, F.FST_F64, _stream())
    assert ei.value.status == F.FST_EINVAL
    assert "fixed scratch" in str(ei.value)
    torch.cuda.synchronize()
    assert torch.all(out == 5.0)
