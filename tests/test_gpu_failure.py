"""Failure paths on the GPU, made without a GPU fault.

* A bounded device wait that runs out: the test hook fst_test_tc_stall makes the
  tensor-core correction wait on a barrier that nothing completes, so it gives up after
  20 ms before issuing any copy or product (its normal give-up path: tensor memory
  freed, NaN partial sums, error word raised).  The status must come back as
  FST_ETIMEOUT through fst_sync, through fst_project_host and through the next call on
  the plan, and the plan must work normally afterwards.
* Recorded ragged batches whose plans are destroyed and rebuilt (the caching allocator
  hands the same addresses back), and whose plans' workspaces move.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1611_04950_gb300 import fst as F  # noqa: E402
from paper_1611_04950_gb300 import workloads  # noqa: E402
from oracle import fst_oracle as O  # noqa: E402


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _stream():
    return torch.cuda.current_stream().cuda_stream


def test_tc_wait_timeout_is_reported_and_recovered():
    _cuda()
    # 40 signals: batches of more than 32 rows take the tensor-core correction
    N, W, B = 65536, 1 / 8, 40
    p = F.Plan(N, W, eps=1e-4)
    y = workloads.gaussian(B, N, seed=41).float().cuda()
    ref = p.project(y)
    F.fst_sync(p.h, _stream())

    # 1) reported by fst_sync; every output carries the NaN correction
    F.fst_test_tc_stall(1, 0.02)
    out = torch.zeros_like(y)
    F.fst_project(p.h, y.data_ptr(), out.data_ptr(), B, N, F.FST_F32, _stream())
    with pytest.raises(F.FSTError) as ei:
        F.fst_sync(p.h, _stream())
    assert ei.value.status == F.FST_ETIMEOUT
    assert torch.isnan(out).all()
    F.fst_sync(p.h, _stream())          # reporting cleared the word

    # 2) the context is intact: the same call gives the same result as before
    again = p.project(y)
    torch.cuda.synchronize()
    assert torch.equal(again, ref)

    # 3) reported by the next call on the plan, which enqueues nothing
    F.fst_test_tc_stall(1, 0.02)
    F.fst_project(p.h, y.data_ptr(), out.data_ptr(), B, N, F.FST_F32, _stream())
    torch.cuda.synchronize()
    marker = torch.full_like(y, 7.0)
    with pytest.raises(F.FSTError) as ei:
        F.fst_project(p.h, y.data_ptr(), marker.data_ptr(), B, N, F.FST_F32, _stream())
    assert ei.value.status == F.FST_ETIMEOUT
    torch.cuda.synchronize()
    assert torch.all(marker == 7.0)

    # 4) reported by the synchronous host-buffer entry point of the same call
    F.fst_test_tc_stall(1, 0.02)
    yh = y.cpu().pin_memory()
    oh = torch.empty_like(yh).pin_memory()
    with pytest.raises(F.FSTError) as ei:
        F.fst_project_host(p.h, yh.data_ptr(), oh.data_ptr(), B, F.FST_F32, _stream())
    assert ei.value.status == F.FST_ETIMEOUT
    F.fst_sync(p.h, _stream())
    assert torch.equal(p.project_host(yh), ref.cpu())


def _ragged_case():
    # single-CTA lengths and two four-step ones (N > 8192)
    params = [(1000, 0.05, 1e-6), (3000, 0.2, 1e-3), (8192, 0.25, 1e-8), (5000, 1 / 64, 1e-6),
              (20000, 0.1, 1e-6), (70000, 0.2, 1e-3)]
    g = np.random.default_rng(17)
    ys64 = [g.standard_normal(N) for (N, W, e) in params]
    ys = [torch.as_tensor(v, dtype=torch.float32, device="cuda") for v in ys64]
    return params, ys64, ys


def _check_ragged(params, ys64, outs):
    for (N, W, e), y, o in zip(params, ys64, outs):
        ref = O.fast_project(O.make_plan(N, W, O.default_K(N, W), e), y)
        err = np.linalg.norm(o.double().cpu().numpy() - ref) / np.linalg.norm(y)
        assert err < 1e-5, (N, W, e, err)


def test_ragged_recording_survives_destroy_and_rebuild():
    _cuda()
    params, ys64, ys = _ragged_case()
    outs = [torch.empty_like(v) for v in ys]
    ps = F.PlanSet(params)
    for _ in range(3):                  # direct, recorded, replayed
        ps.project(ys, outs)
    torch.cuda.synchronize()
    _check_ragged(params, ys64, outs)
    ps.close()                          # drops the recorded batch with its plans
    torch.cuda.empty_cache()
    for o in outs:
        o.fill_(float("nan"))
    ps2 = F.PlanSet(params)             # same parameters, same signal buffers
    for _ in range(3):
        ps2.project(ys, outs)
    torch.cuda.synchronize()
    _check_ragged(params, ys64, outs)


def test_ragged_recording_follows_a_moved_workspace():
    _cuda()
    params, ys64, ys = _ragged_case()
    outs = [torch.empty_like(v) for v in ys]
    ps = F.PlanSet(params)
    for _ in range(3):
        ps.project(ys, outs)
    torch.cuda.synchronize()
    # a large batch on the longest signal's plan reallocates that plan's workspace
    i = max(range(len(params)), key=lambda k: params[k][0])
    N = params[i][0]
    big = workloads.gaussian(96, N, seed=5).float().cuda()
    res = torch.empty_like(big)
    F.fst_project(ps.h[i], big.data_ptr(), res.data_ptr(), 96, N, F.FST_F32, _stream())
    del big, res
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    for o in outs:
        o.fill_(float("nan"))
    for _ in range(3):                  # direct again, recorded again, replayed
        ps.project(ys, outs)
    torch.cuda.synchronize()
    _check_ragged(params, ys64, outs)

