"""Failure detection on the GPU without a fault: a device-side wait that runs out.

Every tensor-core kernel of the library bounds its mbarrier waits by %globaltimer and,
when one runs out, raises NEGF_ERR_TIMEOUT on the context and returns.  The self test
launches one thread that waits, with that same bounded wait, on an mbarrier that
nothing arrives on; nothing else is in flight.  The test checks that the status reaches
the host through negf_ctx_sync, that the wait lasted its budget, that the status is
cleared, and that the context still computes correctly afterwards.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_device_wait_runs_out_and_reports_timeout():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2602_03438_gb300 as P
    ctx = P.Context(0, 64 << 20)
    assert ctx.sync() == 0
    budget = 200_000_000   # 0.2 s of GPU time
    t0 = time.perf_counter()
    ctx.selftest_wait_timeout(budget)
    st = ctx.sync()
    dt = time.perf_counter() - t0
    assert st == P.negf.NEGF_ERR_TIMEOUT
    assert dt >= 0.9 * budget * 1e-9
    # the status was cleared, and the context still works: a small product checks out
    assert ctx.sync() == 0
    rng = np.random.default_rng(5)
    n, u = 24, 3
    A = rng.standard_normal((u, n, n)) + 1j * rng.standard_normal((u, n, n))
    B = rng.standard_normal((u, n, n)) + 1j * rng.standard_normal((u, n, n))
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dD = torch.empty_like(dA)
    P.negf.negf_block_gemm(ctx, P.FP64, dA, dB, dD)
    assert ctx.sync() == 0
    assert np.abs(dD.cpu().numpy() - A @ B).max() <= 1e-10 * np.abs(A @ B).max()


def test_self_test_budget_is_checked():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2602_03438_gb300 as P
    ctx = P.Context(0, 64 << 20)
    with pytest.raises(P.negf.NegfError):
        ctx.selftest_wait_timeout(10)
    with pytest.raises(P.negf.NegfError):
        ctx.selftest_wait_timeout(5_000_000_000)
    assert ctx.sync() == 0
