"""negf_block_gemm_noalloc through the C ABI, against negf_block_gemm.

The no-allocation entry point serves callers that may not allocate device memory
(an application that owns all device memory in its own arena, or a loop that
cannot afford cudaMalloc/cudaFree synchronizing the device).  It must give the
same product as the context-based entry point, on consecutive calls that share
its static scratch array.  This file sorts last so that a run stopping at the
first failure has already run every other test; it also passes on its own.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

# the tolerance of the sliced (NEGF_MIXED) product in the block tests
TOL = 1e-13


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_03438_gb300 as P
    P.negf.load_library()
    return P


def _rand(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _err(got, ref, A, B, alpha):
    scale = np.linalg.norm(A[0]) * np.linalg.norm(B[0]) * abs(alpha) / A.shape[-1]
    return np.abs(got - ref).max() / max(scale, 1e-300)


@pytest.mark.parametrize("n,opA,opB", [(128, 0, 0), (64, 2, 0), (100, 0, 2), (8, 2, 2)])
def test_noalloc_matches_context_gemm_on_two_calls(P, n, opA, opB):
    ctx = P.Context(0, 64 << 20)
    try:
        rng = np.random.default_rng(1000 + n + opA + 3 * opB)
        for call in range(2):   # two calls in a row share the static scratch
            U = 5 if call == 0 else 3
            A, B, Cm = _rand(rng, (U, n, n)), _rand(rng, (U, n, n)), _rand(rng, (U, n, n))
            if call == 1:       # a different dynamic range than the first call
                A *= 10.0 ** rng.uniform(-6, 6, size=(1, n, 1))
            alpha, beta = (-1.0, 1.0) if call == 0 else (0.3 + 0.7j, -0.5j)
            D_ref = torch.empty((U, n, n), dtype=torch.complex128, device="cuda")
            P.negf.negf_block_gemm(ctx, P.MIXED, _t(A), _t(B), D_ref, opA, opB, alpha, beta, _t(Cm))
            D = torch.empty_like(D_ref)
            status = torch.zeros(1, dtype=torch.int32, device="cuda")
            P.negf.negf_block_gemm_noalloc(_t(A), _t(B), D, opA, opB, alpha, beta, _t(Cm), status)
            torch.cuda.synchronize()
            assert int(status.item()) == 0
            assert ctx.sync() == 0
            ref = D_ref.cpu().numpy()
            got = D.cpu().numpy()
            assert _err(got, ref, A, B, alpha) <= TOL, call
            # and both agree with the definition
            op = lambda x, o: x if o == 0 else np.conj(np.swapaxes(x, -1, -2))
            exact = alpha * (op(A, opA) @ op(B, opB)) + beta * Cm
            rn = np.linalg.norm(op(A, opA), axis=2)[:, :, None]
            cn = np.linalg.norm(op(B, opB), axis=1)[:, None, :]
            # error relative to the size of the two summands (row x column norms, |beta C|)
            size = abs(alpha) * rn * cn + abs(beta) * np.abs(Cm)
            assert (np.abs(got - exact) / size).max() <= TOL
    finally:
        ctx.close()


def test_noalloc_rejects_batches_beyond_its_scratch(P):
    n = 128
    limit = P.negf.C.c_uint32(1 << 20).value // (2 * 4 * n)   # units whose scales fit 1 MiB
    A = torch.zeros((limit + 1, n, n), dtype=torch.complex128, device="cuda")
    D = torch.empty_like(A)
    with pytest.raises(P.NegfError) as ei:
        P.negf.negf_block_gemm_noalloc(A, A[0], D)
    assert ei.value.code == P.negf.NEGF_ERR_ARG
    assert "static array" in str(ei.value)


def test_noalloc_on_a_second_device(P):
    """The kernels' shared-memory attributes are set per device: the first call on a
    second GPU must work like the first (skipped when one GPU is visible)."""
    if torch.cuda.device_count() < 2:
        pytest.skip("one CUDA device visible")
    n, U = 128, 4
    rng = np.random.default_rng(77)
    A, B = _rand(rng, (U, n, n)), _rand(rng, (U, n, n))
    exact = A @ B
    for dev in (0, 1):
        with torch.cuda.device(dev):
            tA = torch.from_numpy(A).to(f"cuda:{dev}")
            tB = torch.from_numpy(B).to(f"cuda:{dev}")
            D = torch.empty_like(tA)
            status = torch.zeros(1, dtype=torch.int32, device=f"cuda:{dev}")
            P.negf.negf_block_gemm_noalloc(tA, tB, D, status=status, stream=torch.cuda.current_stream(dev))
            torch.cuda.synchronize(dev)
            assert int(status.item()) == 0
            got = D.cpu().numpy()
            size = np.linalg.norm(A, axis=2)[:, :, None] * np.linalg.norm(B, axis=1)[:, None, :]
            assert (np.abs(got - exact) / size).max() <= TOL, dev
