"""The two building blocks of the sweeps through the C ABI against numpy
complex128: the batched block product (rows a8: FP64 and 3-term TF32 split on
the tensor cores) and the batched block inverse (row a7)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

H = lambda x: np.conj(np.swapaxes(x, -1, -2))


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_03438_gb300 as P
    P.negf.load_library()
    return P


@pytest.fixture(scope="module")
def ctx(P):
    c = P.Context(0, 1 << 30)
    yield c
    c.close()


def _rand(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def _op(x, op):
    return x if op == 0 else H(x)


GEMM_TOL = {"FP64": 1e-13, "MIXED": 1e-13, "MIXED_TF32": 2e-6}


@pytest.mark.parametrize("n", [1, 8, 16, 33, 64, 100, 128, 130, 192, 256, 300, 512])
@pytest.mark.parametrize("opA,opB", [(0, 0), (2, 0), (0, 2), (2, 2)])
@pytest.mark.parametrize("prec", ["FP64", "MIXED", "MIXED_TF32"])
def test_block_gemm(P, ctx, n, opA, opB, prec):
    rng = np.random.default_rng(n * 7 + opA + 3 * opB)
    U = 3
    A, B, Cm = _rand(rng, (U, n, n)), _rand(rng, (U, n, n)), _rand(rng, (U, n, n))
    alpha, beta = 0.7 - 0.2j, -1.1 + 0.4j
    ref = alpha * (_op(A, opA) @ _op(B, opB)) + beta * Cm
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    D = torch.empty((U, n, n), dtype=torch.complex128, device="cuda")
    P.negf.negf_block_gemm(ctx, getattr(P, prec), t(A), t(B), D, opA, opB, alpha, beta, t(Cm))
    assert ctx.sync() == 0
    got = D.cpu().numpy()
    # normwise error relative to |alpha| ||A|| ||B|| (the size of the summands)
    scale = np.linalg.norm(A[0]) * np.linalg.norm(B[0]) * abs(alpha) / n
    err = np.abs(got - ref).max() / max(scale, 1e-300)
    tol = 1e-13 if n < 16 else GEMM_TOL[prec]
    assert err <= tol, err


@pytest.mark.parametrize("n,opA,opB", [(100, 0, 0), (128, 2, 2), (128, 0, 2), (120, 2, 0)])
def test_sliced_gemm_many_units(P, ctx, n, opA, opB):
    """More units than resident clusters: every cluster of the persistent kernel walks
    several units, its epilogue overlapping the next unit's products."""
    rng = np.random.default_rng(400 + n + opA + opB)
    U = 160
    A, B, Cm = _rand(rng, (U, n, n)), _rand(rng, (U, n, n)), _rand(rng, (U, n, n))
    alpha, beta = -1.0, 1.0
    ref = alpha * (_op(A, opA) @ _op(B, opB)) + beta * Cm
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    D = torch.empty((U, n, n), dtype=torch.complex128, device="cuda")
    P.negf.negf_block_gemm(ctx, P.MIXED, t(A), t(B), D, opA, opB, alpha, beta, t(Cm))
    assert ctx.sync() == 0
    got = D.cpu().numpy()
    for u in range(U):
        scale = np.linalg.norm(A[u]) * np.linalg.norm(B[u]) / n
        assert np.abs(got[u] - ref[u]).max() <= 1e-13 * scale, u


def test_sliced_gemm_wide_dynamic_range(P, ctx):
    """Rows and columns spanning 1e-12..1e3 (the decaying couplings of banded
    Hamiltonians): the sliced product keeps each row/column on its own scale."""
    rng = np.random.default_rng(9)
    n = 96
    ra = 10.0 ** rng.uniform(-12, 3, size=n)
    cb = 10.0 ** rng.uniform(-12, 3, size=n)
    A = _rand(rng, (2, n, n)) * ra[None, :, None]
    B = _rand(rng, (2, n, n)) * cb[None, None, :]
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    D = torch.empty((2, n, n), dtype=torch.complex128, device="cuda")
    P.negf.negf_block_gemm(ctx, P.MIXED, t(A), t(B), D)
    assert ctx.sync() == 0
    ref = A @ B
    # error of entry (m, j) relative to ||row m of A|| ||column j of B||
    rn = np.linalg.norm(A, axis=2)[:, :, None]
    cn = np.linalg.norm(B, axis=1)[:, None, :]
    assert (np.abs(D.cpu().numpy() - ref) / (rn * cn)).max() <= 1e-13


def test_block_gemm_shared_operand_and_in_place(P, ctx):
    rng = np.random.default_rng(5)
    n, U = 64, 4
    A = _rand(rng, (n, n))          # shared by all units
    B = _rand(rng, (U, n, n))
    Cm = _rand(rng, (U, n, n))
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    D = t(Cm)                       # D == C: in-place accumulate
    P.negf.negf_block_gemm(ctx, P.MIXED, t(A), t(B), D, 0, 0, 1.0, 1.0, D)
    assert ctx.sync() == 0
    ref = A[None] @ B + Cm
    assert np.abs(D.cpu().numpy() - ref).max() <= 2e-6 * np.linalg.norm(A) * np.linalg.norm(B[0]) / n


@pytest.mark.parametrize("n", [1, 5, 32, 64, 100, 128, 192])
@pytest.mark.parametrize("prec", ["FP64", "MIXED", "MIXED_TF32"])
def test_block_inverse(P, ctx, n, prec):
    rng = np.random.default_rng(n)
    U = 3
    M = _rand(rng, (U, n, n)) + 2.0 * np.sqrt(n) * np.eye(n)[None] * np.exp(1j * rng.uniform(0, 6, size=(U, 1, 1)))
    ref = np.linalg.inv(M)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    X = torch.empty((U, n, n), dtype=torch.complex128, device="cuda")
    st = torch.zeros(U, dtype=torch.int32, device="cuda")
    P.negf.negf_block_inverse(ctx, getattr(P, prec), t(M), X, st)
    assert ctx.sync() == 0
    assert st.cpu().numpy().tolist() == [0] * U
    for u in range(U):
        err = np.linalg.norm(X[u].cpu().numpy() - ref[u]) / np.linalg.norm(ref[u])
        tol = {"FP64": 1e-13, "MIXED": 1e-11, "MIXED_TF32": 1e-9}[prec]
        assert err <= tol, (u, err)


@pytest.mark.parametrize("n", [16, 24, 70, 128])
def test_block_inverse_with_interchanges(P, ctx, n):
    """Dense complex normal matrices (no diagonal dominance): partial pivoting interchanges
    rows at most steps, across the panels of the blocked FP32 Gauss-Jordan (8 columns per
    panel; n = 70 ends on a panel of 6).  Mixed: the FP32 inverse refined twice."""
    rng = np.random.default_rng(900 + n)
    U = 4
    M = _rand(rng, (U, n, n))
    ref = np.linalg.inv(M)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    for prec, tol in (("MIXED", 1e-10), ("FP64", 1e-12)):
        X = torch.empty((U, n, n), dtype=torch.complex128, device="cuda")
        st = torch.zeros(U, dtype=torch.int32, device="cuda")
        P.negf.negf_block_inverse(ctx, getattr(P, prec), t(M), X, st)
        assert ctx.sync() == 0
        assert st.cpu().numpy().tolist() == [0] * U
        for u in range(U):
            err = np.linalg.norm(X[u].cpu().numpy() - ref[u]) / np.linalg.norm(ref[u])
            assert err <= tol, (prec, u, err)


def test_block_inverse_singular_panels(P, ctx):
    """A zero column found by the blocked FP32 Gauss-Jordan (n = 24, column 13, in the
    second panel) flags its unit; the identity next to it does not."""
    n = 24
    rng = np.random.default_rng(7)
    M = np.stack([_rand(rng, (n, n)), np.eye(n, dtype=complex)])
    M[0, :, 13] = 0.0
    X = torch.empty((2, n, n), dtype=torch.complex128, device="cuda")
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    P.negf.negf_block_inverse(ctx, P.MIXED, torch.from_numpy(M).cuda(), X, st)
    assert ctx.sync() == 0
    assert st.cpu().numpy().tolist() == [P.negf.NEGF_ERR_SINGULAR, 0]
    assert np.abs(X[1].cpu().numpy() - np.eye(n)).max() <= 1e-14


def test_block_inverse_singular(P, ctx):
    n = 6
    M = np.zeros((2, n, n), complex)
    M[1] = np.eye(n)
    M[0, :, 2] = 0.0
    M[0] += np.diag([1, 1, 0, 1, 1, 1])
    X = torch.empty((2, n, n), dtype=torch.complex128, device="cuda")
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    P.negf.negf_block_inverse(ctx, P.FP64, torch.from_numpy(M).cuda(), X, st)
    assert ctx.sync() == 0
    assert st.cpu().numpy().tolist() == [P.negf.NEGF_ERR_SINGULAR, 0]
