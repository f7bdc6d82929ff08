"""The blocked Gauss-Jordan inversion of the FP32 block inverse, restated step by step in
numpy (host logic, no GPU): panels of w columns whose pivot steps act on the panel's own
columns only, with the row interchanges kept as positions and each row's multipliers
recorded, then one rank-w pass over the other columns through the staged (moved) rows,
and the interchanges undone as column swaps at the end.  Checked against
numpy.linalg.inv, with partial pivoting that interchanges rows across panels, a ragged
last panel, and a zero column that must be flagged."""
import numpy as np
import pytest


def panel_gauss_jordan(A, w):
    """Returns (X, singular).  The data flow of the kernel: W is the working matrix in
    positions; per panel, the panel threads hold rows by their original index r and
    track mypos[r]; F[pos][j] are the multipliers at the rows' final positions."""
    n = A.shape[0]
    W = A.astype(complex).copy()
    piv = list(range(n))
    singular = False
    for k0 in range(0, n, w):
        ww = min(w, n - k0)
        pw = W[:, k0:k0 + ww].copy()          # row r of the panel (rows by index)
        pf = np.zeros((n, ww), complex)       # row r's multipliers
        mypos = np.arange(n)
        dinv = np.zeros(ww, complex)
        for j in range(ww):
            k = k0 + j
            cand = [(abs(pw[r, j]) ** 2, mypos[r]) for r in range(n) if mypos[r] >= k]
            best = max(c[0] for c in cand)
            p = min(c[1] for c in cand if c[0] == best)   # first position of the largest
            if not best > 0:
                singular, p = True, k
            win = int(np.nonzero(mypos == p)[0][0])
            d = pw[win, j]
            dinv[j] = np.conj(d) / abs(d) ** 2 if abs(d) > 0 else 0.0
            prow = pw[win] * dinv[j]
            prow[j] = dinv[j]
            piv[k] = p
            for r in range(n):
                if r == win:
                    pf[r, j] = d
                    pw[r] = prow
                else:
                    f = pw[r, j]
                    pf[r, j] = f
                    new = pw[r] - f * prow
                    new[j] = -f * dinv[j]
                    pw[r] = new
            at_k = mypos == k
            mypos[at_k] = p
            mypos[win] = k
        rowsrc = np.empty(n, int)
        F = np.zeros((n, ww), complex)
        for r in range(n):
            W[mypos[r], k0:k0 + ww] = pw[r]
            F[mypos[r]] = pf[r]
            rowsrc[mypos[r]] = r
        # the other columns: y = the rows the interchanges put at each position; the pivot
        # rows' new values from the w x w triangle, then the rank-w update
        others = [c for c in range(n) if not (k0 <= c < k0 + ww)]
        Y = W[rowsrc][:, others]
        V = np.zeros((ww, len(others)), complex)
        for j in range(ww):
            V[j] = (Y[k0 + j] - F[k0 + j, :j] @ V[:j]) * dinv[j]
        new = Y - F @ V
        for j in range(ww):
            new[k0 + j] = V[j] - F[k0 + j, j + 1:] @ V[j + 1:]
        W[:, others] = new
    for k in range(n - 1, -1, -1):
        p = piv[k]
        if p != k:
            W[:, [k, p]] = W[:, [p, k]]
    return W, singular


@pytest.mark.parametrize("n,w", [(1, 8), (5, 8), (16, 8), (24, 8), (30, 8), (33, 4), (40, 8)])
def test_panel_gauss_jordan_is_the_inverse(n, w):
    rng = np.random.default_rng(n * 10 + w)
    A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))   # no diagonal dominance
    X, sing = panel_gauss_jordan(A, w)
    ref = np.linalg.inv(A)
    assert not sing
    assert np.abs(X - ref).max() <= 1e-11 * np.abs(ref).max()


def test_panel_gauss_jordan_interchanges_rows_across_panels():
    """The largest entries of the first columns sit in rows of a later panel: the pivots
    come from there, and the result is still the inverse."""
    n, w = 24, 8
    rng = np.random.default_rng(3)
    A = 0.01 * (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    for j in range(8):
        A[20 - j, j] = 5.0 + j
    X, sing = panel_gauss_jordan(A, w)
    assert not sing
    assert np.abs(X @ A - np.eye(n)).max() <= 1e-12


def test_panel_gauss_jordan_flags_a_zero_column():
    n = 24
    rng = np.random.default_rng(7)
    A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    A[:, 13] = 0.0
    _, sing = panel_gauss_jordan(A, 8)
    assert sing
