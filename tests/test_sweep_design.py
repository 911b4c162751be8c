"""CPU checks of the identities the mixed form's SPD-inverse kernels rely on,
as plain numpy emulations of the kernels' steps (no GPU, no oracle, no
library code):

* the panel-blocked symmetric sweep with look-ahead (Goodnight's sweep
  operator taken four 64-pivots at a time on a gathered column panel: the
  pivots sweep the panel's own rows K, which leaves W_KK = -A_KK^-1; every
  other row takes the whole panel as one product U = W (-W_KK)^T, the rest
  of the matrix one low-rank update A -= U W^T; the next panel is gathered
  before that update reached it and patched, its rows K copied from U)
  reproduces A^-1, also with a ragged last panel and garbage in the unused
  upper triangle;
* the double-float pivot-tile sweep (hi + lo binary32 pairs, Dekker's
  two-sum / two-product with fused multiply-adds, one Newton step for 1/d)
  tracks the binary64 inverse to about cond x 1e-15, far below binary32.
"""
import numpy as np
import pytest

B = 64  # pivot tile


def _tile(M, i, j):
    return M[B * i:B * i + B, B * j:B * j + B]


def _gather(A, W, k0, bw, nt):
    for i in range(nt):
        for q in range(bw):
            j = k0 + q
            S = _tile(A, max(i, j), min(i, j))
            blk = S if i > j else (S.T if i < j else np.tril(S) + np.tril(S, -1).T)
            W[B * i:B * i + B, B * q:B * q + B] = blk


def _panel_rows_K(W, U, V, k0, bw):
    """The pivots of the panel, one after another, on the panel's own rows."""
    for q in range(bw):
        k = k0 + q
        Vk = W[B * k0:B * (k0 + bw), B * q:B * q + B].copy()
        Wkk = W[B * k:B * k + B, B * q:B * q + B]
        P = np.linalg.inv(np.tril(Wkk) + np.tril(Wkk, -1).T)
        Wn = W.copy()
        for i in range(k0, k0 + bw):
            rows = slice(B * i, B * i + B)
            col_q = slice(B * q, B * q + B)
            if i == k:
                Wn[rows, col_q] = -P
                U[rows, col_q] = 0.0
                V[rows, col_q] = 0.0
                continue
            Ui = W[rows, col_q] @ P
            V[rows, col_q] = W[rows, col_q]
            U[rows, col_q] = Ui
            Wn[rows, col_q] = Ui
            Wn[B * k:B * k + B, B * (i - k0):B * (i - k0) + B] = Ui.T
            for jj in range(bw):
                if jj != q:
                    cj = slice(B * jj, B * jj + B)
                    Wn[rows, cj] = W[rows, cj] - Ui @ Vk[B * jj:B * jj + B].T
        W[:] = Wn


def _rows(tiles):
    return np.concatenate([np.arange(B * i, B * i + B) for i in tiles]) if tiles else np.zeros(0, dtype=int)


def _update_lower(A, U, V, K):
    n = A.shape[0]
    C = A - U[:, :K] @ V[:, :K].T
    nb = (n + 127) // 128
    for bm in range(nb):
        for bn in range(bm + 1):   # 128-row tiles on or below the diagonal
            A[128 * bm:128 * bm + 128, 128 * bn:128 * bn + 128] = C[128 * bm:128 * bm + 128, 128 * bn:128 * bn + 128]


def _scatter(A, W, U, k0, bw, nt):
    for i in range(nt):
        in_panel = k0 <= i < k0 + bw
        src_m = W if in_panel else U     # rows K stand in W, the other rows in U
        for q in range(bw):
            j = k0 + q
            src = src_m[B * i:B * i + B, B * q:B * q + B]
            if i >= j:
                A[B * i:B * i + B, B * j:B * j + B] = src
            elif not in_panel:
                A[B * j:B * j + B, B * i:B * i + B] = src.T


def blocked_sweep_inverse(A0, panel=4, seed=0):
    """Emulation of the panel-blocked sweep with look-ahead, in the order the
    two streams' dependencies allow (panel p on its rows, the other rows'
    product, gather + patch of panel p+1, update and scatter of panel p)."""
    n = A0.shape[0]
    nt = n // B
    rng = np.random.default_rng(seed)
    A = np.tril(A0) + np.triu(rng.uniform(-1e3, 1e3, (n, n)), 1)   # only lower tiles are meaningful
    ldw = B * panel
    W = [np.full((n, ldw), np.nan) for _ in range(2)]
    U = [np.full((n, ldw), np.nan) for _ in range(2)]
    V = [np.full((n, ldw), np.nan) for _ in range(2)]
    panels = [(k0, min(panel, nt - k0)) for k0 in range(0, nt, panel)]
    _gather(A, W[0], *panels[0], nt)
    for p, (k0, bw) in enumerate(panels):
        cur, nxt = p & 1, (p & 1) ^ 1
        K = B * bw
        _panel_rows_K(W[cur], U[cur], V[cur], k0, bw)
        Wkk = W[cur][B * k0:B * (k0 + bw), :K].copy()                 # -A_KK^-1
        other = _rows([i for i in range(nt) if not k0 <= i < k0 + bw])
        U[cur][other, :K] = -W[cur][other, :K] @ Wkk.T                 # A_iK A_KK^-1
        if p + 1 < len(panels):
            k1, bw1 = panels[p + 1]
            _gather(A, W[nxt], k1, bw1, nt)           # before the update of panel p reaches it
            W[nxt][other, :B * bw1] -= U[cur][other, :K] @ W[cur][B * k1:B * (k1 + bw1), :K].T
            W[nxt][B * k0:B * (k0 + bw), :B * bw1] = U[cur][B * k1:B * (k1 + bw1), :K].T
        if nt > bw:
            _update_lower(A, U[cur], W[cur], K)
        _scatter(A, W[cur], U[cur], k0, bw, nt)
    L = np.tril(A)
    return -(L + np.tril(L, -1).T)   # the sweep leaves -A^-1


@pytest.mark.parametrize("nt,panel", [(6, 4), (9, 4), (9, 2), (5, 1)])
def test_blocked_sweep_with_lookahead_inverts(nt, panel):
    rng = np.random.default_rng(nt)
    n = B * nt
    X = rng.standard_normal((n, n))
    A = X @ X.T / n + np.eye(n)
    R = blocked_sweep_inverse(A, panel)
    E = np.linalg.inv(A)
    assert np.abs(R - E).max() / np.abs(E).max() < 1e-12


# ---------------------------------------------------------------- double-float
f32 = np.float32


def _add(a, b):
    return f32(f32(a) + f32(b))


def _sub(a, b):
    return f32(f32(a) - f32(b))


def _mul(a, b):
    return f32(f32(a) * f32(b))


def _fma(a, b, c):
    # a*b is exact in binary64 for binary32 a, b; one rounding of the sum
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def _two_sum(a, b):
    s = _add(a, b)
    bb = _sub(s, a)
    return s, _add(_sub(a, _sub(s, bb)), _sub(b, bb))


def _fast_two_sum(a, b):
    s = _add(a, b)
    return s, _sub(b, _sub(s, a))


def df_mul(a, b):
    p = _mul(a[0], b[0])
    e = _fma(a[0], b[0], -p)
    e = _fma(a[0], b[1], e)
    e = _fma(a[1], b[0], e)
    return _fast_two_sum(p, e)


def df_sub(a, b):
    s, e = _two_sum(a[0], -b[0])
    return _fast_two_sum(s, _add(e, _sub(a[1], b[1])))


def df_recip(d):
    r = f32(f32(1.0) / d[0])
    t = _fma(-d[0], r, f32(1.0))
    t = _fma(-d[1], r, t)
    return _fast_two_sum(r, _mul(r, t))


def df_sweep_inverse(A32):
    """The pivot kernel's sweep on the lower triangle in double-float."""
    m = A32.shape[0]
    S = [[(A32[i, j], f32(0)) for j in range(i + 1)] for i in range(m)]
    for p in range(m):
        inv = df_recip(S[p][p])
        col = [S[i][p] if i >= p else S[p][i] for i in range(m)]
        wv = [df_mul(c, inv) for c in col]
        for i in range(m):
            for j in range(i + 1):
                if i == p and j == p:
                    S[i][j] = (-inv[0], -inv[1])
                elif i == p:
                    S[i][j] = wv[j]
                elif j == p:
                    S[i][j] = wv[i]
                else:
                    S[i][j] = df_sub(S[i][j], df_mul(col[i], wv[j]))
    val = lambda x: np.float64(x[0]) + np.float64(x[1])
    return np.array([[-val(S[max(i, j)][min(i, j)]) for j in range(m)] for i in range(m)])


@pytest.mark.parametrize("shift", [1.0, 1e-3])
def test_double_float_sweep_tracks_binary64(shift):
    rng = np.random.default_rng(3)
    m = 24
    X = rng.standard_normal((m, m))
    A32 = (X @ X.T / m + shift * np.eye(m)).astype(np.float32)
    A = A32.astype(np.float64)
    E = np.linalg.inv(A)
    R = df_sweep_inverse(A32)
    err = np.abs(R - E).max() / np.abs(E).max()
    cond = np.linalg.cond(A)
    # binary32 would give cond x 6e-8; double-float stays near binary64
    assert err < cond * 2e-14, (err, cond)
    R32 = np.linalg.inv(A32).astype(np.float64)
    assert err < 1e-3 * np.abs(R32 - E).max() / np.abs(E).max()
