"""FastFCA reference oracle: plain complex128 NumPy, one frequency bin at a time.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute this
module; only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
use it.  It shares no code with the CUDA path.

Every function follows the paper's equations in the paper's order and notation (the frequency
index i is dropped, as in Sec. III-IV; the frame index j runs over T frames, so J = T):

* ``Xhat_from_x``        Eq. 14, X^_j = x_j x_j^H (or the block average of Sec. VI-B)
* ``sigma2``             Eq. 28 with Eq. 38: sigma^2_{mj} = [L H]_{mj}
* ``weighted_cov``       Eq. 33: Q_m = (1/J) sum_j X^_j / sigma^2_{mj}
* ``ip_update_column``   Eq. 34 then Eq. 35 (one column of W)
* ``decorrelated_power`` Eq. 37: U_{mj} = w_m^H X^_j w_m
* ``nmf_em_step``        Algorithm 1, the body of the n-loop (G_n, Phi_n, L[:, n], H[n, :])
* ``iterate``            Algorithm 1, one pass of the repeat loop
* ``nmf_mm_step``        Algorithm 2, the L and H lines (MM for IS-NMF)
* ``iterate_mm``         Algorithm 2, one pass of the repeat loop
* ``loglik``             Eq. 31 (negated, with its additive constant -M J ln(pi) restored)
* ``mwf``/``separate``   Eq. 39: F_jn = W^{-H} diag(L[:, n] H[n, j] / sigma^2_{:, j}) W^H
* ``separate_blocks``    Eq. 39 with the block powers of Sec. VI-B

Readings where the paper is silent:
* Inside the n-loop the updates are Gauss-Seidel: G_n uses L and H as already updated for
  n' < n; L[:, n] divides by the old H[n, :]; H[n, :] divides by the new L[:, n].
* Eq. 34 uses W with columns 1..m-1 already updated in this sweep.
* The square root of Eq. 35 takes the real part of w^H Q w (real for Hermitian Q).
* No floors are applied to sigma^2, L or H (the paper has none).
* Algorithm 2 lists the L line before the H line: H is updated with sigma^2 = LH recomputed
  from the new L.
"""
from __future__ import annotations

import numpy as np

LN_PI = float(np.log(np.pi))


def Xhat_from_x(x: np.ndarray, B: int = 1) -> np.ndarray:
    """Eq. 14: X^_j = x_j x_j^H for frames x (J, M).  With B > 1, Sec. VI-B: the average of
    x x^H over each block of B consecutive frames (J must be a multiple of B)."""
    x = np.asarray(x, dtype=np.complex128)
    outer = x[:, :, None] * x[:, None, :].conj()
    if B == 1:
        return outer
    J = x.shape[0] // B
    return outer[: J * B].reshape(J, B, *outer.shape[1:]).mean(axis=1)


def sigma2(L: np.ndarray, H: np.ndarray) -> np.ndarray:
    """Eq. 28 with Eq. 38: sigma^2 = L H, an M x J matrix."""
    return L @ H


def weighted_cov(Xhat: np.ndarray, s2_row: np.ndarray) -> np.ndarray:
    """Eq. 33: Q_m = (1/J) sum_j X^_j / sigma^2_{mj} for one m (s2_row has shape (J,))."""
    J = Xhat.shape[0]
    return (Xhat / s2_row[:, None, None]).sum(axis=0) / J


def ip_update_column(W: np.ndarray, Q_m: np.ndarray, m: int) -> np.ndarray:
    """Eq. 34 (w_m <- (W^H Q_m)^{-1} e_m) then Eq. 35 (w_m <- w_m / sqrt(w_m^H Q_m w_m)).

    Returns a new W with column m replaced; the other columns are unchanged."""
    M = W.shape[0]
    e_m = np.zeros(M, dtype=np.complex128)
    e_m[m] = 1.0
    w = np.linalg.solve(W.conj().T @ Q_m, e_m)
    quad = np.real(w.conj() @ Q_m @ w)
    if not quad > 0.0:
        raise FloatingPointError("w^H Q_m w is not positive")
    W = W.copy()
    W[:, m] = w / np.sqrt(quad)
    return W


def decorrelated_power(Xhat: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Eq. 37: U_{mj} = w_m^H X^_j w_m, an M x J matrix."""
    return np.real(np.einsum("am,jab,bm->mj", W.conj(), Xhat, W))


def nmf_em_step(U: np.ndarray, L: np.ndarray, H: np.ndarray, n: int):
    """Algorithm 1, one pass of the n-loop body.  Returns new (L, H) (copies)."""
    L = L.copy()
    H = H.copy()
    M, J = U.shape
    S = np.outer(L[:, n], H[n, :])                       # [L]_{:,n} [H]_{n,:}
    G = S / (L @ H)                                      # G_n = S (.) (LH)^{o-1}
    Phi = G ** 2 * U + (1.0 - G) * S                     # Phi_n
    L[:, n] = (Phi @ (1.0 / H[n, :])) / J                # (1/J) Phi_n [(H^T)^{o-1}]_{:,n}
    H[n, :] = ((1.0 / L[:, n]) @ Phi) / M                # (1/M) [(L^T)^{o-1}]_{n,:} Phi_n
    return L, H


def nmf_mm_step(U: np.ndarray, L: np.ndarray, H: np.ndarray):
    """Algorithm 2, the L and H lines: multiplicative MM updates of IS-NMF U ~ LH with the
    exponent 1/2.  Returns new (L, H)."""
    S = sigma2(L, H)
    L = L * np.sqrt(((U * S ** -2) @ H.T) / ((S ** -1) @ H.T))     # L (.) {[U (.) (LH)^-2] H^T / (LH)^-1 H^T}^1/2
    S = sigma2(L, H)                                                # with the new L
    H = H * np.sqrt((L.T @ (U * S ** -2)) / (L.T @ (S ** -1)))     # H (.) {L^T [U (.) (LH)^-2] / L^T (LH)^-1}^1/2
    return L, H


def ip_sweep(Xhat: np.ndarray, W: np.ndarray, L: np.ndarray, H: np.ndarray) -> np.ndarray:
    """Algorithm 1, the m-loop: Q_m from the current L, H, then Eq. 34-35 for m = 1..M."""
    M = W.shape[0]
    s2 = sigma2(L, H)
    for m in range(M):
        Q_m = weighted_cov(Xhat, s2[m])
        W = ip_update_column(W, Q_m, m)
    return W


def iterate(Xhat: np.ndarray, W: np.ndarray, L: np.ndarray, H: np.ndarray):
    """Algorithm 1, one pass of the repeat loop for one frequency bin.

    Xhat (J, M, M) complex128; W (M, M) complex128; L (M, N); H (N, J), both float64.
    Returns the updated (W, L, H)."""
    W = ip_sweep(Xhat, W, L, H)
    U = decorrelated_power(Xhat, W)
    N = L.shape[1]
    for n in range(N):
        L, H = nmf_em_step(U, L, H, n)
    return W, L, H


def iterate_mm(Xhat: np.ndarray, W: np.ndarray, L: np.ndarray, H: np.ndarray):
    """Algorithm 2, one pass of the repeat loop for one frequency bin (shapes as ``iterate``):
    the same IP sweep and U, then the MM updates of L and H."""
    W = ip_sweep(Xhat, W, L, H)
    U = decorrelated_power(Xhat, W)
    L, H = nmf_mm_step(U, L, H)
    return W, L, H


def loglik(Xhat: np.ndarray, W: np.ndarray, L: np.ndarray, H: np.ndarray) -> float:
    """Log-likelihood of one frequency bin: the negative of Eq. 31 minus M J ln(pi).

    l = J ln|det W|^2 - sum_{m,j} (U_{mj} / sigma^2_{mj} + ln sigma^2_{mj}) - M J ln(pi)."""
    J = Xhat.shape[0]
    M = W.shape[0]
    U = decorrelated_power(Xhat, W)
    s2 = sigma2(L, H)
    _, logabsdet = np.linalg.slogdet(W)
    return float(J * 2.0 * logabsdet - np.sum(U / s2 + np.log(s2)) - M * J * LN_PI)


def mwf(W: np.ndarray, L: np.ndarray, H: np.ndarray, n: int, j: int) -> np.ndarray:
    """Eq. 39: the M x M Wiener filter F_jn = W^{-H} diag(g) W^H, g_m = L_mn H_nj / sigma^2_mj."""
    s2 = sigma2(L, H)[:, j]
    g = L[:, n] * H[n, j] / s2
    return np.linalg.inv(W.conj().T) @ np.diag(g) @ W.conj().T


def separate(x: np.ndarray, W: np.ndarray, L: np.ndarray, H: np.ndarray) -> np.ndarray:
    """Source images c_jn = F_jn x_j (Eq. 39) for one bin; x (J, M) -> c (J, N, M)."""
    x = np.asarray(x, dtype=np.complex128)
    J, M = x.shape
    N = L.shape[1]
    c = np.zeros((J, N, M), dtype=np.complex128)
    for j in range(J):
        for n in range(N):
            c[j, n] = mwf(W, L, H, n, j) @ x[j]
    return c


def separate_fast(x: np.ndarray, W: np.ndarray, L: np.ndarray, H: np.ndarray) -> np.ndarray:
    """Eq. 39 evaluated frame-vectorised (same arithmetic as ``separate``, without the
    per-(j, n) loops): decorrelate, scale by the diagonal gains, project back."""
    x = np.asarray(x, dtype=np.complex128)
    WH = W.conj().T
    y = x @ WH.T                                           # y_j = W^H x_j, (J, M)
    s2 = sigma2(L, H)                                      # (M, J)
    g = L[:, :, None] * H[None, :, :] / s2[:, None, :]     # (M, N, J)
    WmH = np.linalg.inv(WH)
    return np.einsum("ab,bnj,jb->jna", WmH, g, y)


# ----------------------------------------------------------------------------- whole problem
def separate_blocks(x: np.ndarray, W: np.ndarray, L: np.ndarray, H: np.ndarray, B: int) -> np.ndarray:
    """Eq. 39 under the piecewise-stationary model of Sec. VI-B: every frame b of block j has
    the block's covariances, so frame t is filtered with the powers H[:, t // B]."""
    return separate_fast(x, W, L, np.repeat(np.asarray(H, dtype=np.float64), B, axis=1))


def run(x: np.ndarray, P: np.ndarray, lam: np.ndarray, v: np.ndarray, iters: int,
        freqs=None, with_ll: bool = True, algorithm: str = "em", block: int = 1):
    """Algorithm 1 ("em", IP+EM) or Algorithm 2 ("mm", IP+MM) for every frequency bin (or the
    listed ones), ``iters`` repeats each.  With block = B > 1 the input is the block average
    X^_j of Sec. VI-B and v has T / B columns.

    x (F, T, M) complex; P (F, M, M); lam (F, M, N); v (F, N, T).
    Returns dict with W, L, H (float64/complex128 copies for the processed bins) and
    ll[f_index, it] = log-likelihood after iteration it (when with_ll)."""
    F = x.shape[0]
    freqs = list(range(F)) if freqs is None else list(freqs)
    step = {"em": iterate, "mm": iterate_mm}[algorithm]
    Ws, Ls, Hs, lls = [], [], [], []
    for f in freqs:
        Xhat = Xhat_from_x(x[f], block)
        W = np.asarray(P[f], dtype=np.complex128).copy()
        L = np.asarray(lam[f], dtype=np.float64).copy()
        H = np.asarray(v[f], dtype=np.float64).copy()
        ll_f = []
        for _ in range(iters):
            W, L, H = step(Xhat, W, L, H)
            if with_ll:
                ll_f.append(loglik(Xhat, W, L, H))
        Ws.append(W)
        Ls.append(L)
        Hs.append(H)
        lls.append(ll_f)
    return {"freqs": freqs, "W": np.array(Ws), "L": np.array(Ls), "H": np.array(Hs),
            "ll": np.array(lls, dtype=np.float64)}
