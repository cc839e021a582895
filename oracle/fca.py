"""Full-rank spatial covariance analysis (FCA) reference oracle, complex128 NumPy.

TEST INFRASTRUCTURE ONLY (see oracle/fastfca.py): the product path never imports it.

Follows Sec. III with the frequency index dropped:

* ``obs_cov``     Eq. 6: X_j = sum_n h_jn R_n
* ``mwf``         Eq. 7: F_jn = h_jn R_n X_j^{-1} (explicit M x M inverse)
* ``psi``         Eq. 12: Psi_jn = F_jn X^_j F_jn^H + (I - F_jn) h_jn R_n
* ``em_iterate``  Eq. 12 then Eq. 13: h_jn <- tr(R_n^{-1} Psi_jn) / M, then
                  R_n <- (1/J) sum_j Psi_jn / h_jn
* ``loglik``      Eq. 10 negated, with its constant -M J ln(pi) restored.
* ``gmean``       the matrix geometric mean A # B = A^1/2 (A^-1/2 B A^-1/2)^1/2 A^1/2
* ``mm_iterate``  Eq. 15-17: X_j = sum_n h_jn R_n; h_jn <- h_jn {tr(X^-1 X^ X^-1 R_n) /
                  tr(X^-1 R_n)}^1/2; R_n <- (sum_j h_jn X_j^-1)^-1 # [R_n (sum_j h_jn X_j^-1
                  X^_j X_j^-1) R_n]

Reading where the paper prints the two M-step updates side by side (Eq. 13): h is updated
first with the old R_n, then R_n with the new h.  Each is the exact maximiser of the EM
Q-function in its own variable with the other fixed, so the likelihood cannot decrease.

Reading of the MM rules (Eq. 15-17, App. B): both right-hand sides are evaluated at the
current parameters (X_j from Eq. 15, the current h and R_n), then h and R are replaced.  Each
printed rule is the exact minimiser of the auxiliary function in its own variable with the
other at its current value (the h inside the eliminated Gamma_jn and the h of Eq. 17 are the
same).
"""
from __future__ import annotations

import numpy as np

LN_PI = float(np.log(np.pi))


def obs_cov(R: np.ndarray, h: np.ndarray, j: int) -> np.ndarray:
    """Eq. 6: X_j = sum_n h_jn R_n.  R (N, M, M); h (N, J)."""
    return np.einsum("n,nab->ab", h[:, j], R)


def mwf(R: np.ndarray, h: np.ndarray, n: int, j: int) -> np.ndarray:
    """Eq. 7: F_jn = h_jn R_n X_j^{-1}."""
    return h[n, j] * R[n] @ np.linalg.inv(obs_cov(R, h, j))


def psi(x_j: np.ndarray, R: np.ndarray, h: np.ndarray, n: int, j: int) -> np.ndarray:
    """Eq. 12 for one (j, n), with X^_j = x_j x_j^H (Eq. 14)."""
    M = R.shape[1]
    F = mwf(R, h, n, j)
    Xhat = np.outer(x_j, x_j.conj())
    return F @ Xhat @ F.conj().T + (np.eye(M) - F) @ (h[n, j] * R[n])


def em_iterate(x: np.ndarray, R: np.ndarray, h: np.ndarray):
    """One EM iteration (Eq. 12-13) for one frequency bin.  x (J, M); R (N, M, M); h (N, J)."""
    x = np.asarray(x, dtype=np.complex128)
    J, M = x.shape
    N = R.shape[0]
    Psi = np.zeros((N, J, M, M), dtype=np.complex128)
    for j in range(J):
        for n in range(N):
            Psi[n, j] = psi(x[j], R, h, n, j)
    h_new = np.zeros_like(h, dtype=np.float64)
    for n in range(N):
        Rinv = np.linalg.inv(R[n])
        for j in range(J):
            h_new[n, j] = np.real(np.trace(Rinv @ Psi[n, j])) / M
    R_new = np.zeros_like(R, dtype=np.complex128)
    for n in range(N):
        R_new[n] = (Psi[n] / h_new[n][:, None, None]).sum(axis=0) / J
    return R_new, h_new


def loglik(x: np.ndarray, R: np.ndarray, h: np.ndarray) -> float:
    """-(Eq. 10) - M J ln(pi) = -sum_j [ln det X_j + x_j^H X_j^{-1} x_j] - M J ln(pi)."""
    x = np.asarray(x, dtype=np.complex128)
    J, M = x.shape
    total = 0.0
    for j in range(J):
        X = obs_cov(R, h, j)
        _, logdet = np.linalg.slogdet(X)
        total += logdet + np.real(x[j].conj() @ np.linalg.solve(X, x[j]))
    return float(-total - M * J * LN_PI)


def psd_power(A: np.ndarray, p: float) -> np.ndarray:
    """A^p = U diag(s^p) U^H from an eigenvalue decomposition of Hermitian PD A (App. B)."""
    s, U = np.linalg.eigh(A)
    return (U * s ** p) @ U.conj().T


def gmean(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A # B = A^1/2 (A^-1/2 B A^-1/2)^1/2 A^1/2 (the geometric mean defined after Eq. 17)."""
    Ah = psd_power(A, 0.5)
    Aih = psd_power(A, -0.5)
    G = Ah @ psd_power(Aih @ B @ Aih, 0.5) @ Ah
    return (G + G.conj().T) / 2


def mm_iterate(x: np.ndarray, R: np.ndarray, h: np.ndarray):
    """One MM iteration (Eq. 15-17) for one frequency bin.  x (J, M); R (N, M, M); h (N, J)."""
    x = np.asarray(x, dtype=np.complex128)
    J, M = x.shape
    N = R.shape[0]
    Xinv = np.stack([np.linalg.inv(obs_cov(R, h, j)) for j in range(J)])        # Eq. 15
    XiXhXi = np.stack([Xinv[j] @ np.outer(x[j], x[j].conj()) @ Xinv[j] for j in range(J)])
    h_new = np.zeros_like(h, dtype=np.float64)
    R_new = np.zeros_like(R, dtype=np.complex128)
    for n in range(N):
        for j in range(J):                                                       # Eq. 16
            num = np.real(np.trace(XiXhXi[j] @ R[n]))
            den = np.real(np.trace(Xinv[j] @ R[n]))
            h_new[n, j] = h[n, j] * np.sqrt(num / den)
        A = np.einsum("j,jab->ab", h[n], Xinv)                                   # Eq. 17
        Bm = R[n] @ np.einsum("j,jab->ab", h[n], XiXhXi) @ R[n]
        R_new[n] = gmean(np.linalg.inv(A), Bm)
    return R_new, h_new


def separate(x: np.ndarray, R: np.ndarray, h: np.ndarray) -> np.ndarray:
    """c_jn = F_jn x_j (Eq. 7) for one bin; x (J, M) -> c (J, N, M)."""
    x = np.asarray(x, dtype=np.complex128)
    J, M = x.shape
    N = R.shape[0]
    c = np.zeros((J, N, M), dtype=np.complex128)
    for j in range(J):
        for n in range(N):
            c[j, n] = mwf(R, h, n, j) @ x[j]
    return c


def run(x: np.ndarray, R0: np.ndarray, h0: np.ndarray, iters: int, freqs=None,
        with_ll: bool = True, algorithm: str = "em"):
    """FCA EM ("em", Eq. 12-13) or MM ("mm", Eq. 15-17) on every (or the listed) frequency bin.
    x (F, T, M); R0 (F, N, M, M); h0 (F, N, T)."""
    step = {"em": em_iterate, "mm": mm_iterate}[algorithm]
    F = x.shape[0]
    freqs = list(range(F)) if freqs is None else list(freqs)
    Rs, hs, lls = [], [], []
    for f in freqs:
        R = np.asarray(R0[f], dtype=np.complex128).copy()
        h = np.asarray(h0[f], dtype=np.float64).copy()
        ll_f = []
        for _ in range(iters):
            R, h = step(x[f], R, h)
            if with_ll:
                ll_f.append(loglik(x[f], R, h))
        Rs.append(R)
        hs.append(h)
        lls.append(ll_f)
    return {"freqs": freqs, "R": np.array(Rs), "h": np.array(hs),
            "ll": np.array(lls, dtype=np.float64)}
