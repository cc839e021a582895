"""FastMNMF reference oracle (Sec. IV-H, App. C): plain complex128 / float64 NumPy.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute this
module; only the tests, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` use it.
It shares no code with the CUDA path.

Model (App. C).  In every frequency i the mixture follows the FastFCA model of Sec. IV: a
demixing matrix W_i and diagonal spatial weights lambda_imn.  The source power
spectrograms are factored across frequencies by NMF, Eq. 52:

    h_ijn = sum_k t_ikn v_jkn,        sigma^2_mij = sum_n lambda_imn h_ijn   (Eq. 28)

and the negative log-likelihood is Eq. 53: -J sum_i ln|det W_i|^2 + sum U/sigma^2 +
sum ln sigma^2, with U_mij = |w_im^H x_ij|^2 (Eq. 37).  The log-likelihood reported here is
its negative with the constant -I M J ln(pi) restored.

Notation: i frequency (I bins), j frame (J), k basis (K), n source (N), m channel (M).
Arrays: x (I, J, M) complex; W (I, M, M); lam (I, M, N); t (I, K, N); v (J, K, N).

One iteration.  App. C alternates ICA updates of every W_i with tensor-factor updates of
Lambda, T and V, and names IP for W and the MM algorithm for the rest without printing them.
* ``ip_all``  for every i, the IP sweep of Eq. 33-35 with sigma^2 of the current parameters
* ``mm_lam``  lambda_imn <- lambda_imn (sum_j h_ijn U/sigma^4 / sum_j h_ijn/sigma^2)^(1/2)
* ``mm_t``    t_ikn <- t_ikn (sum_mj lambda_imn v_jkn U/sigma^4 / sum_mj lambda_imn v_jkn/sigma^2)^(1/2)
* ``mm_v``    v_jkn <- v_jkn (sum_mi lambda_imn t_ikn U/sigma^4 / sum_mi lambda_imn t_ikn/sigma^2)^(1/2)

Readings where the paper is silent:
* The MM rules are the exponent-1/2 multiplicative updates of IS-NMF that Algorithm 2 gives
  for L and H, applied to each factor of the three-way model.  Each one is the minimiser of
  the standard auxiliary function of the IS divergence in that factor.
* Order per iteration: IP for every i, then U from the new W (Eq. 37), then Lambda, T, V in
  the order App. C lists them.  sigma^2 is recomputed from the current factors before each
  of the three updates, as Algorithm 2 recomputes LH between its L and H lines.
* No normalisation of the scale that lambda, t and v share, and no floors (the paper has
  none).
"""
from __future__ import annotations

import numpy as np

from oracle import fastfca as off

LN_PI = float(np.log(np.pi))


def h_of(t: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Eq. 52: h[i, j, n] = sum_k t[i, k, n] v[j, k, n]."""
    return np.einsum("ikn,jkn->ijn", t, v)


def sigma2(lam: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Eq. 28 with h from Eq. 52: s2[i, m, j] = sum_n lam[i, m, n] h[i, j, n]."""
    return np.einsum("imn,ijn->imj", lam, h)


def decorrelated_power(x: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Eq. 37 for every frequency: U[i, m, j] = |w_im^H x_ij|^2."""
    y = np.einsum("iam,ija->imj", W.conj(), x)
    return np.abs(y) ** 2


def ip_all(x: np.ndarray, W: np.ndarray, lam: np.ndarray, t: np.ndarray, v: np.ndarray) -> np.ndarray:
    """The IP sweep of Eq. 33-35 in every frequency, with sigma^2 of the given parameters."""
    h = h_of(t, v)
    Wn = np.empty_like(W)
    for i in range(x.shape[0]):
        Xhat = off.Xhat_from_x(x[i])
        Wn[i] = off.ip_sweep(Xhat, W[i].astype(np.complex128), lam[i], h[i].T)
    return Wn


def mm_lam(U, lam, t, v):
    """MM update of lambda (all i, m, n at once)."""
    h = h_of(t, v)
    s2 = sigma2(lam, h)
    num = np.einsum("imj,ijn->imn", U / s2 ** 2, h)
    den = np.einsum("imj,ijn->imn", 1.0 / s2, h)
    return lam * np.sqrt(num / den)


def mm_t(U, lam, t, v):
    """MM update of the bases t (all i, k, n at once)."""
    s2 = sigma2(lam, h_of(t, v))
    num = np.einsum("imn,jkn,imj->ikn", lam, v, U / s2 ** 2)
    den = np.einsum("imn,jkn,imj->ikn", lam, v, 1.0 / s2)
    return t * np.sqrt(num / den)


def mm_v(U, lam, t, v):
    """MM update of the activations v (all j, k, n at once): the sums run over every
    frequency, which is what couples the bins."""
    s2 = sigma2(lam, h_of(t, v))
    num = np.einsum("imn,ikn,imj->jkn", lam, t, U / s2 ** 2)
    den = np.einsum("imn,ikn,imj->jkn", lam, t, 1.0 / s2)
    return v * np.sqrt(num / den)


def iterate(x, W, lam, t, v):
    """One iteration: IP in every frequency, U, then the MM updates of lambda, t, v."""
    W = ip_all(x, W, lam, t, v)
    U = decorrelated_power(x, W)
    lam = mm_lam(U, lam, t, v)
    t = mm_t(U, lam, t, v)
    v = mm_v(U, lam, t, v)
    return W, lam, t, v


def loglik_per_f(x, W, lam, t, v) -> np.ndarray:
    """Eq. 53 negated per frequency, with the constant -M J ln(pi):
    l_i = J ln|det W_i|^2 - sum_{m,j} (U/sigma^2 + ln sigma^2) - M J ln(pi)."""
    I, J, M = x.shape
    U = decorrelated_power(x, W)
    s2 = sigma2(lam, h_of(t, v))
    _, logabsdet = np.linalg.slogdet(W)
    return J * 2.0 * logabsdet - np.sum(U / s2 + np.log(s2), axis=(1, 2)) - M * J * LN_PI


def loglik(x, W, lam, t, v) -> float:
    return float(np.sum(loglik_per_f(x, W, lam, t, v)))


def separate(x, W, lam, t, v) -> np.ndarray:
    """Source images by the FastFCA Wiener filter (Eq. 39) with h from Eq. 52:
    c[i, j, n] = W_i^{-H} diag(lambda_i[:, n] h_ijn / sigma^2_ij) W_i^H x_ij, shape (I, J, N, M)."""
    h = h_of(t, v)
    return np.stack([off.separate_fast(x[i], W[i], lam[i], h[i].T) for i in range(x.shape[0])])


def run(x, W0, lam0, t0, v0, iters: int, with_ll: bool = True):
    """``iters`` iterations from the given start.  Returns dict with W, lam, t, v (float64 /
    complex128 copies) and ll[it] = total log-likelihood after iteration it (when with_ll)."""
    x = np.asarray(x, dtype=np.complex128)
    W = np.asarray(W0, dtype=np.complex128).copy()
    lam = np.asarray(lam0, dtype=np.float64).copy()
    t = np.asarray(t0, dtype=np.float64).copy()
    v = np.asarray(v0, dtype=np.float64).copy()
    ll = []
    for _ in range(iters):
        W, lam, t, v = iterate(x, W, lam, t, v)
        if with_ll:
            ll.append(loglik(x, W, lam, t, v))
    return {"W": W, "lam": lam, "t": t, "v": v, "ll": np.array(ll, dtype=np.float64)}
