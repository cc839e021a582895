"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and the oracle's tests.

This module draws random numbers and nothing else of the separation method: it holds no
step of FCA or FastFCA estimation (no covariance weighting, no IP update, no NMF update,
no Wiener filter).  It produces

* mixtures drawn from the local Gaussian model of Sec. III-A, Eq. 4: each source image is
  c_n(t,f) ~ CN(0, v_n(t,f) R_n(f)) and the mixture is their sum (Eq. 2), with
  v_n(t,f) = sum_k B_n(f,k) A_n(k,t) (nonnegative factors with Gamma(1,1) entries) and
  R_n(f) = a_n(f) a_n(f)^H + 0.01 I, a_n(f) the far-field steering vector of the array;
* the random starting point that both the CUDA path and the oracle are given:
  P_f = I, lambda_n(f) = 1 and v_n(t,f) = (||x(t,f)||^2 / (M N)) * u, u ~ U[0.5, 1.5);
* the FastMNMF starting point (App. C): W_i = I, lambda = 1, bases and activations from the
  frequency and frame marginals of ||x||^2 / (M N), each times its own u ~ U[0.5, 1.5).

The paper evaluates on recorded room impulse responses and speech (Sec. VII); those are not
available, so these model-generated mixtures with the paper's STFT shape family stand in.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SPEED_OF_SOUND = 343.0
FS = 16000.0


@dataclass(frozen=True)
class Workload:
    """One synthetic separation problem: F frequency bins, T frames, M mics, N sources."""
    name: str
    M: int
    N: int
    F: int
    T: int
    K: int
    iters: int
    array: str = "linear"          # "linear" or "circular"
    spacing: float = 0.04          # linear: mic spacing (m); circular: radius (m)
    seed: int = 1000
    extra: dict = field(default_factory=dict)


# The five workload families of the hot-path scope (sizes as named there).
WORKLOADS = {
    "small": Workload("fastfca_m2n3_f257_t250", M=2, N=3, F=257, T=250, K=4, iters=20,
                      array="linear", spacing=0.04, seed=1000),
    "fca_cmp": Workload("fastfca_m4n6_f513_t1250", M=4, N=6, F=513, T=1250, K=8, iters=100,
                        array="linear", spacing=0.03, seed=2000),
    "learned": Workload("fastfca_m3n5_f257_t500", M=3, N=5, F=257, T=500, K=8, iters=200,
                        array="linear", spacing=0.03, seed=4000),
    "large": Workload("fastfca_m8n12_f1025_t4000", M=8, N=12, F=1025, T=4000, K=16, iters=50,
                      array="circular", spacing=0.05, seed=5000),
}


def mic_positions(M: int, array: str, spacing: float) -> np.ndarray:
    """(M, 2) microphone coordinates in metres."""
    m = np.arange(M, dtype=np.float64)
    if array == "linear":
        return np.stack([m * spacing, np.zeros(M)], axis=1)
    if array == "circular":
        ang = 2.0 * np.pi * m / M
        return np.stack([spacing * np.cos(ang), spacing * np.sin(ang)], axis=1)
    raise ValueError(f"unknown array geometry {array!r}")


def steering_vectors(F: int, pos: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Far-field steering vectors a_n(f), shape (N, F, M), complex128.

    a_m(f) = exp(-i 2 pi nu_f (p_m . u(theta)) / c), nu_f = f fs / (2 (F - 1)).
    """
    nu = np.arange(F, dtype=np.float64) * FS / (2.0 * (F - 1))
    u = np.stack([np.cos(theta), np.sin(theta)], axis=1)          # (N, 2)
    delay = (u @ pos.T) / SPEED_OF_SOUND                            # (N, M)
    return np.exp(-2j * np.pi * nu[None, :, None] * delay[:, None, :])


@dataclass
class Mixture:
    x: np.ndarray            # (F, T, M) complex64, m fastest
    v_true: np.ndarray       # (N, F, T) float64 source powers
    R_true: np.ndarray       # (N, F, M, M) complex128 spatial covariances
    c_true: np.ndarray | None  # (N, F, T, M) complex64 source images (optional)


def generate_mixture(M: int, N: int, F: int, T: int, K: int, *, seed: int,
                     array: str = "linear", spacing: float = 0.04,
                     keep_images: bool = False) -> Mixture:
    """Draw one mixture from the model (see the module docstring).  F >= 2: the frequency
    grid nu_f = f fs / (2 (F - 1)) runs from 0 to fs / 2."""
    if F < 2:
        raise ValueError("the frequency grid needs F >= 2 (take one bin of a larger mixture)")
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = rng.uniform(0.0, np.pi, size=N)
    B = rng.gamma(1.0, 1.0, size=(N, F, K))
    A = rng.gamma(1.0, 1.0, size=(N, K, T))
    v = np.einsum("nfk,nkt->nft", B, A)
    a = steering_vectors(F, mic_positions(M, array, spacing), theta)   # (N, F, M)
    R = np.einsum("nfa,nfb->nfab", a, a.conj()) + 0.01 * np.eye(M)[None, None]
    chol = np.linalg.cholesky(R)                                        # (N, F, M, M)
    x = np.zeros((F, T, M), dtype=np.complex128)
    c_all = np.zeros((N, F, T, M), dtype=np.complex64) if keep_images else None
    for n in range(N):
        z = (rng.standard_normal((F, T, M)) + 1j * rng.standard_normal((F, T, M))) * np.sqrt(0.5)
        c = np.sqrt(v[n])[:, :, None] * np.einsum("fab,ftb->fta", chol[n], z)
        x += c
        if keep_images:
            c_all[n] = c.astype(np.complex64)
    return Mixture(x=x.astype(np.complex64), v_true=v, R_true=R, c_true=c_all)


def workload_mixture(w: Workload, index: int = 0, keep_images: bool = False) -> Mixture:
    return generate_mixture(w.M, w.N, w.F, w.T, w.K, seed=w.seed + index, array=w.array,
                            spacing=w.spacing, keep_images=keep_images)


@dataclass
class InitParams:
    P: np.ndarray     # (F, M, M) complex128, the joint diagonalizer (W in the paper)
    lam: np.ndarray   # (F, M, N) float32, [L]_{mn} = [Lambda_n]_{mm}
    v: np.ndarray     # (F, N, T) float32, [H]_{nt} = h_{tn}


def random_init(x: np.ndarray, N: int, *, seed: int) -> InitParams:
    """P = I, lambda = 1, v = (||x_t||^2 / (M N)) u with u ~ U[0.5, 1.5) (float32 values).

    The random factor breaks the symmetry between sources: with equal starting powers every
    source would receive identical updates forever.
    """
    F, T, M = x.shape
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x5EED))
    u = rng.uniform(0.5, 1.5, size=(F, N, T))
    pw = (np.abs(x.astype(np.complex128)) ** 2).sum(axis=2) / (M * N)   # (F, T)
    v = (pw[:, None, :] * u).astype(np.float32)
    v = np.maximum(v, np.float32(1e-30))
    P = np.broadcast_to(np.eye(M, dtype=np.complex128), (F, M, M)).copy()
    lam = np.ones((F, M, N), dtype=np.float32)
    return InitParams(P=P, lam=lam, v=v)


def fca_random_init(x: np.ndarray, N: int, *, seed: int):
    """Starting point for the full-matrix FCA comparison path: R_n = I, h as in random_init.

    Returns (R (F, N, M, M) complex128, h (F, N, T) float32).
    """
    F, T, M = x.shape
    p = random_init(x, N, seed=seed)
    R = np.broadcast_to(np.eye(M, dtype=np.complex128), (F, N, M, M)).copy()
    return R, p.v


@dataclass
class FastMNMFInit:
    W: np.ndarray     # (F, M, M) complex128, demixing matrices
    lam: np.ndarray   # (F, M, N) float32, spatial weights lambda_imn
    t: np.ndarray     # (F, K, N) float32, bases t_ikn
    v: np.ndarray     # (T, K, N) float32, activations v_jkn


def fastmnmf_random_init(x: np.ndarray, N: int, K: int, *, seed: int) -> FastMNMFInit:
    """W = I, lambda = 1; with p_ij = ||x_ij||^2 / (M N):
    t_ikn = (mean_j p_ij / K) u and v_jkn = (mean_i p_ij / mean_ij p_ij) u', u, u' ~ U[0.5, 1.5),
    so that sum_k t v starts near the separable part of p (float32 values)."""
    F, T, M = x.shape
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x3A3F))
    p = (np.abs(x.astype(np.complex128)) ** 2).sum(axis=2) / (M * N)     # (F, T)
    pf = p.mean(axis=1)
    pt = p.mean(axis=0) / p.mean()
    t = (pf[:, None, None] / K * rng.uniform(0.5, 1.5, size=(F, K, N))).astype(np.float32)
    v = (pt[:, None, None] * rng.uniform(0.5, 1.5, size=(T, K, N))).astype(np.float32)
    W = np.broadcast_to(np.eye(M, dtype=np.complex128), (F, M, M)).copy()
    lam = np.ones((F, M, N), dtype=np.float32)
    return FastMNMFInit(W=W, lam=lam, t=np.maximum(t, np.float32(1e-30)), v=np.maximum(v, np.float32(1e-30)))
