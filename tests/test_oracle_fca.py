"""Pins of the full-matrix FCA oracle (Sec. III, App. A) against independent facts."""
import numpy as np
import pytest

from oracle import fca
from tests.conftest import rand_complex, rand_hpd


def problem(rng, M=2, N=3, J=6):
    x = rand_complex(rng, J, M) * 1.5
    R = np.array([rand_hpd(rng, M) for _ in range(N)])
    h = rng.uniform(0.3, 2.0, size=(N, J))
    return x, R, h


def test_psi_equals_posterior_moments(rng):
    """Eq. 12 equals mu mu^H + Sigma with App. A's marginal posterior mean
    mu = h R X^{-1} x and covariance Sigma = h R - h^2 R X^{-1} R."""
    x, R, h = problem(rng, 3, 4, 3)
    for j in range(3):
        X = fca.obs_cov(R, h, j)
        Xi = np.linalg.inv(X)
        for n in range(4):
            mu = h[n, j] * R[n] @ Xi @ x[j]
            Sig = h[n, j] * R[n] - h[n, j] ** 2 * R[n] @ Xi @ R[n]
            assert np.allclose(fca.psi(x[j], R, h, n, j), np.outer(mu, mu.conj()) + Sig, atol=1e-11)


def test_psi_matches_stacked_gaussian_conditioning(rng):
    """App. A: the posterior of the stacked images c~ = (c_1, ..., c_N) given x = E c~ is
    Gaussian; Psi_n is the n-th diagonal block of its second moment (numpy on the MN system)."""
    M, N = 2, 3
    x, R, h = problem(rng, M, N, 2)
    for j in range(2):
        C = np.zeros((M * N, M * N), dtype=complex)
        for n in range(N):
            C[n * M:(n + 1) * M, n * M:(n + 1) * M] = h[n, j] * R[n]
        E = np.hstack([np.eye(M)] * N)
        K = np.linalg.solve((E @ C @ E.T).T, (C @ E.T).T).T     # C E^T (E C E^T)^{-1}
        mu = K @ x[j]
        Sig = C - K @ E @ C
        second = np.outer(mu, mu.conj()) + Sig
        for n in range(N):
            blk = second[n * M:(n + 1) * M, n * M:(n + 1) * M]
            assert np.allclose(fca.psi(x[j], R, h, n, j), blk, atol=1e-11)


def q_function(Psi, R, h):
    """App. A Q-function (up to constants): -sum_{j,n} [ln det(h R_n) + tr((h R_n)^{-1} Psi_jn)]."""
    N, J = h.shape
    tot = 0.0
    for n in range(N):
        Ri = np.linalg.inv(R[n])
        ld = np.linalg.slogdet(R[n])[1]
        for j in range(J):
            M = R.shape[1]
            tot -= M * np.log(h[n, j]) + ld + np.real(np.trace(Ri @ Psi[n, j])) / h[n, j]
    return tot


def test_m_step_updates_maximise_q_function(rng):
    """Eq. 13: h <- tr(R^{-1} Psi)/M maximises Q over h with R fixed, and R <- mean(Psi/h)
    maximises it over R with the new h fixed (brute-force perturbation)."""
    M, N, J = 2, 3, 5
    x, R, h = problem(rng, M, N, J)
    Psi = np.array([[fca.psi(x[j], R, h, n, j) for j in range(J)] for n in range(N)])
    R_new, h_new = fca.em_iterate(x, R, h)
    base = q_function(Psi, R, h_new)
    for n in range(N):
        for j in range(J):
            for eps in (1e-4, -1e-4):
                hp = h_new.copy()
                hp[n, j] *= 1 + eps
                assert q_function(Psi, R, hp) < base
    base = q_function(Psi, R_new, h_new)
    for n in range(N):
        for _ in range(4):
            D = rand_hpd(rng, M) - rand_hpd(rng, M)
            D = (D + D.conj().T) / 2
            for eps in (1e-4, -1e-4):
                Rp = R_new.copy()
                Rp[n] = R_new[n] + eps * D
                assert q_function(Psi, Rp, h_new) < base


def test_em_does_not_decrease_loglik(rng):
    """Sec. III-C: EM never decreases the likelihood."""
    x, R, h = problem(rng, 3, 4, 12)
    ll = fca.loglik(x, R, h)
    for _ in range(15):
        R, h = fca.em_iterate(x, R, h)
        ll_new = fca.loglik(x, R, h)
        assert ll_new >= ll - 1e-9 * abs(ll)
        ll = ll_new


def test_fca_images_sum_to_mixture(rng):
    """Eq. 2 with Eq. 7: sum_n h_n R_n X^{-1} = I, so the images add up to x."""
    x, R, h = problem(rng, 3, 4, 5)
    assert np.allclose(fca.separate(x, R, h).sum(axis=1), x, atol=1e-11)
