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


# ---------------------------------------------------------------------------- MM (Eq. 15-17)
def test_geometric_mean_solves_the_riccati_equation(rng):
    """A # B is the PD solution X of X A^-1 X = B (the footnote to Eq. 17); M = 1 gives sqrt(ab)."""
    for M in (1, 2, 3, 4):
        A = rand_hpd(rng, M)
        B = rand_hpd(rng, M, scale=2.0)
        G = fca.gmean(A, B)
        assert np.allclose(G, G.conj().T, atol=1e-12)
        assert np.all(np.linalg.eigvalsh(G) > 0)
        assert np.allclose(G @ np.linalg.solve(A, G), B, rtol=1e-9, atol=1e-9)
    a, b = 2.5, 7.0
    assert np.isclose(fca.gmean(np.array([[a]]), np.array([[b]]))[0, 0].real, np.sqrt(a * b))


def _mm_aux(x, R, h, R_cur, h_cur):
    """The auxiliary function J+ of App. B at the auxiliary variables of (R_cur, h_cur)."""
    J, M = x.shape
    N = R.shape[0]
    val = 0.0
    for j in range(J):
        Pi = fca.obs_cov(R_cur, h_cur, j)
        Pii = np.linalg.inv(Pi)
        val += np.linalg.slogdet(Pi)[1] - M
        q = 0.0
        for n in range(N):
            G = h_cur[n, j] * R_cur[n] @ Pii
            val += h[n, j] * np.real(np.trace(R[n] @ Pii))
            q += np.real(x[j].conj() @ G.conj().T @ np.linalg.solve(R[n], G @ x[j])) / h[n, j]
        val += q
    return val


def test_mm_updates_are_coordinate_minimisers_of_the_auxiliary_function(rng):
    """Each rule of Eq. 16-17 minimises J+ (App. B) in its own variable at the current point:
    the h update is the 1-D minimiser; the R update satisfies the stationarity (Riccati)
    condition R (sum h Pi^-1) R = sum Gamma x x^H Gamma^H / h and lowers J+ against nearby R."""
    M, N, J = 2, 3, 6
    x = rand_complex(rng, J, M)
    R = np.stack([rand_hpd(rng, M) for _ in range(N)])
    h = rng.uniform(0.3, 2.0, (N, J))
    R1, h1 = fca.mm_iterate(x, R, h)
    from scipy.optimize import minimize_scalar
    for n in range(N):
        for j in range(J):
            def f(val, n=n, j=j):
                hh = h.copy()
                hh[n, j] = val
                return _mm_aux(x, R, hh, R, h)
            best = minimize_scalar(f, bounds=(1e-4, 50.0), method="bounded", options={"xatol": 1e-12})
            assert abs(best.x - h1[n, j]) <= 1e-5 * h1[n, j]
    for n in range(N):
        Xi = [np.linalg.inv(fca.obs_cov(R, h, j)) for j in range(J)]
        A = sum(h[n, j] * Xi[j] for j in range(J))
        Bm = sum(h[n, j] * R[n] @ Xi[j] @ np.outer(x[j], x[j].conj()) @ Xi[j] @ R[n] for j in range(J))
        assert np.allclose(R1[n] @ A @ R1[n], Bm, rtol=1e-9, atol=1e-9)
        base = _mm_aux(x, np.where(np.arange(N)[:, None, None] == n, R1, R), h, R, h)
        for _ in range(5):
            D = rand_hpd(rng, M) * 1e-3
            D = D - np.trace(D) / M * np.eye(M)
            Rp = R.copy()
            Rp[n] = R1[n] + D
            if np.all(np.linalg.eigvalsh(Rp[n]) > 0):
                assert _mm_aux(x, Rp, h, R, h) >= base - 1e-12 * abs(base)


def test_fca_mm_log_likelihood_is_monotone(rng):
    for _ in range(5):
        M, N, J = 3, 4, 25
        x = rand_complex(rng, J, M)
        R = np.stack([rand_hpd(rng, M) for _ in range(N)])
        h = rng.uniform(0.3, 2.0, (N, J))
        ll = fca.loglik(x, R, h)
        for _ in range(15):
            R, h = fca.mm_iterate(x, R, h)
            l2 = fca.loglik(x, R, h)
            assert l2 >= ll - 1e-9 * abs(ll)
            ll = l2
