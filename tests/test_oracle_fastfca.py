"""Pins of the FastFCA oracle against facts fixed by the paper and by mathematics.

Each test ties one oracle function to something other than itself: a library routine that
computes the same quantity another way, a closed form, an identity the paper states, or a
brute-force search.  A plausible slip in the oracle (a dropped term, a wrong sign or index,
a transposed or unconjugated operand) breaks at least one of them.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

from oracle import fastfca as ff
from oracle import fca
from paper_2101_08563_gb300 import synth  # noqa: E402
from tests.conftest import rand_complex, rand_hpd

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_problem(rng, M=2, N=3, J=7):
    x = rand_complex(rng, J, M) * 2.0
    W = rand_complex(rng, M, M) + 2.0 * np.eye(M)
    L = rng.uniform(0.2, 2.0, size=(M, N))
    H = rng.uniform(0.2, 2.0, size=(N, J))
    return x, W, L, H


def jd_covariances(W, L):
    """Eq. 19: R_n = W^{-H} Lambda_n W^{-1}, [Lambda_n]_mm = L_mn."""
    Wi = np.linalg.inv(W)
    return np.array([Wi.conj().T @ np.diag(L[:, n]) @ Wi for n in range(L.shape[1])])


def complex_gauss_logpdf_via_real(x, S):
    """log CN(x | 0, S) through the equivalent real 2M-dimensional Gaussian (scipy)."""
    M = S.shape[0]
    C = 0.5 * np.block([[S.real, -S.imag], [S.imag, S.real]])
    return scipy.stats.multivariate_normal(mean=np.zeros(2 * M), cov=C).logpdf(
        np.concatenate([x.real, x.imag]))


# ----------------------------------------------------------------------------- shapes (Sec. VII)
def test_paper_shape_family_golden():
    """Sec. III-D and Table I: 8 s at 16 kHz, 1024-point frames, 512 shift -> 513 x 249 bins."""
    g = json.load(open(os.path.join(GOLDEN, "paper_shapes.json")))
    frames = (g["fs_hz"] * g["seconds"] - g["frame_len"]) // g["frame_shift"] + 1
    bins = g["frame_len"] // 2 + 1
    assert frames == g["frames"]
    assert bins == g["bins"]
    assert bins * frames == g["tf_points"]


# ----------------------------------------------------------------------------- log-likelihood
def test_loglik_matches_explicit_gaussian_density(rng):
    """Eq. 31 (with Eq. 25's |det W|^2 and the -MJ ln(pi) constant) equals the sum of proper
    complex Gaussian log-densities N_c(x_j | 0, sum_n h_jn R_n), evaluated by scipy through
    the real 2M-dimensional representation, with R_n from Eq. 19."""
    for M, N in [(2, 3), (3, 5)]:
        x, W, L, H = small_problem(rng, M, N, J=6)
        R = jd_covariances(W, L)
        ref = sum(complex_gauss_logpdf_via_real(x[j], np.einsum("n,nab->ab", H[:, j], R))
                  for j in range(x.shape[0]))
        got = ff.loglik(ff.Xhat_from_x(x), W, L, H)
        assert got == pytest.approx(ref, rel=1e-11, abs=1e-9)


def test_fca_loglik_matches_explicit_gaussian_density(rng):
    """Eq. 10 negated (with constant) against scipy's Gaussian density, general (non-JD) R."""
    M, N, J = 3, 4, 5
    x = rand_complex(rng, J, M)
    R = np.array([rand_hpd(rng, M) for _ in range(N)])
    h = rng.uniform(0.1, 3.0, size=(N, J))
    ref = sum(complex_gauss_logpdf_via_real(x[j], np.einsum("n,nab->ab", h[:, j], R))
              for j in range(J))
    assert fca.loglik(x, R, h) == pytest.approx(ref, rel=1e-11, abs=1e-9)


def test_cost_at_identity_is_isnmf(rng):
    """Footnote of Sec. IV-E: with W = I the cost is the IS-NMF cost of U ~ LH (Eq. 36):
    -loglik = sum D_IS(U | LH) + sum ln U + MJ + MJ ln(pi)."""
    x, _, L, H = small_problem(rng, 3, 4, J=9)
    M, J = 3, 9
    U = np.abs(x.T) ** 2
    S = L @ H
    d_is = np.sum(U / S - np.log(U / S) - 1.0)
    got = -ff.loglik(ff.Xhat_from_x(x), np.eye(M, dtype=complex), L, H)
    assert got == pytest.approx(d_is + np.log(U).sum() + M * J + M * J * np.log(np.pi), rel=1e-12)


def test_ajd_plus_isnmf_identity_piecewise(rng):
    """Eq. 45 (Sec. VI-C): for block-averaged X^_j with B >= M, the piecewise cost (Eq. 44)
    equals sum_j D_LD(W^H X^_j W | ddiag(.)) + sum D_IS(<|y|^2> | sigma^2) up to terms free
    of (W, L, H); here that constant is sum_j ln det X^_j + MJ."""
    M, N, B, J = 3, 4, 5, 6
    x = rand_complex(rng, J * B, M)
    Xh = ff.Xhat_from_x(x, B=B)
    consts = []
    for _ in range(3):
        W = rand_complex(rng, M, M) + 1.5 * np.eye(M)
        L = rng.uniform(0.2, 2.0, size=(M, N))
        H = rng.uniform(0.2, 2.0, size=(N, J))
        negll = -ff.loglik(Xh, W, L, H) - M * J * np.log(np.pi)
        dld = 0.0
        for j in range(J):
            A = W.conj().T @ Xh[j] @ W
            D = np.diag(np.real(np.diag(A)))
            Z = A @ np.linalg.inv(D)
            dld += np.real(np.trace(Z)) - np.linalg.slogdet(Z)[1] - M
        u = np.real(np.einsum("am,jab,bm->mj", W.conj(), Xh, W))
        s = L @ H
        dis = np.sum(u / s - np.log(u / s) - 1.0)
        consts.append(negll - dld - dis)
    expect = sum(np.linalg.slogdet(Xh[j])[1] for j in range(J)) + M * J
    assert np.allclose(consts, expect, rtol=1e-10, atol=1e-9)


def test_log_det_divergence_nonnegative(rng):
    """Theorem 2 (App. B): D_LD(A | B) >= 0 with equality iff A = B."""
    for _ in range(20):
        A, B = rand_hpd(rng, 3), rand_hpd(rng, 3)
        Z = A @ np.linalg.inv(B)
        d = np.real(np.trace(Z)) - np.linalg.slogdet(Z)[1] - 3
        assert d > 0
    Z = np.eye(3)
    assert np.real(np.trace(Z)) - np.linalg.slogdet(Z)[1] - 3 == pytest.approx(0.0, abs=1e-14)


# ----------------------------------------------------------------------------- IP (Eq. 32-35)
def test_ip_column_is_stationary(rng):
    """Eq. 32: after updating column m by Eq. 34-35, W^H Q_m w_m = e_m."""
    M = 4
    W = rand_complex(rng, M, M) + 2 * np.eye(M)
    for m in range(M):
        Q = rand_hpd(rng, M)
        W = ff.ip_update_column(W, Q, m)
        e = np.zeros(M)
        e[m] = 1
        assert np.allclose(W.conj().T @ Q @ W[:, m], e, atol=1e-12)
        assert np.real(W[:, m].conj() @ Q @ W[:, m]) == pytest.approx(1.0, abs=1e-12)


def test_ip_two_channels_reaches_generalized_eigenvectors(rng):
    """Sec. IV-A / Sec. VI-A: two HPD matrices are exactly jointly diagonalised by the
    generalised eigenvectors of (Q_2, Q_1).  Iterating IP (Eq. 34-35) with fixed Q_1, Q_2
    must converge to them (scipy.linalg.eigh), up to phase, with w_m^H Q_m w_m = 1."""
    Q1, Q2 = rand_hpd(rng, 2), rand_hpd(rng, 2)
    W = np.eye(2, dtype=complex)
    for _ in range(300):
        W = ff.ip_update_column(W, Q1, 0)
        W = ff.ip_update_column(W, Q2, 1)
    _, V = scipy.linalg.eigh(Q2, Q1)          # V^H Q1 V = I, V^H Q2 V diagonal
    for m, Q in [(0, Q1), (1, Q2)]:
        w = W[:, m]
        # w is parallel to exactly one generalised eigenvector
        cos = [abs(v.conj() @ Q1 @ w) / np.sqrt(np.real(v.conj() @ Q1 @ v) * np.real(w.conj() @ Q1 @ w))
               for v in V.T]
        assert max(cos) == pytest.approx(1.0, abs=1e-10)
        assert np.real(w.conj() @ Q @ w) == pytest.approx(1.0, abs=1e-12)
    assert abs(W[:, 0].conj() @ Q1 @ W[:, 1]) < 1e-10
    assert abs(W[:, 0].conj() @ Q2 @ W[:, 1]) < 1e-10


def test_weighted_cov_matches_matrix_product(rng):
    """Eq. 33 equals X^T diag(1/sigma^2_m) conj(X) / J (a BLAS product, not a sum of outer products)."""
    x, W, L, H = small_problem(rng, 3, 4, J=11)
    s2 = L @ H
    for m in range(3):
        Q = ff.weighted_cov(ff.Xhat_from_x(x), s2[m])
        ref = (x.T * (1.0 / s2[m])) @ x.conj() / x.shape[0]
        assert np.allclose(Q, ref, atol=1e-13)


def test_ip_does_not_decrease_loglik(rng):
    """Sec. IV-E: IP never decreases the likelihood; checked after every column update."""
    x, W, L, H = small_problem(rng, 3, 5, J=20)
    Xh = ff.Xhat_from_x(x)
    s2 = L @ H
    ll = ff.loglik(Xh, W, L, H)
    for _ in range(3):
        for m in range(3):
            W = ff.ip_update_column(W, ff.weighted_cov(Xh, s2[m]), m)
            ll_new = ff.loglik(Xh, W, L, H)
            assert ll_new >= ll - 1e-9 * abs(ll)
            ll = ll_new


def sweep_problem(rng, M=4, N=3, J=40):
    """A problem whose rows of sigma^2 = LH differ in shape, not only in scale (L spans three
    decades per row), so each Q_m of Eq. 33 is a genuinely different matrix."""
    x = rand_complex(rng, J, M) * 2.0
    W = rand_complex(rng, M, M) + 2.0 * np.eye(M)
    L = np.exp(rng.uniform(-3.5, 3.5, size=(M, N)))
    H = rng.uniform(0.05, 3.0, size=(N, J))
    return x, W, L, H


def q_by_definition(x, L, H):
    """Eq. 33 written out frame by frame, with sigma^2_{mj} = sum_n L_mn H_nj (Eq. 28, 38)."""
    J, M = x.shape
    Q = np.zeros((M, M, M), complex)
    for m in range(M):
        for j in range(J):
            s2 = sum(L[m, n] * H[n, j] for n in range(L.shape[1]))
            Q[m] += np.outer(x[j], x[j].conj()) / s2
        Q[m] /= J
    return Q


def test_ip_sweep_last_column_is_stationary_for_its_own_q(rng):
    """Eq. 32 after a whole sweep (Algorithm 1's m-loop): the last column was updated with every
    other column already final, so W^H Q_M w_M = e_M holds exactly for its own Q_M, and for
    no other Q_m (the rows of sigma^2 differ)."""
    M = 4
    x, W0, L, H = sweep_problem(rng, M)
    Q = q_by_definition(x, L, H)
    W = ff.ip_sweep(ff.Xhat_from_x(x), W0, L, H)
    e = np.zeros(M)
    e[M - 1] = 1.0
    scale = np.linalg.norm(W) ** 2 * np.linalg.norm(Q[M - 1])
    assert np.allclose(W.conj().T @ Q[M - 1] @ W[:, M - 1], e, atol=1e-12 * scale)
    for m in range(M - 1):
        assert np.linalg.norm(W.conj().T @ Q[m] @ W[:, M - 1] - e) > 1e-3


def test_ip_sweep_is_the_sequence_of_column_updates(rng):
    """The sweep equals M calls of Eq. 34-35 in order, column m with its own Q_m and the W that
    the previous columns left (each call pinned on its own above); each column satisfies
    Eq. 32 for its Q_m at the moment it is updated.  A sweep that solved every column with the
    W it started from, or used one Q for all m, gives a different W."""
    M = 4
    x, W0, L, H = sweep_problem(rng, M)
    Q = q_by_definition(x, L, H)
    W = W0.copy()
    for m in range(M):
        W = ff.ip_update_column(W, Q[m], m)
        e = np.zeros(M)
        e[m] = 1.0
        assert np.allclose(W.conj().T @ Q[m] @ W[:, m], e, atol=1e-10)
    Wsweep = ff.ip_sweep(ff.Xhat_from_x(x), W0, L, H)
    assert np.allclose(Wsweep, W, rtol=0, atol=1e-12 * np.abs(W).max())
    # the slips this pins against give visibly different results on this problem
    W_stale = W0.copy()
    for m in range(M):
        W_stale[:, m] = ff.ip_update_column(W0, Q[m], m)[:, m]
    W_oneq = W0.copy()
    for m in range(M):
        W_oneq = ff.ip_update_column(W_oneq, Q[0], m)
    for bad in (W_stale, W_oneq):
        assert np.abs(bad - W).max() > 1e-3 * np.abs(W).max()


# ----------------------------------------------------------------------------- NMF EM (Alg. 1)
def test_phi_is_gaussian_posterior_second_moment(rng):
    """Phi_n of Algorithm 1 is E[|s_n|^2 | y] for y = sum_n s_n, s_n ~ CN(0, S_n) independent:
    checked against textbook Gaussian conditioning on the N-vector s (numpy solve)."""
    M, N, J = 2, 3, 4
    x, W, L, H = small_problem(rng, M, N, J)
    U = np.abs(rand_complex(rng, M, J)) ** 2 + 0.1
    y_abs = np.sqrt(U)
    n = 1
    S = np.outer(L[:, n], H[n, :])
    G = S / (L @ H)
    Phi = G ** 2 * U + (1 - G) * S
    for m in range(M):
        for j in range(J):
            D = np.diag(L[m, :] * H[:, j])
            one = np.ones((N, 1))
            k = D @ one @ np.linalg.inv(one.T @ D @ one)
            mean = (k * y_abs[m, j])[:, 0]
            cov = D - k @ one.T @ D
            assert Phi[m, j] == pytest.approx(abs(mean[n]) ** 2 + cov[n, n], rel=1e-12)


def em_aux(Phi, Ln, Hn):
    """EM auxiliary (negative expected complete log-likelihood) of source n's component:
    sum_{m,j} ln(L_mn H_nj) + Phi_mj / (L_mn H_nj)."""
    S = np.outer(Ln, Hn)
    return np.sum(np.log(S) + Phi / S)


def test_nmf_em_updates_are_coordinate_minimisers(rng):
    """The L[:, n] and H[n, :] updates of Algorithm 1 minimise the EM auxiliary in their own
    block with the other fixed: every +-eps perturbation raises it (brute force)."""
    M, N, J = 2, 3, 5
    _, _, L, H = small_problem(rng, M, N, J)
    U = np.abs(rand_complex(rng, M, J)) ** 2 + 0.1
    for n in range(N):
        S = np.outer(L[:, n], H[n, :])
        G = S / (L @ H)
        Phi = G ** 2 * U + (1 - G) * S
        L2, H2 = ff.nmf_em_step(U, L, H, n)
        base = em_aux(Phi, L2[:, n], H[n, :])          # L step uses the old H[n, :]
        for m in range(M):
            for eps in (1e-4, -1e-4):
                Lp = L2[:, n].copy()
                Lp[m] *= 1 + eps
                assert em_aux(Phi, Lp, H[n, :]) > base
        base = em_aux(Phi, L2[:, n], H2[n, :])         # H step uses the new L[:, n]
        for j in range(J):
            for eps in (1e-4, -1e-4):
                Hp = H2[n, :].copy()
                Hp[j] *= 1 + eps
                assert em_aux(Phi, L2[:, n], Hp) > base
        L, H = L2, H2


def test_each_nmf_step_does_not_decrease_loglik(rng):
    """Sec. IV-E: the EM updates of L and H never decrease the likelihood (checked per n)."""
    x, W, L, H = small_problem(rng, 3, 5, J=30)
    Xh = ff.Xhat_from_x(x)
    U = ff.decorrelated_power(Xh, W)
    ll = ff.loglik(Xh, W, L, H)
    for _ in range(4):
        for n in range(5):
            L, H = ff.nmf_em_step(U, L, H, n)
            ll_new = ff.loglik(Xh, W, L, H)
            assert ll_new >= ll - 1e-9 * abs(ll)
            ll = ll_new


def test_iterate_monotone_on_generated_mixture():
    """Algorithm 1 on a model-generated mixture: log-likelihood non-decreasing every iteration."""
    from paper_2101_08563_gb300 import synth
    mix = synth.generate_mixture(2, 3, 6, 40, 4, seed=7)
    p = synth.random_init(mix.x, 3, seed=7)
    out = ff.run(mix.x, p.P, p.lam, p.v, iters=25)
    d = np.diff(out["ll"], axis=1)
    assert np.all(d >= -1e-9 * np.abs(out["ll"][:, 1:]))


def test_decorrelated_power_is_abs_y_squared(rng):
    """Eq. 37 equals |y_mj|^2 with y_j = W^H x_j (Eq. 22)."""
    x, W, L, H = small_problem(rng, 3, 4, J=5)
    y = x @ W.conj()
    assert np.allclose(ff.decorrelated_power(ff.Xhat_from_x(x), W), (np.abs(y) ** 2).T, atol=1e-12)


# ----------------------------------------------------------------------------- MWF (Eq. 39)
def test_mwf_equals_fca_mwf_under_jd(rng):
    """Eq. 39 is Eq. 7 with R_n from Eq. 19: both oracles give the same filter and images."""
    x, W, L, H = small_problem(rng, 3, 5, J=4)
    R = jd_covariances(W, L)
    for n in range(5):
        for j in range(4):
            assert np.allclose(ff.mwf(W, L, H, n, j), fca.mwf(R, H, n, j), atol=1e-11)
    assert np.allclose(ff.separate(x, W, L, H), fca.separate(x, R, H), atol=1e-11)
    assert np.allclose(ff.separate_fast(x, W, L, H), ff.separate(x, W, L, H), atol=1e-12)


def test_images_sum_to_mixture(rng):
    """Eq. 2: the Wiener gains sum to one over n, so the separated images add up to x."""
    x, W, L, H = small_problem(rng, 3, 5, J=6)
    c = ff.separate(x, W, L, H)
    assert np.allclose(c.sum(axis=1), x, atol=1e-12)


def test_mwf_is_least_squares_regression():
    """Sec. III-B: the MWF is the LMMSE estimator.  A least-squares regression (numpy lstsq)
    of sampled source images on sampled mixtures recovers F_jn = h_jn R_n X_j^{-1}."""
    rng = np.random.Generator(np.random.PCG64(99))
    M, N, S = 2, 3, 200000
    R = np.array([rand_hpd(rng, M) for _ in range(N)])
    h = rng.uniform(0.5, 2.0, size=(N, 1))
    c = np.stack([rand_complex(rng, S, M) @ np.linalg.cholesky(h[n, 0] * R[n]).T for n in range(N)])
    xs = c.sum(axis=0)
    for n in range(N):
        Ft, *_ = np.linalg.lstsq(xs, c[n], rcond=None)     # c ~ x F^T
        assert np.allclose(Ft.T, fca.mwf(R, h, n, 0), atol=2e-2)


def test_mwf_ica_special_case_is_selector(rng):
    """Sec. V-C (Eq. 40): with N = M and Lambda_n = e_n e_n^T the MWF reduces to
    W^{-H} e_n e_n^T W^H, i.e. separation then projection back of the n-th output."""
    M = 3
    x = rand_complex(rng, 5, M)
    W = rand_complex(rng, M, M) + 2 * np.eye(M)
    L = np.eye(M)
    H = rng.uniform(0.3, 2.0, size=(M, 5))
    c = ff.separate(x, W, L, H)
    Wi = np.linalg.inv(W.conj().T)
    for j in range(5):
        y = W.conj().T @ x[j]
        for n in range(M):
            assert np.allclose(c[j, n], Wi[:, n] * y[n], atol=1e-12)


def test_fastfca_posterior_equals_fca_posterior(rng):
    """With R_n = W^{-H} Lambda_n W^{-1}, FCA's posterior statistics (Eq. 12, explicit
    inverse) seen through W^H are FastFCA's: W^H mu_jn = G_n y_j and
    diag(W^H Psi_jn W) = Phi_n[:, j] of Algorithm 1."""
    M, N, J = 2, 3, 4
    x, W, L, H = small_problem(rng, M, N, J)
    R = jd_covariances(W, L)
    U = ff.decorrelated_power(ff.Xhat_from_x(x), W)
    y = x @ W.conj()
    for n in range(N):
        S = np.outer(L[:, n], H[n, :])
        G = S / (L @ H)
        Phi = G ** 2 * U + (1 - G) * S
        for j in range(J):
            mu = fca.mwf(R, H, n, j) @ x[j]
            assert np.allclose(W.conj().T @ mu, G[:, j] * y[j], atol=1e-11)
            P = W.conj().T @ fca.psi(x[j], R, H, n, j) @ W
            assert np.allclose(np.real(np.diag(P)), Phi[:, j], rtol=1e-10, atol=1e-12)
            # the posterior covariance part (Psi minus mu mu^H) is diagonal after W^H . W
            mu_y = W.conj().T @ mu
            C = P - np.outer(mu_y, mu_y.conj())
            assert np.allclose(C - np.diag(np.diag(C)), 0.0, atol=1e-10)


def test_golden_trajectory_regression():
    """The oracle reproduces its committed trajectory (written by tests/golden/make_golden.py
    from the oracle alone); guards against unintended changes of the oracle's arithmetic."""
    g = json.load(open(os.path.join(GOLDEN, "oracle_trajectory_m2n3.json")))
    from paper_2101_08563_gb300 import synth
    mix = synth.generate_mixture(g["M"], g["N"], g["F"], g["T"], g["K"], seed=g["seed"])
    p = synth.random_init(mix.x, g["N"], seed=g["seed"])
    out = ff.run(mix.x, p.P, p.lam, p.v, iters=g["iters"])
    assert np.allclose(out["ll"], np.array(g["ll"]), rtol=1e-12, atol=1e-9)


# ---------------------------------------------------------------------------- Algorithm 2 (IP+MM)
def _is_cost(U, L, H):
    S = L @ H
    return float(np.sum(U / S + np.log(S)))


def test_mm_update_minimises_the_written_out_majoriser(rng):
    """The L and H lines of Algorithm 2 are the exact minimisers of the IS-NMF auxiliary
    function: Jensen's bound on U/sigma^2 with weights lam_n = L~ H~_n / sigma~^2 and the
    tangent bound on ln sigma^2.  Each entry's 1-D majoriser is minimised numerically here."""
    from scipy.optimize import minimize_scalar
    M, N, J = 2, 3, 7
    U = rng.uniform(0.2, 3.0, (M, J))
    L0 = rng.uniform(0.3, 2.0, (M, N))
    H0 = rng.uniform(0.3, 2.0, (N, J))
    L1, H1 = ff.nmf_mm_step(U, L0, H0)
    S0 = L0 @ H0
    for m in range(M):
        for n in range(N):
            lam = L0[m, n] * H0[n] / S0[m]
            f = lambda l: np.sum(lam ** 2 * U[m] / (l * H0[n]) + l * H0[n] / S0[m])
            best = minimize_scalar(f, bounds=(1e-6, 100.0), method="bounded", options={"xatol": 1e-12})
            assert abs(best.x - L1[m, n]) <= 1e-6 * L1[m, n]
    S1 = L1 @ H0                               # H uses sigma^2 from the new L
    for n in range(N):
        for j in range(J):
            lam = L1[:, n] * H0[n, j] / S1[:, j]
            f = lambda h: np.sum(lam ** 2 * U[:, j] / (L1[:, n] * h) + L1[:, n] * h / S1[:, j])
            best = minimize_scalar(f, bounds=(1e-6, 100.0), method="bounded", options={"xatol": 1e-12})
            assert abs(best.x - H1[n, j]) <= 1e-6 * H1[n, j]


def test_mm_step_never_increases_the_is_cost(rng):
    for _ in range(20):
        M, N, J = int(rng.integers(2, 5)), int(rng.integers(1, 6)), int(rng.integers(3, 30))
        U = rng.uniform(0.01, 5.0, (M, J))
        L = rng.uniform(0.05, 3.0, (M, N))
        H = rng.uniform(0.05, 3.0, (N, J))
        c0 = _is_cost(U, L, H)
        L1, H1 = ff.nmf_mm_step(U, L, H)
        assert _is_cost(U, L1, H1) <= c0 + 1e-12 * abs(c0)


def test_mm_fixed_points_are_stationary_points_of_the_is_cost(rng):
    """Run the MM updates to convergence (W = I is IS-NMF, footnote of Sec. IV-E); the
    finite-difference gradient of the IS cost then vanishes at the limit."""
    M, N, J = 2, 2, 6
    U = rng.uniform(0.2, 3.0, (M, J))
    L = rng.uniform(0.5, 1.5, (M, N))
    H = rng.uniform(0.5, 1.5, (N, J))
    for _ in range(20000):
        L, H = ff.nmf_mm_step(U, L, H)
    eps = 1e-6
    for A in (L, H):
        for idx in np.ndindex(A.shape):
            old = A[idx]
            A[idx] = old * (1 + eps)
            cp = _is_cost(U, L, H)
            A[idx] = old * (1 - eps)
            cm = _is_cost(U, L, H)
            A[idx] = old
            # d cost / d ln A  (scale-free): zero at a stationary point
            assert abs(cp - cm) / (2 * eps) <= 1e-6 * abs(_is_cost(U, L, H))


def test_ip_mm_log_likelihood_is_monotone():
    mix = synth.generate_mixture(3, 4, 3, 150, 4, seed=33)
    init = synth.random_init(mix.x, 4, seed=33)
    ref = ff.run(mix.x, init.P, init.lam, init.v, iters=25, algorithm="mm")
    for f in range(3):
        ll = ref["ll"][f]
        assert np.all(np.diff(ll) >= -1e-9 * np.abs(ll[1:]))


def test_block_separation_equals_the_frame_filter_with_repeated_powers(rng):
    """Sec. VI-B: frames of one block share their covariances, so the block filter of every
    frame is the frame-wise Eq. 39 filter with that block's powers (checked per frame with the
    explicit FCA filter of Eq. 7 under Eq. 19)."""
    M, N, B, J = 3, 4, 5, 4
    x = rand_complex(rng, B * J, M)
    W = rand_complex(rng, M, M) + 2 * np.eye(M)
    L = rng.uniform(0.3, 2.0, (M, N))
    H = rng.uniform(0.3, 2.0, (N, J))
    c = ff.separate_blocks(x, W, L, H, B)
    Wi = np.linalg.inv(W)
    for t in range(B * J):
        j = t // B
        Rs = [Wi.conj().T @ np.diag(L[:, n] * H[n, j]) @ Wi for n in range(N)]
        X = sum(Rs)
        for n in range(N):
            assert np.allclose(c[t, n], Rs[n] @ np.linalg.solve(X, x[t]), atol=1e-10)
