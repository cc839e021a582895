"""Pins of the FastMNMF oracle (App. C, Eq. 52-53) against what the model and the
mathematics fix, independently of the oracle's own index expressions."""
import numpy as np
import pytest
from scipy import stats

from oracle import fastmnmf as mn


@pytest.fixture
def rng():
    return np.random.Generator(np.random.PCG64(7))


def problem(rng, I=3, J=7, M=2, N=2, K=2):
    x = (rng.standard_normal((I, J, M)) + 1j * rng.standard_normal((I, J, M))) * np.sqrt(0.5)
    W = np.eye(M)[None] + 0.3 * (rng.standard_normal((I, M, M)) + 1j * rng.standard_normal((I, M, M)))
    lam = rng.uniform(0.3, 2.0, (I, M, N))
    t = rng.uniform(0.3, 2.0, (I, K, N))
    v = rng.uniform(0.3, 2.0, (J, K, N))
    return x, W, lam, t, v


def neg_cost(x, W, lam, t, v):
    """Eq. 53 without its constant (the negative log-likelihood up to I M J ln(pi))."""
    return -mn.loglik(x, W, lam, t, v)


def test_loglik_is_the_complex_gaussian_density(rng):
    """Eq. 53: x_ij ~ CN(0, W_i^{-H} diag(sigma^2_ij) W_i^{-1}) (Eq. 19, 28, 52), evaluated by
    scipy on the real 2M-dimensional form."""
    x, W, lam, t, v = problem(rng)
    I, J, M = x.shape
    N, K = lam.shape[2], t.shape[1]
    ref = 0.0
    for i in range(I):
        Wi_inv = np.linalg.inv(W[i])
        for j in range(J):
            s2 = np.array([sum(lam[i, m, n] * sum(t[i, k, n] * v[j, k, n] for k in range(K))
                               for n in range(N)) for m in range(M)])
            S = Wi_inv.conj().T @ np.diag(s2) @ Wi_inv
            C = 0.5 * np.block([[S.real, -S.imag], [S.imag, S.real]])
            z = np.concatenate([x[i, j].real, x[i, j].imag])
            ref += stats.multivariate_normal(mean=np.zeros(2 * M), cov=C).logpdf(z)
    assert np.isclose(mn.loglik(x, W, lam, t, v), ref, rtol=1e-11)


def _coefficients(sig_fn, theta):
    """a[l, p] = d sigma^2_p / d theta_l, found by probing the (linear) map with unit
    vectors: independent of how the update writes its index sums."""
    flat = theta.ravel()
    a = np.empty((flat.size, sig_fn(theta).size))
    for l in range(flat.size):
        e = np.zeros_like(flat)
        e[l] = 1.0
        a[l] = sig_fn(e.reshape(theta.shape)).ravel()
    return a


def _aux(theta_flat, theta0_flat, a, U):
    """Auxiliary function of the IS divergence sum_p U_p/s_p + ln s_p for s = a^T theta,
    touching it at theta0: Jensen on 1/s (weights phi_lp = theta0_l a_lp / s0_p) and the
    tangent of ln s at s0."""
    s0 = a.T @ theta0_flat
    phi = theta0_flat[:, None] * a / s0[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        jensen = np.where(a > 0, phi ** 2 * U[None, :] / (theta_flat[:, None] * a), 0.0).sum(axis=0)
    s = a.T @ theta_flat
    return float(np.sum(jensen + np.log(s0) + (s - s0) / s0))


FACTORS = ["lam", "t", "v"]


def _factor_setup(name, x, W, lam, t, v):
    U = mn.decorrelated_power(x, W)
    if name == "lam":
        sig = lambda th: mn.sigma2(th, mn.h_of(t, v))
        return U, lam, sig, mn.mm_lam(U, lam, t, v)
    if name == "t":
        sig = lambda th: mn.sigma2(lam, mn.h_of(th, v))
        return U, t, sig, mn.mm_t(U, lam, t, v)
    sig = lambda th: mn.sigma2(lam, mn.h_of(t, th))
    return U, v, sig, mn.mm_v(U, lam, t, v)


@pytest.mark.parametrize("name", FACTORS)
def test_mm_update_minimises_the_auxiliary_function(rng, name):
    """Each MM update is the exact minimiser of the IS auxiliary function in its factor: the
    auxiliary touches the cost at the current point, lies above it, and no coordinate move
    away from the update lowers it."""
    x, W, lam, t, v = problem(rng)
    U, theta0, sig, theta1 = _factor_setup(name, x, W, lam, t, v)
    a = _coefficients(sig, theta0)
    Uf = U.ravel()
    th0 = theta0.ravel()
    th1 = theta1.ravel()

    def cost(th):
        s = a.T @ th
        return float(np.sum(Uf / s + np.log(s)))

    assert np.isclose(_aux(th0, th0, a, Uf), cost(th0), rtol=1e-12)
    assert _aux(th1, th0, a, Uf) >= cost(th1) - 1e-9
    g1 = _aux(th1, th0, a, Uf)
    for l in range(th1.size):
        for eps in (1e-3, -1e-3):
            th = th1.copy()
            th[l] *= 1.0 + eps
            assert _aux(th, th0, a, Uf) >= g1 - 1e-12, (name, l, eps)


@pytest.mark.parametrize("name", FACTORS)
def test_mm_ratio_matches_the_cost_gradient(rng, name):
    """(theta_new / theta)^2 = num/den, and the cost gradient is den - num: finite
    differences of Eq. 53 give d cost / d theta_l = den_l (1 - (theta_new_l / theta_l)^2)
    with den_l = sum_p a_lp / sigma^2_p."""
    x, W, lam, t, v = problem(rng)
    U, theta0, sig, theta1 = _factor_setup(name, x, W, lam, t, v)
    a = _coefficients(sig, theta0)
    s0 = a.T @ theta0.ravel()
    den = a @ (1.0 / s0)
    ratio2 = (theta1.ravel() / theta0.ravel()) ** 2

    def c(th):
        args = {"lam": lam, "t": t, "v": v}
        args[name] = th
        return neg_cost(x, W, args["lam"], args["t"], args["v"])

    h = 1e-6
    for l in range(theta0.size):
        e = np.zeros(theta0.size)
        e[l] = h
        g = (c(theta0 + e.reshape(theta0.shape)) - c(theta0 - e.reshape(theta0.shape))) / (2 * h)
        assert np.isclose(g, den[l] * (1.0 - ratio2[l]), rtol=1e-5, atol=1e-7), (name, l)


def test_each_update_does_not_increase_the_cost(rng):
    x, W, lam, t, v = problem(rng, I=4, J=9, M=3, N=3, K=2)
    for _ in range(4):
        c0 = neg_cost(x, W, lam, t, v)
        W = mn.ip_all(x, W, lam, t, v)
        c1 = neg_cost(x, W, lam, t, v)
        U = mn.decorrelated_power(x, W)
        lam = mn.mm_lam(U, lam, t, v)
        c2 = neg_cost(x, W, lam, t, v)
        t = mn.mm_t(U, lam, t, v)
        c3 = neg_cost(x, W, lam, t, v)
        v = mn.mm_v(U, lam, t, v)
        c4 = neg_cost(x, W, lam, t, v)
        for a_, b_ in ((c0, c1), (c1, c2), (c2, c3), (c3, c4)):
            assert b_ <= a_ + 1e-9 * abs(a_)


def test_rescaling_bases_and_activations_leaves_the_trajectory_unchanged(rng):
    """h = T V is invariant under t -> c t, v -> v / c per (k, n), and so is every update of
    h, W and lambda (the MM rules are scale-equivariant)."""
    x, W, lam, t, v = problem(rng, K=3)
    c = rng.uniform(0.2, 5.0, (1, t.shape[1], t.shape[2]))
    r1 = mn.run(x, W, lam, t, v, iters=3)
    r2 = mn.run(x, W, lam, t * c, v / c, iters=3)
    assert np.allclose(r1["ll"], r2["ll"], rtol=1e-11)
    assert np.allclose(mn.h_of(r1["t"], r1["v"]), mn.h_of(r2["t"], r2["v"]), rtol=1e-9)
    assert np.allclose(r1["W"], r2["W"], rtol=1e-9, atol=1e-12)


def test_images_sum_to_the_mixture(rng):
    x, W, lam, t, v = problem(rng, M=3, N=4, K=2)
    c = mn.separate(x, W, lam, t, v)
    assert np.allclose(c.sum(axis=2), x, atol=1e-11)


def test_one_frequency_one_basis_reduces_to_algorithm_2(rng):
    """With I = 1 and K = 1, h_jn = t_n v_jn and the lambda update is Algorithm 2's L line
    with H = h^T; the v update is Algorithm 2's H line with L = lambda diag(t)."""
    from oracle import fastfca as off
    x, W, lam, t, v = problem(rng, I=1, J=8, M=2, N=3, K=1)
    U = mn.decorrelated_power(x, W)
    H = (t[0, 0][:, None] * v[:, 0, :].T)                        # (N, J)
    L_alg2, _ = off.nmf_mm_step(U[0], lam[0], H)
    assert np.allclose(mn.mm_lam(U, lam, t, v)[0], L_alg2, rtol=1e-12)
    # H line of Algorithm 2 with L' = lambda diag(t) and H' = v^T
    Lp = lam[0] * t[0, 0][None, :]
    S = Lp @ v[:, 0, :].T
    v_alg2 = v[:, 0, :].T * np.sqrt((Lp.T @ (U[0] * S ** -2)) / (Lp.T @ (S ** -1)))
    assert np.allclose(mn.mm_v(U, lam, t, v)[:, 0, :].T, v_alg2, rtol=1e-12)


def test_iterations_never_decrease_the_loglik_on_a_generated_mixture():
    from paper_2101_08563_gb300 import synth
    mix = synth.generate_mixture(3, 3, 6, 40, 2, seed=31)
    st = synth.fastmnmf_random_init(mix.x, 3, 2, seed=31)
    r = mn.run(mix.x, st.W, st.lam, st.t, st.v, iters=8)
    assert np.all(np.diff(r["ll"]) >= -1e-9 * np.abs(r["ll"][1:]))


def test_images_are_the_gaussian_posterior_mean(rng):
    """Eq. 39 under Eq. 52: c_ijn = C_ijn (sum_n' C_ijn')^{-1} x_ij with the source image
    covariance C_ijn = h_ijn W_i^{-H} diag(lambda_i[:, n]) W_i^{-1}, built here per bin from
    explicit loops over k."""
    x, W, lam, t, v = problem(rng, I=2, J=5, M=3, N=3, K=2)
    I, J, M = x.shape
    N, K = lam.shape[2], t.shape[1]
    c = mn.separate(x, W, lam, t, v)
    for i in range(I):
        A = np.linalg.inv(W[i])
        for j in range(J):
            C = []
            for n in range(N):
                h = 0.0
                for k in range(K):
                    h += t[i, k, n] * v[j, k, n]
                C.append(h * A.conj().T @ np.diag(lam[i, :, n]) @ A)
            X = sum(C)
            for n in range(N):
                assert np.allclose(c[i, j, n], C[n] @ np.linalg.solve(X, x[i, j]), atol=1e-10)


def test_iteration_strictly_lowers_the_cost_and_composes_the_pinned_steps(rng):
    """One iteration is the IP sweep, then U of the new W (Eq. 37), then the three MM
    updates; from a start far from the IP optimum it lowers the cost by more than the IP step
    alone."""
    x, W, lam, t, v = problem(rng, I=3, J=12, M=3, N=2, K=2)
    W = W * rng.uniform(0.2, 3.0, (3, 1, 3))
    W1, lam1, t1, v1 = mn.iterate(x, W, lam, t, v)
    Wa = mn.ip_all(x, W, lam, t, v)
    U = mn.decorrelated_power(x, Wa)
    la = mn.mm_lam(U, lam, t, v)
    ta = mn.mm_t(U, la, t, v)
    va = mn.mm_v(U, la, ta, v)
    for p, q in ((W1, Wa), (lam1, la), (t1, ta), (v1, va)):
        assert np.allclose(p, q, rtol=1e-13, atol=1e-15)
    c0 = neg_cost(x, W, lam, t, v)
    cip = neg_cost(x, Wa, lam, t, v)
    c1 = neg_cost(x, W1, lam1, t1, v1)
    assert cip < c0 and c1 < cip
