"""Pins of the FP64 reference of the learned initialiser (features, conv, loss gradients)."""
import numpy as np

from oracle import learned as ol
from tests.conftest import rand_complex


def small_params(rng, M, N, hidden=ol.HIDDEN, scale=0.05):
    D = ol.out_dim(M, N)
    return {"W1": rng.standard_normal((hidden, ol.D_IN)) * scale, "b1": rng.standard_normal(hidden) * scale,
            "W2": rng.standard_normal((hidden, hidden)) * scale, "b2": rng.standard_normal(hidden) * scale,
            "W3": rng.standard_normal((D, hidden)) * scale, "b3": rng.standard_normal(D) * scale}


def test_features_match_direct_definitions(rng):
    x = rand_complex(rng, 40, 3)
    phi, q = ol.features(x, 5, 11)
    R = sum(np.outer(x[t], x[t].conj()) for t in range(40)) / 40
    tr = np.trace(R).real
    assert np.allclose(phi[:3], np.diag(R).real / tr)
    assert np.isclose(phi[3], (R[0, 1] / tr).real) and np.isclose(phi[4], (R[0, 1] / tr).imag)
    p = np.log(np.sum(np.abs(x) ** 2, axis=1) / 3)
    assert np.isclose(phi[9], np.log(tr / 3)) and np.isclose(phi[10], p.mean()) and np.isclose(phi[11], p.std())
    assert np.isclose(phi[12], 0.5) and phi[13] == 1.0
    assert np.allclose(q, p - p.mean())


def test_conv_is_numpy_convolution(rng):
    kw = rng.standard_normal((4, 9))
    q = rng.standard_normal(30)
    out = ol.conv_logv(kw, np.zeros(4), np.zeros(4), q)
    for n in range(4):
        # correlation with zero padding = convolution with the reversed kernel, 'same' size
        assert np.allclose(out[n], np.convolve(q, kw[n][::-1], mode="same"))


def test_gelu_gradient_by_finite_differences():
    z = np.linspace(-4, 4, 41)
    h = 1e-6
    fd = (ol.gelu(z + h) - ol.gelu(z - h)) / (2 * h)
    assert np.allclose(ol.gelu_grad(z), fd, atol=1e-7)


def test_batch_gradients_by_finite_differences():
    rng = np.random.Generator(np.random.PCG64(5))
    M, N, T, S = 3, 4, 20, 3
    params = small_params(rng, M, N, hidden=16, scale=0.3)
    conv = {"k": rng.standard_normal((N, 9)) * 0.1, "c": rng.standard_normal(N) * 0.1}
    phis = rng.standard_normal((S, ol.D_IN))
    qs = rng.standard_normal((S, T))
    targets = []
    for s in range(S):
        W = rand_complex(rng, M, M) + np.eye(M)
        L = rng.uniform(0.3, 2.0, (M, N))
        H = rng.uniform(0.3, 2.0, (N, T))
        targets.append(ol.canon_target(W, L, H))
    loss, g, _ = ol.batch_loss_and_grads(params, conv, phis, qs, targets, M, N)
    eps = 1e-6
    for name, store in [("W1", params), ("b2", params), ("W3", params), ("b3", params), ("k", conv), ("c", conv)]:
        arr = store[name]
        flat = arr.reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _, _ = ol.batch_loss_and_grads(params, conv, phis, qs, targets, M, N)
            flat[idx] = old - eps
            lm, _, _ = ol.batch_loss_and_grads(params, conv, phis, qs, targets, M, N)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[name].reshape(-1)[idx]) <= 1e-5 + 1e-4 * abs(fd), (name, idx, fd, g[name].reshape(-1)[idx])


def test_canonical_target_keeps_the_model_covariances(rng):
    # W^{-H} diag(L h_t) W^{-1} must be the same for (W, L, H) and the scale-free target
    M, N, T = 3, 4, 7
    W = rand_complex(rng, M, M) + 2 * np.eye(M)
    L = rng.uniform(0.2, 3.0, (M, N))
    H = rng.uniform(0.2, 3.0, (N, T))
    Wn, lt, ht = ol.canon_target(W, L, H)
    assert np.allclose(np.linalg.norm(Wn, axis=0), 1.0)
    assert np.allclose(lt.mean(axis=0), 0.0)

    def covs(W_, L_, H_):
        Wi = np.linalg.inv(W_)
        return [Wi.conj().T @ np.diag(L_ @ H_[:, t]) @ Wi for t in range(T)]

    for a, b in zip(covs(W, L, H), covs(Wn, np.exp(lt), np.exp(ht))):
        assert np.allclose(a, b, rtol=1e-12, atol=1e-12)
    # a column rescaling of W or a per-source rescaling of (L, H) leaves the target unchanged
    d = rng.uniform(0.5, 2.0, M) * np.exp(1j * rng.uniform(0, 6.28, M))
    s = rng.uniform(0.5, 2.0, N)
    Wn2, lt2, ht2 = ol.canon_target(W * d[None, :], L * np.abs(d)[:, None] ** 2 * s[None, :], H / s[:, None])
    assert np.allclose(np.abs(np.sum(Wn2.conj() * Wn, axis=0)), 1.0)
    assert np.allclose(lt2, lt) and np.allclose(ht2, ht)
