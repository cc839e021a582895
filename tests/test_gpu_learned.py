"""The learned initialiser on the GPU against the FP64 reference (oracle/learned.py).

Products run on BF16 tensor cores with FP32 accumulation, so the comparison with the FP64
reference uses tolerances derived from BF16 rounding (unit roundoff 2^-8 per operand: about
1e-2 of an output's rms after three layers).  Parts computed in FP32 only (features, targets,
the head given the network output, the bias-gradient sums) are compared tightly, and the
forward pass is also compared tightly with the same products on BF16-rounded operands.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import learned as ol  # noqa: E402
from tests.conftest import rand_complex  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2101_08563_gb300 import build, fastfca
    build.build()
    fastfca.load()
    from paper_2101_08563_gb300 import learned
    return learned


def oracle_params(L, flat, M, N):
    p = {k: np.asarray(v, dtype=np.float64) for k, v in L.unpack(flat, M, N).items()}
    D = ol.out_dim(M, N)
    mlp = {"W1": p["W1"], "b1": p["b1"], "W2": p["W2"], "b2": p["b2"], "W3": p["W3"][:D], "b3": p["b3"][:D]}
    return mlp, {"k": p["k"], "c": p["c"]}


def bf16(a):
    """Round float32 values to BF16 (nearest, ties to even), returned as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def random_net(L, M, N, rows, T, seed):
    net = L.InitNet(M, N, max_rows=rows, max_T=T, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed))
    flat = net.get_params()
    blocks = L.unpack(flat, M, N)
    # give every block visible values (the default last layer is 100x smaller)
    blocks["W3"][:] = rng.uniform(-1, 1, blocks["W3"].shape) * np.sqrt(3.0 / L.HIDDEN)
    blocks["b1"][:] = rng.uniform(-0.2, 0.2, blocks["b1"].shape)
    blocks["b2"][:] = rng.uniform(-0.2, 0.2, blocks["b2"].shape)
    blocks["b3"][:] = rng.uniform(-0.5, 0.5, blocks["b3"].shape)
    blocks["c"][:] = rng.uniform(-0.5, 0.5, blocks["c"].shape)
    net.set_params(flat)
    return net, flat


def random_inputs(rng, rows, T):
    feats = rng.standard_normal((rows, ol.D_IN)).astype(np.float32)
    feats[:, -2:] = 0.0
    q = rng.standard_normal((rows, T)).astype(np.float32)
    return feats, q


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ---------------------------------------------------------------------------- generator
def test_generator_is_seeded_and_has_model_power(L):
    a = L.generate_mixtures(16, 65, 200, 3, 5, 4, 0.03, seed=5)
    b = L.generate_mixtures(16, 65, 200, 3, 5, 4, 0.03, seed=5)
    c = L.generate_mixtures(16, 65, 200, 3, 5, 4, 0.03, seed=6)
    assert torch.equal(a, b) and not torch.equal(a, c)
    assert torch.isfinite(torch.view_as_real(a)).all()
    # E|x_m|^2 = sum_n E[v_n] R_n[m, m] = N K (1 + 0.01)
    pw = (a.abs() ** 2).mean(dim=(0, 1, 2)).cpu().numpy()
    assert np.allclose(pw, 5 * 4 * 1.01, rtol=0.06), pw


def test_generator_steering_geometry(L):
    # one source: per-frequency correlation of two mics is a_0 conj(a_1) / 1.01 in magnitude,
    # with phase 2 pi nu_f d cos(theta) / c growing linearly in f (d small: no wrap)
    F, T = 17, 4000
    x = L.generate_mixtures(3, F, T, 2, 1, 4, 0.01, seed=9).cpu().numpy().astype(np.complex128)
    for b in range(3):
        R01 = (x[b, :, :, 0] * x[b, :, :, 1].conj()).mean(axis=1)
        R00 = (np.abs(x[b, :, :, 0]) ** 2).mean(axis=1)
        R11 = (np.abs(x[b, :, :, 1]) ** 2).mean(axis=1)
        rho = np.abs(R01) / np.sqrt(R00 * R11)
        assert np.all(rho > 0.97) and np.all(rho < 1.0 + 1e-6)
        ph = np.angle(R01)
        slope = ph[F - 1] / (F - 1)
        assert abs(slope) <= 2 * np.pi * 8000 * 0.01 / 343 / (F - 1) * 1.05
        assert np.allclose(ph, slope * np.arange(F), atol=0.05)


# ---------------------------------------------------------------------------- features, targets
def test_features_match_oracle(L):
    F, T, M = 7, 203, 3
    x = L.generate_mixtures(2, F, T, M, 5, 4, 0.03, seed=11).view(2 * F, T, M)
    feats, q = L.features(x, F)
    feats, q = feats.cpu().numpy(), q.cpu().numpy()
    xh = x.cpu().numpy().astype(np.complex128)
    for r in range(2 * F):
        phi, qo = ol.features(xh[r], r % F, F)
        assert np.allclose(feats[r], phi, rtol=1e-4, atol=1e-4), (r, feats[r], phi)
        assert np.allclose(q[r], qo, atol=1e-4)


def test_features_m2(L):
    F, T, M = 5, 64, 2
    x = L.generate_mixtures(1, F, T, M, 3, 4, 0.04, seed=3).view(F, T, M)
    feats, q = L.features(x, F)
    xh = x.cpu().numpy().astype(np.complex128)
    for r in range(F):
        phi, qo = ol.features(xh[r], r, F)
        assert np.allclose(feats[r].cpu().numpy(), phi, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("M,N,T", [(3, 5, 41), (2, 3, 9)])
def test_targets_match_oracle(L, M, N, T, rng):
    rows = 13
    P = rand_complex(rng, rows, M, M) + 2.0 * np.eye(M)[None]
    lam = rng.uniform(0.05, 4.0, (rows, M, N)).astype(np.float32)
    v = rng.uniform(0.05, 4.0, (rows, N, T)).astype(np.float32)
    wt, lt, ht = L.targets(cuda(P), cuda(lam), cuda(v))
    wt, lt, ht = wt.cpu().numpy(), lt.cpu().numpy(), ht.cpu().numpy()
    for r in range(rows):
        Wn, l, h = ol.canon_target(P[r], lam[r].astype(np.float64), v[r].astype(np.float64))
        assert np.allclose(wt[r][..., 0] + 1j * wt[r][..., 1], Wn, atol=1e-6)
        assert np.allclose(lt[r], l, atol=1e-5)
        assert np.allclose(ht[r], h, atol=1e-5)


# ---------------------------------------------------------------------------- network
@pytest.mark.parametrize("M,N,rows", [(3, 5, 150), (2, 3, 37)])
def test_forward_matches_oracle(L, M, N, rows):
    rng = np.random.Generator(np.random.PCG64(rows))
    net, flat = random_net(L, M, N, rows, 16, seed=rows)
    feats, _ = random_inputs(rng, rows, 16)
    o = net.forward(cuda(feats)).astype(np.float64)
    D = ol.out_dim(M, N)
    mlp, _ = oracle_params(L, flat, M, N)
    ref, _ = ol.forward(mlp, feats.astype(np.float64))
    rms = np.sqrt((ref ** 2).mean())
    assert np.abs(o[:, :D] - ref).max() <= 3e-2 * rms
    # the same products on BF16-rounded operands, FP64 accumulation: FP32-accumulation close
    z1 = bf16(feats) @ bf16(mlp["W1"]).T + mlp["b1"]
    z2 = bf16(ol.gelu(z1)) @ bf16(mlp["W2"]).T + mlp["b2"]
    o3 = bf16(ol.gelu(z2)) @ bf16(L.unpack(flat, M, N)["W3"]).T + L.unpack(flat, M, N)["b3"]
    assert np.abs(o - o3).max() <= 2e-3 * rms
    # padding columns (unused outputs) follow the same products
    assert np.allclose(o[:, D:], o3[:, D:], atol=2e-3 * rms)


def clear_targets(L, rng, net, flat, feats, q, M, N, noise=0.2):
    """Targets built from the reference prediction with a known permutation plus noise, so
    that the optimal permutations are clear-cut (no near-ties between FP32 and FP64)."""
    mlp, conv = oracle_params(L, flat, M, N)
    rows, T = q.shape
    o, _ = ol.forward(mlp, feats.astype(np.float64))
    base = 2 * M * M
    wt = np.empty((rows, M, M, 2), np.float32)
    lt = np.empty((rows, M, N), np.float32)
    ht = np.empty((rows, N, T), np.float32)
    for r in range(rows):
        W = (o[r, 0:base:2] + 1j * o[r, 1:base:2]).reshape(M, M)
        lnL = o[r, base: base + M * N].reshape(M, N)
        lnv = ol.conv_logv(conv["k"], conv["c"], o[r, base + M * N: base + M * N + N], q[r].astype(np.float64))
        sig = rng.permutation(M)
        pi = rng.permutation(N)
        d = rng.uniform(0.5, 2.0, M) * np.exp(1j * rng.uniform(0, 6.28, M))
        s = rng.uniform(0.5, 2.0, N)
        Wt = W[:, sig] * d[None, :] + noise * 0.2 * rand_complex(rng, M, M)
        Lt = np.exp(lnL[np.ix_(sig, pi)] + noise * rng.standard_normal((M, N))) * s[None, :]
        Ht = np.exp(lnv[pi] + noise * rng.standard_normal((N, T))) / s[:, None]
        Wn, l, h = ol.canon_target(Wt, Lt, Ht)
        wt[r, ..., 0], wt[r, ..., 1] = Wn.real, Wn.imag
        lt[r], ht[r] = l, h
    return wt, lt, ht


@pytest.mark.parametrize("M,N,rows,T", [(3, 5, 150, 77), (2, 3, 70, 130)])
def test_loss_and_gradients_match_oracle(L, M, N, rows, T):
    rng = np.random.Generator(np.random.PCG64(1000 + rows))
    net, flat = random_net(L, M, N, rows, T, seed=rows + 1)
    feats, q = random_inputs(rng, rows, T)
    wt, lt, ht = clear_targets(L, rng, net, flat, feats, q, M, N)
    loss, g = net.loss_grad(cuda(feats), cuda(q), cuda(wt), cuda(lt), cuda(ht))
    mlp, conv = oracle_params(L, flat, M, N)
    targets = [((wt[r, ..., 0] + 1j * wt[r, ..., 1]).astype(np.complex128), lt[r].astype(np.float64),
                ht[r].astype(np.float64)) for r in range(rows)]
    ref_loss, ref_g, _ = ol.batch_loss_and_grads(mlp, conv, feats.astype(np.float64), q.astype(np.float64),
                                                 targets, M, N)
    assert abs(loss - ref_loss) <= 2e-2 * abs(ref_loss)
    D = ol.out_dim(M, N)
    gb = {k: np.asarray(v, np.float64) for k, v in L.unpack(g, M, N).items()}
    assert np.all(gb["W3"][D:] == 0) and np.all(gb["b3"][D:] == 0)
    gb["W3"], gb["b3"] = gb["W3"][:D], gb["b3"][:D]
    for k in ("W1", "b1", "W2", "b2", "W3", "b3", "k", "c"):
        err = np.linalg.norm(gb[k] - ref_g[k]) / np.linalg.norm(ref_g[k])
        assert err <= 5e-2, (k, err)

    # the head alone, in FP32, given the GPU's own network output: tight
    o = net.forward(cuda(feats)).astype(np.float64)
    base = 2 * M * M + M * N
    tot, do_sum, dk, dc = 0.0, np.zeros(D), np.zeros((N, L.CONV_K)), np.zeros(N)
    for r in range(rows):
        lnv = ol.conv_logv(conv["k"], conv["c"], o[r, base: base + N], q[r].astype(np.float64))
        lr, do, dlnv, _ = ol.loss_and_grads(o[r, :D], lnv, targets[r], M, N)
        dks, dcs, db = ol.conv_grads(conv["k"], dlnv, q[r].astype(np.float64))
        do[base: base + N] += db
        tot += lr
        do_sum += do
        dk += dks
        dc += dcs
    assert abs(loss - tot / rows) <= 1e-4 * abs(tot / rows)
    assert np.allclose(gb["b3"], do_sum / rows, rtol=1e-3, atol=1e-5 * np.abs(do_sum / rows).max())
    assert np.allclose(gb["k"], dk / rows, rtol=1e-3, atol=1e-5 * np.abs(dk / rows).max())
    assert np.allclose(gb["c"], dc / rows, rtol=1e-3, atol=1e-5 * np.abs(dc / rows).max())


def test_adam_first_step(L):
    M, N, rows, T = 3, 5, 64, 50
    rng = np.random.Generator(np.random.PCG64(77))
    net, flat = random_net(L, M, N, rows, T, seed=77)
    feats, q = random_inputs(rng, rows, T)
    wt, lt, ht = clear_targets(L, rng, net, flat, feats, q, M, N)
    args = [cuda(a) for a in (feats, q, wt, lt, ht)]
    _, g = net.loss_grad(*args)
    lr = 1e-3
    net.train_step(*args, lr)
    after = net.get_params()
    # first Adam step: m / (1 - b1) = g and sqrt(v / (1 - b2)) = |g|
    expect = flat - lr * g / (np.abs(g) + 1e-8)
    assert np.allclose(after, expect, atol=lr * 2e-3, rtol=0)


def test_training_reduces_loss(L):
    # teacher-student: targets are the (permuted, rescaled) prediction of a teacher network,
    # so the minimum is reachable; the student starts from perturbed teacher weights
    M, N, rows, T = 3, 5, 96, 60
    rng = np.random.Generator(np.random.PCG64(5))
    net, teacher = random_net(L, M, N, rows, T, seed=5)
    feats, q = random_inputs(rng, rows, T)
    wt, lt, ht = clear_targets(L, rng, net, teacher, feats, q, M, N, noise=0.0)
    student = teacher.copy()
    blocks = L.unpack(student, M, N)
    blocks["W3"][:] += 0.3 * np.abs(blocks["W3"]).mean() * rng.standard_normal(blocks["W3"].shape)
    blocks["b3"][:] += rng.uniform(-0.3, 0.3, blocks["b3"].shape)
    blocks["k"][:] += rng.uniform(-0.1, 0.1, blocks["k"].shape)
    net.set_params(student)
    args = [cuda(a) for a in (feats, q, wt, lt, ht)]
    first = net.train_step(*args, 1e-3, want_loss=True)
    for _ in range(300):
        last = net.train_step(*args, 1e-3, want_loss=True)
    assert last < 0.3 * first, (first, last)


@pytest.mark.parametrize("M,N,rows,T", [(3, 5, 70, 45), (2, 3, 20, 200)])
def test_predict_matches_oracle(L, M, N, rows, T):
    rng = np.random.Generator(np.random.PCG64(rows * 3))
    net, flat = random_net(L, M, N, rows, T, seed=rows * 3)
    feats, q = random_inputs(rng, rows, T)
    P, lam, v = net.predict(cuda(feats), cuda(q))
    P, lam, v = P.cpu().numpy(), lam.cpu().numpy(), v.cpu().numpy()
    mlp, conv = oracle_params(L, flat, M, N)
    o = net.forward(cuda(feats)).astype(np.float64)
    base = 2 * M * M
    for r in range(rows):
        # exact given the GPU network output
        W = (o[r, 0:base:2] + 1j * o[r, 1:base:2]).reshape(M, M)
        Wn = W / np.linalg.norm(W, axis=0, keepdims=True)
        assert np.allclose(P[r], Wn, atol=1e-6)
        assert np.allclose(lam[r], np.exp(o[r, base: base + M * N]).reshape(M, N), rtol=1e-5)
        lnv = ol.conv_logv(conv["k"], conv["c"], o[r, base + M * N: base + M * N + N], q[r].astype(np.float64))
        assert np.allclose(v[r], np.exp(lnv), rtol=1e-4)
        # FP64 reference prediction: BF16-level agreement
        Wr, Lr, Hr = ol.predict(mlp, conv, feats[r].astype(np.float64), q[r].astype(np.float64), M, N)
        assert np.abs(P[r] - Wr).max() <= 3e-2
        assert np.abs(np.log(lam[r]) - np.log(Lr)).max() <= 5e-2
        assert np.abs(np.log(v[r]) - np.log(Hr)).max() <= 5e-2


def test_unsupported_shapes_are_refused(L):
    from paper_2101_08563_gb300.fastfca import FastFCAError
    with pytest.raises(FastFCAError, match="EUNSUPPORTED"):
        L.InitNet(4, 6, 10, 10)
    with pytest.raises(FastFCAError, match="EINVAL"):
        L.InitNet(3, 5, 10, 60000)


# ---------------------------------------------------------------------------- what it gains
@pytest.fixture(scope="module")
def trained(L):
    """A network trained on 3000 generated mixtures of the learned-initialiser workload's shape
    (M=3, N=5, F=257, T=500, K=8, linear array 3 cm) with 200-iteration FastFCA targets."""
    M, N, F, T, K, d = 3, 5, 257, 500, 8, 0.03
    data, _ = L.make_training_set(3000, F, T, M, N, K, d, seed=31, iters=200)
    net = L.InitNet(M, N, max_rows=32 * F, max_T=T, seed=32)
    before = L.mean_loss(net, data)
    L.train(net, data, epochs=6, batch=2048, lr=1e-3, seed=33)
    after = L.mean_loss(net, data)
    del data
    torch.cuda.empty_cache()
    return net, before, after, (M, N, F, T, K, d)


def test_trained_network_gains_early_and_stays_near_the_converged_optimum(L, trained):
    net, before, after, (M, N, F, T, K, d) = trained
    assert after < 0.5 * before
    res = L.evaluate(net, 32, F, T, M, N, K, d, seed=(0xFFFF << 32) + 31, max_iters=1000)
    p, q = res["plain"], res["learned"]
    early = res["to_default_200"]
    # what the network gains: it reaches the default start's 200-iteration log-likelihood (the
    # training targets' iteration count, within 1e-3 per bin) on most held-out mixtures, in
    # less measured time than the default start, and it is far ahead after 10 iterations
    assert early["learned"]["reached_fraction"] >= 0.9
    assert early["learned"]["seconds_p50"] is not None and early["plain"]["seconds_p50"] is not None
    assert early["learned"]["seconds_p50"] < early["plain"]["seconds_p50"]
    assert q["ll_per_bin_after_10"] > p["ll_per_bin_after_10"]
    # against the converged reference (both starts run until the log-likelihood stops moving)
    # the learned start may settle in a lower optimum; the loss stays small
    assert q["final_ll_per_bin_minus_ref"] >= -0.05
    assert p["final_ll_per_bin_minus_ref"] >= -0.05
    # the network's W alone (default L and H) is reported beside them, timed the same way
    w = res["learned_w"]
    assert w["final_ll_per_bin_minus_ref"] >= -0.05 and res["to_default_200"]["learned_w"]["reached_fraction"] > 0


def test_trajectory_from_the_learned_start_matches_the_oracle(L, trained):
    from oracle import fastfca as off
    from paper_2101_08563_gb300 import fastfca as ffm
    net, _, _, (M, N, F, T, K, d) = trained
    x = L.generate_mixtures(1, F, T, M, N, K, d, seed=(0xFFFF << 32) + 77).view(F, T, M)
    feats, q = L.features(x, F)
    P, lam, v = net.predict(feats, q)
    freqs = [0, 40, 128, 256]
    xs = x[freqs].contiguous()
    sep = ffm.Separator(xs, N)
    sep.set_params(P[freqs].contiguous(), lam[freqs].contiguous(), v[freqs].contiguous())
    ll_gpu = sep.iterate(10)
    ref = off.run(xs.cpu().numpy(), P[freqs].cpu().numpy(), lam[freqs].cpu().numpy(), v[freqs].cpu().numpy(),
                  iters=10)
    ll_ref = ref["ll"].sum(axis=0)
    assert np.all(np.abs(ll_gpu - ll_ref) <= 1e-5 * np.abs(ll_ref))
    assert np.all(np.diff(ll_ref) >= -1e-9 * np.abs(ll_ref[1:]))
