"""Parity of the one-SM IP+EM kernel (fastfca_em_sm.cuh: one CTA per frequency, sigma^2 and U
of every frame in tensor memory) with the complex128 oracle, through the C ABI.

Tolerances as for the other kernels: total log-likelihood relative error <= 1e-5 per
iteration, source images <= 1e-4 per (frequency, source) block, relative Frobenius and
element-wise.  The cases cover M = 5..8, one to eight frame slots per thread with ragged
last slots, the largest T the kernel takes (4096), one source and sixteen, the
log-likelihood of given parameters (no iteration), bitwise resumption, long runs and the
large workload at full size in the benchmark's launch configuration.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fastfca as off  # noqa: E402
from paper_2101_08563_gb300 import synth  # noqa: E402
from parity import assert_images  # noqa: E402

pytestmark = pytest.mark.gpu

LL_TOL = 1e-5
IMG_TOL = 1e-4


@pytest.fixture(scope="module")
def ff():
    """The library with IP+EM on the large-bin shapes forced onto the one-SM kernel."""
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2101_08563_gb300 import build, fastfca
    build.build()
    fastfca.load()
    fastfca.large_bin_kernel("sm")
    yield fastfca
    fastfca.large_bin_kernel("auto")


def mixture(M, N, F, T, seed, K=8):
    return synth.generate_mixture(M, N, F, T, K, seed=seed, array="circular" if M >= 5 else "linear",
                                  spacing=0.05 if M >= 5 else 0.03)


def check_parity(ff, M, N, F, T, iters, seed=1):
    mix = mixture(M, N, F, T, seed)
    init = synth.random_init(mix.x, N, seed=seed)
    sep = ff.Separator(torch.from_numpy(mix.x).cuda(), N)
    sep.set_params(init.P, init.lam, init.v)
    ll = sep.iterate(iters)
    c = sep.separate()
    P, lam, v = sep.get_params()
    _, ll_f = sep.loglik(per_f=True)
    sep.close()
    ref = off.run(mix.x, init.P, init.lam, init.v, iters=iters)
    ll_ref = ref["ll"].sum(axis=0)
    assert np.all(np.abs(ll - ll_ref) <= LL_TOL * np.abs(ll_ref)), (ll, ll_ref)
    assert np.allclose(ll_f, ref["ll"][:, -1], rtol=LL_TOL, atol=0)
    cr = np.stack([off.separate_fast(mix.x[f], ref["W"][f], ref["L"][f], ref["H"][f]) for f in range(F)])
    assert_images(c, cr, IMG_TOL)
    assert np.linalg.norm(c.sum(axis=2) - mix.x) / np.linalg.norm(mix.x) < 1e-5
    s2 = np.einsum("fmn,fnt->fmt", lam.astype(np.float64), v.astype(np.float64))
    s2_ref = np.einsum("fmn,fnt->fmt", ref["L"], ref["H"])
    assert np.allclose(s2, s2_ref, rtol=2e-3)
    return ll


@pytest.mark.parametrize("M,N,F,T,iters", [
    (8, 12, 3, 300, 4),     # one frame slot, most threads idle in it
    (8, 12, 2, 1001, 3),    # two slots, ragged
    (8, 12, 2, 4000, 2),    # the large workload's frames and sources
    (8, 12, 2, 4096, 2),    # the most frames: every slot of every thread full
    (5, 7, 3, 257, 4),      # odd M: idle lanes in the Q pass
    (6, 9, 2, 611, 3),
    (7, 16, 2, 3333, 3),    # the most sources
    (8, 1, 2, 2500, 3),     # one source: sigma^2 = L H is the whole model
    (5, 16, 2, 4095, 2),
])
def test_sm_parity(ff, M, N, F, T, iters):
    check_parity(ff, M, N, F, T, iters)


def test_sm_loglik_of_given_parameters(ff):
    """fastfca_loglik (no iteration: the kernel's U pass, then pass A) equals Eq. 31 of the
    oracle at arbitrary parameters."""
    rng = np.random.Generator(np.random.PCG64(8))
    M, N, F, T = 8, 12, 3, 2000
    mix = mixture(M, N, F, T, 8)
    P = (rng.standard_normal((F, M, M)) + 1j * rng.standard_normal((F, M, M))) * 0.2 + np.eye(M)
    lam = rng.uniform(0.2, 2.0, (F, M, N)).astype(np.float32)
    v = rng.uniform(0.2, 5.0, (F, N, T)).astype(np.float32)
    sep = ff.Separator(torch.from_numpy(mix.x).cuda(), N)
    sep.set_params(P, lam, v)
    tot, per_f = sep.loglik(per_f=True)
    sep.close()
    ref = [off.loglik(off.Xhat_from_x(mix.x[f]), P[f], lam[f].astype(np.float64), v[f].astype(np.float64))
           for f in range(F)]
    assert np.allclose(per_f, ref, rtol=1e-6, atol=0)
    assert tot == pytest.approx(sum(ref), rel=1e-6)


def test_sm_resume_is_bitwise_and_loglik_matches_the_history(ff):
    """iterate(3) then iterate(4) equals iterate(7) bit for bit (W^{-H} and |det W|^2 carried
    between launches, fixed-order reductions); the log-likelihood of the final parameters is
    the history's last value."""
    M, N, F, T = 8, 12, 2, 2222
    mix = mixture(M, N, F, T, 4)
    init = synth.random_init(mix.x, N, seed=4)
    xd = torch.from_numpy(mix.x).cuda()
    a = ff.Separator(xd, N)
    a.set_params(init.P, init.lam, init.v)
    ll_a = np.concatenate([a.iterate(3), a.iterate(4)])
    b = ff.Separator(xd, N)
    b.set_params(init.P, init.lam, init.v)
    ll_b = b.iterate(7)
    for u, w in zip(a.get_params(), b.get_params()):
        assert np.array_equal(u, w)
    assert np.array_equal(ll_a, ll_b)
    assert np.all(np.diff(ll_b) >= -1e-6 * np.abs(ll_b[1:]))
    tot = a.loglik()
    assert tot == pytest.approx(ll_b[-1], rel=1e-9)
    a.close()
    b.close()


def test_sm_and_cluster_kernels_agree(ff):
    """The two large-bin kernels run the same steps: after five iterations from one start their
    log-likelihoods and images agree to FP32 rounding."""
    M, N, F, T = 8, 12, 2, 3000
    mix = mixture(M, N, F, T, 12)
    init = synth.random_init(mix.x, N, seed=12)
    xd = torch.from_numpy(mix.x).cuda()
    out = {}
    for kernel in ("sm", "cluster"):
        ff.large_bin_kernel(kernel)
        sep = ff.Separator(xd, N)
        sep.set_params(init.P, init.lam, init.v)
        out[kernel] = (sep.iterate(5), sep.separate())
        sep.close()
    ff.large_bin_kernel("sm")
    assert np.allclose(out["sm"][0], out["cluster"][0], rtol=1e-6, atol=0)
    assert_images(out["sm"][1], out["cluster"][1], IMG_TOL, "one-SM vs cluster")


def test_sm_long_run_stays_finite_and_monotone(ff):
    """500 IP+EM iterations: every log-likelihood finite and non-decreasing within FP32
    rounding (Algorithm 1 is an ascent method)."""
    M, N, T = 8, 12, 4000
    mix = mixture(M, N, 4, T, 901, K=16)
    init = synth.random_init(mix.x, N, seed=901)
    sep = ff.Separator(torch.from_numpy(mix.x).cuda(), N)
    sep.set_params(init.P, init.lam, init.v)
    ll = np.concatenate([sep.iterate(100) for _ in range(5)])
    c = sep.separate()
    sep.close()
    assert np.all(np.isfinite(ll))
    assert np.all(np.diff(ll) >= -2e-6 * np.abs(ll[1:])), np.min(np.diff(ll) / np.abs(ll[1:]))
    assert np.all(np.isfinite(c)) and np.linalg.norm(c.sum(axis=2) - mix.x) / np.linalg.norm(mix.x) < 1e-5


def test_large_workload_full_size_on_the_sm_kernel(ff, large_workload):
    """The large single instance (M=8 circular 5 cm, N=12, F=1025, T=4000, K=16, 50
    iterations) in the benchmark's launch configuration (one CTA per frequency); the oracle
    follows four frequencies across the band."""
    w, x, init = large_workload
    ff.large_bin_kernel("auto")                 # the benchmark's choice for this shape
    xd = torch.from_numpy(x).cuda()
    sep = ff.Separator(xd, w.N)
    sep.set_params(init.P, init.lam, init.v)
    hist = sep.iterate(w.iters)
    _, ll_f = sep.loglik(per_f=True)
    c = torch.empty((w.F, w.T, w.N, w.M), dtype=torch.complex64, device="cuda")
    sep.separate(c)
    sep.close()
    ff.large_bin_kernel("sm")
    assert np.all(np.diff(hist) >= -1e-6 * np.abs(hist[1:]))
    freqs = [1, 333, 700, 1024]
    ref = off.run(x, init.P, init.lam, init.v, iters=w.iters, freqs=freqs)
    for i, f in enumerate(freqs):
        assert abs(ll_f[f] - ref["ll"][i, -1]) <= LL_TOL * abs(ref["ll"][i, -1]), f
        cr = off.separate_fast(x[f], ref["W"][i], ref["L"][i], ref["H"][i])
        assert_images(c[f:f + 1].cpu().numpy(), cr[None], IMG_TOL, f"f={f}")
    xs = c.sum(dim=2)
    assert float((xs - xd).abs().pow(2).sum().sqrt() / xd.abs().pow(2).sum().sqrt()) < 1e-5


def test_frequency_ranges_run_alone_equal_the_whole_run(ff):
    """The premise of sharding one mixture over ranks by frequency (shard.py): each frequency
    is computed on its own, so contexts on contiguous frequency ranges give, bit for bit, the
    rows of one context on the whole mixture, and their per-iteration log-likelihoods sum to
    the whole run's."""
    from paper_2101_08563_gb300 import shard
    M, N, F, T = 8, 12, 5, 2500
    mix = mixture(M, N, F, T, 31)
    init = synth.random_init(mix.x, N, seed=31)
    xd = torch.from_numpy(mix.x).cuda()
    whole = ff.Separator(xd, N)
    whole.set_params(init.P, init.lam, init.v)
    ll_whole = whole.iterate(3)
    Pw, lw, vw = whole.get_params()
    whole.close()
    ll_sum = np.zeros(3)
    for f0, f1 in shard.frequency_ranges(F, 2):
        part = ff.Separator(xd[f0:f1].clone(), N)
        part.set_params(init.P[f0:f1], init.lam[f0:f1], init.v[f0:f1])
        ll_sum += part.iterate(3)
        P, lam, v = part.get_params()
        part.close()
        assert np.array_equal(P, Pw[f0:f1]) and np.array_equal(lam, lw[f0:f1]) and np.array_equal(v, vw[f0:f1])
    assert np.allclose(ll_sum, ll_whole, rtol=1e-12, atol=0)


@pytest.mark.parametrize("M,N,T", [(8, 12, 1001), (6, 9, 611)])
def test_filter_output_on_an_8_byte_boundary(ff, M, N, T):
    """The large-bin filter writes each frame's images with one bulk copy when the output
    starts on 16 bytes, and with plain stores otherwise (c on an 8-byte boundary, which the
    API accepts): both give the same bits, ragged last tile included."""
    mix = mixture(M, N, 2, T, 3)
    init = synth.random_init(mix.x, N, seed=3)
    sep = ff.Separator(torch.from_numpy(mix.x).cuda(), N)
    sep.set_params(init.P, init.lam, init.v)
    sep.iterate(2, return_ll=False)
    n = 2 * T * N * M
    aligned = torch.empty(n, dtype=torch.complex64, device="cuda")
    base = torch.empty(n + 1, dtype=torch.complex64, device="cuda")
    shifted = base[1:]
    assert aligned.data_ptr() % 16 == 0 and shifted.data_ptr() % 16 == 8
    sep.separate(aligned.view(2, T, N, M))
    sep.separate(shifted.view(2, T, N, M))
    torch.cuda.synchronize()
    sep.close()
    assert torch.equal(aligned, shifted)
