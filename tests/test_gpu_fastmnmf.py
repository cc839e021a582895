"""Parity of the CUDA FastMNMF path (App. C) with the complex128 FastMNMF oracle.

The oracle keeps the paper's index order (t as (I, K, N), v as (J, K, N)); the C ABI stores
t as [F][N][K] and v as [N][K][T].  The conversions below are the only glue."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fastmnmf as omn  # noqa: E402
from paper_2101_08563_gb300 import synth  # noqa: E402
from parity import assert_images  # noqa: E402

pytestmark = pytest.mark.gpu

LL_TOL = 1e-5
IMG_TOL = 1e-4


@pytest.fixture(scope="module")
def ff():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2101_08563_gb300 import build, fastfca
    build.build()
    fastfca.load()
    return fastfca


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def to_abi(st):
    return (st.W, st.lam, np.ascontiguousarray(st.t.transpose(0, 2, 1)),
            np.ascontiguousarray(st.v.transpose(2, 1, 0)))


def from_abi(t, v):
    return t.transpose(0, 2, 1).astype(np.float64), v.transpose(2, 1, 0).astype(np.float64)


def run_gpu(ff, x, N, K, st, iters):
    sep = ff.Separator(torch.from_numpy(x).cuda(), N, model="fastmnmf", bases=K)
    sep.set_params_mnmf(*to_abi(st))
    ll = sep.iterate(iters)
    c = sep.separate()
    W, lam, t, v = sep.get_params_mnmf()
    _, ll_f = sep.loglik(per_f=True)
    sep.close()
    return ll, c, W, lam, t, v, ll_f


@pytest.mark.parametrize("M,N,K,F,T,iters", [
    (2, 3, 2, 6, 150, 3),
    (3, 4, 4, 5, 300, 2),
    (4, 6, 8, 4, 517, 2),       # ragged last warp of frames
    (2, 2, 1, 3, 64, 3),        # one basis
    (3, 2, 16, 2, 96, 2),       # the most bases, several (n, k) chunks
    (4, 8, 3, 2, 2048, 1),      # the most frames one CTA holds
    (3, 2, 5, 1, 333, 3),       # one frequency: the v update sums over a single bin
    (8, 12, 4, 2, 600, 2),      # thread-block clusters from here on
    (3, 10, 3, 3, 400, 3),
    (4, 6, 4, 2, 3000, 2),      # more frames than one frequency-resident CTA holds
    (2, 1, 2, 2, 200, 3),       # one source
    (6, 16, 2, 2, 150, 2),      # the most sources
])
def test_fastmnmf_parity(ff, M, N, K, F, T, iters):
    """Log-likelihood after every iteration, per-frequency log-likelihood, images, W and the
    scale-free h = t v against the oracle from the same start."""
    # the generator's frequency grid needs F >= 2: one frequency is the upper bin of two
    mix = synth.generate_mixture(M, N, max(F, 2), T, K, seed=300 + M + N + K)
    mix.x = np.ascontiguousarray(mix.x[-F:])
    st = synth.fastmnmf_random_init(mix.x, N, K, seed=17)
    ll, c, W, lam, t, v, ll_f = run_gpu(ff, mix.x, N, K, st, iters)
    ref = omn.run(mix.x, st.W, st.lam, st.t, st.v, iters=iters)
    assert np.all(np.abs(ll - ref["ll"]) <= LL_TOL * np.abs(ref["ll"])), (ll, ref["ll"])
    ll_f_ref = omn.loglik_per_f(mix.x.astype(np.complex128), ref["W"], ref["lam"], ref["t"], ref["v"])
    assert np.allclose(ll_f, ll_f_ref, rtol=LL_TOL)
    c_ref = omn.separate(mix.x.astype(np.complex128), ref["W"], ref["lam"], ref["t"], ref["v"])
    assert_images(c, c_ref, IMG_TOL)
    assert rel(c.sum(axis=2), mix.x) < 1e-5
    assert np.max(np.abs(W - ref["W"])) <= 1e-3 * np.max(np.abs(ref["W"]))
    tg, vg = from_abi(t, v)
    assert rel(omn.h_of(tg, vg), omn.h_of(ref["t"], ref["v"])) <= 1e-3
    assert rel(lam, ref["lam"]) <= 1e-3


def test_fastmnmf_loglik_of_given_parameters(ff):
    """fastfca_loglik on a FastMNMF context (no iteration) is Eq. 53 of the oracle."""
    rng = np.random.Generator(np.random.PCG64(5))
    M, N, K, F, T = 3, 3, 2, 4, 200
    mix = synth.generate_mixture(M, N, F, T, K, seed=5)
    st = synth.fastmnmf_random_init(mix.x, N, K, seed=5)
    W = st.W + 0.2 * (rng.standard_normal(st.W.shape) + 1j * rng.standard_normal(st.W.shape))
    st = synth.FastMNMFInit(W=W, lam=st.lam, t=st.t, v=st.v)
    sep = ff.Separator(torch.from_numpy(mix.x).cuda(), N, model="fastmnmf", bases=K)
    sep.set_params_mnmf(*to_abi(st))
    tot, per_f = sep.loglik(per_f=True)
    sep.close()
    ref = omn.loglik_per_f(mix.x.astype(np.complex128), W, st.lam.astype(np.float64),
                           st.t.astype(np.float64), st.v.astype(np.float64))
    assert np.allclose(per_f, ref, rtol=1e-6)
    assert abs(tot - ref.sum()) <= 1e-6 * abs(ref.sum())


def test_fastmnmf_default_start_is_monotone(ff):
    """The library's own start (Philox) on a generated mixture: finite and non-decreasing."""
    mix = synth.generate_mixture(4, 5, 16, 700, 4, seed=41)
    sep = ff.Separator(torch.from_numpy(mix.x).cuda(), 5, model="fastmnmf", bases=4, seed=3)
    ll = sep.iterate(12)
    c = sep.separate()
    sep.close()
    assert np.all(np.isfinite(ll))
    assert np.all(np.diff(ll) >= -1e-6 * np.abs(ll[1:]))
    assert rel(c.sum(axis=2), mix.x) < 1e-5


def test_fastmnmf_full_size(ff):
    """M=4, N=6, K=8, F=513, T=1250 in the benchmark's configuration, two iterations against
    the whole oracle (the frequencies are coupled, so no frequency can be recomputed alone);
    images compared at sampled frequencies."""
    w = synth.WORKLOADS["fca_cmp"]
    K = 8
    mix = synth.workload_mixture(w)
    st = synth.fastmnmf_random_init(mix.x, w.N, K, seed=w.seed)
    ll, c, W, lam, t, v, ll_f = run_gpu(ff, mix.x, w.N, K, st, 2)
    ref = omn.run(mix.x, st.W, st.lam, st.t, st.v, iters=2)
    assert np.all(np.abs(ll - ref["ll"]) <= LL_TOL * np.abs(ref["ll"])), (ll, ref["ll"])
    x = mix.x.astype(np.complex128)
    for f in (0, 100, 256, 512):
        cr = omn.separate(x[f:f + 1], ref["W"][f:f + 1], ref["lam"][f:f + 1], ref["t"][f:f + 1], ref["v"])
        assert_images(c[f:f + 1], cr, IMG_TOL, f"f={f}")


@pytest.mark.parametrize("M,N,K,T,why", [
    (9, 3, 4, 100, "M"), (3, 17, 4, 100, "N"), (3, 3, 4, 40000, "T")])
def test_fastmnmf_unsupported_shapes(ff, M, N, K, T, why):
    x = torch.zeros((2, T, M), dtype=torch.complex64, device="cuda")
    with pytest.raises(ff.FastFCAError, match="EUNSUPPORTED"):
        ff.Separator(x, N, model="fastmnmf", bases=K)


@pytest.mark.parametrize("K", [0, 17])
def test_fastmnmf_bases_out_of_range(ff, K):
    x = torch.ones((2, 64, 3), dtype=torch.complex64, device="cuda")
    with pytest.raises(ff.FastFCAError, match="EINVAL"):
        ff.Separator(x, 3, model="fastmnmf", bases=K)


def test_fastmnmf_params_on_other_models_are_rejected(ff):
    x = torch.ones((2, 64, 3), dtype=torch.complex64, device="cuda")
    sep = ff.Separator(x, 3)
    with pytest.raises(ff.FastFCAError, match="EINVAL"):
        sep.get_params_mnmf()
    sep.close()
