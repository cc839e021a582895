"""Parity of the cluster kernel (large bins: M up to 8, N up to 16, T beyond one CTA) with the
complex128 oracle, through the C ABI.

The same tolerances as the frequency-resident path: total log-likelihood relative error
<= 1e-5 per iteration, source images relative Frobenius error <= 1e-4.  The cases choose T so
that the cluster size (1, 2, 4 or 8 CTAs per frequency, picked from the shared memory the
frames need) takes every value, with ragged last CTAs.
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
    """The library with IP+EM on the large-bin shapes forced onto the cluster kernel (the
    one-SM kernel takes some of these shapes by default; tests/test_gpu_sm.py covers it)."""
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2101_08563_gb300 import build, fastfca
    build.build()
    fastfca.load()
    fastfca.large_bin_kernel("cluster")
    yield fastfca
    fastfca.large_bin_kernel("auto")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def check_parity(ff, M, N, F, T, iters, K=4, array="linear", spacing=0.03, seed=1):
    mix = synth.generate_mixture(M, N, F, T, K, seed=seed, array=array, spacing=spacing)
    init = synth.random_init(mix.x, N, seed=seed)
    sep = ff.Separator(torch.from_numpy(mix.x).cuda(), N)
    sep.set_params(init.P, init.lam, init.v)
    ll = sep.iterate(iters)
    c = sep.separate()
    sep.close()
    ref = off.run(mix.x, init.P, init.lam, init.v, iters=iters)
    ll_ref = ref["ll"].sum(axis=0)
    assert np.all(np.abs(ll - ll_ref) <= LL_TOL * np.abs(ll_ref)), (ll, ll_ref)
    cr = np.stack([off.separate_fast(mix.x[f], ref["W"][f], ref["L"][f], ref["H"][f]) for f in range(F)])
    assert_images(c, cr, IMG_TOL)
    assert rel(c.sum(axis=2), mix.x) < 1e-5
    return ll


@pytest.mark.parametrize("M,N,F,T,iters", [
    (8, 12, 3, 300, 4),     # C = 1
    (8, 12, 2, 1001, 3),    # C = 2, ragged
    (8, 12, 2, 2003, 2),    # C = 4, ragged
    (8, 12, 2, 4000, 2),    # C = 8: the large workload's frames and sources
    (5, 7, 3, 257, 4),      # odd M
    (6, 9, 2, 611, 3),
    (7, 16, 2, 333, 3),     # the most sources
    (3, 10, 3, 400, 4),     # N beyond the frequency-resident kernel
    (2, 3, 3, 2500, 3),     # T beyond one CTA of the frequency-resident kernel
    (4, 6, 2, 3001, 2),
])
def test_cluster_parity(ff, M, N, F, T, iters):
    check_parity(ff, M, N, F, T, iters, array="circular" if M >= 5 else "linear",
                 spacing=0.05 if M >= 5 else 0.03)


def max_frames(ff, M, N):
    """The largest T a context accepts for (M, N), found by bisection on creation (a T beyond
    what eight CTAs hold is rejected with EUNSUPPORTED before any kernel runs)."""
    def accepted(T):
        try:
            ff.Separator(torch.zeros((1, T, M), dtype=torch.complex64, device="cuda"), N).close()
            return True
        except ff.FastFCAError as e:
            assert "EUNSUPPORTED" in str(e), str(e)
            return False
    lo, hi = 4000, 65536
    assert accepted(lo) and not accepted(hi)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        lo, hi = (mid, hi) if accepted(mid) else (lo, mid)
    return lo


@pytest.mark.parametrize("M,N", [(8, 16), (3, 4)])
def test_cluster_parity_at_the_most_frames(ff, M, N):
    """Parity at the largest T the cluster kernel takes for (M, N): the last CTA of the
    eight is full or nearly so, and shared memory is at its carve-out."""
    T = max_frames(ff, M, N)
    check_parity(ff, M, N, 2, T, 2, array="circular" if M >= 5 else "linear",
                 spacing=0.05 if M >= 5 else 0.03)


def test_cluster_loglik_resume_and_monotone(ff):
    M, N, F, T = 8, 12, 2, 1500
    mix = synth.generate_mixture(M, N, F, T, 8, seed=4, array="circular", spacing=0.05)
    init = synth.random_init(mix.x, N, seed=4)
    xd = torch.from_numpy(mix.x).cuda()
    a = ff.Separator(xd, N)
    a.set_params(init.P, init.lam, init.v)
    ll_a = np.concatenate([a.iterate(3), a.iterate(4)])
    b = ff.Separator(xd, N)
    b.set_params(init.P, init.lam, init.v)
    ll_b = b.iterate(7)
    pa, pb = a.get_params(), b.get_params()
    for u, w in zip(pa, pb):
        assert np.array_equal(u, w)
    assert np.array_equal(ll_a, ll_b)
    assert np.all(np.diff(ll_b) >= -1e-6 * np.abs(ll_b[1:]))
    # log-likelihood of the current parameters without iterating: the last value again
    tot, per_f = a.loglik(per_f=True)
    assert tot == pytest.approx(ll_b[-1], rel=1e-9)
    ref = [off.loglik(off.Xhat_from_x(mix.x[f]), pa[0][f], pa[1][f].astype(np.float64), pa[2][f].astype(np.float64))
           for f in range(F)]
    assert np.allclose(per_f, ref, rtol=1e-6)
    a.close()
    b.close()


def test_large_workload_sampled_frequencies(ff, large_workload):
    """The large single instance at full size (M=8 circular 5 cm, N=12, F=1025, T=4000, K=16,
    50 iterations) on the cluster kernel (clusters of 8 CTAs); the oracle follows three
    frequencies."""
    w, x, init = large_workload
    xd = torch.from_numpy(x).cuda()
    sep = ff.Separator(xd, w.N)
    sep.set_params(init.P, init.lam, init.v)
    hist = sep.iterate(w.iters)
    _, ll_f = sep.loglik(per_f=True)
    freqs = [1, 512, 1024]
    ref = off.run(x, init.P, init.lam, init.v, iters=w.iters, freqs=freqs)
    c = torch.empty((w.F, w.T, w.N, w.M), dtype=torch.complex64, device="cuda")
    sep.separate(c)
    sep.close()
    assert np.all(np.diff(hist) >= -1e-6 * np.abs(hist[1:]))
    for i, f in enumerate(freqs):
        assert abs(ll_f[f] - ref["ll"][i, -1]) <= LL_TOL * abs(ref["ll"][i, -1]), f
        cr = off.separate_fast(x[f], ref["W"][i], ref["L"][i], ref["H"][i])
        assert_images(c[f:f + 1].cpu().numpy(), cr[None], IMG_TOL, f"f={f}")
    xs = c.sum(dim=2)
    assert float((xs - xd).abs().pow(2).sum().sqrt() / xd.abs().pow(2).sum().sqrt()) < 1e-5


def test_cluster_limits(ff):
    x = torch.zeros((2, 64, 9), dtype=torch.complex64, device="cuda")
    with pytest.raises(ff.FastFCAError, match="EUNSUPPORTED"):
        ff.Separator(x, 10)                               # M = 9
    x = torch.zeros((2, 64, 8), dtype=torch.complex64, device="cuda")
    with pytest.raises(ff.FastFCAError, match="EUNSUPPORTED"):
        ff.Separator(x, 17)                               # N = 17
    x = torch.zeros((1, 20000, 8), dtype=torch.complex64, device="cuda")
    with pytest.raises(ff.FastFCAError, match="EUNSUPPORTED"):
        ff.Separator(x, 16)                               # frames beyond eight CTAs


def test_cluster_reports_non_positive_power(ff):
    M, N, F, T = 6, 8, 2, 2000              # clusters of two CTAs of 1000 frames
    mix = synth.generate_mixture(M, N, F, T, 4, seed=6, array="circular", spacing=0.05)
    init = synth.random_init(mix.x, N, seed=6)
    sep = ff.Separator(torch.from_numpy(mix.x).cuda(), N)
    bad_v = init.v.copy()
    bad_v[1, :, 1500] = 0.0                # a frame of the second CTA: sigma^2 = 0 there
    sep.set_params(init.P, init.lam, bad_v)
    with pytest.raises(ff.FastFCAError, match="ENUMERIC"):
        sep.iterate(2)
    sep.set_params(init.P, init.lam, init.v)
    assert np.all(np.isfinite(sep.iterate(2)))
    sep.close()
