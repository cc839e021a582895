"""Parity of the CUDA full-rank FCA comparison path with the complex128 FCA oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fca as ofca  # noqa: E402
from paper_2101_08563_gb300 import synth  # noqa: E402
from parity import assert_images  # noqa: E402

pytestmark = pytest.mark.gpu


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


CASES = [(2, 3, 4, 150, 3), (3, 4, 3, 200, 2), (4, 6, 2, 300, 2)]


@pytest.mark.parametrize("algorithm", ["em", "mm"])
@pytest.mark.parametrize("M,N,F,T,iters", CASES + [(2, 8, 2, 517, 3), (4, 2, 3, 1029, 2)])
def test_fca_parity_small(ff, M, N, F, T, iters, algorithm):
    """EM (Eq. 12-13) or MM (Eq. 15-17) on the GPU against the oracle: log-likelihood after
    every iteration, the final R and h, the images.  T spans several 128-frame slots and ends
    in a ragged one."""
    mix = synth.generate_mixture(M, N, F, T, 4, seed=200 + M + N)
    R0, h0 = synth.fca_random_init(mix.x, N, seed=11)
    sep = ff.Separator(torch.from_numpy(mix.x).cuda(), N, model="fca" if algorithm == "em" else "fca_mm")
    sep.set_params_fca(R0, h0)
    ll = sep.iterate(iters)
    c = sep.separate()
    R, h = sep.get_params_fca()
    _, ll_f = sep.loglik(per_f=True)
    sep.close()
    ref = ofca.run(mix.x, R0, h0, iters=iters, algorithm=algorithm)
    ll_ref = ref["ll"].sum(axis=0)
    assert np.all(np.abs(ll - ll_ref) <= 1e-5 * np.abs(ll_ref)), (ll, ll_ref)
    assert np.allclose(ll_f, ref["ll"][:, -1], rtol=1e-5)
    c_ref = np.stack([ofca.separate(mix.x[f], ref["R"][i], ref["h"][i]) for i, f in enumerate(ref["freqs"])])
    assert_images(c, c_ref, 1e-4)
    assert rel(R, ref["R"]) <= 1e-4
    assert rel(h, ref["h"]) <= 1e-3
    assert rel(c.sum(axis=2), mix.x) < 1e-5


@pytest.mark.parametrize("model", ["fca", "fca_mm"])
def test_fca_loglik_monotone_full_width(ff, model):
    """The M=4, N=6 comparison workload's frame count at reduced F: neither EM (Sec. III-C)
    nor MM (App. B) decreases the likelihood."""
    mix = synth.generate_mixture(4, 6, 8, 1250, 8, seed=2000)
    R0, h0 = synth.fca_random_init(mix.x, 6, seed=2000)
    sep = ff.Separator(torch.from_numpy(mix.x).cuda(), 6, model=model)
    sep.set_params_fca(R0, h0)
    ll = sep.iterate(10)
    sep.close()
    assert np.all(np.diff(ll) >= -1e-6 * np.abs(ll[1:]))


def test_fca_mm_sampled_frequencies_of_the_comparison_workload(ff):
    """MM on the full M=4, N=6, F=513, T=1250 comparison workload, 10 iterations, in the
    benchmark's launch configuration; the oracle recomputes sampled frequencies."""
    w = synth.WORKLOADS["fca_cmp"]
    mix = synth.workload_mixture(w)
    R0, h0 = synth.fca_random_init(mix.x, w.N, seed=w.seed)
    sep = ff.Separator(torch.from_numpy(mix.x).cuda(), w.N, model="fca_mm")
    sep.set_params_fca(R0, h0)
    sep.iterate(10)
    R, h = sep.get_params_fca()
    _, ll_f = sep.loglik(per_f=True)
    sep.close()
    freqs = [0, 200, 512]
    ref = ofca.run(mix.x, R0, h0, iters=10, freqs=freqs, algorithm="mm")
    for i, f in enumerate(freqs):
        assert abs(ll_f[f] - ref["ll"][i, -1]) <= 1e-5 * abs(ref["ll"][i, -1]), f
        assert rel(R[f], ref["R"][i]) <= 1e-4, f
