"""Parity of the CUDA full-rank FCA comparison path with the complex128 FCA oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fca as ofca  # noqa: E402
from paper_2101_08563_gb300 import synth  # noqa: E402

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


@pytest.mark.parametrize("M,N,F,T,iters", [(2, 3, 4, 150, 3), (3, 4, 3, 200, 2), (4, 6, 2, 300, 2)])
def test_fca_parity_small(ff, M, N, F, T, iters):
    mix = synth.generate_mixture(M, N, F, T, 4, seed=200 + M + N)
    R0, h0 = synth.fca_random_init(mix.x, N, seed=11)
    sep = ff.Separator(torch.from_numpy(mix.x).cuda(), N, model="fca")
    sep.set_params_fca(R0, h0)
    ll = sep.iterate(iters)
    c = sep.separate()
    R, h = sep.get_params_fca()
    _, ll_f = sep.loglik(per_f=True)
    sep.close()
    ref = ofca.run(mix.x, R0, h0, iters=iters)
    ll_ref = ref["ll"].sum(axis=0)
    assert np.all(np.abs(ll - ll_ref) <= 1e-5 * np.abs(ll_ref)), (ll, ll_ref)
    assert np.allclose(ll_f, ref["ll"][:, -1], rtol=1e-5)
    c_ref = np.stack([ofca.separate(mix.x[f], ref["R"][i], ref["h"][i]) for i, f in enumerate(ref["freqs"])])
    assert rel(c, c_ref) <= 1e-4
    assert rel(R, ref["R"]) <= 1e-4
    assert rel(h, ref["h"]) <= 1e-3
    assert rel(c.sum(axis=2), mix.x) < 1e-5


def test_fca_loglik_monotone_full_width(ff):
    """The M=4, N=6 comparison workload's frequency width at reduced F and T: EM never
    decreases the likelihood (Sec. III-C)."""
    mix = synth.generate_mixture(4, 6, 8, 1250, 8, seed=2000)
    R0, h0 = synth.fca_random_init(mix.x, 6, seed=2000)
    sep = ff.Separator(torch.from_numpy(mix.x).cuda(), 6, model="fca")
    sep.set_params_fca(R0, h0)
    ll = sep.iterate(10)
    sep.close()
    assert np.all(np.diff(ll) >= -1e-6 * np.abs(ll[1:]))
