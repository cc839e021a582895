"""The batched path (many mixtures, mixed M, N, T, one CUDA-graph launch) against the
single-mixture path and the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fastfca as off  # noqa: E402
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


def mixed_batch(seed=7, B=9, F=6):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(B):
        M = int(rng.integers(2, 5))
        N = int(rng.integers(M + 1, M + 4))
        T = int(rng.integers(60, 700))
        mix = synth.generate_mixture(M, N, F, T, 4, seed=seed * 100 + b)
        init = synth.random_init(mix.x, N, seed=b)
        out.append((mix, init, N))
    return out


def test_batch_fine_schedule_equals_single_path_bitwise(ff):
    items = mixed_batch()
    xs = [torch.from_numpy(m.x).cuda() for m, _, _ in items]
    bt = ff.Batch(xs, [N for _, _, N in items])
    bt.schedule("fine", 1.0)
    for b, (m, init, N) in enumerate(items):
        bt.set_params(b, init.P, init.lam, init.v)
    ll, sec = bt.iterate(4)
    assert np.all(sec > 0)
    for b, (m, init, N) in enumerate(items):
        sep = ff.Separator(xs[b], N)
        sep.set_params(init.P, init.lam, init.v)
        sep.iterate(4, return_ll=False)
        tot = sep.loglik()
        Ps, ls, vs = sep.get_params()
        sep.close()
        Pb, lb, vb = bt.get_params(b)
        assert np.array_equal(Pb, Ps) and np.array_equal(lb, ls) and np.array_equal(vb, vs), b
        assert ll[b] == pytest.approx(tot, rel=1e-12)
    bt.close()


def test_batch_tuned_matches_oracle_and_resumes(ff):
    items = mixed_batch(seed=3, B=6, F=4)
    xs = [torch.from_numpy(m.x).cuda() for m, _, _ in items]
    bt = ff.Batch(xs, [N for _, _, N in items])
    for b, (m, init, N) in enumerate(items):
        bt.set_params(b, init.P, init.lam, init.v)
    scheme, factor = bt.tune(2)                  # probes restore the parameters
    assert scheme in ("fine", "coarse", "single") and factor > 0
    ll1, _ = bt.iterate(3)
    ll2, _ = bt.iterate(2)                       # graph reuse for a new n_iter, resume
    for b, (m, init, N) in enumerate(items):
        ref = off.run(m.x, init.P, init.lam, init.v, iters=5)
        assert ll2[b] == pytest.approx(ref["ll"][:, -1].sum(), rel=1e-5), b
        c = torch.empty((m.x.shape[0], m.x.shape[1], N, m.x.shape[2]), dtype=torch.complex64, device="cuda")
        bt.separate(b, c)
        torch.cuda.synchronize()
        cr = np.stack([off.separate_fast(m.x[f], ref["W"][i], ref["L"][i], ref["H"][i])
                       for i, f in enumerate(ref["freqs"])])
        assert np.linalg.norm(c.cpu().numpy() - cr) / np.linalg.norm(cr) <= 1e-4, b
    assert np.all(ll2 >= ll1 - 1e-6 * np.abs(ll1))
    bt.close()


def test_batch_mixed_algorithms(ff):
    """A batch whose mixtures take Algorithm 1 or Algorithm 2 each: every mixture matches the
    single-mixture path of its own algorithm bit for bit, and the oracle's run."""
    items = mixed_batch(seed=11, B=8, F=4)
    models = ["fastfca_mm" if b % 2 else "fastfca" for b in range(len(items))]
    xs = [torch.from_numpy(m.x).cuda() for m, _, _ in items]
    bt = ff.Batch(xs, [N for _, _, N in items], models=models)
    for b, (m, init, N) in enumerate(items):
        bt.set_params(b, init.P, init.lam, init.v)
    scheme, factor = bt.tune(2)
    for b, (m, init, N) in enumerate(items):
        bt.set_params(b, init.P, init.lam, init.v)
    ll, _ = bt.iterate(4)
    for b, (m, init, N) in enumerate(items):
        sep = ff.Separator(xs[b], N, model=models[b])
        sep.set_params(init.P, init.lam, init.v)
        sep.iterate(4, return_ll=False)
        Ps, ls, vs = sep.get_params()
        sep.close()
        Pb, lb, vb = bt.get_params(b)
        assert np.array_equal(Pb, Ps) and np.array_equal(lb, ls) and np.array_equal(vb, vs), (b, models[b])
        ref = off.run(m.x, init.P, init.lam, init.v, iters=4, algorithm="mm" if b % 2 else "em")
        assert ll[b] == pytest.approx(ref["ll"][:, -1].sum(), rel=1e-5), b
    bt.close()
