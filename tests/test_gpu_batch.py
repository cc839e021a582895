"""The batched path (many mixtures, mixed M, N, T, one CUDA-graph launch) against the
single-mixture path and the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fastfca as off  # noqa: E402
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


def test_batch_fine_schedule_matches_single_path(ff):
    """The persistent class schedule (fine buckets) against the single-mixture path and the
    oracle: the single path keeps sigma^2 in tensor memory and updates it by each source's
    change where the persistent kernel recomputes it as L H, so the two agree to rounding
    (log-likelihoods within 1e-5 of each other and of the oracle), not bit for bit."""
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
        sep.close()
        ref = off.run(m.x, init.P, init.lam, init.v, iters=4)
        assert ll[b] == pytest.approx(tot, rel=1e-5), b
        assert ll[b] == pytest.approx(ref["ll"][:, -1].sum(), rel=1e-5), b
    bt.close()


def test_batch_mixture_schedule(ff):
    """One single-mixture launch per mixture on concurrent graph branches (schedule 3), with
    Algorithm 1 and Algorithm 2 mixtures mixed.  The first call after set_params equals the
    single-mixture path bit for bit (both form B = W^{-H} from W at the start); a second call
    (B formed again, where the single path carries it) continues the oracle's trajectory; the
    timed form (seconds requested: direct launches between events) gives the same results as
    the graph."""
    items = mixed_batch(seed=21, B=7, F=5)
    models = ["fastfca_mm" if b % 3 == 1 else "fastfca" for b in range(len(items))]
    xs = [torch.from_numpy(m.x).cuda() for m, _, _ in items]
    bt = ff.Batch(xs, [N for _, _, N in items], models=models)
    bt.schedule("mixture", 2.0)
    for b, (m, init, N) in enumerate(items):
        bt.set_params(b, init.P, init.lam, init.v)
    ll1, sec = bt.iterate(3)
    assert np.all(sec > 0)
    for b, (m, init, N) in enumerate(items):
        sep = ff.Separator(xs[b], N, model=models[b])
        sep.set_params(init.P, init.lam, init.v)
        sep.iterate(3, return_ll=False)
        tot = sep.loglik()
        Ps, ls, vs = sep.get_params()
        sep.close()
        Pb, lb, vb = bt.get_params(b)
        assert np.array_equal(Pb, Ps) and np.array_equal(lb, ls) and np.array_equal(vb, vs), (b, models[b])
        assert ll1[b] == pytest.approx(tot, rel=1e-12)
    bt.iterate(2, stats=False)                   # through the graph
    ll2, _ = bt.iterate(1, seconds=False)        # through the graph, log-likelihoods read back
    for b, (m, init, N) in enumerate(items):
        ref = off.run(m.x, init.P, init.lam, init.v, iters=6, algorithm="mm" if models[b] == "fastfca_mm" else "em")
        assert ll2[b] == pytest.approx(ref["ll"][:, -1].sum(), rel=1e-5), b
    bt.close()


def test_batch_tuned_matches_oracle_and_resumes(ff):
    items = mixed_batch(seed=3, B=6, F=4)
    xs = [torch.from_numpy(m.x).cuda() for m, _, _ in items]
    bt = ff.Batch(xs, [N for _, _, N in items])
    for b, (m, init, N) in enumerate(items):
        bt.set_params(b, init.P, init.lam, init.v)
    scheme, factor = bt.tune(2)                  # probes restore the parameters
    assert scheme in ("fine", "coarse", "single", "mixture") and factor > 0
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
        assert_images(c.cpu().numpy(), cr, 1e-4, f"mixture {b}")
    assert np.all(ll2 >= ll1 - 1e-6 * np.abs(ll1))
    bt.close()


def test_batch_mixed_algorithms(ff):
    """A batch whose mixtures take Algorithm 1 or Algorithm 2 each.  Under the per-mixture
    schedule (the single-mixture path's own launches) every mixture matches that path of its
    own algorithm bit for bit; under whatever schedule the tuner picks (its CTA size sets the
    order of the frame sums, so the bits may differ) each matches the oracle's run."""
    items = mixed_batch(seed=11, B=8, F=4)
    models = ["fastfca_mm" if b % 2 else "fastfca" for b in range(len(items))]
    xs = [torch.from_numpy(m.x).cuda() for m, _, _ in items]
    bt = ff.Batch(xs, [N for _, _, N in items], models=models)
    for b, (m, init, N) in enumerate(items):
        bt.set_params(b, init.P, init.lam, init.v)
    scheme, factor = bt.tune(2)
    for b, (m, init, N) in enumerate(items):
        bt.set_params(b, init.P, init.lam, init.v)
    ll_tuned, _ = bt.iterate(4)
    for b, (m, init, N) in enumerate(items):
        ref = off.run(m.x, init.P, init.lam, init.v, iters=4, algorithm="mm" if b % 2 else "em")
        assert ll_tuned[b] == pytest.approx(ref["ll"][:, -1].sum(), rel=1e-5), (b, scheme)
    bt.schedule("mixture", 2.0)
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


@pytest.mark.parametrize("scheme,factor", [("fine", 4.0), ("mixture", 8.0)])
def test_batch_bench_schedule_matches_oracle(ff, scheme, factor):
    """The schedules the benchmark's tuner picks for its 64-mixture batch (one launch per
    mixture on 16 branches; before that, fine frame buckets with grid share factor 4) on
    mixtures of the benchmark's frequency count range (F = 64) and frame range (T up to 2000):
    every mixture's log-likelihood after each iteration, its final parameters and its images
    against the oracle from the same start."""
    shapes = [(4, 7, 2000), (3, 6, 1650), (2, 5, 1210), (4, 5, 731), (3, 4, 203), (2, 3, 1999)]
    F, iters = 64, 3
    mixes, inits = [], []
    for b, (M, N, T) in enumerate(shapes):
        mix = synth.generate_mixture(M, N, F, T, 8, seed=5100 + b, keep_images=False)
        mixes.append(mix)
        inits.append(synth.random_init(mix.x, N, seed=5100 + b))
    xs = [torch.from_numpy(m.x).cuda() for m in mixes]
    bt = ff.Batch(xs, [N for _, N, _ in shapes])
    bt.schedule(scheme, factor)
    for b, init in enumerate(inits):
        bt.set_params(b, init.P, init.lam, init.v)
    lls = [bt.iterate(1)[0] for _ in range(iters)]      # the log-likelihood after each iteration
    for b, ((M, N, T), m, init) in enumerate(zip(shapes, mixes, inits)):
        ref = off.run(m.x, init.P, init.lam, init.v, iters=iters)
        for it in range(iters):
            tot = ref["ll"][:, it].sum()
            assert abs(lls[it][b] - tot) <= 1e-5 * abs(tot), (b, it, lls[it][b], tot)
        P, lam, v = bt.get_params(b)
        s2 = np.einsum("fmn,fnt->fmt", lam.astype(np.float64), v.astype(np.float64))
        s2_ref = np.einsum("fmn,fnt->fmt", ref["L"], ref["H"])
        assert np.allclose(s2, s2_ref, rtol=2e-3), b
        c = torch.empty((F, T, N, M), dtype=torch.complex64, device="cuda")
        bt.separate(b, c)
        torch.cuda.synchronize()
        cr = np.stack([off.separate_fast(m.x[f], ref["W"][f], ref["L"][f], ref["H"][f]) for f in range(F)])
        assert_images(c.cpu().numpy(), cr, 1e-4, f"mixture {b} (M={M}, N={N}, T={T})")
    bt.close()
