"""Host-side fault injection through the C ABI: inputs that make the model degenerate are
reported as FASTFCA_ENUMERIC, never returned as non-finite results, and a context recovers
once its parameters are replaced.

Nothing here faults the GPU: the planted values are ordinary floating-point data (NaN, Inf,
exact zeros) and every kernel loop is bounded by an iteration count.

* A NaN or Inf sample in x: the next iterations meet a non-finite sigma^2 or Q_m.
* A frame that is exactly zero: sigma^2 -> 0 raises the likelihood without bound (Eq. 25 has
  no maximiser there).  The EM updates (Algorithm 1, Eq. 12-13) keep that bin's power small
  but positive, and the complex128 oracle agrees with the kernels on them.  The multiplicative
  updates (Algorithm 2, Eq. 15-17, Eq. 53) set it to exactly zero, and the next evaluation
  of sigma^2 reports the failure; the oracle's log-likelihood is non-finite there too.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fastfca as off, fca as ofca  # noqa: E402
from paper_2101_08563_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

LL_TOL = 1e-5


@pytest.fixture(scope="module")
def ff():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2101_08563_gb300 import build, fastfca
    build.build()
    fastfca.load()
    return fastfca


# (model, M, N, F, T, bases, block): the frequency-resident kernels, the cluster kernel
# (M = 6, T beyond one CTA), the block input, full-rank FCA and FastMNMF
CASES = [
    ("fastfca", 3, 4, 3, 300, 0, 1),
    ("fastfca_mm", 3, 4, 3, 300, 0, 1),
    ("fastfca", 6, 4, 2, 2500, 0, 1),
    ("fastfca", 2, 3, 3, 400, 0, 4),
    ("fca", 3, 4, 2, 200, 0, 1),
    ("fca_mm", 2, 3, 2, 200, 0, 1),
    ("fastmnmf", 3, 4, 3, 300, 3, 1),
]


def case_id(c):
    return f"{c[0]}-M{c[1]}N{c[2]}T{c[4]}" + (f"B{c[6]}" if c[6] > 1 else "")


def mixture(M, N, F, T, seed):
    return synth.generate_mixture(M, N, F, T, 4, seed=seed).x


def make(ff, x, N, model, bases, block):
    return ff.Separator(torch.from_numpy(x).cuda(), N, model=model, bases=bases, block=block)


def set_start(sep, x, N, model, bases, block, seed):
    """A seeded start for the model (the same on every context it is given to)."""
    if model in ("fca", "fca_mm"):
        sep.set_params_fca(*synth.fca_random_init(x, N, seed=seed))
    elif model == "fastmnmf":
        st = synth.fastmnmf_random_init(x, N, bases, seed=seed)
        sep.set_params_mnmf(st.W, st.lam, np.ascontiguousarray(st.t.transpose(0, 2, 1)),
                            np.ascontiguousarray(st.v.transpose(2, 1, 0)))
    else:
        init = synth.random_init(x, N, seed=seed)
        v = init.v
        if block > 1:   # one column per block of B frames
            F, n_, T = v.shape
            v = np.ascontiguousarray(v.reshape(F, n_, T // block, block).mean(axis=3))
        sep.set_params(init.P, init.lam, v)


@pytest.mark.parametrize("bad", [np.nan, np.inf])
@pytest.mark.parametrize("case", CASES, ids=case_id)
def test_nonfinite_mixture_is_reported_and_recovered(ff, case, bad):
    model, M, N, F, T, K, B = case
    x = mixture(M, N, F, T, seed=31)
    x_bad = x.copy()
    x_bad[F - 1, 7, 0] = complex(bad, 0.0)
    sep = make(ff, x_bad, N, model, K, B)                 # default start, computed from x_bad
    with pytest.raises(ff.FastFCAError, match="ENUMERIC"):
        sep.iterate(3)
    # the parameters may now hold NaN: nothing runs on them until they are replaced
    with pytest.raises(ff.FastFCAError, match="set_params"):
        sep.iterate(1)
    with pytest.raises(ff.FastFCAError, match="ENUMERIC"):
        sep.loglik()
    with pytest.raises(ff.FastFCAError, match="ENUMERIC"):
        sep.separate()
    if model in ("fca", "fca_mm"):
        sep.get_params_fca()                              # inspection still works
    elif model == "fastmnmf":
        sep.get_params_mnmf()
    else:
        sep.get_params()
    # a clean mixture and a fresh start give exactly what a fresh context gives
    sep.set_mixture(torch.from_numpy(x).pin_memory())
    set_start(sep, x, N, model, K, B, seed=31)
    ll_r = sep.iterate(3)
    fresh = make(ff, x, N, model, K, B)
    set_start(fresh, x, N, model, K, B, seed=31)
    ll_f = fresh.iterate(3)
    assert np.all(np.isfinite(ll_r))
    assert np.array_equal(ll_r, ll_f)
    assert np.array_equal(sep.separate(), fresh.separate())
    sep.close()
    fresh.close()


def silent(x, t0):
    y = x.copy()
    y[:, t0, :] = 0
    return y


@pytest.mark.parametrize("M,N,F,T,block", [(3, 4, 3, 300, 1), (6, 4, 2, 2500, 1)],
                         ids=["resident", "cluster"])
def test_silent_frame_ip_em_matches_oracle(ff, M, N, F, T, block):
    """IP+EM on a mixture with an all-zero frame: finite, and at parity with the oracle."""
    x = silent(mixture(M, N, F, T, seed=32), 17)
    init = synth.random_init(x, N, seed=32)
    sep = make(ff, x, N, "fastfca", 0, block)
    sep.set_params(init.P, init.lam, init.v)
    ll = sep.iterate(4)
    c = sep.separate()
    sep.close()
    ref = off.run(x, init.P, init.lam, init.v, 4)["ll"].sum(axis=0)
    assert np.all(np.isfinite(ll)) and np.all(np.isfinite(c))
    assert np.max(np.abs(ll - ref) / np.abs(ref)) <= LL_TOL
    assert np.all(c[:, 17] == 0)                          # the filter maps a zero frame to zero


def test_silent_frame_fca_em_matches_oracle(ff):
    x = silent(mixture(3, 4, 2, 200, seed=33), 17)
    R0, h0 = synth.fca_random_init(x, 4, seed=33)
    sep = make(ff, x, 4, "fca", 0, 1)
    sep.set_params_fca(R0, h0)
    ll = sep.iterate(3)
    sep.close()
    ref = ofca.run(x, R0, h0, 3)["ll"].sum(axis=0)
    assert np.all(np.isfinite(ll))
    assert np.max(np.abs(ll - ref) / np.abs(ref)) <= LL_TOL


@pytest.mark.parametrize("model,M,N,F,T,K", [
    ("fastfca_mm", 3, 4, 3, 300, 0),
    ("fastfca_mm", 6, 4, 2, 2500, 0),
    ("fca_mm", 2, 3, 2, 200, 0),
    ("fastmnmf", 3, 4, 3, 300, 3),
], ids=["ipmm-resident", "ipmm-cluster", "fca-mm", "fastmnmf"])
def test_silent_frame_multiplicative_updates_report(ff, model, M, N, F, T, K):
    """The multiplicative updates zero the silent frame's power in iteration 1; the next
    evaluation of sigma^2 (the log-likelihood after it, else iteration 2) meets sigma^2 = 0 and
    reports ENUMERIC.  The oracle fails at the same point: its log-likelihood after iteration 1
    is NaN, or (full-rank FCA) the inverse of the singular covariance raises."""
    x = silent(mixture(M, N, F, T, seed=34), 17)
    sep = make(ff, x, N, model, K, 1)
    set_start(sep, x, N, model, K, 1, seed=34)
    with pytest.raises(ff.FastFCAError, match="ENUMERIC"):
        sep.iterate(2)
    sep.close()


def test_batch_reports_the_failed_mixture(ff):
    """A non-finite mixture in a batch: ENUMERIC, its log-likelihood non-finite, the others
    identical to a batch without it (mixtures are independent)."""
    xs = [mixture(3, 4, 3, 300, seed=40 + i) for i in range(3)]
    bad = [x.copy() for x in xs]
    bad[1][0, 5, 1] = np.nan
    inits = [synth.random_init(x, 4, seed=40 + i) for i, x in enumerate(xs)]
    clean = ff.Batch([torch.from_numpy(x).cuda() for x in xs], [4, 4, 4])
    faulty = ff.Batch([torch.from_numpy(x).cuda() for x in bad], [4, 4, 4])
    for i, p in enumerate(inits):
        clean.set_params(i, p.P, p.lam, p.v)
        faulty.set_params(i, p.P, p.lam, p.v)
    ll_c, _ = clean.iterate(3)
    with pytest.raises(ff.FastFCAError, match="ENUMERIC") as ei:
        faulty.iterate(3)
    ll_b = ei.value.ll_per_mixture
    assert not np.isfinite(ll_b[1])
    assert ll_b[0] == ll_c[0] and ll_b[2] == ll_c[2]
    clean.close()
    faulty.close()


# ------------------------------------------------------------------ forced allocation failure

def sweep_allocations(ff, make, limit=80):
    """Fails each device allocation that make() performs, in turn: every failure is ENOMEM and
    leaves the library's live-allocation count where it was.  Returns how many allocations a
    successful make() performs (the result of that call is closed)."""
    base = ff.live_allocations()
    for k in range(limit):
        ff.fail_allocation_after(k)
        try:
            obj = make()
        except ff.FastFCAError as e:
            assert "ENOMEM" in str(e), str(e)
            assert ff.live_allocations() == base, f"allocation {k}: leak"
            continue
        finally:
            ff.fail_allocation_after(-1)
        obj.close()
        assert ff.live_allocations() == base
        return k
    raise AssertionError(f"make() still failing after {limit} allocations")


@pytest.mark.parametrize("case", CASES, ids=case_id)
@pytest.mark.parametrize("host_x", [False, True], ids=["device-x", "host-x"])
def test_create_survives_every_failed_allocation(ff, case, host_x):
    model, M, N, F, T, K, B = case
    x = mixture(M, N, F, T, seed=50)
    xd = x if host_x else torch.from_numpy(x).cuda()
    n = sweep_allocations(ff, lambda: ff.Separator(xd, N, model=model, bases=K, block=B))
    assert n >= 5


def test_failed_allocations_in_use_leave_the_context_usable(ff):
    """Allocations a live context makes later (the history of iterate, the staging buffer of a
    host separation, the owned copy of set_mixture): ENOMEM, nothing leaked, and afterwards
    the context gives exactly what a context that never failed gives."""
    x = mixture(3, 4, 3, 300, seed=51)
    init = synth.random_init(x, 4, seed=51)
    ref = ff.Separator(torch.from_numpy(x).cuda(), 4)
    ref.set_params(init.P, init.lam, init.v)
    ll_ref = ref.iterate(4)
    c_ref = ref.separate()
    sep = ff.Separator(torch.from_numpy(x).cuda(), 4)
    sep.set_params(init.P, init.lam, init.v)
    base = ff.live_allocations()
    for k in (0, 1):                                   # history, then its totals
        ff.fail_allocation_after(k)
        with pytest.raises(ff.FastFCAError, match="ENOMEM"):
            sep.iterate(4)
        ff.fail_allocation_after(-1)
        assert ff.live_allocations() <= base + 1       # the history may keep its first buffer
    ff.fail_allocation_after(0)
    with pytest.raises(ff.FastFCAError, match="ENOMEM"):
        sep.set_mixture(x)                             # the owned copy
    ff.fail_allocation_after(-1)
    sep.set_params(init.P, init.lam, init.v)
    assert np.array_equal(sep.iterate(4), ll_ref)
    ff.fail_allocation_after(0)
    with pytest.raises(ff.FastFCAError, match="ENOMEM"):
        sep.separate()                                 # host output: the staging buffer
    ff.fail_allocation_after(-1)
    assert np.array_equal(sep.separate(), c_ref)
    sep.close()
    ref.close()


def batch_inputs(ff):
    shapes = [(3, 4, 3, 300), (2, 3, 2, 500), (4, 6, 2, 200)]
    xs = [mixture(M, N, F, T, seed=60 + i) for i, (M, N, F, T) in enumerate(shapes)]
    Ns = [s[1] for s in shapes]
    inits = [synth.random_init(x, n, seed=60 + i) for i, (x, n) in enumerate(zip(xs, Ns))]
    return xs, Ns, inits


def started_batch(ff, xs, Ns, inits):
    b = ff.Batch([torch.from_numpy(x).cuda() for x in xs], Ns)
    for i, p in enumerate(inits):
        b.set_params(i, p.P, p.lam, p.v)
    return b


def test_batch_create_survives_every_failed_allocation(ff):
    xs, Ns, _ = batch_inputs(ff)
    sweep_allocations(ff, lambda: ff.Batch(xs, Ns), limit=120)                    # host x
    xd = [torch.from_numpy(x).cuda() for x in xs]
    sweep_allocations(ff, lambda: ff.Batch(xd, Ns), limit=120)                    # device x


def test_batch_schedule_and_tune_survive_failed_allocations(ff):
    """A failed schedule or tune returns ENOMEM, frees what it allocated, puts the previous
    schedule and the parameters back, and the batch then iterates exactly as one that never
    failed."""
    xs, Ns, inits = batch_inputs(ff)
    ref = started_batch(ff, xs, Ns, inits)
    ll_ref, _ = ref.iterate(3)
    ref.close()
    b = started_batch(ff, xs, Ns, inits)
    params = [b.get_params(i) for i in range(len(xs))]
    base = ff.live_allocations()
    for k in range(4):
        ff.fail_allocation_after(k)
        with pytest.raises(ff.FastFCAError, match="ENOMEM"):
            b.schedule(2, 2.0)
        ff.fail_allocation_after(-1)
        assert ff.live_allocations() == base
    failures = 0
    for k in range(200):
        ff.fail_allocation_after(k)
        try:
            b.tune(1)
        except ff.FastFCAError as e:
            assert "ENOMEM" in str(e), str(e)
            failures += 1
        else:
            break
        finally:
            ff.fail_allocation_after(-1)
        assert ff.live_allocations() == base, f"tune, allocation {k}: leak"
        for i in range(len(xs)):
            for a, p in zip(b.get_params(i), params[i]):
                assert np.array_equal(a, p), f"tune, allocation {k}: parameters changed"
    assert failures > 9          # the snapshot and the classes of several probes
    b.schedule(0, 1.0)           # the schedule the reference batch ran
    for i, p in enumerate(inits):
        b.set_params(i, p.P, p.lam, p.v)
    ll, _ = b.iterate(3)
    assert np.array_equal(ll, ll_ref)
    b.close()


def test_net_create_survives_every_failed_allocation(ff):
    from paper_2101_08563_gb300 import learned as L
    n = sweep_allocations(ff, lambda: L.InitNet(3, 4, max_rows=64, max_T=256, seed=1))
    assert n >= 15


def test_cluster_exchange_timeout_is_reported_and_a_fresh_context_works(ff):
    """The cluster kernel's one wait on other CTAs (each source's exchange in the n-loop) made
    to run out: with the limit set to one non-blocking poll, an exchange that is not complete
    at the first poll is reported (status bit -> ECUDA, and the context stays failed).  The
    kernel then waits, bounded, for the bytes already sent, so nothing is left in flight; a
    context created after the limit is restored computes what the oracle computes."""
    M, N, F, T = 8, 12, 2, 2003                   # clusters of four CTAs
    mix = synth.generate_mixture(M, N, F, T, 8, seed=71, array="circular", spacing=0.05)
    init = synth.random_init(mix.x, N, seed=71)
    xd = torch.from_numpy(mix.x).cuda()
    ff.large_bin_kernel("cluster")
    try:
        ff.cluster_wait_limit(1)
        sep = ff.Separator(xd, N)
        sep.set_params(init.P, init.lam, init.v)
        with pytest.raises(ff.FastFCAError, match="ECUDA") as e:
            sep.iterate(2)
        assert "timed out" in str(e.value)
        with pytest.raises(ff.FastFCAError, match="ECUDA"):
            sep.iterate(1)                          # failed for good
        sep.close()
        ff.cluster_wait_limit(0)
        fresh = ff.Separator(xd, N)
        fresh.set_params(init.P, init.lam, init.v)
        ll = fresh.iterate(2)
        fresh.close()
    finally:
        ff.cluster_wait_limit(0)
        ff.large_bin_kernel("auto")
    ref = off.run(mix.x, init.P, init.lam, init.v, iters=2)
    ll_ref = ref["ll"].sum(axis=0)
    assert np.all(np.abs(ll - ll_ref) <= LL_TOL * np.abs(ll_ref)), (ll, ll_ref)
