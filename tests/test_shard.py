"""One mixture split over ranks by contiguous frequency ranges (FastFCA's frequencies are
independent, Sec. IV-G), on CPU ranks (gloo, world size 2): each rank runs its own range,
with the complex128 oracle standing in for the kernel, and one FP64 all-reduce per call
gives the whole mixture's log-likelihood.  It must equal the oracle's on the whole mixture."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

from paper_2101_08563_gb300 import shard  # noqa: E402


@pytest.mark.parametrize("F,world", [(1, 1), (7, 2), (8, 2), (1025, 8), (5, 8), (513, 3)])
def test_frequency_ranges_partition_the_band(F, world):
    rs = shard.frequency_ranges(F, world)
    assert len(rs) == world and rs[0][0] == 0 and rs[-1][1] == F
    assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))            # contiguous, no gap
    sizes = [f1 - f0 for f0, f1 in rs]
    assert max(sizes) - min(sizes) <= 1 and sum(sizes) == F


def _mixture():
    from paper_2101_08563_gb300 import synth
    mix = synth.generate_mixture(2, 3, 7, 60, 4, seed=81)
    init = synth.random_init(mix.x, 3, seed=81)
    return mix.x, init


class OracleRange:
    """The oracle on frequencies [f0, f1) of a mixture, keeping its state between calls."""

    def __init__(self, x, init, f0, f1):
        from oracle import fastfca as off
        self.off = off
        self.x = x[f0:f1]
        self.W, self.L, self.H = init.P[f0:f1].copy(), init.lam[f0:f1].astype(np.float64), init.v[f0:f1].astype(np.float64)

    def iterate(self, n):
        out = self.off.run(self.x, self.W, self.L, self.H, iters=n)
        self.W, self.L, self.H = np.stack(out["W"]), np.stack(out["L"]), np.stack(out["H"])
        return out["ll"].sum(axis=0)

    def loglik(self):
        off = self.off
        return sum(off.loglik(off.Xhat_from_x(self.x[i]), self.W[i], self.L[i], self.H[i]) for i in range(len(self.x)))


def _rank_main(rank, world, port, out_dir):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x, init = _mixture()
    f0, f1 = shard.frequency_ranges(x.shape[0], world)[rank]
    s = shard.FrequencyShard(OracleRange(x, init, f0, f1), x.shape[0], rank, world)
    ll = np.concatenate([s.iterate(2), s.iterate(1)])
    tot = s.loglik()
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.append(ll, tot))
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def test_sharded_log_likelihood_equals_the_whole_mixture(tmp_path):
    world = 2
    port = _free_port()
    ctx = torch.multiprocessing.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    from oracle import fastfca as off
    x, init = _mixture()
    ref = off.run(x, init.P, init.lam, init.v, iters=3)
    want = np.append(ref["ll"].sum(axis=0), None)
    whole_final = sum(off.loglik(off.Xhat_from_x(x[f]), ref["W"][f], ref["L"][f], ref["H"][f]) for f in range(x.shape[0]))
    want[-1] = whole_final
    for r in range(world):
        got = np.load(tmp_path / f"rank{r}.npy")
        assert np.allclose(got, want.astype(np.float64), rtol=1e-12, atol=0), (r, got, want)
