"""Benchmark: FastFCA IP+EM throughput (time-frequency-bin iterations per second) on GB300.

One step = one complete FastFCA run on the M=4, N=6, F=513, T=1250 workload (100 IP+EM
iterations, Algorithm 1, then the Wiener-filter separation of Eq. 39), starting from the
seeded random initialisation, through the library's C ABI.  The metric counts F*T*iters
bin-iterations per step.  Inputs are model-generated (synthetic) and resident in HBM when a
timed step starts; L2 is flushed (a 512 MiB write) between steps, outside the timed spans.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank separates its own mixture (independent problems, no data
collective): weak scaling, value = all ranks' bin-iterations / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2101_08563_gb300 import synth  # noqa: E402

WORKLOAD = synth.WORKLOADS["fca_cmp"]
MNMF_K = 8            # FastMNMF bases per source on the bench mixture (its generator's K)
MNMF_ITERS = 20


def mnmf_abi_params(st):
    """A FastMNMF start in the C ABI's layouts: t (F, N, K), v (N, K, T)."""
    return (st.W, st.lam, np.ascontiguousarray(st.t.transpose(0, 2, 1)),
            np.ascontiguousarray(st.v.transpose(2, 1, 0)))
METRIC = "FastFCA EM TF-bin-iters/s"
UNIT = "bin-iters/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP32 arithmetic peak from unit counts and the maximum clock: 152 SMs x 128 FP32 lanes x
# 2 flop (FMA) x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def algorithmic_flops_per_bin_iter(M: int, N: int) -> float:
    """FP32 flops one bin-iteration of Algorithm 1 needs (excluding the per-frequency IP):
    Q accumulation 6*M(M+1)/2 + 4*M*M(M+1)/2, decorrelation 8M^2, U 3M, NMF EM 13*M*N,
    log-likelihood terms 4M."""
    tri = M * (M + 1) / 2
    return 6 * tri + 4 * M * tri + 8 * M * M + 3 * M + 13 * M * N + 4 * M


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle timing
_WORKER_STATE = {}


def _pool_init(seed_index):
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    w = WORKLOAD
    mix = synth.workload_mixture(w, seed_index)
    init = synth.random_init(mix.x, w.N, seed=w.seed + seed_index)
    _WORKER_STATE["x"] = mix.x
    _WORKER_STATE["init"] = init


def _noop(_):
    return 0


def _oracle_worker(args):
    """Algorithm 1 (with the per-iteration log-likelihood) and Eq. 39 on a list of
    frequencies of the workload mixture held by this worker process."""
    freqs, iters = args
    from oracle import fastfca as off
    x, init = _WORKER_STATE["x"], _WORKER_STATE["init"]
    out = off.run(x, init.P, init.lam, init.v, iters=iters, freqs=freqs, with_ll=True)
    for i, f in enumerate(out["freqs"]):
        off.separate_fast(x[f], out["W"][i], out["L"][i], out["H"][i])
    return len(freqs)


class OraclePool:
    """Spawned worker processes, each holding the workload mixture (generated at start-up,
    outside any timed span); `run` times the oracle over frequencies split across them."""

    def __init__(self, workers, seed_index=0):
        import multiprocessing as mp
        self.workers = workers
        self.pool = mp.get_context("spawn").Pool(workers, initializer=_pool_init, initargs=(seed_index,))
        self.pool.map(_noop, range(workers))

    def run(self, freqs, iters):
        chunks = [c for c in (freqs[i::self.workers] for i in range(self.workers)) if c]
        t0 = time.perf_counter()
        self.pool.map(_oracle_worker, [(c, iters) for c in chunks], chunksize=1)
        return time.perf_counter() - t0, len(chunks)

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline():
    """The oracle on the whole workload (every frequency, all iterations, separation) across
    the host's cores."""
    w = WORKLOAD
    cores = os.cpu_count() or 1
    pool = OraclePool(cores)
    try:
        wall, used = pool.run(list(range(w.F)), w.iters)
    finally:
        pool.close()
    sample = (f"whole workload: {w.F} frequencies x {w.iters} iterations (+ log-likelihood each "
              f"iteration) + separation, split over {used} processes")
    # the same oracle on one core, on a sample of frequencies (each frequency costs the same)
    n1 = 16
    pool1 = OraclePool(1)
    try:
        wall1, _ = pool1.run(list(range(n1)), w.iters)
    finally:
        pool1.close()
    return {"value": w.F * w.T * w.iters / wall, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": sample, "seconds": round(wall, 3),
            "single_core": {"value": n1 * w.T * w.iters / wall1, "unit": UNIT, "cores": 1,
                            "sample": f"{n1} of the {w.F} frequencies x {w.iters} iterations, one process",
                            "seconds": round(wall1, 3)}}


# ----------------------------------------------------------------------------- batch workload
BATCH_B, BATCH_F, BATCH_ITERS, BATCH_SEED = 64, 513, 20, 3000


def batch_shapes():
    """The mixed-shape batch: M in {2,3,4}, N in M+1..M+3, T uniform in [200, 2000]."""
    rng = np.random.Generator(np.random.PCG64(BATCH_SEED))
    out = []
    for b in range(BATCH_B):
        M = int(rng.integers(2, 5))
        N = int(rng.integers(M + 1, M + 4))
        T = int(rng.integers(200, 2001))
        out.append((M, N, T))
    return out


def _gen_batch_item(args):
    b, M, N, T = args
    mix = synth.generate_mixture(M, N, BATCH_F, T, 8, seed=BATCH_SEED + b)
    init = synth.random_init(mix.x, N, seed=BATCH_SEED + b)
    return mix.x, init.P, init.lam, init.v


def generate_batch():
    import multiprocessing as mp
    shapes = batch_shapes()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        data = pool.map(_gen_batch_item, [(b, M, N, T) for b, (M, N, T) in enumerate(shapes)])
    return shapes, data


def run_batch(shapes, data, dev, stream, clocks_ok=True):
    import torch
    from paper_2101_08563_gb300 import fastfca
    xs = [torch.from_numpy(d[0]).to(dev) for d in data]
    inits = [(torch.from_numpy(d[1]).to(dev), torch.from_numpy(d[2]).to(dev), torch.from_numpy(d[3]).to(dev))
             for d in data]
    bt = fastfca.Batch(xs, [N for _, N, _ in shapes], stream=stream.cuda_stream)

    def reset():
        for b, (P, lam, v) in enumerate(inits):
            bt.set_params(b, P, lam, v)

    reset()
    scheme, factor = bt.tune(3)
    for _ in range(3):
        reset()
        bt.iterate(BATCH_ITERS, stats=False)
    torch.cuda.synchronize()
    units = sum(BATCH_F * T for _, _, T in shapes) * BATCH_ITERS
    times, secs = [], []
    for _ in range(5):
        reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bt.iterate(BATCH_ITERS, stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        _, sec = bt.iterate(BATCH_ITERS, stats=True)     # per-mixture spans (stamps)
        secs.append(sec)
    bt.close()
    sec = np.median(np.array(secs), axis=0)
    ms = float(np.median(times))
    return {"value": units / (ms * 1e-3), "unit": UNIT, "mixtures": BATCH_B, "iters": BATCH_ITERS,
            "ms_per_launch": ms, "per_mixture_ms_p50": float(np.percentile(sec, 50) * 1e3),
            "per_mixture_ms_p99": float(np.percentile(sec, 99) * 1e3),
            "schedule": {"bucketing": scheme, "grid_factor": factor},
            "config": "M in {2,3,4}, N in M+1..M+3, F=513, T uniform [200,2000], one CUDA-graph launch"}


# ----------------------------------------------------------------------------- GPU arm
def run_learned(n_train):
    """The learned initialiser end to end on the GPU: n_train generated mixtures of the
    learned-initialiser workload with 200-iteration FastFCA targets, 6 epochs of training, and
    the comparison with the default start on 512 held-out mixtures (batched as one context)."""
    import torch
    from paper_2101_08563_gb300 import learned as L
    w = synth.WORKLOADS["learned"]
    data, t_data = L.make_training_set(n_train, w.F, w.T, w.M, w.N, w.K, w.spacing, seed=w.seed, iters=w.iters)
    n_eval = 512
    net = L.InitNet(w.M, w.N, max_rows=n_eval * w.F, max_T=w.T, seed=w.seed + 1)
    loss0 = L.mean_loss(net, data)
    hist, t_train = L.train(net, data, epochs=6, batch=2048, lr=1e-3, seed=w.seed)
    loss1 = L.mean_loss(net, data)
    del data
    torch.cuda.empty_cache()
    res = L.evaluate(net, n_eval, w.F, w.T, w.M, w.N, w.K, w.spacing, seed=(0xFFFF << 32) + w.seed, iters=w.iters)
    net.close()
    res.update({"workload": w.name, "train_mixtures": n_train, "target_iters": w.iters,
                "train_data_seconds": t_data, "train_seconds": t_train, "epochs": 6, "batch_rows": 2048,
                "loss_untrained": loss0, "loss_trained": loss1,
                "held_out": "512 mixtures, generator key disjoint from the training keys",
                "reference_ll": "default start after 200 iterations (GPU FastFCA, oracle-parity tested)"})
    return res


def separation_roofline(w, sep_ms, peaks):
    """The Wiener separation (W^{-H} per frequency + Eq. 39 filter) of one step as an HBM-bound
    kernel: algorithmic bytes x (8 M) + v (4 N) read and c (8 N M) written per bin, over its
    event-timed span inside the step (it follows the IP+EM launch, so x and v may still be
    partly in L2)."""
    per_bin = 8 * w.M + 4 * w.N + 8 * w.N * w.M
    bytes_ = per_bin * w.F * w.T
    ms = statistics.mean(sep_ms)
    hbm = peaks.get("hbm_gbs")
    gbs = bytes_ / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "bst_to_winv_kernel + fastfca_mwf_kernel", "achieved": gbs,
            "peak": hbm, "unit": "GB/s", "frac": (gbs / hbm) if hbm else None,
            "bytes_per_bin": per_bin, "ms": ms,
            "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}


def run_large(peaks):
    """The large single instance (M=8 circular, N=12, F=1025, T=4000, K=16, 50 iterations)
    on the cluster kernel: IP+EM launch throughput (event-timed, L2 flushed between steps)
    and the Wiener separation's HBM bandwidth (x and v read, 3.15 GB of images written)."""
    import torch
    from paper_2101_08563_gb300 import fastfca
    w = synth.WORKLOADS["large"]
    mix = synth.workload_mixture(w)
    init = synth.random_init(mix.x, w.N, seed=w.seed)
    x = torch.from_numpy(mix.x).cuda()
    P0, lam0, v0 = (torch.from_numpy(a).cuda() for a in (init.P, init.lam, init.v))
    c = torch.empty((w.F, w.T, w.N, w.M), dtype=torch.complex64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    sep = fastfca.Separator(x, w.N)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    em_ms, mwf_ms = [], []
    for rep in range(4):
        sep.set_params(P0, lam0, v0)
        flush.zero_()
        torch.cuda.synchronize()
        ev[0].record()
        sep.iterate(w.iters, return_ll=False)
        ev[1].record()
        sep.separate(c)
        ev[2].record()
        torch.cuda.synchronize()
        if rep > 0:                                   # the first is a warm-up
            em_ms.append(ev[0].elapsed_time(ev[1]))
            mwf_ms.append(ev[1].elapsed_time(ev[2]))
    ll_em = float(sep.loglik()) / (w.F * w.T)
    sep.close()
    # the same start and iterations by IP+MM (Algorithm 2) on the same cluster kernel
    msep = fastfca.Separator(x, w.N, model="fastfca_mm")
    mm_ms = []
    for rep in range(3):
        msep.set_params(P0, lam0, v0)
        flush.zero_()
        torch.cuda.synchronize()
        ev[0].record()
        msep.iterate(w.iters, return_ll=False)
        ev[1].record()
        torch.cuda.synchronize()
        if rep > 0:
            mm_ms.append(ev[0].elapsed_time(ev[1]))
    ll_mm = float(msep.loglik()) / (w.F * w.T)
    msep.close()
    em = statistics.mean(em_ms)
    mwf = statistics.mean(mwf_ms)
    mm = statistics.mean(mm_ms)
    flops = algorithmic_flops_per_bin_iter(w.M, w.N) * w.F * w.T * w.iters
    mwf_bytes = x.numel() * 8 + v0.numel() * 4 + c.numel() * 8
    hbm = peaks.get("hbm_gbs")
    return {
        "workload": w.name, "metric": METRIC, "value": w.F * w.T * w.iters / (em * 1e-3), "unit": UNIT,
        "iters": w.iters, "em_launch_ms": em, "kernel": "fastfca_em_cluster_kernel<8> (clusters of 8 CTAs)",
        "roofline": {"bound": "alu", "achieved": flops / (em * 1e-3) / 1e12, "peak": FP32_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": flops / (em * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                     "flops_per_bin_iter": algorithmic_flops_per_bin_iter(w.M, w.N)},
        "separation": {"kernel": "fastfca_mwf_wide_kernel<8>", "ms": mwf, "bytes": mwf_bytes,
                       "achieved_gbs": mwf_bytes / (mwf * 1e-3) / 1e9,
                       "frac_of_measured_hbm": (mwf_bytes / (mwf * 1e-3) / 1e9 / hbm) if hbm else None},
        "l2": "flushed before each step (512 MiB write, untimed)",
        "loglik_per_bin": ll_em,
        "ip_mm": {"algorithm": "IP+MM (Algorithm 2), same start and iterations", "launch_ms": mm,
                  "value": w.F * w.T * w.iters / (mm * 1e-3), "unit": UNIT, "loglik_per_bin": ll_mm},
    }


def precision_report():
    """Error of every output of the CUDA path against the FP64 oracle from the same start:
    the whole small workload (M=2, N=3, F=257, T=250, 20 iterations) and four frequencies of
    the bench workload (100 iterations).  Images c and log-likelihood per iteration are
    compared directly; the parameters through W (fixed scale: the IP normalises it) and the
    scale-free sigma^2 = LH and per-source powers L[:, n] H[n, :]."""
    import torch
    from oracle import fastfca as off
    from paper_2101_08563_gb300 import fastfca
    out = {}
    for name, freqs in (("small", None), ("fca_cmp", [3, 130, 257, 511])):
        w = synth.WORKLOADS[name]
        mix = synth.workload_mixture(w)
        init = synth.random_init(mix.x, w.N, seed=w.seed)
        fs = list(range(w.F)) if freqs is None else freqs
        x = np.ascontiguousarray(mix.x[fs])
        sep = fastfca.Separator(torch.from_numpy(x).cuda(), w.N)
        sep.set_params(np.ascontiguousarray(init.P[fs]), np.ascontiguousarray(init.lam[fs]),
                       np.ascontiguousarray(init.v[fs]))
        ll = sep.iterate(w.iters)
        c = sep.separate()
        P, lam, v = sep.get_params()
        sep.close()
        ref = off.run(x, init.P[fs], init.lam[fs], init.v[fs], iters=w.iters)
        ll_ref = ref["ll"].sum(axis=0)
        cr = np.stack([off.separate_fast(x[i], ref["W"][i], ref["L"][i], ref["H"][i]) for i in range(len(fs))])
        s2 = np.einsum("fmn,fnt->fmt", lam.astype(np.float64), v.astype(np.float64))
        s2r = np.einsum("fmn,fnt->fmt", ref["L"], ref["H"])
        pw = lam.astype(np.float64)[:, :, :, None] * v.astype(np.float64)[:, None, :, :]
        pwr = ref["L"][:, :, :, None] * ref["H"][:, None, :, :]
        out[name] = {
            "frequencies": "all" if freqs is None else freqs, "iters": w.iters,
            "loglik_rel_err_max": float(np.max(np.abs(ll - ll_ref) / np.abs(ll_ref))),
            "images_rel_err": float(np.linalg.norm(c - cr) / np.linalg.norm(cr)),
            "W_rel_err": float(np.max(np.abs(P - ref["W"])) / np.max(np.abs(ref["W"]))),
            "sigma2_rel_err_max": float(np.max(np.abs(s2 - s2r) / s2r)),
            "source_power_rel_err_median": float(np.median(np.abs(pw - pwr) / pwr)),
            "tolerance": {"loglik": 1e-5, "images": 1e-4},
        }
    return out


def load_peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except Exception:
        return {}


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_2101_08563_gb300 import build, fastfca

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = WORKLOAD
    mix = synth.workload_mixture(w, rank)
    init = synth.random_init(mix.x, w.N, seed=w.seed + rank)
    build.build()
    x = torch.from_numpy(mix.x).to(dev)
    P0 = torch.from_numpy(init.P).to(dev)
    lam0 = torch.from_numpy(init.lam).to(dev)
    v0 = torch.from_numpy(init.v).to(dev)
    c = torch.empty((w.F, w.T, w.N, w.M), dtype=torch.complex64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sep = fastfca.Separator(x, w.N, stream=stream.cuda_stream)

    def step():
        sep.set_params(P0, lam0, v0)
        sep.iterate(w.iters, return_ll=False)
        sep.separate(c)

    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()

    # per-launch timing of the dominant kernel (the fused IP+EM launch) inside each step
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    mids = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):
        flush.zero_()
        sep.set_params(P0, lam0, v0)
        starts[i].record(stream)
        sep.iterate(w.iters, return_ll=False)
        mids[i].record(stream)
        sep.separate(c)
        ends[i].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clock_info = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    em_ms = [s.elapsed_time(m) for s, m in zip(starts, mids)]
    sep_ms = [m.elapsed_time(e) for m, e in zip(mids, ends)]
    # the set_params copies are outside the event spans; one step is iterate + separate
    units = w.F * w.T * w.iters
    value = weak_scaling_value(units * args.steps, sum(step_ms) * 1e-3, world, dev)
    tot_ms = world * units * args.steps / value * 1e3          # the max over ranks

    # the same model fitted by IP+MM (Algorithm 2) on the same mixture and start, for the
    # paper's iteration count (20, Table I): time per launch and the log-likelihood reached,
    # beside IP+EM's after as many iterations.  (Run longer on this mixture, IP+MM reaches a
    # point where a decorrelated channel and its model variance vanish together at one frame
    # and the likelihood has no upper bound; the FP64 oracle does the same.)
    mm_iters = 20
    msep = fastfca.Separator(x, w.N, model="fastfca_mm", stream=stream.cuda_stream)
    msep.set_params(P0, lam0, v0)
    msep.iterate(2, return_ll=False)
    mm_ms = []
    for _ in range(3):
        flush.zero_()
        msep.set_params(P0, lam0, v0)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        msep.iterate(mm_iters, return_ll=False)
        a1.record(stream)
        torch.cuda.synchronize()
        mm_ms.append(a0.elapsed_time(a1))
    msep.set_params(P0, lam0, v0)
    mm_ll = float(msep.iterate(mm_iters)[-1])
    msep.close()
    sep.set_params(P0, lam0, v0)
    em_ll_same = float(sep.iterate(mm_iters)[-1])
    em_ms_same = []
    for _ in range(3):
        flush.zero_()
        sep.set_params(P0, lam0, v0)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        sep.iterate(mm_iters, return_ll=False)
        a1.record(stream)
        torch.cuda.synchronize()
        em_ms_same.append(a0.elapsed_time(a1))

    # piecewise-stationary input (Sec. VI-B): the same mixture in blocks of 5 frames (250 blocks), the
    # default start of a block context, the bench's iterations
    blk = 5
    bsep = fastfca.Separator(x, w.N, stream=stream.cuda_stream, block=blk, seed=w.seed)
    Pb, lamb, vb = bsep.get_params()
    Pb, lamb, vb = (torch.from_numpy(a).to(dev) for a in (Pb, lamb, vb))
    bsep.iterate(2, return_ll=False)
    blk_ms = []
    for _ in range(3):
        flush.zero_()
        bsep.set_params(Pb, lamb, vb)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        bsep.iterate(w.iters, return_ll=False)
        a1.record(stream)
        torch.cuda.synchronize()
        blk_ms.append(a0.elapsed_time(a1))
    bsep.close()

    # FCA comparison path on the same GPU (fewer iterations: it is ~an order slower)
    fca_iters = 10
    R0, h0 = synth.fca_random_init(mix.x, w.N, seed=w.seed + rank)
    R0d = torch.from_numpy(R0).to(dev)
    h0d = torch.from_numpy(h0).to(dev)
    fca_ms, fca_ll = {}, {}
    for model in ("fca", "fca_mm"):      # EM (Eq. 12-13) and MM (Eq. 15-17)
        fsep = fastfca.Separator(x, w.N, model=model, stream=stream.cuda_stream)
        fsep.set_params_fca(R0d, h0d)
        fsep.iterate(2, return_ll=False)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        fsep.set_params_fca(R0d, h0d)
        f0.record(stream)
        fsep.iterate(fca_iters, return_ll=False)
        f1.record(stream)
        torch.cuda.synchronize()
        fca_ms[model] = f0.elapsed_time(f1)
        fca_ll[model] = float(fsep.loglik()) / (w.F * w.T)
        fsep.close()

    # FastMNMF (App. C) on the same mixture, K bases per source, from the same kind of start
    st = synth.fastmnmf_random_init(mix.x, w.N, MNMF_K, seed=w.seed + rank)
    mparams = [torch.from_numpy(a).to(dev) for a in mnmf_abi_params(st)]
    mnsep = fastfca.Separator(x, w.N, model="fastmnmf", bases=MNMF_K, stream=stream.cuda_stream)
    mnsep.set_params_mnmf(*mparams)
    mnsep.iterate(2, return_ll=False)
    mn_ms = []
    for _ in range(3):
        flush.zero_()
        mnsep.set_params_mnmf(*mparams)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        mnsep.iterate(MNMF_ITERS, return_ll=False)
        a1.record(stream)
        torch.cuda.synchronize()
        mn_ms.append(a0.elapsed_time(a1))
    mn_ll = float(mnsep.loglik()) / (w.F * w.T)
    mnsep.close()

    # end-to-end through the public API with host buffers (pinned), copies inside the span:
    # every step uploads its mixture and start, runs the iterations (reading back the
    # log-likelihood per iteration) and downloads the images.  Two long-lived contexts on two
    # streams take the steps in turn, so one step's copies overlap the other's kernels.
    x_h = torch.from_numpy(mix.x).pin_memory()
    P_h = torch.from_numpy(init.P).pin_memory()
    lam_h = torch.from_numpy(init.lam).pin_memory()
    v_h = torch.from_numpy(init.v).pin_memory()
    c_hs = [torch.empty((w.F, w.T, w.N, w.M), dtype=torch.complex64).pin_memory() for _ in range(2)]
    ll_hs = [torch.empty(w.iters, dtype=torch.float64).pin_memory() for _ in range(2)]
    e2e_streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
    ctxs = [fastfca.Separator(x_h, w.N, stream=st.cuda_stream) for st in e2e_streams]
    e2e_steps = max(4, min(args.steps, 10))

    def e2e_step(i):
        s = ctxs[i % 2]
        s.sync()                         # this context's previous step has landed on the host
        s.set_mixture(x_h)
        s.set_params(P_h, lam_h, v_h)
        s.iterate_async(w.iters, ll_hs[i % 2])
        s.separate_async(c_hs[i % 2])
        return ll_hs[i % 2]

    e2e_step(0)
    e2e_step(1)
    for s_ in ctxs:
        s_.sync()
    # three windows of e2e_steps steps; the median is reported.  The leg is host-bound and the
    # host is shared, so one window alone can catch a stall of the host's own.
    e2e_windows = []
    for _ in range(3):
        barrier(world)
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            ll = e2e_step(i)
        for s_ in ctxs:
            s_.sync()
        e2e_windows.append(weak_scaling_value(units * e2e_steps, time.perf_counter() - t0, world, dev))
    e2e_value = statistics.median(e2e_windows)
    h2d = mix.x.nbytes + init.P.nbytes + init.lam.nbytes + init.v.nbytes
    d2h = c_hs[0].numel() * 8 + w.iters * 8
    for s_ in ctxs:
        s_.close()
    sep.close()
    return {
        "value": value, "ms_per_step": tot_ms / args.steps, "em_ms": em_ms, "step_ms": step_ms, "sep_ms": sep_ms,
        "clocks": clock_info, "fca_ms": fca_ms, "fca_ll": fca_ll, "fca_iters": fca_iters, "mn_ms": mn_ms,
        "mn_ll": mn_ll, "mm_ms": mm_ms, "mm_ll": mm_ll,
        "mm_iters": mm_iters, "em_ll_same": em_ll_same, "em_ms_same": em_ms_same, "blk": blk, "blk_ms": blk_ms,
        "e2e_value": e2e_value, "e2e_windows": e2e_windows, "e2e_steps": e2e_steps, "h2d": h2d, "d2h": d2h,
        "final_ll": float(ll[-1].item() if hasattr(ll[-1], "item") else ll[-1]),
    }


def run_profile_case(F, iters, workload="fca_cmp", model="fastfca", separate=False):
    """A workload's first 8 frequencies tiled to F (so the launch has F frequencies of the
    workload's shape), two launches of the IP+EM kernel (model "fastfca_mm": IP+MM): 2
    iterations, then `iters`.
    workload "fastmnmf": the full M=4 N=6 K=8 F=513 T=1250 mixture, FastMNMF, 2 iterations
    then `iters` (each iteration one fastmnmf_freq_kernel and one fastmnmf_v_kernel launch)."""
    import torch
    from paper_2101_08563_gb300 import build, fastfca
    if workload == "fastmnmf":
        w = WORKLOAD
        mix = synth.workload_mixture(w)
        st = synth.fastmnmf_random_init(mix.x, w.N, MNMF_K, seed=w.seed)
        build.build()
        sep = fastfca.Separator(torch.from_numpy(mix.x).cuda(), w.N, model="fastmnmf", bases=MNMF_K)
        params = mnmf_abi_params(st)
        for n in (2, iters):
            sep.set_params_mnmf(*params)
            sep.iterate(n, return_ll=False)
        torch.cuda.synchronize()
        sep.close()
        print("profile case done")
        return
    w = synth.WORKLOADS[workload]
    mix = synth.generate_mixture(w.M, w.N, 8, w.T, w.K, seed=w.seed, array=w.array, spacing=w.spacing,
                                 keep_images=False)
    x = np.tile(mix.x, (F // 8 + 1, 1, 1))[:F].copy()
    init = synth.random_init(x, w.N, seed=w.seed)
    build.build()
    sep = fastfca.Separator(torch.from_numpy(x).cuda(), w.N, model=model)
    sep.set_params(init.P, init.lam, init.v)
    sep.iterate(2, return_ll=False)
    sep.set_params(init.P, init.lam, init.v)
    sep.iterate(iters, return_ll=False)
    if separate:                          # two separations into a device buffer
        out = torch.empty((F, w.T, w.N, w.M), dtype=torch.complex64, device="cuda")
        for _ in range(2):
            sep.separate(out)
    torch.cuda.synchronize()
    sep.close()
    print("profile case done")


def em_traffic():
    """DRAM bytes per bench launch of the IP+EM kernel from the committed ncu capture, or None
    when the kernel source changed since that capture."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(prof))["fastfca_em_kernel"]
        csrc = os.path.join(ROOT, "paper_2101_08563_gb300", "csrc")
        src = b"".join(open(os.path.join(csrc, f), "rb").read() for f in ("fastfca_em.cuh", "common.cuh"))
        if hashlib.sha1(src).hexdigest() != rec["source_sha1"]:
            return None
        return rec["bytes_per_launch"]
    except Exception:
        return None


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def weak_scaling_value(units_per_rank, local_seconds, world, dev):
    """Whole-job throughput of independent per-rank problems: every rank processed
    units_per_rank, the job took the slowest rank's time (max over ranks)."""
    return world * units_per_rank / allreduce_max(local_seconds, world, dev)


def allreduce_max(v, world, dev):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--learned-mixtures", type=int, default=20000)
    ap.add_argument("--profile", action="store_true",
                    help="only run the IP+EM kernel on the bench mixture's first frequencies tiled to "
                         "--profile-F, once untimed then once with --profile-iters iterations (for ncu)")
    ap.add_argument("--profile-F", type=int, default=608)
    ap.add_argument("--profile-iters", type=int, default=5)
    ap.add_argument("--profile-separate", action="store_true",
                    help="with --profile: end with two separations (the Wiener filter kernels)")
    ap.add_argument("--profile-model", default="fastfca", choices=["fastfca", "fastfca_mm"])
    ap.add_argument("--profile-workload", default="fca_cmp", choices=["fca_cmp", "large", "fastmnmf"])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    w = WORKLOAD
    config = {"workload": w.name, "M": w.M, "N": w.N, "F": w.F, "T": w.T, "iters": w.iters,
              "K_nmf": w.K, "array": f"{w.array} {w.spacing * 100:.0f} cm",
              "step": "IP+EM x iters + Wiener separation, from the seeded init",
              "l2": "flushed between steps (512 MiB write, untimed)"}

    if args.profile:
        run_profile_case(args.profile_F, args.profile_iters, args.profile_workload, args.profile_model,
                         args.profile_separate)
        return

    if args.impl == "reference":
        if rank != 0:
            return
        cores = os.cpu_count() or 1
        freqs = list(range(0, w.F, max(1, w.F // (2 * cores))))[: 2 * cores]
        iters = 25
        pool = OraclePool(cores)
        try:
            for _ in range(args.warmup):
                pool.run(freqs, iters)
            times = []
            for _ in range(args.steps):
                wall, used = pool.run(freqs, iters)
                times.append(wall)
        finally:
            pool.close()
        units = len(freqs) * w.T * iters
        value = units * len(times) / sum(times)
        sample = (f"{len(freqs)} of {w.F} frequencies x {iters} iterations + separation per step, "
                  f"{used} processes")
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()                   # spawned workers, before any CUDA work
    batch_data = None
    if rank == 0 and not args.no_batch:
        batch_data = generate_batch()          # spawned workers, before any CUDA work

    r = run_gpu(args, rank, world, local_rank)
    batch = None
    if batch_data is not None:
        import torch
        batch = run_batch(*batch_data, torch.device("cuda", local_rank), torch.cuda.current_stream())
    learned = None
    if rank == 0 and not args.no_learned:
        learned = run_learned(args.learned_mixtures)
    precision = None
    if rank == 0 and world == 1 and not args.no_precision:
        precision = precision_report()
    large = None
    if rank == 0 and world == 1 and not args.no_large:
        large = run_large(load_peaks())
    if rank != 0:
        return
    peaks = load_peaks()
    flops = algorithmic_flops_per_bin_iter(w.M, w.N) * w.F * w.T * w.iters
    em_avg_s = statistics.mean(r["em_ms"]) * 1e-3
    achieved = flops / em_avg_s / 1e12
    traffic = em_traffic()
    out = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "dtype_detail": "complex64 bins in FP32; the IP (Eq. 34-35) and the log-likelihood sums in FP64",
        "data": "synthetic (model-generated mixtures, seeded)", "config": config,
        "gpu_launches": 3 * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                     "kernel": "fastfca_em_kernel", "flops_per_bin_iter": algorithmic_flops_per_bin_iter(w.M, w.N),
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (unit counts and max clock)"},
        "roofline_separation": separation_roofline(w, r["sep_ms"], peaks),
        "clocks": r["clocks"],
        "e2e": {"value": r["e2e_value"], "unit": UNIT, "h2d_bytes_per_step": r["h2d"],
                "d2h_bytes_per_step": r["d2h"],
                "windows": r["e2e_windows"], "note": f"median of 3 windows of {r['e2e_steps']} steps"},
        "ip_mm": {"algorithm": "IP+MM (Algorithm 2), same mixture and start, 20 iterations (Table I)",
                  "iters": r["mm_iters"],
                  "value": w.F * w.T * r["mm_iters"] / (statistics.mean(r["mm_ms"]) * 1e-3), "unit": UNIT,
                  "launch_ms": statistics.mean(r["mm_ms"]), "loglik": r["mm_ll"],
                  "ip_em_same_iters": {"value": w.F * w.T * r["mm_iters"] / (statistics.mean(r["em_ms_same"]) * 1e-3),
                                       "launch_ms": statistics.mean(r["em_ms_same"]), "loglik": r["em_ll_same"]}},
        "block_input": {"model": "piecewise-stationary FastFCA (Sec. VI-B), IP+EM, blocks of %d frames" % r["blk"],
                        "B": r["blk"], "launch_ms": statistics.mean(r["blk_ms"]),
                        "block_iters_per_s": w.F * (w.T // r["blk"]) * w.iters / (statistics.mean(r["blk_ms"]) * 1e-3),
                        "frame_bin_iters_per_s": w.F * w.T * w.iters / (statistics.mean(r["blk_ms"]) * 1e-3)},
        "fca_comparison": {
            model: {"value": w.F * w.T * r["fca_iters"] / (r["fca_ms"][model] * 1e-3), "unit": UNIT,
                    "iters": r["fca_iters"], "ms": r["fca_ms"][model],
                    "loglik_per_bin": r["fca_ll"][model],
                    "update": {"fca": "EM, Eq. 12-13", "fca_mm": "MM with the geometric mean, Eq. 15-17"}[model]}
            for model in ("fca", "fca_mm")},
        "fastmnmf": {"model": "FastMNMF (App. C), K = %d bases per source, same mixture" % MNMF_K,
                     "iters": MNMF_ITERS, "ms": statistics.mean(r["mn_ms"]),
                     "value": w.F * w.T * MNMF_ITERS / (statistics.mean(r["mn_ms"]) * 1e-3), "unit": UNIT,
                     "launches_per_iter": 4, "loglik_per_bin": r["mn_ll"]},
        "em_launch_ms": statistics.mean(r["em_ms"]),
        "final_loglik": r["final_ll"],
        "hbm_peak_gbs_measured": peaks.get("hbm_gbs"),
    }
    if batch is not None:
        out["batch"] = batch
    if learned is not None:
        out["learned_init"] = learned
    if precision is not None:
        out["precision"] = precision
    if large is not None:
        out["large"] = large
    if cpu is not None:
        out["cpu_baseline"] = cpu
    print(json.dumps(out))


if __name__ == "__main__":
    main()
