"""Benchmark: FastFCA IP+EM throughput (time-frequency-bin iterations per second) on GB300.

Headline workload: the large single instance, M=8 (circular array, r = 5 cm), N=12, F=1025,
T=4000, K=16.  One step = one complete FastFCA run on it through the library's C ABI: 50
IP+EM iterations (Algorithm 1) from the seeded random start, then the Wiener-filter
separation of Eq. 39.  The metric counts F*T*iters bin-iterations per step.  Inputs are
model-generated (synthetic) and resident in HBM when a timed step starts; the inputs are
larger than L2 and L2 is also flushed (a 512 MiB write) between steps, outside the timed
spans.

Also reported, each under its own key: the end-to-end figure through the C ABI with host
buffers (copies inside the span), the roofline of the IP+EM launch (FP32 ALU and the
streaming schedule's HBM bytes), the separation's HBM bandwidth, the oracle's throughput on
the host cores, the precision of every output against the FP64 oracle, and the other
workloads (M=4, N=6, F=513, T=1250 with IP+MM, block input, FCA and FastMNMF on it; the
64-mixture batch; the learned initialiser).

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

HEADLINE = synth.WORKLOADS["large"]       # M=8, N=12, F=1025, T=4000, 50 iterations
SECOND = synth.WORKLOADS["fca_cmp"]       # M=4, N=6, F=513, T=1250, 100 iterations
MNMF_K = 8            # FastMNMF bases per source on the M=4 mixture (its generator's K)
MNMF_ITERS = 20
METRIC = "FastFCA EM TF-bin-iters/s"
UNIT = "bin-iters/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP32 arithmetic peak from unit counts and the maximum clock: 152 SMs x 128 FP32 lanes x
# 2 flop (FMA) x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# oracle samples of the headline workload (frequencies spread over the band)
CPU_SAMPLE_FREQS, CPU_SAMPLE_ITERS = 64, 4
PRECISION_FREQS = [1, 300, 700, 1024]


def mnmf_abi_params(st):
    """A FastMNMF start in the C ABI's layouts: t (F, N, K), v (N, K, T)."""
    return (st.W, st.lam, np.ascontiguousarray(st.t.transpose(0, 2, 1)),
            np.ascontiguousarray(st.v.transpose(2, 1, 0)))


def algorithmic_flops_per_bin_iter(M: int, N: int) -> float:
    """FP32 flops one bin-iteration of Algorithm 1 needs (excluding the per-frequency IP):
    Q accumulation 6*M(M+1)/2 + 4*M*M(M+1)/2, decorrelation 8M^2, U 3M, NMF EM 13*M*N,
    log-likelihood terms 4M."""
    tri = M * (M + 1) / 2
    return 6 * tri + 4 * M * tri + 8 * M * M + 3 * M + 13 * M * N + 4 * M


def streaming_bytes_per_bin_iter(M: int, N: int) -> int:
    """HBM bytes one bin-iteration moves in the streaming schedule (x read twice as complex64,
    for the Q pass and the U pass; v read and written once as float32): 16 M + 8 N."""
    return 16 * M + 8 * N


def separation_bytes_per_bin(M: int, N: int) -> int:
    """Eq. 39 per bin: x read (8 M), v read (4 N), the N images written (8 N M)."""
    return 8 * M + 4 * N + 8 * N * M


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


# ----------------------------------------------------------------------------- oracle on the host
_WORKER_STATE = {}


def _pool_init(x, P, lam, v):
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    _WORKER_STATE.update(x=x, P=P, lam=lam, v=v)


def _noop(_):
    return 0


def _oracle_worker(args):
    """Algorithm 1 (with the per-iteration log-likelihood) and Eq. 39 on rows `idx` of the
    sampled frequencies this worker holds; returns each row's final W, L, H, log-likelihood
    and images when `keep`."""
    idx, iters, keep = args
    from oracle import fastfca as off
    s = _WORKER_STATE
    out = off.run(s["x"], s["P"], s["lam"], s["v"], iters=iters, freqs=idx, with_ll=True)
    res = []
    for i, f in enumerate(out["freqs"]):
        c = off.separate_fast(s["x"][f], out["W"][i], out["L"][i], out["H"][i])
        if keep:
            res.append((f, out["W"][i], out["L"][i], out["H"][i], out["ll"][i], c))
    return res if keep else len(idx)


class OraclePool:
    """Spawned worker processes, each holding the sampled frequencies of a mixture and its start
    (handed over at start-up, outside any timed span); `run` times the oracle over rows split
    across them."""

    def __init__(self, workers, data):
        import multiprocessing as mp
        self.workers = workers
        self.pool = mp.get_context("spawn").Pool(workers, initializer=_pool_init, initargs=data)
        self.pool.map(_noop, range(workers))

    def run(self, rows, iters, keep=False):
        chunks = [c for c in (rows[i::self.workers] for i in range(self.workers)) if c]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, [(c, iters, keep) for c in chunks], chunksize=1)
        return time.perf_counter() - t0, len(chunks), res

    def close(self):
        self.pool.close()
        self.pool.join()


def sample_freqs(F, n):
    return sorted(set(int(round(f)) for f in np.linspace(0, F - 1, n)))


def sampled_data(x, init, freqs):
    return (np.ascontiguousarray(x[freqs]), np.ascontiguousarray(init.P[freqs]),
            np.ascontiguousarray(init.lam[freqs]), np.ascontiguousarray(init.v[freqs]))


def cpu_baseline(w, x, init):
    """The oracle on a bounded sample of the headline workload (frequencies spread over the
    band, a few iterations each with the log-likelihood, then the separation) across the
    host's cores; each frequency costs the same, so the rate is that of the whole workload."""
    cores = os.cpu_count() or 1
    freqs = sample_freqs(w.F, CPU_SAMPLE_FREQS)
    pool = OraclePool(cores, sampled_data(x, init, freqs))
    try:
        wall, used, _ = pool.run(list(range(len(freqs))), CPU_SAMPLE_ITERS)
    finally:
        pool.close()
    sample = (f"{len(freqs)} of the {w.F} frequencies (spread over the band) x {CPU_SAMPLE_ITERS} IP+EM "
              f"iterations (+ log-likelihood each iteration) + separation, split over {used} processes")
    n1 = 4
    pool1 = OraclePool(1, sampled_data(x, init, freqs[:n1]))
    try:
        wall1, _, _ = pool1.run(list(range(n1)), 2)
    finally:
        pool1.close()
    return {"value": len(freqs) * w.T * CPU_SAMPLE_ITERS / wall, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": sample, "seconds": round(wall, 3),
            "single_core": {"value": n1 * w.T * 2 / wall1, "unit": UNIT, "cores": 1,
                            "sample": f"{n1} of the {w.F} frequencies x 2 iterations, one process",
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


def run_batch(shapes, data, dev, stream):
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
    # the same mixtures one at a time: one single-mixture context each, launched in a row on
    # one stream (device-resident, the same iterations), for the comparison with the batch
    seps = [fastfca.Separator(xs[b], shapes[b][1], stream=stream.cuda_stream) for b in range(len(shapes))]
    seq = []
    for _ in range(3):
        for b, s_ in enumerate(seps):
            s_.set_params(*inits[b])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s_ in seps:
            s_.iterate_async(BATCH_ITERS)
        e1.record(stream)
        torch.cuda.synchronize()
        seq.append(e0.elapsed_time(e1))
    for s_ in seps:
        s_.close()
    ms_seq = float(np.median(seq))
    return {"value": units / (ms * 1e-3), "unit": UNIT, "mixtures": BATCH_B, "iters": BATCH_ITERS,
            "ms_per_launch": ms, "per_mixture_ms_p50": float(np.percentile(sec, 50) * 1e3),
            "per_mixture_ms_p99": float(np.percentile(sec, 99) * 1e3),
            "one_at_a_time_value": units / (ms_seq * 1e-3), "one_at_a_time_ms": ms_seq,
            "schedule": {"bucketing": scheme, "grid_factor": factor},
            "config": "M in {2,3,4}, N in M+1..M+3, F=513, T uniform [200,2000], one CUDA-graph launch"}


# ----------------------------------------------------------------------------- learned initialiser
def run_learned(n_train):
    """The learned initialiser end to end on the GPU: n_train generated mixtures of the
    learned-initialiser workload with 200-iteration FastFCA targets, 6 epochs of training, and
    the comparison of the default start with two learned starts (the network's W, L and H; the
    network's W with the default L and H) on 512 held-out mixtures (batched as one context)."""
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
    res = L.evaluate(net, n_eval, w.F, w.T, w.M, w.N, w.K, w.spacing, seed=(0xFFFF << 32) + w.seed, max_iters=1000)
    net.close()
    res.update({"workload": w.name, "train_mixtures": n_train, "target_iters": w.iters,
                "train_data_seconds": t_data, "train_seconds": t_train, "epochs": 6, "batch_rows": 2048,
                "loss_untrained": loss0, "loss_trained": loss1,
                "held_out": "512 mixtures, generator key disjoint from the training keys"})
    return res


# ----------------------------------------------------------------------------- rooflines
def load_peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except Exception:
        return {}


_FP32_MEASURED = {}


def measured_fp32_tflops():
    """The FP32 FMA rate of this GPU from the library's probe (measured once per process)."""
    if "tf" not in _FP32_MEASURED:
        try:
            from paper_2101_08563_gb300 import fastfca
            _FP32_MEASURED["tf"] = fastfca.measure_fp32_fma(2000)
        except Exception:
            _FP32_MEASURED["tf"] = None
    return _FP32_MEASURED["tf"]


def em_roofline(w, em_ms, peaks, kernel, traffic):
    """The IP+EM launch against both ceilings: FP32 arithmetic (algorithmic flops per
    bin-iteration, unit-count peak) and HBM (the streaming schedule's 16 M + 8 N bytes per
    bin-iteration, measured copy bandwidth).  The binding one (the lower ceiling on
    bin-iters/s) is named in `bound`."""
    units = w.F * w.T * w.iters
    s = statistics.mean(em_ms) * 1e-3
    flops = algorithmic_flops_per_bin_iter(w.M, w.N)
    by = streaming_bytes_per_bin_iter(w.M, w.N)
    hbm = peaks.get("hbm_gbs")
    alu = {"achieved": flops * units / s / 1e12, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
           "frac": flops * units / s / 1e12 / FP32_PEAK_TFLOPS, "flops_per_bin_iter": flops,
           "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (unit counts and max clock)",
           "peak_measured_tflops": measured_fp32_tflops(),
           "peak_measured_source": "fastfca_measure_fp32_fma: 8 independent FMA chains per thread, 2048 threads "
                                   "on every SM, CUDA events"}
    mem = {"achieved": by * units / s / 1e9, "peak": hbm, "unit": "GB/s",
           "frac": (by * units / s / 1e9 / hbm) if hbm else None, "bytes_per_bin_iter": by,
           "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
           "note": "algorithmic bytes of the streaming schedule (x read twice, v read and written once)"}
    alu_ceiling = FP32_PEAK_TFLOPS * 1e12 / flops
    hbm_ceiling = (hbm * 1e9 / by) if hbm else float("inf")
    bound = "alu" if alu_ceiling < hbm_ceiling else "hbm"
    main = alu if bound == "alu" else mem
    return {"bound": bound, "achieved": main["achieved"], "peak": main["peak"], "unit": main["unit"],
            "frac": main["frac"], "traffic": traffic, "kernel": kernel, "launch_ms": statistics.mean(em_ms),
            "alu": alu, "hbm": mem,
            "ceilings_bin_iters_per_s": {"alu": alu_ceiling, "hbm": hbm_ceiling}}


def separation_roofline(w, sep_ms, peaks, kernel):
    """The Wiener separation (W^{-H} per frequency + Eq. 39 filter) of one step as an HBM-bound
    kernel: algorithmic bytes x (8 M) + v (4 N) read and c (8 N M) written per bin, over its
    event-timed span inside the step."""
    per_bin = separation_bytes_per_bin(w.M, w.N)
    bytes_ = per_bin * w.F * w.T
    ms = statistics.mean(sep_ms)
    hbm = peaks.get("hbm_gbs")
    gbs = bytes_ / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": gbs, "peak": hbm, "unit": "GB/s",
            "frac": (gbs / hbm) if hbm else None, "bytes_per_bin": per_bin, "ms": ms,
            "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}


def em_traffic(kernel_key):
    """DRAM bytes per launch of a kernel from the committed ncu record, or None when the
    kernel's sources changed since that capture."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(prof))[kernel_key]
        csrc = os.path.join(ROOT, "paper_2101_08563_gb300", "csrc")
        src = b"".join(open(os.path.join(csrc, f), "rb").read() for f in rec["sources"])
        if hashlib.sha1(src).hexdigest() != rec["source_sha1"]:
            return None
        return rec["bytes_per_launch"]
    except Exception:
        return None


# ----------------------------------------------------------------------------- the headline
def run_headline(args, rank, world, local_rank, w, x_np, init):
    """The headline workload on this rank: K timed steps (50 IP+EM iterations + separation, one
    stream, L2 flushed between steps), the end-to-end leg through the C ABI with host buffers,
    and one untimed run whose outputs feed the precision report."""
    import torch
    from paper_2101_08563_gb300 import fastfca

    dev = torch.device("cuda", local_rank)
    x = torch.from_numpy(x_np).to(dev)
    P0 = torch.from_numpy(init.P).to(dev)
    lam0 = torch.from_numpy(init.lam).to(dev)
    v0 = torch.from_numpy(init.v).to(dev)
    c = torch.empty((w.F, w.T, w.N, w.M), dtype=torch.complex64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sep = fastfca.Separator(x, w.N, stream=stream.cuda_stream)

    for _ in range(args.warmup):
        sep.set_params(P0, lam0, v0)
        sep.iterate(w.iters, return_ll=False)
        sep.separate(c)
        flush.zero_()
    torch.cuda.synchronize()

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
    units = w.F * w.T * w.iters
    value = weak_scaling_value(units * args.steps, sum(step_ms) * 1e-3, world, dev)
    tot_ms = world * units * args.steps / value * 1e3          # the max over ranks

    # one untimed run whose outputs the precision report compares with the oracle
    sep.set_params(P0, lam0, v0)
    hist = sep.iterate(w.iters)
    P, lam, v = sep.get_params()
    _, ll_f = sep.loglik(per_f=True)
    sep.separate(c)
    torch.cuda.synchronize()
    fs = PRECISION_FREQS
    outputs = {"freqs": fs, "ll_hist": hist, "ll_f": ll_f[fs], "P": P[fs], "lam": lam[fs], "v": v[fs],
               "c": c[fs].cpu().numpy()}
    x_sum_err = float((c.sum(dim=2) - x).abs().pow(2).sum().sqrt() / x.abs().pow(2).sum().sqrt())
    sep.close()
    del c
    torch.cuda.empty_cache()

    # end to end through the public API with host buffers (pinned), copies inside the span:
    # every step uploads its mixture and start, runs the iterations (reading back the
    # log-likelihood per iteration) and downloads the images.  Three long-lived contexts on
    # three streams take the steps in turn, so one step's copies overlap the others' kernels.
    n_ctx = 3
    x_h = torch.from_numpy(x_np).pin_memory()
    P_h = torch.from_numpy(init.P).pin_memory()
    lam_h = torch.from_numpy(init.lam).pin_memory()
    v_h = torch.from_numpy(init.v).pin_memory()
    c_hs = [torch.empty((w.F, w.T, w.N, w.M), dtype=torch.complex64).pin_memory() for _ in range(n_ctx)]
    ll_hs = [torch.empty(w.iters, dtype=torch.float64).pin_memory() for _ in range(n_ctx)]
    e2e_streams = [torch.cuda.Stream(dev) for _ in range(n_ctx)]
    ctxs = [fastfca.Separator(x_h, w.N, stream=st.cuda_stream) for st in e2e_streams]
    e2e_steps = max(6, min(args.steps, 12))

    def e2e_step(i):
        s = ctxs[i % n_ctx]
        s.sync()                         # this context's previous step has landed on the host
        s.set_mixture(x_h)
        s.set_params(P_h, lam_h, v_h)
        s.iterate_async(w.iters, ll_hs[i % n_ctx])
        s.separate_async(c_hs[i % n_ctx])
        return ll_hs[i % n_ctx]

    for i in range(n_ctx):
        e2e_step(i)
    for s_ in ctxs:
        s_.sync()
    e2e_windows = []
    ll = None
    for _ in range(3):
        barrier(world)
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            ll = e2e_step(i)
        for s_ in ctxs:
            s_.sync()
        e2e_windows.append(weak_scaling_value(units * e2e_steps, time.perf_counter() - t0, world, dev))
    e2e_value = statistics.median(e2e_windows)
    h2d = x_np.nbytes + init.P.nbytes + init.lam.nbytes + init.v.nbytes
    d2h = c_hs[0].numel() * 8 + w.iters * 8
    e2e_ll_ok = bool(np.allclose(ll.numpy(), hist, rtol=0, atol=0))
    for s_ in ctxs:
        s_.close()
    return {
        "value": value, "ms_per_step": tot_ms / args.steps, "em_ms": em_ms, "step_ms": step_ms, "sep_ms": sep_ms,
        "clocks": clock_info, "e2e_value": e2e_value, "e2e_windows": e2e_windows, "e2e_steps": e2e_steps,
        "h2d": h2d, "d2h": d2h, "e2e_ll_equal": e2e_ll_ok, "outputs": outputs, "images_sum_err": x_sum_err,
        "final_ll": float(hist[-1]),
    }


# ----------------------------------------------------------------------------- the M=4 workload
def run_second(args, rank, local_rank):
    """The M=4, N=6, F=513, T=1250 workload: IP+EM (100 iterations) + separation per step,
    device-timed; then IP+MM, the block input, FCA (EM and MM) and FastMNMF on the same mixture."""
    import torch
    from paper_2101_08563_gb300 import fastfca

    w = SECOND
    dev = torch.device("cuda", local_rank)
    mix = synth.workload_mixture(w, rank)
    init = synth.random_init(mix.x, w.N, seed=w.seed + rank)
    x = torch.from_numpy(mix.x).to(dev)
    P0, lam0, v0 = (torch.from_numpy(a).to(dev) for a in (init.P, init.lam, init.v))
    c = torch.empty((w.F, w.T, w.N, w.M), dtype=torch.complex64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sep = fastfca.Separator(x, w.N, stream=stream.cuda_stream)

    def timed(fn, reps=3, reset=None):
        out = []
        for _ in range(reps):
            flush.zero_()
            if reset:
                reset()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            fn()
            a1.record(stream)
            torch.cuda.synchronize()
            out.append(a0.elapsed_time(a1))
        return out

    reset = lambda: sep.set_params(P0, lam0, v0)   # noqa: E731
    for _ in range(3):
        reset()
        sep.iterate(w.iters, return_ll=False)
        sep.separate(c)
    steps = max(5, min(args.steps, 20))
    em_ms, sep_ms = [], []
    for _ in range(steps):
        flush.zero_()
        reset()
        a0, a1, a2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a0.record(stream)
        sep.iterate(w.iters, return_ll=False)
        a1.record(stream)
        sep.separate(c)
        a2.record(stream)
        torch.cuda.synchronize()
        em_ms.append(a0.elapsed_time(a1))
        sep_ms.append(a1.elapsed_time(a2))
    step_ms = [a + b for a, b in zip(em_ms, sep_ms)]

    # IP+MM (Algorithm 2) for the paper's iteration count (20, Table I), beside IP+EM's 20
    mm_iters = 20
    msep = fastfca.Separator(x, w.N, model="fastfca_mm", stream=stream.cuda_stream)
    msep.set_params(P0, lam0, v0)
    msep.iterate(2, return_ll=False)
    mm_ms = timed(lambda: msep.iterate(mm_iters, return_ll=False), reset=lambda: msep.set_params(P0, lam0, v0))
    msep.set_params(P0, lam0, v0)
    mm_ll = float(msep.iterate(mm_iters)[-1])
    msep.close()
    reset()
    em_ll_same = float(sep.iterate(mm_iters)[-1])
    em_ms_same = timed(lambda: sep.iterate(mm_iters, return_ll=False), reset=reset)

    # piecewise-stationary input (Sec. VI-B): blocks of 5 frames (250 blocks), its default start
    blk = 5
    bsep = fastfca.Separator(x, w.N, stream=stream.cuda_stream, block=blk, seed=w.seed)
    Pb, lamb, vb = (torch.from_numpy(a).to(dev) for a in bsep.get_params())
    bsep.iterate(2, return_ll=False)
    blk_ms = timed(lambda: bsep.iterate(w.iters, return_ll=False), reset=lambda: bsep.set_params(Pb, lamb, vb))
    bsep.close()

    # FCA comparison path on the same GPU (fewer iterations: it is ~an order slower)
    fca_iters = 10
    R0, h0 = synth.fca_random_init(mix.x, w.N, seed=w.seed + rank)
    R0d, h0d = torch.from_numpy(R0).to(dev), torch.from_numpy(h0).to(dev)
    fca = {}
    for model in ("fca", "fca_mm"):      # EM (Eq. 12-13) and MM (Eq. 15-17)
        fsep = fastfca.Separator(x, w.N, model=model, stream=stream.cuda_stream)
        fsep.set_params_fca(R0d, h0d)
        fsep.iterate(2, return_ll=False)
        ms = timed(lambda: fsep.iterate(fca_iters, return_ll=False), reps=1,
                   reset=lambda: fsep.set_params_fca(R0d, h0d))[0]
        fca[model] = {"value": w.F * w.T * fca_iters / (ms * 1e-3), "unit": UNIT, "iters": fca_iters, "ms": ms,
                      "loglik_per_bin": float(fsep.loglik()) / (w.F * w.T),
                      "update": {"fca": "EM, Eq. 12-13", "fca_mm": "MM with the geometric mean, Eq. 15-17"}[model]}
        fsep.close()

    # FastMNMF (App. C) on the same mixture, K bases per source
    st = synth.fastmnmf_random_init(mix.x, w.N, MNMF_K, seed=w.seed + rank)
    mparams = [torch.from_numpy(a).to(dev) for a in mnmf_abi_params(st)]
    mnsep = fastfca.Separator(x, w.N, model="fastmnmf", bases=MNMF_K, stream=stream.cuda_stream)
    mnsep.set_params_mnmf(*mparams)
    mnsep.iterate(2, return_ll=False)
    mn_ms = timed(lambda: mnsep.iterate(MNMF_ITERS, return_ll=False), reset=lambda: mnsep.set_params_mnmf(*mparams))
    mn_ll = float(mnsep.loglik()) / (w.F * w.T)
    mnsep.close()
    sep.close()

    peaks = load_peaks()
    units = w.F * w.T * w.iters
    return {
        "workload": w.name, "M": w.M, "N": w.N, "F": w.F, "T": w.T, "iters": w.iters,
        "metric": METRIC, "value": units / (statistics.mean(step_ms) * 1e-3), "unit": UNIT,
        "ms_per_step": statistics.mean(step_ms), "em_launch_ms": statistics.mean(em_ms),
        "roofline": em_roofline(w, em_ms, peaks, "fastfca_em_kernel<4,6> (one CTA per frequency)",
                                em_traffic("fastfca_em_kernel")),
        "roofline_separation": separation_roofline(w, sep_ms, peaks, "bst_to_winv_kernel + fastfca_mwf_kernel"),
        "l2_note": "x and v (36 MB) fit L2: the IP+EM launch reads HBM once per launch, so its HBM "
                   "fraction is an equivalent, not DRAM traffic",
        "ip_mm": {"algorithm": "IP+MM (Algorithm 2), same mixture and start, 20 iterations (Table I)",
                  "iters": mm_iters, "value": w.F * w.T * mm_iters / (statistics.mean(mm_ms) * 1e-3), "unit": UNIT,
                  "launch_ms": statistics.mean(mm_ms), "loglik": mm_ll,
                  "ip_em_same_iters": {"value": w.F * w.T * mm_iters / (statistics.mean(em_ms_same) * 1e-3),
                                       "launch_ms": statistics.mean(em_ms_same), "loglik": em_ll_same}},
        "block_input": {"model": "piecewise-stationary FastFCA (Sec. VI-B), IP+EM, blocks of %d frames" % blk,
                        "B": blk, "launch_ms": statistics.mean(blk_ms),
                        "block_iters_per_s": w.F * (w.T // blk) * w.iters / (statistics.mean(blk_ms) * 1e-3),
                        "frame_bin_iters_per_s": w.F * w.T * w.iters / (statistics.mean(blk_ms) * 1e-3)},
        "fca_comparison": fca,
        "fastmnmf": {"model": "FastMNMF (App. C), K = %d bases per source, same mixture" % MNMF_K,
                     "iters": MNMF_ITERS, "ms": statistics.mean(mn_ms),
                     "value": w.F * w.T * MNMF_ITERS / (statistics.mean(mn_ms) * 1e-3), "unit": UNIT,
                     "launches_per_iter": 4, "loglik_per_bin": mn_ll},
    }


# ----------------------------------------------------------------------------- precision
def _errors(ll, ll_ref, c, cr, P, W_ref, lam, v, L_ref, H_ref):
    """Every output against the oracle: log-likelihood, images per (f, n) block, W (fixed scale:
    the IP normalises it), the scale-free sigma^2 = LH and per-source powers L[:, n] H[n, :]."""
    d = np.abs(c.astype(np.complex128) - cr)
    a = np.abs(cr)
    fro = np.sqrt((d ** 2).sum(axis=(1, 3))) / np.sqrt((a ** 2).sum(axis=(1, 3)))
    ele = d.max(axis=(1, 3)) / a.max(axis=(1, 3))
    s2 = np.einsum("fmn,fnt->fmt", lam.astype(np.float64), v.astype(np.float64))
    s2r = np.einsum("fmn,fnt->fmt", L_ref, H_ref)
    pw = lam.astype(np.float64)[:, :, :, None] * v.astype(np.float64)[:, None, :, :]
    pwr = L_ref[:, :, :, None] * H_ref[:, None, :, :]
    return {
        "loglik_rel_err_max": float(np.max(np.abs(ll - ll_ref) / np.abs(ll_ref))),
        "images_rel_err": float(np.linalg.norm(c - cr) / np.linalg.norm(cr)),
        "images_rel_err_worst_f_n_block": float(fro.max()),
        "images_elementwise_err_worst_f_n_block": float(ele.max()),
        "W_rel_err": float(np.max(np.abs(P - W_ref)) / np.max(np.abs(W_ref))),
        "sigma2_rel_err_max": float(np.max(np.abs(s2 - s2r) / s2r)),
        "source_power_rel_err_median": float(np.median(np.abs(pw - pwr) / pwr)),
        "tolerance": {"loglik": 1e-5, "images": 1e-4},
    }


def precision_report(headline_outputs, x_head, init_head):
    """Error of every output of the CUDA path against the FP64 oracle from the same start: the
    whole small workload (M=2, N=3, F=257, T=250, 20 iterations), four frequencies of the M=4
    workload (100 iterations) and four frequencies of the headline workload (50 iterations,
    the outputs of the benchmark's own run)."""
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
        cr = np.stack([off.separate_fast(x[i], ref["W"][i], ref["L"][i], ref["H"][i]) for i in range(len(fs))])
        e = _errors(ll, ref["ll"].sum(axis=0), c, cr, P, ref["W"], lam, v, ref["L"], ref["H"])
        e.update({"workload": w.name, "frequencies": "all" if freqs is None else freqs, "iters": w.iters})
        out[name] = e
    if headline_outputs is not None:
        w = HEADLINE
        o = headline_outputs
        fs = o["freqs"]
        pool = OraclePool(len(fs), sampled_data(x_head, init_head, fs))
        try:
            _, _, res = pool.run(list(range(len(fs))), w.iters, keep=True)
        finally:
            pool.close()
        rows = sorted(r for chunk in res for r in chunk)
        W_ref = np.stack([r[1] for r in rows])
        L_ref = np.stack([r[2] for r in rows])
        H_ref = np.stack([r[3] for r in rows])
        ll_ref = np.array([r[4][-1] for r in rows])
        cr = np.stack([r[5] for r in rows])
        e = _errors(o["ll_f"], ll_ref, o["c"], cr, o["P"], W_ref, o["lam"], o["v"], L_ref, H_ref)
        e["loglik_rel_err_max"] = float(np.max(np.abs(o["ll_f"] - ll_ref) / np.abs(ll_ref)))
        e.update({"workload": w.name, "frequencies": fs, "iters": w.iters,
                  "note": "the benchmark's own run; log-likelihood compared per frequency after the last "
                          "iteration"})
        out["large"] = e
    return out


# ----------------------------------------------------------------------------- profiling cases
def run_profile_case(F, iters, workload="fca_cmp", model="fastfca", separate=False):
    """A workload's first 8 frequencies tiled to F (so the launch has F frequencies of the
    workload's shape), two launches of the IP+EM kernel (model "fastfca_mm": IP+MM): 2
    iterations, then `iters`.
    workload "fastmnmf": the full M=4 N=6 K=8 F=513 T=1250 mixture, FastMNMF, 2 iterations
    then `iters` (each iteration one fastmnmf_freq_kernel and one fastmnmf_v_kernel launch)."""
    import torch
    from paper_2101_08563_gb300 import build, fastfca
    if workload == "fastmnmf":
        w = SECOND
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


# ----------------------------------------------------------------------------- multi-rank helpers
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


def headline_config(w):
    return {"workload": w.name, "M": w.M, "N": w.N, "F": w.F, "T": w.T, "iters": w.iters,
            "K_nmf": w.K, "array": f"{w.array} r = {w.spacing * 100:.0f} cm" if w.array == "circular"
            else f"{w.array} {w.spacing * 100:.0f} cm",
            "step": "IP+EM (Algorithm 1) x iters + Wiener separation (Eq. 39), from the seeded random start",
            "l2": "inputs larger than L2 (x 262 MB, v 197 MB); L2 also flushed between steps (512 MiB write, "
                  "untimed)"}


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
    ap.add_argument("--no-second", action="store_true")
    ap.add_argument("--learned-mixtures", type=int, default=20000)
    ap.add_argument("--profile", action="store_true",
                    help="only run the IP+EM kernel on a workload's first frequencies tiled to "
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
    w = HEADLINE
    config = headline_config(w)

    if args.profile:
        run_profile_case(args.profile_F, args.profile_iters, args.profile_workload, args.profile_model,
                         args.profile_separate)
        return

    if args.impl == "reference":
        if rank != 0:
            return
        mix = synth.workload_mixture(w)
        init = synth.random_init(mix.x, w.N, seed=w.seed)
        cores = os.cpu_count() or 1
        freqs = sample_freqs(w.F, 2 * cores)
        iters = 2
        pool = OraclePool(cores, sampled_data(mix.x, init, freqs))
        rows = list(range(len(freqs)))
        try:
            for _ in range(args.warmup):
                pool.run(rows, iters)
            times = []
            for _ in range(args.steps):
                wall, used, _ = pool.run(rows, iters)
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

    # inputs first (host work, before any CUDA context): this rank's headline mixture and start
    mix = synth.workload_mixture(w, rank)
    x_head = mix.x
    init_head = synth.random_init(x_head, w.N, seed=w.seed + rank)
    del mix
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, x_head, init_head)      # spawned workers
    batch_data = None
    if rank == 0 and not args.no_batch:
        batch_data = generate_batch()

    import torch
    from paper_2101_08563_gb300 import build
    torch.cuda.set_device(local_rank)
    build.build()
    r = run_headline(args, rank, world, local_rank, w, x_head, init_head)
    if rank != 0:
        return
    dev = torch.device("cuda", local_rank)
    second = None if args.no_second else run_second(args, rank, local_rank)
    batch = run_batch(*batch_data, dev, torch.cuda.current_stream()) if batch_data is not None else None
    learned = None if args.no_learned else run_learned(args.learned_mixtures)
    precision = None
    if world == 1 and not args.no_precision:
        precision = precision_report(r["outputs"], x_head, init_head)
    peaks = load_peaks()
    out = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "dtype_detail": "complex64 bins in FP32; the IP (Eq. 34-35) and the log-likelihood sums in FP64",
        "data": "synthetic (model-generated mixtures, seeded)", "config": config,
        "gpu_launches": 3 * args.steps,
        "roofline": em_roofline(w, r["em_ms"], peaks, "fastfca_em_sm_kernel<8> (one CTA per frequency, sigma^2 and U in TMEM)",
                                em_traffic("fastfca_em_large")),
        "roofline_separation": separation_roofline(w, r["sep_ms"], peaks,
                                                   "bst_to_winv_kernel + fastfca_mwf_tile_kernel<8>"),
        "clocks": r["clocks"],
        "e2e": {"value": r["e2e_value"], "unit": UNIT, "h2d_bytes_per_step": r["h2d"],
                "d2h_bytes_per_step": r["d2h"], "windows": r["e2e_windows"],
                "note": f"median of 3 windows of {r['e2e_steps']} steps; three contexts on three streams; the "
                        f"last step's log-likelihood history equals the device run's: {r['e2e_ll_equal']}"},
        "em_launch_ms": statistics.mean(r["em_ms"]),
        "separation_ms": statistics.mean(r["sep_ms"]),
        "final_loglik": r["final_ll"],
        "loglik_per_bin": r["final_ll"] / (w.F * w.T),
        "images_sum_to_mixture_rel_err": r["images_sum_err"],
        "hbm_peak_gbs_measured": peaks.get("hbm_gbs"),
    }
    if cpu is not None:
        out["cpu_baseline"] = cpu
    if precision is not None:
        out["precision"] = precision
    if second is not None:
        out["m4n6"] = second
    if batch is not None:
        out["batch"] = batch
    if learned is not None:
        out["learned_init"] = learned
    print(json.dumps(out))


if __name__ == "__main__":
    main()
