"""Learned initialiser of FastFCA: ctypes binding of the fastfca_net_* and generator calls.

Argument marshalling and host orchestration only: data generation, features, targets, the
network's forward and backward passes, Adam and the prediction all run in the library's CUDA
kernels (include/fastfca.h gives the definitions).  Device arrays are torch CUDA tensors.

The paper initialises Algorithm 1 from masks (Sec. VII) and leaves better starting points
open; this module trains a small network on converged FastFCA runs over model-generated
mixtures and uses its output as the starting point instead of W = I, L = 1.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np
import torch

from . import fastfca as ff
from .fastfca import FastFCAError, _ptr

D_IN = 16
HIDDEN = 256
OUT_PAD = 40
CONV_K = 9


def _stream(stream=None):
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream if stream is None else stream)


def _check_global(st):
    if st != 0:
        raise FastFCAError(st, ff.load().fastfca_net_last_error(None).decode())


def _dev(t, dtype, shape, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name}: expected a CUDA tensor")
    return _ptr(t, dtype, shape, name)[0]


def generate_mixtures(B, F, T, M, N, K, spacing, seed, stream=None):
    """complex64 (B, F, T, M) CUDA tensor of model-generated mixtures (fastfca_generate_mixtures)."""
    x = torch.empty((B, F, T, M), dtype=torch.complex64, device="cuda")
    _check_global(ff.load().fastfca_generate_mixtures(B, F, T, M, N, K, float(spacing), int(seed) & (2**64 - 1),
                                                      _dev(x, np.complex64, x.shape, "x"), _stream(stream)))
    return x


def features(x, F, stream=None):
    """feats (rows, 16) and q (rows, T) for x complex64 (rows, T, M) on the GPU."""
    rows, T, M = (int(s) for s in x.shape)
    feats = torch.empty((rows, D_IN), dtype=torch.float32, device="cuda")
    q = torch.empty((rows, T), dtype=torch.float32, device="cuda")
    _check_global(ff.load().fastfca_net_features(rows, F, T, M, _dev(x, np.complex64, x.shape, "x"),
                                                 _dev(feats, np.float32, feats.shape, "feats"),
                                                 _dev(q, np.float32, q.shape, "q"), _stream(stream)))
    return feats, q


def targets(P, lam, v, stream=None):
    """Scale-free targets (wt (rows, M, M, 2), lt (rows, M, N), ht (rows, N, T)) on the GPU."""
    rows, M, _ = (int(s) for s in P.shape)
    N, T = int(v.shape[1]), int(v.shape[2])
    wt = torch.empty((rows, M, M, 2), dtype=torch.float32, device="cuda")
    lt = torch.empty((rows, M, N), dtype=torch.float32, device="cuda")
    ht = torch.empty((rows, N, T), dtype=torch.float32, device="cuda")
    _check_global(ff.load().fastfca_net_targets(
        rows, T, M, N, _dev(P, np.complex128, (rows, M, M), "P"), _dev(lam, np.float32, (rows, M, N), "lam"),
        _dev(v, np.float32, (rows, N, T), "v"), _dev(wt, np.float32, wt.shape, "wt"),
        _dev(lt, np.float32, lt.shape, "lt"), _dev(ht, np.float32, ht.shape, "ht"), _stream(stream)))
    return wt, lt, ht


def param_layout(M, N):
    """(name, offset, shape) of each block of the flat parameter vector."""
    blocks = [("W1", (HIDDEN, D_IN)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
              ("W3", (OUT_PAD, HIDDEN)), ("b3", (OUT_PAD,)), ("k", (N, CONV_K)), ("c", (N,))]
    out, off = [], 0
    for name, shape in blocks:
        out.append((name, off, shape))
        off += int(np.prod(shape))
    return out


def unpack(flat, M, N):
    """Dict of parameter blocks (views of flat) in the layout of include/fastfca.h."""
    return {name: flat[off: off + int(np.prod(shape))].reshape(shape) for name, off, shape in param_layout(M, N)}


class InitNet:
    """The initialiser network for (M, N) held by the library (fastfca_net_*)."""

    def __init__(self, M, N, max_rows, max_T, seed=0, stream=None):
        self.lib = ff.load()
        self.M, self.N, self.max_rows, self.max_T = int(M), int(N), int(max_rows), int(max_T)
        self.stream = _stream(stream)
        h = ctypes.c_void_p()
        st = self.lib.fastfca_net_create(self.M, self.N, self.max_rows, self.max_T, int(seed) & (2**64 - 1),
                                         self.stream, ctypes.byref(h))
        if st != 0:
            raise FastFCAError(st, self.lib.fastfca_net_last_error(None).decode())
        self._h = h
        self.count = int(self.lib.fastfca_net_param_count(self._h))

    def _check(self, st):
        if st != 0:
            raise FastFCAError(st, self.lib.fastfca_net_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self.lib.fastfca_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        out = np.empty(self.count, np.float32)
        self._check(self.lib.fastfca_net_get_params(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        if flat.shape != (self.count,):
            raise ValueError(f"expected {self.count} parameters")
        self._check(self.lib.fastfca_net_set_params(self._h, flat.ctypes.data_as(ctypes.c_void_p)))

    def forward(self, feats):
        rows = int(feats.shape[0])
        out = np.empty((rows, OUT_PAD), np.float32)
        self._check(self.lib.fastfca_net_forward(self._h, rows, _dev(feats, np.float32, (rows, D_IN), "feats"),
                                                 out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def _batch(self, feats, q, wt, lt, ht):
        rows, T = int(q.shape[0]), int(q.shape[1])
        M, N = self.M, self.N
        return rows, T, [_dev(feats, np.float32, (rows, D_IN), "feats"), _dev(q, np.float32, (rows, T), "q"),
                         _dev(wt, np.float32, (rows, M, M, 2), "wt"), _dev(lt, np.float32, (rows, M, N), "lt"),
                         _dev(ht, np.float32, (rows, N, T), "ht")]

    def loss_grad(self, feats, q, wt, lt, ht):
        """(mean loss, flat gradient as a host array) of one batch."""
        rows, T, ptrs = self._batch(feats, q, wt, lt, ht)
        loss = ctypes.c_double()
        g = np.empty(self.count, np.float32)
        self._check(self.lib.fastfca_net_loss_grad(self._h, rows, T, *ptrs, ctypes.byref(loss),
                                                   g.ctypes.data_as(ctypes.c_void_p)))
        return loss.value, g

    def train_step(self, feats, q, wt, lt, ht, lr, want_loss=False):
        rows, T, ptrs = self._batch(feats, q, wt, lt, ht)
        loss = ctypes.c_double()
        self._check(self.lib.fastfca_net_train_step(self._h, rows, T, *ptrs, ctypes.c_float(lr),
                                                    ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def predict(self, feats, q):
        """Starting point (P complex128 (rows, M, M), lam (rows, M, N), v (rows, N, T)) on the GPU."""
        rows, T = int(q.shape[0]), int(q.shape[1])
        M, N = self.M, self.N
        P = torch.empty((rows, M, M), dtype=torch.complex128, device="cuda")
        lam = torch.empty((rows, M, N), dtype=torch.float32, device="cuda")
        v = torch.empty((rows, N, T), dtype=torch.float32, device="cuda")
        self._check(self.lib.fastfca_net_predict(self._h, rows, T, _dev(feats, np.float32, (rows, D_IN), "feats"),
                                                 _dev(q, np.float32, (rows, T), "q"),
                                                 _dev(P, np.complex128, P.shape, "P"),
                                                 _dev(lam, np.float32, lam.shape, "lam"),
                                                 _dev(v, np.float32, v.shape, "v")))
        return P, lam, v


# ---------------------------------------------------------------------------- training data
def make_training_set(n_mix, F, T, M, N, K, spacing, seed, iters=200, chunk=256, stream=None):
    """Features and targets of n_mix generated mixtures (all resident on the GPU).

    Each chunk of mixtures is generated on the GPU, run through `iters` iterations of
    Algorithm 1 from the default start (fastfca_create's seeded W = I, L = 1 start) as one
    context over all its frequencies (frequencies are independent, Sec. IV-G), and reduced to
    features and scale-free targets.  Returns a dict of CUDA tensors with one row per (mixture, f)
    and the seconds spent.
    """
    R = n_mix * F
    dev = dict(device="cuda")
    data = {"feats": torch.empty((R, D_IN), dtype=torch.float32, **dev),
            "q": torch.empty((R, T), dtype=torch.float32, **dev),
            "wt": torch.empty((R, M, M, 2), dtype=torch.float32, **dev),
            "lt": torch.empty((R, M, N), dtype=torch.float32, **dev),
            "ht": torch.empty((R, N, T), dtype=torch.float32, **dev)}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j, b0 in enumerate(range(0, n_mix, chunk)):
        c = min(chunk, n_mix - b0)
        x = generate_mixtures(c, F, T, M, N, K, spacing, int(seed) + (j << 32), stream).view(c * F, T, M)
        sep = ff.Separator(x, N, stream=stream, seed=(int(seed) * 7919 + j) & 0x7fffffff)
        sep.iterate(iters, return_ll=False)
        P = torch.empty((c * F, M, M), dtype=torch.complex128, **dev)
        lam = torch.empty((c * F, M, N), dtype=torch.float32, **dev)
        v = torch.empty((c * F, N, T), dtype=torch.float32, **dev)
        sep.get_params_into(P, lam, v)
        r0, r1 = b0 * F, (b0 + c) * F
        wt, lt, ht = targets(P, lam, v, stream)
        feats, q = features(x, F, stream)
        for k, val in (("feats", feats), ("q", q), ("wt", wt), ("lt", lt), ("ht", ht)):
            data[k][r0:r1].copy_(val)
        sep.close()
        del x, P, lam, v, wt, lt, ht, feats, q
    torch.cuda.synchronize()
    return data, time.perf_counter() - t0


def train(net, data, epochs=4, batch=2048, lr=1e-3, seed=0, log_every=0):
    """Adam over contiguous row batches in a shuffled order each epoch, cosine learning rate.
    Returns (mean loss per epoch, seconds)."""
    R = int(data["q"].shape[0])
    starts = np.arange(0, R, batch)
    rng = np.random.default_rng(seed)
    total = epochs * len(starts)
    hist = []
    step = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ep in range(epochs):
        losses = []
        for s0 in rng.permutation(starts):
            s1 = min(s0 + batch, R)
            cur = lr * 0.5 * (1.0 + np.cos(np.pi * step / total))
            want = log_every > 0 and step % log_every == 0
            loss = net.train_step(*(data[k][s0:s1] for k in ("feats", "q", "wt", "lt", "ht")), cur,
                                  want_loss=want)
            if want:
                losses.append(loss)
            step += 1
        hist.append(float(np.mean(losses)) if losses else None)
    torch.cuda.synchronize()
    return hist, time.perf_counter() - t0


def mean_loss(net, data, batch=4096):
    """Mean loss over all rows of a data set (no update)."""
    R = int(data["q"].shape[0])
    tot = 0.0
    for s0 in range(0, R, batch):
        s1 = min(s0 + batch, R)
        loss, _ = net.loss_grad(*(data[k][s0:s1] for k in ("feats", "q", "wt", "lt", "ht")))
        tot += loss * (s1 - s0)
    return tot / R


# ---------------------------------------------------------------------------- evaluation
def _ll_trace(sep, n_mix, F, T, max_iters, conv):
    """Log-likelihood per mixture after each iteration, (iters run, n_mix), until no mixture's
    log-likelihood moves by more than conv per bin in one iteration, or max_iters, or the first
    numerical failure (ENUMERIC: after many iterations a nearly degenerate bin can leave the
    FP32 range of its Q_m or sigma^2); the trace then holds the iterations before it.
    Returns (trace, why it stopped)."""
    out = []
    prev = None
    why = "max_iters"
    for k in range(max_iters):
        try:
            sep.iterate(1, return_ll=False)
            _, pf = sep.loglik(per_f=True)
        except ff.FastFCAError as e:
            if "ENUMERIC" not in str(e) or not out:
                raise
            why = f"numerical failure reported after iteration {k + 1} ({e}); the trace ends at iteration {k}"
            break
        cur = pf.reshape(n_mix, F).sum(axis=1)
        out.append(cur)
        if prev is not None and np.max(np.abs(cur - prev)) < conv * F * T:
            why = "converged"
            break
        prev = cur
    return np.array(out), why


def _timed_replay(sep, iters, before=None):
    """(seconds the start `before()` took, seconds from the beginning to the end of each of
    `iters` single iterations), from CUDA events on the current stream, which the contexts
    here run on."""
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(iters)]
    torch.cuda.synchronize()
    e0.record(st)
    if before is not None:
        before()
    e1.record(st)
    for k in range(iters):
        sep.iterate(1, return_ll=False)
        ev[k].record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3, np.array([e0.elapsed_time(e) / 1e3 for e in ev])


def evaluate(net, n_mix, F, T, M, N, K, spacing, seed, max_iters=1000, tol=1e-3, conv=1e-6, early_iters=200,
             stream=None):
    """Learned starts vs the default start on n_mix held-out mixtures, batched as one context.

    Three starts: the default one ("plain"), the network's W, L and H ("learned"), and the
    network's W with the default start's L and H ("learned_w").  Each is run to convergence
    (until no mixture's log-likelihood changes by more than `conv` per bin in an iteration, at
    most max_iters iterations).  The reference of a mixture is the best of the three converged
    log-likelihoods; a start has reached it once it is within tol per bin (tol F T) of it.  Each start is then replayed, bit for bit the same
    run, with a CUDA event after every iteration: its time to the reference is measured from
    the start (for the learned start: features, network, prediction, upload) to the iteration
    that crosses.  Reports, per start, the iterations and seconds at which 50 % and 90 % of the
    mixtures have reached the reference, the fraction that reaches it at all, the converged
    log-likelihood per bin relative to the reference, and the fraction of mixtures on which the
    learned start ends below the default one (by more than tol per bin).

    The same is reported (under "to_default_<early_iters>") for a second reference: the
    default start's log-likelihood after early_iters iterations, the iteration count of the
    network's training targets.
    """
    x = generate_mixtures(n_mix, F, T, M, N, K, spacing, seed, stream).view(n_mix * F, T, M)
    bins = F * T
    plain_seed = (int(seed) * 31 + 7) & 0x7fffffff
    # default start: its parameters, then a trace to convergence
    plain = ff.Separator(x, N, stream=stream, seed=plain_seed)
    P0, lam0, v0 = (torch.from_numpy(a).cuda() for a in plain.get_params())
    tr_plain, why_plain = _ll_trace(plain, n_mix, F, T, max_iters, conv)
    # learned start: features, network, prediction, then a trace to convergence
    sep = ff.Separator(x, N, stream=stream, seed=0)

    def learned_start():
        feats, q = features(x, F, stream)
        P, lam, v = net.predict(feats, q)
        sep.set_params(P, lam, v)

    learned_start()
    tr_learned, why_learned = _ll_trace(sep, n_mix, F, T, max_iters, conv)
    # the network's W alone, with the default start's L and H
    sep_w = ff.Separator(x, N, stream=stream, seed=0)

    def learned_w_start():
        feats, q = features(x, F, stream)
        P, _, _ = net.predict(feats, q)
        sep_w.set_params(P, lam0, v0)

    learned_w_start()
    tr_w, why_w = _ll_trace(sep_w, n_mix, F, T, max_iters, conv)
    ref = np.maximum(np.maximum(tr_plain[-1], tr_learned[-1]), tr_w[-1])
    ref_early = tr_plain[min(early_iters, tr_plain.shape[0]) - 1]

    def first_hit(tr, r):
        hit = tr >= (r - tol * bins)[None, :]
        return np.where(hit.any(axis=0), hit.argmax(axis=0) + 1, np.inf)

    traces = (("plain", tr_plain), ("learned", tr_learned), ("learned_w", tr_w))
    hits = {name: first_hit(tr, ref) for name, tr in traces}
    hits_early = {name: first_hit(tr, ref_early) for name, tr in traces}
    # timed replays of the same runs, up to the last crossing of either reference
    times, t_start = {}, {}
    for name, ctx, start in (("plain", plain, lambda: plain.set_params(P0, lam0, v0)),
                             ("learned", sep, learned_start), ("learned_w", sep_w, learned_w_start)):
        fin = np.concatenate([hits[name][np.isfinite(hits[name])], hits_early[name][np.isfinite(hits_early[name])]])
        kmax = int(fin.max()) if fin.size else 1
        t_start[name], times[name] = _timed_replay(ctx, kmax, before=start)
    plain.close()
    sep.close()
    sep_w.close()
    res = {"n_mix": n_mix, "max_iters": max_iters, "tol_per_bin": tol, "conv_per_bin": conv,
           "iters_run": {"plain": int(tr_plain.shape[0]), "learned": int(tr_learned.shape[0]),
                         "learned_w": int(tr_w.shape[0])},
           "trace_stopped": {"plain": why_plain, "learned": why_learned, "learned_w": why_w},
           "starts": {"plain": "the default start (fastfca_create's W = I, L = 1, seeded H)",
                      "learned": "the network's W, L and H",
                      "learned_w": "the network's W with the default start's L and H"},
           "reference": "per mixture, the best of the three starts' converged log-likelihoods",
           "timing": "CUDA events after every iteration of a replay of the same run, from the start "
                     "(the learned start's features, network, prediction and upload included)",
           "learned_ends_below_default_fraction": float(np.mean(tr_learned[-1] < tr_plain[-1] - tol * bins)),
           "learned_w_ends_above_default_fraction": float(np.mean(tr_w[-1] > tr_plain[-1] + tol * bins)),
           "learned_w_ends_below_default_fraction": float(np.mean(tr_w[-1] < tr_plain[-1] - tol * bins)),
           "learned_start_seconds": float(t_start["learned"]),
           "seconds_per_iteration": float(np.median(np.diff(times["plain"]))) if len(times["plain"]) > 1 else None}
    def crossing(name, its):
        sec = np.array([times[name][int(k) - 1] if np.isfinite(k) else np.inf for k in its])
        out = {"reached_fraction": float(np.isfinite(its).mean())}
        for pct in (50, 90):
            q = int(max(np.ceil(pct / 100.0 * len(its)) - 1, 0))
            k, t = np.sort(its)[q], np.sort(sec)[q]
            out[f"iters_p{pct}"] = float(k) if np.isfinite(k) else None
            out[f"seconds_p{pct}"] = float(t) if np.isfinite(t) else None
        return out

    res[f"to_default_{early_iters}"] = {
        "reference": f"per mixture, the default start's log-likelihood after {early_iters} iterations "
                     f"(the training targets' iteration count), within tol per bin"}
    for name, tr in traces:
        out = crossing(name, hits[name])
        out["converged_fraction"] = out.pop("reached_fraction")
        out.update({"final_ll_per_bin_minus_ref": float(np.median((tr[-1] - ref) / bins)),
                    "ll_per_bin_after_1": float(np.median((tr[0] - ref) / bins)),
                    "ll_per_bin_after_10": float(np.median((tr[min(9, tr.shape[0] - 1)] - ref) / bins))})
        res[name] = out
        res[f"to_default_{early_iters}"][name] = crossing(name, hits_early[name])
    return res
