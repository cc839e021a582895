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
def _ll_trace(sep, n_mix, F, iters):
    """Log-likelihood per mixture after each of `iters` iterations: (iters, n_mix)."""
    out = np.empty((iters, n_mix))
    for it in range(iters):
        sep.iterate(1, return_ll=False)
        _, pf = sep.loglik(per_f=True)
        out[it] = pf.reshape(n_mix, F).sum(axis=1)
    return out


def _time_iters(sep, k=10):
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record()
    sep.iterate(k, return_ll=False)
    end.record()
    torch.cuda.synchronize()
    return start.elapsed_time(end) / 1e3 / k


def evaluate(net, n_mix, F, T, M, N, K, spacing, seed, iters=200, tol=1e-3, stream=None):
    """Learned start vs the default start on n_mix held-out mixtures, batched as one context.

    The reference is the log-likelihood the default start reaches after `iters` iterations; a
    mixture has converged once its log-likelihood is within tol per bin (tol F T) of that.
    Reports, per start, the iterations at which 50 % and 90 % of the mixtures have converged,
    the batched wall time to get there (start cost + iterations x measured time per
    iteration), the fraction that converges at all within `iters`, and the final
    log-likelihood per bin relative to the reference.
    """
    x = generate_mixtures(n_mix, F, T, M, N, K, spacing, seed, stream).view(n_mix * F, T, M)
    bins = F * T
    # default start
    plain = ff.Separator(x, N, stream=stream, seed=(int(seed) * 31 + 7) & 0x7fffffff)
    t_iter = _time_iters(plain)
    plain.close()
    plain = ff.Separator(x, N, stream=stream, seed=(int(seed) * 31 + 7) & 0x7fffffff)
    ll_plain = _ll_trace(plain, n_mix, F, iters)
    plain.close()
    # learned start (timed: features, network, prediction, parameter upload)
    sep = ff.Separator(x, N, stream=stream, seed=0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    feats, q = features(x, F, stream)
    P, lam, v = net.predict(feats, q)
    sep.set_params(P, lam, v)
    ev1.record()
    torch.cuda.synchronize()
    t_start = ev0.elapsed_time(ev1) / 1e3
    ll_learned = _ll_trace(sep, n_mix, F, iters)
    sep.close()
    ref = ll_plain[-1]
    thresh = ref - tol * bins

    def first_hit(tr):
        hit = tr >= thresh[None, :]
        its = np.where(hit.any(axis=0), hit.argmax(axis=0) + 1, np.inf)
        return its

    res = {"n_mix": n_mix, "iters": iters, "tol_per_bin": tol, "seconds_per_iteration": t_iter,
           "learned_start_seconds": t_start}
    for name, tr, t0 in (("plain", ll_plain, 0.0), ("learned", ll_learned, t_start)):
        its = first_hit(tr)
        out = {"converged_fraction": float(np.isfinite(its).mean()),
               "final_ll_per_bin_minus_ref": float(np.median((tr[-1] - ref) / bins)),
               "ll_per_bin_after_1": float(np.median((tr[0] - ref) / bins)),
               "ll_per_bin_after_10": float(np.median((tr[min(9, iters - 1)] - ref) / bins))}
        srt = np.sort(its)
        for pct in (50, 90):
            k = srt[max(int(np.ceil(pct / 100.0 * len(srt))) - 1, 0)]   # order statistic; inf = never
            k = float(k) if np.isfinite(k) else None
            out[f"iters_p{pct}"] = k
            out[f"seconds_p{pct}"] = None if k is None else t0 + k * t_iter
        res[name] = out
    return res
