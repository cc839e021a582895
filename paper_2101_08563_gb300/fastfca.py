"""ctypes binding of libfastfca.so (C ABI in include/fastfca.h).

Argument marshalling only: every step of the method runs in the library's CUDA kernels.
Arrays may be torch tensors (CPU or CUDA) or NumPy arrays (host); they must be C-contiguous
with the dtype and shape that include/fastfca.h gives.  The library reports errors through
status codes, raised here as FastFCAError.  Importing this module loads the library and
raises if it has not been built (``paper_2101_08563_gb300.build.build()``): there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

try:  # torch is optional for host-only use
    import torch
except Exception:  # pragma: no cover
    torch = None

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENUMERIC", 5: "EUNSUPPORTED"}
STATUS_ENUMERIC = 4
MODEL_FASTFCA = 0
MODEL_FCA = 1
MODEL_FASTFCA_MM = 2
MODEL_FCA_MM = 3
MODEL_FASTMNMF = 4

# Every entry point of include/fastfca.h with (restype, argtypes).
_P = ctypes.c_void_p
_SIGNATURES = {
    "fastfca_create": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(_P)]),
    "fastfca_create_blocks": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.POINTER(_P)]),
    "fastfca_create_mnmf": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.POINTER(_P)]),
    "fastfca_set_params_mnmf": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "fastfca_get_params_mnmf": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "fastfca_set_params": (ctypes.c_int, [_P, _P, _P, _P]),
    "fastfca_get_params": (ctypes.c_int, [_P, _P, _P, _P]),
    "fastfca_set_params_fca": (ctypes.c_int, [_P, _P, _P]),
    "fastfca_get_params_fca": (ctypes.c_int, [_P, _P, _P]),
    "fastfca_iterate": (ctypes.c_int, [_P, ctypes.c_int32, _P]),
    "fastfca_loglik": (ctypes.c_int, [_P, _P, _P]),
    "fastfca_separate": (ctypes.c_int, [_P, _P]),
    "fastfca_set_mixture": (ctypes.c_int, [_P, _P]),
    "fastfca_sync": (ctypes.c_int, [_P]),
    "fastfca_last_error": (ctypes.c_char_p, [_P]),
    "fastfca_destroy": (None, [_P]),
    "fastfca_version": (ctypes.c_char_p, []),
    "fastfca_debug_fail_alloc": (None, [ctypes.c_int64]),
    "fastfca_debug_live_allocs": (ctypes.c_int64, []),
    "fastfca_debug_large_bin_kernel": (None, [ctypes.c_int32]),
    "fastfca_debug_cluster_wait_limit": (None, [ctypes.c_int32]),
    "fastfca_measure_fp32_fma": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "fastfca_debug_f64_reciprocals": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                     ctypes.c_void_p]),
    "fastfca_separate_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                _P, _P, _P, _P, _P, _P]),
    "fastfca_batch_create": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, ctypes.POINTER(_P)]),
    "fastfca_batch_set_params": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P]),
    "fastfca_batch_get_params": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P]),
    "fastfca_batch_iterate": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "fastfca_batch_tune": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "fastfca_batch_schedule": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double]),
    "fastfca_batch_separate": (ctypes.c_int, [_P, ctypes.c_int32, _P]),
    "fastfca_batch_last_error": (ctypes.c_char_p, [_P]),
    "fastfca_batch_destroy": (None, [_P]),
    "fastfca_generate_mixtures": (ctypes.c_int, [ctypes.c_int32] * 6 + [ctypes.c_double, ctypes.c_uint64, _P, _P]),
    "fastfca_net_features": (ctypes.c_int, [ctypes.c_int32] * 4 + [_P, _P, _P, _P]),
    "fastfca_net_targets": (ctypes.c_int, [ctypes.c_int32] * 4 + [_P] * 7),
    "fastfca_net_create": (ctypes.c_int, [ctypes.c_int32] * 4 + [ctypes.c_uint64, _P, ctypes.POINTER(_P)]),
    "fastfca_net_param_count": (ctypes.c_int64, [_P]),
    "fastfca_net_get_params": (ctypes.c_int, [_P, _P]),
    "fastfca_net_set_params": (ctypes.c_int, [_P, _P]),
    "fastfca_net_forward": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "fastfca_net_loss_grad": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32] + [_P] * 7),
    "fastfca_net_train_step": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32] + [_P] * 5
                               + [ctypes.c_float, _P]),
    "fastfca_net_predict": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32] + [_P] * 5),
    "fastfca_net_last_error": (ctypes.c_char_p, [_P]),
    "fastfca_net_destroy": (None, [_P]),
}


class FastFCAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("F", ctypes.c_int32), ("T", ctypes.c_int32), ("M", ctypes.c_int32),
                ("N", ctypes.c_int32), ("model", ctypes.c_int32), ("seed", ctypes.c_int32)]


_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load() -> ctypes.CDLL:
    """Loads libfastfca.so (built in-tree); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run paper_2101_08563_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a, dtype_np, shape, name, writable=False):
    """(pointer, keepalive) for a torch tensor or NumPy array with the expected layout."""
    if a is None:
        return None, None
    if torch is not None and isinstance(a, torch.Tensor):
        want = {np.complex64: torch.complex64, np.complex128: torch.complex128,
                np.float32: torch.float32, np.float64: torch.float64}[dtype_np]
        if a.dtype != want:
            raise TypeError(f"{name}: expected {want}, got {a.dtype}")
        if tuple(a.shape) != tuple(shape):
            raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(a.shape)}")
        if not a.is_contiguous():
            raise ValueError(f"{name}: must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), a
    arr = a
    if not isinstance(arr, np.ndarray):
        raise TypeError(f"{name}: expected a torch tensor or NumPy array")
    if arr.dtype != dtype_np:
        raise TypeError(f"{name}: expected {np.dtype(dtype_np)}, got {arr.dtype}")
    if tuple(arr.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(arr.shape)}")
    if not arr.flags["C_CONTIGUOUS"]:
        raise ValueError(f"{name}: must be C-contiguous")
    if writable and not arr.flags["WRITEABLE"]:
        raise ValueError(f"{name}: must be writable")
    return ctypes.c_void_p(arr.ctypes.data), arr


def _default_stream():
    if torch is not None and torch.cuda.is_available():
        return torch.cuda.current_stream().cuda_stream
    return 0


class Separator:
    """One separation problem (one mixture) held by the library.

    x: complex64 (F, T, M), host or CUDA.  N: number of sources.  model: "fastfca" (IP+EM,
    Algorithm 1), "fastfca_mm" (the same model by IP+MM, Algorithm 2), "fca" (full-rank FCA by EM,
    Eq. 12-13), "fca_mm" (the same model by MM, Eq. 15-17) or "fastmnmf" (App. C, with
    `bases` = K NMF bases per source; parameters through set/get_params_mnmf).
    A CUDA x is borrowed (kept referenced here); a host x is copied by the library.  seed
    selects the random factor of the default initial v (see fastfca_create).
    """

    def __init__(self, x, N: int, model: str = "fastfca", stream=None, seed: int = 0, block: int = 1,
                 bases: int = 0):
        self.lib = load()
        shape = tuple(x.shape)
        if len(shape) != 3:
            raise ValueError("x must have shape (F, T, M)")
        self.F, self.T, self.M = (int(s) for s in shape)
        self.N = int(N)
        self.model = {"fastfca": MODEL_FASTFCA, "fca": MODEL_FCA, "fastfca_mm": MODEL_FASTFCA_MM,
                      "fca_mm": MODEL_FCA_MM, "fastmnmf": MODEL_FASTMNMF}[model]
        self.K = int(bases)
        cfg = Config(self.F, self.T, self.M, self.N, self.model, int(seed) & 0x7fffffff)
        px, self._x = _ptr(x, np.complex64, shape, "x")
        self.stream = _default_stream() if stream is None else stream
        h = ctypes.c_void_p()
        self.block = int(block)
        self.J = self.T // self.block if self.block >= 1 else self.T   # parameter columns
        if self.model == MODEL_FASTMNMF:
            st = self.lib.fastfca_create_mnmf(ctypes.byref(cfg), self.K, px, ctypes.c_void_p(self.stream),
                                              ctypes.byref(h))
        elif self.block == 1:
            st = self.lib.fastfca_create(ctypes.byref(cfg), px, ctypes.c_void_p(self.stream), ctypes.byref(h))
        else:
            st = self.lib.fastfca_create_blocks(ctypes.byref(cfg), self.block, px, ctypes.c_void_p(self.stream),
                                                ctypes.byref(h))
        if st != 0:
            raise FastFCAError(st, self.lib.fastfca_last_error(None).decode())
        self._h = h

    # ------------------------------------------------------------------ plumbing
    def _check(self, st):
        if st != 0:
            raise FastFCAError(st, self.lib.fastfca_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self.lib.fastfca_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ parameters
    def set_params(self, P, lam, v):
        F, M, N, T = self.F, self.M, self.N, self.J
        pP, kP = _ptr(P, np.complex128, (F, M, M), "P")
        pl, kl = _ptr(lam, np.float32, (F, M, N), "lam")
        pv, kv = _ptr(v, np.float32, (F, N, T), "v")
        self._check(self.lib.fastfca_set_params(self._h, pP, pl, pv))

    def get_params(self):
        F, M, N, T = self.F, self.M, self.N, self.J
        P = np.empty((F, M, M), np.complex128)
        lam = np.empty((F, M, N), np.float32)
        v = np.empty((F, N, T), np.float32)
        self._check(self.lib.fastfca_get_params(self._h, _ptr(P, np.complex128, P.shape, "P", True)[0],
                                                _ptr(lam, np.float32, lam.shape, "lam", True)[0],
                                                _ptr(v, np.float32, v.shape, "v", True)[0]))
        return P, lam, v

    def get_params_into(self, P=None, lam=None, v=None):
        F, M, N, T = self.F, self.M, self.N, self.J
        self._check(self.lib.fastfca_get_params(self._h, _ptr(P, np.complex128, (F, M, M), "P", True)[0],
                                                _ptr(lam, np.float32, (F, M, N), "lam", True)[0],
                                                _ptr(v, np.float32, (F, N, T), "v", True)[0]))

    def set_params_fca(self, R, h):
        F, M, N, T = self.F, self.M, self.N, self.T
        pR, kR = _ptr(R, np.complex128, (F, N, M, M), "R")
        ph, kh = _ptr(h, np.float32, (F, N, T), "h")
        self._check(self.lib.fastfca_set_params_fca(self._h, pR, ph))

    def get_params_fca(self):
        F, M, N, T = self.F, self.M, self.N, self.T
        R = np.empty((F, N, M, M), np.complex128)
        h = np.empty((F, N, T), np.float32)
        self._check(self.lib.fastfca_get_params_fca(self._h, _ptr(R, np.complex128, R.shape, "R", True)[0],
                                                    _ptr(h, np.float32, h.shape, "h", True)[0]))
        return R, h

    def set_params_mnmf(self, W, lam, t, v):
        """FastMNMF parameters: W complex128 (F, M, M), lam float32 (F, M, N), t float32
        (F, N, K) bases, v float32 (N, K, T) activations; host or CUDA."""
        F, M, N, K, T = self.F, self.M, self.N, self.K, self.T
        pW, kW = _ptr(W, np.complex128, (F, M, M), "W")
        pl, kl = _ptr(lam, np.float32, (F, M, N), "lam")
        pt, kt = _ptr(t, np.float32, (F, N, K), "t")
        pv, kv = _ptr(v, np.float32, (N, K, T), "v")
        self._check(self.lib.fastfca_set_params_mnmf(self._h, pW, pl, pt, pv))

    def get_params_mnmf(self):
        F, M, N, K, T = self.F, self.M, self.N, self.K, self.T
        W = np.empty((F, M, M), np.complex128)
        lam = np.empty((F, M, N), np.float32)
        t = np.empty((F, N, K), np.float32)
        v = np.empty((N, K, T), np.float32)
        self._check(self.lib.fastfca_get_params_mnmf(self._h, _ptr(W, np.complex128, W.shape, "W", True)[0],
                                                     _ptr(lam, np.float32, lam.shape, "lam", True)[0],
                                                     _ptr(t, np.float32, t.shape, "t", True)[0],
                                                     _ptr(v, np.float32, v.shape, "v", True)[0]))
        return W, lam, t, v

    # ------------------------------------------------------------------ algorithm
    def iterate(self, n_iter: int, return_ll: bool = True):
        """n_iter iterations; returns the total log-likelihood after each (np.float64), after
        synchronising (numerical failures raise here), or None without waiting."""
        if return_ll:
            ll = np.empty(n_iter, np.float64)
            self._check(self.lib.fastfca_iterate(self._h, int(n_iter), ll.ctypes.data_as(ctypes.c_void_p)))
            self.sync()
            return ll
        self._check(self.lib.fastfca_iterate(self._h, int(n_iter), None))
        return None

    def iterate_async(self, n_iter: int, ll_out=None):
        """Stream-ordered iterations; ll_out (host or CUDA float64 (n_iter,), pinned host for an
        asynchronous copy) receives the log-likelihood per iteration once the stream has passed
        the call (see sync)."""
        p = _ptr(ll_out, np.float64, (int(n_iter),), "ll_out", True)[0] if ll_out is not None else None
        self._check(self.lib.fastfca_iterate(self._h, int(n_iter), p))
        return ll_out

    def loglik(self, per_f: bool = False):
        tot = np.zeros(1, np.float64)
        pf = np.empty(self.F, np.float64) if per_f else None
        self._check(self.lib.fastfca_loglik(self._h, tot.ctypes.data_as(ctypes.c_void_p),
                                            pf.ctypes.data_as(ctypes.c_void_p) if per_f else None))
        return (float(tot[0]), pf) if per_f else float(tot[0])

    def separate(self, out=None):
        """Source images complex64 (F, T, N, M); into `out` (host or CUDA) when given.  A host
        result is complete on return (the call synchronises); a CUDA one is stream-ordered."""
        shape = (self.F, self.T, self.N, self.M)
        if out is None:
            out = np.empty(shape, np.complex64)
        self.separate_async(out)
        if not (torch is not None and isinstance(out, torch.Tensor) and out.is_cuda):
            self.sync()
        return out

    def separate_async(self, out):
        """Stream-ordered separation into `out` (host or CUDA, caller-allocated); a host buffer
        is complete once the context's stream has passed the call (see sync)."""
        shape = (self.F, self.T, self.N, self.M)
        p, keep = _ptr(out, np.complex64, shape, "c", True)
        self._check(self.lib.fastfca_separate(self._h, p))
        return out

    def set_mixture(self, x):
        """Replaces the mixture (same shape; host or CUDA), copied stream-ordered into a
        buffer the library owns."""
        p, keep = _ptr(x, np.complex64, (self.F, self.T, self.M), "x")
        self._check(self.lib.fastfca_set_mixture(self._h, p))
        self._x = keep

    def sync(self):
        self._check(self.lib.fastfca_sync(self._h))


def fail_allocation_after(n: int):
    """Fault injection: after n more device allocations by the library succeed, the next one
    fails as an out of memory would (one-shot; n < 0 disarms)."""
    load().fastfca_debug_fail_alloc(int(n))


def large_bin_kernel(which: str):
    """Kernel for IP+EM on the large-bin shapes in contexts created from now on: "auto" (by
    shape), "cluster" (thread-block clusters) or "sm" (one SM per frequency, T <= 4096)."""
    load().fastfca_debug_large_bin_kernel({"auto": 0, "cluster": 1, "sm": 2}[which])


def cluster_wait_limit(spins: int):
    """Failure injection: a cluster exchange of the cluster kernel is reported as timed out
    after `spins` polls (0 restores the default)."""
    load().fastfca_debug_cluster_wait_limit(int(spins))


def measure_fp32_fma(iters: int = 2000, stream=None) -> float:
    """The FP32 FMA rate of the current GPU in TFLOP/s (one timed launch over every SM)."""
    lib = load()
    out = ctypes.c_double()
    st = lib.fastfca_measure_fp32_fma(int(iters), ctypes.byref(out), ctypes.c_void_p(stream or _default_stream()))
    if st != 0:
        raise FastFCAError(st, lib.fastfca_last_error(None).decode())
    return float(out.value)


def live_allocations() -> int:
    """Device allocations the library holds now (all contexts, batches and networks)."""
    return int(load().fastfca_debug_live_allocs())


def abi_symbols_from_header(path: str | None = None):
    """Names of the functions declared in include/fastfca.h."""
    import re
    path = path or os.path.join(_build.ROOT, "include", "fastfca.h")
    txt = open(path).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b(fastfca_[a-z0-9_]+)\s*\(",
                                 txt, flags=re.M)))


class Batch:
    """Many independent FastFCA mixtures iterated together in one CUDA-graph launch.

    xs: list of complex64 (F_b, T_b, M_b) arrays (host or CUDA); Ns: sources per mixture;
    seeds: per-mixture seeds of the default initial v (default: the mixture index);
    models: per-mixture "fastfca" (IP+EM, Algorithm 1, the default) or "fastfca_mm" (IP+MM,
    Algorithm 2).
    """

    SCHEMES = {0: "fine", 1: "coarse", 2: "single", 3: "mixture"}

    def __init__(self, xs, Ns, stream=None, seeds=None, models=None):
        self.lib = load()
        if len(xs) != len(Ns) or not xs:
            raise ValueError("xs and Ns must be non-empty and of equal length")
        self.B = len(xs)
        self.shapes = []
        cfgs = (Config * self.B)()
        ptrs = (ctypes.c_void_p * self.B)()
        self._xs = []
        for i, (x, N) in enumerate(zip(xs, Ns)):
            F, T, M = (int(s) for s in x.shape)
            self.shapes.append((F, T, M, int(N)))
            seed = i if seeds is None else int(seeds[i]) & 0x7fffffff
            model = MODEL_FASTFCA if models is None else {"fastfca": MODEL_FASTFCA,
                                                          "fastfca_mm": MODEL_FASTFCA_MM}[models[i]]
            cfgs[i] = Config(F, T, M, int(N), model, seed)
            p, keep = _ptr(x, np.complex64, (F, T, M), f"xs[{i}]")
            ptrs[i] = p.value
            self._xs.append(keep)
        self.stream = _default_stream() if stream is None else stream
        h = ctypes.c_void_p()
        st = self.lib.fastfca_batch_create(self.B, cfgs, ptrs, ctypes.c_void_p(self.stream), ctypes.byref(h))
        if st != 0:
            raise FastFCAError(st, self.lib.fastfca_last_error(None).decode())
        self._h = h

    def _check(self, st):
        if st != 0:
            raise FastFCAError(st, self.lib.fastfca_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self.lib.fastfca_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, b, P, lam, v):
        F, T, M, N = self.shapes[b]
        pP, kP = _ptr(P, np.complex128, (F, M, M), "P")
        pl, kl = _ptr(lam, np.float32, (F, M, N), "lam")
        pv, kv = _ptr(v, np.float32, (F, N, T), "v")
        self._check(self.lib.fastfca_batch_set_params(self._h, b, pP, pl, pv))

    def get_params(self, b):
        F, T, M, N = self.shapes[b]
        P = np.empty((F, M, M), np.complex128)
        lam = np.empty((F, M, N), np.float32)
        v = np.empty((F, N, T), np.float32)
        self._check(self.lib.fastfca_batch_get_params(self._h, b, _ptr(P, np.complex128, P.shape, "P", True)[0],
                                                      _ptr(lam, np.float32, lam.shape, "lam", True)[0],
                                                      _ptr(v, np.float32, v.shape, "v", True)[0]))
        return P, lam, v

    def iterate(self, n_iter, stats=True, seconds=True):
        """Returns (log-likelihood per mixture, seconds per mixture or None) when stats, else
        None; seconds=False leaves the per-mixture spans out."""
        if not stats:
            self._check(self.lib.fastfca_batch_iterate(self._h, int(n_iter), None, None))
            return None
        ll = np.empty(self.B, np.float64)
        sec = np.empty(self.B, np.float64) if seconds else None
        st = self.lib.fastfca_batch_iterate(self._h, int(n_iter), ll.ctypes.data_as(ctypes.c_void_p),
                                            sec.ctypes.data_as(ctypes.c_void_p) if seconds else None)
        if st == STATUS_ENUMERIC:
            # the log-likelihoods are filled anyway: non-finite for the mixtures that failed
            err = FastFCAError(st, self.lib.fastfca_batch_last_error(self._h).decode())
            err.ll_per_mixture = ll
            raise err
        self._check(st)
        return ll, sec

    def tune(self, n_iter):
        scheme = ctypes.c_int32()
        factor = ctypes.c_double()
        self._check(self.lib.fastfca_batch_tune(self._h, int(n_iter), ctypes.byref(scheme), ctypes.byref(factor)))
        return self.SCHEMES[scheme.value], factor.value

    def schedule(self, scheme, factor=1.0):
        """Sets the schedule: "fine", "coarse" or "single" frame bucketing of the persistent
        class launches (factor scales each class's grid), or "mixture": one single-mixture
        launch per mixture on round(2 factor) concurrent graph branches."""
        code = {v: k for k, v in self.SCHEMES.items()}[scheme] if isinstance(scheme, str) else int(scheme)
        self._check(self.lib.fastfca_batch_schedule(self._h, code, ctypes.c_double(factor)))

    def separate(self, b, out):
        F, T, M, N = self.shapes[b]
        p, keep = _ptr(out, np.complex64, (F, T, N, M), "c", True)
        self._check(self.lib.fastfca_batch_separate(self._h, b, p))
        return out
