"""fastfca_separate_noalloc: the separation entry point for callers that cannot allocate.

Code that separates audio inside a real-time callback (or any section where an allocator
call may block the thread or synchronise the device) cannot call cudaMalloc there.  The
library gives such callers one entry point that takes every input and output from them and
keeps its single intermediate in a fixed array compiled into the library.  This test calls it
through the C ABI, twice in a row, with the library's next device allocation armed to fail
(so any allocation inside the call would surface as an error), and checks both outputs
against the context-based fastfca_separate on the same parameters and against the oracle's
Eq. 39, per (frequency, source) block.  Two shapes cover both filter kernels.  It lives in its own
file, collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fastfca as off  # noqa: E402
from paper_2101_08563_gb300 import synth  # noqa: E402
from parity import assert_images  # noqa: E402

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4   # the source-image tolerance the other GPU tests use


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("M,N,F,T", [
    (3, 4, 11, 300),      # the frequency-resident filter
    (6, 8, 5, 1300),      # the wide filter (the shapes the cluster kernel fits)
])
def test_noalloc_separation_matches_context_separation(M, N, F, T):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2101_08563_gb300 import build, fastfca
    build.build()
    lib = fastfca.load()

    mix = synth.generate_mixture(M, N, F, T, 4, seed=21, array="circular" if M >= 5 else "linear",
                                 spacing=0.05 if M >= 5 else 0.03)
    rng = np.random.Generator(np.random.PCG64(21))
    P = (rng.standard_normal((F, M, M)) + 1j * rng.standard_normal((F, M, M))) * 0.3 + np.eye(M)
    lam = rng.uniform(0.2, 2.0, (F, M, N)).astype(np.float32)
    v = rng.uniform(0.2, 5.0, (F, N, T)).astype(np.float32)

    xd = torch.from_numpy(mix.x).cuda()
    sep = fastfca.Separator(xd, N)
    sep.set_params(P, lam, v)
    ref = sep.separate()
    sep.close()
    # the oracle's Eq. 39 with the same parameters (FP64)
    oracle_ref = np.stack([off.separate_fast(mix.x[f], P[f], lam[f].astype(np.float64), v[f].astype(np.float64))
                           for f in range(F)])

    Pd = torch.from_numpy(P).cuda()
    lamd = torch.from_numpy(lam).cuda()
    vd = torch.from_numpy(v).cuda()
    c = torch.empty((F, T, N, M), dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    live = fastfca.live_allocations()
    for call in range(2):
        c.fill_(float("nan"))
        # the next device allocation of the library would fail: this call must make none
        fastfca.fail_allocation_after(0)
        try:
            st = lib.fastfca_separate_noalloc(F, T, M, N, _p(xd), _p(Pd), _p(lamd), _p(vd), _p(c),
                                              ctypes.c_void_p(stream))
        finally:
            fastfca.fail_allocation_after(-1)
        assert st == 0, lib.fastfca_last_error(None)
        assert fastfca.live_allocations() == live
        torch.cuda.synchronize()
        got = c.cpu().numpy()
        assert np.all(np.isfinite(got)), f"call {call}: output not fully written"
        assert_images(got, ref, IMG_TOL, f"call {call} against fastfca_separate")
        assert_images(got, oracle_ref, IMG_TOL, f"call {call} against the oracle")

    # sizes beyond the static scratch are refused before any launch
    big_F = 65536 // (M * M) + 1
    st = lib.fastfca_separate_noalloc(big_F, T, M, N, _p(xd), _p(Pd), _p(lamd), _p(vd), _p(c),
                                      ctypes.c_void_p(stream))
    assert st == 1 and b"exceeds" in lib.fastfca_last_error(None)
