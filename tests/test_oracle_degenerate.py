"""Degenerate input: an all-zero frame (digital silence).  The likelihood of Eq. 25 has no
maximiser there (sigma^2 -> 0 raises it without bound).  These pins fix what each update does
with such a frame, which the kernels must reproduce: the EM updates keep the frame's power
positive and still never lower the likelihood, and the multiplicative updates set it to
exactly zero in one step."""
import warnings

import numpy as np
import pytest

from oracle import fastfca as off, fca as ofca, fastmnmf as omn
from paper_2101_08563_gb300 import synth


def silent_mixture(M, N, F, T, seed, t0=5):
    x = synth.generate_mixture(M, N, F, T, 4, seed=seed).x.copy()
    x[:, t0, :] = 0
    return x, t0


def test_ip_em_keeps_a_silent_frame_positive_and_ascends():
    """Algorithm 1: Phi_n = G^2 U + (1 - G) S reduces to (1 - G) S with U = 0, positive for
    N >= 2; the likelihood still rises every iteration (EM)."""
    x, t0 = silent_mixture(2, 3, 2, 60, seed=1)
    init = synth.random_init(x, 3, seed=1)
    r = off.run(x, init.P, init.lam, init.v, 6)
    ll = r["ll"].sum(axis=0)
    assert np.all(np.isfinite(ll)) and np.all(np.diff(ll) > 0)
    H = r["H"][:, :, t0]
    assert np.all(H > 0) and np.all(H < init.v[:, :, t0])   # shrinks, stays positive


def test_ip_mm_zeroes_a_silent_frame_in_one_update():
    """Algorithm 2: h <- h sqrt(L^T (U / (LH)^2) / L^T (1 / LH)) with U = 0 gives h = 0."""
    x, t0 = silent_mixture(2, 3, 2, 60, seed=2)
    init = synth.random_init(x, 3, seed=2)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        r = off.run(x, init.P, init.lam, init.v, 1, algorithm="mm")
    assert np.all(r["H"][:, :, t0] == 0)
    assert np.all(r["H"][:, :, np.arange(60) != t0] > 0)
    assert not np.all(np.isfinite(r["ll"]))


def test_fca_em_keeps_a_silent_frame_positive_and_ascends():
    x, t0 = silent_mixture(2, 3, 2, 60, seed=3)
    R0, h0 = synth.fca_random_init(x, 3, seed=3)
    r = ofca.run(x, R0, h0, 4)
    ll = r["ll"].sum(axis=0)
    assert np.all(np.isfinite(ll)) and np.all(np.diff(ll) > 0)


def test_fca_mm_zeroes_a_silent_frame():
    """Eq. 15: z = X^{-1} x = 0 makes the ratio, hence every h_nj at that frame, zero; the
    covariance there is then singular."""
    x, _ = silent_mixture(2, 3, 2, 60, seed=4)
    R0, h0 = synth.fca_random_init(x, 3, seed=4)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        with pytest.raises(np.linalg.LinAlgError):
            ofca.run(x, R0, h0, 2, algorithm="mm")


def test_fastmnmf_zeroes_a_frame_silent_at_every_frequency():
    """Eq. 53's v update sums over frequencies; with U = 0 at every one, v_jkn becomes 0."""
    x, t0 = silent_mixture(2, 3, 3, 60, seed=5)
    st = synth.fastmnmf_random_init(x, 3, 2, seed=5)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        r = omn.run(x, st.W, st.lam, st.t, st.v, 1)
    assert np.all(r["v"][t0] == 0)
    assert not np.all(np.isfinite(r["ll"]))
