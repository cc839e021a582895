"""The library's FP64 reciprocal helpers against CUDA's correctly rounded division and square
root, and the FP32 FMA rate probe the benchmark reports (GPU).

The IP (Eq. 34-35) divides by the pivots of Q_m and by sqrt(w^H Q_m w) through
rcp_pos_f64 / rsqrt_pos_f64: an FP32 hardware approximation of the scaled argument refined by
one Newton-Raphson step, so the relative error is about the square of the FP32 seed's
(~2^-22), i.e. ~2^-44, plus FP64 rounding.  Held here to 1e-13 relative over twenty decades."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ff():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2101_08563_gb300 import build, fastfca
    build.build()
    fastfca.load()
    return fastfca


def test_f64_reciprocals_match_cuda_division_and_sqrt(ff):
    rng = np.random.Generator(np.random.PCG64(5))
    x = np.concatenate([10.0 ** rng.uniform(-150, 150, 200000),       # the exponents the IP can meet
                        rng.uniform(0.5, 4.0, 100000),
                        np.array([1.0, 2.0, 4.0, 0.5, 0.25, 1.5, 3.999999999999, 1e-300, 1e300])])
    xd = torch.from_numpy(x).cuda()
    rcp = torch.empty_like(xd)
    rsq = torch.empty_like(xd)
    lib = ff.load()
    st = lib.fastfca_debug_f64_reciprocals(len(x), ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(rcp.data_ptr()),
                                            ctypes.c_void_p(rsq.data_ptr()),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    ref_rcp = (1.0 / xd)                      # CUDA's IEEE division
    ref_rsq = torch.rsqrt(xd)
    torch.cuda.synchronize()
    e_rcp = ((rcp - ref_rcp).abs() / ref_rcp).max().item()
    e_rsq = ((rsq - ref_rsq).abs() / ref_rsq).max().item()
    assert e_rcp <= 1e-13, e_rcp
    assert e_rsq <= 1e-13, e_rsq


def test_fp32_fma_probe_is_near_the_unit_count_peak(ff):
    """The measured FP32 FMA rate lies between half of and slightly above the peak from unit
    counts (SMs x 128 lanes x 2 flops at the 2.07 GHz maximum clock)."""
    dev = torch.cuda.get_device_properties(0)
    tf = ff.measure_fp32_fma(2000)
    unit_peak = dev.multi_processor_count * 128 * 2 * 2.07e9 / 1e12      # at the 2.07 GHz maximum clock
    assert 0.5 * unit_peak <= tf <= 1.05 * unit_peak, (tf, unit_peak)
