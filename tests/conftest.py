import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture
def rng():
    return np.random.Generator(np.random.PCG64(12345))


def rand_hpd(rng, M, scale=1.0):
    """A random Hermitian positive definite M x M matrix."""
    A = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    return scale * (A @ A.conj().T + 0.5 * np.eye(M))


def rand_complex(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


_LARGE = {}


@pytest.fixture(scope="session")
def large_workload():
    """The large single instance (M=8 circular 5 cm, N=12, F=1025, T=4000, K=16) and its seeded
    start, generated once per test session (the generator takes a while at this size)."""
    if not _LARGE:
        from paper_2101_08563_gb300 import synth
        w = synth.WORKLOADS["large"]
        mix = synth.generate_mixture(w.M, w.N, w.F, w.T, w.K, seed=w.seed, array=w.array, spacing=w.spacing,
                                     keep_images=False)
        _LARGE.update(w=w, x=mix.x, init=synth.random_init(mix.x, w.N, seed=w.seed))
    return _LARGE["w"], _LARGE["x"], _LARGE["init"]
