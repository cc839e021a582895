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
