"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/fastfca.h declares.  No compute call is made (no GPU needed)."""
import ctypes
import os
import subprocess

import pytest

from paper_2101_08563_gb300 import build, fastfca

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return fastfca.load()


def test_header_declares_the_boundary():
    names = fastfca.abi_symbols_from_header()
    for required in ("fastfca_create", "fastfca_iterate", "fastfca_separate", "fastfca_loglik",
                     "fastfca_destroy", "fastfca_set_params", "fastfca_get_params"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    names = fastfca.abi_symbols_from_header()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding's signature table covers the header exactly
    assert sorted(fastfca._SIGNATURES) == names


def test_exported_symbols_are_c_linkage():
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB_PATH], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("nm unavailable")
    exported = {ln.split()[-1] for ln in out.stdout.splitlines() if " T " in ln}
    for n in fastfca.abi_symbols_from_header():
        assert n in exported, n


def test_version_string(lib):
    assert b"sm_103a" in lib.fastfca_version()


def test_create_rejects_null_arguments_without_touching_the_gpu(lib):
    h = ctypes.c_void_p()
    # NULL cfg / x are rejected before any CUDA call
    assert lib.fastfca_create(None, None, None, ctypes.byref(h)) == 1
    assert h.value is None
    assert b"required" in lib.fastfca_last_error(None)


def test_config_struct_matches_header():
    assert ctypes.sizeof(fastfca.Config) == 24


def test_allocation_fault_injection_is_host_state(lib):
    """The allocation counters live on the host: nothing is held before any context exists,
    and arming or disarming the injected failure touches no device."""
    assert fastfca.live_allocations() == 0
    fastfca.fail_allocation_after(3)
    fastfca.fail_allocation_after(-1)          # disarmed again: later tests allocate normally
    assert fastfca.live_allocations() == 0


def test_noalloc_separation_refuses_misaligned_buffers_before_any_device_work(lib):
    """fastfca_separate_noalloc checks the alignment its kernels' vector accesses need (x and
    P 16 bytes, c 8 bytes, lam and v 4 bytes) before it looks at a pointer's memory type or
    touches a device, so a misaligned buffer is an EINVAL here, on a machine with no GPU,
    instead of a misaligned-address fault on one.  The addresses are never dereferenced."""
    F, T, M, N = 4, 64, 6, 8                   # the wide filter's shape class
    good = [ctypes.c_void_p(0x10000 * (k + 1)) for k in range(5)]    # x, P, lam, v, c

    def call(x, P, lam, v, c):
        return lib.fastfca_separate_noalloc(F, T, M, N, x, P, lam, v, c, None)

    for k, bad, what in ((4, 0x50004, b"c must start on an 8-byte"), (0, 0x10008, b"x and P"),
                         (1, 0x20008, b"x and P"), (2, 0x30002, b"lam and v"), (3, 0x40001, b"lam and v")):
        args = list(good)
        args[k] = ctypes.c_void_p(bad)
        assert call(*args) == 1, what                    # FASTFCA_EINVAL
        assert what in lib.fastfca_last_error(None)
    # M = 9 has no filter kernel; a zero size is refused
    assert lib.fastfca_separate_noalloc(F, T, 9, N, *good, None) == 5        # FASTFCA_EUNSUPPORTED
    assert lib.fastfca_separate_noalloc(0, T, M, N, *good, None) == 1
