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
