"""Source checks of the library's failure policy (CPU, no build needed): a kernel reports a
problem through the context's status word and returns; it never traps, never fails a device
assert, and never waits without a bound.  These are the properties that keep a GPU usable
for the next call after a numerical or configuration failure.  Every device allocation goes
through the counted allocator, which the fault-injection tests rely on."""
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2101_08563_gb300", "csrc")


def sources():
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(CSRC, name)) as f:
                yield name, f.read()


def strip_comments(text):
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.sub(r"//[^\n]*", "", text)


def test_no_trap_and_no_device_assert():
    for name, text in sources():
        code = strip_comments(text)
        assert "__trap" not in code, name
        assert not re.search(r"\btrap\s*;", code), name                  # inline PTX trap
        assert not re.search(r"(?<!static_)\bassert\s*\(", code), name     # only static_assert


def test_every_open_ended_loop_is_bounded():
    """Loops with no bound of their own: the persistent batch kernel's item loop (it ends when
    the atomic counter passes the item count) is the only `for (;;)`; every mbarrier wait (the
    cluster exchange's, and the tensor-core product's completion in the learned network's
    GEMM) counts its spins against a limit."""
    forever = []
    for name, text in sources():
        code = strip_comments(text)
        forever += [name for _ in re.finditer(r"for\s*\(\s*;\s*;\s*\)|while\s*\(\s*(true|1)\s*\)", code)]
    assert forever == ["fastfca_em.cuh"]
    em = strip_comments(dict(sources())["fastfca_em.cuh"])
    loop = em[em.index("for (;;)"):]
    assert re.search(r"if \(i >= n_items\) return;", loop[:400])
    spins = [m.group(0) for _, t in sources() for m in re.finditer(r"while \(!mbar_try_wait[^\n]*", strip_comments(t))]
    assert spins and all(("kMbarSpinLimit" in s) or ("kGemmSpin" in s) for s in spins)
    # the injected-limit form polls without blocking, against the launch's limit
    polls = [m.group(0) for _, t in sources()
             for m in re.finditer(r"while \(!\(done = mbar_test_wait[^\n]*", strip_comments(t))]
    assert polls and all("wait_limit" in s for s in polls)



def test_device_allocations_go_through_the_counted_allocator():
    """cudaMalloc and cudaMallocAsync appear only in dev_malloc_raw / dev_malloc_async_raw, so
    the library's live-allocation count and its injected allocation failures see every
    device allocation (the allocation-free separation is checked against that count)."""
    calls = []
    for name, text in sources():
        code = strip_comments(text)
        for m in re.finditer(r"\bcuda(Malloc|MallocAsync|MallocManaged|MallocPitch|Malloc3D)\s*\(", code):
            head = code[:m.start()]
            fn = re.findall(r"cudaError_t (\w+)\(", head)
            calls.append((name, fn[-1] if fn else None, m.group(1)))
    assert sorted(calls) == [("api.cu", "dev_malloc_async_raw", "MallocAsync"),
                             ("api.cu", "dev_malloc_raw", "Malloc")], calls
