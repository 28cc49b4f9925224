"""Device memory through the caller's allocator hook (hfdib_set_allocator).

The binding installs PyTorch's caching allocator: a handle's buffers then
show up in torch.cuda.memory_allocated() and go back at destroy.  A handle
made while cudaMalloc is installed runs the same sweeps bit for bit, and a
counting hook sees every block returned with the size it was allocated with.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2606_06135_gb300 import geometry as G
from paper_2606_06135_gb300 import hfdib

pytestmark = pytest.mark.gpu


def test_torch_caching_allocator_serves_the_handle():
    import torch
    hfdib.use_torch_allocator()
    case = G.case_cylinder(64, 32)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    s = hfdib.Solver(case, precision=1)
    held = torch.cuda.memory_allocated() - before
    # about 60 FP64 arrays of N cells and more (fields, hierarchy, mirrors)
    assert held >= 40 * 8 * case["lam"].size, held
    r1 = s.sweep(3)
    f1 = {n: s.field(n).cpu().numpy() for n in ("ux", "uy", "p", "k")}
    s.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
    # the same sweeps with cudaMalloc'd buffers
    hfdib.use_cuda_malloc()
    try:
        s2 = hfdib.Solver(case, precision=1)
        assert torch.cuda.memory_allocated() == before
        r2 = s2.sweep(3)
        np.testing.assert_array_equal(r1, r2)
        for n, v in f1.items():
            np.testing.assert_array_equal(s2.field(n).cpu().numpy(), v)
        s2.close()
    finally:
        hfdib.use_torch_allocator()


def test_counting_hook_sees_every_block_back():
    import torch
    lib = hfdib.load_library()
    live = {}
    log = {"alloc": 0, "free": 0}

    def alloc(nbytes, stream, ctx):
        p = torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        live[int(p)] = int(nbytes)
        log["alloc"] += 1
        return int(p)

    def free(ptr, nbytes, stream, ctx):
        assert live.pop(int(ptr)) == int(nbytes)
        log["free"] += 1
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = hfdib.ALLOC_FN(alloc), hfdib.FREE_FN(free)
    assert lib.hfdib_set_allocator(a, f, None) == 0
    try:
        b = hfdib.BatchSolver([G.case_cylinder(48, 24), G.case_cylinder(32, 16)], precision=1)
        b.sweep(2)
        assert log["alloc"] > 0 and live
        b.close()
        assert not live and log["free"] == log["alloc"]
    finally:
        hfdib._ALLOCATOR = None
        hfdib.use_torch_allocator()


def _poison_cache(torch):
    """Leave blocks of many sizes in the caching allocator, every byte 0xFF
    (a NaN in FP32 and in FP64)."""
    junk = []
    for nbytes, count in ((1 << 12, 64), (1 << 16, 64), (1 << 19, 64), (1 << 20, 32), (1 << 22, 8),
                          (1 << 24, 8)):
        for _ in range(count):
            junk.append(torch.full((nbytes,), 255, dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()
    del junk


CASES = {"cylinder_45x23": lambda: G.case_cylinder(45, 23), "sphere_20x12x10": lambda: G.case_sphere(20, 12, 10)}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("precision", [0, 1])
def test_stale_memory_from_the_cache_does_not_reach_the_solve(precision, name):
    """Blocks from the caching allocator keep what their last user wrote.
    With the cache filled with NaN bit patterns, a handle's sweeps equal those
    of a handle on cudaMalloc'd memory bit for bit: no kernel lets a value it
    has not written reach a result (a term that is dropped is selected away,
    never multiplied by zero: 0 * NaN is NaN).  Odd sizes give ragged x-pairs
    and coarse levels."""
    import torch
    case = CASES[name]()
    hfdib.use_cuda_malloc()
    try:
        ref = hfdib.Solver(case, precision=precision)
        r_ref = ref.sweep(6)
        f_ref = ref.fields()
        ref.close()
    finally:
        hfdib.use_torch_allocator()
    _poison_cache(torch)
    s = hfdib.Solver(case, precision=precision)
    r = s.sweep(6)
    assert np.all(np.isfinite(r)), r
    np.testing.assert_array_equal(r, r_ref)
    f = s.fields()
    for n, v in f_ref.items():
        np.testing.assert_array_equal(f[n], v, err_msg=n)
    s.close()
