"""The allocation-free classification entry point against the allocating one.

hfdib_classify_noalloc exists for callers that cannot allocate device memory
when they need the cell groups (their memory belongs to another framework's
pool, they run under a fixed budget, or they must stay out of the driver's
allocator); its scratch is a fixed array inside the library.  Here it is
called several times in a row through the C ABI, on different lambda fields
(2D and 3D), and each result must equal -- bit for bit, as every integer output in these tests
-- what a handle made by hfdib_create reports for the same field.  The file
is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2606_06135_gb300 import geometry as G

pytestmark = pytest.mark.gpu


def noalloc(lib, case, torch, stream):
    from paper_2606_06135_gb300 import hfdib
    g = case["grid"]
    N = g["nx"] * g["ny"] * g["nz"]
    lam = torch.as_tensor(np.ascontiguousarray(case["lam"])).cuda()
    tags = torch.full((N,), 255, dtype=torch.uint8, device="cuda")
    cells = torch.full((N,), -7, dtype=torch.int32, device="cuda")
    n_bc = C.c_int64(-1)
    torch.cuda.synchronize()
    rc = lib.hfdib_classify_noalloc(C.byref(hfdib.grid_struct(g)), C.c_void_p(lam.data_ptr()),
                                    C.c_void_p(tags.data_ptr()), C.c_void_p(cells.data_ptr()), N,
                                    C.byref(n_bc), C.c_void_p(stream.cuda_stream))
    assert rc == 0, rc
    return tags.cpu().numpy().reshape(case["lam"].shape), cells.cpu().numpy()[: n_bc.value], n_bc.value


def reference(case):
    from paper_2606_06135_gb300.hfdib import Solver
    s = Solver(case)
    tags, nbc = s.tags()
    cells = s.bc_list()["cell"] if nbc else np.zeros(0, np.int64)
    s.close()
    return tags, cells, nbc


def test_noalloc_matches_create_on_two_calls_in_a_row():
    import torch
    from paper_2606_06135_gb300 import hfdib
    lib = hfdib.load_library()
    stream = torch.cuda.Stream()
    for case in (G.case_bfs(1024, 256), G.case_cylinder(64, 32), G.case_sphere(32, 16, 16)):
        t_ref, c_ref, n_ref = reference(case)
        t, c, n = noalloc(lib, case, torch, stream)
        assert n == n_ref
        np.testing.assert_array_equal(t, t_ref)
        np.testing.assert_array_equal(c.astype(np.int64), c_ref)


def test_noalloc_rejects_sizes_beyond_its_capacity():
    from paper_2606_06135_gb300 import hfdib
    lib = hfdib.load_library()
    g = hfdib.Grid(4097, 4096, 1, 0, 0, 0, 1, 1, 1)      # 2^24 + 4096 cells
    n_bc = C.c_int64(0)
    rc = lib.hfdib_classify_noalloc(C.byref(g), C.c_void_p(8), C.c_void_p(8), C.c_void_p(8), 0,
                                    C.byref(n_bc), None)
    assert rc == hfdib.STATUS_TOO_LARGE
    assert lib.hfdib_error_string(rc) == b"problem exceeds a fixed capacity of the call"


@pytest.mark.parametrize("bad", [float("nan"), -0.25, 1.5])
def test_noalloc_rejects_lambda_outside_the_unit_interval(bad):
    """A NaN or out-of-range lambda value fails the call, as it fails
    hfdib_create; the next call with a valid field succeeds (the flag is
    cleared per call)."""
    import torch
    from paper_2606_06135_gb300 import hfdib
    lib = hfdib.load_library()
    stream = torch.cuda.Stream()
    case = G.case_cylinder(32, 16)
    lam = np.ascontiguousarray(case["lam"]).copy()
    lam.flat[37] = bad
    g = case["grid"]
    N = lam.size
    lam_d = torch.as_tensor(lam).cuda()
    tags = torch.empty((N,), dtype=torch.uint8, device="cuda")
    cells = torch.empty((N,), dtype=torch.int32, device="cuda")
    n_bc = C.c_int64(-1)
    torch.cuda.synchronize()
    rc = lib.hfdib_classify_noalloc(C.byref(hfdib.grid_struct(g)), C.c_void_p(lam_d.data_ptr()),
                                    C.c_void_p(tags.data_ptr()), C.c_void_p(cells.data_ptr()), N,
                                    C.byref(n_bc), C.c_void_p(stream.cuda_stream))
    assert rc == -1 and n_bc.value == 0
    t, c, n = noalloc(lib, case, torch, stream)
    t_ref, c_ref, n_ref = reference(case)
    assert n == n_ref
    np.testing.assert_array_equal(t, t_ref)
