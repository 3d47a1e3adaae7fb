"""nek_dot_c_noalloc, the weighted dot for callers that cannot allocate.

Some callers may not allocate device memory once their set-up is over: a host
framework that owns every device allocation, or a time-critical loop in which
cudaMalloc/cudaFree (which synchronise the device) are not allowed.  For them
the library keeps the reduction's partial sums in a fixed array of its own, and
nek_dot_c_noalloc must give the same result as nek_dot_c.  Two calls in a row
check that the shared array's leftover contents never leak into a result.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2011_04981_gb300 import inputs, nekax  # noqa: E402


def _call_noalloc(lib, n, c, a, b, out):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.nek_dot_c_noalloc(n, c.data_ptr(), a.data_ptr(), b.data_ptr(), out.data_ptr(), stream)


def test_noalloc_dot_matches_dot_c_on_two_calls_in_a_row():
    lib = nekax.load()
    dev = torch.device("cuda")
    cases = [((24, 16, 12), 6), ((4, 3, 2), 5)]  # ~1.0 M points (all blocks), then a few blocks
    for call, (dims, nx) in enumerate(cases):
        mesh = inputs.box_mesh(*dims, nx, perturb=0.1, seed=call)
        n = mesh.npts
        gs = nekax.GsPlan(mesh.nelt, nx, mesh.glo_num)
        c = torch.empty(n, dtype=torch.float64, device=dev)
        gs.inv_multiplicity(c)
        a = torch.from_numpy(inputs.random_global_field(mesh, seed=10 + call).reshape(-1)).to(dev)
        b = torch.from_numpy(inputs.random_global_field(mesh, seed=20 + call).reshape(-1)).to(dev)
        expect = torch.zeros(1, dtype=torch.float64, device=dev)
        nekax.dot_c(gs, a, b, expect)
        got = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        assert _call_noalloc(lib, n, c, a, b, got) == nekax.OK
        torch.cuda.synchronize()
        # same kernels, same grid, same partials: the header promises bit equality
        assert float(got.item()) == float(expect.item()), (call, got.item(), expect.item())
    # n = 0: one block, no loads, a sum of nothing (and no stale partial from the calls above)
    zero = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
    assert _call_noalloc(lib, 0, c, a, b, zero) == nekax.OK
    torch.cuda.synchronize()
    assert float(zero.item()) == 0.0


def test_noalloc_dot_rejects_oversize_and_bad_pointers():
    lib = nekax.load()
    A = 0x10000
    assert lib.nek_dot_c_noalloc(1 << 31, A, A, A, A, None) == nekax.ERR_TOO_LARGE
    assert lib.nek_dot_c_noalloc(-1, A, A, A, A, None) == nekax.ERR_INVALID_ARG
    assert lib.nek_dot_c_noalloc(10, None, A, A, A, None) == nekax.ERR_INVALID_ARG
    assert lib.nek_dot_c_noalloc(10, A, A, A, None, None) == nekax.ERR_INVALID_ARG
    for bad in range(4):  # a pointer that is not 8-byte aligned, rejected before any launch
        args = [A, A, A, A]
        args[bad] = A + 4
        assert lib.nek_dot_c_noalloc(10, *args, None) == nekax.ERR_INVALID_ARG, bad
