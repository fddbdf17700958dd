"""The allocation-free H^1 entry point, hpse_h1_error_noalloc.

It serves callers that cannot call cudaMalloc: programs whose device memory
is owned entirely by another allocator (a framework caching allocator or a
fixed arena reserved at start-up), and latency-critical loops that must not
pay the device-wide synchronisation cudaFree implies.  Its scratch is a
fixed-size file-scope device array shared by every call.

The test calls it through the C ABI and checks it against hpse_h1_error (the
allocating entry point) on two calls in a row with different inputs, so that
contents left over from the first call cannot pass for the second result.  It
also checks that sizes beyond the array's capacity are refused before any
device work.  This file is collected last: it must pass in a fresh process and
after every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12  # the two entry points share the partial sums; only the final summation order differs


@pytest.fixture(scope="module")
def api():
    from paper_1110_2316_gb300.build import build
    build()
    from paper_1110_2316_gb300 import api as A
    return A


def _call(lib, fn, mesh, u, ref=None, vq=None, gq=None):
    out = np.zeros(2 * mesh.n_rhs)
    st = getattr(lib, fn)(mesh._h, C.c_void_p(u.data_ptr()),
                          None if ref is None else C.c_void_p(ref.data_ptr()),
                          None if vq is None else C.c_void_p(vq.data_ptr()),
                          None if gq is None else C.c_void_p(gq.data_ptr()),
                          out.ctypes.data_as(C.c_void_p),
                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


def test_noalloc_matches_allocating_entry_point(api):
    from paper_1110_2316_gb300 import _lib
    lib = _lib.load()
    pb = wl.varcoef_manufactured(n=(3, 2, 2), W=5)
    mesh = api.Mesh(pb.mesh, n_rhs=3, coef_kind=api.COEF_SCALAR)
    n = mesh.n_rhs * mesh.ndof
    for call, seed in enumerate((1, 2)):
        g = torch.Generator(device="cuda").manual_seed(seed)
        u = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
        ref = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
        st0, want = _call(lib, "hpse_h1_error", mesh, u, ref=ref)
        st1, got = _call(lib, "hpse_h1_error_noalloc", mesh, u, ref=ref)
        assert st0 == 0 and st1 == 0, (st0, st1)
        assert np.all(want > 0)
        assert np.allclose(got, want, rtol=REL_TOL, atol=0), (call, got, want)
    mesh.close()


def test_noalloc_refuses_sizes_beyond_its_array(api):
    from paper_1110_2316_gb300 import _lib
    lib = _lib.load()
    # 512 elements x 257 right-hand sides = 131584 items > 131072
    mesh = api.Mesh(wl.box_mesh(8, W=1), n_rhs=257, coef_kind=api.COEF_LAPLACE)
    u = torch.zeros(8, dtype=torch.float64, device="cuda")
    st, _ = _call(lib, "hpse_h1_error_noalloc", mesh, u, ref=u)
    assert st == 10  # HPSE_ERR_CAPACITY
    mesh.close()
