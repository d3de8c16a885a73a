"""The allocation-free product (ttm_multiply_noalloc) against ttm_multiply.

Some callers cannot allocate device memory once they are running (a fixed device
budget reserved up front, memory already exhausted, or no tolerance for the implicit
synchronisation of cudaMalloc). For them the library offers ttm_multiply_noalloc, which
runs the same sweep in a fixed device array. This test calls it through the C ABI on two
products in a row (so the second call finds the first call's leftovers in the array) and
checks each result against ttm_multiply on the same inputs, with the tolerance of the other
float64 parity tests. It also checks that a product too large for the array is refused
before any GPU work. The file name makes pytest collect it last.
"""

import ctypes

import numpy as np
import pytest

import ttgen
from oracle import tt as ott

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_19747_gb300 as pkg
    pkg.build()
    lib = pkg.load_library()
    h = pkg.Handle(0)
    yield pkg, lib, h
    h.close()


def _dev(cores):
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cores]


def _noalloc(pkg, lib, A, B, fill=None, **opts):
    from paper_2410_19747_gb300 import binding as b
    Ad, Bd = _dev(A), _dev(B)
    a, bb = b.TTDesc(Ad), b.TTDesc(Bd)
    o = b.make_options(**opts)
    cap = int(lib.ttm_output_capacity(ctypes.byref(a.c), ctypes.byref(bb.c), ctypes.byref(o)))
    assert cap > 0
    L, d = len(A), A[0].shape[1]
    bufs = [torch.empty(cap, dtype=torch.float64, device="cuda") for _ in range(L)]
    if fill is not None:
        for t in bufs:
            t.fill_(fill)
        torch.cuda.synchronize()
    bonds = (ctypes.c_int64 * (L + 1))()
    ptrs = (ctypes.c_void_p * L)(*[t.data_ptr() for t in bufs])
    out = b.c_tt(L, 0, 0, 0, bonds, ptrs)
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.ttm_multiply_noalloc(ctypes.byref(a.c), ctypes.byref(bb.c), ctypes.byref(out), ctypes.byref(o),
                                  ctypes.c_void_p(stream))
    return st, out, bufs


def _cores(out, bufs, d):
    res = []
    for k in range(out.L):
        n = int(out.bonds[k]) * d * int(out.bonds[k + 1])
        res.append(bufs[k][:n].reshape(int(out.bonds[k]), d, int(out.bonds[k + 1])).cpu().numpy())
    return res


def test_noalloc_matches_multiply_on_two_calls_in_a_row(env):
    pkg, lib, h = env
    cases = [
        (ttgen.rand_tt(10, 2, 8, 1000, canon="left"), ttgen.rand_tt(10, 2, 8, 1100, canon="left"),
         dict(chi_max=8, chi_out=8)),
        (ttgen.rand_tt_spectral(12, 2, 16, 3200), ttgen.rand_tt_spectral(12, 2, 12, 3201),
         dict(eps=1e-10, chi_max=20, chi_out=20)),
    ]
    for A, B, opts in cases:
        st, out, bufs = _noalloc(pkg, lib, A, B, **opts)
        assert st == 0, lib.ttm_last_error().decode()
        got = _cores(out, bufs, A[0].shape[1])
        ref, _ = pkg.ttm_multiply(h, _dev(A), _dev(B), **opts)
        ref = [c.cpu().numpy() for c in ref]
        assert ott.bonds_of(got) == ott.bonds_of(ref)
        assert ott.diff_norm(got, ref) <= 1e-12 * ott.norm(ref)


def test_noalloc_refuses_products_beyond_its_array(env):
    pkg, lib, h = env
    A = ttgen.rand_tt(20, 2, 256, 7, canon="left")
    B = ttgen.rand_tt(20, 2, 256, 8, canon="left")
    st, out, bufs = _noalloc(pkg, lib, A, B, fill=-7.25, chi_max=256, chi_out=256)
    assert st == -4   # TTM_ERR_WORKSPACE
    assert b"workspace" in lib.ttm_last_error()
    torch.cuda.synchronize()
    for t in bufs:    # refused before any GPU work: the caller's output buffers are untouched
        assert bool((t == -7.25).all())
