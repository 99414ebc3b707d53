"""kr_block_reduce_noalloc: the block reduction without library allocations (GPU).

Some callers cannot let a library allocate device memory (their own pool
allocator owns all of it, or they cannot afford cudaMalloc's possible device
synchronisation inside the call).  This checks that the allocation-free entry
point, called through the C interface on two calls in a row, returns what the
allocating entry point kr_block_reduce returns, within the tolerance of the
other reduction tests, and that it rejects block widths beyond its static
scratch before doing any GPU work.  The file sorts last so that a stopping run
has executed every other test first.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import gaussian_block  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_04395_gb300 import build
    build.build()
    import paper_1504_04395_gb300 as m
    m.load_library()
    return m


@pytest.mark.parametrize("s", [1, 3, 8, 16])
@pytest.mark.parametrize("kind", ["gram", "trace", "sumv", "norm2"])
def test_noalloc_matches_allocating_entry_point(kr, s, kind):
    n = 300_007  # many CTAs with a ragged tail
    Y = torch.from_numpy(gaussian_block(n, s, seed=s)).cuda()
    U = None
    if kind in ("gram", "trace"):
        U = torch.from_numpy(gaussian_block(n, s, seed=100 + s)).cuda()
    elif kind == "sumv":
        U = torch.from_numpy(np.ascontiguousarray(gaussian_block(n, 1, seed=7)[:, 0])).cuda()
    ref = kr.kr_block_reduce(U, Y, kind=kind)
    Yh = Y.cpu().numpy()
    Uh = None if U is None else U.cpu().numpy().reshape(n, -1)
    bound = float(np.sum(np.abs(Yh) ** 2)) if kind == "norm2" else float(np.sum(np.abs(Uh).T @ np.abs(Yh)))
    code = kr.RED[kind]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    uptr = ctypes.c_void_p(0) if U is None else ctypes.c_void_p(U.data_ptr())
    for _ in range(2):  # two calls in a row share the static scratch
        out = torch.full_like(ref, complex(np.nan, np.nan))
        st = kr.lib().kr_block_reduce_noalloc(n, s, uptr, ctypes.c_void_p(Y.data_ptr()), code,
                                              ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 0, kr.kr_last_error()
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        if kind == "norm2":
            got, want = got.real, want.real
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - want)) <= 1e-13 * bound


def test_noalloc_rejects_width_beyond_scratch(kr):
    Y = torch.zeros((10, 17), dtype=torch.complex128, device="cuda")
    out = torch.zeros((17, 17), dtype=torch.complex128, device="cuda")
    st = kr.lib().kr_block_reduce_noalloc(10, 17, ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                          1, ctypes.c_void_p(out.data_ptr()), None)
    assert st == 9  # KR_UNSUPPORTED
    assert "s must be in [1, 16]" in kr.kr_last_error()
