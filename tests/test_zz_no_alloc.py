"""kr_block_reduce_noalloc: the block reduction without library allocations (GPU).

Some callers cannot let a library allocate device memory (their own pool
allocator owns all of it, or they cannot afford cudaMalloc's possible device
synchronisation inside the call).  This checks that the allocation-free entry
point, called through the C interface on two calls in a row, returns the FP64
reduction computed on the host from the same blocks (U^H Y, its trace, u^H Y
summed, ||Y||_F^2) and what the allocating entry point kr_block_reduce returns,
within the tolerance of the other reduction tests; that the Python wrapper
rejects outputs and operands of the wrong shape; and that block widths beyond
the static scratch are rejected before any GPU work.  The file sorts last so
that a stopping run has executed every other test first.
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
    # the reduction in FP64 on the host, from its definition
    if kind == "gram":
        host = Uh.conj().T @ Yh
    elif kind == "trace":
        host = np.array([np.sum(Uh.conj() * Yh)])
    elif kind == "sumv":
        host = np.array([np.sum(Uh[:, 0].conj() @ Yh)])
    else:
        host = np.array([np.sum(np.abs(Yh) ** 2)])
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
        got, want = out.cpu().numpy().reshape(host.shape), ref.cpu().numpy().reshape(host.shape)
        if kind == "norm2":
            got, want, hv = got.real, want.real, host.real
        else:
            hv = host
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - hv)) <= 1e-13 * bound
        assert np.max(np.abs(got - want)) <= 1e-13 * bound


@pytest.mark.parametrize("kind", ["gram", "sumv"])
def test_noalloc_python_wrapper(kr, kind):
    n, s = 5003, 4
    Y = torch.from_numpy(gaussian_block(n, s, seed=1)).cuda()
    if kind == "gram":
        U = torch.from_numpy(gaussian_block(n, s, seed=2)).cuda()
        out = torch.empty((s, s), dtype=torch.complex128, device="cuda")
        host = U.cpu().numpy().conj().T @ Y.cpu().numpy()
    else:
        U = torch.from_numpy(np.ascontiguousarray(gaussian_block(n, 1, seed=2)[:, 0])).cuda()
        out = torch.empty((1,), dtype=torch.complex128, device="cuda")
        host = np.array([np.sum(U.cpu().numpy().conj() @ Y.cpu().numpy())])
    got = kr.kr_block_reduce_noalloc(U, Y, out, kind=kind)
    torch.cuda.synchronize()
    bound = float(np.sum(np.abs(U.cpu().numpy()).reshape(n, -1).T @ np.abs(Y.cpu().numpy())))
    assert np.max(np.abs(got.cpu().numpy().reshape(host.shape) - host)) <= 1e-13 * bound


def test_noalloc_wrapper_rejects_wrong_shapes(kr):
    n, s = 1000, 4
    Y = torch.zeros((n, s), dtype=torch.complex128, device="cuda")
    U = torch.zeros((n, s), dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):  # a Gram needs an (s, s) output
        kr.kr_block_reduce_noalloc(U, Y, torch.zeros((1,), dtype=torch.complex128, device="cuda"), kind="gram")
    with pytest.raises(TypeError):  # wrong dtype of the output
        kr.kr_block_reduce_noalloc(U, Y, torch.zeros((s, s), dtype=torch.float64, device="cuda"), kind="gram")
    with pytest.raises(ValueError):  # U narrower than Y
        kr.kr_block_reduce_noalloc(U[:, :2].contiguous(), Y, torch.zeros((s, s), dtype=torch.complex128,
                                                                         device="cuda"), kind="gram")
    with pytest.raises(ValueError):  # sumv takes an n-vector
        kr.kr_block_reduce_noalloc(U, Y, torch.zeros((1,), dtype=torch.complex128, device="cuda"), kind="sumv")


def test_noalloc_rejects_host_memory(kr):
    Y = torch.zeros((10, 2), dtype=torch.complex128)
    out = torch.zeros((2, 2), dtype=torch.complex128, device="cuda")
    st = kr.lib().kr_block_reduce_noalloc(10, 2, ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(Y.data_ptr()), 1,
                                          ctypes.c_void_p(out.data_ptr()), None)
    assert st == 6  # KR_BAD_ARG, before any GPU work
    assert "device memory" in kr.kr_last_error()


def test_noalloc_rejects_width_beyond_scratch(kr):
    Y = torch.zeros((10, 17), dtype=torch.complex128, device="cuda")
    out = torch.zeros((17, 17), dtype=torch.complex128, device="cuda")
    st = kr.lib().kr_block_reduce_noalloc(10, 17, ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                          1, ctypes.c_void_p(out.data_ptr()), None)
    assert st == 9  # KR_UNSUPPORTED
    assert "s must be in [1, 16]" in kr.kr_last_error()
