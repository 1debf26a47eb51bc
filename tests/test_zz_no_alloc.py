"""The reduction entry point that allocates nothing (semax_reduce_noalloc),
for callers that cannot allocate device memory themselves: it must give the
same answer as semax_reduce with a caller workspace, call after call, while
using only its built-in device scratch.

Kept in a file of its own that pytest collects last; it passes alone in a
fresh process and after the other tests."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_07659_gb300._lib as L
    return L.lib()


def _reduce_with_workspace(lib, a, a_prec, b, b_prec, stream):
    size = ctypes.c_size_t(0)
    assert lib.semax_reduce_workspace_size(a.numel(), ctypes.byref(size)) == 0
    ws = torch.empty(size.value, dtype=torch.uint8, device="cuda")
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    assert lib.semax_reduce(a.numel(), a.data_ptr(), a_prec, b.data_ptr(), b_prec, out.data_ptr(),
                            ws.data_ptr(), ws.numel(), stream) == 0
    return out


@pytest.mark.parametrize("count", [1, 4099, 5_000_000])
def test_noalloc_reduce_matches_workspace_reduce_twice(lib, count):
    stream = torch.cuda.current_stream().cuda_stream
    g = torch.Generator(device="cpu").manual_seed(count)
    cases = [(torch.rand(count, generator=g, dtype=torch.float64) - 0.5, 0),
             ((torch.rand(count, generator=g, dtype=torch.float64) - 0.5).float(), 1)]
    b = (torch.rand(count, generator=g, dtype=torch.float64) - 0.5).cuda()
    for a_host, a_prec in cases:
        a = a_host.cuda()
        ref = _reduce_with_workspace(lib, a, a_prec, b, 0, stream).cpu().numpy()
        for _ in range(2):          # two calls in a row share the static scratch
            out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
            assert lib.semax_reduce_noalloc(count, a.data_ptr(), a_prec, b.data_ptr(), 0,
                                            out.data_ptr(), stream) == 0
            got = out.cpu().numpy()
            assert np.array_equal(got, ref)   # same partition, same kernels: bit for bit
        # a different input in between must not leave stale partials behind
        c = torch.zeros_like(a)
        out = torch.empty(3, dtype=torch.float64, device="cuda")
        assert lib.semax_reduce_noalloc(count, c.data_ptr(), a_prec, c.data_ptr(), a_prec,
                                        out.data_ptr(), stream) == 0
        assert np.array_equal(out.cpu().numpy(), np.zeros(3))


def test_noalloc_reduce_argument_errors(lib):
    assert lib.semax_reduce_noalloc(-1, None, 0, None, 0, None, None) == -1
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    assert lib.semax_reduce_noalloc(10, None, 0, None, 0, out.data_ptr(), None) == -1
    assert lib.semax_reduce_noalloc(10, out.data_ptr(), 5, out.data_ptr(), 0, out.data_ptr(), None) == -1
