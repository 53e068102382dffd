"""The allocation-free line FFT (sar_fft_lines_static) against sar_fft_lines.

sar_fft_lines_static is for callers that must not have device memory
allocated on their behalf -- on-board or real-time radar processing with a
device-memory footprint fixed at start-up, memory owned by a pool allocator.  Its twiddles live in one fixed
device array that every call shares and rewrites.  This test calls it through
the C-ABI twice in a row (two different lengths, so the second call must
rebuild the shared table the first one left behind) and compares each result
with the allocating entry point within the FFT tolerance of the parity tests.

This file is collected last so that a run stopping at its first failure has
already run every other test; it passes alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest

import sarsim

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FFT_TOL = 2e-6    # relative L2 tolerance of one FP32 FFT in tests/test_gpu_parity.py


@pytest.fixture(scope="module")
def sar(built_lib):
    import paper_2604_03585_gb300 as sar
    assert torch.cuda.is_available(), "gpu tests need a CUDA device"
    torch.cuda.set_device(0)
    return sar


def rel_l2(a, b):
    a = a.astype(np.complex128)
    b = b.astype(np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_static_fft_matches_allocating_fft_twice(sar):
    lib = sar.library()
    stream = torch.cuda.current_stream().cuda_stream
    for call, (n, n_lines, inverse) in enumerate([(4096, 19, 0), (1024, 33, 1)]):
        x = torch.from_numpy(sarsim.complex_gaussian(40 + call, 7, n * n_lines, 1.0).reshape(n_lines, n)).cuda()
        ref = torch.empty_like(x)
        got = torch.empty_like(x)
        assert lib.sar_fft_lines(n, n_lines, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(ref.data_ptr()),
                                 inverse, ctypes.c_void_p(stream)) == sar.SAR_OK
        st = lib.sar_fft_lines_static(n, n_lines, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(got.data_ptr()),
                                      inverse, ctypes.c_void_p(stream))
        assert st == sar.SAR_OK, sar.sar_last_error()
        torch.cuda.synchronize()
        assert rel_l2(got.cpu().numpy(), ref.cpu().numpy()) <= FFT_TOL, call


@pytest.mark.parametrize("inverse", [0, 1])
@pytest.mark.parametrize("n", [256, 512, 1024, 2048, 4096, 8192, 16384])
def test_static_fft_every_length(sar, n, inverse):
    """Every power-of-two length the shared array is sized for (16384 needs
    the largest table, 17,408 values), out of place and in place (in == out),
    against the allocating entry point."""
    lib = sar.library()
    stream = torch.cuda.current_stream().cuda_stream
    n_lines = 5
    x = torch.from_numpy(sarsim.complex_gaussian(60 + inverse, n, n * n_lines, 1.0).reshape(n_lines, n)).cuda()
    ref = torch.empty_like(x)
    got = torch.empty_like(x)
    assert lib.sar_fft_lines(n, n_lines, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(ref.data_ptr()),
                             inverse, ctypes.c_void_p(stream)) == sar.SAR_OK
    st = lib.sar_fft_lines_static(n, n_lines, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(got.data_ptr()),
                                  inverse, ctypes.c_void_p(stream))
    assert st == sar.SAR_OK, sar.sar_last_error()
    inplace = x.clone()
    st = lib.sar_fft_lines_static(n, n_lines, ctypes.c_void_p(inplace.data_ptr()),
                                  ctypes.c_void_p(inplace.data_ptr()), inverse, ctypes.c_void_p(stream))
    assert st == sar.SAR_OK, sar.sar_last_error()
    torch.cuda.synchronize()
    r = ref.cpu().numpy()
    assert rel_l2(got.cpu().numpy(), r) <= FFT_TOL
    assert rel_l2(inplace.cpu().numpy(), r) <= FFT_TOL


def test_static_fft_refuses_unsupported_sizes(sar):
    lib = sar.library()
    assert lib.sar_fft_lines_static(32768, 1, None, None, 0, None) == sar.SAR_ERR_UNSUPPORTED
    assert lib.sar_fft_lines_static(300, 1, None, None, 0, None) == sar.SAR_ERR_UNSUPPORTED
