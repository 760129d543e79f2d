"""lbm_field_sum_noalloc: the sum entry point that allocates nothing.

It serves callers that may not allocate device memory at the point where they need a
sum (a fixed, pre-planned memory budget; a framework that forbids cudaMalloc/cudaFree
on its hot path).  Its scratch is an array compiled into the library.  The GPU test
checks it, through the C ABI, against the existing lbm_reduce on two consecutive calls.
This file is collected last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1507_07294_gb300 import inputs as I
from paper_1507_07294_gb300 import lbm as L


def test_rejects_bad_arguments_without_a_gpu():
    lib = L.load_library()
    out = (ctypes.c_double * 2)()
    assert lib.lbm_field_sum_noalloc(None, -1, ctypes.cast(out, ctypes.c_void_p), None) == L.LBM_EINVAL
    assert "outside" in lib.lbm_last_error(None).decode()
    assert lib.lbm_field_sum_noalloc(None, 2 ** 31, ctypes.cast(out, ctypes.c_void_p), None) == L.LBM_EINVAL
    assert "outside" in lib.lbm_last_error(None).decode()
    assert lib.lbm_field_sum_noalloc(None, 10, None, None) == L.LBM_EINVAL
    assert lib.lbm_field_sum_noalloc(None, 10, ctypes.cast(out, ctypes.c_void_p), None) == L.LBM_EINVAL


@pytest.mark.gpu
def test_matches_lbm_reduce_on_two_calls_in_a_row():
    """Sum of phi by the no-allocation entry point vs sum_phi of lbm_reduce, for two
    problems one right after the other on the shared scratch.  The second array is
    smaller (fewer partial sums) than the first, so partials left over from the first
    call would show in the second result."""
    import torch

    lib = L.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    problems = [
        I.perturbed(I.rayleigh_taylor(W=24, nz=40, Re=200.0), seed=13, phi_amp=0.05, u_amp=0.01),
        I.perturbed(I.droplet(n=14, R=4.0), seed=14, u_amp=0.01),
    ]
    sums = []
    for w in problems:
        with L.Solver(w, stream=stream) as s:
            s.step(5)
            ref_sum, _ = s.reduce()
            phi = s.fields(L.LBM_FIELD_PHI)["phi"].astype(np.float32).ravel()
        x = torch.from_numpy(phi).to("cuda")
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.lbm_field_sum_noalloc(ctypes.c_void_p(x.data_ptr()), x.numel(),
                                       ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert st == L.LBM_OK, lib.lbm_last_error(None).decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # the same FP32 values summed in FP64, possibly in another order
        assert abs(got[0] - ref_sum) <= 1e-12 * float(np.abs(phi).sum()) + 1e-12
        assert got[1] == 0.0
        sums.append(got[0])
    assert abs(sums[0] - sums[1]) > 1.0


@pytest.mark.gpu
def test_grid_stride_and_the_largest_admitted_size():
    """Arrays longer than 1024 blocks x 256 threads, so each block of the fixed grid
    strides over several elements, down to n = 2^31 - 1, the largest size the entry
    point admits (an 8.6 GB FP32 array): the 64-bit stride must neither wrap nor skip
    the last element."""
    import torch

    lib = L.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.empty(2, dtype=torch.float64, device="cuda")

    def call(x, n):
        st = lib.lbm_field_sum_noalloc(ctypes.c_void_p(x.data_ptr()), n,
                                       ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert st == L.LBM_OK, lib.lbm_last_error(None).decode()
        torch.cuda.synchronize()
        return out.cpu().numpy()

    gen = torch.Generator(device="cuda").manual_seed(5)
    for n in (1024 * 256 + 1, 3 * 1024 * 256 + 77, 40_000_003):
        x = torch.rand(n, generator=gen, device="cuda", dtype=torch.float32) - 0.25
        x[n // 3] = float("inf")
        got = call(x, n - 1)  # the last element is outside the summed range
        assert got[1] == 1.0
        x[n // 3] = 0.0
        ref = float(x[: n - 1].double().sum())
        got = call(x, n - 1)
        assert got[1] == 0.0
        assert abs(got[0] - ref) <= 1e-12 * float(x.abs().double().sum())
        del x

    n = 2 ** 31 - 1
    free, _ = torch.cuda.mem_get_info()
    if free < 4 * n + (2 << 30):
        pytest.skip("not enough free device memory for a 2^31 - 1 element array")
    x = torch.full((n,), 0.25, dtype=torch.float32, device="cuda")
    x[-1] = 1.0
    got = call(x, n)
    # every partial sum is a multiple of 1/4 below 2^30: exact in FP64
    assert got[0] == (n - 1) * 0.25 + 1.0
    assert got[1] == 0.0
    x[-1] = float("nan")
    assert call(x, n)[1] == 1.0
    del x
    torch.cuda.empty_cache()
