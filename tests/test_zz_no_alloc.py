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
