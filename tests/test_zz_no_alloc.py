"""The allocation-free width selection (trd_sigma_from_residuals_noalloc) gives the same
kernel width as the handle-based trd_sigma_from_residuals, twice in a row on the same
inputs, while the fixed device array it works in is shared between calls.

Callers of the allocation-free entry point cannot allocate device memory themselves (hosts
that own all device memory through their own allocator, fixed device-memory budgets, loops
that cannot take cudaMalloc's implicit synchronisation), which is why the entry point takes
no handle.  This file is collected last so a
run that stops at the first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_09044_gb300 import build, binding
    build.build()
    return torch, binding.load()


def test_noalloc_width_matches_handle_path(env):
    torch, lib = env
    from paper_2305_09044_gb300 import TRD
    t = TRD((4, 4, 4), (1, 1, 1), "fp32")
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(7)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for n in (1, 1000, 300_001, 1 << 20):
        r = rng.standard_normal(n).astype(np.float32) * 0.3
        r[: n // 10] *= 40.0
        rd = torch.from_numpy(r).cuda()
        for prev in (-1.0, 5.0):
            want = t.sigma_from_residuals(rd, 1.7, prev)
            for _ in range(2):                      # two calls in a row share the scratch
                out.fill_(-1.0)
                st = lib.trd_sigma_from_residuals_noalloc(C.c_void_p(rd.data_ptr()), n, 1.7, prev,
                                                          C.c_void_p(out.data_ptr()),
                                                          C.c_void_p(stream.cuda_stream))
                assert st == 0
                stream.synchronize()
                got = float(out.item())
                assert abs(got - want) <= 1e-12 * want, (n, prev, got, want)


def test_noalloc_rejects_oversize_and_bad_arguments(env):
    torch, lib = env
    rd = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.trd_sigma_from_residuals_noalloc(C.c_void_p(rd.data_ptr()), (1 << 20) + 1, 1.0, -1.0,
                                                C.c_void_p(out.data_ptr()), s) == 1
    assert lib.trd_sigma_from_residuals_noalloc(C.c_void_p(rd.data_ptr()), 0, 1.0, -1.0,
                                                C.c_void_p(out.data_ptr()), s) == 1
    assert lib.trd_sigma_from_residuals_noalloc(None, 16, 1.0, -1.0, C.c_void_p(out.data_ptr()), s) == 1
    assert lib.trd_sigma_from_residuals_noalloc(C.c_void_p(rd.data_ptr()), 16, float("nan"), -1.0,
                                                C.c_void_p(out.data_ptr()), s) == 1
