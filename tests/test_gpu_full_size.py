"""The sketched workloads at their full sizes, in the benchmark's launch configuration, on
sampled outputs the oracle can compute: one RStS core update per listed core from identical
state, against the FP64 oracle on the same sketch (the oracle gathers X_I from the same
host tensor).  64^5 rank 10 (4.3 GB, sketch 24 per non-updated mode, K' = 100) on the
tensor-core paths; 1024 x 1024 x 256 rank 16 (sketch 128, K' = 256) on the FP32 path and the
BF16 tensor-core path.

Tolerances: BF16 5e-3, FP32 1e-5 relative per step (d, eta, core change).
"""
import functools

import numpy as np
import pytest

from oracle import trd_oracle as O

from .helpers import big_problem, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_09044_gb300 import build
    build.build()
    return torch


@functools.lru_cache(maxsize=1)
def _problem(name, cut, cols):
    from paper_2305_09044_gb300 import synth
    return big_problem(synth.WORKLOADS[name], cut, cols)


def _run(torch, w, prec, cut, cols, ks, sigma, tol):
    from paper_2305_09044_gb300 import TRD, synth
    X, mask, truth = _problem(w.name, cut, cols)
    dims, N = tuple(w.dims), len(w.dims)
    t = TRD(dims, w.ranks, prec)
    Xd = torch.from_numpy(X).cuda()
    Md = torch.from_numpy(synth.pack_mask(mask).view(np.int32)).cuda()
    t.set_data(Xd, Md)
    Xv = X.reshape(dims, order="F")
    Pv = mask.reshape(dims, order="F")
    cores = O.init_cores(dims, w.ranks, seed=w.init_seed)
    for k in ks:
        t.set_cores(cores)
        sample = [None if j == k else O.draw_indices(w.sample_seed, 0, k, j, N, dims[j], w.sketch)
                  for j in range(N)]
        t.sample_subtensor(k, sample)
        st = O.core_update(Xv, Pv, cores, k, sigma, lam=-1e-10, sample=sample)
        s = t.residual_weights(k, sigma)
        assert s["n_slots"] == dims[k] * w.sketch ** (N - 1) and s["n_obs"] == st.n_obs
        d = t.core_gradient(k)
        assert rel(d, st.d) <= tol, (k, rel(d, st.d))
        eta = t.core_update(k, -1e-10)
        assert abs(eta - st.eta) <= tol * abs(st.eta), (k, eta, st.eta)
        assert rel(t.get_core(k) - cores[k], st.cores[k] - cores[k]) <= tol
        cores = st.cores
    t.close()


def test_full_size_64x5_rank10_sketched_bf16(torch_cuda):
    from paper_2305_09044_gb300 import synth
    w = synth.WORKLOADS["cfg64"]
    _run(torch_cuda, w, "bf16", cut=2, cols=16384, ks=(0, 2, 4), sigma=3.0, tol=5e-3)


def test_full_size_64x5_rank10_sketched_tf32x3(torch_cuda):
    """64^5 rank 10 (K' = 100) with TF32 operands: the FP32 CUDA-core passes take it."""
    from paper_2305_09044_gb300 import synth
    w = synth.WORKLOADS["cfg64"]
    _run(torch_cuda, w, "tf32x3", cut=2, cols=16384, ks=(0, 2), sigma=3.0, tol=1e-5)


def test_full_size_video_rank16_sketched_fp32(torch_cuda):
    from paper_2305_09044_gb300 import synth
    w = synth.WORKLOADS["video"]
    _run(torch_cuda, w, "fp32", cut=1, cols=16384, ks=(0, 2), sigma=1.5, tol=1e-5)


def test_full_size_video_rank16_sketched_bf16(torch_cuda):
    """The same 1024 x 1024 x 256 rank-16 workload (K' = 256) on the tensor-core path."""
    from paper_2305_09044_gb300 import synth
    w = synth.WORKLOADS["video"]
    _run(torch_cuda, w, "bf16", cut=1, cols=16384, ks=(0, 2), sigma=1.5, tol=5e-3)


def test_full_size_video_rank16_sketched_tf32x3(torch_cuda):
    """K' = 256 with TF32 operands: the FP32 CUDA-core passes take the contraction."""
    from paper_2305_09044_gb300 import synth
    w = synth.WORKLOADS["video"]
    _run(torch_cuda, w, "tf32x3", cut=1, cols=16384, ks=(0,), sigma=1.5, tol=1e-5)
