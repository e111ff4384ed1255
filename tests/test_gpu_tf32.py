"""Parity of the FP32-accurate tensor-core path (TF32 operands, 3-term split of both
operands in every product of both data passes) with the FP64 oracle (needs a GB300).

Tolerance: the FP32 contract, 1e-5 relative (Frobenius) per step for d, eta and the core
change, from identical state.  Shapes cover contractions up to 64 wide (on the tensor cores),
ragged tiles everywhere, an inner block size that is not a multiple of 4, both orientations
of the stationary block, and contractions wider than 64 (the FP32 CUDA-core passes take
them).
"""
import math

import numpy as np
import pytest

from oracle import trd_oracle as O

from .helpers import flat, problem, rel

pytestmark = pytest.mark.gpu

TOL = 1e-5

SHAPES = [
    ((48, 40, 36, 32), (8, 8, 8, 8)),       # K' = 64
    ((23, 17, 9, 13), (2, 3, 4, 3)),        # odd inner block, K' = 8 / 6
    ((64, 40, 36), (8, 8, 8)),              # order 3, one ragged stationary block
    ((20, 16, 12, 10, 9), (2, 3, 2, 2, 3)), # order 5
    ((52, 44, 30, 28), (4, 3, 4, 2)),       # small ranks, 2288 x 840
    ((24, 20, 18, 16), (10, 10, 10, 10)),   # K' = 100: CUDA-core FP32 passes
    ((24, 20, 18), (16, 16, 16)),           # K' = 256: CUDA-core FP32 passes
]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_09044_gb300 import build
    build.build()
    return torch


def _make(torch, dims, ranks, missing=0.3, outliers=0.1, seed=5):
    from paper_2305_09044_gb300 import TRD
    X, P, words, truth, Xt = problem(dims, ranks, missing, outliers, seed)
    t = TRD(dims, ranks, "tf32x3")
    Xd = torch.from_numpy(flat(X)).cuda()
    Md = torch.from_numpy(words.view(np.int32)).cuda()
    t.set_data(Xd, Md)
    return t, X, P, Xt, (Xd, Md)


def _check_step(t, X, P, cores, k, sigma, sample=None, gram="global"):
    st = O.core_update(X, P, cores, k, sigma, lam=-1e-10, sample=sample, gram=gram)
    s = t.residual_weights(k, sigma)
    assert s["n_obs"] == st.n_obs
    assert abs(s["sum_w"] - st.sum_w) <= TOL * st.sum_w
    assert abs(s["sum_we2"] - 2 * st.objective) <= TOL * 2 * st.objective
    d = t.core_gradient(k)
    assert rel(d, st.d) <= TOL, (k, rel(d, st.d))
    eta = t.core_update(k, -1e-10, gram=gram)
    assert abs(eta - st.eta) <= TOL * abs(st.eta), (k, eta, st.eta)
    assert rel(t.get_core(k) - cores[k], st.cores[k] - cores[k]) <= TOL
    return st.cores


@pytest.mark.parametrize("dims,ranks", SHAPES)
def test_tf32x3_core_step_parity(torch_cuda, dims, ranks):
    t, X, P, Xt, keep = _make(torch_cuda, dims, ranks)
    cores = O.init_cores(dims, ranks, seed=11)
    for k in range(len(dims)):
        t.set_cores(cores)
        cores = _check_step(t, X, P, cores, k, 1.3)


@pytest.mark.parametrize("dims,ranks,s", [((16, 12, 12, 12, 12), (10, 10, 10, 10, 10), 8),
                                           ((40, 33, 29, 21), (3, 2, 4, 2), 7)])
def test_tf32x3_sketched_step_parity(torch_cuda, dims, ranks, s):
    """SAWRTRD: RStS gather by the specified draw, then the per-step checks on the sketch
    (order 5 with ranks 10 is the 64^5 workload's shape class, K' = 100)."""
    t, X, P, Xt, keep = _make(torch_cuda, dims, ranks, missing=0.5, seed=8)
    cores = O.init_cores(dims, ranks, seed=12)
    N = len(dims)
    for k in range(N):
        t.set_cores(cores)
        idx = [None if m == k else O.draw_indices(99, 0, k, m, N, dims[m], s) for m in range(N)]
        t.sample_subtensor(k, idx)
        cores = _check_step(t, X, P, cores, k, 2.0, sample=idx)


@pytest.mark.parametrize("gram", ["local", "none"])
def test_tf32x3_ablation_variants(torch_cuda, gram):
    dims, ranks, s = (30, 26, 24), (3, 2, 3), 12
    t, X, P, Xt, keep = _make(torch_cuda, dims, ranks, seed=9)
    cores = O.init_cores(dims, ranks, seed=13)
    for k in range(3):
        t.set_cores(cores)
        idx = [None if m == k else O.draw_indices(5, 0, k, m, 3, dims[m], s) for m in range(3)]
        t.sample_subtensor(k, idx)
        cores = _check_step(t, X, P, cores, k, 1.0, sample=idx, gram=gram)


def test_tf32x3_row_sampling(torch_cuda):
    from paper_2305_09044_gb300 import TRD
    dims, ranks, J = (24, 20, 16, 12), (3, 2, 3, 2), 700
    X, P, words, truth, Xt = problem(dims, ranks, 0.3, 0.1, 61)
    t = TRD(dims, ranks, "tf32x3")
    keep = (torch_cuda.from_numpy(flat(X)).cuda(), torch_cuda.from_numpy(words.view(np.int32)).cuda())
    t.set_data(*keep)
    cores = O.init_cores(dims, ranks, seed=9)
    for k in range(len(dims)):
        rows = O.draw_rows(5, 0, k, dims, J)
        t.set_cores(cores)
        t.sample_rows(k, rows)
        st = O.core_update_rows(X, P, cores, k, 1.4, rows, lam=-1e-10)
        s = t.residual_weights(k, 1.4)
        assert s["n_obs"] == st.n_obs
        assert rel(t.core_gradient(k), st.d) <= TOL
        eta = t.core_update(k, -1e-10)
        assert abs(eta - st.eta) <= TOL * abs(st.eta)
        assert rel(t.get_core(k) - cores[k], st.cores[k] - cores[k]) <= TOL
        cores = st.cores


def test_tf32x3_sigma_inf_least_squares(torch_cuda):
    """W = 1, no mask, lambda = 0: the step is the least-squares solution and eta = 1."""
    from paper_2305_09044_gb300 import TRD
    dims, ranks = (48, 40, 36, 32), (4, 4, 4, 4)
    X, P, words, truth, Xt = problem(dims, ranks, 0.0, 0.0, 3)
    t = TRD(dims, ranks, "tf32x3")
    Xd = torch_cuda.from_numpy(flat(X)).cuda()
    t.set_data(Xd, None)
    cores = O.init_cores(dims, ranks, seed=4)
    for k in range(4):
        t.set_cores(cores)
        st = O.core_update(X, np.ones_like(X), cores, k, math.inf, lam=0.0)
        s = t.residual_weights(k, math.inf)
        assert s["n_obs"] == X.size and abs(s["sum_w"] - X.size) < 1e-6 * X.size
        assert rel(t.core_gradient(k), st.d) <= TOL
        assert abs(t.core_update(k, 0.0) - 1.0) <= TOL
        cores = st.cores


def test_tf32x3_trajectory_matches_oracle(torch_cuda):
    """A few full AWRTRD iterations (adaptive width) on the TF32 tensor-core path: every
    step size within 1e-5 of the oracle's, the final model within 1e-5."""
    dims, ranks = (36, 30, 28, 24), (3, 3, 2, 2)
    t, X, P, Xt, keep = _make(torch_cuda, dims, ranks, missing=0.4, seed=21)
    cores = O.init_cores(dims, ranks, seed=77)
    t.set_cores(cores)
    D = O.D_matrix(cores)
    obs = P > 0
    rms = float(np.sqrt(np.mean(X[obs] ** 2)))
    sigma = None
    for it in range(4):
        sigma = O.adaptive_sigma((X - O.reconstruct(cores))[obs], rms, sigma)
        cores, e, D, steps = O.sawrtrd_iteration(X, P, cores, sigma, it, D_prev=D)
        r = t.step(sigma=-1.0)
        assert abs(r["sigma"] - sigma) <= 1e-5 * sigma
        for k in range(4):
            assert abs(r["eta"][k] - steps[k].eta) <= TOL * abs(steps[k].eta), (it, k)
    assert rel(O.reconstruct(t.get_cores()), O.reconstruct(cores)) <= TOL


def test_tf32x3_full_size_workload(torch_cuda):
    """The 100^4 rank-8 workload at full size in the benchmark's launch configuration: one
    update of core 1 (stationary inner block) and core 4 (stationary outer block)."""
    from paper_2305_09044_gb300 import TRD, synth
    w = synth.WORKLOADS["cfg100"]
    truth = synth.gaussian_cores(w.dims, w.ranks, w.data_seed)
    Xt = O.reconstruct_unfold(truth)
    c = synth.draw_corruption(w)
    X = synth.assemble(Xt, c).astype(np.float32)
    P = c.mask.astype(np.float64)
    t = TRD(w.dims, w.ranks, "tf32x3")
    Xd = torch_cuda.from_numpy(flat(X)).cuda()
    Md = torch_cuda.from_numpy(synth.pack_mask(c.mask).view(np.int32)).cuda()
    t.set_data(Xd, Md)
    X = X.astype(np.float64)
    del Xt
    cores = O.init_cores(w.dims, w.ranks, seed=w.init_seed)
    for k in (0, 3):
        t.set_cores(cores)
        cores = _check_step(t, X, P, cores, k, 2.0)
