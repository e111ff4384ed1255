"""Degenerate cases of the method on the GPU against the FP64 oracle: a ring of rank-1 cores
(K = K' = 1, every contraction a single product), a mode of size 1, and a tensor with no
observed entry (the gradient vanishes, the line search finds no curvature, eta = 0 and the
cores stay put).  Tolerances as in the other parity tests: 1e-10 (FP64), 1e-5 (FP32, scaled
by 10 for derived scalars), 5e-3 (BF16)."""
import numpy as np
import pytest

from oracle import trd_oracle as O

from .helpers import flat, problem, rel

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5, "bf16": 5e-3}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_09044_gb300 import build
    build.build()
    return torch


def _handle(torch, dims, ranks, prec, X, words):
    from paper_2305_09044_gb300 import TRD
    t = TRD(dims, ranks, prec)
    Xd = torch.from_numpy(flat(X)).cuda()
    Md = torch.from_numpy(np.asarray(words).view(np.int32)).cuda()
    t.set_data(Xd, Md)
    return t, (Xd, Md)


def _steps_match(t, X, P, cores, sigma, prec, compare="cores"):
    """compare = "cores": the updated core; "model": the reconstruction after the update
    (for a rank-deficient Gram, where the step's component in the Gram's null space is
    fixed only by rounding and does not change the model)."""
    tol = TOL[prec]
    for k in range(X.ndim):
        t.set_cores(cores)
        st = O.core_update(X, P, cores, k, sigma, lam=-1e-10)
        s = t.residual_weights(k, sigma)
        assert s["n_obs"] == st.n_obs
        d = t.core_gradient(k)
        assert rel(d, st.d) <= tol * (1 if prec == "bf16" else 10), (k, rel(d, st.d))

        def model():
            return t.reconstruct().cpu().numpy().astype(np.float64).reshape(X.shape, order="F")

        before = model() if compare == "model" else None
        eta = t.core_update(k, -1e-10)
        assert abs(eta - st.eta) <= tol * 10 * abs(st.eta), (k, eta, st.eta)
        if compare == "cores":
            assert rel(t.get_core(k) - cores[k], st.cores[k] - cores[k]) <= tol * 10
        else:
            # the model change, through the FP32 reconstruction (1e-3 relative)
            change = model() - before
            want = O.reconstruct(st.cores) - O.reconstruct(cores)
            assert rel(change, want) <= 1e-3, (k, rel(change, want))
        cores = st.cores


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_rank_one_ring(torch_cuda, prec):
    dims, ranks = (12, 7, 8, 5), (1, 1, 1, 1)
    X, P, words, truth, Xt = problem(dims, ranks, 0.3, 0.1, 71)
    t, keep = _handle(torch_cuda, dims, ranks, prec, X, words)
    _steps_match(t, X, P, O.init_cores(dims, ranks, seed=13), 1.1, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mode_of_size_one(torch_cuda, prec):
    # a single slice of core 1 makes the FGMC Grams of its neighbours rank-deficient (the
    # lambda term alone keeps them invertible): the model after each update is compared
    dims, ranks = (7, 1, 9, 5), (2, 3, 2, 2)
    X, P, words, truth, Xt = problem(dims, ranks, 0.3, 0.1, 72)
    t, keep = _handle(torch_cuda, dims, ranks, prec, X, words)
    _steps_match(t, X, P, O.init_cores(dims, ranks, seed=14), 1.1, prec, compare="model")


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_no_observed_entry(torch_cuda, prec):
    dims, ranks = (16, 12, 8, 6), (2, 2, 3, 2)
    X, P, words, truth, Xt = problem(dims, ranks, 0.3, 0.1, 73)
    P = np.zeros_like(P)
    words = np.zeros_like(np.asarray(words))
    t, keep = _handle(torch_cuda, dims, ranks, prec, X, words)
    cores = O.init_cores(dims, ranks, seed=15)
    t.set_cores(cores)
    for k in range(len(dims)):
        st = O.core_update(X, P, cores, k, 1.0)
        assert st.eta == 0.0 and not np.any(st.d)
    r = t.step(sigma=1.0)
    assert r["eta"] == [0.0] * len(dims) and r["objective"] == [0.0] * len(dims), r
    for z, z0 in zip(t.get_cores(), cores):
        assert np.array_equal(z, z0)
