"""Uniform row sampling (the paper's ablation, Sec. 5) on the GPU against the oracle: J
sampled rows of Z^{!=k}_[2] and the matching fibres of X along mode k, then the same
residual / weight / gradient / scaled-step / line-search path.  Tolerances as elsewhere:
FP64 1e-10, FP32 1e-5, BF16 5e-3 relative per step."""
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


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("dims,ranks,J", [((24, 20, 16, 12), (3, 2, 3, 2), 700),
                                           ((20, 16, 12, 8, 8), (2, 3, 2, 2, 3), 1500)])
def test_row_sampled_step_parity(torch_cuda, prec, dims, ranks, J):
    from paper_2305_09044_gb300 import TRD
    X, P, words, truth, Xt = problem(dims, ranks, 0.3, 0.1, 61)
    t = TRD(dims, ranks, prec)
    Xd = torch_cuda.from_numpy(flat(X)).cuda()
    Md = torch_cuda.from_numpy(words.view(np.int32)).cuda()
    t.set_data(Xd, Md)
    cores = O.init_cores(dims, ranks, seed=9)
    sigma = 1.4
    tol = TOL[prec]
    for k in range(len(dims)):
        rows = O.draw_rows(5, 0, k, dims, J)
        t.set_cores(cores)
        t.sample_rows(k, rows)
        st = O.core_update_rows(X, P, cores, k, sigma, rows, lam=-1e-10)
        s = t.residual_weights(k, sigma)
        assert s["n_slots"] == dims[k] * J and s["n_obs"] == st.n_obs
        d = t.core_gradient(k)
        assert rel(d, st.d) <= tol, (k, rel(d, st.d))
        eta = t.core_update(k, -1e-10)
        assert abs(eta - st.eta) <= tol * abs(st.eta), (k, eta, st.eta)
        assert rel(t.get_core(k) - cores[k], st.cores[k] - cores[k]) <= tol
        cores = st.cores


def test_row_sample_rejects_bad_rows(torch_cuda):
    from paper_2305_09044_gb300 import TRD, TrdError
    dims, ranks = (8, 6, 5), (2, 2, 2)
    X, P, words, truth, Xt = problem(dims, ranks, 0.3, 0.1, 62)
    t = TRD(dims, ranks, "fp32")
    t.set_data(torch_cuda.from_numpy(flat(X)).cuda(), torch_cuda.from_numpy(words.view(np.int32)).cuda())
    rows = O.draw_rows(1, 0, 0, dims, 10)
    rows[3, 2] = 5                      # I_3 = 5: out of range
    with pytest.raises(TrdError):
        t.sample_rows(0, rows)
