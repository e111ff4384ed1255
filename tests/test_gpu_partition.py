"""The partitioned core update on the GPU (needs a GB300): one problem split over two (and
three) library handles in one process, each on a slab of the largest non-updated mode; the
exchange steps (sum of the partial d, sum of the partial line-search denominators) are host
sums between the phases, as an all-reduce across GPUs would make them.  After updates of every
core the handles hold identical cores equal to the unpartitioned oracle update, within the
per-step tolerance of each precision (FP64 1e-10, FP32 1e-5, BF16 5e-3)."""
import numpy as np
import pytest

from oracle import trd_oracle as O

from .helpers import flat, problem, rel

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5, "tf32x3": 1e-5, "bf16": 5e-3}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_09044_gb300 import build
    build.build()
    return torch


@pytest.mark.parametrize("prec,nparts,sketched", [("fp64", 2, False), ("fp32", 2, False), ("fp32", 3, True),
                                                  ("tf32x3", 2, False), ("bf16", 2, False), ("bf16", 2, True)])
def test_partitioned_update_equals_unpartitioned(torch_cuda, prec, nparts, sketched):
    from paper_2305_09044_gb300 import TRD
    from paper_2305_09044_gb300 import partition as PT
    dims, ranks = (48, 40, 36, 32), (4, 3, 4, 2)
    X, P, words, truth, Xt = problem(dims, ranks, 0.3, 0.1, 71)
    Xd = torch_cuda.from_numpy(flat(X)).cuda()
    Md = torch_cuda.from_numpy(words.view(np.int32)).cuda()
    cores = O.init_cores(dims, ranks, seed=72)
    hs = []
    for _ in range(nparts):
        t = TRD(dims, ranks, prec)
        t.set_data(Xd, Md)
        t.set_cores(cores)
        hs.append(t)
    tol = TOL[prec]
    sigma = 1.4
    for k in range(4):
        sk = ([None if m == k else O.draw_indices(9, 0, k, m, 4, dims[m], 16) for m in range(4)]
              if sketched else None)
        st = O.core_update(X, P, cores, k, sigma, lam=-1e-10, sample=sk)
        pus = [PT.PartitionedUpdate(t, k, p, nparts, sigma, sketch=sk) for p, t in enumerate(hs)]
        parts = [pu.partial_gradient() for pu in pus]
        d = sum(parts)
        assert rel(d, st.d) <= tol, (k, rel(d, st.d))
        assert sum(pu.stats["n_obs"] for pu in pus) == st.n_obs
        den = sum(pu.partial_denominator(d) for pu in pus)
        etas = [pu.apply(den) for pu in pus]
        for e in etas:
            assert abs(e - st.eta) <= tol * abs(st.eta), (k, e, st.eta)
        new = [t.get_core(k) for t in hs]
        for z in new[1:]:
            assert np.array_equal(z, new[0])             # replicated cores stay identical
        assert rel(new[0] - cores[k], st.cores[k] - cores[k]) <= tol
        cores = st.cores
        for t in hs:                                     # continue from the oracle's state
            t.set_core(k, cores[k])
