"""The partitioned core update (one problem split over handles, one exchange step per core
update) on the CPU: the orchestration in paper_2305_09044_gb300.partition driven with an
oracle-backed stand-in for the library handle, one part per process.

Checked against the unpartitioned oracle update (Eq. hatd, Eq. hI and the exact line search
of Sec. 3.2 are column sums, so the parts must reproduce it to rounding): the cores after
updates of every core, on the full tensor and on an RStS sketch, for 2 and 3 parts in one
process, and for 2 gloo ranks (world size 2, 127.0.0.1) exchanging through
torch.distributed."""
import math
import os
import socket

import numpy as np
import pytest

from oracle import trd_oracle as O
from paper_2305_09044_gb300 import partition as PT


class OracleHandle:
    """Stand-in for binding.TRD on one part, computed by the FP64 oracle (test only)."""

    def __init__(self, X, P, cores):
        self.X, self.P, self.cores = X, P, [c.copy() for c in cores]
        self.dims = list(X.shape)
        self.N = len(self.dims)

    def K(self, k):
        return self.cores[k].shape[0] * self.cores[k].shape[2]

    def sample_subtensor(self, k, idx):
        self.idx = [np.arange(self.dims[m]) if (m == k or idx[m] is None) else np.asarray(idx[m])
                    for m in range(self.N)]

    def _sub(self, k):
        XI = self.X[np.ix_(*self.idx)]
        PI = self.P[np.ix_(*self.idx)]
        cs = [self.cores[m][:, self.idx[m], :] for m in range(self.N)]
        B = O.cyclic_unfold2(O.subchain(cs, k))
        return O.unfold_k(XI, k), O.unfold_k(PI, k), B

    def residual_weights(self, k, sigma):
        self.sigma = sigma
        Xk, Pk, B = self._sub(k)
        E = Xk - O.mode2(self.cores[k]) @ B.T
        W = O.hq_weight(E, sigma)
        self.d = (W * Pk * E) @ B
        obs = Pk > 0
        return {"n_obs": int(obs.sum()), "sum_w": float(W[obs].sum()), "sum_we2": float((W * Pk * E * E).sum())}

    def core_gradient(self, k):
        return self.d.copy()

    def set_gradient(self, k, d):
        self.d = np.array(d)

    def line_search_terms(self, k, lam, gram):
        assert gram == "global"
        G = O.fgmc_gram(self.cores, k)
        self.h = O.right_solve_spd(self.d, G + O.resolve_lambda(lam, G) * np.eye(G.shape[0]))
        Xk, Pk, B = self._sub(k)
        W = O.hq_weight(Xk - O.mode2(self.cores[k]) @ B.T, self.sigma)
        HB = self.h @ B.T
        return float(np.sum(self.d * self.h)), float(np.sum(W * Pk * HB * HB))

    def core_update(self, k, lam, eta, gram):
        Z = self.cores[k]
        self.cores[k] = O.fold2(O.mode2(Z) + eta * self.h, Z.shape[0], Z.shape[2])


def _problem(seed=3, dims=(9, 8, 11, 7), ranks=(2, 3, 2, 2)):
    rng = np.random.default_rng(seed)
    N = len(dims)
    cores = [rng.standard_normal((ranks[k], dims[k], ranks[(k + 1) % N])) * 0.8 for k in range(N)]
    X = O.reconstruct([rng.standard_normal(c.shape) * 0.8 for c in cores]) + 0.1 * rng.standard_normal(dims)
    X[rng.random(dims) < 0.1] = 7.0                      # a few outliers
    P = (rng.random(dims) < 0.7).astype(np.float64)
    return X, P, cores


def _sketch(dims, k, seed):
    return [None if m == k else O.draw_indices(seed, 0, k, m, len(dims), dims[m], max(3, dims[m] // 2))
            for m in range(len(dims))]


def test_split_mode_and_ranges():
    assert PT.part_range(10, 0, 3) == (0, 3) and PT.part_range(10, 2, 3) == (6, 10)
    assert PT.split_mode((9, 8, 11, 7), 2) == 0 and PT.split_mode((9, 8, 11, 7), 0) == 2
    idx = PT.part_indices((9, 8, 11, 7), 0, 1, 2)
    assert idx[0] is None and idx[1] is None and idx[3] is None and list(idx[2]) == list(range(5, 11))
    sk = [None, [1, 4, 6], [0, 2, 3, 9], [5]]
    idx = PT.part_indices((9, 8, 11, 7), 0, 0, 2, sk)
    assert list(idx[2]) == [0, 2] and list(idx[1]) == [1, 4, 6] and list(idx[3]) == [5]
    with pytest.raises(ValueError):
        PT.PartitionedUpdate(OracleHandle(*_problem()), 0, 0, 12, 1.0)   # 11 indices, 12 parts


@pytest.mark.parametrize("nparts", [2, 3])
@pytest.mark.parametrize("sketched", [False, True])
def test_parts_in_one_process_equal_unpartitioned_update(nparts, sketched):
    X, P, cores = _problem()
    hs = [OracleHandle(X, P, cores) for _ in range(nparts)]
    ref = [c.copy() for c in cores]
    sigma = 1.5
    for k in range(4):
        sk = _sketch(X.shape, k, 17) if sketched else None
        st = O.core_update(X, P, ref, k, sigma, lam=-1e-10, sample=sk)
        ref = st.cores
        pus = [PT.PartitionedUpdate(h, k, p, nparts, sigma, sketch=sk) for p, h in enumerate(hs)]
        d = sum(pu.partial_gradient() for pu in pus)
        assert np.linalg.norm(d - st.d) <= 1e-12 * np.linalg.norm(st.d)
        assert sum(pu.stats["n_obs"] for pu in pus) == st.n_obs
        den = sum(pu.partial_denominator(d) for pu in pus)
        assert abs(den - st.den) <= 1e-12 * st.den
        etas = [pu.apply(den) for pu in pus]
        assert all(abs(e - st.eta) <= 1e-12 * st.eta for e in etas)
        for h in hs:
            assert np.linalg.norm(h.cores[k] - ref[k]) <= 1e-12 * np.linalg.norm(ref[k])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port)})
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, P, cores = _problem(seed=5)
        h = OracleHandle(X, P, cores)
        red = PT.torch_allreduce()
        etas = []
        for it in range(2):
            for k in range(4):
                sk = _sketch(X.shape, k, 100 + it) if it == 1 else None
                etas.append(PT.partitioned_core_update(h, k, 1.2, red, rank, world, sketch=sk)["eta"])
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.concatenate([c.ravel() for c in h.cores] + [etas]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_equal_unpartitioned_update(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    X, P, cores = _problem(seed=5)
    ref, etas = [c.copy() for c in cores], []
    for it in range(2):
        for k in range(4):
            sk = _sketch(X.shape, k, 100 + it) if it == 1 else None
            st = O.core_update(X, P, ref, k, 1.2, lam=-1e-10, sample=sk)
            ref, _ = st.cores, etas.append(st.eta)
    want = np.concatenate([c.ravel() for c in ref] + [etas])
    got = [np.load(os.path.join(tmp_path, f"rank{r}.npy")) for r in range(world)]
    assert np.array_equal(got[0], got[1])                 # the ranks hold identical cores
    assert np.linalg.norm(got[0] - want) <= 1e-11 * np.linalg.norm(want)
