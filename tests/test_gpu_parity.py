"""GPU-vs-oracle parity of every hot-path step, through the C ABI (needs a GB300).

Per-step tests start each core update from identical cores (the oracle's), so every
reported difference belongs to that step alone.  Tolerances (relative Frobenius norm per
tensor): FP64 path 1e-10, FP32 path 1e-5; the FGMC Gram is FP64 on both paths (1e-12).
"""
import math

import numpy as np
import pytest

from oracle import trd_oracle as O

from .helpers import flat, problem, rel

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}

SHAPES = [
    # dims, ranks (mixed ranks, ragged tiles: no size is a multiple of the 64-wide tile)
    ((30, 30, 30), (3, 3, 3)),
    ((23, 17, 9, 13), (2, 3, 4, 3)),
    ((11, 7, 5, 6, 9), (2, 2, 3, 2, 2)),
    ((70, 65, 3), (4, 5, 2)),
]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_09044_gb300 import build
    build.build()
    return torch


def _make(torch, dims, ranks, prec, missing=0.3, outliers=0.1, seed=5):
    from paper_2305_09044_gb300 import TRD
    X, P, words, truth, Xt = problem(dims, ranks, missing, outliers, seed)
    t = TRD(dims, ranks, prec)
    Xd = torch.from_numpy(flat(X)).cuda()
    Md = torch.from_numpy(words.view(np.int32)).cuda()
    t.set_data(Xd, Md)
    return t, X, P, Xt, (Xd, Md)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dims,ranks", SHAPES)
def test_core_step_parity_full(torch_cuda, prec, dims, ranks):
    """AWRTRD (no sketch): residual/weights, gradient d, FGMC G, step size eta and the
    updated core, for every k, against the oracle from identical state."""
    t, X, P, Xt, keep = _make(torch_cuda, dims, ranks, prec)
    cores = O.init_cores(dims, ranks, seed=11)
    sigma = 1.3
    for k in range(len(dims)):
        t.set_cores(cores)
        st = O.core_update(X, P, cores, k, sigma, lam=-1e-10)
        s = t.residual_weights(k, sigma)
        assert s["n_obs"] == st.n_obs and s["n_slots"] == X.size
        assert abs(s["sum_w"] - st.sum_w) <= TOL[prec] * st.sum_w
        assert abs(s["sum_we2"] - 2 * st.objective) <= TOL[prec] * 2 * st.objective
        d = t.core_gradient(k)
        assert rel(d, st.d) <= TOL[prec], (k, rel(d, st.d))
        G = t.fgmc_gram(k)
        assert rel(G, st.G) <= 1e-12
        eta = t.core_update(k, -1e-10)
        assert abs(eta - st.eta) <= TOL[prec] * abs(st.eta), (eta, st.eta)
        Znew = t.get_core(k)
        assert rel(Znew - cores[k], st.cores[k] - cores[k]) <= TOL[prec]
        cores = st.cores


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dims,ranks,s", [((40, 33, 29, 21), (3, 2, 4, 2), 7),
                                           ((24, 20, 18, 16, 12), (2, 3, 2, 3, 2), 5)])
def test_core_step_parity_sketched(torch_cuda, prec, dims, ranks, s):
    """SAWRTRD: RStS gather with index sets drawn by the specified generator, then the same
    per-step checks on the sketch (G stays the global FGMC Gram)."""
    t, X, P, Xt, keep = _make(torch_cuda, dims, ranks, prec, missing=0.5, seed=8)
    cores = O.init_cores(dims, ranks, seed=12)
    N = len(dims)
    sigma = 2.0
    for k in range(N):
        t.set_cores(cores)
        idx = [None if m == k else O.draw_indices(99, 0, k, m, N, dims[m], s) for m in range(N)]
        t.sample_subtensor(k, idx)
        st = O.core_update(X, P, cores, k, sigma, lam=-1e-10, sample=idx)
        s_ = t.residual_weights(k, sigma)
        assert s_["n_slots"] == dims[k] * s ** (N - 1)
        assert s_["n_obs"] == st.n_obs
        d = t.core_gradient(k)
        assert rel(d, st.d) <= TOL[prec], (k, rel(d, st.d))
        eta = t.core_update(k, -1e-10)
        assert abs(eta - st.eta) <= TOL[prec] * abs(st.eta)
        assert rel(t.get_core(k), st.cores[k]) <= TOL[prec]
        assert rel(t.get_core(k) - cores[k], st.cores[k] - cores[k]) <= TOL[prec]
        cores = st.cores


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("gram", ["local", "none"])
def test_ablation_variants(torch_cuda, gram, prec):
    """Ablations of Sec. 5.1: 'local scaled term' (Gram of the sampled cores) and
    'gradient descent' (h = d) on a sketch, on every precision of the data passes."""
    dims, ranks, s = (30, 26, 24), (3, 2, 3), 12
    tol = {"fp64": 1e-10, "fp32": 1e-5, "bf16": 5e-3}[prec]
    t, X, P, Xt, keep = _make(torch_cuda, dims, ranks, prec, seed=9)
    cores = O.init_cores(dims, ranks, seed=13)
    for k in range(3):
        t.set_cores(cores)
        idx = [None if m == k else O.draw_indices(5, 0, k, m, 3, dims[m], s) for m in range(3)]
        t.sample_subtensor(k, idx)
        st = O.core_update(X, P, cores, k, 1.0, lam=-1e-10, sample=idx, gram=gram)
        t.residual_weights(k, 1.0)
        t.core_gradient(k)
        eta = t.core_update(k, -1e-10, gram=gram)
        assert abs(eta - st.eta) <= tol * abs(st.eta), (k, eta, st.eta)
        assert rel(t.get_core(k) - cores[k], st.cores[k] - cores[k]) <= tol
        cores = st.cores


def test_fixed_step_and_sigma_inf(torch_cuda):
    """sigma = inf gives W = 1 (Sec. 3.2 limit); a fixed step size bypasses the line search."""
    dims, ranks = (20, 18, 16), (2, 3, 2)
    t, X, P, Xt, keep = _make(torch_cuda, dims, ranks, "fp64")
    cores = O.init_cores(dims, ranks, seed=3)
    t.set_cores(cores)
    st = O.core_update(X, P, cores, 1, math.inf, lam=0.0, eta=0.37)
    s = t.residual_weights(1, math.inf)
    assert abs(s["sum_w"] - s["n_obs"]) < 1e-9
    assert rel(t.core_gradient(1), st.d) <= 1e-10
    assert abs(t.core_update(1, 0.0, eta=0.37) - 0.37) == 0.0
    assert rel(t.get_core(1), st.cores[1]) <= 1e-10


def test_init_cores_matches_generator(torch_cuda):
    from paper_2305_09044_gb300 import TRD
    dims, ranks = (9, 7, 5, 4), (2, 3, 4, 2)
    t = TRD(dims, ranks, "fp64")
    t.init_cores(2024)
    want = O.init_cores(dims, ranks, seed=2024)
    for k in range(4):
        assert rel(t.get_core(k), want[k]) <= 1e-14


@pytest.mark.parametrize("dims,ranks", [((30, 30, 30), (3, 3, 3)), ((12, 11, 10, 9), (2, 3, 2, 3))])
def test_reconstruct_and_recovery_error(torch_cuda, dims, ranks):
    from paper_2305_09044_gb300 import TRD
    rng = np.random.default_rng(4)
    cores = [rng.standard_normal((ranks[k], dims[k], ranks[(k + 1) % len(dims)])) for k in range(len(dims))]
    t = TRD(dims, ranks, "fp32")
    Xg = t.reconstruct_from(cores).cpu().numpy()
    Xo = flat(O.reconstruct(cores))
    assert rel(Xg, Xo) <= 1e-6
    t.set_cores(cores)
    ref = O.reconstruct(cores) * 1.01
    err = t.recovery_error(torch_cuda.from_numpy(flat(ref)).cuda())
    assert abs(err - 0.01 / 1.01) < 1e-6


def test_adaptive_sigma_selection_parity(torch_cuda):
    """The width rule has no pin in the paper (parity unpinned); GPU and oracle must agree
    on identical residuals: exact order statistics, type-7 quartiles, population std."""
    from paper_2305_09044_gb300 import TRD
    t = TRD((4, 4, 4), (1, 1, 1), "fp32")
    rng = np.random.default_rng(0)
    for n in [1, 2, 5, 1000, 4097, 300_001]:
        r = rng.standard_normal(n).astype(np.float32) * 0.3
        r[: n // 10] *= 50   # heavy tail
        rd = torch_cuda.from_numpy(r).cuda()
        for prev in [-1.0, 10.0]:
            got = t.sigma_from_residuals(rd, 1.7, prev)
            want = O.adaptive_sigma(r.astype(np.float64), 1.7, prev if prev > 0 else None)
            assert abs(got - want) <= 1e-12 * want, (n, got, want)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adaptive_sigma_on_tensor(torch_cuda, prec):
    dims, ranks = (30, 30, 30), (3, 3, 3)
    t, X, P, Xt, keep = _make(torch_cuda, dims, ranks, prec)
    cores = O.init_cores(dims, ranks, seed=2001)
    t.set_cores(cores)
    obs = P > 0
    want = O.adaptive_sigma((X - O.reconstruct(cores))[obs], float(np.sqrt(np.mean(X[obs] ** 2))))
    got = t.adaptive_sigma()
    assert abs(got - want) <= (1e-12 if prec == "fp64" else 1e-5) * want


def test_trajectory_tiny_fp64_adaptive(torch_cuda):
    """The 30^3 rank-3 workload (30 % missing, 10 % outliers), FP64, adaptive width, 100
    iterations of Algorithm 1 on the GPU against the oracle: per-iteration e and sigma
    track, and the final recovery errors differ by at most 1e-4."""
    from paper_2305_09044_gb300 import synth
    w = synth.WORKLOADS["tiny3"]
    dims, ranks = w.dims, w.ranks
    truth = synth.gaussian_cores(dims, ranks, w.data_seed)
    Xt = O.reconstruct_unfold(truth)
    c = synth.draw_corruption(w)
    X = synth.assemble(Xt, c).astype(np.float32).astype(np.float64)
    P = c.mask.astype(np.float64)
    from paper_2305_09044_gb300 import TRD
    t = TRD(dims, ranks, "fp64")
    Xd = torch_cuda.from_numpy(flat(X)).cuda()
    Md = torch_cuda.from_numpy(synth.pack_mask(c.mask).view(np.int32)).cuda()
    t.set_data(Xd, Md)
    t.init_cores(w.init_seed)
    cores = O.init_cores(dims, ranks, seed=w.init_seed)
    obs = P > 0
    rms = float(np.sqrt(np.mean(X[obs] ** 2)))
    D = O.D_matrix(cores)
    sigma = None
    for it in range(100):
        sigma = O.adaptive_sigma((X - O.reconstruct(cores))[obs], rms, sigma)
        cores, e, D, steps = O.sawrtrd_iteration(X, P, cores, sigma, it, D_prev=D)
        r = t.step(sigma=-1.0)
        assert abs(r["sigma"] - sigma) <= 1e-8 * sigma, (it, r["sigma"], sigma)
        assert abs(r["e"] - e) <= 1e-6 * max(e, 1e-12) + 1e-12, (it, r["e"], e)
    err_o = O.relative_error(cores, Xt)
    err_g = t.recovery_error(torch_cuda.from_numpy(flat(Xt)).cuda())
    assert abs(err_o - err_g) <= 1e-4, (err_o, err_g)


def test_trajectory_sketched_fp32(torch_cuda):
    """A sketched (SAWRTRD) trajectory in FP32: index draws inside trd_step follow the
    specified generator, so GPU and oracle see the same sketches."""
    dims, ranks = (36, 30, 28, 24), (3, 3, 2, 2)
    t, X, P, Xt, keep = _make(torch_cuda, dims, ranks, "fp32", missing=0.4, seed=21)
    cores = O.init_cores(dims, ranks, seed=77)
    t.set_cores(cores)
    sizes = [[dims[m] if m == k else 12 for m in range(4)] for k in range(4)]
    D = O.D_matrix(cores)
    for it in range(5):
        cores, e, D, steps = O.sawrtrd_iteration(X, P, cores, 1.5, it, sizes=sizes, seed=31, D_prev=D)
        r = t.step(sketch=[12] * 4, sigma=1.5, seed=31)
        for k in range(4):
            assert abs(r["eta"][k] - steps[k].eta) <= 1e-5 * abs(steps[k].eta), (it, k)
    assert rel(O.reconstruct(t.get_cores()), O.reconstruct(cores)) <= 1e-4


@pytest.mark.parametrize("prec,dims,ranks", [("fp64", (12, 10, 9, 8), (10, 10, 10, 10)),
                                             ("fp32", (10, 9, 8, 7), (8, 16, 8, 16)),
                                             ("fp32", (9, 8, 7, 6, 5), (11, 11, 11, 11, 11)),
                                             ("fp64", (8, 20, 120), (3, 20, 20)),
                                             ("fp64", (5, 24, 22, 6), (4, 12, 17, 4)),
                                             ("fp64", (40, 36, 3, 8), (20, 20, 3, 4)),
                                             ("fp64", (6, 30, 5, 24), (36, 36, 3, 3)),
                                             ("fp64", (4, 48, 6, 30), (46, 46, 2, 2))])
def test_scaled_step_large_gram(torch_cuda, prec, dims, ranks):
    """K = r_k r_{k+1} of 100, 128 and 121: the FP64 LDL^T factorisation and the
    row-parallel solves of the scaled step (Eq. sg, Eq. hI) at the Gram sizes of the 64^5 rank-10
    workload and beyond, against the oracle's Cholesky, from identical state.  K = 400 (the
    image ranks (3, 20, 20)) and 204 take the blocked multi-CTA Cholesky, both with a ragged
    last panel, and the FGMC factor of their r_k r_{k+1} > 128 cores comes from the tiled
    slice-Gram kernel (compared here through G^{!=k}, 1e-12).  Ranks (20, 20, 3, 4): the most
    balanced cut of the ring (through the two rank-20 edges, r_1 r_c = 400) is wider than the
    FP64 data pass takes, so the pass cuts through the rank-3 edge (r_1 r_c = 60).  K = 1296
    and 2116 (two large neighbouring ranks, as in the paper's video rank [80, 80, 3, 20]) take
    the wide back-contraction (8 and 32 outputs per thread) and the row solves with the factor
    read from L2."""
    t, X, P, Xt, keep = _make(torch_cuda, dims, ranks, prec)
    cores = O.init_cores(dims, ranks, seed=13)
    sigma = 2.0
    for k in range(len(dims)):
        t.set_cores(cores)
        st = O.core_update(X, P, cores, k, sigma, lam=-1e-10)
        t.residual_weights(k, sigma)
        d = t.core_gradient(k)
        assert rel(d, st.d) <= TOL[prec]
        assert rel(t.fgmc_gram(k), st.G) <= 1e-12
        eta = t.core_update(k, -1e-10)
        assert abs(eta - st.eta) <= TOL[prec] * abs(st.eta), (k, eta, st.eta)
        assert rel(t.get_core(k) - cores[k], st.cores[k] - cores[k]) <= TOL[prec]
        cores = st.cores


def test_video_rank_fp32(torch_cuda):
    """The paper's video rank [80, 80, 3, 20] on a small video-shaped tensor in FP32, against
    the oracle from identical state: the data pass cuts the ring through the rank-3 edge
    (r_1 r_c = 240), d (Eq. sd) of the K = 6400 and 1600 cores comes from the wide
    back-contraction, the FGMC Gram (Eq. FGMC) at K = 6400 and 1600 equals the explicit B^T B,
    and the updates (blocked Cholesky and row solves at K = 6400) give the oracle's step size.
    G is singular for the K = 6400 and 1600 cores here (1440 and 576 rows), so the test
    regularises with lambda = 1e-6 tr(G) / K and compares the step size of the better-posed
    K = 240 and 60 cores only."""
    dims, ranks = (8, 24, 3, 20), (80, 80, 3, 20)
    t, X, P, Xt, keep = _make(torch_cuda, dims, ranks, "fp32")
    cores = O.init_cores(dims, ranks, seed=11)
    sigma = 1.3
    for k in range(len(dims)):
        t.set_cores(cores)
        st = O.core_update(X, P, cores, k, sigma, gram="none")
        t.residual_weights(k, sigma)
        d = t.core_gradient(k)
        assert rel(d, st.d) <= TOL["fp32"], (k, rel(d, st.d))
        if k in (0, 3):
            assert rel(t.fgmc_gram(k), O.explicit_gram(cores, k)) <= 1e-12, k
        eta = t.core_update(k, -1e-6)
        assert math.isfinite(eta) and eta > 0, (k, eta)
        if k in (1, 2):
            ref = O.core_update(X, P, cores, k, sigma, lam=-1e-6)
            assert abs(eta - ref.eta) <= TOL["fp32"] * abs(ref.eta), (k, eta, ref.eta)
        cores = t.get_cores()


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_graph_replay_equals_eager(torch_cuda, prec):
    """Repeated unsketched steps replayed from a captured CUDA graph give bit-identical
    reports and cores to the same steps run eagerly; a state-changing call in between (a core
    set from the host) ends the replay and the results still agree."""
    from paper_2305_09044_gb300 import TRD
    dims, ranks = (24, 20, 16, 12), (3, 2, 3, 2)
    X, P, words, truth, Xt = problem(dims, ranks, 0.3, 0.1, 51)
    Xd = torch_cuda.from_numpy(flat(X)).cuda()
    Md = torch_cuda.from_numpy(words.view(np.int32)).cuda()
    runs = []
    for graphs in (True, False):
        t = TRD(dims, ranks, prec)
        t.set_graphs(graphs)
        t.set_data(Xd, Md)
        t.init_cores(7)
        reps = [t.step(sigma=-1.0) for _ in range(6)]
        mid = t.get_core(1)
        t.set_core(1, mid)                    # ends the replay; state unchanged
        reps += [t.step(sigma=-1.0) for _ in range(4)]
        runs.append((reps, t.get_cores()))
    (ra, ca), (rb, cb) = runs
    for a, b in zip(ra, rb):
        assert a["e"] == b["e"] and a["sigma"] == b["sigma"] and a["eta"] == b["eta"], (a, b)
    for za, zb in zip(ca, cb):
        assert np.array_equal(za, zb)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_reattach_after_content_change(torch_cuda, prec):
    """New contents written behind the attached pointers and re-attached with trd_set_data
    give the same steps as a fresh handle on the new data: nothing derived from the old
    contents (mask layouts, probe values) survives the re-attach."""
    from paper_2305_09044_gb300 import TRD
    dims, ranks = (32, 24, 16, 16), (2, 3, 2, 2)
    Xa, _, wa, _, _ = problem(dims, ranks, 0.3, 0.1, 61)
    Xb, _, wb, _, _ = problem(dims, ranks, 0.5, 0.2, 62)
    assert not np.array_equal(wa, wb)
    Xd = torch_cuda.from_numpy(flat(Xa)).cuda()
    Md = torch_cuda.from_numpy(wa.view(np.int32)).cuda()
    t = TRD(dims, ranks, prec)
    t.set_data(Xd, Md)
    t.init_cores(9)
    for _ in range(3):
        t.step(sigma=-1.0)                      # caches and a captured graph for the old data
    cores = t.get_cores()
    Xd.copy_(torch_cuda.from_numpy(flat(Xb)))
    Md.copy_(torch_cuda.from_numpy(wb.view(np.int32)))
    t.set_data(Xd, Md)
    u = TRD(dims, ranks, prec)
    Xe = torch_cuda.from_numpy(flat(Xb)).cuda()
    Me = torch_cuda.from_numpy(wb.view(np.int32)).cuda()
    u.set_data(Xe, Me)
    for k, z in enumerate(cores):
        u.set_core(k, z)
    assert t.adaptive_sigma() == u.adaptive_sigma()      # probe values of the new contents
    ra = [t.step(sigma=2.0) for _ in range(3)]           # mask layouts of the new contents
    rb = [u.step(sigma=2.0) for _ in range(3)]
    for a, b in zip(ra, rb):
        assert a["e"] == b["e"] and a["eta"] == b["eta"] and a["objective"] == b["objective"], (a, b)
    for za, zb in zip(t.get_cores(), u.get_cores()):
        assert np.array_equal(za, zb)
