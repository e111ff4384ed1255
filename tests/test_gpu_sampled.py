"""Sampled correntropy loss and its hand-written adjoint (GPU) against the FP64 oracle and
central finite differences; the torch.autograd.Function through torch.autograd.gradcheck.

Tolerances: FP64 adjoint vs oracle 1e-10, vs central differences (step 1e-6) 1e-6 relative;
FP32 loss 1e-5 and gradient 1e-4 relative (FP32 scatter sums over ~10^3 entries per slice).
"""
import numpy as np
import pytest

from oracle import trd_oracle as O

from .helpers import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_09044_gb300 import build
    build.build()
    return torch


def _abi(torch, cores, dtype):
    """Paper-shaped cores (r_k, I_k, r_{k+1}) -> library layout (I_k, r_{k+1}, r_k) on the GPU."""
    return [torch.from_numpy(np.ascontiguousarray(Z.transpose(1, 2, 0))).to(dtype).cuda() for Z in cores]


def _grad_to_paper(g):
    return np.ascontiguousarray(g.transpose(2, 0, 1))


def _instance(dims, ranks, M, seed, scale=0.5):
    rng = np.random.default_rng(seed)
    N = len(dims)
    cores = [scale * rng.standard_normal((ranks[k], dims[k], ranks[(k + 1) % N])) for k in range(N)]
    lin = rng.choice(int(np.prod(dims)), M, replace=False)
    idx = np.stack(np.unravel_index(lin, dims, order="F"), axis=1).astype(np.int32)
    x = rng.standard_normal(M)
    return cores, idx, x


def test_adjoint_fp64_oracle_and_finite_differences(torch_cuda):
    """8^4, rank 4 (the finite-difference check's instance): loss and gradient equal the oracle's, and
    the gradient matches FP64 central differences of the GPU loss at step 1e-6."""
    torch = torch_cuda
    from paper_2305_09044_gb300 import TRD
    dims, ranks, M, sigma = (8, 8, 8, 8), (4, 4, 4, 4), 500, 0.9
    cores, idx, x = _instance(dims, ranks, M, 21)
    t = TRD(dims, ranks, "fp64")
    cd = _abi(torch, cores, torch.float64)
    idd = torch.from_numpy(idx).cuda()
    xd = torch.from_numpy(x).cuda()
    loss = t.sampled_fwd(cd, idd, xd, sigma)
    lo, e, w, go = O.sampled_loss_grad(cores, idx, x, sigma)
    assert abs(loss - lo) <= 1e-12 * abs(lo)
    grads = [_grad_to_paper(g.cpu().numpy()) for g in t.sampled_bwd(cd, idd, xd, sigma)]
    for k in range(4):
        assert rel(grads[k], go[k]) <= 1e-10, (k, rel(grads[k], go[k]))
    rng = np.random.default_rng(3)
    num, ana = [], []
    h = 1e-6
    for _ in range(40):
        k = int(rng.integers(0, 4))
        a, i, b = (int(rng.integers(0, s)) for s in cores[k].shape)
        for sgn in (1, -1):
            cp = [c.clone() for c in cd]
            cp[k][i, b, a] += sgn * h          # library layout (I_k, r_{k+1}, r_k)
            val = t.sampled_fwd(cp, idd, xd, sigma)
            if sgn == 1:
                lp = val
            else:
                lm = val
        num.append((lp - lm) / (2 * h))
        ana.append(grads[k][a, i, b])
    assert rel(num, ana) <= 1e-6, rel(num, ana)


def test_adjoint_fp32_matches_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2305_09044_gb300 import TRD
    dims, ranks, M, sigma = (24, 20, 18, 16), (5, 6, 4, 6), 20000, 1.1
    cores, idx, x = _instance(dims, ranks, M, 22, 0.6)
    t = TRD(dims, ranks, "fp32")
    cd = _abi(torch, cores, torch.float32)
    idd = torch.from_numpy(idx).cuda()
    x32 = x.astype(np.float32)
    xd = torch.from_numpy(x32).cuda()
    c32 = [c.cpu().numpy().astype(np.float64).transpose(2, 0, 1) for c in cd]
    lo, e, w, go = O.sampled_loss_grad_vec(c32, idx, x32.astype(np.float64), sigma)
    resid = torch.empty_like(xd)
    loss = t.sampled_fwd(cd, idd, xd, sigma, resid)
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    assert rel(resid.cpu().numpy(), e) <= 1e-5
    grads = [_grad_to_paper(g.cpu().numpy().astype(np.float64)) for g in t.sampled_bwd(cd, idd, xd, sigma)]
    for k in range(4):
        assert rel(grads[k], go[k]) <= 1e-4, (k, rel(grads[k], go[k]))


def test_bad_index_is_rejected(torch_cuda):
    torch = torch_cuda
    from paper_2305_09044_gb300 import TRD, TrdError
    dims, ranks = (6, 6, 6), (2, 2, 2)
    cores, idx, x = _instance(dims, ranks, 40, 5)
    idx[7, 1] = 6                          # out of range: skipped, reported
    t = TRD(dims, ranks, "fp64")
    with pytest.raises(TrdError):
        t.sampled_fwd(_abi(torch, cores, torch.float64), torch.from_numpy(idx).cuda(),
                      torch.from_numpy(x).cuda(), 1.0)


def test_autograd_function_gradcheck(torch_cuda):
    torch = torch_cuda
    from paper_2305_09044_gb300 import TRD
    from paper_2305_09044_gb300.autograd import TRCorrentropy
    dims, ranks, M, sigma = (5, 4, 6, 3), (2, 2, 3, 2), 60, 0.7
    cores, idx, x = _instance(dims, ranks, M, 23, 0.8)
    t = TRD(dims, ranks, "fp64")
    cd = [c.requires_grad_(True) for c in _abi(torch, cores, torch.float64)]
    idd = torch.from_numpy(idx).cuda()
    xd = torch.from_numpy(x).cuda()
    fn = lambda *cs: TRCorrentropy.apply(t, idd, xd, sigma, *cs)
    # the adjoint scatter-adds with atomics, so repeated backward passes may differ in the
    # last bits (summation order); nondet_tol bounds that at FP64 rounding level
    assert torch.autograd.gradcheck(fn, tuple(cd), eps=1e-6, atol=1e-7, rtol=1e-5, nondet_tol=1e-12)
    loss = fn(*cd)
    loss.backward()
    lo, e, w, go = O.sampled_loss_grad(cores, idx, x, sigma)
    for k in range(4):
        assert rel(_grad_to_paper(cd[k].grad.cpu().numpy()), go[k]) <= 1e-10


def test_full_size_sampled_workload(torch_cuda):
    """128^4, TR ranks 20, 2^24 sampled entries, FP32 (the sampled-loss workload's size):
    residuals at 2000 entries and the gradient slice Z_1(i_1 = 5) against the oracle."""
    torch = torch_cuda
    from paper_2305_09044_gb300 import TRD, synth
    w = synth.WORKLOADS["grad128"]
    cores = synth.gaussian_cores(w.dims, w.ranks, w.data_seed)
    idx = synth.sample_entries(w.dims, w.n_sampled, w.sample_seed)
    M = idx.shape[0]
    x = np.random.default_rng(w.data_seed + 5).standard_normal(M).astype(np.float32)
    t = TRD(w.dims, w.ranks, "fp32")
    cd = _abi(torch, cores, torch.float32)
    idd = torch.from_numpy(idx).cuda()
    xd = torch.from_numpy(x).cuda()
    resid = torch.empty_like(xd)
    sigma = 1.0
    t.sampled_fwd(cd, idd, xd, sigma, resid)
    grads = t.sampled_bwd(cd, idd, xd, sigma)
    c32 = [c.cpu().numpy().astype(np.float64).transpose(2, 0, 1) for c in cd]
    pick = np.random.default_rng(1).choice(M, 2000, replace=False)
    r = resid.cpu().numpy()
    want = x[pick].astype(np.float64) - np.array([O.entry(c32, idx[m]) for m in pick])
    assert rel(r[pick], want) <= 1e-5
    sel = np.flatnonzero(idx[:, 0] == 5)
    lo, e, wv, go = O.sampled_loss_grad_vec(c32, idx[sel], x[sel].astype(np.float64), sigma)
    g0 = _grad_to_paper(grads[0].cpu().numpy().astype(np.float64))
    assert rel(g0[:, 5, :], go[0][:, 5, :]) <= 1e-4
