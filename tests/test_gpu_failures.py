"""Failure detection on the GPU path, made on the host side or by a wait that runs out:
a singular FGMC system (lambda = 0 with a zero core), a non-finite residual at an observed
entry, NaN stored at unobserved entries (must be ignored), and the bounded device wait of
the tensor-core pass giving up.  No test faults, traps or hangs the device; after every
failure the same handle is used again and must give the oracle's result.
"""
import math

import numpy as np
import pytest

from oracle import trd_oracle as O

from .helpers import flat, problem, rel

pytestmark = pytest.mark.gpu

DIMS, RANKS = (24, 20, 16, 12), (3, 2, 3, 2)
TOL = {"fp64": 1e-10, "fp32": 1e-4, "bf16": 5e-3}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_09044_gb300 import build
    build.build()
    return torch


def _handle(torch, prec, X, words, dims=DIMS, ranks=RANKS):
    from paper_2305_09044_gb300 import TRD
    t = TRD(dims, ranks, prec)
    xd = torch.from_numpy(flat(X)).cuda()
    md = torch.from_numpy(words.view(np.int32)).cuda()
    t.set_data(xd, md)
    return t, (xd, md)


def _update_matches_oracle(t, X, P, cores, k, tol, sigma=1.5):
    t.set_cores(cores)
    st = O.core_update(X, P, cores, k, sigma, lam=-1e-10)
    t.residual_weights(k, sigma)
    t.core_gradient(k)
    eta = t.core_update(k, -1e-10)
    assert abs(eta - st.eta) <= tol * abs(st.eta)
    assert rel(t.get_core(k) - cores[k], st.cores[k] - cores[k]) <= tol


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_singular_system_is_reported_and_step_rejected(torch_cuda, prec):
    """A zero core makes every Gram G^{!=k} (k != that core) zero; with lambda = 0 the
    factorisation meets a zero pivot: TRD_ESINGULAR, eta forced to 0, core unchanged."""
    from paper_2305_09044_gb300 import TrdError, binding
    X, P, words, truth, Xt = problem(DIMS, RANKS, 0.3, 0.1, 41)
    t, keep = _handle(torch_cuda, prec, X, words)
    cores = O.init_cores(DIMS, RANKS, seed=5)
    broken = [c.copy() for c in cores]
    broken[2][:] = 0.0
    t.set_cores(broken)
    t.residual_weights(0, 1.5)
    t.core_gradient(0)
    with pytest.raises(TrdError) as ei:
        t.core_update(0, 0.0)
    assert ei.value.status == binding.TRD_ESINGULAR
    assert np.array_equal(t.get_core(0), broken[0])
    _update_matches_oracle(t, X, P, cores, 1, TOL[prec])


def test_singular_system_blocked_cholesky(torch_cuda):
    """The same failure at K = 204 (ranks (4, 12, 17, 4)), where the blocked multi-CTA
    Cholesky factors the Gram: the zero pivot is met in the first diagonal block, the later
    panels are skipped, the step is rejected, and the next update of that core is the
    oracle's."""
    from paper_2305_09044_gb300 import TrdError, binding
    dims, ranks = (5, 24, 22, 6), (4, 12, 17, 4)
    X, P, words, truth, Xt = problem(dims, ranks, 0.3, 0.1, 43)
    t, keep = _handle(torch_cuda, "fp64", X, words, dims, ranks)
    cores = O.init_cores(dims, ranks, seed=6)
    broken = [c.copy() for c in cores]
    broken[3][:] = 0.0
    t.set_cores(broken)
    t.residual_weights(1, 1.5)
    t.core_gradient(1)
    with pytest.raises(TrdError) as ei:
        t.core_update(1, 0.0)
    assert ei.value.status == binding.TRD_ESINGULAR
    assert np.array_equal(t.get_core(1), broken[1])
    _update_matches_oracle(t, X, P, cores, 1, TOL["fp64"])


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_nonfinite_observed_entry_is_reported(torch_cuda, prec):
    from paper_2305_09044_gb300 import TrdError, binding
    X, P, words, truth, Xt = problem(DIMS, RANKS, 0.3, 0.1, 42)
    obs = np.flatnonzero(flat(P) > 0)
    Xbad = flat(X).copy()
    Xbad[obs[[3, len(obs) // 2]]] = [np.nan, np.inf]
    t, keep = _handle(torch_cuda, prec, Xbad.reshape(X.shape, order="F"), words)
    cores = O.init_cores(DIMS, RANKS, seed=6)
    t.set_cores(cores)
    s = t.residual_weights(1, 1.5, raise_nonfinite=False)
    assert s["n_nonfinite"] == 2 and s["n_obs"] == len(obs)
    with pytest.raises(TrdError) as ei:
        t.residual_weights(1, 1.5)
    assert ei.value.status == binding.TRD_ENONFINITE


def test_nonfinite_residual_rejects_the_bf16_step(torch_cuda):
    """A NaN at an observed entry: the residual pass reports it, and the scaled step that
    follows is rejected (its line-search denominator is not finite) and leaves the core as it
    was.  On the BF16 path the line search reads the weights pass 1 cached, which carry 0 for
    that entry; pass 1's non-finite count makes the denominator NaN all the same."""
    from paper_2305_09044_gb300 import TrdError, binding
    X, P, words, truth, Xt = problem(DIMS, RANKS, 0.3, 0.1, 44)
    obs = np.flatnonzero(flat(P) > 0)
    Xbad = flat(X).copy()
    Xbad[obs[len(obs) // 3]] = np.nan
    t, keep = _handle(torch_cuda, "bf16", Xbad.reshape(X.shape, order="F"), words)
    cores = O.init_cores(DIMS, RANKS, seed=9)
    t.set_cores(cores)
    s = t.residual_weights(2, 1.5, raise_nonfinite=False)
    assert s["n_nonfinite"] == 1
    t.core_gradient(2)
    with pytest.raises(TrdError) as ei:
        t.core_update(2, -1e-10)
    assert ei.value.status == binding.TRD_ENONFINITE
    assert np.array_equal(t.get_core(2), cores[2].astype(t.get_core(2).dtype))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_nan_at_unobserved_entries_is_ignored(torch_cuda, prec):
    """Unobserved entries take no part in the method (P masks them, Eq. 6): storing NaN
    there changes nothing."""
    X, P, words, truth, Xt = problem(DIMS, RANKS, 0.3, 0.1, 43)
    Xn = np.where(P > 0, X, np.nan)
    t, keep = _handle(torch_cuda, prec, Xn, words)
    cores = O.init_cores(DIMS, RANKS, seed=7)
    for k in (0, 3):
        _update_matches_oracle(t, X, P, cores, k, TOL[prec])
        t.set_cores(cores)
        s = t.residual_weights(k, 1.5)
        assert s["n_nonfinite"] == 0 and math.isfinite(s["sum_we2"])


def test_device_wait_gives_up_with_status(torch_cuda):
    """The bounded mbarrier wait of the tensor-core pass, on a barrier nothing arrives on,
    gives up after its limit and reports TRD_ETIMEOUT; the handle stays usable."""
    from paper_2305_09044_gb300 import binding
    X, P, words, truth, Xt = problem(DIMS, RANKS, 0.3, 0.1, 44)
    t, keep = _handle(torch_cuda, "bf16", X, words)
    assert t.wait_selftest(True, 1 << 10) == binding.TRD_OK
    assert t.wait_selftest(False, 1 << 12) == binding.TRD_ETIMEOUT
    assert t.wait_selftest(False, 0) == binding.TRD_EINVAL
    assert t.wait_selftest(True, 1 << 10) == binding.TRD_OK
    _update_matches_oracle(t, X, P, O.init_cores(DIMS, RANKS, seed=8), 2, TOL["bf16"])


def test_width_rejects_nan_floor(torch_cuda):
    """A NaN rms of the observed data (the floor of the adaptive width) is rejected with
    TRD_EINVAL by the handle path, as by the allocation-free form; the handle stays usable."""
    from paper_2305_09044_gb300 import TRD, TrdError
    t = TRD((4, 4, 4), (1, 1, 1), "fp32")
    rd = torch_cuda.ones(100, dtype=torch_cuda.float32, device="cuda")
    with pytest.raises(TrdError):
        t.sigma_from_residuals(rd, float("nan"), -1.0)
    assert t.sigma_from_residuals(rd, 1.0, -1.0) > 0
