"""The C-ABI library builds, loads and exports every symbol declared in include/trd.h, and
its host-only logic matches the oracle (no GPU compute is called here)."""
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2305_09044_gb300 import build, binding
    build.build()
    return binding.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "trd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(trd_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for need in ["trd_init_cores", "trd_sample_subtensor", "trd_residual_weights", "trd_core_gradient",
                 "trd_fgmc_gram", "trd_core_update", "trd_step"]:
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2305_09044_gb300.binding import EXPORTS
    names = _declared()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(EXPORTS) == names


def test_status_strings(lib):
    lib.trd_status_string.restype = __import__("ctypes").c_char_p
    assert lib.trd_status_string(0) == b"TRD_OK"
    assert lib.trd_status_string(4) == b"TRD_ESINGULAR"


def test_create_rejects_bad_shapes(lib):
    import ctypes as C
    h = C.c_void_p()
    I = (C.c_int64 * 2)(4, 4)
    R = (C.c_int32 * 2)(2, 2)
    assert lib.trd_create(C.byref(h), 2, I, R, 1, None) == 1      # N < 3
    I3 = (C.c_int64 * 3)(4, 4, 4)
    R3 = (C.c_int32 * 3)(2, 129, 2)
    assert lib.trd_create(C.byref(h), 3, I3, R3, 1, None) == 1    # rank too large
    R3 = (C.c_int32 * 3)(2, 100, 100)
    assert lib.trd_create(C.byref(h), 3, I3, R3, 1, None) == 1    # r_k r_{k+1} too large
    assert lib.trd_create(C.byref(h), 3, I3, (C.c_int32 * 3)(2, 2, 2), 9, None) == 1  # precision


def test_draw_indices_matches_oracle(lib):
    from oracle import trd_oracle as O
    from paper_2305_09044_gb300 import draw_indices
    for (seed, t, k, j, N, I, s) in [(7, 3, 1, 2, 4, 64, 24), (0, 0, 0, 1, 3, 1024, 128),
                                      (2**63 + 5, 17, 4, 0, 5, 64, 24), (3, 1, 2, 1, 3, 10, 10)]:
        assert np.array_equal(draw_indices(seed, t, k, j, N, I, s), O.draw_indices(seed, t, k, j, N, I, s))


def _cut_rule(dims, ranks, precision):
    """The cut rule as include/trd.h states it, written out: c = 1..N-1 in order, the c whose
    blocks' log entry counts differ least among those with R[0] R[c] <= 256 (112 on FP64),
    the lowest c on a tie; when none fits, the most balanced c overall."""
    kmax = 112 if precision == "fp64" else 256
    best, best_c, fit, fit_c = math.inf, 1, math.inf, None
    for c in range(1, len(dims)):
        cost = abs(sum(math.log(d) for d in dims[:c]) - sum(math.log(d) for d in dims[c:]))
        if cost < best - 1e-12:
            best, best_c = cost, c
        if ranks[0] * ranks[c] <= kmax and cost < fit - 1e-12:
            fit, fit_c = cost, c
    c = fit_c if fit_c is not None else best_c
    return c, ranks[0] * ranks[c], fit_c is not None


def test_ring_cut(lib):
    """Where the data passes cut the ring (host only): the paper's video rank [80, 80, 3, 20] is
    cut through its rank-3 edge (width 240) on BF16 although the balanced cut runs through the
    two rank-80 edges (width 6400), and has no cut the FP64 passes take; the image ranks
    (3, 20, 20) keep the balanced width-60 cut; random shapes follow the stated rule."""
    from paper_2305_09044_gb300 import TrdError, ring_cut
    assert ring_cut((1920, 1080, 3, 50), (80, 80, 3, 20), "bf16") == (2, 240, True)
    assert ring_cut((1920, 200, 3, 50), (80, 80, 3, 20), "bf16") == (2, 240, True)
    assert ring_cut((1920, 1080, 3, 50), (80, 80, 3, 20), "fp64") == (1, 6400, False)
    assert ring_cut((3, 1352, 2000), (3, 20, 20), "bf16") == (2, 60, True)
    assert ring_cut((40, 36, 3, 8), (20, 20, 3, 4), "fp64") == (2, 60, True)
    rng = np.random.default_rng(5)
    for _ in range(2000):
        N = int(rng.integers(3, 9))
        dims = [int(x) for x in rng.integers(1, 3000, N)]
        ranks = [int(x) for x in rng.integers(1, 65, N)]
        prec = ["fp64", "fp32", "bf16", "tf32x3"][int(rng.integers(0, 4))]
        if sum(math.log2(d) for d in dims) >= 40:
            continue
        assert ring_cut(dims, ranks, prec) == _cut_rule(dims, ranks, prec), (dims, ranks, prec)
    with pytest.raises(TrdError):
        ring_cut((4, 4, 4), (2, 129, 2), "fp32")
    with pytest.raises(TrdError):
        ring_cut((4, 4, 4), (2, 100, 100), "fp32")
