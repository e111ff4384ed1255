"""The C-ABI library builds, loads and exports every symbol declared in include/trd.h, and
its host-only logic matches the oracle (no GPU compute is called here)."""
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
