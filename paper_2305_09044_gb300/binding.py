"""Thin ctypes binding of libtrd (include/trd.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels.  PyTorch supplies device
memory and the CUDA stream.  There is no CPU fallback: if libtrd.so is missing or no CUDA
device is present, constructing a handle raises.

Core arrays on the Python side use the paper's shape (r_k, I_k, r_{k+1}) (Def. 1); the
library's layout is the row-major mode-2 unfolding (I_k, r_{k+1}, r_k).
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import List, Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtrd.so")

TRD_OK, TRD_EINVAL, TRD_ENOMEM, TRD_ECUDA, TRD_ESINGULAR, TRD_ENONFINITE, TRD_ETIMEOUT, TRD_ENOTIMPL = range(8)
PRECISIONS = {"fp64": 0, "fp32": 1, "bf16": 2, "tf32x3": 3}
GRAMS = {"global": 0, "local": 1, "none": 2}
MAX_ORDER = 8

STATUS_NAMES = ["TRD_OK", "TRD_EINVAL", "TRD_ENOMEM", "TRD_ECUDA", "TRD_ESINGULAR",
                "TRD_ENONFINITE", "TRD_ETIMEOUT", "TRD_ENOTIMPL"]

# every symbol the header declares
EXPORTS = [
    "trd_create", "trd_destroy", "trd_last_error", "trd_status_string", "trd_set_data",
    "trd_init_cores", "trd_set_core", "trd_get_core", "trd_reset_iteration",
    "trd_sample_subtensor", "trd_draw_indices", "trd_residual_weights", "trd_core_gradient",
    "trd_fgmc_gram", "trd_core_update", "trd_step", "trd_adaptive_sigma",
    "trd_sigma_from_residuals", "trd_reconstruct", "trd_reconstruct_from",
    "trd_recovery_error", "trd_sampled_fwd", "trd_sampled_bwd", "trd_set_profiling",
    "trd_get_profile", "trd_kernel_launches", "trd_sigma_from_residuals_noalloc",
    "trd_wait_selftest", "trd_set_graphs", "trd_sample_rows", "trd_psnr", "trd_set_gradient",
    "trd_line_search_terms", "trd_ring_cut",
]


class TrdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class ResidStats(C.Structure):
    _fields_ = [("sigma", C.c_double), ("sum_w", C.c_double), ("sum_e2", C.c_double),
                ("sum_we2", C.c_double), ("n_obs", C.c_int64), ("n_nonfinite", C.c_int64),
                ("n_slots", C.c_int64)]


class Params(C.Structure):
    _fields_ = [("sketch", C.c_int32 * MAX_ORDER), ("sigma", C.c_double), ("lambda_", C.c_double),
                ("seed", C.c_uint64), ("gram", C.c_int32), ("reserved", C.c_int32)]


class Report(C.Structure):
    _fields_ = [("e", C.c_double), ("sigma", C.c_double), ("eta", C.c_double * MAX_ORDER),
                ("objective", C.c_double * MAX_ORDER), ("slots", C.c_int64), ("t", C.c_int32),
                ("reserved", C.c_int32)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libtrd.so once (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libtrd.so not found at {path}: run __graft_entry__.build() "
                          "(python -m paper_2305_09044_gb300.build)")
    lib = C.CDLL(path)
    vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    P = C.POINTER
    sig = {
        "trd_create": [P(vp), C.c_int, P(i64), P(i32), C.c_int, vp],
        "trd_destroy": [vp],
        "trd_last_error": [vp],
        "trd_status_string": [C.c_int],
        "trd_set_data": [vp, vp, vp],
        "trd_init_cores": [vp, u64, dbl],
        "trd_set_core": [vp, C.c_int, P(dbl)],
        "trd_get_core": [vp, C.c_int, P(dbl)],
        "trd_reset_iteration": [vp, i32],
        "trd_sample_subtensor": [vp, C.c_int, P(P(i32)), P(i32)],
        "trd_draw_indices": [u64, i32, C.c_int, C.c_int, C.c_int, i64, i32, P(i32)],
        "trd_residual_weights": [vp, C.c_int, dbl, P(ResidStats)],
        "trd_core_gradient": [vp, C.c_int, P(dbl)],
        "trd_fgmc_gram": [vp, C.c_int, P(dbl)],
        "trd_core_update": [vp, C.c_int, dbl, dbl, C.c_int, P(dbl)],
        "trd_step": [vp, P(Params), P(Report)],
        "trd_adaptive_sigma": [vp, dbl, P(dbl)],
        "trd_sigma_from_residuals": [vp, vp, i64, dbl, dbl, P(dbl)],
        "trd_reconstruct": [vp, vp],
        "trd_reconstruct_from": [vp, P(P(dbl)), vp],
        "trd_recovery_error": [vp, vp, P(dbl)],
        "trd_sampled_fwd": [vp, P(vp), vp, vp, i64, dbl, C.c_int, vp, P(dbl)],
        "trd_sampled_bwd": [vp, P(vp), vp, vp, i64, dbl, C.c_int, dbl, P(vp)],
        "trd_set_profiling": [vp, C.c_int],
        "trd_get_profile": [vp, C.c_int, P(dbl)],
        "trd_kernel_launches": [],
        "trd_sigma_from_residuals_noalloc": [vp, i64, dbl, dbl, vp, vp],
        "trd_wait_selftest": [vp, C.c_int, i64],
        "trd_set_graphs": [vp, C.c_int],
        "trd_sample_rows": [vp, C.c_int, P(i32), i64],
        "trd_psnr": [vp, vp, dbl, P(dbl)],
        "trd_set_gradient": [vp, C.c_int, P(dbl)],
        "trd_line_search_terms": [vp, C.c_int, dbl, C.c_int, P(dbl), P(dbl)],
        "trd_ring_cut": [C.c_int, P(i64), P(i32), C.c_int, P(i32), P(i32)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.trd_destroy.restype = None
    lib.trd_kernel_launches.restype = C.c_int64
    lib.trd_last_error.restype = C.c_char_p
    lib.trd_status_string.restype = C.c_char_p
    _lib = lib
    return lib


def _dptr(t) -> Optional[int]:
    """Device pointer of a CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def core_to_abi(Z: np.ndarray) -> np.ndarray:
    """(r_k, I_k, r_{k+1}) -> row-major mode-2 unfolding (I_k, r_{k+1}, r_k), float64."""
    return np.ascontiguousarray(np.asarray(Z, dtype=np.float64).transpose(1, 2, 0))


def core_from_abi(A: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(A.transpose(2, 0, 1))


def kernel_launches() -> int:
    return int(load().trd_kernel_launches())


def draw_indices(seed: int, t: int, k: int, j: int, N: int, I: int, s: int) -> np.ndarray:
    lib = load()
    out = np.empty(s, dtype=np.int32)
    st = lib.trd_draw_indices(seed, t, k, j, N, I, s, out.ctypes.data_as(C.POINTER(C.c_int32)))
    if st != TRD_OK:
        raise TrdError(st, "trd_draw_indices")
    return out


def ring_cut(dims: Sequence[int], ranks: Sequence[int], precision: str = "fp32"):
    """(c, r_1 r_{c+1}, fits) of trd_ring_cut: where the data passes cut the ring for these
    mode sizes and ranks, and whether that width is one they take (host only)."""
    lib = load()
    N = len(dims)
    I = (C.c_int64 * N)(*[int(d) for d in dims])
    R = (C.c_int32 * N)(*[int(r) for r in ranks])
    c, w = C.c_int32(), C.c_int32()
    st = lib.trd_ring_cut(N, I, R, PRECISIONS[precision], C.byref(c), C.byref(w))
    if st not in (TRD_OK, TRD_ENOTIMPL):
        raise TrdError(st, "trd_ring_cut")
    return int(c.value), int(w.value), st == TRD_OK


class TRD:
    """One decomposition problem on the current CUDA device (wraps a trd_t handle)."""

    def __init__(self, dims: Sequence[int], ranks: Sequence[int], precision: str = "fp32",
                 stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libtrd needs a CUDA device; there is no CPU fallback")
        self.lib = load()
        self.dims = [int(d) for d in dims]
        self.ranks = [int(r) for r in ranks]
        self.N = len(self.dims)
        self.precision = precision
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        I = (C.c_int64 * self.N)(*self.dims)
        R = (C.c_int32 * self.N)(*self.ranks)
        st = self.lib.trd_create(C.byref(h), self.N, I, R, PRECISIONS[precision],
                                 C.c_void_p(stream.cuda_stream))
        if st != TRD_OK:
            raise TrdError(st, "trd_create failed")
        self.h = h
        self._data = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.trd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str):
        if st != TRD_OK:
            msg = self.lib.trd_last_error(self.h).decode() if self.h else ""
            raise TrdError(st, f"{what}: {msg}")

    def K(self, k: int) -> int:
        return self.ranks[k] * self.ranks[(k + 1) % self.N]

    # ------------------------------------------------------------------ data / cores
    def set_data(self, X, mask=None):
        """X: CUDA float32 tensor with prod(dims) entries in linear order (i_1 fastest);
        mask: CUDA int32/uint32 tensor of packed words or None (fully observed)."""
        import torch
        if X.dtype != torch.float32 or X.numel() != int(np.prod(self.dims)):
            raise ValueError("X must be float32 with prod(dims) entries")
        self._data = (X, mask)   # keep the borrowed buffers alive
        self._check(self.lib.trd_set_data(self.h, C.c_void_p(_dptr(X)),
                                          C.c_void_p(_dptr(mask)) if mask is not None else None),
                    "trd_set_data")

    def init_cores(self, seed: int, stddev: float = -1.0):
        self._check(self.lib.trd_init_cores(self.h, seed, stddev), "trd_init_cores")

    def set_core(self, k: int, Z: np.ndarray):
        A = core_to_abi(Z)
        self._check(self.lib.trd_set_core(self.h, k, A.ctypes.data_as(C.POINTER(C.c_double))),
                    "trd_set_core")

    def set_cores(self, cores: Sequence[np.ndarray], t: int = 0):
        for k, Z in enumerate(cores):
            self.set_core(k, Z)
        self._check(self.lib.trd_reset_iteration(self.h, t), "trd_reset_iteration")

    def get_core(self, k: int) -> np.ndarray:
        A = np.empty((self.dims[k], self.ranks[(k + 1) % self.N], self.ranks[k]))
        self._check(self.lib.trd_get_core(self.h, k, A.ctypes.data_as(C.POINTER(C.c_double))),
                    "trd_get_core")
        return core_from_abi(A)

    def get_cores(self) -> List[np.ndarray]:
        return [self.get_core(k) for k in range(self.N)]

    # ------------------------------------------------------------------ hot path
    def sample_subtensor(self, k: int, idx: Optional[Sequence[Optional[np.ndarray]]]):
        if idx is None:
            self._check(self.lib.trd_sample_subtensor(self.h, k, None, None), "trd_sample_subtensor")
            return
        arrs = [np.ascontiguousarray(np.asarray(a if a is not None else [0], dtype=np.int32))
                for a in idx]
        ptrs = (C.POINTER(C.c_int32) * self.N)(*[
            (a.ctypes.data_as(C.POINTER(C.c_int32)) if (m != k and idx[m] is not None) else None)
            for m, a in enumerate(arrs)])
        sizes = (C.c_int32 * self.N)(*[len(a) if (m != k and idx[m] is not None) else 0
                                        for m, a in enumerate(arrs)])
        self._keep = arrs
        self._check(self.lib.trd_sample_subtensor(self.h, k, ptrs, sizes), "trd_sample_subtensor")

    def sample_rows(self, k: int, rows: np.ndarray):
        """Uniform row sampling for core k: rows is a (J, N) integer array of multi-indices
        (column k ignored); see trd_sample_rows."""
        r = np.ascontiguousarray(np.asarray(rows, dtype=np.int32))
        if r.ndim != 2 or r.shape[1] != self.N:
            raise ValueError("rows must have shape (J, N)")
        self._check(self.lib.trd_sample_rows(self.h, k, r.ctypes.data_as(C.POINTER(C.c_int32)), r.shape[0]),
                    "trd_sample_rows")

    def residual_weights(self, k: int, sigma: float, raise_nonfinite: bool = True) -> dict:
        s = ResidStats()
        st = self.lib.trd_residual_weights(self.h, k, sigma, C.byref(s))
        if st != TRD_ENONFINITE or raise_nonfinite:
            self._check(st, "trd_residual_weights")
        return {f: getattr(s, f) for f, _ in ResidStats._fields_}

    def core_gradient(self, k: int) -> np.ndarray:
        d = np.empty((self.dims[k], self.K(k)))
        self._check(self.lib.trd_core_gradient(self.h, k, d.ctypes.data_as(C.POINTER(C.c_double))),
                    "trd_core_gradient")
        return d

    def fgmc_gram(self, k: int) -> np.ndarray:
        G = np.empty((self.K(k), self.K(k)))
        self._check(self.lib.trd_fgmc_gram(self.h, k, G.ctypes.data_as(C.POINTER(C.c_double))),
                    "trd_fgmc_gram")
        return G

    def core_update(self, k: int, lam: float = -1e-10, eta: float = -1.0, gram: str = "global") -> float:
        out = C.c_double()
        self._check(self.lib.trd_core_update(self.h, k, lam, eta, GRAMS[gram], C.byref(out)),
                    "trd_core_update")
        return out.value

    def set_gradient(self, k: int, d: np.ndarray):
        """Replace the device gradient of core k (I_k x K) by d (the summed partial gradients of
        a partitioned update)."""
        a = np.ascontiguousarray(d, dtype=np.float64)
        assert a.shape == (self.dims[k], self.K(k))
        self._check(self.lib.trd_set_gradient(self.h, k, a.ctypes.data_as(C.POINTER(C.c_double))),
                    "trd_set_gradient")

    def line_search_terms(self, k: int, lam: float = -1e-10, gram: str = "global"):
        """(<d, h>, this handle's line-search denominator) without changing core k."""
        num, den = C.c_double(), C.c_double()
        self._check(self.lib.trd_line_search_terms(self.h, k, lam, GRAMS[gram], C.byref(num), C.byref(den)),
                    "trd_line_search_terms")
        return num.value, den.value

    def step(self, sketch: Optional[Sequence[int]] = None, sigma: float = -1.0,
             lam: float = -1e-10, seed: int = 0, gram: str = "global") -> dict:
        p = Params()
        for m in range(self.N):
            p.sketch[m] = int(sketch[m]) if sketch is not None else 0
        p.sigma, p.lambda_, p.seed, p.gram = sigma, lam, seed, GRAMS[gram]
        r = Report()
        self._check(self.lib.trd_step(self.h, C.byref(p), C.byref(r)), "trd_step")
        return {"e": r.e, "sigma": r.sigma, "eta": list(r.eta)[: self.N],
                "objective": list(r.objective)[: self.N], "slots": r.slots, "t": r.t}

    # ------------------------------------------------------------------ evaluation helpers
    def adaptive_sigma(self, sigma_prev: float = -1.0) -> float:
        out = C.c_double()
        self._check(self.lib.trd_adaptive_sigma(self.h, sigma_prev, C.byref(out)), "trd_adaptive_sigma")
        return out.value

    def sigma_from_residuals(self, resid, rms: float, sigma_prev: float = -1.0) -> float:
        out = C.c_double()
        self._check(self.lib.trd_sigma_from_residuals(self.h, C.c_void_p(_dptr(resid)), resid.numel(),
                                                      rms, sigma_prev, C.byref(out)),
                    "trd_sigma_from_residuals")
        return out.value

    def reconstruct(self, out=None):
        import torch
        if out is None:
            out = torch.empty(int(np.prod(self.dims)), dtype=torch.float32, device="cuda")
        self._check(self.lib.trd_reconstruct(self.h, C.c_void_p(_dptr(out))), "trd_reconstruct")
        return out

    def reconstruct_from(self, cores: Sequence[np.ndarray], out=None):
        import torch
        if out is None:
            out = torch.empty(int(np.prod(self.dims)), dtype=torch.float32, device="cuda")
        arrs = [core_to_abi(Z) for Z in cores]
        ptrs = (C.POINTER(C.c_double) * self.N)(*[a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs])
        self._check(self.lib.trd_reconstruct_from(self.h, ptrs, C.c_void_p(_dptr(out))),
                    "trd_reconstruct_from")
        return out

    def set_profiling(self, on=True):
        """Tracing level: False/0 off, 1 the data passes only, True/2 every phase."""
        level = 2 if on is True else (0 if on is False else int(on))
        self._check(self.lib.trd_set_profiling(self.h, level), "trd_set_profiling")

    PHASES = ["pass1", "pass2", "merge", "reduce", "backcontract", "gram", "cholesky", "solve",
              "update", "sigma", "stop", "gather"]

    def get_profile(self, reset: bool = False) -> dict:
        """Per-phase totals (ms) and counts of the traced intervals (see trd_get_profile)."""
        out = (C.c_double * 24)()
        self._check(self.lib.trd_get_profile(self.h, 1 if reset else 0, out), "trd_get_profile")
        res = {}
        for q, name in enumerate(self.PHASES):
            res[name + "_ms"] = out[2 * q]
            res[name + "_n"] = int(out[2 * q + 1])
        return res

    # ------------------------------------------------------------------ sampled correntropy loss
    def sampled_fwd(self, cores, idx, x, sigma: float, resid=None) -> float:
        """cores: CUDA tensors in the library layout (I_k, r_{k+1}, r_k), all float32 or all
        float64; idx: CUDA int32 (M, N); x: CUDA values (M,), same dtype as the cores."""
        import torch
        fp64 = cores[0].dtype == torch.float64
        ptrs = (C.c_void_p * self.N)(*[_dptr(t) for t in cores])
        out = C.c_double()
        self._check(self.lib.trd_sampled_fwd(self.h, ptrs, C.c_void_p(_dptr(idx)), C.c_void_p(_dptr(x)),
                                             idx.shape[0], sigma, 1 if fp64 else 0,
                                             C.c_void_p(_dptr(resid)) if resid is not None else None,
                                             C.byref(out)), "trd_sampled_fwd")
        return out.value

    def sampled_bwd(self, cores, idx, x, sigma: float, g_scale: float = 1.0, grads=None):
        import torch
        fp64 = cores[0].dtype == torch.float64
        if grads is None:
            grads = [torch.empty_like(t) for t in cores]
        ptrs = (C.c_void_p * self.N)(*[_dptr(t) for t in cores])
        gptrs = (C.c_void_p * self.N)(*[_dptr(t) for t in grads])
        self._check(self.lib.trd_sampled_bwd(self.h, ptrs, C.c_void_p(_dptr(idx)), C.c_void_p(_dptr(x)),
                                             idx.shape[0], sigma, 1 if fp64 else 0, g_scale, gptrs),
                    "trd_sampled_bwd")
        return grads

    def set_graphs(self, on: bool = True):
        """Capture and replay repeated unsketched steps as a CUDA graph (default on)."""
        self._check(self.lib.trd_set_graphs(self.h, 1 if on else 0), "trd_set_graphs")

    def wait_selftest(self, arrive: bool, limit: int) -> int:
        """Run the bounded device wait once (see trd_wait_selftest); returns the raw status
        (TRD_OK or TRD_ETIMEOUT) instead of raising, so a test can check it."""
        return int(self.lib.trd_wait_selftest(self.h, 1 if arrive else 0, int(limit)))

    def recovery_error(self, Xref) -> float:
        out = C.c_double()
        self._check(self.lib.trd_recovery_error(self.h, C.c_void_p(_dptr(Xref)), C.byref(out)),
                    "trd_recovery_error")
        return out.value

    def psnr(self, Xref, peak: float = 1.0) -> float:
        """PSNR (dB) of the current reconstruction against the device tensor Xref."""
        out = C.c_double()
        self._check(self.lib.trd_psnr(self.h, C.c_void_p(_dptr(Xref)), float(peak), C.byref(out)),
                    "trd_psnr")
        return out.value
