"""Shared test helpers: seeded problems built from the workload generator, with the clean
tensor computed by the FP64 oracle (never by the CUDA path)."""
import math

import numpy as np

from oracle import trd_oracle as O
from paper_2305_09044_gb300 import synth


def problem(dims, ranks, missing=0.3, outliers=0.1, seed=5, noise_var=0.0):
    """Returns (X32 as float64, P as float64 0/1, packed mask, true cores, X_true)."""
    w = synth.Workload("t", tuple(dims), tuple(ranks), missing, outliers, noise_var=noise_var,
                       data_seed=seed)
    cores = synth.gaussian_cores(dims, ranks, seed)
    Xt = O.reconstruct_unfold(cores)
    c = synth.draw_corruption(w)
    X = synth.assemble(Xt, c)
    X32 = X.astype(np.float32).astype(np.float64)
    P = c.mask.astype(np.float64)
    return X32, P, synth.pack_mask(c.mask), cores, Xt


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def flat(X):
    """Linear (i_1 fastest) float32 vector of a tensor."""
    return np.asarray(X, dtype=np.float32).reshape(-1, order="F")


def big_problem(w, cut: int, cols: int):
    """Full-size workload `w` built chunk by chunk (for tensors of ~1e9 entries): the clean
    tensor from the oracle's two-half reconstruction of the seeded true cores, the
    corruption from synth.corruption_chunks.  Returns (X float32 flat, mask bool flat,
    true cores); arrays are in linear order (i_1 fastest)."""
    dims = tuple(w.dims)
    n = int(np.prod(dims))
    truth = synth.gaussian_cores(dims, w.ranks, w.data_seed, w.smooth_modes, w.smooth_width)
    Xc = np.empty(n, dtype=np.float32)
    s1 = s2 = 0.0
    lo, hi = math.inf, -math.inf
    for s, v in O.reconstruct_chunks(truth, cut, cols):
        Xc[s:s + v.size] = v
        s1 += float(v.sum())
        s2 += float(np.dot(v, v))
        lo, hi = min(lo, float(v.min())), max(hi, float(v.max()))
    std = math.sqrt(max(s2 / n - (s1 / n) ** 2, 0.0))
    X = np.empty(n, dtype=np.float32)
    mask = np.empty(n, dtype=bool)
    for s, m, o, u, nz in synth.corruption_chunks(w):
        e = s + m.size
        X[s:e] = synth.assemble_chunk(Xc[s:e].astype(np.float64), o, u, nz, w.outlier_kind, std, lo, hi)
        mask[s:e] = m
    del Xc
    return X, mask, truth
