"""Seeded synthetic workloads for the robust tensor-ring decomposition.

This module only draws random numbers and assembles them element-wise; it holds none of
the method's arithmetic (no TR contraction, no weights, no gradients).  A clean tensor
X_true = R(Z_true) is produced by the caller from the cores drawn here (the CPU oracle in
tests, the library's reconstruction kernel in the benchmark).

Layout shared with the library: a tensor of dims (I_1, ..., I_N) is flattened with i_1
fastest (Def. 2's multi-index), i.e. numpy Fortran order; the observation mask is
bit-packed, bit b of 32-bit word w <-> linear index 32 w + b (1 = observed), padded with
zero words to a multiple of four words.

Workloads (the paper's image/video data sets are not used; these stand in for them with
the orders 3-5, TR ranks 3-20, 20-80 % missing and 10-20 % outliers of its experiments):
  tiny3   30 x 30 x 30, ranks 3, N(0, 1/3) cores, 30 % missing, 10 % outliers
  cfg100  100^4, ranks 8, 50 % missing, 20 % outliers U[-10 std, 10 std] + N(0, 1e-3) noise
  cfg64   64^5, ranks 10, 70 % missing, 10 % outliers; sketch 24 per non-updated mode
  video   1024 x 1024 x 256, ranks 16, smooth modes 1-2, 80 % missing, 15 % salt-and-pepper
  grad128 128^4, ranks 20, 10 % outliers, 2^24 sampled observed entries
  image   3 x 1352 x 2000 (a colour image, channel mode first so that the ring's cut keeps
          r_1 r_c = 60), ranks (3, 20, 20), fully observed (decomposition), noise on every
          entry from the two-component mixture 0.8 N(0, 1e-3) + 0.2 N(0, 0.5) on the [0, 1]
          scale (here scaled by the clean tensor's range), PSNR against the clean tensor
  imagec  the same image tensor and noise with 70 % of the entries missing (completion)
  videop  1920 x 1080 x 3 x 50 (a 50-frame colour video) at the paper's video TR rank
          (80, 80, 3, 20), 70 % missing, the image workloads' mixture noise on every entry,
          RStS sketch 200 per non-updated mode (J = 200 x 3 x 50 = 3e4 sampled fibres when a
          frame mode is updated)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    dims: Tuple[int, ...]
    ranks: Tuple[int, ...]
    missing: float                  # fraction of entries unobserved
    outlier_frac: float             # fraction of observed entries replaced
    outlier_kind: str = "uniform"   # 'uniform' U[-10 std, 10 std], 'saltpepper' or 'gmm'
                                    # (every entry noisy; outlier_frac = weight of the wide
                                    # component)
    noise_var: float = 0.0          # additive Gaussian noise variance
    sketch: Optional[int] = None    # RStS size per non-updated mode (None: full tensor)
    smooth_modes: Tuple[int, ...] = ()
    smooth_width: float = 0.0
    data_seed: int = 1000
    init_seed: int = 2000
    sample_seed: int = 3000
    n_sampled: int = 0              # sampled-entry workload (differentiation)


WORKLOADS = {
    "tiny3": Workload("tiny3", (30, 30, 30), (3, 3, 3), 0.3, 0.1,
                      data_seed=1001, init_seed=2001, sample_seed=3001),
    "cfg100": Workload("cfg100", (100, 100, 100, 100), (8, 8, 8, 8), 0.5, 0.2, noise_var=1e-3,
                       data_seed=1002, init_seed=2002, sample_seed=3002),
    "cfg64": Workload("cfg64", (64,) * 5, (10,) * 5, 0.7, 0.1, sketch=24,
                      data_seed=1003, init_seed=2003, sample_seed=3003),
    "video": Workload("video", (1024, 1024, 256), (16, 16, 16), 0.8, 0.15,
                      outlier_kind="saltpepper", sketch=128, smooth_modes=(0, 1),
                      smooth_width=8.0, data_seed=1004, init_seed=2004, sample_seed=3004),
    "grad128": Workload("grad128", (128,) * 4, (20,) * 4, 0.0, 0.1,
                        data_seed=1005, init_seed=2005, sample_seed=3005, n_sampled=1 << 24),
    "image": Workload("image", (3, 1352, 2000), (3, 20, 20), 0.0, 0.2, outlier_kind="gmm",
                      data_seed=1006, init_seed=2006, sample_seed=3006),
    "imagec": Workload("imagec", (3, 1352, 2000), (3, 20, 20), 0.7, 0.2, outlier_kind="gmm",
                       data_seed=1006, init_seed=2006, sample_seed=3006),
    "videop": Workload("videop", (1920, 1080, 3, 50), (80, 80, 3, 20), 0.7, 0.2, outlier_kind="gmm",
                       sketch=200, data_seed=1007, init_seed=2007, sample_seed=3007),
}

# variances of the two mixture components of the 'gmm' noise, on data rescaled to [0, 1]
GMM_VARS = (1e-3, 0.5)


def gaussian_cores(dims: Sequence[int], ranks: Sequence[int], seed: int,
                   smooth_modes: Sequence[int] = (), smooth_width: float = 0.0) -> List[np.ndarray]:
    """i.i.d. Gaussian cores Z_k of shape (r_k, I_k, r_{k+1}), variance 1/sqrt(r_k r_{k+1})
    (unit-variance entries for equal ranks).  Cores of `smooth_modes` are low-pass filtered
    along i with a periodic Gaussian of std `smooth_width` and rescaled to that variance."""
    rng = np.random.default_rng(seed)
    N = len(dims)
    cores = []
    for k in range(N):
        rk, rk1 = ranks[k], ranks[(k + 1) % N]
        std = (rk * rk1) ** -0.25
        Z = rng.standard_normal((rk, dims[k], rk1))
        if k in smooth_modes and smooth_width > 0:
            n = dims[k]
            off = np.minimum(np.arange(n), n - np.arange(n)).astype(np.float64)
            ker = np.exp(-0.5 * (off / smooth_width) ** 2)
            Z = np.real(np.fft.ifft(np.fft.fft(Z, axis=1) * np.fft.fft(ker)[None, :, None], axis=1))
            Z /= Z.std()
        cores.append(std * Z)
    return cores


def bernoulli_mask(dims: Sequence[int], observed: float, seed: int) -> np.ndarray:
    """Boolean observation mask, uniform Bernoulli(observed), numpy Fortran order."""
    rng = np.random.default_rng(seed + 7)
    n = int(np.prod(dims))
    return (rng.random(n) < observed).reshape(dims, order="F")


def pack_mask(mask: np.ndarray) -> np.ndarray:
    """Bit-pack a boolean tensor in linear (Fortran) order into uint32 words."""
    flat = np.asarray(mask, dtype=bool).reshape(-1, order="F")
    n_words = (flat.size + 31) // 32
    n_words = (n_words + 3) // 4 * 4
    bits = np.zeros(n_words * 32, dtype=bool)
    bits[: flat.size] = flat
    return np.packbits(bits, bitorder="little").view("<u4").astype(np.uint32)


def unpack_mask(words: np.ndarray, dims: Sequence[int]) -> np.ndarray:
    n = int(np.prod(dims))
    bits = np.unpackbits(np.asarray(words, dtype="<u4").view(np.uint8), bitorder="little")
    return bits[:n].astype(bool).reshape(dims, order="F")


@dataclass
class Corruption:
    """Random draws that turn a clean tensor into an observed one."""
    mask: np.ndarray                 # bool, observed entries
    outlier: np.ndarray              # bool, observed entries that are replaced
    outlier_u: np.ndarray            # float64 in [-1, 1] (uniform) or {-1, +1} (salt/pepper)
    noise: Optional[np.ndarray] = field(default=None)


def draw_corruption(w: Workload, dims: Optional[Sequence[int]] = None) -> Corruption:
    dims = tuple(dims or w.dims)
    mask = bernoulli_mask(dims, 1.0 - w.missing, w.data_seed)
    rng = np.random.default_rng(w.data_seed + 11)
    n = int(np.prod(dims))
    outl = (rng.random(n) < w.outlier_frac).reshape(dims, order="F")
    if w.outlier_kind == "saltpepper":
        # salt-and-pepper hits entries whether observed or not; only observed ones matter
        u = np.where(rng.random(n) < 0.5, -1.0, 1.0).reshape(dims, order="F")
    elif w.outlier_kind == "gmm":
        # every entry gets mixture noise: outl picks the wide component, u is N(0, 1)
        u = rng.standard_normal(n).reshape(dims, order="F")
    else:
        outl &= mask
        u = rng.uniform(-1.0, 1.0, n).reshape(dims, order="F")
    noise = None
    if w.noise_var > 0:
        noise = math.sqrt(w.noise_var) * np.random.default_rng(w.data_seed + 13).standard_normal(
            n).reshape(dims, order="F")
    return Corruption(mask, outl, u, noise)


def assemble(x_true, c: Corruption, kind: str = "uniform", scale: float = 10.0):
    """Observed tensor: x_true + noise, with outliers U[-scale std, scale std] (std of the
    clean entries) or salt-and-pepper (max or min of the clean tensor) at c.outlier.
    Works element-wise on numpy arrays."""
    x = np.array(x_true, dtype=np.float64, copy=True)
    if c.noise is not None:
        x = x + c.noise
    if kind == "saltpepper":
        hi, lo = float(np.max(x_true)), float(np.min(x_true))
        x = np.where(c.outlier, np.where(c.outlier_u > 0, hi, lo), x)
    elif kind == "gmm":
        # mixture noise on the [0, 1] scale: standard deviations times the clean range
        rng_ = float(np.max(x_true)) - float(np.min(x_true))
        sd = np.where(c.outlier, math.sqrt(GMM_VARS[1]), math.sqrt(GMM_VARS[0]))
        x = x + rng_ * sd * c.outlier_u
    else:
        std = float(np.std(x_true))
        x = np.where(c.outlier, scale * std * c.outlier_u, x)
    return x


def corruption_chunks(w: Workload, chunk: int = 1 << 26):
    """Chunked form of the corruption draw for tensors too large for whole-tensor arrays:
    yields (start, mask, outlier, u, noise) over consecutive linear-index ranges.  Each
    component has its own generator (mask: data_seed + 7, outlier: + 11, u: + 12, noise:
    + 13), drawn sequentially chunk after chunk, so the result does not depend on `chunk`.
    Same distributions as draw_corruption; a different stream from it."""
    n = int(np.prod(w.dims))
    g_mask = np.random.default_rng(w.data_seed + 7)
    g_out = np.random.default_rng(w.data_seed + 11)
    g_u = np.random.default_rng(w.data_seed + 12)
    g_noise = np.random.default_rng(w.data_seed + 13) if w.noise_var > 0 else None
    for s in range(0, n, chunk):
        c = min(chunk, n - s)
        mask = g_mask.random(c) < (1.0 - w.missing)
        outl = g_out.random(c) < w.outlier_frac
        if w.outlier_kind == "saltpepper":
            u = np.where(g_u.random(c) < 0.5, -1.0, 1.0)
        elif w.outlier_kind == "gmm":
            u = g_u.standard_normal(c)
        else:
            outl &= mask
            u = g_u.uniform(-1.0, 1.0, c)
        noise = math.sqrt(w.noise_var) * g_noise.standard_normal(c) if g_noise is not None else None
        yield s, mask, outl, u, noise


def assemble_chunk(x_true, outl, u, noise, kind: str, std: float, lo: float, hi: float,
                   scale: float = 10.0):
    """assemble() for one chunk, with the clean tensor's std / min / max given."""
    x = np.array(x_true, dtype=np.float64, copy=True)
    if noise is not None:
        x = x + noise
    if kind == "saltpepper":
        return np.where(outl, np.where(u > 0, hi, lo), x)
    if kind == "gmm":
        sd = np.where(outl, math.sqrt(GMM_VARS[1]), math.sqrt(GMM_VARS[0]))
        return x + (hi - lo) * sd * u
    return np.where(outl, scale * std * u, x)


def sample_entries(dims: Sequence[int], M: int, seed: int) -> np.ndarray:
    """About M distinct multi-indices (rows of an int32 array, N columns), sorted by linear
    index: each entry is kept independently with probability M / numel (a few draws more),
    then the first M are returned (fewer when the draw falls short)."""
    rng = np.random.default_rng(seed)
    n = int(np.prod(dims))
    p = min(1.0, M / n * 1.001 + 64.0 / n)
    lin = np.flatnonzero(rng.random(n) < p)[:M]
    idx = np.stack(np.unravel_index(lin, dims, order="F"), axis=1)
    return np.ascontiguousarray(idx.astype(np.int32))
