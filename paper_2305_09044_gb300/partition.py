"""Partitioned core update: one problem split over several handles (one per GPU).

The data terms of a core update are sums over the columns j of the unfolding X_[k] (Eq. hatd
for d, the exact line search of Sec. 3.2 for its denominator), while the FGMC Gram G
(Prop. 2), the factorisation of G + lambda I and the step direction h = d (G + lambda I)^-1
depend only on the cores and on d.  Splitting the columns over P handles therefore needs one
exchange step per core update and nothing else:

  1. every handle: residuals, weights and the partial d over its columns (data pass 1);
  2. all-reduce (sum) of d -- I_k x K doubles;
  3. every handle: h from the summed d (replicated), <d, h>, and the partial line-search
     denominator sum w (h B^T)^2 over its columns (data pass 2);
  4. all-reduce (sum) of the denominator -- one double;
  5. every handle applies Z_k <- Z_k + eta fold(h) with eta = <d, h> / sum of denominators.

The columns are split by a contiguous range of one non-updated mode (the largest, so every
part has work), selected on each handle with trd_sample_subtensor; inside a sketched update
(RStS) the range applies to that mode's sketch indices.  The cores, G and h stay replicated,
so after every update all handles hold identical cores.  The exchange is a caller-supplied
sum over parts: torch.distributed all_reduce (NCCL between GPUs, gloo on CPU ranks) through
`torch_allreduce`, or a plain host sum when one process drives several handles.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence

import numpy as np


def part_range(n: int, part: int, nparts: int):
    """Contiguous range [lo, hi) of part `part` of `nparts` over n items."""
    return n * part // nparts, n * (part + 1) // nparts


def split_mode(dims: Sequence[int], k: int, sketch: Optional[Sequence[Optional[Sequence[int]]]] = None) -> int:
    """The non-updated mode whose (sketch) indices are split: the largest one, the last on ties."""
    sizes = [(len(sketch[m]) if sketch is not None and sketch[m] is not None else dims[m]) if m != k else -1
             for m in range(len(dims))]
    best = max(sizes)
    return max(m for m in range(len(dims)) if sizes[m] == best)


def part_indices(dims: Sequence[int], k: int, part: int, nparts: int,
                 sketch: Optional[Sequence[Optional[Sequence[int]]]] = None) -> List[Optional[np.ndarray]]:
    """Index sets (trd_sample_subtensor form: None = whole mode) selecting this part's columns."""
    N = len(dims)
    m = split_mode(dims, k, sketch)
    idx: List[Optional[np.ndarray]] = [None] * N
    for j in range(N):
        if j != k and sketch is not None and sketch[j] is not None:
            idx[j] = np.asarray(sketch[j], dtype=np.int64)
    base = idx[m] if idx[m] is not None else np.arange(dims[m], dtype=np.int64)
    lo, hi = part_range(len(base), part, nparts)
    idx[m] = base[lo:hi]
    return idx


class PartitionedUpdate:
    """The phases of one partitioned update of core k on one handle, between the exchanges.

    handle: a binding.TRD (or any object with the same methods); part / nparts: this handle's
    share of the columns; sketch: optional RStS index sets of the update (None entries = whole
    mode)."""

    def __init__(self, handle, k: int, part: int, nparts: int, sigma: float, lam: float = -1e-10,
                 gram: str = "global", sketch=None):
        self.t, self.k, self.sigma, self.lam, self.gram = handle, k, sigma, lam, gram
        self.idx = part_indices(handle.dims, k, part, nparts, sketch)
        if len(self.idx[split_mode(handle.dims, k, sketch)]) == 0:
            raise ValueError("more parts than indices of the split mode")
        self.num = None

    def partial_gradient(self) -> np.ndarray:
        """Phase 1: this part's residual statistics and partial d (I_k x K)."""
        t, k = self.t, self.k
        t.sample_subtensor(k, self.idx)
        self.stats = t.residual_weights(k, self.sigma)
        return t.core_gradient(k)

    def partial_denominator(self, d_total: np.ndarray) -> float:
        """Phase 2: install the summed d, form h, <d, h> and this part's denominator."""
        self.t.set_gradient(self.k, d_total)
        self.num, den = self.t.line_search_terms(self.k, self.lam, self.gram)
        return den

    def apply(self, den_total: float) -> float:
        """Phase 3: the global exact step eta = <d, h> / den_total, applied to core k."""
        eta = self.num / den_total if den_total > 0 else 0.0
        if eta > 0:
            self.t.core_update(self.k, self.lam, eta=eta, gram=self.gram)
        return eta


def partitioned_core_update(handle, k: int, sigma: float, allreduce: Callable[[np.ndarray], np.ndarray],
                            part: int, nparts: int, lam: float = -1e-10, gram: str = "global",
                            sketch=None) -> dict:
    """One partitioned update of core k on this part; `allreduce` sums an array over the
    parts.  Returns eta and the summed residual statistics."""
    pu = PartitionedUpdate(handle, k, part, nparts, sigma, lam, gram, sketch)
    d = allreduce(pu.partial_gradient())
    st = allreduce(np.array([pu.stats["n_obs"], pu.stats["sum_w"], pu.stats["sum_we2"]], dtype=np.float64))
    den = float(allreduce(np.array([pu.partial_denominator(d)]))[0])
    eta = pu.apply(den)
    return {"eta": eta, "n_obs": int(st[0]), "sum_w": float(st[1]), "objective": 0.5 * float(st[2])}


def torch_allreduce(group=None, device: Optional[str] = None) -> Callable[[np.ndarray], np.ndarray]:
    """Sum over the ranks of a torch.distributed process group: FP64 tensors on `device`
    ('cuda' for NCCL, 'cpu' for gloo; default: cuda when the group's backend is NCCL)."""
    import torch
    import torch.distributed as dist
    if device is None:
        device = "cuda" if dist.get_backend(group) == "nccl" else "cpu"

    def _sum(a: np.ndarray) -> np.ndarray:
        x = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(device)
        dist.all_reduce(x, op=dist.ReduceOp.SUM, group=group)
        return x.cpu().numpy()

    return _sum
