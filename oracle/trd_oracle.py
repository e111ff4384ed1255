"""FP64 CPU oracle for the per-core hot path of AWRTRD / SAWRTRD.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / reference leg of ``bench.py`` may import this module.  It
shares no code with the CUDA path: it restates He & Atia, "Scalable and Robust Tensor
Ring Decomposition for Large-scale Data" (UAI 2023) step by step in plain numpy float64,
in the paper's order and notation.  Indices are 0-based here (the paper's are 1-based).

Conventions (all from the paper):
  * A TR core Z_k has shape (r_k, I_k, r_{k+1}) with r_{N+1} = r_1 (Def. 1).
  * The multi-index overline{i_1 ... i_N} puts i_1 fastest (Def. 2), i.e. numpy
    Fortran order; a tensor is stored flat in that order.
  * Z_{k(2)} is the classical mode-2 unfolding, I_k x (r_k r_{k+1}), column alpha + beta*r_k.
  * X_[k] is the cyclic mode-k unfolding of Thm. 1, columns overline{i_{k+1}..i_N i_1..i_{k-1}}.

Readings where the paper is silent or garbled (each is listed in the design notes):
  * weight sign: w = -g'(e)/e = exp(-e^2/(2 sigma^2)) in (0, 1]  (Eq. updatew with Eq. corr)
  * update sign: Z_k <- Z_k + eta fold(h); d of Eq. sd is the negative gradient (Eq. updatessd)
  * FGMC's Phi is the realignment G[a + b q, a' + b' q] = T[b p + b', a q + a'] (Prop. 2)
  * sketch size s_j = min(I_j, ceil(J^(1/(N-1)))) (Sec. 3.3, Algorithm 1)
  * no rescaling of the sketched gradient; W is recomputed per core update
  * adaptive sigma (cited but not stated by the paper, Sec. 5): PARITY UNPINNED against
    the paper; sigma = max(sigma_min, 2 min(std(e), IQR(e)/1.349)).
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np

# ----------------------------------------------------------------------------------------
# Counter-based generator: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014; Vigna's public
# reference implementation).  Used for core initialisation and RStS index draws, so the
# random numbers the method draws are defined independently of either implementation.
# ----------------------------------------------------------------------------------------
_M64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


def splitmix64_mix(z: int) -> int:
    """SplitMix64 output function (the variant-13 finaliser) on one 64-bit word."""
    z &= _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def splitmix64_stream(seed: int, n: int) -> List[int]:
    """First n outputs of SplitMix64 seeded with `seed` (output m = mix(seed + (m+1) gamma))."""
    return [splitmix64_mix((seed + (m + 1) * GOLDEN_GAMMA) & _M64) for m in range(n)]


def _splitmix64_vec(seed: int, counters: np.ndarray) -> np.ndarray:
    """Vectorised output `counters` of the stream seeded with `seed` (uint64 wrap-around)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counters.astype(np.uint64) + np.uint64(1)) * np.uint64(GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def gaussian_from_counter(seed: int, g: np.ndarray) -> np.ndarray:
    """Standard normal number g of the init stream: Box-Muller (1958) on the
    outputs 2g and 2g+1, u1 = ((z>>11)+1) 2^-53 in (0,1], u2 = (z>>11) 2^-53 in [0,1)."""
    z1 = _splitmix64_vec(seed, 2 * g)
    z2 = _splitmix64_vec(seed, 2 * g + 1)
    u1 = ((z1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (z2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def init_cores(dims: Sequence[int], ranks: Sequence[int], seed: int, stddev: float = -1.0):
    """Algorithm 1 initialisation (the paper leaves the law unstated).  Reading: i.i.d.
    N(0, s^2) with s = (r_k r_{k+1})^(-1/4) unless stddev > 0.  Entry (alpha, i, beta) of
    core k takes global counter base_k + (i r_{k+1} + beta) r_k + alpha, base_k being the
    number of entries of the cores before k."""
    N = len(dims)
    cores = []
    base = 0
    for k in range(N):
        rk, rk1, Ik = ranks[k], ranks[(k + 1) % N], dims[k]
        s = stddev if stddev > 0 else (rk * rk1) ** -0.25
        n = rk * Ik * rk1
        g = base + np.arange(n, dtype=np.uint64)
        vals = s * gaussian_from_counter(seed, g)
        # flat order (i, beta, alpha) -> core[alpha, i, beta]
        cores.append(np.ascontiguousarray(vals.reshape(Ik, rk1, rk).transpose(2, 0, 1)))
        base += n
    return cores


def draw_indices(seed: int, t: int, k: int, j: int, N: int, I: int, s: int) -> np.ndarray:
    """RStS index set I_j for core update k of outer iteration t (Algorithm 1, step
    'randomly generate index set'): s distinct indices from [0, I), uniform, without
    replacement, sorted.  Key = output (t N + k) N + j of the seed stream; then a partial
    Fisher-Yates shuffle (Durstenfeld 1964) driven by the key's stream, pick m uniform on
    [m, I) as m + (z_m mod (I - m))."""
    if s >= I:
        return np.arange(I, dtype=np.int64)
    key = splitmix64_mix((seed + ((t * N + k) * N + j + 1) * GOLDEN_GAMMA) & _M64)
    z = splitmix64_stream(key, s)
    perm = list(range(I))
    for m in range(s):
        pick = m + (z[m] % (I - m))
        perm[m], perm[pick] = perm[pick], perm[m]
    return np.sort(np.array(perm[:s], dtype=np.int64))


def sketch_sizes(J: float, dims: Sequence[int], k: int) -> List[int]:
    """Sec. 3.3 / Algorithm 1 sketch sizes.  The printed formula is dimensionally garbled;
    reading: s_k = I_k and s_j = min(I_j, ceil(J^(1/(N-1)))) for j != k."""
    N = len(dims)
    per = math.ceil(J ** (1.0 / (N - 1)) - 1e-9)
    return [dims[m] if m == k else min(dims[m], per) for m in range(N)]


# ----------------------------------------------------------------------------------------
# Tensor-ring algebra: Def. 1, Def. 2, Thm. 1
# ----------------------------------------------------------------------------------------

def merge(Za: np.ndarray, Zb: np.ndarray) -> np.ndarray:
    """Def. 2 core merging: Z^{(a,b)}(overline{i_a i_b}) = Z_a(i_a) Z_b(i_b), i_a fastest."""
    ra, Ia, _ = Za.shape
    _, Ib, rc = Zb.shape
    out = np.tensordot(Za, Zb, axes=(2, 0))            # [x, i_a, i_b, z] = (Z_a(i_a) Z_b(i_b))[x, z]
    return out.reshape(ra, Ia * Ib, rc, order="F")     # overline{i_a i_b} = i_a + i_b I_a


def subchain(cores: Sequence[np.ndarray], k: int) -> np.ndarray:
    """Thm. 1 subchain Z^{!=k}: merge Z_{k+1}, ..., Z_N, Z_1, ..., Z_{k-1} in that order.
    Shape (r_{k+1}, prod_{j!=k} I_j, r_k); slice index overline{i_{k+1}..i_N i_1..i_{k-1}}."""
    N = len(cores)
    order = [(k + 1 + m) % N for m in range(N - 1)]
    S = cores[order[0]]
    for m in order[1:]:
        S = merge(S, cores[m])
    return S


def mode2(Z: np.ndarray) -> np.ndarray:
    """Classical mode-2 unfolding of a 3-way array (p, I, q): M[i, a + b p] = Z[a, i, b]."""
    p, I, q = Z.shape
    return Z.transpose(1, 2, 0).reshape(I, q * p)   # column b*p + a


def fold2(M: np.ndarray, p: int, q: int) -> np.ndarray:
    """Inverse of mode2 (the paper's fold)."""
    I = M.shape[0]
    return M.reshape(I, q, p).transpose(2, 0, 1)


def cyclic_unfold2(S: np.ndarray) -> np.ndarray:
    """Cyclic mode-2 unfolding Z_[2] of a 3-way array (p, J, q) (Thm. 1, [n] unfolding):
    columns overline{i_3 i_1} = i_3 + i_1 q, i.e. B[j, a + b q] = S[b, j, a]."""
    p, J, q = S.shape
    return S.transpose(1, 0, 2).reshape(J, p * q)    # column b*q + a


def unfold_k(X: np.ndarray, k: int) -> np.ndarray:
    """Thm. 1: X_[k](i_k, overline{i_{k+1}..i_N i_1..i_{k-1}}) = X(i_1..i_N)."""
    N = X.ndim
    axes = [k] + [(k + 1 + m) % N for m in range(N - 1)]
    Xt = np.transpose(X, axes)
    return Xt.reshape(X.shape[k], -1, order="F")


def reconstruct(cores: Sequence[np.ndarray]) -> np.ndarray:
    """Def. 1: X(i_1..i_N) = Tr(prod_k Z_k(i_k)), via merging all cores (Def. 2)."""
    S = cores[0]
    for Z in cores[1:]:
        S = merge(S, Z)
    vals = np.einsum("aja->j", S)
    return vals.reshape([Z.shape[1] for Z in cores], order="F")


def reconstruct_unfold(cores: Sequence[np.ndarray]) -> np.ndarray:
    """Thm. 1 with k = 1: X_[1] = Z_{1(2)} (Z^{!=1}_[2])^T, folded back (i_1 fastest)."""
    B = cyclic_unfold2(subchain(cores, 0))
    X1 = mode2(cores[0]) @ B.T
    return X1.reshape([Z.shape[1] for Z in cores], order="F")


def reconstruct_chunks(cores: Sequence[np.ndarray], c: int, cols: int):
    """Def. 1 for tensors too large to form a subchain of N - 1 cores: cut the ring after
    core c, merge both halves (Def. 2), A = Z^{(1..c)} of shape (r_1, P_in, r_{c+1}) and
    C = Z^{(c+1..N)} of shape (r_{c+1}, P_out, r_1); then X(a + P_in b) = Tr(A(a) C(b)) =
    sum_{x,z} A[x, a, z] C[z, b, x].  Yields (start, values) for consecutive column blocks
    of `cols` outer indices b, in linear (i_1 fastest) order."""
    A = cores[0]
    for Z in cores[1:c]:
        A = merge(A, Z)
    C = cores[c]
    for Z in cores[c + 1:]:
        C = merge(C, Z)
    r1, P_in, rc = A.shape
    P_out = C.shape[1]
    Ahat = A.transpose(1, 0, 2).reshape(P_in, r1 * rc)          # [a, x rc + z]
    for b0 in range(0, P_out, cols):
        b1 = min(P_out, b0 + cols)
        Chat = C[:, b0:b1, :].transpose(1, 2, 0).reshape(b1 - b0, r1 * rc)   # [b, x rc + z]
        yield b0 * P_in, (Ahat @ Chat.T).reshape(-1, order="F")


def entry(cores: Sequence[np.ndarray], idx: Sequence[int]) -> float:
    """Def. 1 for one entry, by explicit matrix products."""
    M = np.eye(cores[0].shape[0])
    for Z, i in zip(cores, idx):
        M = M @ Z[:, i, :]
    return float(np.trace(M))


# ----------------------------------------------------------------------------------------
# Correntropy, HQ weights (Eq. corr, Eq. hq_w2, Eq. updatew)
# ----------------------------------------------------------------------------------------

def g_sigma(x, sigma):
    """Gaussian kernel of Eq. corr: g(x) = sigma^2 exp(-x^2 / (2 sigma^2))."""
    return sigma ** 2 * np.exp(-np.asarray(x, dtype=np.float64) ** 2 / (2.0 * sigma ** 2))


def hq_weight(e, sigma):
    """Eq. updatew with the sign reading: w = -g'(e)/e = exp(-e^2/(2 sigma^2)); w(0) = 1;
    sigma = +inf gives w = 1 (Sec. 3.2, the sigma -> infinity limit)."""
    e = np.asarray(e, dtype=np.float64)
    if math.isinf(sigma):
        return np.ones_like(e)
    return np.exp(-(e * e) / (2.0 * sigma * sigma))


def welsch_loss(e, sigma):
    """sum sigma^2 (1 - exp(-e^2/(2 sigma^2))) = sum (sigma^2 - g_sigma(e)): minimising it
    maximises the correntropy objective of Eq. corr."""
    e = np.asarray(e, dtype=np.float64)
    return float(np.sum(sigma ** 2 - g_sigma(e, sigma)))


# ----------------------------------------------------------------------------------------
# FGMC (Prop. 2)
# ----------------------------------------------------------------------------------------

def fgmc_Q(Z: np.ndarray, swap: bool = False) -> np.ndarray:
    """Prop. 2: Q(:, i r_{k+1} + j) = vec(Z(:,:,i) Z(:,:,j)^T) (vec column-major); with
    swap=True (the first core when the chain length c is odd) the factors are exchanged."""
    rk, Ik, rk1 = Z.shape
    Q = np.empty((rk * rk, rk1 * rk1))
    for i in range(rk1):
        for j in range(rk1):
            M = Z[:, :, j] @ Z[:, :, i].T if swap else Z[:, :, i] @ Z[:, :, j].T
            Q[:, i * rk1 + j] = M.reshape(-1, order="F")
    return Q


def fgmc_Phi(T: np.ndarray, p: int, q: int) -> np.ndarray:
    """Phi of Prop. 2 (undefined in the paper; reading): realign the (p^2 x q^2) chain
    product into the (pq x pq) Gram, G[a + b q, a' + b' q] = T[b p + b', a q + a'] for a
    subchain whose slices are p x q."""
    G = np.empty((p * q, p * q))
    for b in range(p):
        for b2 in range(p):
            for a in range(q):
                for a2 in range(q):
                    G[a + b * q, a2 + b2 * q] = T[b * p + b2, a * q + a2]
    return G


def fgmc_gram(cores: Sequence[np.ndarray], k: int) -> np.ndarray:
    """Eq. FGMC for the subchain Z^{!=k}: the chain starts at core k+1 and has c = N-1
    factors; Q of its first core is swapped when c is odd.  Returns G = B^T B (K x K,
    K = r_k r_{k+1}) without forming B."""
    N = len(cores)
    order = [(k + 1 + m) % N for m in range(N - 1)]
    c = N - 1
    T = fgmc_Q(cores[order[0]], swap=(c % 2 == 1))
    for m in order[1:]:
        T = T @ fgmc_Q(cores[m])
    p = cores[order[0]].shape[0]      # r_{k+1}
    q = cores[order[-1]].shape[2]     # r_k
    return fgmc_Phi(T, p, q)


def explicit_gram(cores: Sequence[np.ndarray], k: int) -> np.ndarray:
    """G = (Z^{!=k}_[2])^T Z^{!=k}_[2] formed explicitly (Eq. sg), for checking FGMC."""
    B = cyclic_unfold2(subchain(cores, k))
    return B.T @ B


# ----------------------------------------------------------------------------------------
# Cholesky (written out; Eq. sg needs (G + lambda I)^{-1})
# ----------------------------------------------------------------------------------------

def cholesky(A: np.ndarray) -> np.ndarray:
    """Lower-triangular L with A = L L^T (Cholesky-Banachiewicz, column by column)."""
    n = A.shape[0]
    L = np.zeros_like(A, dtype=np.float64)
    for j in range(n):
        s = A[j, j] - np.dot(L[j, :j], L[j, :j])
        if not s > 0.0:
            raise np.linalg.LinAlgError(f"matrix not positive definite at pivot {j}")
        L[j, j] = math.sqrt(s)
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def right_solve_spd(d: np.ndarray, A: np.ndarray) -> np.ndarray:
    """h = d A^{-1} for SPD A via A = L L^T: solve L y = d^T, L^T h^T = y, column by column."""
    L = cholesky(A)
    n = A.shape[0]
    Y = np.array(d.T, dtype=np.float64)
    for j in range(n):                       # forward substitution
        Y[j] = (Y[j] - L[j, :j] @ Y[:j]) / L[j, j]
    for j in range(n - 1, -1, -1):           # back substitution
        Y[j] = (Y[j] - L[j + 1:, j] @ Y[j + 1:]) / L[j, j]
    return Y.T


def resolve_lambda(lam: float, G: np.ndarray) -> float:
    """Eq. sg regulariser ('sufficiently small'): lam >= 0 is absolute; lam < 0 means
    |lam| tr(G)/K."""
    return lam if lam >= 0 else abs(lam) * float(np.trace(G)) / G.shape[0]


# ----------------------------------------------------------------------------------------
# One core update (Sec. 3.2 steps 1-2; Sec. 3.3 with a sketch; Algorithm 1 inner loop)
# ----------------------------------------------------------------------------------------

class CoreStep:
    """Everything one core update produces, for step-by-step parity checks."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def core_update(X: np.ndarray, P: np.ndarray, cores: List[np.ndarray], k: int, sigma: float,
                lam: float = -1e-10, eta: Optional[float] = None,
                sample: Optional[Sequence[np.ndarray]] = None,
                gram: str = "global") -> CoreStep:
    """One update of core k (0-based).

    X, P    : full data tensor and 0/1 mask (numpy arrays, shape I_1 x ... x I_N)
    sample  : None (AWRTRD, full tensor) or the RStS index sets I_j (I_k ignored, kept full)
    sigma   : kernel width (inf gives W = 1)
    lam     : Eq. sg regulariser (see resolve_lambda)
    eta     : None for the exact line search, else a fixed step size
    gram    : 'global' (Eq. hI: G from the full cores by FGMC), 'local' (ablation 'local
              scaled term': explicit Gram of the sampled subchain), 'none' (ablation
              'gradient descent': h = d)
    Returns a CoreStep with the new core list in .cores (the input list is not modified).
    """
    N = X.ndim
    rk, rk1 = cores[k].shape[0], cores[k].shape[2]
    if sample is None:
        XI, PI, cs = X, P, list(cores)
    else:
        idx = [np.arange(X.shape[m]) if m == k else np.asarray(sample[m]) for m in range(N)]
        XI = X[np.ix_(*idx)]                                  # RStS sketch X_I (Sec. 3.2.2)
        PI = P[np.ix_(*idx)]
        cs = [cores[m][:, idx[m], :] for m in range(N)]       # sampled cores (Z_m)_{I_m}
    B = cyclic_unfold2(subchain(cs, k))                       # Z^{!=k}_{I[2]}
    Xk = unfold_k(XI, k)                                      # X_{I[k]}
    Pk = unfold_k(PI, k).astype(np.float64)
    Zk2 = mode2(cores[k])                                     # Z_{k(2)}
    Xhat = Zk2 @ B.T                                          # Thm. 1
    E = Xk - Xhat                                             # residual
    W = hq_weight(E, sigma)                                   # Eq. updatew
    Y = W * Pk * E
    d = Y @ B                                                 # Eq. sd / Eq. hatd
    if gram == "global":
        G = fgmc_gram(cores, k)                               # Eq. FGMC, full cores
    elif gram == "local":
        G = B.T @ B
    elif gram == "none":
        G = None
    else:
        raise ValueError(gram)
    if G is None:
        lam_used, h = 0.0, d.copy()
    else:
        lam_used = resolve_lambda(lam, G)
        h = right_solve_spd(d, G + lam_used * np.eye(G.shape[0]))   # Eq. sg / Eq. hI
    num = float(np.sum(d * h))                                # <d, h>
    HB = h @ B.T
    den = float(np.sum(W * Pk * HB * HB))                     # ||sqrt(W) o P o (h B^T)||^2
    eta_used = (num / den if den > 0 else 0.0) if eta is None else float(eta)
    new = list(cores)
    new[k] = fold2(Zk2 + eta_used * h, rk, rk1)               # Eq. updatessd (sign reading)
    obs = Pk > 0
    return CoreStep(cores=new, d=d, G=G, h=h, num=num, den=den, eta=eta_used,
                    lam=lam_used, sum_w=float(np.sum(W[obs])),
                    sum_e2=float(np.sum(E[obs] ** 2)), n_obs=int(obs.sum()),
                    objective=float(0.5 * np.sum(W * Pk * E * E)))


def sampled_rows(cores: Sequence[np.ndarray], k: int, rows: np.ndarray) -> np.ndarray:
    """Rows of Z^{!=k}_[2] at the multi-indices `rows` (J x N integer array, column k
    ignored): S(j) = Z_{k+1}(i_{k+1}) ... Z_N(i_N) Z_1(i_1) ... Z_{k-1}(i_{k-1}) (Thm. 1
    order), unfolded as in cyclic_unfold2: B[j, a + b r_k] = S(j)[b, a].  Shape J x K."""
    N = len(cores)
    order = [(k + 1 + m) % N for m in range(N - 1)]
    S = cores[order[0]][:, rows[:, order[0]], :]                       # (r_{k+1}, J, .)
    for m in order[1:]:
        S = np.einsum("ajb,bjc->ajc", S, cores[m][:, rows[:, m], :])   # slice products per j
    return cyclic_unfold2(S)


def row_fibres(X: np.ndarray, k: int, rows: np.ndarray) -> np.ndarray:
    """Columns of X_[k] at the sampled multi-indices: F[i, j] = X(rows[j] with i_k = i)."""
    idx = tuple(rows[:, m] for m in range(X.ndim))
    out = np.empty((X.shape[k], rows.shape[0]), dtype=np.float64)
    for i in range(X.shape[k]):
        full = list(idx)
        full[k] = np.full(rows.shape[0], i)
        out[i] = X[tuple(full)]
    return out


def core_update_rows(X: np.ndarray, P: np.ndarray, cores: List[np.ndarray], k: int, sigma: float,
                     rows: np.ndarray, lam: float = -1e-10, eta: Optional[float] = None,
                     gram: str = "global") -> CoreStep:
    """Ablation 'uniform row sampling' (Sec. 5, ablation experiments): Z^{!=k}_{I[2]} is a set
    of sampled rows of Z^{!=k}_[2] (the multi-indices `rows`, J x N, column k ignored)
    instead of the RStS sketch; X_{I[k]} and P_{I[k]} are the matching columns of X_[k] and
    P_[k].  Every other step as in core_update (Eq. updatew, Eq. hatd, Eq. hI, line search)."""
    rk, rk1 = cores[k].shape[0], cores[k].shape[2]
    B = sampled_rows(cores, k, rows)                           # Z^{!=k}_{I[2]}
    Xk = row_fibres(X, k, rows)                                # X_{I[k]}
    Pk = row_fibres(P.astype(np.float64), k, rows)
    Zk2 = mode2(cores[k])
    E = Xk - Zk2 @ B.T                                         # Thm. 1
    W = hq_weight(E, sigma)                                    # Eq. updatew
    d = (W * Pk * E) @ B                                       # Eq. hatd
    if gram == "global":
        G = fgmc_gram(cores, k)
    elif gram == "local":
        G = B.T @ B
    elif gram == "none":
        G = None
    else:
        raise ValueError(gram)
    if G is None:
        lam_used, h = 0.0, d.copy()
    else:
        lam_used = resolve_lambda(lam, G)
        h = right_solve_spd(d, G + lam_used * np.eye(G.shape[0]))
    num = float(np.sum(d * h))
    HB = h @ B.T
    den = float(np.sum(W * Pk * HB * HB))
    eta_used = (num / den if den > 0 else 0.0) if eta is None else float(eta)
    new = list(cores)
    new[k] = fold2(Zk2 + eta_used * h, rk, rk1)
    obs = Pk > 0
    return CoreStep(cores=new, d=d, G=G, h=h, num=num, den=den, eta=eta_used, lam=lam_used,
                    sum_w=float(np.sum(W[obs])), sum_e2=float(np.sum(E[obs] ** 2)),
                    n_obs=int(obs.sum()), objective=float(0.5 * np.sum(W * Pk * E * E)))


def draw_rows(seed: int, t: int, k: int, dims: Sequence[int], J: int) -> np.ndarray:
    """J multi-indices drawn i.i.d. uniformly (with replacement) for core update k of
    iteration t: entry m of row j is z mod I_m with z = output (j (N + 1) + m) of the
    SplitMix64 stream keyed by output (t N + k) N + N of the seed's stream (the RStS keys use
    outputs (t N + k) N + j, j < N); column k is 0."""
    N = len(dims)
    key = splitmix64_mix((seed + ((t * N + k) * N + N + 1) * GOLDEN_GAMMA) & _M64)
    z = splitmix64_stream(key, J * (N + 1))
    out = np.zeros((J, N), dtype=np.int64)
    for j in range(J):
        for m in range(N):
            if m != k:
                out[j, m] = z[j * (N + 1) + m] % dims[m]
    return out


def weighted_objective(X, P, cores, W=None):
    """0.5 ||sqrt(W) o P o (X - R(Z))||_F^2 (the data term of Eq. tc_hq)."""
    E = (X - reconstruct(cores)) * P
    return 0.5 * float(np.sum(E * E if W is None else W * E * E))


# ----------------------------------------------------------------------------------------
# Stopping rule (Algorithm 1) and recovery error
# ----------------------------------------------------------------------------------------

def D_matrix(cores: Sequence[np.ndarray]) -> np.ndarray:
    """Algorithm 1: D^t = Z_{N(2)} G_{Z^{!=N}} Z_{N(2)}^T (equals X_[N] X_[N]^T)."""
    N = len(cores)
    ZN = mode2(cores[N - 1])
    return ZN @ fgmc_gram(cores, N - 1) @ ZN.T


def stop_error(D_new: np.ndarray, D_old: np.ndarray) -> float:
    """Algorithm 1: e = ||D^t - D^{t-1}||_F / ||D^t||_F."""
    return float(np.linalg.norm(D_new - D_old) / np.linalg.norm(D_new))


def relative_error(cores, X_true) -> float:
    """||R(Z) - X_true||_F / ||X_true||_F over all entries."""
    return float(np.linalg.norm(reconstruct(cores) - X_true) / np.linalg.norm(X_true))


def psnr(X_hat, X_ref, peak: float = 1.0) -> float:
    """Peak signal-to-noise ratio between the recovered and the original data, the quality
    measure of Sec. 5: 10 log10(peak^2 / MSE) with MSE the mean squared difference over all
    entries (peak = 1 for data rescaled to [0, 1]; +inf for identical tensors)."""
    mse = float(np.mean((np.asarray(X_hat, dtype=np.float64) - np.asarray(X_ref, dtype=np.float64)) ** 2))
    return math.inf if mse == 0.0 else 10.0 * math.log10(peak * peak / mse)


# ----------------------------------------------------------------------------------------
# Adaptive kernel width (Sec. 5 cites a rule it does not state).  PARITY UNPINNED.
# ----------------------------------------------------------------------------------------

def adaptive_sigma(resid_obs: np.ndarray, x_obs_rms: float, sigma_prev: Optional[float] = None,
                   c_sigma: float = 2.0, rho: float = 0.9) -> float:
    """Reading: sigma_t = max(1e-6 rms(X_obs), c_sigma min(std(e), IQR(e)/1.349),
    rho sigma_{t-1}) with the population std and type-7 (linear interpolation) quartiles
    of the observed residuals e.  The rho-limiter keeps the width from shrinking faster
    than the fit converges (without it the width collapses onto the best-fit subset)."""
    e = np.asarray(resid_obs, dtype=np.float64)
    std = float(np.sqrt(np.mean((e - e.mean()) ** 2)))
    q1, q3 = np.percentile(e, [25.0, 75.0])               # numpy 'linear' = type 7
    s = max(1e-6 * x_obs_rms, c_sigma * min(std, (q3 - q1) / 1.349))
    if sigma_prev is not None and math.isfinite(sigma_prev):
        s = max(s, rho * sigma_prev)
    return s


# ----------------------------------------------------------------------------------------
# Algorithm 1: one outer iteration
# ----------------------------------------------------------------------------------------

def sawrtrd_iteration(X, P, cores, sigma, t, *, lam=-1e-10, sizes=None, seed=0,
                      D_prev=None, gram="global"):
    """One REPEAT pass of Algorithm 1: for k = 1..N sample (if sizes given), reweight,
    gradient, FGMC Gram, update; then D^t and the stopping quantity e.
    sizes: None for AWRTRD (full tensor) or per-core lists s (s[k] ignored)."""
    N = X.ndim
    steps = []
    if D_prev is None:
        D_prev = D_matrix(cores)
    for k in range(N):
        sample = None
        if sizes is not None:
            sample = [None if m == k else
                      draw_indices(seed, t, k, m, N, X.shape[m], sizes[k][m]) for m in range(N)]
        st = core_update(X, P, cores, k, sigma, lam=lam, sample=sample, gram=gram)
        steps.append(st)
        cores = st.cores
    D = D_matrix(cores)
    return cores, stop_error(D, D_prev), D, steps


# ----------------------------------------------------------------------------------------
# Sampled correntropy loss and its adjoint (differentiation pattern built on Def. 1, Eq. corr)
# ----------------------------------------------------------------------------------------

def sampled_loss_grad(cores, idx: np.ndarray, x: np.ndarray, sigma: float):
    """loss = sum_m sigma^2 (1 - exp(-e_m^2/(2 sigma^2))), e_m = x_m - Tr(prod Z_k(i_mk)).
    d loss / d Z_k(i)[a, b] = sum_{m: i_mk = i} -w_m e_m S_m^{!=k}[b, a] with w the HQ weight.
    Returns (loss, e, w, grads) with grads[k] shaped like core k."""
    N = len(cores)
    M = idx.shape[0]
    xhat = np.empty(M)
    for m in range(M):
        xhat[m] = entry(cores, idx[m])
    e = x - xhat
    w = hq_weight(e, sigma)
    loss = welsch_loss(e, sigma)
    grads = [np.zeros_like(Z) for Z in cores]
    for m in range(M):
        for k in range(N):
            S = np.eye(cores[(k + 1) % N].shape[0])
            for j in [(k + 1 + q) % N for q in range(N - 1)]:
                S = S @ cores[j][:, idx[m, j], :]
            grads[k][:, idx[m, k], :] += -w[m] * e[m] * S.T
    return loss, e, w, grads


def sampled_loss_grad_vec(cores, idx: np.ndarray, x: np.ndarray, sigma: float):
    """Same quantities as sampled_loss_grad, with the per-entry products batched over the
    entries (numpy matmul on stacks of slices) for large samples."""
    N = len(cores)
    idx = np.asarray(idx)
    slices = [np.transpose(cores[k][:, idx[:, k], :], (1, 0, 2)) for k in range(N)]  # (M, r_k, r_k+1)
    # prefix P_k = Z_1 ... Z_{k-1} and suffix Q_k = Z_{k+1} ... Z_N, per entry
    M = idx.shape[0]
    pre = [None] * N
    P = np.broadcast_to(np.eye(cores[0].shape[0]), (M,) + (cores[0].shape[0],) * 2)
    for k in range(N):
        pre[k] = P
        P = np.matmul(P, slices[k])
    xhat = np.trace(P, axis1=1, axis2=2)
    e = x - xhat
    w = hq_weight(e, sigma)
    loss = welsch_loss(e, sigma)
    g = -w * e
    grads = [np.zeros_like(Z) for Z in cores]
    suf = np.broadcast_to(np.eye(cores[0].shape[0]), (M,) + (cores[0].shape[0],) * 2)
    for k in range(N - 1, -1, -1):
        # S^{!=k} = (Z_{k+1} ... Z_N)(Z_1 ... Z_{k-1}) = suf @ pre[k]
        S = np.matmul(suf, pre[k])                          # (M, r_{k+1}, r_k)
        contrib = g[:, None, None] * np.transpose(S, (0, 2, 1))
        np.add.at(grads[k], (slice(None), idx[:, k], slice(None)),
                  np.transpose(contrib, (1, 0, 2)))
        suf = np.matmul(slices[k], suf)
    return loss, e, w, grads
