"""Plain FP64 CPU oracle for approximate mini-batch kernel k-means.

Ferrarotti, Decherchi & Rocchia, "Distributed kernel k-means for large scale
clustering" (arXiv 1710.03013).

TEST INFRASTRUCTURE ONLY.  This module is the independent checker of the CUDA
library.  It is imported only by ``tests/``, by ``__graft_entry__.smoke()`` and
by the CPU-baseline legs of ``bench.py``.  The library never imports it, and it
shares no code with the library: both sides implement the SplitMix64 generator
from its published definition, and nothing else is common.

Everything is float64 and written for a reader who checks it against the
paper by eye: kernels are evaluated from direct differences (no norm
expansion), sums are plain numpy reductions, and every step follows the order
of Algorithm 1.  Each function names the equation or section it restates.

Readings of the paper (where it is silent, garbled or at odds with itself):
  R1  RBF kernel: K(x, y) = exp(-||x - y||^2 / (2 sigma^2)).
  R2  MD kernel: K = exp(-rmsd^2 / (2 sigma^2)), rmsd after optimal proper
      superposition of the mean-centred frames, equal atom weights.
  R3  The normalisers |w_j| of Eq. 14, 16, 17 are the landmark counts
      n_j = |S_j| (so w_j is the mean of its landmark support).
  R4  Landmarks L are drawn once per mini-batch; S_j is re-derived from the
      labels at every inner iteration.
  R5  |L| = clamp(ceil(s * N_i - 1e-9), 1, N_i) (Eq. 18).
  R6  Eq. 8 gets the constant term +K(m_j, m_j), i.e. the full Eq. 2 distance.
  R7  Ties: lowest cluster index for labels, lowest local sample index for
      medoids and k-means++ picks.
  R8  d_ij = +inf when n_j = 0 inside the inner loop.
  R9  Eq. 12 is skipped for an empty cluster (alpha = 0 keeps m_j).
  R10 |w_j| in alpha is the cumulative member count of earlier mini-batches;
      |w_j^i| counts every member of X^i, not only landmarks.
  R11 ``iters`` caps the inner loop; with early stop the loop also ends at the
      first iteration that changes no label (Algorithm 1, while condition).
  R13 Omega_t of an inner iteration is sum_i min_j d_ij for the labels of that
      iteration, i.e. the cost right after the assignment (Eq. 9).
  R18 Restarts (Section 4.5: of several k-means++ initialisations the one of
      least cost is kept): the cost is Eq. 1 over the whole data set against
      the final global medoids;
      restart r uses the r-th output of SplitMix64(seed); ties go to the
      lowest restart; all restarts share one bandwidth.
  R19 The elbow criterion (Sections 4.4, 4.5) is not defined in the paper:
      the C whose cost lies farthest below the chord joining the end points of
      the cost curve, both axes scaled to [0, 1] (lowest C on ties).
  R20 The centre displacement of Fig. 4(b): per outer iteration, the mean over
      clusters of the feature-space distance between the global medoid before
      and after the mini-batch.
"""

import math

import numpy as np

_MASK64 = (1 << 64) - 1

KIND_RBF = "rbf"
KIND_RMSD = "rmsd"
KIND_LINEAR = "linear"


# ---------------------------------------------------------------------------
# Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
# pseudorandom number generators", OOPSLA 2014), from its published
# definition.  u01 takes the top 53 bits.
# ---------------------------------------------------------------------------
class SplitMix64:
    def __init__(self, seed):
        self.state = int(seed) & _MASK64

    def next_u64(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def u01(self):
        return (self.next_u64() >> 11) * (2.0 ** -53)


def rng_streams(seed, B):
    """Sub-streams of one fit: master = SplitMix64(seed); its draws, in order,
    seed the k-means++ stream, the bandwidth stream and one landmark stream per
    mini-batch."""
    master = SplitMix64(seed)
    kpp = SplitMix64(master.next_u64())
    bw = SplitMix64(master.next_u64())
    lm = [SplitMix64(master.next_u64()) for _ in range(B)]
    return kpp, bw, lm


# ---------------------------------------------------------------------------
# Kernels (Section 2: a Mercer kernel replaces the feature-space product).
# ---------------------------------------------------------------------------
def sq_dists(X, Y, chunk_elems=1 << 23):
    """||x - y||^2 for every pair, from explicit differences (float64)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    out = np.empty((X.shape[0], Y.shape[0]), dtype=np.float64)
    rows = max(1, chunk_elems // max(1, Y.shape[0] * X.shape[1]))
    for a in range(0, X.shape[0], rows):
        diff = X[a:a + rows, None, :] - Y[None, :, :]
        out[a:a + rows] = np.einsum("ijk,ijk->ij", diff, diff)
    return out


def centre_frames(F):
    """Frames [n][n_atoms][3] moved to their arithmetic mean (equal weights)."""
    F = np.asarray(F, dtype=np.float64)
    return F - F.mean(axis=1, keepdims=True)


def horn_matrix(S):
    """Horn's symmetric 4x4 quaternion matrix of a 3x3 correlation matrix
    S[a][b] = sum_k x_k[a] y_k[b] (Horn 1987, closed-form absolute
    orientation).  Its largest eigenvalue is max_R sum_k y_k . (R x_k) over
    proper rotations R."""
    Sxx, Sxy, Sxz = S[..., 0, 0], S[..., 0, 1], S[..., 0, 2]
    Syx, Syy, Syz = S[..., 1, 0], S[..., 1, 1], S[..., 1, 2]
    Szx, Szy, Szz = S[..., 2, 0], S[..., 2, 1], S[..., 2, 2]
    N = np.empty(S.shape[:-2] + (4, 4), dtype=np.float64)
    N[..., 0, 0] = Sxx + Syy + Szz
    N[..., 0, 1] = Syz - Szy
    N[..., 0, 2] = Szx - Sxz
    N[..., 0, 3] = Sxy - Syx
    N[..., 1, 1] = Sxx - Syy - Szz
    N[..., 1, 2] = Sxy + Syx
    N[..., 1, 3] = Szx + Sxz
    N[..., 2, 2] = -Sxx + Syy - Szz
    N[..., 2, 3] = Syz + Szy
    N[..., 3, 3] = -Sxx - Syy + Szz
    for a in range(4):
        for b in range(a):
            N[..., a, b] = N[..., b, a]
    return N


def rmsd2(A, Bf, chunk_pairs=1 << 15):
    """Squared minimum RMSD after optimal proper superposition, for every pair
    of frames A[i] (shape [n_atoms][3]) and Bf[j].  Reading R2: both frames are
    centred on their mean; rmsd^2 = max(0, (G_a + G_b - 2 lambda_max) / n)
    with lambda_max the top eigenvalue of Horn's matrix (LAPACK eigvalsh)."""
    A = centre_frames(A)
    Bc = centre_frames(Bf)
    n = A.shape[1]
    Ga = np.einsum("ikc,ikc->i", A, A)
    Gb = np.einsum("jkc,jkc->j", Bc, Bc)
    out = np.empty((A.shape[0], Bc.shape[0]), dtype=np.float64)
    rows = max(1, chunk_pairs // max(1, Bc.shape[0]))
    for a in range(0, A.shape[0], rows):
        S = np.einsum("ika,jkb->ijab", A[a:a + rows], Bc)
        lam = np.linalg.eigvalsh(horn_matrix(S))[..., -1]
        r2 = (Ga[a:a + rows, None] + Gb[None, :] - 2.0 * lam) / n
        out[a:a + rows] = np.maximum(r2, 0.0)
    return out


class Kernel:
    """Kernel choice.  ``n_atoms`` is used by the MD kernel only; its samples
    are rows of length 3*n_atoms holding [n_atoms][3] coordinates."""

    def __init__(self, kind, sigma=1.0, n_atoms=0):
        self.kind = kind
        self.sigma = float(sigma)
        self.n_atoms = int(n_atoms)

    def frames(self, X):
        X = np.asarray(X, dtype=np.float64)
        return X.reshape(X.shape[0], self.n_atoms, 3)

    def distance(self, X, Y):
        """The distance the bandwidth heuristic takes the median of."""
        if self.kind == KIND_RMSD:
            return np.sqrt(rmsd2(self.frames(X), self.frames(Y)))
        return np.sqrt(sq_dists(X, Y))

    def __call__(self, X, Y):
        """K(X, Y) as an [len(X)][len(Y)] float64 matrix."""
        if self.kind == KIND_RBF:
            return np.exp(-sq_dists(X, Y) / (2.0 * self.sigma ** 2))
        if self.kind == KIND_RMSD:
            r2 = rmsd2(self.frames(X), self.frames(Y))
            return np.exp(-r2 / (2.0 * self.sigma ** 2))
        if self.kind == KIND_LINEAR:
            return np.asarray(X, np.float64) @ np.asarray(Y, np.float64).T
        raise ValueError(self.kind)

    def self_terms(self, X):
        """K(x, x): exactly 1 for both Gaussian kernels, ||x||^2 for linear."""
        X = np.asarray(X, dtype=np.float64)
        if self.kind == KIND_LINEAR:
            return np.einsum("ij,ij->i", X, X)
        return np.ones(X.shape[0], dtype=np.float64)


def median_bandwidth(X, kernel, bw_rng, max_samples=2048):
    """Bandwidth heuristic: the lower median of all pairwise distances among
    M = min(N, 2048) samples picked by a partial Fisher-Yates shuffle of the
    bandwidth stream.  (The paper's sigma = 4 d_max is replaced by the median
    rule of the workloads it is measured on.)"""
    N = X.shape[0]
    M = min(N, max_samples)
    pick = partial_fisher_yates(N, M, bw_rng)
    if M < 2:
        return 1.0
    D = kernel.distance(X[pick], X[pick])
    iu = np.triu_indices(M, k=1)
    vals = np.sort(D[iu])
    return float(vals[(vals.size - 1) // 2])


# ---------------------------------------------------------------------------
# Mini-batches and landmarks (Section 3.1 "Mini-batch fetching"; Eq. 18).
# ---------------------------------------------------------------------------
def minibatch_indices(N, B, sampling="stride"):
    """Global indices of the B disjoint mini-batches, each in increasing order.
    stride: X^i = {x_{i + jB}};  block: contiguous, the first N mod B batches
    one longer."""
    if sampling == "stride":
        return [np.arange(i, N, B, dtype=np.int64) for i in range(B)]
    if sampling == "block":
        base, extra = divmod(N, B)
        out, start = [], 0
        for i in range(B):
            size = base + (1 if i < extra else 0)
            out.append(np.arange(start, start + size, dtype=np.int64))
            start += size
        return out
    raise ValueError(sampling)


def partial_fisher_yates(n, k, rng):
    """First k entries of a Fisher-Yates shuffle of [0, n) (unsorted)."""
    idx = np.arange(n, dtype=np.int64)
    for a in range(k):
        r = a + int(math.floor(rng.u01() * (n - a)))
        idx[a], idx[r] = idx[r], idx[a]
    return idx[:k].copy()


def n_landmarks(Ni, s):
    """Eq. 18 solved for |L| (reading R5)."""
    return int(min(max(math.ceil(s * Ni - 1e-9), 1), Ni))


def landmark_indices(Ni, s, rng):
    """Landmarks L: uniform without replacement from the mini-batch (Eq. 14),
    returned sorted.  s = 1 takes the whole mini-batch and draws nothing."""
    nl = n_landmarks(Ni, s)
    if nl == Ni:
        return np.arange(Ni, dtype=np.int64)
    return np.sort(partial_fisher_yates(Ni, nl, rng))


# ---------------------------------------------------------------------------
# Initialisation (Section 3.1, "Kernel evaluation and mini-batch
# initialization").
# ---------------------------------------------------------------------------
def kmeanspp(X0, C, kernel, rng):
    """Kernel k-means++ seeding (Arthur & Vassilvitskii 2007, kernelised):
    the first medoid is uniform; each next one is drawn with probability
    proportional to D^2(x) = min over chosen m of
    K(x,x) - 2K(x,m) + K(m,m).  The draw takes target = u01 * sum(D^2) and
    the first index whose running sum exceeds it; if every D^2 is zero, the
    lowest unchosen index.  Returns local indices."""
    N0 = X0.shape[0]
    kself = kernel.self_terms(X0)
    chosen = [int(math.floor(rng.u01() * N0))]
    D2 = np.full(N0, np.inf)
    for _ in range(1, C):
        m = chosen[-1]
        km = kernel(X0, X0[m:m + 1])[:, 0]
        D2 = np.minimum(D2, kself - 2.0 * km + kself[m])
        D2 = np.maximum(D2, 0.0)
        u = rng.u01()
        prefix = np.cumsum(D2)          # running sum in index order
        total = float(prefix[-1])
        if total > 0.0:
            target = u * total          # u < 1, so target < total
            pick = int(np.searchsorted(prefix, target, side="right"))
        else:
            taken = set(chosen)
            pick = next(idx for idx in range(N0) if idx not in taken)
        chosen.append(pick)
    return np.asarray(chosen, dtype=np.int64)


def nearest_medoid_labels(kself, Kt, kmm):
    """Eq. 8 with the constant K(m_j, m_j) (reading R6): label = argmin_j
    K(x,x) - 2K(x, m_j) + K(m_j, m_j), lowest j on ties."""
    d = kself[:, None] - 2.0 * Kt + kmm[None, :]
    return np.argmin(d, axis=1).astype(np.int64), d


# ---------------------------------------------------------------------------
# Inner iteration (Eq. 15-17 with Eq. 4-6; Eq. 9 cost).
# ---------------------------------------------------------------------------
def support_stats(Kb, L, u, C):
    """n_j = |S_j| (landmarks labelled j), compactness g_hat (Eq. 16) and
    similarity f_hat (Eq. 17) of every row of the block Kb = K(X^i, X^i[L]).
    Rows at landmark positions give the L x L block, so g_hat needs no extra
    kernel values.  Reading R3: both are normalised by n_j."""
    uL = u[L]
    n = np.bincount(uL, minlength=C)[:C].astype(np.int64)
    fhat = np.full((Kb.shape[0], C), np.nan)
    ghat = np.full(C, np.nan)
    for j in range(C):
        if n[j] == 0:
            continue
        Sj = np.nonzero(uL == j)[0]
        fhat[:, j] = Kb[:, Sj].sum(axis=1) / n[j]
        ghat[j] = Kb[np.ix_(L[Sj], Sj)].sum() / float(n[j]) ** 2
    return n, ghat, fhat


def inner_step(Kb, kself, L, u, C):
    """One inner GD iteration on mini-batch i (Eq. 15): the distances
    d_ij = K_ii - 2 f_hat_ij + g_hat_j (+inf for n_j = 0, reading R8), the new
    labels (lowest j on ties), the cost Omega (reading R13), the margin
    d_(2) - d_(1) of every row and the number of changed labels."""
    n, ghat, fhat = support_stats(Kb, L, u, C)
    d = kself[:, None] - 2.0 * fhat + ghat[None, :]
    d[:, n == 0] = np.inf
    u_new = np.argmin(d, axis=1).astype(np.int64)
    rows = np.arange(d.shape[0])
    dmin = d[rows, u_new]
    if C > 1:
        part = np.partition(d, 1, axis=1)
        margin = part[:, 1] - part[:, 0]
    else:
        margin = np.full(d.shape[0], np.inf)
    return {
        "u": u_new,
        "omega": float(np.sum(dmin)),
        "changed": int(np.count_nonzero(u_new != u)),
        "margin": margin,
        "d": d,
        "n": n,
        "ghat": ghat,
        "fhat": fhat,
    }


# ---------------------------------------------------------------------------
# Mini-batch medoids and merge (Eq. 10-13, empty-cluster rule).
# ---------------------------------------------------------------------------
def minibatch_medoids(kself, fhat, n, c):
    """Eq. 10 (via Eq. 7): m_j^i = argmin_l K_ll - 2 f_hat_lj over the whole
    mini-batch, lowest l on ties.  -1 marks an empty cluster (c_j = 0 or
    n_j = 0)."""
    C = fhat.shape[1]
    mi = np.full(C, -1, dtype=np.int64)
    for j in range(C):
        if c[j] == 0 or n[j] == 0:
            continue
        mi[j] = int(np.argmin(kself - 2.0 * fhat[:, j]))
    return mi


def merge_medoids(kself, Kt, Kmi, mi, c, W):
    """Eq. 12 with alpha = |w_j^i| / (|w_j^i| + |w_j|) (Eq. 13): the new global
    medoid is argmin_l K_ll - 2(1-alpha) K(x_l, m_j) - 2 alpha K(x_l, m_j^i)
    over the mini-batch (lowest l on ties).  Empty clusters keep m_j
    (reading R9).  Returns local indices (-1 = keep) and the new counts."""
    C = len(mi)
    new_local = np.full(C, -1, dtype=np.int64)
    W = W.copy()
    for j in range(C):
        if mi[j] < 0:
            continue
        alpha = c[j] / float(c[j] + W[j])
        val = kself - 2.0 * (1.0 - alpha) * Kt[:, j] - 2.0 * alpha * Kmi[:, j]
        new_local[j] = int(np.argmin(val))
        W[j] += c[j]
    return new_local, W


# ---------------------------------------------------------------------------
# Algorithm 1 on one process (no distribution: the P-node split of
# Section 3.3 does not change the arithmetic).
# ---------------------------------------------------------------------------
def fit(X, C, B, s, kernel, iters, seed, early_stop=True, init_medoids=None,
        sampling="stride"):
    """Approximate mini-batch kernel k-means (Algorithm 1, Eq. 8-18).

    Returns a dict with the per-sample labels (each sample's final label in its
    own mini-batch), the global medoids (global indices and coordinates), the
    cumulative counts W, the final supports of the last mini-batch (landmark
    coordinates, their labels, n_j and g_hat), the Omega trace and the
    per-mini-batch details used by the tests.
    """
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    kpp_rng, bw_rng, lm_rngs = rng_streams(seed, B)
    if kernel.sigma <= 0.0 and kernel.kind != KIND_LINEAR:
        kernel = Kernel(kernel.kind, median_bandwidth(X, kernel, bw_rng),
                        kernel.n_atoms)
    batches = minibatch_indices(N, B, sampling)
    labels = np.full(N, -1, dtype=np.int64)
    W = np.zeros(C, dtype=np.int64)
    M_idx = None
    trace = []
    details = []
    for i, gidx in enumerate(batches):
        Xi = X[gidx]
        Ni = Xi.shape[0]
        L = landmark_indices(Ni, s, lm_rngs[i])
        Kb = kernel(Xi, Xi[L])                          # Alg. 1 line 3
        kself = kernel.self_terms(Xi)
        if i == 0:                                      # Alg. 1 lines 4-6
            if init_medoids is not None:
                M_idx = np.asarray(init_medoids, dtype=np.int64).copy()
            else:
                M_idx = gidx[kmeanspp(Xi, C, kernel, kpp_rng)]
        MX = X[M_idx]
        Kt = kernel(Xi, MX)                             # aux block, N_i x C
        u, _ = nearest_medoid_labels(kself, Kt, kernel.self_terms(MX))
        u_init = u.copy()
        steps = []
        for t in range(iters):                          # Alg. 1 lines 9-16
            st = inner_step(Kb, kself, L, u, C)
            trace.append((i, t, st["omega"], st["changed"]))
            steps.append(st)
            u = st["u"]
            if early_stop and st["changed"] == 0:
                break
        n, ghat, fhat = support_stats(Kb, L, u, C)
        c = np.bincount(u, minlength=C)[:C].astype(np.int64)
        mi = minibatch_medoids(kself, fhat, n, c)       # Eq. 10
        Kmi = np.zeros((Ni, C))
        ok = mi >= 0
        if ok.any():
            Kmi[:, ok] = kernel(Xi, Xi[mi[ok]])
        new_local, W_new = merge_medoids(kself, Kt, Kmi, mi, c, W)
        M_old = M_idx.copy()
        for j in range(C):
            if new_local[j] >= 0:
                M_idx[j] = gidx[new_local[j]]
        W = W_new
        labels[gidx] = u
        details.append({
            "gidx": gidx, "L": L, "u_init": u_init, "u": u.copy(),
            "n": n, "ghat": ghat, "c": c, "mi": mi, "M_before": M_old,
            "M_after": M_idx.copy(), "steps": steps, "kernel_sigma": kernel.sigma,
        })
    last = details[-1]
    XL = X[last["gidx"][last["L"]]]
    return {
        "labels": labels,
        "medoids": M_idx.copy(),
        "medoid_coords": X[M_idx].copy(),
        "W": W,
        "support_coords": XL,
        "support_labels": last["u"][last["L"]].copy(),
        "n": last["n"],
        "ghat": last["ghat"],
        "trace": trace,
        "details": details,
        "kernel": kernel,
        "C": C,
    }


# ---------------------------------------------------------------------------
# Using a fitted model (Eq. 2 / Eq. 15 for new samples, Eq. 1 cost).
# ---------------------------------------------------------------------------
def assign_distances(model, Xnew, mode="supports"):
    """Distances of new samples to the C prototypes.  ``supports``: the sparse
    centroids of Eq. 14 kept from the last mini-batch, d_j = K(x,x) -
    2 f_hat_j(x) + g_hat_j (+inf for n_j = 0).  ``medoids``: Eq. 2 against the
    global medoids, d_j = K(x,x) - 2K(x, m_j) + K(m_j, m_j)."""
    kernel = model["kernel"]
    C = model["C"]
    Xnew = np.asarray(Xnew, dtype=np.float64)
    kself = kernel.self_terms(Xnew)
    if mode == "medoids":
        MX = model["medoid_coords"]
        return kself[:, None] - 2.0 * kernel(Xnew, MX) + kernel.self_terms(MX)[None, :]
    Ks = kernel(Xnew, model["support_coords"])
    uL = model["support_labels"]
    d = np.full((Xnew.shape[0], C), np.inf)
    for j in range(C):
        nj = int(np.count_nonzero(uL == j))
        if nj == 0:
            continue
        f = Ks[:, uL == j].sum(axis=1) / nj
        d[:, j] = kself - 2.0 * f + model["ghat"][j]
    return d


def assign(model, Xnew, mode="supports"):
    """Labels (argmin, lowest j on ties) and distances of new samples."""
    d = assign_distances(model, Xnew, mode)
    u = np.argmin(d, axis=1).astype(np.int64)
    return u, d[np.arange(d.shape[0]), u]


def cost(model, X, mode="supports"):
    """Eq. 1 against the model's prototypes: sum_i min_j d_ij."""
    _, dmin = assign(model, X, mode)
    return float(np.sum(dmin))


# ---------------------------------------------------------------------------
# Model selection and diagnostics around Algorithm 1 (Section 4.1, Fig. 4b;
# Sections 4.4 and 4.5).
# ---------------------------------------------------------------------------
def medoid_displacement(kernel, X, M_before, M_after):
    """Average displacement of the cluster centres across one outer
    iteration (the control observable of Section 4.1, Fig. 4b): the mean over
    the C clusters of the feature-space distance between the global medoid
    before and after the mini-batch, sqrt(K(a,a) - 2K(a,b) + K(b,b))."""
    X = np.asarray(X, dtype=np.float64)
    A = X[np.asarray(M_before)]
    Bm = X[np.asarray(M_after)]
    kab = np.array([kernel(A[j:j + 1], Bm[j:j + 1])[0, 0] for j in range(len(A))])
    d2 = kernel.self_terms(A) - 2.0 * kab + kernel.self_terms(Bm)
    same = np.asarray(M_before) == np.asarray(M_after)
    d2[same] = 0.0
    return float(np.mean(np.sqrt(np.maximum(d2, 0.0))))


def displacement_trace(result, X):
    """medoid_displacement of every mini-batch of a fit() result."""
    return [medoid_displacement(result["kernel"], X, det["M_before"], det["M_after"])
            for det in result["details"]]


def restart_seeds(seed, n):
    """Seeds of n restarts: the first n outputs of SplitMix64(seed)."""
    g = SplitMix64(seed)
    return [g.next_u64() for _ in range(n)]


def fit_restarts(X, C, B, s, kernel, iters, seeds, early_stop=True, sampling="stride"):
    """Section 4.5: the method initialised several times with k-means++ (one
    seed each) and the solution of minimum cost kept.  Reading: the cost is
    Eq. 1 over the whole data set against the final global medoids (the
    output M of Algorithm 1); ties go to the lowest restart.  Every restart
    uses the same bandwidth (the caller resolves the median rule first)."""
    fits = [fit(X, C, B, s, kernel, iters, sd, early_stop=early_stop, sampling=sampling) for sd in seeds]
    costs = np.array([cost(f, X, "medoids") for f in fits])
    best = int(np.argmin(costs))
    return {"costs": costs, "best": best, "fit": fits[best], "fits": fits}


def elbow_index(costs):
    """The elbow of a cost curve over consecutive C (Sections 4.4 and 4.5
    pick C "via the elbow criterion"; reading: the point farthest below the
    chord joining the curve's end points, both axes scaled to [0, 1]; lowest
    C on ties).  Returns the index into `costs`."""
    y = np.asarray(costs, dtype=np.float64)
    n = y.size
    if n <= 2:
        return 0
    x = np.arange(n) / (n - 1.0)
    span = y.max() - y.min()
    if span <= 0.0:
        return 0
    yn = (y - y.min()) / span
    chord = yn[0] + (yn[-1] - yn[0]) * x
    return int(np.argmax(chord - yn))


def elbow(X, C_lo, C_hi, B, s, kernel, iters, seed, n_restarts=1, early_stop=True, sampling="stride"):
    """Cost of the best of n_restarts fits for every C in [C_lo, C_hi] (the
    same restart seeds for every C) and the elbow C."""
    seeds = restart_seeds(seed, n_restarts)
    Cs = list(range(C_lo, C_hi + 1))
    costs = np.array([fit_restarts(X, C, B, s, kernel, iters, seeds, early_stop, sampling)["costs"].min()
                      for C in Cs])
    return {"Cs": np.array(Cs), "costs": costs, "C": Cs[elbow_index(costs)]}
