"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these checks re-types the oracle's own formula: each compares it with
a different formulation (matrix algebra, explicit feature-space means, brute
force, SVD superposition, closed forms, a library median, published generator
outputs).  CPU only.
"""

import itertools
import math

import numpy as np
import pytest

from oracle import kkm_oracle as O
from synth import blobs, random_rigid_motion

# ---------------------------------------------------------------------------
# SplitMix64: outputs of the published reference generator.
# ---------------------------------------------------------------------------


def test_splitmix64_reference_outputs():
    r = O.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    r = O.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_u01_range_and_resolution():
    r = O.SplitMix64(99)
    v = np.array([r.u01() for _ in range(2000)])
    assert v.min() >= 0.0 and v.max() < 1.0
    assert np.all(v * 2.0 ** 53 == np.floor(v * 2.0 ** 53))


# ---------------------------------------------------------------------------
# Textbook kernel k-means in matrix form (Zhang & Rudnicky's g/f form written
# with one-hot matrices): an independent formulation for P1 and P5.
# ---------------------------------------------------------------------------


def textbook_step(K, u, C):
    N = K.shape[0]
    Z = np.zeros((N, C))
    Z[np.arange(N), u] = 1.0
    cnt = Z.sum(axis=0)
    live = cnt > 0
    F = np.full((N, C), np.inf)
    g = np.zeros(C)
    F[:, live] = (K @ Z[:, live]) / cnt[live]
    g[live] = np.einsum("ij,ik,kj->j", Z[:, live], K, Z[:, live]) / cnt[live] ** 2
    D = np.diag(K)[:, None] - 2.0 * F + g[None, :]
    D[:, ~live] = np.inf
    un = np.argmin(D, axis=1)
    return un, float(D[np.arange(N), un].sum())


def _blob_data(N=240, d=5, C=4, problem=0):
    X, y = blobs(N, d, C, workload=90, problem=problem)
    return X.astype(np.float64), y


def test_P1_full_batch_equals_textbook_kernel_kmeans():
    X, _ = _blob_data()
    ker = O.Kernel(O.KIND_RBF, sigma=3.0)
    res = O.fit(X, 4, 1, 1.0, ker, iters=25, seed=11, early_stop=False)
    det = res["details"][0]
    K = ker(X, X)
    u = det["u_init"].copy()
    for st in det["steps"]:
        un, om = textbook_step(K, u, 4)
        assert np.array_equal(un, st["u"])
        assert abs(om - st["omega"]) <= 1e-12 * abs(om)
        u = un
    assert np.array_equal(res["labels"], u)


def test_P2_linear_kernel_is_lloyd():
    X, _ = _blob_data(N=300, d=3, C=5, problem=1)
    ker = O.Kernel(O.KIND_LINEAR)
    res = O.fit(X, 5, 1, 1.0, ker, iters=20, seed=5, early_stop=False)
    det = res["details"][0]
    u = det["u_init"].copy()
    for st in det["steps"]:
        mus = np.stack([X[u == j].mean(axis=0) if np.any(u == j)
                        else np.full(X.shape[1], np.nan) for j in range(5)])
        dist = ((X[:, None, :] - mus[None, :, :]) ** 2).sum(axis=2)
        dist[np.isnan(dist)] = np.inf
        un = np.argmin(dist, axis=1)
        om = dist[np.arange(len(X)), un].sum()
        assert np.array_equal(un, st["u"])
        assert abs(om - st["omega"]) <= 1e-10 * abs(om)
        u = un


def _feature_space_cost(K, u, C):
    total = 0.0
    for j in range(C):
        S = np.nonzero(u == j)[0]
        if S.size == 0:
            continue
        # sum_i ||phi(x_i) - mean||^2 = sum_i K_ii - (1/|S|) sum_{m,n} K_mn
        total += np.trace(K[np.ix_(S, S)]) - K[np.ix_(S, S)].sum() / S.size
    return total


@pytest.mark.parametrize("C", [2, 3])
def test_P3_brute_force_minimum_is_fixed_point(C):
    g = np.random.Generator(np.random.PCG64(3 + C))
    centres = np.array([[0.0, 0.0], [6.0, 0.0], [0.0, 6.0]])[:C]
    y = np.arange(9) % C
    X = centres[y] + g.normal(0, 0.4, size=(9, 2))
    ker = O.Kernel(O.KIND_RBF, sigma=2.5)
    K = ker(X, X)
    best, best_u = np.inf, None
    for lab in itertools.product(range(C), repeat=9):
        u = np.array(lab)
        if len(set(lab)) < C:
            continue
        c = _feature_space_cost(K, u, C)
        if c < best - 1e-12:
            best, best_u = c, u
    st = O.inner_step(K, np.ones(9), np.arange(9), best_u, C)
    assert np.array_equal(st["u"], best_u)
    assert st["changed"] == 0
    assert abs(st["omega"] - best) <= 1e-12 * best
    reached = min(O.fit(X, C, 1, 1.0, ker, 20, seed)["trace"][-1][2]
                  for seed in range(20))
    assert abs(reached - best) <= 1e-12 * best


@pytest.mark.parametrize("kind", [O.KIND_RBF, O.KIND_LINEAR])
def test_P4_omega_monotone_full_landmarks(kind):
    X, _ = _blob_data(N=400, d=6, C=6, problem=2)
    ker = O.Kernel(kind, sigma=2.0)
    res = O.fit(X, 6, 2, 1.0, ker, iters=30, seed=3, early_stop=False)
    for det in res["details"]:
        om = [st["omega"] for st in det["steps"]]
        for a, b in zip(om, om[1:]):
            assert b <= a + 1e-12 * abs(a)


def test_P4_landmark_cost_monotone_sparse():
    X, _ = _blob_data(N=600, d=4, C=5, problem=3)
    ker = O.Kernel(O.KIND_RBF, sigma=2.0)
    res = O.fit(X, 5, 2, 0.3, ker, iters=30, seed=8, early_stop=False)
    for det in res["details"]:
        L = det["L"]
        costs = [float(np.min(st["d"][L], axis=1).sum()) for st in det["steps"]]
        for a, b in zip(costs, costs[1:]):
            assert b <= a + 1e-12 * abs(a)


def test_P5_landmark_trajectory_is_kernel_kmeans_on_L():
    X, _ = _blob_data(N=500, d=4, C=4, problem=4)
    ker = O.Kernel(O.KIND_RBF, sigma=2.0)
    res = O.fit(X, 4, 1, 0.25, ker, iters=15, seed=21, early_stop=False)
    det = res["details"][0]
    L = det["L"]
    KLL = ker(X[L], X[L])
    uL = det["u_init"][L].copy()
    KfullL = ker(X, X[L])
    for st in det["steps"]:
        un, _ = textbook_step(KLL, uL, 4)
        assert np.array_equal(st["u"][L], un)
        # non-landmarks: nearest landmark-mean in feature space
        Z = np.zeros((len(L), 4))
        Z[np.arange(len(L)), uL] = 1
        cnt = Z.sum(0)
        live = cnt > 0
        F = np.full((len(X), 4), np.inf)
        F[:, live] = KfullL @ Z[:, live] / cnt[live]
        g = np.zeros(4)
        g[live] = np.einsum("ij,ik,kj->j", Z[:, live], KLL, Z[:, live]) / cnt[live] ** 2
        D = 1.0 - 2 * F + g
        assert np.array_equal(np.argmin(D, axis=1), st["u"])
        uL = un


# ---------------------------------------------------------------------------
# P6: the MD kernel.
# ---------------------------------------------------------------------------


def _kabsch_rmsd2(A, B):
    A = A - A.mean(axis=0)
    B = B - B.mean(axis=0)
    H = A.T @ B
    U, S, Vt = np.linalg.svd(H)
    d = np.sign(np.linalg.det(U @ Vt))
    best = S[0] + S[1] + d * S[2]
    return max(0.0, ((A * A).sum() + (B * B).sum() - 2 * best) / A.shape[0])


def _frames(n=6, atoms=40, problem=0):
    g = np.random.Generator(np.random.PCG64(77 + problem))
    base = np.cumsum(g.normal(size=(atoms, 3)), axis=0)
    F = base[None] + g.normal(0, 0.8, size=(n, atoms, 3))
    return F, g


def test_P6_rmsd_matches_svd_kabsch():
    F, _ = _frames(8, 50)
    r2 = O.rmsd2(F, F)
    for a in range(8):
        for b in range(8):
            assert abs(r2[a, b] - _kabsch_rmsd2(F[a], F[b])) <= 1e-10 * max(1.0, r2[a, b])


def test_P6_rmsd_self_zero_symmetric_triangle():
    F, _ = _frames(7, 30, problem=1)
    r = np.sqrt(O.rmsd2(F, F))
    assert np.all(np.abs(np.diag(r)) <= 1e-6)
    assert np.allclose(r, r.T, atol=1e-10)
    for a, b, c in itertools.product(range(7), repeat=3):
        assert r[a, c] <= r[a, b] + r[b, c] + 1e-9


def test_P6_rmsd_rigid_motion_invariance():
    F, g = _frames(5, 60, problem=2)
    R, t = random_rigid_motion(g, 5)
    G = np.einsum("nij,nkj->nki", R, F) + t[:, None, :]
    assert np.allclose(O.rmsd2(F, F), O.rmsd2(G, F), atol=1e-9)
    assert np.allclose(O.rmsd2(F, F), O.rmsd2(F, G), atol=1e-9)


@pytest.mark.parametrize("eps", [-0.5, -0.1, 0.05, 0.3, 2.0])
def test_P6_rmsd_scaling_closed_form(eps):
    F, _ = _frames(1, 45, problem=3)
    x = F[0] - F[0].mean(axis=0)
    y = (1.0 + eps) * x
    want = abs(eps) * math.sqrt((x * x).sum() / x.shape[0])
    got = math.sqrt(O.rmsd2(x[None], y[None])[0, 0])
    assert abs(got - want) <= 1e-9 * max(1.0, want)


def test_P6_rmsd_kernel_values():
    F, _ = _frames(4, 20, problem=4)
    ker = O.Kernel(O.KIND_RMSD, sigma=1.5, n_atoms=20)
    X = F.reshape(4, 60)
    K = ker(X, X)
    want = np.exp(-np.array([[_kabsch_rmsd2(F[a], F[b]) for b in range(4)]
                             for a in range(4)]) / (2 * 1.5 ** 2))
    assert np.allclose(K, want, rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------------------
# P7: medoids and the merge, checked with explicit coordinates (linear kernel).
# ---------------------------------------------------------------------------


def test_P7_first_batch_merge_keeps_batch_medoids_gaussian():
    X, _ = _blob_data(N=300, d=4, C=4, problem=5)
    ker = O.Kernel(O.KIND_RBF, sigma=2.0)
    res = O.fit(X, 4, 3, 0.5, ker, iters=10, seed=2)
    det0 = res["details"][0]
    for j in range(4):
        if det0["mi"][j] >= 0:
            assert det0["M_after"][j] == det0["gidx"][det0["mi"][j]]


def test_P7_B1_medoids_are_eq10_medoids_linear():
    X, _ = _blob_data(N=200, d=3, C=3, problem=6)
    ker = O.Kernel(O.KIND_LINEAR)
    res = O.fit(X, 3, 1, 1.0, ker, iters=15, seed=4)
    u = res["labels"]
    for j in range(3):
        mu = X[u == j].mean(axis=0)
        want = int(np.argmin(((X - mu) ** 2).sum(axis=1)))
        assert res["medoids"][j] == want


def test_P7_merge_convex_combination_linear():
    X, _ = _blob_data(N=400, d=3, C=3, problem=7)
    ker = O.Kernel(O.KIND_LINEAR)
    res = O.fit(X, 3, 2, 1.0, ker, iters=15, seed=6)
    d0, d1 = res["details"]
    Xi = X[d1["gidx"]]
    for j in range(3):
        if d1["mi"][j] < 0:
            assert d1["M_after"][j] == d1["M_before"][j]
            continue
        cj = d1["c"][j]
        Wj = d0["c"][j]
        alpha = cj / (cj + Wj)
        target = (1 - alpha) * X[d1["M_before"][j]] + alpha * Xi[d1["mi"][j]]
        want = d1["gidx"][int(np.argmin(((Xi - target) ** 2).sum(axis=1)))]
        assert d1["M_after"][j] == want
    assert np.array_equal(res["W"], d0["c"] + d1["c"])


def test_P7_empty_cluster_keeps_medoid():
    # Two far groups and C=3 with two initial medoids in the same group: one
    # cluster can lose every landmark; its global medoid must not move.
    X = np.concatenate([np.zeros((20, 2)) + [0, 0], np.zeros((20, 2)) + [50, 0]])
    X += np.random.Generator(np.random.PCG64(1)).normal(0, 0.1, X.shape)
    ker = O.Kernel(O.KIND_RBF, sigma=1.0)
    init = np.array([0, 1, 20])
    res = O.fit(X, 3, 2, 1.0, ker, iters=10, seed=1, init_medoids=init)
    for det in res["details"]:
        for j in range(3):
            if det["mi"][j] < 0:
                assert det["M_after"][j] == det["M_before"][j]
    assert any((det["mi"] < 0).any() for det in res["details"])


# ---------------------------------------------------------------------------
# P8: mini-batches and landmarks.
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("sampling", ["stride", "block"])
@pytest.mark.parametrize("N,B", [(10, 3), (1000, 7), (5, 5), (17, 1)])
def test_P8_partition(sampling, N, B):
    bs = O.minibatch_indices(N, B, sampling)
    allidx = np.concatenate(bs)
    assert np.array_equal(np.sort(allidx), np.arange(N))
    assert all(np.all(np.diff(b) > 0) for b in bs)
    sizes = [len(b) for b in bs]
    assert max(sizes) - min(sizes) <= 1
    if sampling == "stride":
        for i, b in enumerate(bs):
            assert np.all(b % B == i)


# Landmarks are a uniform random subset of the mini-batch (Section 3.2, Eq. 14).
# The draw is the first k steps of a Fisher-Yates shuffle (Durstenfeld's
# form): step a swaps position a with r = a + floor(u * (n - a)), u uniform in
# [0, 1).  The two hand-worked cases below start from published SplitMix64
# outputs (the same values as test_splitmix64_reference_outputs), so neither
# depends on the oracle's generator plumbing.


def _u01_of(x):
    return (x >> 11) * 2.0 ** -53      # top 53 bits, as in the generator pin


def test_P8_fisher_yates_hand_worked_seed0():
    # SplitMix64(0): u = 0.88331..., 0.43152..., 0.02643...
    # a = 0: r = 0 + floor(0.88331 * 10) = 8   -> [8 1 2 3 4 5 6 7 0 9]
    # a = 1: r = 1 + floor(0.43152 *  9) = 4   -> [8 4 2 3 1 5 6 7 0 9]
    # a = 2: r = 2 + floor(0.02643 *  8) = 2   (no move)
    outs = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [a + math.floor(_u01_of(x) * (10 - a)) for a, x in enumerate(outs)] == [8, 4, 2]
    got = O.partial_fisher_yates(10, 3, O.SplitMix64(0))
    assert got.tolist() == [8, 4, 2]


def test_P8_fisher_yates_hand_worked_seed1234567():
    # SplitMix64(1234567): u = 0.35008, 0.17364, 0.53221, 0.24901, 0.88953
    # a = 0: r = 0 + floor(0.35008 * 20) =  7  -> pos0 = 7,  pos7 = 0
    # a = 1: r = 1 + floor(0.17364 * 19) =  4  -> pos1 = 4,  pos4 = 1
    # a = 2: r = 2 + floor(0.53221 * 18) = 11  -> pos2 = 11, pos11 = 2
    # a = 3: r = 3 + floor(0.24901 * 17) =  7  -> pos3 = 0 (moved there at a=0), pos7 = 3
    # a = 4: r = 4 + floor(0.88953 * 16) = 18  -> pos4 = 18, pos18 = 1
    outs = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    assert [a + math.floor(_u01_of(x) * (20 - a)) for a, x in enumerate(outs)] == [7, 4, 11, 7, 18]
    assert O.partial_fisher_yates(20, 5, O.SplitMix64(1234567)).tolist() == [7, 4, 11, 0, 18]
    # landmark_indices returns the same set sorted
    assert O.landmark_indices(20, 0.25, O.SplitMix64(1234567)).tolist() == [0, 4, 7, 11, 18]


def _fy_frequencies_ok(draw, n=12, k=4, T=20000):
    """A uniform k-subset in uniform order: every (position, value) cell has
    probability 1/n, every value is included with probability k/n, and a
    given pair with probability k(k-1)/(n(n-1)).  T seeds; every frequency
    must lie within 4 standard deviations."""
    pos = np.zeros((k, n))
    inc = np.zeros(n)
    pair = 0
    for seed in range(1, T + 1):
        p = np.asarray(draw(n, k, O.SplitMix64(seed)))
        pos[np.arange(k), p] += 1
        inc[p] += 1
        pair += int(0 in p and 1 in p)

    def within(freq, prob):
        return bool(np.all(np.abs(freq / T - prob) <= 4.0 * math.sqrt(prob * (1.0 - prob) / T)))
    return (within(pos, 1.0 / n), within(inc, k / n),
            within(np.array([pair]), k * (k - 1) / (n * (n - 1))))


def test_P8_fisher_yates_uniform_over_seeds():
    assert _fy_frequencies_ok(O.partial_fisher_yates) == (True, True, True)


def _fy_mutant(rule):
    def draw(n, k, rng):
        idx = list(range(n))
        for a in range(k):
            r = rule(a, n, rng.u01())
            idx[a], idx[r] = idx[r], idx[a]
        return idx[:k]
    return draw


@pytest.mark.parametrize("name,rule", [
    ("no swap", lambda a, n, u: a),
    ("r = floor(u n)", lambda a, n, u: int(math.floor(u * n))),
    ("last element unreachable", lambda a, n, u: a + int(math.floor(u * (n - a - 1)))),
])
def test_P8_fisher_yates_pins_reject_plausible_mistakes(name, rule):
    # the same checks fail for draws with a plausible mistake planted in them
    draw = _fy_mutant(rule)
    assert not all(_fy_frequencies_ok(draw)), name
    assert list(draw(10, 3, O.SplitMix64(0))) != [8, 4, 2] or \
        list(draw(20, 5, O.SplitMix64(1234567))) != [7, 4, 11, 0, 18], name


@pytest.mark.parametrize("Ni,s", [(100, 0.2), (3000, 0.05), (7, 0.01), (50, 1.0), (15000, 0.2)])
def test_P8_landmarks(Ni, s):
    L = O.landmark_indices(Ni, s, O.SplitMix64(42))
    assert len(L) == max(1, min(Ni, math.ceil(s * Ni - 1e-9)))
    assert np.all(np.diff(L) > 0) and L.min() >= 0 and L.max() < Ni


# ---------------------------------------------------------------------------
# P9: kernel values and the bandwidth heuristic.
# ---------------------------------------------------------------------------


def test_P9_rbf_values():
    X, _ = _blob_data(N=50, d=7, C=3, problem=8)
    ker = O.Kernel(O.KIND_RBF, sigma=1.7)
    K = ker(X, X)
    assert np.allclose(K, K.T, rtol=0, atol=0)
    assert np.all(K > 0) and np.all(K <= 1)
    assert np.all(np.diag(K) == 1.0)
    from scipy.spatial.distance import cdist
    assert np.allclose(K, np.exp(-cdist(X, X, "sqeuclidean") / (2 * 1.7 ** 2)), rtol=1e-12)


@pytest.mark.parametrize("N", [3, 6, 11])
def test_P9_median_bandwidth_is_lower_median(N):
    from scipy.spatial.distance import pdist
    X, _ = _blob_data(N=N, d=3, C=2, problem=9)
    ker = O.Kernel(O.KIND_RBF, sigma=0.0)
    sig = O.median_bandwidth(X, ker, O.SplitMix64(5))
    dist = np.sort(pdist(X))
    assert sig == pytest.approx(dist[(len(dist) - 1) // 2], rel=1e-12)
    if len(dist) % 2 == 1:
        assert sig == pytest.approx(np.median(dist), rel=1e-12)


# ---------------------------------------------------------------------------
# k-means++ and Eq. 8 on hand-checkable cases.
# ---------------------------------------------------------------------------


def test_kmeanspp_hand_case_linear_1d():
    X = np.array([[0.0], [1.0], [3.0], [10.0]])
    ker = O.Kernel(O.KIND_LINEAR)
    rng = O.SplitMix64(123)
    got = O.kmeanspp(X, 2, ker, rng)
    r = O.SplitMix64(123)
    m0 = int(math.floor(r.u01() * 4))
    d2 = [(X[k, 0] - X[m0, 0]) ** 2 for k in range(4)]
    target = r.u01() * sum(d2)
    run, pick = 0.0, None
    for k in range(4):
        run += d2[k]
        if run > target:
            pick = k
            break
    assert list(got) == [m0, pick]


def test_kmeanspp_separated_groups_pick_one_each():
    g = np.random.Generator(np.random.PCG64(2))
    centres = np.array([[0, 0], [100, 0], [0, 100], [100, 100]], float)
    X = np.repeat(centres, 25, axis=0) + g.normal(0, 0.01, (100, 2))
    ker = O.Kernel(O.KIND_LINEAR)
    for seed in range(10):
        picks = O.kmeanspp(X, 4, ker, O.SplitMix64(seed))
        assert len({int(p) // 25 for p in picks}) == 4


def test_eq8_nearest_medoid_linear_explicit():
    X, _ = _blob_data(N=100, d=3, C=3, problem=10)
    M = X[[0, 1, 2]]
    ker = O.Kernel(O.KIND_LINEAR)
    u, _ = O.nearest_medoid_labels(ker.self_terms(X), ker(X, M), ker.self_terms(M))
    want = np.argmin(((X[:, None] - M[None]) ** 2).sum(axis=2), axis=1)
    assert np.array_equal(u, want)


def test_assign_and_cost_linear_explicit_means():
    X, _ = _blob_data(N=300, d=3, C=3, problem=11)
    ker = O.Kernel(O.KIND_LINEAR)
    res = O.fit(X, 3, 2, 0.5, ker, iters=10, seed=9)
    Xn = X[:40] + 0.1
    mus = np.stack([res["support_coords"][res["support_labels"] == j].mean(0)
                    for j in range(3)])
    dist = ((Xn[:, None] - mus[None]) ** 2).sum(axis=2)
    u, dmin = O.assign(res, Xn, "supports")
    assert np.array_equal(u, np.argmin(dist, axis=1))
    assert np.allclose(dmin, dist.min(axis=1), rtol=1e-9, atol=1e-9)
    MX = res["medoid_coords"]
    dm = ((Xn[:, None] - MX[None]) ** 2).sum(axis=2)
    um, _ = O.assign(res, Xn, "medoids")
    assert np.array_equal(um, np.argmin(dm, axis=1))
    assert O.cost(res, Xn, "medoids") == pytest.approx(dm.min(axis=1).sum(), rel=1e-9)


# ---------------------------------------------------------------------------
# Model selection and diagnostics (Section 4.1 Fig. 4b; Sections 4.4, 4.5).
# ---------------------------------------------------------------------------
def test_displacement_linear_is_mean_euclidean_distance():
    X, _ = _blob_data(N=300, d=3, C=4, problem=20)
    ker = O.Kernel(O.KIND_LINEAR)
    a, b = np.array([3, 10, 55, 7]), np.array([3, 99, 12, 250])
    want = np.mean(np.linalg.norm(X[a] - X[b], axis=1))      # explicit coordinates
    assert abs(O.medoid_displacement(ker, X, a, b) - want) <= 1e-12 * want
    assert O.medoid_displacement(ker, X, a, a) == 0.0


def test_displacement_rbf_closed_form():
    from scipy.spatial.distance import cdist
    X, _ = _blob_data(N=200, d=5, C=3, problem=21)
    sig = 2.5
    ker = O.Kernel(O.KIND_RBF, sig)
    a, b = np.array([0, 5, 9]), np.array([1, 5, 150])
    r = np.diag(cdist(X[a], X[b]))
    want = np.mean(np.sqrt(2.0 - 2.0 * np.exp(-r ** 2 / (2 * sig ** 2))))
    assert abs(O.medoid_displacement(ker, X, a, b) - want) <= 1e-12
    res = O.fit(X, 3, 2, 0.5, ker, 5, 4)
    tr = O.displacement_trace(res, X)
    assert len(tr) == 2 and all(v >= 0.0 for v in tr)


def test_elbow_index_hand_worked():
    # costs 100 50 10 8 6 4 over six consecutive C; scaled y = 1, .5, .0625,
    # .0417, .0208, 0; the chord from (0, 1) to (1, 0) is 1 - x with x = k/5;
    # chord - y = 0, .3, .5375, .3583, .1792, 0: the elbow is the third C
    assert O.elbow_index([100, 50, 10, 8, 6, 4]) == 2
    # the same under any positive affine change of the cost
    assert O.elbow_index([3 + 0.5 * c for c in [100, 50, 10, 8, 6, 4]]) == 2
    # a straight line has no elbow below its chord: the first C
    assert O.elbow_index([10, 8, 6, 4, 2]) == 0
    assert O.elbow_index([5.0]) == 0


def test_elbow_finds_separated_groups():
    # four well separated groups: the cost drops steeply up to C = 4, then flattens
    g = np.random.Generator(np.random.PCG64(31))
    centres = np.array([[0.0, 0.0], [20.0, 0.0], [0.0, 20.0], [20.0, 20.0]])
    X = centres[np.arange(240) % 4] + g.normal(0, 1.0, size=(240, 2))
    res = O.elbow(X, 2, 8, 1, 1.0, O.Kernel(O.KIND_LINEAR), 15, seed=5, n_restarts=3)
    assert res["C"] == 4
    assert np.all(np.diff(res["costs"]) <= 1e-9 * res["costs"][0])


def test_restarts_keep_the_minimum_explicit_cost():
    X, _ = _blob_data(N=400, d=2, C=6, problem=22)
    ker = O.Kernel(O.KIND_LINEAR)
    seeds = O.restart_seeds(9, 5)
    res = O.fit_restarts(X, 6, 2, 0.5, ker, 10, seeds)
    # explicit Eq. 1 cost against each restart's medoids (squared Euclidean distances)
    explicit = []
    for f in res["fits"]:
        M = X[f["medoids"]]
        explicit.append(float(((X[:, None, :] - M[None, :, :]) ** 2).sum(axis=2).min(axis=1).sum()))
    assert np.allclose(res["costs"], explicit, rtol=1e-12)
    assert res["best"] == int(np.argmin(explicit))
    assert res["fit"] is res["fits"][res["best"]]
    assert len(set(seeds)) == 5
