"""Parity of the CUDA library with the FP64 oracle, through the C ABI.

Sizes span several CTA tiles and ragged tails; edge cases cover C = 1, one
landmark, zero iterations, host buffers and invalid arguments.
"""

import numpy as np
import pytest

from oracle import kkm_oracle as O
from synth import blobs, md_trajectory
from tests.helpers import (DIST_REL, KERNEL_ABS, OMEGA_REL, assert_close_rel, assert_labels,
                           clear_rows, first_divergence)

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _np(t):
    return t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)


def _median_sigma(X, kind="rbf", n_atoms=0):
    """A bandwidth computed once by the oracle and passed to both sides."""
    k = O.Kernel(O.KIND_RBF if kind == "rbf" else O.KIND_RMSD, 0.0, n_atoms)
    return float(np.float32(O.median_bandwidth(X.astype(np.float64), k, O.SplitMix64(99), 512)))


# ------------------------------------------------------------ kernel block
@pytest.mark.parametrize("nA,nB,d", [(300, 517, 37), (7, 1029, 16), (129, 130, 784), (1, 33, 5),
                                     (33, 64, 8)])
def test_kernel_matrix_rbf(lib, nA, nB, d):
    X, _ = blobs(nA + nB, d, 4, workload=50, problem=d)
    A, Bm = X[:nA], X[nA:]
    sig = _median_sigma(X)
    got = _np(lib.kkm_kernel_matrix(_dev(A), _dev(Bm), "rbf", sig))
    want = O.Kernel(O.KIND_RBF, sig)(A, Bm)
    assert np.max(np.abs(got - want)) <= KERNEL_ABS


def test_kernel_matrix_rbf_host_buffers_and_diagonal(lib):
    X, _ = blobs(200, 12, 3, workload=50, problem=1)
    sig = _median_sigma(X)
    got = lib.kkm_kernel_matrix(X, X, "rbf", sig)
    want = O.Kernel(O.KIND_RBF, sig)(X, X)
    assert np.max(np.abs(got - want)) <= KERNEL_ABS


def test_kernel_matrix_linear(lib):
    X, _ = blobs(400, 23, 3, workload=50, problem=2)
    A, Bm = X[:150], X[150:]
    got = _np(lib.kkm_kernel_matrix(_dev(A), _dev(Bm), "linear"))
    want = A.astype(np.float64) @ Bm.astype(np.float64).T
    scale = np.linalg.norm(A, axis=1)[:, None] * np.linalg.norm(Bm, axis=1)[None, :]
    assert np.max(np.abs(got - want) / scale) <= 1e-5



@pytest.mark.parametrize("nA,nB,d,kind", [(3, 1000, 784, "rbf"), (17, 2051, 100, "rbf"), (32, 777, 8, "rbf"),
                                          (2, 5000, 33, "rbf"), (5, 3001, 129, "linear"), (16, 1500, 256, "linear"),
                                          (31, 300, 64, "linear")])
def test_kernel_matrix_few_references(lib, nA, nB, d, kind):
    """At most 32 reference rows (the medoid and k-means++ columns): the
    reference rows held in shared memory as pairs (an odd count padded), two
    or four sample rows per warp, row lengths that are not a multiple of the
    128-value step; Gaussian and linear kinds against the oracle."""
    X, _ = blobs(nA + nB, d, 5, workload=53, problem=nA * 1000 + d)
    A, Bm = X[:nA], X[nA:]
    if kind == "rbf":
        sig = _median_sigma(X)
        got = _np(lib.kkm_kernel_matrix(_dev(A), _dev(Bm), "rbf", sig))
        want = O.Kernel(O.KIND_RBF, sig)(A, Bm)
        assert np.max(np.abs(got - want)) <= KERNEL_ABS
        assert np.mean(want > 0.05) > 0.05  # non-negligible values are covered
    else:
        got = _np(lib.kkm_kernel_matrix(_dev(A), _dev(Bm), "linear"))
        want = A.astype(np.float64) @ Bm.astype(np.float64).T
        scale = np.linalg.norm(A, axis=1)[:, None] * np.linalg.norm(Bm, axis=1)[None, :]
        assert np.max(np.abs(got - want) / scale) <= 1e-5

@pytest.mark.parametrize("atoms", [300, 57])
def test_kernel_matrix_rmsd(lib, atoms):
    F, _ = md_trajectory(n_frames=260, n_atoms=atoms, n_states=3, dwell=40.0, workload=51,
                         problem=atoms)
    X = F.reshape(len(F), -1)
    A, Bm = X[:70], X[70:]
    got = _np(lib.kkm_kernel_matrix(_dev(A), _dev(Bm), "rmsd", 1.5, n_atoms=atoms))
    want = O.Kernel(O.KIND_RMSD, 1.5, atoms)(A, Bm)
    assert np.max(np.abs(got - want)) <= KERNEL_ABS
    assert np.mean(want > 0.1) > 0.1  # the test covers non-negligible values


def test_rmsd_self_and_rigid_motion(lib):
    from synth import random_rigid_motion
    F, _ = md_trajectory(n_frames=40, n_atoms=120, n_states=2, workload=52)
    g = np.random.Generator(np.random.PCG64(5))
    R, t = random_rigid_motion(g, len(F))
    G = (np.einsum("nij,nkj->nki", R, F) + t[:, None, :]).astype(np.float32)
    X, Y = F.reshape(40, -1), G.reshape(40, -1)
    k_xy = _np(lib.kkm_kernel_matrix(_dev(X), _dev(Y), "rmsd", 1.5, n_atoms=120))
    assert np.all(np.abs(np.diag(k_xy) - 1.0) <= 1e-5)
    k_xx = _np(lib.kkm_kernel_matrix(_dev(X), _dev(X), "rmsd", 1.5, n_atoms=120))
    assert np.max(np.abs(k_xx - k_xy)) <= KERNEL_ABS


@pytest.mark.parametrize("kind", ["rbf", "rbf_long", "rbf_long_small", "rmsd"])
def test_median_bandwidth(lib, kind):
    """The median rule on 2,048 drawn samples; long rows (>= 256 floats) take
    the split-K distance path, a ragged sample count the partial tiles."""
    if kind.startswith("rbf"):
        N, d = {"rbf": (3000, 16), "rbf_long": (2600, 300), "rbf_long_small": (1500, 257)}[kind]
        X, _ = blobs(N, d, 5, workload=0, problem=d)
        k = O.Kernel(O.KIND_RBF, 0.0)
        kind = "rbf"
    else:
        F, _ = md_trajectory(n_frames=900, n_atoms=40, n_states=3, dwell=100.0, workload=53)
        X = F.reshape(len(F), -1)
        k = O.Kernel(O.KIND_RMSD, 0.0, 40)
    got = lib.kkm_median_bandwidth(_dev(X), kind, n_atoms=k.n_atoms, seed=17)
    _, bw, _ = O.rng_streams(17, 1)
    want = O.median_bandwidth(X.astype(np.float64), k, bw)
    assert_close_rel(got, want, 1e-5, "median bandwidth")


# ------------------------------------------------------- teacher-forced step
def _step_case(lib, X, L, u, C, kind, sig, n_atoms=0):
    got = lib.kkm_debug_step(_dev(X), L, u, C, kind, sig, n_atoms)
    k = O.Kernel({"rbf": O.KIND_RBF, "rmsd": O.KIND_RMSD, "linear": O.KIND_LINEAR}[kind], sig, n_atoms)
    Xd = X.astype(np.float64)
    Kb = k(Xd, Xd[L])
    ref = O.inner_step(Kb, k.self_terms(Xd), np.asarray(L, np.int64), np.asarray(u, np.int64), C)
    assert np.array_equal(got["n"], ref["n"])
    live = ref["n"] > 0
    assert np.all(np.isnan(got["ghat"][~live]))
    scale = k.self_terms(Xd)[:, None] + np.where(live, ref["ghat"], 0.0)[None, :]
    assert np.allclose(got["ghat"][live], ref["ghat"][live], rtol=1e-6, atol=1e-9)
    fd = np.abs(got["fhat"][:, live] - ref["fhat"][:, live])
    assert np.max(2 * fd / scale[:, live]) <= DIST_REL
    mask = assert_labels(got["u"], ref["u"], ref["d"], "step labels")
    assert_close_rel(got["omega"], ref["omega"], OMEGA_REL, "step Omega")
    fin = np.isfinite(ref["margin"]) & mask
    if fin.any():
        assert np.max(np.abs(got["margin"][fin] - ref["margin"][fin]) / scale.max(axis=1)[fin]) <= 4 * DIST_REL
    assert abs(got["changed"] - ref["changed"]) <= int(np.sum(~mask))
    return got, ref


@pytest.mark.parametrize("Ni,nL,C,d", [(2000, 700, 5, 16), (2000, 2000, 5, 16), (777, 65, 9, 30),
                                       (5000, 1, 3, 8), (300, 300, 1, 4)])
def test_debug_step_rbf(lib, Ni, nL, C, d):
    X, y = blobs(Ni, d, max(C, 2), workload=54, problem=Ni + nL)
    sig = _median_sigma(X)
    g = np.random.Generator(np.random.PCG64(Ni))
    L = np.sort(g.choice(Ni, nL, replace=False)).astype(np.int32)
    u = np.where(g.random(Ni) < 0.7, y % C, g.integers(0, C, Ni)).astype(np.int32)
    _step_case(lib, X, L, u, C, "rbf", sig)


def test_debug_step_empty_cluster_and_linear(lib):
    X, y = blobs(900, 6, 3, workload=54, problem=3)
    L = np.arange(0, 900, 3, dtype=np.int32)
    u = (y % 3).astype(np.int32)
    u[L] = np.where(u[L] == 2, 0, u[L])  # cluster 2 keeps members but no landmark
    got, ref = _step_case(lib, X, L, u, 3, "rbf", _median_sigma(X))
    assert ref["n"][2] == 0 and np.all(got["u"] != 2)
    _step_case(lib, X, L, (y % 3).astype(np.int32), 3, "linear", 0.0)


def test_debug_step_rmsd(lib):
    F, st = md_trajectory(n_frames=600, n_atoms=60, n_states=4, dwell=50.0, workload=55)
    X = F.reshape(600, -1)
    L = np.arange(0, 600, 5, dtype=np.int32)
    u = (st % 4).astype(np.int32)
    _step_case(lib, X, L, u, 4, "rmsd", 1.5, 60)


# ----------------------------------------------------------- whole fits
def _fit_pair(lib, X, C, B, s, iters, seed, kind="rbf", sig=None, n_atoms=0, sampling="stride",
              early_stop=True, use_oracle_init=True, iteration="auto"):
    okind = {"rbf": O.KIND_RBF, "rmsd": O.KIND_RMSD, "linear": O.KIND_LINEAR}[kind]
    ref = O.fit(X.astype(np.float64), C, B, s, O.Kernel(okind, sig or 0.0, n_atoms), iters, seed,
                early_stop=early_stop, sampling=sampling)
    init = ref["details"][0]["M_before"] if use_oracle_init else None
    lab, model = lib.kkm_fit(_dev(X), C, B, s, kind, sig or 0.0, n_atoms, iters, seed, sampling=sampling,
                             early_stop=early_stop, init_medoids=init, iteration=iteration)
    return _np(lab), model, ref


def _check_fit(lab, model, ref):
    om, ch = model.trace()
    want = np.array([t[2] for t in ref["trace"]])
    div = first_divergence(om, want)
    assert om.shape == want.shape, f"trace lengths {om.shape} vs {want.shape}"
    assert div is None, f"Omega trace diverges at iteration {div}: {om[div]} vs {want[div]}"
    for det in ref["details"]:
        assert_labels(lab[det["gidx"]], det["u"], det["steps"][-1]["d"] if det["steps"] else
                      np.zeros((len(det["gidx"]), 2)), "fit labels")
    idx, cnt, coords = model.medoids()
    assert np.array_equal(idx, ref["medoids"])
    assert np.array_equal(cnt, ref["W"])
    lab_s, gh, n = model.supports()
    assert np.array_equal(n, ref["n"])
    live = ref["n"] > 0
    assert np.allclose(gh[live], ref["ghat"][live], rtol=1e-6)


def test_fit_exact_kernel_kmeans_2000x16(lib):
    """Exact kernel k-means: N=2000, d=16, 5 blobs, median bandwidth, C=5, B=1, s=1, 20 iterations."""
    X, _ = blobs(2000, 16, 5, workload=0)
    sig = _median_sigma(X)
    lab, model, ref = _fit_pair(lib, X, 5, 1, 1.0, 20, seed=1, sig=sig, early_stop=False)
    _check_fit(lab, model, ref)


@pytest.mark.parametrize("iteration", ["fused", "split"])
@pytest.mark.parametrize("sampling", ["stride", "block"])
def test_fit_minibatch_landmarks(lib, sampling, iteration):
    X, _ = blobs(3001, 20, 6, workload=56)
    sig = _median_sigma(X)
    lab, model, ref = _fit_pair(lib, X, 6, 3, 0.3, 15, seed=4, sig=sig, sampling=sampling, iteration=iteration)
    _check_fit(lab, model, ref)


def test_fit_kmeanspp_on_device(lib):
    X, _ = blobs(2500, 10, 7, workload=57)
    sig = _median_sigma(X)
    lab, model, ref = _fit_pair(lib, X, 7, 2, 0.5, 12, seed=9, sig=sig, use_oracle_init=False)
    _check_fit(lab, model, ref)


def test_kmeanspp_picks(lib):
    X, _ = blobs(4000, 16, 8, workload=58)
    sig = _median_sigma(X)
    for seed in range(4):
        got = lib.kkm_debug_kmeanspp(_dev(X), 8, seed, "rbf", sig)
        kpp, _, _ = O.rng_streams(seed, 1)
        want = O.kmeanspp(X.astype(np.float64), 8, O.Kernel(O.KIND_RBF, sig), kpp)
        assert np.array_equal(got, want)


@pytest.mark.parametrize("iteration", ["fused", "split"])
def test_fit_rmsd(lib, iteration):
    F, _ = md_trajectory(n_frames=1500, n_atoms=60, n_states=4, dwell=60.0, workload=59)
    X = F.reshape(1500, -1)
    lab, model, ref = _fit_pair(lib, X, 4, 2, 0.2, 10, seed=2, kind="rmsd", sig=1.5, n_atoms=60,
                                iteration=iteration)
    _check_fit(lab, model, ref)


@pytest.mark.parametrize("iteration", ["fused", "split"])
def test_fit_linear_is_lloyd_on_device(lib, iteration):
    X, _ = blobs(1200, 5, 4, workload=60)
    lab, model, ref = _fit_pair(lib, X, 4, 1, 1.0, 15, seed=3, kind="linear", sig=0.0, iteration=iteration)
    _check_fit(lab, model, ref)


# ------------------------------------------------ fused iteration shapes
def test_fused_iteration_many_clusters_ragged(lib):
    """The fused iteration at its largest C (64) on a ragged mini-batch (1,237
    samples: the last column group and strip are partial) against the oracle;
    C = 65 is refused for KKM_ITER_FUSED and runs split under AUTO."""
    X, _ = blobs(1237, 8, 40, workload=90)
    sig = _median_sigma(X)
    lab, model, ref = _fit_pair(lib, X, 64, 1, 0.6, 12, seed=5, sig=sig, iteration="fused")
    _check_fit(lab, model, ref)
    with pytest.raises(lib.KKMError) as e:
        lib.kkm_fit(_dev(X), 65, 1, 0.6, "rbf", sig, iters=2, seed=5, iteration="fused")
    assert e.value.status == lib.STATUS_EINVAL
    lab, model, ref = _fit_pair(lib, X, 65, 1, 0.6, 6, seed=5, sig=sig)
    _check_fit(lab, model, ref)


def test_fused_iteration_matches_split_long_landmark_list(lib):
    """More landmarks than the fused kernel stages in shared memory (9,000 >
    8,192: the sorted list is read from global memory), and landmark labels
    that change between iterations (supports re-sorted by the closing CTA):
    the fused and split forms give the same trace to 1e-6 and the same labels
    on all but near-tied rows."""
    X, _ = blobs(20000, 4, 5, workload=91)
    sig = _median_sigma(X)
    runs = {it: lib.kkm_fit(_dev(X), 5, 1, 0.45, "rbf", sig, iters=12, seed=2, early_stop=False, iteration=it)
            for it in ("fused", "split")}
    (lf, mf), (ls, ms) = runs["fused"], runs["split"]
    of, os_ = mf.trace()[0], ms.trace()[0]
    assert of.shape == os_.shape == (12,)
    assert np.max(np.abs(of - os_) / os_) <= 1e-6
    assert np.mean(_np(lf) == _np(ls)) >= 0.999
    assert mf.trace()[1].max() > 0  # labels did change during the loop


def test_fit_median_bandwidth_inside(lib):
    X, _ = blobs(2200, 12, 4, workload=61)
    ref = O.fit(X.astype(np.float64), 4, 2, 0.5, O.Kernel(O.KIND_RBF, 0.0), 8, 5)
    lab, model = lib.kkm_fit(_dev(X), 4, 2, 0.5, "rbf", 0.0, iters=8, seed=5,
                             init_medoids=ref["details"][0]["M_before"])
    assert_close_rel(model.info()["sigma"], ref["kernel"].sigma, 1e-5, "sigma")


# ---------------------------------------------------------------- edge cases
def test_fit_edge_cases(lib):
    X, _ = blobs(640, 6, 3, workload=62)
    sig = _median_sigma(X)
    for C, B, s, iters in [(1, 1, 1.0, 5), (3, 2, 0.001, 5), (3, 2, 0.5, 0), (3, 1, 1.0, 1)]:
        lab, model, ref = _fit_pair(lib, X, C, B, s, iters, seed=7, sig=sig)
        _check_fit(lab, model, ref)
    # C equal to the mini-batch size
    Xs = X[:12]
    lab, model, ref = _fit_pair(lib, Xs, 4, 3, 1.0, 3, seed=7, sig=sig)
    _check_fit(lab, model, ref)


def test_fit_host_buffers_equal_device(lib):
    X, _ = blobs(1500, 9, 4, workload=63)
    sig = _median_sigma(X)
    lab_d, m_d = lib.kkm_fit(_dev(X), 4, 2, 0.4, "rbf", sig, iters=10, seed=8)
    lab_h, m_h = lib.kkm_fit(X, 4, 2, 0.4, "rbf", sig, iters=10, seed=8)
    assert isinstance(lab_h, np.ndarray)
    assert np.array_equal(_np(lab_d), lab_h)
    assert np.array_equal(m_d.trace()[0], m_h.trace()[0])


def test_fit_pinned_host_input(lib):
    """Pinned host input is copied and checked by one kernel that reads it
    directly (a ragged tail of 10,507 floats); a pinned view that is not
    16-byte aligned takes the copy-then-check path; both give the bits of the
    device-input fit.  A NaN in pinned input is refused."""
    import torch
    X, _ = blobs(1501, 7, 4, workload=63, problem=1)
    sig = _median_sigma(X)
    lab_d, m_d = lib.kkm_fit(_dev(X), 4, 2, 0.4, "rbf", sig, iters=8, seed=8)
    Xp = torch.from_numpy(X).pin_memory()
    big = torch.from_numpy(np.concatenate([[0.0], X.ravel()]).astype(np.float32)).pin_memory()
    Xu = big[1:].view(1501, 7)
    assert Xu.data_ptr() % 16 != 0
    for Xh in (Xp, Xu):
        lab_h, m_h = lib.kkm_fit(Xh, 4, 2, 0.4, "rbf", sig, iters=8, seed=8)
        assert np.array_equal(_np(lab_d), _np(lab_h))
        assert np.array_equal(m_d.trace()[0], m_h.trace()[0])
    la_d, da_d = lib.kkm_assign(m_d, _dev(X))
    la_p, da_p = lib.kkm_assign(m_d, Xp)
    assert np.array_equal(_np(la_d), _np(la_p)) and np.array_equal(_np(da_d), _np(da_p))
    bad = Xp.clone().pin_memory()
    bad[1500, 6] = float("nan")
    with pytest.raises(lib.KKMError) as e:
        lib.kkm_fit(bad, 4, 2, 0.4, "rbf", sig, iters=2, seed=8)
    assert "NaN" in str(e.value)


@pytest.mark.parametrize("prec,pipeline", [("fp32", "auto"), ("fp32", "serial"), ("bf16", "auto"), ("bf16", "overlap")])
def test_fit_pinned_host_input_in_place(lib, prec, pipeline):
    """Pinned host input whose rows are a multiple of 4 floats stays on the
    host in a whole fit: each mini-batch's rows are read over the link as they
    are gathered (and checked there), the medoid and sample rows likewise.
    Every result is the bits of the device-input fit; a NaN in the last row
    (the last mini-batch to be fetched) is refused with no model."""
    import torch
    X, _ = blobs(3003, 16, 5, workload=63, problem=2)
    sig = _median_sigma(X)
    p = lib.KKM_BF16 if prec == "bf16" else lib.KKM_FP32
    kw = dict(iters=8, seed=8, precision=p, pipeline=pipeline)
    lab_d, m_d = lib.kkm_fit(_dev(X), 5, 3, 0.3, "rbf", 0.0, **kw)
    Xp = torch.from_numpy(X).pin_memory()
    assert Xp.data_ptr() % 16 == 0
    lab_h, m_h = lib.kkm_fit(Xp, 5, 3, 0.3, "rbf", 0.0, **kw)
    assert np.array_equal(_np(lab_d), _np(lab_h))
    assert np.array_equal(m_d.trace()[0], m_h.trace()[0]) and np.array_equal(m_d.trace()[1], m_h.trace()[1])
    for a, b in zip(m_d.medoids(), m_h.medoids()):
        assert np.array_equal(np.asarray(a), np.asarray(b))
    for a, b in zip(m_d.supports(), m_h.supports()):
        assert np.array_equal(np.asarray(a), np.asarray(b), equal_nan=True)
    bad = Xp.clone().pin_memory()
    bad[3002, 15] = float("nan")
    with pytest.raises(lib.KKMError) as e:
        lib.kkm_fit(bad, 5, 3, 0.3, "rbf", sig, **kw)
    assert "NaN" in str(e.value)
    bad[3002, 15] = float("inf")
    with pytest.raises(lib.KKMError):
        lib.kkm_fit(bad, 5, 3, 0.3, "rbf", sig, **kw)


@pytest.mark.parametrize("n_atoms", [20, 21])
def test_fit_pinned_host_md_frames_in_place(lib, n_atoms):
    """Pinned host MD frames stay on the host in a whole fit: each
    mini-batch's frames are staged by the copy engine, checked and prepared
    from the staging buffer.  Every result is the bits of the device-input
    fit (frames of 60 and 63 floats); a NaN in the last frame is refused."""
    import torch
    from synth import md_trajectory
    F, _ = md_trajectory(2400, n_atoms, dwell=50.0, workload=63, problem=3)
    X = np.ascontiguousarray(F.reshape(2400, -1).astype(np.float32))
    kw = dict(iters=5, seed=4, pipeline="overlap")
    lab_d, m_d = lib.kkm_fit(_dev(X), 4, 3, 0.2, "rmsd", 1.5, n_atoms, **kw)
    Xp = torch.from_numpy(X).pin_memory()
    lab_h, m_h = lib.kkm_fit(Xp, 4, 3, 0.2, "rmsd", 1.5, n_atoms, **kw)
    assert np.array_equal(_np(lab_d), _np(lab_h))
    assert np.array_equal(m_d.trace()[0], m_h.trace()[0])
    for a, b in zip(m_d.medoids(), m_h.medoids()):
        assert np.array_equal(np.asarray(a), np.asarray(b))
    bad = Xp.clone().pin_memory()
    bad[2399, 0] = float("nan")
    with pytest.raises(lib.KKMError) as e:
        lib.kkm_fit(bad, 4, 3, 0.2, "rmsd", 1.5, n_atoms, **kw)
    assert "NaN" in str(e.value)


def test_fit_deterministic(lib):
    X, _ = blobs(5000, 32, 6, workload=64)
    sig = _median_sigma(X)
    runs = [lib.kkm_fit(_dev(X), 6, 2, 0.3, "rbf", sig, iters=10, seed=3) for _ in range(2)]
    assert np.array_equal(_np(runs[0][0]), _np(runs[1][0]))
    assert np.array_equal(runs[0][1].trace()[0], runs[1][1].trace()[0])


def test_invalid_arguments(lib):
    X, _ = blobs(100, 4, 2, workload=65)
    Xd = _dev(X)
    bad = [dict(C=0), dict(C=300), dict(B=0), dict(B=101), dict(s=0.0), dict(s=1.5), dict(iters=-1),
           dict(C=60, B=2)]
    for kw in bad:
        args = dict(C=2, B=1, s=1.0, iters=3)
        args.update(kw)
        with pytest.raises(lib.KKMError) as e:
            lib.kkm_fit(Xd, args["C"], args["B"], args["s"], "rbf", 1.0, iters=args["iters"], seed=1)
        assert e.value.status == lib.STATUS_EINVAL, kw
    Xn = X.copy()
    Xn[5, 2] = np.nan
    with pytest.raises(lib.KKMError) as e:
        lib.kkm_fit(_dev(Xn), 2, 1, 1.0, "rbf", 1.0, iters=3, seed=1)
    assert e.value.status == lib.STATUS_EINVAL
    with pytest.raises(lib.KKMError):
        lib.kkm_fit(Xd, 2, 1, 1.0, "rmsd", 1.0, n_atoms=3, iters=3, seed=1)  # d != 3 n_atoms
    with pytest.raises(lib.KKMError):
        lib.kkm_fit(Xd, 2, 1, 1.0, "rbf", 1.0, iters=3, seed=1, init_medoids=[0, 100])
    # the library still works after rejected calls
    lab, _ = lib.kkm_fit(Xd, 2, 1, 1.0, "rbf", 1.0, iters=3, seed=1)
    assert _np(lab).min() >= 0


# ------------------------------------------------------------ assign / cost
@pytest.mark.parametrize("mode", ["supports", "medoids"])
def test_assign_and_cost(lib, mode):
    X, _ = blobs(3000, 14, 5, workload=66)
    sig = _median_sigma(X)
    lab, model, ref = _fit_pair(lib, X, 5, 2, 0.4, 10, seed=6, sig=sig)
    Xn, _ = blobs(1234, 14, 5, workload=66, problem=1)
    u, dist = lib.kkm_assign(model, _dev(Xn), mode)
    d_ref = O.assign_distances(ref, Xn, mode)
    u_ref = np.argmin(d_ref, axis=1)
    assert_labels(_np(u), u_ref, d_ref, "assign labels")
    dmin = d_ref[np.arange(len(Xn)), u_ref]
    scale = 1.0 + (np.nanmax(ref["ghat"]) if mode == "supports" else 1.0)
    ok = clear_rows(d_ref)
    assert np.max(np.abs(_np(dist)[ok] - dmin[ok])) <= DIST_REL * scale
    assert_close_rel(lib.kkm_cost(model, _dev(Xn), mode), O.cost(ref, Xn, mode), OMEGA_REL, "cost")
    # host buffers and empty input
    u_h, _ = lib.kkm_assign(model, Xn, mode)
    assert np.array_equal(u_h, _np(u))
    u0, _ = lib.kkm_assign(model, Xn[:0], mode)
    assert len(u0) == 0


def test_assign_rmsd_supports(lib):
    F, _ = md_trajectory(n_frames=1200, n_atoms=48, n_states=3, dwell=80.0, workload=67)
    X = F.reshape(1200, -1)
    lab, model, ref = _fit_pair(lib, X, 3, 2, 0.25, 8, seed=3, kind="rmsd", sig=1.5, n_atoms=48)
    Fn, _ = md_trajectory(n_frames=300, n_atoms=48, n_states=3, dwell=80.0, workload=67, problem=1)
    Xn = Fn.reshape(300, -1)
    u, _ = lib.kkm_assign(model, _dev(Xn), "supports")
    d_ref = O.assign_distances(ref, Xn, "supports")
    assert_labels(_np(u), np.argmin(d_ref, axis=1), d_ref, "rmsd assign")
