"""Parity at the benchmark workloads' full sizes, in the launch configuration
the benchmark times, on sampled outputs the oracle computes one by one, and
properties of the whole fit that hold at any size.  Oracle inputs come from
the generators and the oracle's own plan functions (mini-batches, landmark
draws); teacher-forced labels are the generators' class / state labels.

MNIST-shaped fit: 60,000 x 784, C = 10, B = 4, s = 0.2 (15,000 samples and
3,000 landmarks per mini-batch), 30 iterations, BF16 kernel block.
MD-shaped mini-batch: 25,000 frames x 300 atoms and 1,250 landmarks (one
mini-batch of the 500,000-frame, B = 20, s = 0.05 workload), RMSD kernel,
sigma = 1.5 A.  The whole MD trajectory is not generated here: a stride
mini-batch of it is a trajectory with a 20 times shorter mean dwell, which is
what is generated.
"""

import json
import os

import numpy as np
import pytest

from oracle import kkm_oracle as O
from synth import md_trajectory, mnist_like
from tests.helpers import DIST_REL, KERNEL_ABS, assert_labels, rel_margin

pytestmark = pytest.mark.gpu

N, D, C, B, S, ITERS, SEED = 60000, 784, 10, 4, 0.2, 30, 1710


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _bf16(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


@pytest.fixture(scope="module")
def mnist(lib):
    X, cls = mnist_like(N, D)
    Xd = _dev(X)
    # the bandwidth is an input given to both sides: the oracle's median rule
    # on 512 samples (the rule itself is tested at 2,048 samples elsewhere)
    sigma = float(np.float32(O.median_bandwidth(X, O.Kernel(O.KIND_RBF, 0.0), O.SplitMix64(SEED), 512)))
    return X, Xd, sigma, cls


def _pairs(rng, na, nb, k):
    return rng.integers(0, na, k), rng.integers(0, nb, k)


def _plan(batch):
    """Mini-batch `batch` and its landmarks, from the oracle's definitions."""
    _, _, lm = O.rng_streams(SEED, B)
    gidx = O.minibatch_indices(N, B)[batch]
    L = O.landmark_indices(len(gidx), S, lm[batch])
    return gidx, L


def test_kernel_block_full_minibatch(lib, mnist):
    """K(L, X^0) of the first mini-batch (3,000 x 15,000), tensor-core BF16 and
    FP32, against the oracle on 4,000 sampled entries."""
    X, _, sigma, _ = mnist
    gidx, L = _plan(0)
    Xb = X[gidx]
    A, Bq = Xb[L], Xb
    rng = np.random.default_rng(1)
    a, b = _pairs(rng, len(L), len(gidx), 4000)
    for prec, (Ar, Br) in ((lib.KKM_BF16, (_bf16(A), _bf16(Bq))), (lib.KKM_FP32, (A, Bq))):
        K = lib.kkm_kernel_matrix(_dev(A), _dev(Bq), "rbf", sigma, precision=prec)
        got = K[_dev(a.astype(np.int64)), _dev(b.astype(np.int64))].cpu().numpy()
        diff = Ar[a].astype(np.float64) - Br[b].astype(np.float64)
        want = np.exp(-np.einsum("ij,ij->i", diff, diff) / (2.0 * float(sigma) ** 2))
        assert np.max(np.abs(got - want)) <= KERNEL_ABS, prec


def _oracle_rows(kernel, Xb, L, u, C, rows):
    """f_hat of the sampled rows and g_hat of every cluster (Eq. 16-17), one
    cluster at a time from its own support."""
    Xl = Xb[L]
    uL = u[L]
    KR = kernel(Xb[rows], Xl)
    n = np.array([np.count_nonzero(uL == j) for j in range(C)])
    fhat = np.full((len(rows), C), np.nan)
    ghat = np.full(C, np.nan)
    for j in range(C):
        if n[j] == 0:
            continue
        Sj = Xl[uL == j]
        fhat[:, j] = KR[:, uL == j].sum(axis=1) / n[j]
        ghat[j] = kernel(Sj, Sj).sum() / (n[j] * n[j])
    kself = kernel.self_terms(Xb[rows])
    d = np.where(n[None, :] > 0, kself[:, None] - 2.0 * fhat + ghat[None, :], np.inf)
    return n, fhat, ghat, d


def test_fp32_step_full_minibatch(lib, mnist):
    """One teacher-forced inner iteration of the plain FP32 path on the first
    mini-batch (15,000 x 3,000 block), labels = the generator's classes; 256
    sampled rows and every cluster's g_hat against the oracle."""
    X, Xd, sigma, cls = mnist
    gidx, L = _plan(0)
    Xb = X[gidx]
    u = cls[gidx].astype(np.int32)
    got = lib.kkm_debug_step(Xb, L, u, C, "rbf", sigma)
    rng = np.random.default_rng(2)
    rows = np.unique(np.concatenate([rng.integers(0, len(gidx), 224), L[rng.integers(0, len(L), 32)]]))
    ker = O.Kernel(O.KIND_RBF, float(sigma))
    n, fhat, ghat, d = _oracle_rows(ker, Xb.astype(np.float64), L, u.astype(np.int64), C, rows)
    assert np.array_equal(got["n"], n)
    live = n > 0
    assert np.allclose(got["ghat"][live], ghat[live], rtol=1e-6, atol=1e-9)
    scale = 1.0 + np.where(live, ghat, 0.0)[None, :]
    fd = np.abs(got["fhat"][rows][:, live] - fhat[:, live])
    assert np.max(2 * fd / scale[:, live]) <= DIST_REL
    assert_labels(got["u"][rows], np.argmin(d, axis=1), d, "full-size step labels")


def test_bf16_fit_full_size(lib, mnist):
    """The benchmark's fit, by properties that hold at any size: trace length
    and values, counts, medoid coordinates, the support equal to the last
    mini-batch's landmarks with the fit's labels, the model's g_hat equal to
    the Eq. 16 mean of its support under its own labels (oracle kernel on the
    rounded rows), and kkm_assign of 2,000 new samples equal to the Eq. 15
    argmin against the model's own support (oracle kernel, the model's g_hat)."""
    X, Xd, sigma, _ = mnist
    lab, model = lib.kkm_fit(Xd, C, B, S, "rbf", 0.0, iters=ITERS, seed=SEED, early_stop=False,
                             precision=lib.KKM_BF16)
    lab = lab.cpu().numpy()
    om, ch = model.trace()
    assert om.shape == (B * ITERS,) and np.all(np.isfinite(om)) and np.all(om > 0)
    assert lab.min() >= 0 and lab.max() < C
    idx, cnt, coords = model.medoids()
    assert cnt.sum() == N and np.all((idx >= 0) & (idx < N))
    assert np.array_equal(coords, X[idx])
    info = model.info()
    # the support: landmarks of the last mini-batch
    gidx, L = _plan(B - 1)
    sup = X[gidx][L]
    lab_s, gh, n = model.supports()
    assert n.sum() == len(L) and np.array_equal(n, np.bincount(lab_s, minlength=C))
    assert np.array_equal(lab_s, lab[gidx][L])
    # g_hat of the BF16 block (rounded rows, FP16 storage): against the oracle
    # on the rounded support, at the storage precision
    ker = O.Kernel(O.KIND_RBF, float(info["sigma"]))
    supr = _bf16(sup).astype(np.float64)
    for j in range(C):
        if n[j]:
            Sj = supr[lab_s == j]
            want = ker(Sj, Sj).sum() / (n[j] * n[j])
            assert abs(gh[j] - want) <= 1e-3 * want, (j, gh[j], want)
    # assign against the resident support (FP32 kernel values; the model's g_hat)
    Xn, _ = mnist_like(2000, D, problem=9)
    la, da = lib.kkm_assign(model, _dev(Xn), mode="supports")
    model_d = O.assign_distances({"kernel": ker, "C": C, "support_coords": sup.astype(np.float64),
                                  "support_labels": lab_s, "ghat": gh}, Xn)
    assert_labels(la.cpu().numpy(), np.argmin(model_d, axis=1), model_d, "full-size assign labels")
    best = model_d[np.arange(2000), la.cpu().numpy()]
    ok = rel_margin(model_d) > 1e-4
    assert np.max(np.abs(da.cpu().numpy()[ok] - best[ok]) / (1.0 + gh.max())) <= DIST_REL


# ------------------------------------------- the benchmark's BF16 path at full size
# Expected values written by tests/golden/make_mnist_minibatch.py (the FP64
# oracle on the same seeded data).
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
U16 = 2.0 ** -11   # unit roundoff of the FP16-stored kernel block


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        g = json.load(f)
    g["u"] = np.frombuffer(g["u"].encode(), np.uint8).astype(np.int64) - ord("0")
    g["clear"] = np.unpackbits(np.frombuffer(bytes.fromhex(g["clear"]), np.uint8))[:g["Ni"]].astype(bool)
    return g


def test_bf16_step_full_minibatch(lib, mnist):
    """One teacher-forced inner iteration on the benchmark's path (BF16
    tensor-core block stored in FP16, FP32 near-tie re-score) on the first
    mini-batch, 15,000 x 3,000, labels = the generator's classes.
      f_hat (before the re-score) of 288 sampled rows and g_hat of every
        cluster against the oracle on the BF16-rounded rows, within the FP16
        storage rounding (2^-11 relative) plus the FP32 kernel tolerance;
      the new labels of every row against the oracle on the unrounded rows,
        wherever its relative margin exceeds 1e-4 (rows inside the re-score
        window are decided from FP32 kernel values);
      Omega against the unrounded oracle within the BF16 path's 5e-3."""
    X, Xd, sigma, cls = mnist
    g = _golden("mnist_step.json")
    assert g["sigma"] == sigma
    gidx, L = _plan(0)
    assert (g["Ni"], g["nL"], g["landmarks_sum"]) == (len(gidx), len(L), int(L.sum()))
    Xb = X[gidx]
    u = cls[gidx].astype(np.int32)
    got = lib.kkm_debug_step(Xb, L, u, C, "rbf", sigma, precision=lib.KKM_BF16, iteration="split")
    fused = lib.kkm_debug_step(Xb, L, u, C, "rbf", sigma, precision=lib.KKM_BF16, iteration="fused")
    for key in ("u", "n"):
        assert np.array_equal(fused[key], got[key]), key
    assert abs(fused["omega"] - got["omega"]) <= 1e-6 * got["omega"]
    # the tensor-core loop the benchmark times (same block, f_hat summed on the
    # tensor cores in another order): the oracle's labels wherever its margin
    # is clear, the counts exactly, Omega and f_hat as the split form's
    tc = lib.kkm_debug_step(Xb, L, u, C, "rbf", sigma, precision=lib.KKM_BF16, iteration="tc")
    assert np.array_equal(tc["n"], got["n"])
    bad_tc = np.nonzero((tc["u"] != g["u"]) & g["clear"])[0]
    assert bad_tc.size == 0, f"{bad_tc.size} clear rows differ from the oracle (tensor-core loop)"
    assert abs(tc["omega"] - got["omega"]) <= 1e-6 * got["omega"]
    live_n = got["n"] > 0
    assert float(np.max(np.abs(tc["fhat"][:, live_n] - got["fhat"][:, live_n]))) <= 2e-6
    assert np.array_equal(got["n"], g["n"])
    bad = np.nonzero((got["u"] != g["u"]) & g["clear"])[0]
    assert bad.size == 0, f"{bad.size} clear rows differ from the oracle, first {bad[:10]}"
    om_rel = abs(got["omega"] - g["omega"]) / g["omega"]
    print(f"BF16 step: Omega rel error vs unrounded oracle {om_rel:.3g}; "
          f"{np.count_nonzero(~g['clear'])} rows inside the 1e-4 margin")
    assert om_rel <= 5e-3
    # f_hat and g_hat of the stored block against the oracle on the rounded rows
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([rng.integers(0, len(gidx), 256), L[rng.integers(0, len(L), 32)]]))
    ker = O.Kernel(O.KIND_RBF, float(sigma))
    n, fhat, ghat, _ = _oracle_rows(ker, _bf16(Xb).astype(np.float64), L, u.astype(np.int64), C, rows)
    live = n > 0
    fd = np.abs(got["fhat"][rows][:, live] - fhat[:, live])
    assert np.all(fd <= U16 * np.abs(fhat[:, live]) + KERNEL_ABS), float(np.max(fd))
    gd = np.abs(got["ghat"][live] - ghat[live])
    assert np.all(gd <= U16 * ghat[live] + KERNEL_ABS), gd
    print(f"BF16 step: max |f_hat - oracle(rounded)| {np.max(fd):.3g}, max |g_hat - oracle(rounded)| "
          f"{np.max(gd):.3g}, max |g_hat - oracle(unrounded)| "
          f"{np.max(np.abs(got['ghat'][live] - np.asarray(g['ghat'])[live])):.3g}")


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_minibatch_fit_vs_oracle_full_size(lib, mnist, precision):
    """The first mini-batch of the benchmark workload fitted on its own
    (15,000 x 784, B = 1, |L| = 3,000, 30 iterations, early stop off, the
    oracle's k-means++ medoids as the initial ones) against the oracle's whole
    fit: labels equal wherever the oracle's last-iteration margin exceeds 1e-4
    relative, the Omega trace within 1e-6 (FP32) or the BF16 path's 5e-3,
    the landmark counts n_j exactly, g_hat within the same relative bound."""
    X, _, sigma, _ = mnist
    g = _golden("mnist_fit.json")
    assert g["sigma"] == sigma
    gidx, _ = _plan(0)
    Xb = X[gidx]
    prec = lib.KKM_BF16 if precision == "bf16" else lib.KKM_FP32
    rel = 5e-3 if precision == "bf16" else 1e-6
    lab, model = lib.kkm_fit(_dev(Xb), C, 1, S, "rbf", sigma, iters=g["iters"], seed=g["seed"], early_stop=False,
                             init_medoids=g["init_medoids"], precision=prec)
    lab = lab.cpu().numpy()
    bad = np.nonzero((lab != g["u"]) & g["clear"])[0]
    assert bad.size == 0, f"{bad.size} clear rows differ from the oracle, first {bad[:10]}"
    om, _ = model.trace()
    want = np.asarray(g["trace"])
    assert om.shape == want.shape
    err = float(np.max(np.abs(om - want) / want))
    print(f"{precision} fit: Omega trace max rel error {err:.3g}; "
          f"{np.count_nonzero(~g['clear'])} rows inside the 1e-4 margin")
    assert err <= rel
    _, gh, n = model.supports()
    assert np.array_equal(n, g["n"])
    live = n > 0
    assert np.all(np.abs(gh[live] - np.asarray(g["ghat"])[live]) <= rel * np.asarray(g["ghat"])[live])
    idx, cnt, _ = model.medoids()
    assert np.all(np.abs(cnt - np.asarray(g["W"])) <= np.count_nonzero(~g["clear"]))
    if precision == "fp32":
        assert np.array_equal(idx, g["medoids"])


@pytest.fixture(scope="module")
def md_batch(lib):
    F, state = md_trajectory(25000, 300, dwell=100.0, workload=2, problem=5)
    Xf = F.reshape(25000, -1)
    L = O.landmark_indices(25000, 0.05, O.SplitMix64(3)).astype(np.int32)
    return Xf, L, state


def test_rmsd_block_full_minibatch(lib, md_batch):
    """K(L, X^i) for the MD mini-batch (1,250 x 25,000 pairs of 300-atom frames)
    against the oracle (Horn + LAPACK) on 1,500 sampled entries."""
    Xf, L, _ = md_batch
    K = lib.kkm_kernel_matrix(_dev(Xf[L]), _dev(Xf), "rmsd", 1.5, n_atoms=300)
    rng = np.random.default_rng(4)
    a, b = _pairs(rng, len(L), Xf.shape[0], 1500)
    got = K[_dev(a.astype(np.int64)), _dev(b.astype(np.int64))].cpu().numpy()
    A = Xf[L][a].reshape(-1, 300, 3).astype(np.float64)
    Bf = Xf[b].reshape(-1, 300, 3).astype(np.float64)
    r2 = np.array([O.rmsd2(A[q:q + 1], Bf[q:q + 1])[0, 0] for q in range(len(a))])
    want = np.exp(-r2 / (2.0 * 1.5 ** 2))
    assert np.max(np.abs(got - want)) <= KERNEL_ABS
    assert np.mean(want > 1e-4) > 0.05   # the sample holds near pairs too


def test_rmsd_step_full_minibatch(lib, md_batch):
    """One teacher-forced inner iteration on the MD mini-batch (C = 8, labels =
    the generator's states): 96 sampled rows and every cluster's g_hat
    against the oracle."""
    Xf, L, state = md_batch
    kern = O.Kernel(O.KIND_RMSD, 1.5, 300)
    u = state.astype(np.int32)
    got = lib.kkm_debug_step(Xf, L, u, 8, "rmsd", 1.5, 300)
    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([rng.integers(0, Xf.shape[0], 80), L[rng.integers(0, len(L), 16)]]))
    n, fhat, ghat, d = _oracle_rows(kern, Xf.astype(np.float64), L, u.astype(np.int64), 8, rows)
    assert np.array_equal(got["n"], n)
    live = n > 0
    scale = 1.0 + np.where(live, ghat, 0.0)[None, :]
    assert np.all(np.abs(got["ghat"][live] - ghat[live]) <= DIST_REL * (1.0 + ghat[live]))
    fd = np.abs(got["fhat"][rows][:, live] - fhat[:, live])
    assert np.max(2 * fd / scale[:, live]) <= DIST_REL
    assert_labels(got["u"][rows], np.argmin(d, axis=1), d, "MD full-size step labels")
