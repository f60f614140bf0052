"""The tensor-core inner loop (KKM_ITER_TC) against the oracle and the split form.

The loop forms the f_hat numerators of Eq. 17 as the product of the
FP16-stored Gaussian block with the one-hot matrix of the landmark labels on
the tensor cores, one CTA per 128 samples, g_hat (Eq. 16) from the landmark
rows, grid barriers between the phases.  Its input is the reduced-precision
path's block, so it is checked
  - against the split form on the same block (the same values summed in
    another order): f_hat within 2e-6 absolute (means of values in [0, 1]),
    g_hat within 1e-6 relative, the same labels wherever the split step's
    relative margin exceeds 1e-5, Omega within 1e-6 relative;
  - against the oracle: labels above the 1e-4 relative margin, f_hat and
    g_hat within the FP16 storage rounding (2^-11 relative) plus the kernel
    tolerance.  Rows of at most 128 values get FP32 kernel values of the
    unrounded rows; longer rows the tensor-core kernel of the BF16-rounded
    rows, so the oracle sees the rounded rows there.
Shapes span several 128-sample tiles with a ragged last tile, landmark counts
that are not a multiple of the 64-landmark tile, an empty cluster, C = 16
(the largest the loop takes) and a single tile."""

import numpy as np
import pytest

from oracle import kkm_oracle as O
from synth import blobs, mnist_like
from tests.helpers import KERNEL_ABS, OMEGA_REL, assert_labels, rel_margin

pytestmark = pytest.mark.gpu

U16 = 2.0 ** -11


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _bf16(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def _sigma(X, seed=7):
    k = O.Kernel(O.KIND_RBF, 0.0)
    return float(np.float32(O.median_bandwidth(X.astype(np.float64), k, O.SplitMix64(seed), 512)))


def _case(Ni, nL, C, d, seed, empty=False):
    X, y = blobs(Ni, d, max(C, 2), workload=130, problem=seed)
    g = np.random.Generator(np.random.PCG64(seed))
    L = np.sort(g.choice(Ni, nL, replace=False)).astype(np.int32)
    u = np.where(g.random(Ni) < 0.7, y % C, g.integers(0, C, Ni)).astype(np.int32)
    if empty:  # the last cluster keeps members but loses its landmarks
        u[L] = np.where(u[L] == C - 1, 0, u[L])
    return X, L, u


def _check_step(lib, X, L, u, C):
    sig = _sigma(X)
    tc = lib.kkm_debug_step(X, L, u, C, "rbf", sig, precision=lib.KKM_BF16, iteration="tc")
    sp = lib.kkm_debug_step(X, L, u, C, "rbf", sig, precision=lib.KKM_BF16, iteration="split")
    # the split form on the same block
    assert np.array_equal(tc["n"], sp["n"])
    live = sp["n"] > 0
    assert np.all(np.isnan(tc["ghat"][~live]))
    assert np.allclose(tc["ghat"][live], sp["ghat"][live], rtol=1e-6, atol=0.0)
    fd = np.abs(tc["fhat"][:, live] - sp["fhat"][:, live])
    assert np.max(fd) <= 2e-6, float(np.max(fd))
    d_sp = np.where(live[None, :], 1.0 - 2.0 * sp["fhat"] + np.where(live, sp["ghat"], 0.0)[None, :], np.inf)
    sure = rel_margin(d_sp) > 1e-5
    assert np.array_equal(tc["u"][sure], sp["u"][sure])
    assert abs(tc["omega"] - sp["omega"]) <= OMEGA_REL * abs(sp["omega"])
    # the oracle on the rows the block was computed from
    Xo = X.astype(np.float64) if X.shape[1] <= 128 else _bf16(X).astype(np.float64)
    k = O.Kernel(O.KIND_RBF, sig)
    ref = O.inner_step(k(Xo, Xo[L]), k.self_terms(Xo), L.astype(np.int64), u.astype(np.int64), C)
    assert np.array_equal(tc["n"], ref["n"])
    fo = np.abs(tc["fhat"][:, live] - ref["fhat"][:, live])
    assert np.all(fo <= U16 * np.abs(ref["fhat"][:, live]) + KERNEL_ABS), float(np.max(fo))
    go = np.abs(tc["ghat"][live] - ref["ghat"][live])
    assert np.all(go <= U16 * ref["ghat"][live] + KERNEL_ABS), go
    assert_labels(tc["u"], ref["u"], ref["d"], "tensor-core step labels")
    return tc, ref


@pytest.mark.parametrize("Ni,nL,C,d", [(1037, 301, 7, 32), (2600, 650, 10, 200), (128, 64, 16, 16),
                                       (5000, 997, 12, 64), (700, 700, 3, 8), (131, 1, 2, 4)])
def test_tc_step_matches_split_and_oracle(lib, Ni, nL, C, d):
    X, L, u = _case(Ni, nL, C, d, seed=Ni + nL)
    _check_step(lib, X, L, u, C)


def test_tc_step_empty_cluster(lib):
    X, L, u = _case(900, 300, 4, 12, seed=3, empty=True)
    tc, ref = _check_step(lib, X, L, u, 4)
    assert ref["n"][3] == 0 and np.all(tc["u"] != 3)


def _fit(lib, X, C, B, s, iters, seed, sig, iteration, early_stop=False):
    ref = O.fit(X.astype(np.float64), C, B, s, O.Kernel(O.KIND_RBF, sig), iters, seed, early_stop=early_stop)
    init = ref["details"][0]["M_before"]
    lab, model = lib.kkm_fit(_dev(X), C, B, s, "rbf", sig, iters=iters, seed=seed, early_stop=early_stop,
                             init_medoids=init, precision=lib.KKM_BF16, iteration=iteration)
    return lab.cpu().numpy(), model, ref


def _check_fit(lab, model, ref, omega_rel=5e-3):
    om, _ = model.trace()
    want = np.array([t[2] for t in ref["trace"]])
    assert om.shape == want.shape
    for det in ref["details"]:
        assert_labels(lab[det["gidx"]], det["u"], det["steps"][-1]["d"], "tensor-core fit labels")
    assert float(np.max(np.abs(om - want) / np.abs(want))) <= omega_rel
    _, _, n = model.supports()
    assert np.array_equal(n, ref["n"])


@pytest.mark.parametrize("early_stop", [False, True])
def test_tc_fit_exact_kernel_kmeans(lib, early_stop):
    """B = 1, s = 1: every sample a landmark (2,000 landmarks, 32 one-hot tiles)."""
    X, _ = blobs(2000, 16, 5, workload=0)
    sig = _sigma(X, 99)
    _check_fit(*_fit(lib, X, 5, 1, 1.0, 20, 1, sig, "tc", early_stop=early_stop))


def test_tc_fit_mnist_shaped(lib):
    X, _ = mnist_like(6000, 784, problem=5)
    _check_fit(*_fit(lib, X, 10, 2, 0.2, 12, 3, _sigma(X), "tc"))


def test_tc_fit_matches_split(lib):
    """The same fit with either loop form: labels agree on at least 99.9 %
    (near ties may fall either way), the Omega traces within 1e-5."""
    X, _ = mnist_like(8000, 784, problem=6)
    Xd = _dev(X)
    runs = {it: lib.kkm_fit(Xd, 10, 2, 0.25, "rbf", 0.0, iters=10, seed=4, early_stop=False,
                            precision=lib.KKM_BF16, iteration=it) for it in ("tc", "split")}
    (lt, mt), (ls, ms) = runs["tc"], runs["split"]
    assert float(np.mean(lt.cpu().numpy() == ls.cpu().numpy())) >= 0.999
    ot, _ = mt.trace()
    os_, _ = ms.trace()
    assert ot.shape == os_.shape
    assert np.max(np.abs(ot - os_) / np.abs(os_)) <= 1e-5


def test_tc_fit_fp8_block(lib):
    """The loop on the FP8 path's block (also FP16-stored)."""
    X, _ = mnist_like(4000, 784, problem=8)
    Xd = _dev(X)
    lt, mt = lib.kkm_fit(Xd, 10, 2, 0.25, "rbf", 0.0, iters=8, seed=2, early_stop=False,
                         precision=lib.KKM_FP8, iteration="tc")
    ls, ms = lib.kkm_fit(Xd, 10, 2, 0.25, "rbf", 0.0, iters=8, seed=2, early_stop=False,
                         precision=lib.KKM_FP8, iteration="split")
    assert float(np.mean(lt.cpu().numpy() == ls.cpu().numpy())) >= 0.999
    ot, _ = mt.trace()
    os_, _ = ms.trace()
    assert np.max(np.abs(ot - os_) / np.abs(os_)) <= 1e-5


def test_tc_refuses_shapes_it_does_not_cover(lib):
    X, _ = blobs(3000, 8, 4, workload=131)
    Xd = _dev(X)
    with pytest.raises(lib.KKMError):   # more than 16 clusters
        lib.kkm_fit(Xd, 17, 1, 0.3, "rbf", 1.0, iters=2, precision=lib.KKM_BF16, iteration="tc")
    with pytest.raises(lib.KKMError):   # the FP32 block
        lib.kkm_fit(Xd, 4, 1, 0.3, "rbf", 1.0, iters=2, iteration="tc")
    with pytest.raises(lib.KKMError):   # the linear kernel
        lib.kkm_fit(Xd, 4, 1, 0.3, "linear", 0.0, iters=2, precision=lib.KKM_BF16, iteration="tc")
    big, _ = blobs(152 * 128 + 1, 4, 3, workload=132)
    with pytest.raises(lib.KKMError):   # more 128-sample tiles than SMs in one mini-batch
        lib.kkm_fit(_dev(big), 3, 1, 0.01, "rbf", 1.0, iters=2, precision=lib.KKM_BF16, iteration="tc")


@pytest.mark.parametrize("iters,B", [(1, 1), (2, 1), (1, 2), (2, 3)])
def test_tc_medoids_of_the_final_supports(lib, iters, B):
    """The tensor-core loop forms the Eq. 10 keys itself: from the f_hat of its
    last iteration when no landmark label moved there, else after one more
    pass with the patched supports (after one or two iterations from the
    k-means++ medoids, labels are still moving).  On separated blobs (no near
    ties) the medoids, counts, g_hat and n_j equal those of the split form,
    which streams the block once more for Eq. 10."""
    X, _ = blobs(4000, 16, 6, workload=133)
    Xd = _dev(X)
    runs = {it: lib.kkm_fit(Xd, 6, B, 0.3, "rbf", 0.0, iters=iters, seed=11, early_stop=False,
                            precision=lib.KKM_BF16, iteration=it) for it in ("tc", "split")}
    (lt, mt), (ls, ms) = runs["tc"], runs["split"]
    _, ch = ms.trace()
    assert np.any(ch[iters - 1::iters] > 0)  # labels still move in a last iteration
    assert np.array_equal(lt.cpu().numpy(), ls.cpu().numpy())
    it_, ct, _ = mt.medoids()
    is_, cs, _ = ms.medoids()
    assert np.array_equal(it_, is_) and np.array_equal(ct, cs)
    _, gt, nt = mt.supports()
    _, gs, ns = ms.supports()
    assert np.array_equal(nt, ns)
    live = ns > 0
    assert np.allclose(gt[live], gs[live], rtol=1e-6, atol=0.0)
