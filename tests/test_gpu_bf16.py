"""The BF16 tensor-core (tcgen05) kernel block against the FP64 oracle.

The tensor-core path evaluates the kernel of the BF16-rounded rows with FP32
accumulation, so it is compared element by element with the oracle's kernel
of the same rounded rows (1e-5, as the FP32 path); its distance from the
oracle on the unrounded rows is the precision cost and is bounded loosely.
"""

import numpy as np
import pytest

from oracle import kkm_oracle as O
from synth import blobs, mnist_like
from tests.helpers import KERNEL_ABS

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _bf16_round(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


@pytest.mark.parametrize("nA,nB,d", [(300, 517, 37), (256, 128, 64), (129, 1029, 784), (1000, 3000, 784),
                                     (33, 64, 8), (3, 1, 16)])
def test_kernel_matrix_bf16_rbf(lib, nA, nB, d):
    X, _ = blobs(nA + nB, d, 4, workload=70, problem=d)
    A, Bm = X[:nA], X[nA:]
    sig = float(np.float32(O.median_bandwidth(X.astype(np.float64), O.Kernel(O.KIND_RBF, 0.0),
                                              O.SplitMix64(1), 300)))
    got = lib.kkm_kernel_matrix(_dev(A), _dev(Bm), "rbf", sig, precision=lib.KKM_BF16).cpu().numpy()
    ker = O.Kernel(O.KIND_RBF, sig)
    want_rounded = ker(_bf16_round(A), _bf16_round(Bm))
    assert np.max(np.abs(got - want_rounded)) <= KERNEL_ABS
    assert np.max(np.abs(got - ker(A, Bm))) <= 2e-2


def test_kernel_matrix_bf16_linear_and_quantised_rows(lib):
    X, _ = mnist_like(600, 784, problem=3)
    A, Bm = X[:200], X[200:]
    got = lib.kkm_kernel_matrix(_dev(A), _dev(Bm), "linear", precision=lib.KKM_BF16).cpu().numpy()
    want = _bf16_round(A).astype(np.float64) @ _bf16_round(Bm).astype(np.float64).T
    scale = np.linalg.norm(A, axis=1)[:, None] * np.linalg.norm(Bm, axis=1)[None, :]
    assert np.max(np.abs(got - want) / scale) <= 1e-5


def test_kernel_matrix_bf16_diagonal_is_one(lib):
    X, _ = blobs(700, 50, 3, workload=71)
    got = lib.kkm_kernel_matrix(_dev(X), _dev(X), "rbf", 5.0, precision=lib.KKM_BF16).cpu().numpy()
    assert np.all(np.abs(np.diag(got) - 1.0) <= 1e-5)


def test_kernel_matrix_bf16_rejects_rmsd(lib):
    X = np.zeros((4, 9), np.float32)
    with pytest.raises(lib.KKMError):
        lib.kkm_kernel_matrix(X, X, "rmsd", 1.5, n_atoms=3, precision=lib.KKM_BF16)


# ---------------------------------------------------------------- BF16 fits
def _fit_bf16(lib, X, C, B, s, iters, seed, sig, kind="rbf"):
    okind = O.KIND_RBF if kind == "rbf" else O.KIND_LINEAR
    ref = O.fit(X.astype(np.float64), C, B, s, O.Kernel(okind, sig), iters, seed, early_stop=False)
    init = ref["details"][0]["M_before"]
    lab, model = lib.kkm_fit(_dev(X), C, B, s, kind, sig, iters=iters, seed=seed, early_stop=False,
                             init_medoids=init, precision=lib.KKM_BF16)
    return lab.cpu().numpy(), model, ref


def _check_bf16_fit(lab, model, ref, omega_rel=5e-3):
    """Labels must equal the oracle's above the margin (the near-tie re-score
    settles the rest in FP32); Omega carries the BF16 error of the distances,
    which is reported and bounded loosely (d = K_ii - 2 f + g cancels, so a
    ~5e-5 absolute error is ~2e-3 of an Omega built from d ~ 0.03)."""
    from tests.helpers import assert_labels
    om, _ = model.trace()
    want = np.array([t[2] for t in ref["trace"]])
    assert om.shape == want.shape
    for det in ref["details"]:
        assert_labels(lab[det["gidx"]], det["u"], det["steps"][-1]["d"], "bf16 fit labels")
    rel = float(np.max(np.abs(om - want) / np.abs(want)))
    print(f"BF16 Omega max rel error vs oracle: {rel:.3g}")
    assert rel <= omega_rel


def test_fit_bf16_exact_kernel_kmeans_2000x16(lib):
    X, _ = blobs(2000, 16, 5, workload=0)
    sig = float(np.float32(O.median_bandwidth(X.astype(np.float64), O.Kernel(O.KIND_RBF, 0.0),
                                              O.SplitMix64(99), 512)))
    _check_bf16_fit(*_fit_bf16(lib, X, 5, 1, 1.0, 20, 1, sig))


def test_fit_bf16_mnist_shaped(lib):
    X, _ = mnist_like(6000, 784, problem=5)
    sig = float(np.float32(O.median_bandwidth(X.astype(np.float64), O.Kernel(O.KIND_RBF, 0.0),
                                              O.SplitMix64(7), 512)))
    _check_bf16_fit(*_fit_bf16(lib, X, 10, 2, 0.2, 12, 3, sig))


def test_fit_bf16_matches_fp32_path(lib):
    X, _ = mnist_like(8000, 784, problem=6)
    Xd = _dev(X)
    l32, m32 = lib.kkm_fit(Xd, 10, 2, 0.25, "rbf", 0.0, iters=10, seed=4, early_stop=False)
    l16, m16 = lib.kkm_fit(Xd, 10, 2, 0.25, "rbf", 0.0, iters=10, seed=4, early_stop=False,
                           precision=lib.KKM_BF16)
    agree = float(np.mean(l32.cpu().numpy() == l16.cpu().numpy()))
    assert agree >= 0.999, agree
    o32, _ = m32.trace()
    o16, _ = m16.trace()
    assert np.max(np.abs(o32 - o16) / np.abs(o32)) <= 5e-3
