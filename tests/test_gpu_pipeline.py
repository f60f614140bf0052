"""The block pipeline of kkm_fit (Section 4, Fig. 3): the next mini-batch's
kernel block computed on a second stream while the current one iterates.

Overlapped and serial scheduling run the same kernels on the same inputs, so
every output must be the same bits: labels, the Omega and #changed traces,
medoids and counts, and the resident supports with their g_hat.  The cases
cover each block kernel (FP32 Gram, BF16 tensor-core Gram with FP16 storage,
the FP32 short-row block stored in FP16, the MD tensor-core screen with its
exact pass, the plain MD kernel, linear), both samplings, uneven mini-batch
sizes, no inner iterations, and early stop.  The overlapped fits are also
compared with the oracle in the parity tests, which run with the default
(overlapped for B >= 2) scheduling.
"""

import numpy as np
import pytest

from synth import blobs, md_trajectory

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _np(t):
    return t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)


def _same_fit(lib, X, C, B, s, kind, sig, n_atoms=0, **kw):
    outs = []
    for pipe in ("serial", "overlap"):
        lab, m = lib.kkm_fit(X, C, B, s, kind, sig, n_atoms, pipeline=pipe, **kw)
        outs.append((_np(lab), m))
    (la, ma), (lb, mb) = outs
    assert np.array_equal(la, lb)
    oa, ca = ma.trace()
    ob, cb = mb.trace()
    assert np.array_equal(oa, ob) and np.array_equal(ca, cb)
    for x, y in zip(ma.medoids(), mb.medoids()):
        assert np.array_equal(x, y)
    for x, y in zip(ma.supports(), mb.supports()):
        assert np.array_equal(x, y, equal_nan=True)
    return la, ma


@pytest.mark.parametrize("prec,d", [(0, 24), (1, 24), (1, 200)])
def test_pipeline_rbf_same_bits(lib, prec, d):
    X, _ = blobs(9001, d, 7, workload=70, problem=d)
    _same_fit(lib, _dev(X), 7, 4, 0.3, "rbf", 0.0, iters=9, seed=11, precision=prec, early_stop=False)


def test_pipeline_block_sampling_uneven_and_early_stop(lib):
    X, _ = blobs(5003, 16, 5, workload=71)
    _same_fit(lib, _dev(X), 5, 3, 0.25, "rbf", 0.0, iters=12, seed=2, sampling="block")
    _same_fit(lib, _dev(X), 5, 7, 0.5, "rbf", 0.0, iters=0, seed=3)


def test_pipeline_rmsd_tensor_core_block(lib):
    """|L| >= 32 takes the MD tensor-core screen plus the exact pass."""
    F, _ = md_trajectory(n_frames=6000, n_atoms=60, n_states=5, dwell=80.0, workload=72)
    X = F.reshape(6000, -1)
    _same_fit(lib, _dev(X), 5, 3, 0.1, "rmsd", 1.5, 60, iters=6, seed=4, early_stop=False)


def test_pipeline_rmsd_small_and_linear_host_input(lib):
    F, _ = md_trajectory(n_frames=600, n_atoms=30, n_states=3, dwell=40.0, workload=73)
    X = F.reshape(600, -1)
    _same_fit(lib, _dev(X), 3, 4, 0.1, "rmsd", 1.5, 30, iters=5, seed=5)  # |L| = 15: plain kernel
    Xl, _ = blobs(3000, 6, 4, workload=74)
    lab, _ = _same_fit(lib, Xl, 4, 2, 0.5, "linear", 0.0, iters=6, seed=6)  # host input and labels
    assert isinstance(lab, np.ndarray)


def test_pipeline_in_a_batch(lib):
    """kkm_fit_batch runs a problem that asks for the pipeline with its own
    two streams beside the other workers (AUTO means serial there): every
    result equals the serial solo fit."""
    probs = []
    for p in range(6):
        X, _ = blobs(2500 + 700 * p, 12, 4, workload=75, problem=p)
        probs.append(dict(X=X, C=4, B=2 + p % 3, s=0.3, iters=6, seed=p, precision=p % 2,
                          pipeline="overlap" if p % 2 == 0 else "auto"))
    res = lib.kkm_fit_batch(probs, n_streams=3)
    for p, (lab, m, st) in zip(probs, res):
        assert st == 0
        ls, ms = lib.kkm_fit(p["X"], p["C"], p["B"], p["s"], "rbf", 0.0, 0, p["iters"], p["seed"],
                             precision=p["precision"], pipeline="serial")
        assert np.array_equal(_np(lab), _np(ls))
        assert np.array_equal(m.trace()[0], ms.trace()[0])


def test_pipeline_streams_reused_across_fits(lib):
    """The pipeline's stream pairs are reused from fit to fit: many small
    overlapped fits in a row, each on fresh data, equal their serial fits."""
    for p in range(12):
        X, _ = blobs(1200 + 50 * p, 6, 3, workload=76, problem=p)
        lo, mo = lib.kkm_fit(_dev(X), 3, 3, 0.4, "rbf", 0.0, iters=4, seed=p, pipeline="overlap")
        ls, ms = lib.kkm_fit(_dev(X), 3, 3, 0.4, "rbf", 0.0, iters=4, seed=p, pipeline="serial")
        assert np.array_equal(_np(lo), _np(ls))
        assert np.array_equal(mo.trace()[0], ms.trace()[0])
