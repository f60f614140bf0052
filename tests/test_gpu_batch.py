"""Batched independent fits (kkm_fit_batch) on the GPU.

Each problem of a batch must give exactly what kkm_fit gives for it alone
with the split inner loop, the form fits take side by side (same kernels on
its own stream, fixed-order reductions), whatever runs beside it; a sample
of the problems is also checked against the FP64 oracle at the usual
tolerances.
"""

import math

import numpy as np
import pytest

from oracle import kkm_oracle as O
from synth import blobs
from tests.helpers import assert_labels, first_divergence

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _np(t):
    return t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)


def _small_problems(n, seed):
    """Uneven shapes in the style of the batched workload, scaled down so
    the oracle and the solo fits finish quickly."""
    g = np.random.default_rng(seed)
    out = []
    for p in range(n):
        N = int(round(math.exp(g.uniform(math.log(300), math.log(6000)))))
        d = int(g.choice([8, 32, 64, 128]))
        C = int(g.integers(2, 17))
        B = -(-N // 2500)
        s = float(g.choice([0.1, 0.5]))
        X, _ = blobs(N, d, C, workload=3, problem=100 + p)
        out.append(dict(X=X, C=C, B=B, s=s, iters=8, seed=int(g.integers(0, 2**31)),
                        precision=int(g.integers(0, 2)), early_stop=bool(g.integers(0, 2))))
    return out


def _same_model(a, b):
    la, ma = a
    lb, mb = b
    assert np.array_equal(_np(la), _np(lb))
    oa, ca = ma.trace()
    ob, cb = mb.trace()
    assert np.array_equal(oa, ob, equal_nan=True) and np.array_equal(ca, cb)
    ia, wa, xa = ma.medoids()
    ib, wb, xb = mb.medoids()
    assert np.array_equal(ia, ib) and np.array_equal(wa, wb) and np.array_equal(xa, xb)
    sa, ga, na = ma.supports()
    sb, gb, nb = mb.supports()
    assert np.array_equal(sa, sb) and np.array_equal(ga, gb, equal_nan=True) and np.array_equal(na, nb)


@pytest.mark.parametrize("n_streams", [1, 4, 12])
def test_batch_equals_solo_fits(lib, n_streams):
    probs = _small_problems(14, seed=5)
    dev = [dict(p, X=_dev(p["X"])) for p in probs]
    res = lib.kkm_fit_batch(dev, n_streams=n_streams)
    for p, (lab, model, status) in zip(dev, res):
        assert status == 0
        solo = lib.kkm_fit(p["X"], p["C"], p["B"], p["s"], "rbf", 0.0, 0, p["iters"], p["seed"],
                           precision=p["precision"], early_stop=p["early_stop"], iteration="split")
        _same_model((lab, model), solo)


@pytest.mark.parametrize("rows", [2, 4, 8])
def test_assign_rows_per_cta_change_nothing(lib, monkeypatch, rows):
    """The work-list assign takes 1, 2, 4 or 8 blocks of 32 rows per CTA (the
    row tuner's candidates, forced here): every result is bit-identical to
    one block per CTA, on problems with C below and above the 8-warp CTA, a
    ragged last block, early stop on and off, both block precisions."""
    probs = _small_problems(10, seed=11)
    probs.append(dict(X=blobs(3001, 8, 40, workload=3, problem=300)[0], C=40, B=2, s=0.5, iters=6, seed=3,
                      precision=1, early_stop=False))
    dev = [dict(p, X=_dev(p["X"])) for p in probs]
    monkeypatch.setenv("KKM_ASSIGN_ROWS", "1")
    ref = lib.kkm_fit_batch(dev, n_streams=6)
    monkeypatch.setenv("KKM_ASSIGN_ROWS", str(rows))
    got = lib.kkm_fit_batch(dev, n_streams=6)
    for (la, ma, sa), (lb, mb, sb) in zip(ref, got):
        assert sa == 0 and sb == 0
        _same_model((la, ma), (lb, mb))



@pytest.mark.parametrize("chains", [2, 3])
def test_loop_chains_change_nothing(lib, monkeypatch, chains):
    """KKM_LOOP_CHAINS runs the work lists as several chains side by side
    (each fit's loops on one chain): every result is bit-identical to one
    chain, with more chains than loops in flight at times and early stop on."""
    probs = _small_problems(9, seed=13)
    probs.append(dict(X=blobs(2500, 8, 20, workload=3, problem=304)[0], C=20, B=3, s=0.4, iters=5, seed=4,
                      precision=1, early_stop=True))
    dev = [dict(p, X=_dev(p["X"])) for p in probs]
    monkeypatch.setenv("KKM_LOOP_CHAINS", "1")
    ref = lib.kkm_fit_batch(dev, n_streams=5)
    monkeypatch.setenv("KKM_LOOP_CHAINS", str(chains))
    got = lib.kkm_fit_batch(dev, n_streams=5)
    for (la, ma, sa), (lb, mb, sb) in zip(ref, got):
        assert sa == 0 and sb == 0
        _same_model((la, ma), (lb, mb))

@pytest.mark.parametrize("rows", [2, 4, 8])
def test_assign_rows_per_cta_solo_split_fit(lib, monkeypatch, rows):
    """A fit's own assign launches (split loop, FP32 and the reduced-precision
    re-score, a linear-kernel fit) take the same rows-per-CTA candidates:
    bit-identical results."""
    cases = [(blobs(5003, 16, 6, workload=3, problem=301)[0], "rbf", 0, 6, 3),
             (blobs(3001, 32, 9, workload=3, problem=302)[0], "rbf", 1, 9, 2),
             (blobs(2000, 8, 4, workload=3, problem=303)[0], "linear", 0, 4, 2)]
    for X, kind, prec, C, B in cases:
        Xd = _dev(X)
        kw = dict(iters=6, seed=5, precision=prec, iteration="split", early_stop=False)
        monkeypatch.setenv("KKM_ASSIGN_ROWS", "1")
        ref = lib.kkm_fit(Xd, C, B, 0.3, kind, 0.0, **kw)
        monkeypatch.setenv("KKM_ASSIGN_ROWS", str(rows))
        got = lib.kkm_fit(Xd, C, B, 0.3, kind, 0.0, **kw)
        _same_model(ref, got)


def test_row_tuner_cache_file(lib, monkeypatch, tmp_path):
    """With KKM_TUNE_CACHE set, the choices the tuner settles on are written as
    'assign_rows <key> <rows>' lines, each a candidate."""
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("KKM_TUNE_CACHE", str(path))
    monkeypatch.delenv("KKM_ASSIGN_ROWS", raising=False)
    probs = [dict(p, X=_dev(p["X"])) for p in _small_problems(6, seed=12)]
    for _ in range(3):  # enough launches for every key seen to settle
        lib.kkm_fit_batch([dict(p, iters=20) for p in probs], n_streams=4)
    assert path.exists()
    lines = [ln.split() for ln in path.read_text().splitlines() if ln.strip()]
    assert lines and all(ln[0] == "assign_rows" and int(ln[2]) in (1, 2, 4, 8) for ln in lines)


def test_batch_against_oracle(lib):
    """FP32 problems of the batch against the oracle (labels above the margin,
    the Omega trace at 1e-6, medoids identical)."""
    probs = []
    for p, (N, d, C, B, s) in enumerate([(1500, 16, 4, 1, 1.0), (2600, 32, 6, 2, 0.3), (900, 8, 3, 1, 0.5)]):
        X, _ = blobs(N, d, C, workload=3, problem=200 + p)
        sig = float(np.float32(O.median_bandwidth(X.astype(np.float64), O.Kernel(O.KIND_RBF, 0.0),
                                                  O.SplitMix64(p), 512)))
        probs.append(dict(X=X, C=C, B=B, s=s, sigma=sig, iters=10, seed=40 + p, early_stop=False))
    refs = [O.fit(p["X"].astype(np.float64), p["C"], p["B"], p["s"], O.Kernel(O.KIND_RBF, p["sigma"]),
                  p["iters"], p["seed"], early_stop=False) for p in probs]
    dev = [dict(p, X=_dev(p["X"]), init_medoids=r["details"][0]["M_before"]) for p, r in zip(probs, refs)]
    res = lib.kkm_fit_batch(dev, n_streams=3)
    for (lab, model, status), ref in zip(res, refs):
        assert status == 0
        lab = _np(lab)
        om, _ = model.trace()
        want = np.array([t[2] for t in ref["trace"]])
        assert om.shape == want.shape
        assert first_divergence(om, want) is None
        for det in ref["details"]:
            assert_labels(lab[det["gidx"]], det["u"], det["steps"][-1]["d"], "batched fit labels")
        idx, cnt, _ = model.medoids()
        assert np.array_equal(idx, ref["medoids"]) and np.array_equal(cnt, ref["W"])


def test_batch_restarts_of_one_data_set(lib):
    """Restarts: one data set, several seeds, each equal to its solo fit."""
    X, _ = blobs(4000, 32, 8, workload=3, problem=300)
    Xd = _dev(X)
    probs = [dict(X=Xd, C=8, B=2, s=0.2, iters=10, seed=sd, precision=lib.KKM_BF16) for sd in range(6)]
    res = lib.kkm_fit_batch(probs, n_streams=6)
    for p, (lab, model, status) in zip(probs, res):
        assert status == 0
        _same_model((lab, model), lib.kkm_fit(Xd, 8, 2, 0.2, "rbf", 0.0, 0, 10, p["seed"],
                                             precision=lib.KKM_BF16, iteration="split"))


def test_batch_host_inputs_and_labels(lib):
    probs = _small_problems(4, seed=9)
    res = lib.kkm_fit_batch(probs, n_streams=2)
    for p, (lab, model, status) in zip(probs, res):
        assert status == 0 and isinstance(lab, np.ndarray)
        solo = lib.kkm_fit(_dev(p["X"]), p["C"], p["B"], p["s"], "rbf", 0.0, 0, p["iters"], p["seed"],
                           precision=p["precision"], early_stop=p["early_stop"], iteration="split")
        _same_model((lab, model), solo)


def test_batch_failed_problem_does_not_stop_others(lib):
    probs = _small_problems(3, seed=11)
    bad = dict(probs[1], C=probs[1]["X"].shape[0] + 1)   # C larger than the mini-batch
    batch = [probs[0], bad, probs[2]]
    res = lib.kkm_fit_batch(batch, n_streams=2, check=False)
    assert [r[2] for r in res] == [0, lib.STATUS_EINVAL, 0]
    assert res[1][1] is None and res[0][1] is not None and res[2][1] is not None
    with pytest.raises(lib.KKMError):
        lib.kkm_fit_batch(batch, n_streams=2)
