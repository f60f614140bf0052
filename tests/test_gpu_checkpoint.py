"""A fit stopped after any mini-batch and resumed from its checkpoint gives
what one uninterrupted fit gives, bit for bit: the labels of every row, the
global medoids and their counts (Eq. 11-13), the trace of Omega and of label
changes, the centre displacements (Fig. 4b) and the model's supports.  The
state carried between outer iterations of Algorithm 1 is exactly the global
medoids and counts; everything else is recomputed from the seed."""

import numpy as np
import pytest

from synth import blobs

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _same_model(a, b):
    ia, wa, ca = a.medoids()
    ib, wb, cb = b.medoids()
    assert np.array_equal(ia, ib) and np.array_equal(wa, wb) and np.array_equal(ca, cb)
    oa, ga = a.trace()
    ob, gb = b.trace()
    assert np.array_equal(oa, ob) and np.array_equal(ga, gb)
    assert np.array_equal(a.displacement(), b.displacement())
    la, ha, na = a.supports()
    lb, hb, nb = b.supports()
    assert np.array_equal(la, lb) and np.array_equal(ha, hb) and np.array_equal(na, nb)
    assert a.info() == b.info()


def _to_np(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)


@pytest.mark.parametrize("precision,sampling,pipeline,device_input,cuts", [
    ("fp32", "stride", "serial", True, [2, 3]),
    ("fp32", "block", "overlap", False, [1]),
    ("bf16", "stride", "overlap", True, [1, 2, 4]),
    ("bf16", "block", "auto", True, [3]),
])
def test_resumed_fit_equals_one_fit(lib, tmp_path, precision, sampling, pipeline, device_input, cuts):
    X, _ = blobs(7200, 24, 6, workload=120, problem=len(cuts))
    prec = {"fp32": lib.KKM_FP32, "bf16": lib.KKM_BF16}[precision]
    Xin = _dev(X) if device_input else X
    args = (Xin, 6, 6, 0.2, "rbf", 0.0)
    kw = dict(iters=15, seed=31, precision=prec, sampling=sampling)
    lab_whole, whole = lib.kkm_fit(*args, **kw, pipeline=pipeline)
    labels, ck = True, None
    bounds = cuts + [6]
    for q, stop in enumerate(bounds):
        last = q == len(bounds) - 1
        labels, model, ck_new = lib.kkm_fit_range(*args, **kw, stop=stop, checkpoint=ck, labels=labels,
                                                  model=last, pipeline=pipeline)
        assert ck_new.info()["next_batch"] == stop
        if not last:
            # through a file, as a resumed process would
            path = str(tmp_path / f"c{q}.ckpt")
            ck_new.save(path)
            ck = lib.Checkpoint.load(path)
            assert np.array_equal(ck.medoids(), ck_new.medoids())
    assert np.array_equal(_to_np(labels), _to_np(lab_whole))
    _same_model(model, whole)
    assert np.array_equal(ck_new.medoids(), whole.medoids()[0])


def test_checkpoint_after_the_first_mini_batch_holds_its_medoids(lib):
    """The checkpoint after mini-batch 0 holds the medoids a one-mini-batch
    prefix produces; the bandwidth in use (median rule) is kept, so that the
    resumed fit does not redraw it."""
    X, _ = blobs(3000, 8, 4, workload=121)
    Xd = _dev(X)
    _, _, ck = lib.kkm_fit_range(Xd, 4, 3, 0.3, "rbf", 0.0, iters=10, seed=5, stop=1)
    inf = ck.info()
    assert inf["next_batch"] == 1 and inf["B"] == 3 and inf["C"] == 4
    _, whole = lib.kkm_fit(Xd, 4, 3, 0.3, "rbf", 0.0, iters=10, seed=5)
    assert inf["sigma"] == whole.info()["sigma"]
    d = whole.displacement()
    labels, model, ck2 = lib.kkm_fit_range(Xd, 4, 3, 0.3, "rbf", 0.0, iters=10, seed=5, stop=3, checkpoint=ck,
                                           model=True)
    assert np.array_equal(model.displacement(), d)
    # rows of mini-batch 0 were not in this range: still -1
    lab = _to_np(labels)
    assert np.all(lab[0::3] == -1) and np.all(lab[1::3] >= 0) and np.all(lab[2::3] >= 0)


def test_resume_rejects_other_arguments(lib):
    X, _ = blobs(2000, 8, 3, workload=122)
    Xd = _dev(X)
    _, _, ck = lib.kkm_fit_range(Xd, 3, 4, 0.3, "rbf", 1.5, iters=5, seed=1, stop=2)
    for kw in (dict(seed=2), dict(iters=6), dict(sigma=1.0)):
        a = dict(kind="rbf", sigma=1.5, iters=5, seed=1)
        a.update(kw)
        with pytest.raises(lib.KKMError) as e:
            lib.kkm_fit_range(Xd, 3, 4, 0.3, checkpoint=ck, stop=4, **a)
        assert e.value.status == lib.STATUS_EINVAL
    with pytest.raises(lib.KKMError):
        lib.kkm_fit_range(Xd, 3, 5, 0.3, "rbf", 1.5, iters=5, seed=1, checkpoint=ck, stop=4)   # another B
