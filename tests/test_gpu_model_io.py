"""kkm_model_save / kkm_model_load: a loaded model answers every query and
labels new samples exactly as the saved one."""

import numpy as np
import pytest

from synth import blobs, md_trajectory

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y), equal_nan=True)


@pytest.mark.parametrize("kind", ["rbf", "rmsd", "linear"])
def test_save_load_roundtrip(lib, kind, tmp_path):
    if kind == "rmsd":
        F, _ = md_trajectory(3000, 40, workload=6, problem=1)
        X = F.reshape(3000, -1)
        lab, m = lib.kkm_fit(_dev(X), 5, 2, 0.2, "rmsd", 1.5, 40, iters=6, seed=2)
        Q = md_trajectory(500, 40, workload=6, problem=2)[0].reshape(500, -1)
    else:
        X, _ = blobs(3000, 24, 6, workload=6, problem=3)
        lab, m = lib.kkm_fit(_dev(X), 6, 2, 0.3, kind, 2.0 if kind == "rbf" else 0.0, iters=6, seed=2,
                             precision=lib.KKM_BF16 if kind == "rbf" else lib.KKM_FP32)
        Q = blobs(500, 24, 6, workload=6, problem=4)[0]
    path = tmp_path / f"{kind}.kkm"
    m.save(str(path))
    m2 = lib.Model.load(str(path))
    assert m.info() == m2.info()
    _same(m.medoids(), m2.medoids())
    _same(m.supports(), m2.supports())
    _same(m.trace(), m2.trace())
    for mode in ("supports", "medoids"):
        a = lib.kkm_assign(m, _dev(Q), mode=mode)
        b = lib.kkm_assign(m2, _dev(Q), mode=mode)
        _same([t.cpu().numpy() for t in a], [t.cpu().numpy() for t in b])
        assert lib.kkm_cost(m, _dev(Q), mode=mode) == lib.kkm_cost(m2, _dev(Q), mode=mode)
    # the loaded model can be saved again, byte for byte
    path2 = tmp_path / f"{kind}2.kkm"
    m2.save(str(path2))
    assert path.read_bytes() == path2.read_bytes()


def test_loaded_model_serves(lib, tmp_path):
    X, _ = blobs(2000, 16, 4, workload=6, problem=5)
    _, m = lib.kkm_fit(_dev(X), 4, 1, 0.5, "rbf", 0.0, iters=5, seed=1)
    m.save(str(tmp_path / "m.kkm"))
    Q = blobs(300, 16, 4, workload=6, problem=6)[0]
    want = lib.kkm_assign(m, _dev(Q))
    srv = lib.Server(budget_bytes=1 << 30, n_workers=2)
    mid = srv.add_model(lib.Model.load(str(tmp_path / "m.kkm")))
    st, (la, da), _, _ = srv.wait(srv.submit_assign(mid, Q))
    assert st == 0
    assert np.array_equal(la, want[0].cpu().numpy()) and np.array_equal(da, want[1].cpu().numpy())
    srv.close()
