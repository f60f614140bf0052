"""kkm_assign_noalloc: labelling without device allocation.

Some callers cannot allocate device memory while they serve a request (an
allocation can synchronise the device, or the memory belongs to another
framework's pool).  For them kkm_assign_noalloc works in a fixed scratch area
inside the library.  Its results must equal kkm_assign's, call after call,
although every call reuses the same scratch.  This file is collected last so
that a run stopping at its first failure has run every other test before.
"""

import numpy as np
import pytest

from synth import blobs, md_trajectory

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _compare(lib, model, queries, mode):
    import torch
    for Xq in queries:  # two calls in a row through the same scratch
        Xd = _dev(Xq)
        lab = torch.empty(len(Xq), dtype=torch.int32, device="cuda:0")
        dist = torch.empty(len(Xq), dtype=torch.float32, device="cuda:0")
        lib.kkm_assign_noalloc(model, Xd, lab, dist, mode)
        ref_lab, ref_dist = lib.kkm_assign(model, Xd, mode)
        torch.cuda.synchronize()
        assert torch.equal(lab, ref_lab)
        assert torch.max(torch.abs(dist - ref_dist)).item() <= 1e-5 * (1.0 + torch.max(torch.abs(ref_dist)).item())


@pytest.mark.parametrize("mode", ["supports", "medoids"])
def test_noalloc_matches_assign_rbf(lib, mode):
    X, _ = blobs(4000, 24, 6, workload=80)
    _, model = lib.kkm_fit(_dev(X), 6, 2, 0.3, "rbf", 0.0, iters=8, seed=2)
    q1, _ = blobs(1000, 24, 6, workload=80, problem=1)
    q2, _ = blobs(777, 24, 6, workload=80, problem=2)
    _compare(lib, model, [q1, q2], mode)


def test_noalloc_matches_assign_rmsd(lib):
    F, _ = md_trajectory(n_frames=1600, n_atoms=40, n_states=3, dwell=80.0, workload=81)
    _, model = lib.kkm_fit(_dev(F.reshape(1600, -1)), 3, 2, 0.25, "rmsd", 1.5, n_atoms=40, iters=6, seed=1)
    Fq, _ = md_trajectory(n_frames=600, n_atoms=40, n_states=3, dwell=80.0, workload=81, problem=1)
    Xq = Fq.reshape(600, -1)
    _compare(lib, model, [Xq[:300], Xq[300:]], "supports")


def test_noalloc_rejects_oversized_input(lib):
    import torch
    X, _ = blobs(2000, 8, 3, workload=82)
    _, model = lib.kkm_fit(_dev(X), 3, 1, 0.5, "rbf", 0.0, iters=4, seed=1)
    n = 1025  # one row more than KKM_NOALLOC_MAX_ROWS
    Xq = _dev(np.zeros((n, 8), np.float32))
    lab = torch.empty(n, dtype=torch.int32, device="cuda:0")
    with pytest.raises(lib.KKMError) as e:
        lib.kkm_assign_noalloc(model, Xq, lab)
    assert e.value.status == lib.STATUS_EINVAL
    assert "KKM_NOALLOC_MAX_ROWS" in str(e.value)
