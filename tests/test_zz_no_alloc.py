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

from tests.helpers import clear_rows
from oracle import kkm_oracle as O
from synth import blobs, md_trajectory

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _compare(lib, model, queries, mode, margin_of=None):
    """Two calls in a row through the same scratch, each against kkm_assign.
    margin_of(Xq) (optional) gives per-row distances whose relative margin
    decides which labels must be equal; without it every label must be."""
    import torch
    for Xq in queries:
        Xd = _dev(Xq)
        lab = torch.empty(len(Xq), dtype=torch.int32, device="cuda:0")
        dist = torch.empty(len(Xq), dtype=torch.float32, device="cuda:0")
        lib.kkm_assign_noalloc(model, Xd, lab, dist, mode)
        ref_lab, ref_dist = lib.kkm_assign(model, Xd, mode)
        torch.cuda.synchronize()
        if margin_of is None:
            assert torch.equal(lab, ref_lab)
        else:
            clear = torch.from_numpy(clear_rows(margin_of(Xq))).to("cuda:0")
            assert torch.equal(lab[clear], ref_lab[clear])
        assert torch.max(torch.abs(dist - ref_dist)).item() <= 1e-5 * (1.0 + torch.max(torch.abs(ref_dist)).item())


@pytest.mark.parametrize("mode", ["supports", "medoids"])
def test_noalloc_matches_assign_rbf(lib, mode):
    X, _ = blobs(4000, 24, 6, workload=80)
    _, model = lib.kkm_fit(_dev(X), 6, 2, 0.3, "rbf", 0.0, iters=8, seed=2)
    q1, _ = blobs(1000, 24, 6, workload=80, problem=1)
    q2, _ = blobs(777, 24, 6, workload=80, problem=2)
    _compare(lib, model, [q1, q2], mode)


def test_noalloc_matches_assign_rmsd(lib):
    # kkm_assign screens this model's pairs on the tensor cores (200 supports,
    # sigma 1.5) while the allocation-free call evaluates every pair exactly:
    # labels must agree above the 1e-4 relative margin, which the oracle
    # measures on the model's own supports
    n_frames, n_atoms, C, B, s, seed = 1600, 40, 3, 2, 0.25, 1
    F, _ = md_trajectory(n_frames=n_frames, n_atoms=n_atoms, n_states=3, dwell=80.0, workload=81)
    X = F.reshape(n_frames, -1)
    _, model = lib.kkm_fit(_dev(X), C, B, s, "rmsd", 1.5, n_atoms=n_atoms, iters=6, seed=seed)
    gidx, L = lib.kkm_minibatch_plan(n_frames, B, s, seed, B - 1)
    sup_lab, ghat, _ = model.supports()
    ref = {"kernel": O.Kernel(O.KIND_RMSD, 1.5, n_atoms), "C": C,
           "support_coords": X[gidx[L]].astype(np.float64), "support_labels": sup_lab.astype(np.int64),
           "ghat": ghat}
    Fq, _ = md_trajectory(n_frames=600, n_atoms=n_atoms, n_states=3, dwell=80.0, workload=81, problem=1)
    Xq = Fq.reshape(600, -1)
    _compare(lib, model, [Xq[:300], Xq[300:]], "supports",
             margin_of=lambda q: O.assign_distances(ref, q, "supports"))


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
