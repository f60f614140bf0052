"""Model selection and diagnostics against the oracle: restarts that keep
the minimum Eq. 1 cost (Section 4.5), the elbow over a range of C (Sections
4.4, 4.5) and the per-mini-batch centre displacement (Section 4.1, Fig. 4b).

Tolerances: costs are Eq. 1 sums, compared at the Omega tolerance (1e-6
relative); a displacement is the mean of sqrt(K(a,a) - 2K(a,b) + K(b,b)),
whose kernel values carry at most 1e-5 absolute error, so it may differ by
sqrt(2 * 2e-5) per cluster at worst (0 exactly when a medoid does not move).
"""

import numpy as np
import pytest

from oracle import kkm_oracle as O
from synth import blobs, md_trajectory
from tests.helpers import KERNEL_ABS, OMEGA_REL, assert_labels

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _sigma(X):
    k = O.Kernel(O.KIND_RBF, 0.0)
    return float(np.float32(O.median_bandwidth(X.astype(np.float64), k, O.SplitMix64(77), 512)))


DISP_TOL = np.sqrt(4.0 * KERNEL_ABS)


@pytest.mark.parametrize("kind,B,sampling", [("rbf", 4, "stride"), ("rbf", 3, "block"), ("linear", 2, "stride")])
def test_displacement_matches_oracle(lib, kind, B, sampling):
    X, _ = blobs(2400, 6, 5, workload=95, problem=B)
    sig = _sigma(X) if kind == "rbf" else 0.0
    okind = O.KIND_RBF if kind == "rbf" else O.KIND_LINEAR
    ref = O.fit(X.astype(np.float64), 5, B, 0.4, O.Kernel(okind, sig), 8, 3, sampling=sampling)
    init = ref["details"][0]["M_before"]
    _, model = lib.kkm_fit(_dev(X), 5, B, 0.4, kind, sig, iters=8, seed=3, init_medoids=init, sampling=sampling)
    assert np.array_equal(model.medoids()[0], ref["medoids"])
    got = model.displacement()
    want = np.array(O.displacement_trace(ref, X))
    assert got.shape == (B,)
    tol = DISP_TOL if kind == "rbf" else 1e-5 * (1.0 + np.abs(want))
    assert np.all(np.abs(got - want) <= tol), (got, want)
    assert np.all((want == 0.0) == (got == 0.0))


def test_displacement_saved_with_the_model(lib, tmp_path):
    X, _ = blobs(1500, 4, 3, workload=96)
    _, model = lib.kkm_fit(_dev(X), 3, 3, 0.5, "rbf", _sigma(X), iters=5, seed=2)
    path = str(tmp_path / "m.kkm")
    model.save(path)
    again = lib.Model.load(path)
    assert np.array_equal(again.displacement(), model.displacement())


def test_restarts_keep_the_minimum_cost(lib):
    X, _ = blobs(1800, 6, 7, workload=97)
    sig = _sigma(X)
    C, B, s, iters, seed, R = 7, 2, 0.5, 10, 11, 5
    ref = O.fit_restarts(X.astype(np.float64), C, B, s, O.Kernel(O.KIND_RBF, sig), iters, O.restart_seeds(seed, R))
    lab, model, costs, best = lib.kkm_fit_restarts(_dev(X), C, B, s, "rbf", sig, iters=iters, seed=seed,
                                                   n_restarts=R)
    assert np.all(np.abs(costs - ref["costs"]) <= OMEGA_REL * ref["costs"])
    # the same winner, unless two restarts tie within the tolerance
    near = np.abs(ref["costs"] - ref["costs"].min()) <= 2 * OMEGA_REL * ref["costs"].min()
    assert near[best] and (best == ref["best"] or near.sum() > 1)
    bf = ref["fits"][best]
    assert np.array_equal(model.medoids()[0], bf["medoids"])
    lab = lab.cpu().numpy()
    for det in bf["details"]:
        assert_labels(lab[det["gidx"]], det["u"], det["steps"][-1]["d"], "restart labels")
    assert len(set(O.restart_seeds(seed, R))) == R and len(set(np.round(costs, 6))) > 1


def test_restarts_share_the_median_bandwidth(lib):
    """sigma <= 0: one median rule (the bandwidth stream of `seed`) for every
    restart; a restart's cost then equals the oracle's with that bandwidth."""
    X, _ = blobs(1200, 5, 4, workload=98)
    seed, R = 21, 3
    _, bw, _ = O.rng_streams(seed, 1)
    sig = float(np.float32(O.median_bandwidth(X.astype(np.float64), O.Kernel(O.KIND_RBF, 0.0), bw)))
    ref = O.fit_restarts(X.astype(np.float64), 4, 1, 0.5, O.Kernel(O.KIND_RBF, sig), 8, O.restart_seeds(seed, R))
    _, model, costs, best = lib.kkm_fit_restarts(_dev(X), 4, 1, 0.5, "rbf", 0.0, iters=8, seed=seed, n_restarts=R)
    assert abs(model.info()["sigma"] - sig) <= 1e-6 * sig
    assert np.all(np.abs(costs - ref["costs"]) <= OMEGA_REL * ref["costs"])


def test_restarts_rmsd_host_input(lib):
    F, _ = md_trajectory(n_frames=900, n_atoms=30, n_states=3, dwell=50.0, workload=99)
    X = F.reshape(900, -1)
    ker = O.Kernel(O.KIND_RMSD, 1.5, 30)
    ref = O.fit_restarts(X.astype(np.float64), 3, 1, 0.3, ker, 6, O.restart_seeds(4, 3))
    lab, _, costs, best = lib.kkm_fit_restarts(X, 3, 1, 0.3, "rmsd", 1.5, n_atoms=30, iters=6, seed=4, n_restarts=3)
    assert isinstance(lab, np.ndarray) and lab.shape == (900,)
    assert np.all(np.abs(costs - ref["costs"]) <= 1e-5 * ref["costs"])


def test_elbow_matches_oracle(lib):
    g = np.random.Generator(np.random.PCG64(41))
    centres = g.uniform(-30, 30, size=(5, 3))
    X = (centres[np.arange(1500) % 5] + g.normal(0, 1.0, size=(1500, 3))).astype(np.float32)
    sig = 6.0
    ref = O.elbow(X.astype(np.float64), 2, 9, 1, 0.5, O.Kernel(O.KIND_RBF, sig), 10, seed=8, n_restarts=2)
    costs, C = lib.kkm_elbow(_dev(X), 2, 9, 1, 0.5, "rbf", sig, iters=10, seed=8, n_restarts=2)
    assert np.all(np.abs(costs - ref["costs"]) <= OMEGA_REL * ref["costs"])
    assert C == ref["C"] == 5


def test_selection_rejects_bad_arguments(lib):
    X, _ = blobs(300, 3, 3, workload=100)
    with pytest.raises(lib.KKMError):
        lib.kkm_fit_restarts(_dev(X), 3, 1, 0.5, "rbf", 1.0, n_restarts=0)
    with pytest.raises(lib.KKMError):
        lib.kkm_elbow(_dev(X), 4, 4, 1, 0.5, "rbf", 1.0)
    with pytest.raises(lib.KKMError):
        lib.kkm_elbow(_dev(X), 2, 300, 1, 0.5, "rbf", 1.0)
