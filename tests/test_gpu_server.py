"""The serving loop (kkm_server) on the GPU.

A request's result must be the same alone and in the mix: each assign is
compared with kkm_assign on the same rows, each fit with kkm_fit on the same
arguments, bit for bit (the per-row computations do not depend on the other
rows of a fused launch, and a fit runs the same kernels on its own stream).
"""

import threading
import time

import numpy as np
import pytest

from synth import blobs, md_trajectory

pytestmark = pytest.mark.gpu

GB = 1 << 30


def _np(t):
    return t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)


@pytest.fixture(scope="module")
def models(lib):
    """One RMSD model (MD frames) and one RBF model, fitted alone."""
    import torch
    F, _ = md_trajectory(3000, 30, workload=4, problem=1)
    Xm = torch.from_numpy(F.reshape(3000, -1)).cuda()
    _, m_rmsd = lib.kkm_fit(Xm, 6, 2, 0.2, "rmsd", 1.5, 30, iters=8, seed=3)
    Xb, _ = blobs(4000, 32, 7, workload=4, problem=2)
    _, m_rbf = lib.kkm_fit(torch.from_numpy(Xb).cuda(), 7, 2, 0.25, "rbf", 0.0, iters=8, seed=5,
                           precision=lib.KKM_BF16)
    return m_rmsd, m_rbf


def _queries(n, seed):
    g = np.random.default_rng(seed)
    F, _ = md_trajectory(4000, 30, workload=4, problem=10 + seed)
    Xq = F.reshape(4000, -1)
    Xb, _ = blobs(4000, 32, 7, workload=4, problem=20 + seed)
    out = []
    for _ in range(n):
        M = int(np.exp(g.uniform(0.0, np.log(1500))))
        a = int(g.integers(0, 4000 - M))
        if g.random() < 0.5:
            out.append(("rmsd", Xq[a:a + M].copy(), str(g.choice(["supports", "medoids"]))))
        else:
            out.append(("rbf", Xb[a:a + M].copy(), str(g.choice(["supports", "medoids"]))))
    return out


def _fit_jobs(n, seed, lib):
    g = np.random.default_rng(seed)
    jobs = []
    for p in range(n):
        N = int(np.exp(g.uniform(np.log(800), np.log(6000))))
        d = int(g.choice([8, 32, 64]))
        C = int(g.integers(2, 12))
        X, _ = blobs(N, d, C, workload=4, problem=100 + p)
        jobs.append(dict(X=X, C=C, B=-(-N // 3000), s=float(g.choice([0.1, 0.5])), iters=6,
                         seed=int(g.integers(0, 1 << 30)), precision=int(g.integers(0, 2))))
    return jobs


def test_results_alone_and_in_the_mix(lib, models):
    import torch
    m_rmsd, m_rbf = models
    qs = _queries(40, seed=1)
    fits = _fit_jobs(6, seed=2, lib=lib)
    # alone
    alone_q = []
    for kind, X, mode in qs:
        m = m_rmsd if kind == "rmsd" else m_rbf
        lab, dist = lib.kkm_assign(m, X, mode=mode)
        alone_q.append((_np(lab), _np(dist)))
    alone_f = []
    for p in fits:
        lab, mod = lib.kkm_fit(p["X"], p["C"], p["B"], p["s"], "rbf", 0.0, 0, p["iters"], p["seed"],
                               precision=p["precision"])
        alone_f.append((_np(lab), mod.trace()[0]))
    # in the mix: fits interleaved with assigns, several workers
    srv = lib.Server(budget_bytes=20 * GB, n_workers=4)
    # the models become resident (the server owns copies made by fresh fits
    # with the same arguments, which are bit-identical)
    F, _ = md_trajectory(3000, 30, workload=4, problem=1)
    _, r1 = lib.kkm_fit(torch.from_numpy(F.reshape(3000, -1)).cuda(), 6, 2, 0.2, "rmsd", 1.5, 30, iters=8, seed=3)
    Xb, _ = blobs(4000, 32, 7, workload=4, problem=2)
    _, r2 = lib.kkm_fit(torch.from_numpy(Xb).cuda(), 7, 2, 0.25, "rbf", 0.0, iters=8, seed=5,
                        precision=lib.KKM_BF16)
    ids = {"rmsd": srv.add_model(r1), "rbf": srv.add_model(r2)}
    tickets = []
    fi = 0
    for k, (kind, X, mode) in enumerate(qs):
        tickets.append(("q", k, srv.submit_assign(ids[kind], X, mode)))
        if k % 7 == 3 and fi < len(fits):
            tickets.append(("f", fi, srv.submit_fit(fits[fi])))
            fi += 1
    while fi < len(fits):
        tickets.append(("f", fi, srv.submit_fit(fits[fi])))
        fi += 1
    for what, k, t in tickets:
        st, out, mid, err = srv.wait(t)
        assert st == 0, err
        if what == "q":
            lab, dist = out
            assert np.array_equal(_np(lab), alone_q[k][0])
            assert np.array_equal(_np(dist), alone_q[k][1])
        else:
            assert np.array_equal(_np(out), alone_f[k][0])
    s = srv.stats()
    assert s["completed_assign"] == len(qs) and s["completed_fit"] == len(fits)
    assert s["failed"] == 0 and s["queued"] == 0
    assert 0 < s["p50_assign_ms"] <= s["p99_assign_ms"]
    assert s["kernel_evals"] > 0
    srv.close()


def test_waiting_assigns_are_fused(lib, models):
    """With one worker busy on a fit, assigns that arrive meanwhile wait
    together and run as fused launches; each result is still its own."""
    import torch
    srv = lib.Server(budget_bytes=20 * GB, n_workers=1)
    Xb, _ = blobs(4000, 32, 7, workload=4, problem=2)
    _, r2 = lib.kkm_fit(torch.from_numpy(Xb).cuda(), 7, 2, 0.25, "rbf", 0.0, iters=8, seed=5,
                        precision=lib.KKM_BF16)
    mid = srv.add_model(r2)
    big, _ = blobs(40000, 64, 8, workload=4, problem=30)
    tf = srv.submit_fit(dict(X=big, C=8, B=1, s=0.5, iters=20, seed=1))
    qs = [q for q in _queries(30, seed=3) if q[0] == "rbf"]
    ts = [srv.submit_assign(mid, X, "supports") for _, X, _ in qs]
    assert srv.wait(tf)[0] == 0
    for (_, X, _), t in zip(qs, ts):
        st, (lab, dist), _, err = srv.wait(t)
        assert st == 0, err
        la, da = lib.kkm_assign(models[1], X, mode="supports")
        assert np.array_equal(_np(lab), _np(la)) and np.array_equal(_np(dist), _np(da))
    s = srv.stats()
    assert s["fused_assign_launches"] < len(qs)
    srv.close()


def test_budget_admission_and_refusal(lib, models):
    srv = lib.Server(budget_bytes=64 << 20, n_workers=2)
    X, _ = blobs(20000, 64, 5, workload=4, problem=40)
    with pytest.raises(lib.KKMError) as e:
        srv.submit_fit(dict(X=X, C=5, B=1, s=1.0, iters=2, seed=0))   # a 1.6 GB kernel block
    assert "KKM_EBUDGET" in str(e.value)
    small, _ = blobs(2000, 16, 3, workload=4, problem=41)
    t = srv.submit_fit(dict(X=small, C=3, B=1, s=0.3, iters=3, seed=0))
    assert srv.wait(t)[0] == 0
    assert srv.stats()["refused"] == 1
    assert srv.stats()["peak_bytes"] <= 64 << 20
    srv.close()


def test_failed_job_does_not_stop_others(lib):
    srv = lib.Server(budget_bytes=8 * GB, n_workers=2)
    X, _ = blobs(1500, 16, 4, workload=4, problem=50)
    bad = np.array(X)
    bad[7, 3] = np.nan
    t_bad = srv.submit_fit(dict(X=bad, C=4, B=1, s=0.5, iters=3, seed=0))
    t_ok = srv.submit_fit(dict(X=X, C=4, B=1, s=0.5, iters=3, seed=0))
    st, _, _, err = srv.wait(t_bad)
    assert st == lib.STATUS_EINVAL and "NaN" in err
    assert srv.wait(t_ok)[0] == 0
    assert srv.stats()["failed"] == 1
    srv.close()


def test_wait_timeout_then_result(lib):
    srv = lib.Server(budget_bytes=20 * GB, n_workers=1)
    big, _ = blobs(40000, 64, 8, workload=4, problem=60)
    t1 = srv.submit_fit(dict(X=big, C=8, B=1, s=0.5, iters=30, seed=2))
    small, _ = blobs(1000, 8, 3, workload=4, problem=61)
    t2 = srv.submit_fit(dict(X=small, C=3, B=1, s=0.5, iters=3, seed=2))
    with pytest.raises(lib.KKMError) as e:
        srv.wait(t2, timeout_ms=0)
    assert "KKM_ETIMEOUT" in str(e.value)
    assert srv.wait(t1)[0] == 0
    assert srv.wait(t2)[0] == 0
    with pytest.raises(lib.KKMError):
        srv.wait(t2)                 # a ticket is consumed by its wait
    srv.close()


def test_fit_kept_resident_then_assign(lib):
    import torch
    srv = lib.Server(budget_bytes=8 * GB, n_workers=2)
    X, _ = blobs(3000, 32, 5, workload=4, problem=70)
    p = dict(X=X, C=5, B=2, s=0.3, iters=5, seed=9)
    st, lab, mid, _ = srv.wait(srv.submit_fit(p, keep_model=True))
    assert st == 0 and mid >= 0
    Xq, _ = blobs(700, 32, 5, workload=4, problem=71)
    st, (la, da), _, _ = srv.wait(srv.submit_assign(mid, Xq, "supports"))
    assert st == 0
    _, m = lib.kkm_fit(torch.from_numpy(X).cuda(), 5, 2, 0.3, "rbf", 0.0, iters=5, seed=9)
    lb, db = lib.kkm_assign(m, Xq, mode="supports")
    assert np.array_equal(_np(la), _np(lb)) and np.array_equal(_np(da), _np(db))
    srv.remove_model(mid)
    with pytest.raises(lib.KKMError):
        srv.submit_assign(mid, Xq, "supports")
    srv.close()


def test_concurrent_submitters(lib, models):
    """Several host threads submit at once; every ticket completes."""
    srv = lib.Server(budget_bytes=20 * GB, n_workers=3)
    import torch
    Xb, _ = blobs(4000, 32, 7, workload=4, problem=2)
    _, r2 = lib.kkm_fit(torch.from_numpy(Xb).cuda(), 7, 2, 0.25, "rbf", 0.0, iters=8, seed=5,
                        precision=lib.KKM_BF16)
    mid = srv.add_model(r2)
    qs = [q for q in _queries(24, seed=5) if q[0] == "rbf"]
    res = {}

    def client(part):
        for k in part:
            res[k] = srv.wait(srv.submit_assign(mid, qs[k][1], qs[k][2]))

    th = [threading.Thread(target=client, args=(list(range(i, len(qs), 3)),)) for i in range(3)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for k, (st, (lab, dist), _, _) in res.items():
        assert st == 0
        la, da = lib.kkm_assign(models[1], qs[k][1], mode=qs[k][2])
        assert np.array_equal(_np(lab), _np(la)) and np.array_equal(_np(dist), _np(da))
    srv.close()
