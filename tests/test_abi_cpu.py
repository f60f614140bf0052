"""The C-ABI library without a GPU: it builds, loads, exports every symbol the
header declares, and its host-only planning (mini-batch geometry and the
SplitMix64 landmark draw, Section 3.1 and Eq. 14/18) equals the oracle's."""

import os
import re

import numpy as np
import pytest

from oracle import kkm_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def kkm():
    from paper_1710_03013_gb300 import build
    build.build()
    from paper_1710_03013_gb300 import kkm as mod
    mod.load()
    return mod


def header_functions():
    text = open(os.path.join(ROOT, "include", "kkm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kkm_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = header_functions()
    for want in ["kkm_fit", "kkm_assign", "kkm_cost", "kkm_model_free", "kkm_kernel_matrix",
                 "kkm_debug_step", "kkm_status_string", "kkm_last_error"]:
        assert want in names


def test_library_exports_every_header_symbol(kkm):
    lib = kkm.load()
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_header_symbol(kkm):
    assert set(header_functions()) <= set(kkm._SIGNATURES)


def test_status_strings(kkm):
    assert kkm.status_string(0) == "KKM_OK"
    assert kkm.status_string(1) == "KKM_EINVAL"


@pytest.mark.parametrize("sampling", ["stride", "block"])
@pytest.mark.parametrize("N,B,s,seed", [(60000, 4, 0.2, 7), (3001, 3, 0.3, 1), (17, 5, 1.0, 2),
                                         (1000, 7, 0.01, 3), (500000, 20, 0.05, 11)])
def test_minibatch_plan_matches_oracle(kkm, sampling, N, B, s, seed):
    batches = O.minibatch_indices(N, B, sampling)
    _, _, lm = O.rng_streams(seed, B)
    for i in range(B):
        gidx, L = kkm.kkm_minibatch_plan(N, B, s, seed, i, sampling)
        assert np.array_equal(gidx, batches[i])
        want = O.landmark_indices(len(batches[i]), s, lm[i])
        assert np.array_equal(L, want)


def test_minibatch_plan_rejects_bad_arguments(kkm):
    for args in [(10, 0, 0.5, 1, 0), (10, 11, 0.5, 1, 0), (10, 2, 0.0, 1, 0), (10, 2, 1.5, 1, 0),
                 (10, 2, 0.5, 1, 2)]:
        with pytest.raises(kkm.KKMError) as e:
            kkm.kkm_minibatch_plan(*args)
        assert e.value.status == kkm.STATUS_EINVAL


def test_batched_workload_shapes_are_valid():
    """Every problem of the 256-problem batched workload passes kkm_fit's
    argument checks: C <= 256 and no larger than any of its mini-batches."""
    from synth import batched_problems
    P = batched_problems()
    assert len(P) == 256
    for p in P:
        assert 1000 <= p["N"] <= 50000 and p["d"] in (8, 32, 64, 128) and 2 <= p["C"] <= 64
        assert p["B"] == -(-p["N"] // 10000) and p["s"] in (0.1, 0.5)
        for i in range(p["B"]):
            assert (p["N"] - i + p["B"] - 1) // p["B"] >= p["C"]


def test_server_rejects_bad_config_before_any_device_call(kkm):
    """kkm_server_create checks its arguments first (no GPU needed)."""
    import ctypes
    lib = kkm.load()
    h = ctypes.c_void_p()
    for cfg in (kkm.kkm_server_config(0, 0, 0, 0), kkm.kkm_server_config(1 << 30, 65, 0, 0),
                kkm.kkm_server_config(1 << 30, -1, 0, 0), kkm.kkm_server_config(1 << 30, 2, 1, 0)):
        assert lib.kkm_server_create(ctypes.byref(cfg), ctypes.byref(h)) == kkm.STATUS_EINVAL
        assert not h.value
    assert lib.kkm_fit_batch(None, -1, 0, None, None, None) == kkm.STATUS_EINVAL
    assert lib.kkm_fit_batch(None, 1, 0, None, None, None) == kkm.STATUS_EINVAL
    assert lib.kkm_fit_batch(None, 0, 65, None, None, None) == kkm.STATUS_EINVAL


def test_model_load_rejects_bad_files_before_device_work(kkm, tmp_path):
    """kkm_model_load checks the magic, the header and the file length on the
    host; a bad file gives KKM_EINVAL without a GPU."""
    import ctypes
    import struct
    lib = kkm.load()
    h = ctypes.c_void_p()
    missing = str(tmp_path / "missing.kkm").encode()
    assert lib.kkm_model_load(missing, ctypes.byref(h)) == kkm.STATUS_EINVAL
    junk = tmp_path / "junk.kkm"
    junk.write_bytes(b"not a model at all" * 4)
    assert lib.kkm_model_load(str(junk).encode(), ctypes.byref(h)) == kkm.STATUS_EINVAL
    # right magic, header of a small RBF model, but the arrays cut short
    hdr = b"KKMMOD01" + struct.pack("<8qd", 3, 16, 0, 0, 16, 20, 3, 5, 1.5)
    short = tmp_path / "short.kkm"
    short.write_bytes(hdr + b"\0" * 100)
    assert lib.kkm_model_load(str(short).encode(), ctypes.byref(h)) == kkm.STATUS_EINVAL
    assert "inconsistent" in kkm.last_error()
    # inconsistent header (dp does not match d)
    bad = tmp_path / "bad.kkm"
    bad.write_bytes(b"KKMMOD01" + struct.pack("<8qd", 3, 16, 0, 0, 24, 20, 3, 5, 1.5))
    assert lib.kkm_model_load(str(bad).encode(), ctypes.byref(h)) == kkm.STATUS_EINVAL
    assert not h.value


def test_fit_rejects_bad_options_before_any_device_call(kkm):
    """kkm_fit checks sizes and options before it touches the GPU: an unknown
    pipeline, sampling or precision gives KKM_EINVAL here, without one."""
    X = np.zeros((64, 4), np.float32)
    for kw in (dict(pipeline=3), dict(pipeline=-1), dict(sampling=2), dict(precision=7)):
        with pytest.raises(kkm.KKMError) as e:
            kkm.kkm_fit(X, 2, 2, 0.5, "rbf", 1.0, iters=2, labels=False, stream=0, **kw)
        assert e.value.status == kkm.STATUS_EINVAL, kw
    with pytest.raises(kkm.KKMError) as e:
        kkm.kkm_fit(X, 2, 65, 0.5, "rbf", 1.0, iters=2, labels=False, stream=0)   # B > N
    assert e.value.status == kkm.STATUS_EINVAL


class _FakeCuda:
    """A CPU tensor that reports itself as a CUDA tensor on cuda:0, so that
    the binding's argument checks can run without a GPU (nothing reaches the
    library: every case below must be refused before the call)."""

    def __init__(self, t, device="cuda:0"):
        import torch
        self._t = t
        self.is_cuda = True
        self.device = torch.device(device)
        self.dtype = t.dtype
        self.shape = t.shape

    def is_contiguous(self):
        return self._t.is_contiguous()

    def dim(self):
        return self._t.dim()

    def numel(self):
        return self._t.numel()


def test_noalloc_binding_rejects_bad_arguments(kkm):
    import torch
    d, M = 8, 10
    X = _FakeCuda(torch.zeros(M, d))
    lab = _FakeCuda(torch.zeros(M, dtype=torch.int32))
    dist = _FakeCuda(torch.zeros(M))
    assert kkm._check_noalloc_args(d, X, lab, dist) == M
    assert kkm._check_noalloc_args(d, X, lab, None) == M
    bad = [
        (torch.zeros(M, d), lab, dist),                                   # Xnew on the host
        (_FakeCuda(torch.zeros(M, d, dtype=torch.float64)), lab, dist),   # wrong dtype
        (_FakeCuda(torch.zeros(d, M).t()), lab, dist),                    # not contiguous
        (_FakeCuda(torch.zeros(M, d + 1)), lab, dist),                    # wrong row length
        (_FakeCuda(torch.zeros(M * d)), lab, dist),                       # not 2-D
        (X, _FakeCuda(torch.zeros(M - 1, dtype=torch.int32)), dist),      # labels too short
        (X, _FakeCuda(torch.zeros(M, dtype=torch.int64)), dist),          # labels wrong dtype
        (X, torch.zeros(M, dtype=torch.int32), dist),                     # labels on the host
        (X, _FakeCuda(torch.zeros(2 * M, dtype=torch.int32)[::2]), dist),  # labels strided
        (X, lab, _FakeCuda(torch.zeros(M - 1))),                          # dist too short
        (X, lab, _FakeCuda(torch.zeros(M, dtype=torch.float64))),         # dist wrong dtype
        (X, _FakeCuda(torch.zeros(M, dtype=torch.int32), "cuda:1"), dist),  # another device
        (X, lab, _FakeCuda(torch.zeros(M), "cuda:1")),                    # another device
    ]
    for k, (x, l, o) in enumerate(bad):
        with pytest.raises(ValueError):
            kkm._check_noalloc_args(d, x, l, o)


def _checkpoint_bytes(N=64, d=4, C=2, B=4, s=0.5, kind=0, n_atoms=0, iters=3, sigma_arg=1.0, seed=9,
                      precision=0, sampling=0, early_stop=1, had_init=0, next_batch=2, sigma=1.0,
                      M=(5, 40), W=(10, 22), omega=(3.0, 2.5, 2.25), changed=(4, 1, 0), disp=(0.0, 0.125)):
    """A checkpoint file written field by field in the documented layout."""
    import struct
    T = len(omega)
    head = b"KKMCKP01" + struct.pack("<qqiidiiifQiiiiifq", N, d, C, B, s, kind, n_atoms, iters, sigma_arg, seed,
                                     precision, sampling, early_stop, had_init, next_batch, sigma, T)
    body = struct.pack(f"<{C}q{C}q{T}d{T}i{next_batch}d", *M, *W, *omega, *changed, *disp)
    return head + body


def test_checkpoint_file_round_trip_on_the_host(kkm, tmp_path):
    """kkm_checkpoint_load reads the documented layout, kkm_checkpoint_info
    reports it, and kkm_checkpoint_save writes the same bytes back."""
    src = tmp_path / "a.ckpt"
    src.write_bytes(_checkpoint_bytes())
    c = kkm.Checkpoint.load(str(src))
    assert c.info() == {"next_batch": 2, "B": 4, "C": 2, "sigma": 1.0}
    assert c.medoids().tolist() == [5, 40]
    out = tmp_path / "b.ckpt"
    c.save(str(out))
    assert out.read_bytes() == src.read_bytes()


@pytest.mark.parametrize("bad", [
    dict(M=(5, 64)),                     # medoid index beyond N
    dict(next_batch=5, disp=(0.0,) * 5),  # beyond B
    dict(next_batch=0, disp=()),          # nothing run
    dict(omega=(1.0,) * 7, changed=(0,) * 7),  # longer trace than next_batch * iters
    dict(C=0, M=(), W=()),
    dict(precision=5),
    dict(kind=3),
])
def test_checkpoint_load_rejects_inconsistent_files(kkm, tmp_path, bad):
    import ctypes
    lib = kkm.load()
    p = tmp_path / "bad.ckpt"
    p.write_bytes(_checkpoint_bytes(**bad))
    h = ctypes.c_void_p()
    assert lib.kkm_checkpoint_load(str(p).encode(), ctypes.byref(h)) == kkm.STATUS_EINVAL
    assert not h.value


def test_checkpoint_load_rejects_truncated_and_foreign_files(kkm, tmp_path):
    import ctypes
    lib = kkm.load()
    h = ctypes.c_void_p()
    good = _checkpoint_bytes()
    for name, data in (("short", good[:-8]), ("long", good + b"\0" * 8), ("magic", b"KKMMOD02" + good[8:]),
                       ("empty", b"")):
        p = tmp_path / f"{name}.ckpt"
        p.write_bytes(data)
        assert lib.kkm_checkpoint_load(str(p).encode(), ctypes.byref(h)) == kkm.STATUS_EINVAL, name
        assert not h.value


def test_fit_range_rejects_a_foreign_checkpoint_before_any_device_call(kkm, tmp_path):
    """A checkpoint resumes only the fit that made it, over a non-empty range
    that ends at B at most, and a model needs the last mini-batch."""
    p = tmp_path / "a.ckpt"
    p.write_bytes(_checkpoint_bytes())
    c = kkm.Checkpoint.load(str(p))
    X = np.zeros((64, 4), np.float32)
    same = dict(kind="rbf", sigma=1.0, iters=3, seed=9, labels=False, stream=0)
    cases = [
        (dict(same, seed=10), 4, False),        # another seed
        (dict(same, iters=4), 4, False),        # another iteration cap
        (dict(same, sigma=2.0), 4, False),      # another bandwidth argument
        (dict(same, sampling="block"), 4, False),
        (dict(same, precision=kkm.KKM_BF16), 4, False),
        (dict(same, early_stop=False), 4, False),
        (dict(same, init_medoids=[1, 2]), 4, False),
        (same, 2, False),                       # empty range
        (same, 5, False),                       # beyond B
        (same, 3, True),                        # a model before the last mini-batch
    ]
    for kw, stop, model in cases:
        with pytest.raises(kkm.KKMError) as e:
            kkm.kkm_fit_range(X, 2, 4, 0.5, checkpoint=c, stop=stop, model=model, **kw)
        assert e.value.status == kkm.STATUS_EINVAL, (kw, stop, model)
    with pytest.raises(kkm.KKMError):
        kkm.kkm_fit_range(X[:32], 2, 4, 0.5, checkpoint=c, stop=4, **same)   # another N
    done = tmp_path / "done.ckpt"
    done.write_bytes(_checkpoint_bytes(next_batch=4, disp=(0.0,) * 4))
    with pytest.raises(kkm.KKMError) as e:
        kkm.kkm_fit_range(X, 2, 4, 0.5, checkpoint=kkm.Checkpoint.load(str(done)), stop=4, **same)
    assert "complete" in str(e.value)
