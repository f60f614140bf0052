"""Writes the expected values of the full-size MNIST-shaped parity tests.

Every stored value comes from the FP64 oracle (``oracle/kkm_oracle.py``) on
the seeded generator's data; nothing here touches the CUDA library.  The
inputs are the benchmark workload's first stride mini-batch: 15,000 of the
60,000 x 784 samples (B = 4), C = 10, s = 0.2 (|L| = 3,000).

  mnist_step.json  one inner iteration (Eq. 15-17) from the generator's class
                   labels, on the unrounded rows: the new labels, which rows
                   have a relative margin above 1e-4, Omega, n_j and g_hat.
  mnist_fit.json   the whole fit of that mini-batch on its own (B = 1, 30
                   iterations, early stop off, k-means++ seeding): its initial
                   medoids, final labels, the clear rows of its last
                   iteration, the Omega trace, medoids, n_j and g_hat.

Labels are stored as a string of digits (C = 10), clear rows as a hex string
of packed bits.  Each part takes a few minutes of one CPU core:
    python tests/golden/make_mnist_minibatch.py step
    python tests/golden/make_mnist_minibatch.py fit
"""

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import kkm_oracle as O  # noqa: E402
from synth import mnist_like  # noqa: E402

N, D, C, B, S, ITERS, SEED = 60000, 784, 10, 4, 0.2, 30, 1710
MARGIN_REL = 1e-4


def inputs():
    """Mini-batch 0 of the stride sampling, the bandwidth both sides use (the
    oracle's median rule on 512 samples, rounded to float32), the class labels
    and the landmarks of mini-batch 0 (Eq. 14, 18)."""
    X, cls = mnist_like(N, D)
    sigma = float(np.float32(O.median_bandwidth(X, O.Kernel(O.KIND_RBF, 0.0), O.SplitMix64(SEED), 512)))
    gidx = O.minibatch_indices(N, B)[0]
    _, _, lm = O.rng_streams(SEED, B)
    L = O.landmark_indices(len(gidx), S, lm[0])
    return X[gidx], cls[gidx], sigma, L


def clear_mask(d):
    part = np.partition(np.where(np.isfinite(d), d, np.inf), 1, axis=1)
    rel = (part[:, 1] - part[:, 0]) / np.maximum(np.abs(part[:, 1]), 1e-12)
    return rel > MARGIN_REL


def labels_str(u):
    assert u.min() >= 0 and u.max() < 10
    return "".join(str(int(v)) for v in u)


def bits_hex(mask):
    return np.packbits(mask.astype(np.uint8)).tobytes().hex()


def step():
    Xb, cls, sigma, L = inputs()
    ker = O.Kernel(O.KIND_RBF, sigma)
    Kb = ker(Xb.astype(np.float64), Xb[L].astype(np.float64))
    st = O.inner_step(Kb, ker.self_terms(Xb), L, cls.astype(np.int64), C)
    return {"sigma": sigma, "Ni": len(Xb), "nL": len(L), "landmarks_sum": int(L.sum()),
            "u": labels_str(st["u"]), "clear": bits_hex(clear_mask(st["d"])),
            "omega": st["omega"], "changed": st["changed"], "n": st["n"].tolist(),
            "ghat": st["ghat"].tolist()}


def fit():
    Xb, _, sigma, _ = inputs()
    ref = O.fit(Xb.astype(np.float64), C, 1, S, O.Kernel(O.KIND_RBF, sigma), ITERS, SEED, early_stop=False)
    det = ref["details"][0]
    return {"sigma": sigma, "Ni": len(Xb), "nL": len(det["L"]), "iters": ITERS, "seed": SEED,
            "init_medoids": det["M_before"].tolist(), "u": labels_str(ref["labels"]),
            "clear": bits_hex(clear_mask(det["steps"][-1]["d"])),
            "trace": [t[2] for t in ref["trace"]], "medoids": ref["medoids"].tolist(),
            "W": ref["W"].tolist(), "n": ref["n"].tolist(), "ghat": ref["ghat"].tolist()}


if __name__ == "__main__":
    parts = sys.argv[1:] or ["step", "fit"]
    for part in parts:
        out = {"step": step, "fit": fit}[part]()
        with open(os.path.join(HERE, f"mnist_{part}.json"), "w") as f:
            json.dump(out, f, indent=0)
            f.write("\n")
