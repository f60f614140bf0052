"""Comparison rules shared by the GPU parity tests.

Tolerances (the clustering is FP32 on the device, FP64 in the oracle):
  labels     identical wherever the oracle's relative margin
             (d_(2) - d_(1)) / max(|d_(2)|, 1e-12) exceeds 1e-4;
  distances  |d_gpu - d_oracle| <= 1e-5 * (K_ii + g_hat_j), the scale of the
             terms of d = K_ii - 2 f_hat + g_hat (d itself cancels near 0);
  Omega      relative 1e-6;
  kernel     |K_gpu - K_oracle| <= 1e-5 (K in [0, 1] for Gaussian kernels).
"""

import numpy as np

MARGIN_REL = 1e-4
DIST_REL = 1e-5
OMEGA_REL = 1e-6
KERNEL_ABS = 1e-5


def rel_margin(d):
    d = np.where(np.isfinite(d), d, np.inf)
    if d.shape[1] < 2:
        return np.full(d.shape[0], np.inf)
    part = np.partition(d, 1, axis=1)
    with np.errstate(invalid="ignore"):
        rel = (part[:, 1] - part[:, 0]) / np.maximum(np.abs(part[:, 1]), 1e-12)
    return np.where(np.isinf(part[:, 1]), np.inf, rel)


def clear_rows(d):
    return rel_margin(d) > MARGIN_REL


def assert_labels(gpu_u, ref_u, ref_d, what="labels"):
    mask = clear_rows(ref_d)
    bad = np.nonzero((np.asarray(gpu_u) != np.asarray(ref_u)) & mask)[0]
    assert bad.size == 0, f"{what}: {bad.size} clear rows differ, first {bad[:10]}"
    return mask


def assert_close_rel(got, want, rel, what):
    got = float(got)
    want = float(want)
    assert abs(got - want) <= rel * max(abs(want), 1e-300), f"{what}: {got} vs {want}"


def first_divergence(gpu_trace, ref_trace, rel=OMEGA_REL):
    for t, (a, b) in enumerate(zip(gpu_trace, ref_trace)):
        if abs(a - b) > rel * max(abs(b), 1e-300):
            return t
    return None
