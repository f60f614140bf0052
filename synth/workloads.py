"""Seeded generators for the five benchmark workloads (numpy PCG64).

Seeds are SEED_BASE + 1000 * workload + problem.  The recipes stand in for the
paper's datasets (MNIST, the PNP molecular-dynamics trajectory), which are not
reproduced: only their shapes and value distributions are imitated.
"""

import numpy as np

SEED_BASE = 1710_03013


def _rng(workload, problem=0, extra=0):
    return np.random.Generator(
        np.random.PCG64(SEED_BASE + 1000 * workload + problem + 7919 * extra))


def blobs(N, d, n_blobs, workload=0, problem=0, centre_box=5.0, blob_sigma=1.0):
    """Isotropic Gaussian blobs: centres uniform in [-box, box]^d, unit width,
    equal weights.  Returns (X float32 [N][d], true labels int32 [N])."""
    g = _rng(workload, problem)
    centres = g.uniform(-centre_box, centre_box, size=(n_blobs, d))
    y = g.integers(0, n_blobs, size=N)
    X = centres[y] + g.normal(0.0, blob_sigma, size=(N, d))
    return X.astype(np.float32), y.astype(np.int32)


def mnist_like(N=60000, d=784, n_classes=10, density=0.2, noise=0.1,
               workload=1, problem=0):
    """MNIST-shaped features in [0, 1], quantised to k/255.

    Each class template keeps a Bernoulli(density) subset of the coordinates
    with values U[0.3, 1]; a sample is clip(template + N(0, noise^2), 0, 1) on
    every coordinate, then rounded to a multiple of 1/255.  Returns
    (X float32 [N][d], labels int32 [N])."""
    g = _rng(workload, problem)
    mask = g.random((n_classes, d)) < density
    templ = np.where(mask, g.uniform(0.3, 1.0, size=(n_classes, d)), 0.0)
    y = g.integers(0, n_classes, size=N).astype(np.int32)
    X = np.empty((N, d), dtype=np.float32)
    step = 8192
    for a in range(0, N, step):
        b = min(N, a + step)
        v = templ[y[a:b]] + g.normal(0.0, noise, size=(b - a, d))
        v = np.clip(v, 0.0, 1.0)
        X[a:b] = (np.rint(v * 255.0) / 255.0).astype(np.float32)
    return X, y


def _random_rotations(g, n):
    """Uniform SO(3) rotations from uniform unit quaternions [n][3][3]."""
    q = g.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def random_rigid_motion(g, n, box=10.0):
    """n random proper rigid motions: rotations [n][3][3], shifts [n][3]."""
    return _random_rotations(g, n), g.uniform(-box, box, size=(n, 3))


def md_trajectory(n_frames=500000, n_atoms=300, n_states=8, dwell=2000.0,
                  noise=0.5, bond=3.8, box=10.0, workload=2, problem=0):
    """MD-shaped trajectory: a Markov jump process among random-coil reference
    conformations (C-alpha-like chains, fixed bond length in uniformly random
    directions), geometric dwell of the given mean, then per frame Gaussian
    noise per coordinate, a uniform random rotation and a translation in
    [-box, box]^3.  Returns (frames float32 [n][n_atoms][3], state int32 [n])."""
    g = _rng(workload, problem)
    steps = g.normal(size=(n_states, n_atoms, 3))
    steps *= bond / np.linalg.norm(steps, axis=2, keepdims=True)
    refs = np.cumsum(steps, axis=1)
    refs -= refs.mean(axis=1, keepdims=True)
    state = np.empty(n_frames, dtype=np.int32)
    cur = int(g.integers(0, n_states))
    p_leave = 1.0 / dwell
    t = 0
    while t < n_frames:
        stay = int(g.geometric(p_leave))
        state[t:t + stay] = cur
        t += stay
        nxt = int(g.integers(0, n_states - 1))
        cur = nxt if nxt < cur else nxt + 1
    out = np.empty((n_frames, n_atoms, 3), dtype=np.float32)
    step = 16384
    for a in range(0, n_frames, step):
        b = min(n_frames, a + step)
        f = refs[state[a:b]] + g.normal(0.0, noise, size=(b - a, n_atoms, 3))
        R, shift = random_rigid_motion(g, b - a, box)
        f = np.einsum("nij,nkj->nki", R, f) + shift[:, None, :]
        out[a:b] = f.astype(np.float32)
    return out, state


def batched_problems(n_problems=256, workload=3):
    """Shapes of the batched-problem workload: N log-uniform in [1e3, 5e4],
    d in {8, 32, 64, 128}, C uniform in [2, 64], B = ceil(N / 1e4),
    s in {0.1, 0.5}.  Returns a list of dicts; data via ``blobs``."""
    g = _rng(workload, 0, extra=1)
    out = []
    for p in range(n_problems):
        N = int(round(np.exp(g.uniform(np.log(1000.0), np.log(50000.0)))))
        d = int(g.choice([8, 32, 64, 128]))
        C = int(g.integers(2, 65))
        B = int(-(-N // 10000))
        s = float(g.choice([0.1, 0.5]))
        out.append({"problem": p, "N": N, "d": d, "C": C, "B": B, "s": s})
    return out
