"""Shared helpers for the parity tests: seeded hierarchies and field conversions."""
import numpy as np

from paper_1009_0798_gb300 import workloads as W


def rand_fields(h, seed, eta_decades=1.0):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((h.nblocks, 3, 8, 8, 8))
    eta = 10.0 ** rng.uniform(-eta_decades / 2, eta_decades / 2, (h.nblocks, 1, 8, 8, 8))
    return B, eta


def amr_two_level(n=16):
    """Base n x n/2 x n/2 periodic box, the blocks with x < 0.45 refined once."""
    return W.refined(n, n // 2, n // 2, 1.0 / n, [lambda lo, hi: lo[0] < 0.45])


def amr_three_level(n=16):
    """Base n^3, two nested refinements about the centre (spheres r < 0.3, 0.12)."""
    c = np.array([0.5, 0.5, 0.5])

    def sphere(r):
        return lambda lo, hi: float(np.sum((np.clip(c, lo, hi) - c) ** 2)) < r * r

    return W.refined(n, n, n, 1.0 / n, [sphere(0.3), sphere(0.12)])


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    den = np.sqrt(np.sum(b * b))
    return float(np.sqrt(np.sum((a - b) ** 2)) / (den if den > 0 else 1.0))


def dense_of_grid(blk, ijk, dims, ncomp):
    """Blocked [nb][ncomp][8][8][8] with block coordinates ijk -> dense [ncomp][nz][ny][nx]."""
    nx, ny, nz = dims
    out = np.zeros((ncomp, nz, ny, nx))
    for n, (bi, bj, bk) in enumerate(ijk):
        out[:, bk * 8:(bk + 1) * 8, bj * 8:(bj + 1) * 8, bi * 8:(bi + 1) * 8] = blk[n]
    return out


def grid_of_dense(dense, ijk):
    out = np.empty((len(ijk), dense.shape[0], 8, 8, 8))
    for n, (bi, bj, bk) in enumerate(ijk):
        out[n] = dense[:, bk * 8:(bk + 1) * 8, bj * 8:(bj + 1) * 8, bi * 8:(bi + 1) * 8]
    return out
