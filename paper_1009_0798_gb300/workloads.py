"""Seeded synthetic inputs shaped like the test problems of Matsumoto (2011), Sec. 3.

This module holds no arithmetic of the solver itself: it only builds block lists,
magnetic fields and resistivity fields.  Both the CUDA path and the CPU reference
receive the identical arrays it returns.

Layouts
-------
* A hierarchy is described by base cell counts (nx, ny, nz), each a multiple of 8,
  the base cell width dx0, and a block list: int32 rows (level, bi, bj, bk), one per
  8^3-cell block, level 0 first.  Level l has cell width dx0 / 2**l.  Refinement is an
  octree (a refined block has all 8 children) with proper nesting (the 26 neighbours of a
  refined block's parent exist one level down), so coarse-fine interfaces lie on coarse
  block faces and the resolution jumps by one level at most.
* Block fields are float64 arrays [nblocks][ncomp][8][8][8] in block-list order with the
  innermost index along x ([comp][k][j][i]).
* Dense fields are float64 arrays [ncomp][nz][ny][nx].
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BS = 8  # cells per block edge


# ----------------------------------------------------------------------------- blocks
def _morton_key(b: np.ndarray) -> np.ndarray:
    """Interleave the bits of (bi, bj, bk) so nearby blocks sit close in memory."""
    key = np.zeros(len(b), dtype=np.int64)
    for bit in range(20):
        for ax in range(3):
            key |= ((b[:, ax].astype(np.int64) >> bit) & 1) << (3 * bit + ax)
    return key


def _level_blocks(nb: tuple[int, int, int]) -> np.ndarray:
    bk, bj, bi = np.meshgrid(np.arange(nb[2]), np.arange(nb[1]), np.arange(nb[0]), indexing="ij")
    b = np.stack([bi.ravel(), bj.ravel(), bk.ravel()], axis=1).astype(np.int32)
    return b[np.argsort(_morton_key(b), kind="stable")]


@dataclasses.dataclass
class Hierarchy:
    base_cells: tuple[int, int, int]
    dx0: float
    blocks: np.ndarray  # int32 [nblocks, 4]: level, bi, bj, bk
    origin: tuple[float, float, float] = (0.0, 0.0, 0.0)

    @property
    def nlevels(self) -> int:
        return int(self.blocks[:, 0].max()) + 1

    @property
    def nblocks(self) -> int:
        return len(self.blocks)

    def level_dims(self, level: int) -> tuple[int, int, int]:
        return tuple(n << level for n in self.base_cells)

    def dx(self, level: int) -> float:
        return self.dx0 / (1 << level)

    def is_leaf(self) -> np.ndarray:
        """True for blocks whose octree children are absent."""
        keys = {tuple(r) for r in self.blocks.tolist()}
        return np.array([(l + 1, 2 * i, 2 * j, 2 * k) not in keys for l, i, j, k in self.blocks.tolist()])

    def leaf_cells(self) -> int:
        return int(self.is_leaf().sum()) * BS ** 3

    def cell_centers(self, b: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
        """Cell-centre coordinates (z, y, x order, each [8,8,8]) of block b."""
        l, bi, bj, bk = (int(v) for v in self.blocks[b])
        h = self.dx(l)
        ar = np.arange(BS) + 0.5
        x = self.origin[0] + (bi * BS + ar) * h
        y = self.origin[1] + (bj * BS + ar) * h
        z = self.origin[2] + (bk * BS + ar) * h
        return np.meshgrid(z, y, x, indexing="ij")


def uniform(nx: int, ny: int, nz: int, dx: float, origin=(0.0, 0.0, 0.0)) -> Hierarchy:
    """One periodic level of nx*ny*nz cells (multiples of 8), blocks in Morton order."""
    for n in (nx, ny, nz):
        if n % BS:
            raise ValueError("cell counts must be multiples of 8")
    b = _level_blocks((nx // BS, ny // BS, nz // BS))
    blocks = np.concatenate([np.zeros((len(b), 1), np.int32), b], axis=1)
    return Hierarchy((nx, ny, nz), dx, blocks, tuple(origin))


def refined(nx: int, ny: int, nz: int, dx: float, flags, origin=(0.0, 0.0, 0.0)) -> Hierarchy:
    """AMR hierarchy from refinement flags.

    ``flags[l]`` is a predicate f(xlo, xhi) -> bool on a level-l block's physical box
    (xlo, xhi: 3-vectors); a flagged block gets 8 children at level l+1.  Flags are then
    grown so the octree is properly nested.
    """
    base = uniform(nx, ny, nz, dx, origin)
    nb0 = np.array([nx, ny, nz]) // BS
    nlev = len(flags) + 1
    org = np.array(origin, dtype=np.float64)
    # refined[l]: set of level-l blocks that have children
    refined_sets: list[set] = [set() for _ in range(nlev)]
    for l in range(nlev - 1):
        nb = nb0 << l
        h = dx / (1 << l)
        for bi in range(nb[0]):
            for bj in range(nb[1]):
                for bk in range(nb[2]):
                    lo = org + np.array([bi, bj, bk]) * BS * h
                    if flags[l](lo, lo + BS * h):
                        refined_sets[l].add((bi, bj, bk))
    # a level-l block can only be refined if it exists, i.e. its parent is refined
    for l in range(1, nlev - 1):
        refined_sets[l] = {b for b in refined_sets[l] if (b[0] // 2, b[1] // 2, b[2] // 2) in refined_sets[l - 1]}
    # proper nesting: if a level-l block is refined (l>=1), all 26 neighbours of its parent
    # at level l-1 must be refined too.  Iterate from the finest level down.
    for l in range(nlev - 2, 0, -1):
        nbp = nb0 << (l - 1)
        need = set()
        for (bi, bj, bk) in refined_sets[l]:
            p = (bi // 2, bj // 2, bk // 2)
            for di in (-1, 0, 1):
                for dj in (-1, 0, 1):
                    for dk in (-1, 0, 1):
                        need.add(((p[0] + di) % nbp[0], (p[1] + dj) % nbp[1], (p[2] + dk) % nbp[2]))
        refined_sets[l - 1] |= need
    # the children of every refined block exist; growing a coarse set may have added
    # blocks at level l whose own refinement is unaffected (nesting only constrains down)
    rows = [base.blocks]
    for l in range(1, nlev):
        parents = sorted(refined_sets[l - 1])
        if not parents:
            break
        kids = np.array([(2 * p[0] + a, 2 * p[1] + b, 2 * p[2] + c)
                         for p in parents for c in (0, 1) for b in (0, 1) for a in (0, 1)], dtype=np.int32)
        kids = kids[np.argsort(_morton_key(kids), kind="stable")]
        rows.append(np.concatenate([np.full((len(kids), 1), l, np.int32), kids], axis=1))
        # drop refinement flags of level-l blocks that do not exist
        if l < nlev - 1:
            kset = {tuple(k) for k in kids.tolist()}
            refined_sets[l] = {b for b in refined_sets[l] if b in kset}
    return Hierarchy((nx, ny, nz), dx, np.concatenate(rows, axis=0).astype(np.int32), tuple(origin))


# ----------------------------------------------------------------------------- layouts
def dense_to_blocks(h: Hierarchy, dense: np.ndarray, level: int = 0) -> np.ndarray:
    """[ncomp][nz][ny][nx] array of one full level -> [nblocks_at_level][ncomp][8][8][8]."""
    sel = h.blocks[h.blocks[:, 0] == level]
    out = np.empty((len(sel), dense.shape[0], BS, BS, BS), dtype=dense.dtype)
    for n, (_, bi, bj, bk) in enumerate(sel.tolist()):
        out[n] = dense[:, bk * BS:(bk + 1) * BS, bj * BS:(bj + 1) * BS, bi * BS:(bi + 1) * BS]
    return out


def blocks_to_dense(h: Hierarchy, blk: np.ndarray, level: int = 0) -> np.ndarray:
    """Inverse of dense_to_blocks for a fully covered level."""
    nx, ny, nz = h.level_dims(level)
    sel = np.nonzero(h.blocks[:, 0] == level)[0]
    out = np.zeros((blk.shape[1], nz, ny, nx), dtype=blk.dtype)
    for n in sel:
        _, bi, bj, bk = h.blocks[n].tolist()
        out[:, bk * BS:(bk + 1) * BS, bj * BS:(bj + 1) * BS, bi * BS:(bi + 1) * BS] = blk[n]
    return out


def sample_blocks(h: Hierarchy, fn, ncomp: int) -> np.ndarray:
    """Evaluate fn(x, y, z) -> tuple of ncomp arrays at the cell centres of every block."""
    out = np.empty((h.nblocks, ncomp, BS, BS, BS))
    for b in range(h.nblocks):
        z, y, x = h.cell_centers(b)
        vals = fn(x, y, z)
        for c in range(ncomp):
            out[b, c] = vals[c]
    return out


# ----------------------------------------------------------------------------- fields
def random_potential_field(dims: tuple[int, int, int], dx: float, seed: int, rms: float) -> np.ndarray:
    """Divergence-free random field [3][nz][ny][nx] on a periodic grid.

    A vector potential A has an amplitude spectrum |k|^-2 (complex normal coefficients for
    every k != 0 up to Nyquist, fixed seed); B is its curl by central differences
    (periodic), scaled to the requested rms |B|.
    """
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.rfftfreq(nx)[None, None, :]
    k2 = (kx * nx) ** 2 + (ky * ny) ** 2 + (kz * nz) ** 2
    amp = np.zeros_like(k2)
    amp[k2 > 0] = 1.0 / k2[k2 > 0]
    A = np.empty((3, nz, ny, nx))
    for c in range(3):
        coef = (rng.standard_normal(k2.shape) + 1j * rng.standard_normal(k2.shape)) * amp
        A[c] = np.fft.irfftn(coef, s=(nz, ny, nx), axes=(0, 1, 2))

    def d0(f, axis):  # central difference along a dense axis (0=z, 1=y, 2=x)
        return (np.roll(f, -1, axis=axis) - np.roll(f, 1, axis=axis)) / (2.0 * dx)

    B = np.empty_like(A)
    B[0] = d0(A[2], 1) - d0(A[1], 0)
    B[1] = d0(A[0], 0) - d0(A[2], 2)
    B[2] = d0(A[1], 2) - d0(A[0], 1)
    cur = math.sqrt(float(np.mean(np.sum(B * B, axis=0))))
    return B * (rms / cur)


def gaussian_bump_eta(dims, dx, eta0=1e-3, contrast=999.0, width=0.05, center=(0.5, 0.5, 0.5)) -> np.ndarray:
    """eta0 * (1 + contrast * exp(-|x-c|^2 / width^2)) at cell centres, [1][nz][ny][nx]."""
    nx, ny, nz = dims
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * dx, (np.arange(ny) + 0.5) * dx,
                          (np.arange(nx) + 0.5) * dx, indexing="ij")
    r2 = (x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2
    return (eta0 * (1.0 + contrast * np.exp(-r2 / width ** 2)))[None]


# ----------------------------------------------------------------------------- configs
@dataclasses.dataclass
class Workload:
    name: str
    hier: Hierarchy
    B: np.ndarray      # [nblocks][3][8][8][8]
    eta: np.ndarray    # [nblocks][1][8][8][8]
    dt: float
    steps: int
    tol: float
    lam: float = 0.5


def periodic_box_32(seed: int = 1, n: int = 32) -> Workload:
    """Uniform 32^3 periodic unit box, eta = 1, B = (0, sin 2pi x, cos 2pi x) plus a
    k^-2 random divergence-free field of rms 0.1; dt = 10x the explicit limit dx^2/6;
    20 CN steps to relative residual 1e-10."""
    dx = 1.0 / n
    h = uniform(n, n, n, dx)
    x = (np.arange(n) + 0.5) * dx
    wave = np.zeros((3, n, n, n))
    wave[1] = np.sin(2 * np.pi * x)[None, None, :]
    wave[2] = np.cos(2 * np.pi * x)[None, None, :]
    B = wave + random_potential_field((n, n, n), dx, seed, 0.1)
    eta = np.ones((1, n, n, n))
    return Workload(f"periodic_{n}^3_eta1", h, dense_to_blocks(h, B), dense_to_blocks(h, eta),
                    dt=10.0 * dx * dx / 6.0, steps=20, tol=1e-10)


def resistive_bump_256(n: int = 256, seed: int = 2) -> Workload:
    """Uniform n^3 periodic unit box (n = 256 for the headline case).  eta = 1e-3 (1 + 999
    exp(-|x-c|^2/0.05^2)), three decades; B = curl of a k^-2 random potential, rms 1;
    dt = 100x the explicit limit dx^2/(6 eta_max); 10 CN steps to relative residual 1e-9."""
    dx = 1.0 / n
    h = uniform(n, n, n, dx)
    B = random_potential_field((n, n, n), dx, seed, 1.0)
    eta = gaussian_bump_eta((n, n, n), dx)
    eta_max = 1e-3 * 1000.0
    return Workload(f"resistive_bump_{n}^3", h, dense_to_blocks(h, B), dense_to_blocks(h, eta),
                    dt=100.0 * dx * dx / (6.0 * eta_max), steps=10, tol=1e-9)


def current_loop_field(x, y, z, center=0.5, radius=0.1, width=0.03, amp=1.0):
    """Uniform B_z = 1 plus the poloidal field of a toroidal current ring: B = curl(A_phi phi)
    with A_phi = amp (rho/R) exp(-((rho-R)^2 + z^2)/w^2) about the box centre."""
    X, Y, Z = x - center, y - center, z - center
    rho = np.sqrt(X * X + Y * Y)
    g = np.exp(-((rho - radius) ** 2 + Z * Z) / width ** 2)
    bx = amp * (X / radius) * (2.0 * Z / width ** 2) * g
    by = amp * (Y / radius) * (2.0 * Z / width ** 2) * g
    bz = 1.0 + amp * g / radius * (2.0 - 2.0 * rho * (rho - radius) / width ** 2)
    return bx, by, bz


def nested_spheres_64(n: int = 64, radii=(0.25, 0.125, 0.0625), eta0: float = 1e-3) -> Workload:
    """Block AMR: base n^3 unit box in 8^3 blocks, refinement levels (ratio 2) on blocks
    that intersect spheres of the given radii about the centre.  eta = eta0 (1 + (0.05/r)^2)
    capped at 1e3 eta0.  B = uniform B_z = 1 plus a current ring of width 0.03 scaled to
    max |B_ring| = 1.  dt = 100x the explicit limit at the finest level and max eta."""
    dx = 1.0 / n
    c = np.array([0.5, 0.5, 0.5])

    def sphere(r):
        def f(lo, hi):
            nearest = np.clip(c, lo, hi)
            return float(np.sum((nearest - c) ** 2)) < r * r
        return f

    h = refined(n, n, n, dx, [sphere(r) for r in radii])
    # scale the ring so that max |B - B_uniform| = 1 on a fine sample
    s = np.linspace(0.3, 0.7, 161)
    X, Y, Z = np.meshgrid(s, s, s, indexing="ij")
    bx, by, bz = current_loop_field(X, Y, Z)
    peak = float(np.sqrt(bx ** 2 + by ** 2 + (bz - 1.0) ** 2).max())
    B = sample_blocks(h, lambda x, y, z: current_loop_field(x, y, z, amp=1.0 / peak), 3)

    def eta_fn(x, y, z):
        r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2
        return (np.minimum(eta0 * (1.0 + 0.05 ** 2 / np.maximum(r2, 1e-300)), 1e3 * eta0),)

    eta = sample_blocks(h, eta_fn, 1)
    dxf = h.dx(h.nlevels - 1)
    return Workload(f"nested_spheres_{n}^3_L{h.nlevels - 1}", h, B, eta,
                    dt=100.0 * dxf * dxf / (6.0 * 1e3 * eta0), steps=10, tol=1e-9)


def sinusoid_half_refined(N: int = 8, lam: float = 0.5, dt: float = 1e-4, t_end: float = 4e-3) -> Workload:
    """Sinusoidal diffusion test of Sec. 3.1: B_z = sin(k.r), k = 2pi (1, 2, 0), eta = 1,
    domain [0,1] x [0,1/2] x [0,1/4] periodic in 4 x 2 x 1 base blocks of N^3 cells (here
    covered by 8^3-cell blocks), the half x < 1/2 refined once."""
    nx, ny, nz = 4 * N, 2 * N, N
    dx = 1.0 / (4 * N)
    h = refined(nx, ny, nz, dx, [lambda lo, hi: hi[0] <= 0.5 + 1e-12])
    k = 2 * np.pi * np.array([1.0, 2.0, 0.0])
    B = sample_blocks(h, lambda x, y, z: (0 * x, 0 * x, np.sin(k[0] * x + k[1] * y + k[2] * z)), 3)
    eta = np.ones((h.nblocks, 1, BS, BS, BS))
    steps = int(round(t_end / dt))
    return Workload(f"sinusoid_half_refined_N{N}", h, B, eta, dt=dt, steps=steps, tol=1e-12, lam=lam)


# ----------------------------------------------------------------------------- batches
BATCH_EDGES = (16, 24, 32, 48, 64)


def smooth_lognormal_eta(n: int, seed: int, decades: float = 2.0, eta_min: float = 1e-3,
                         sigma_cells: float = 2.0) -> np.ndarray:
    """Dense [1][n][n][n] resistivity eta = eta_min 10^(decades u): u is seeded normal noise
    smoothed by a periodic Gaussian filter of width sigma_cells (applied as its Fourier
    transfer function exp(-2 pi^2 sigma^2 k^2), k in cycles per cell) and rescaled to [0, 1]."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((n, n, n))
    k = np.fft.fftfreq(n)
    kr = np.fft.rfftfreq(n)
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + kr[None, None, :] ** 2
    u = np.fft.irfftn(np.fft.rfftn(noise) * np.exp(-2.0 * math.pi ** 2 * sigma_cells ** 2 * k2), s=(n, n, n), axes=(0, 1, 2))
    u = (u - u.min()) / (u.max() - u.min())
    return (eta_min * 10.0 ** (decades * u))[None]


@dataclasses.dataclass
class Instance:
    n: int
    hier: Hierarchy
    B: np.ndarray      # [nblocks][3][8][8][8]
    eta: np.ndarray    # [nblocks][1][8][8][8]
    dt: float


def batched_instances(count: int = 512, seed: int = 4, edges=BATCH_EDGES, tol: float = 1e-9) -> list[Instance]:
    """Independent periodic unit boxes: edge drawn uniformly from `edges` (seeded), eta from
    smooth_lognormal_eta (2 decades), B = curl of a k^-2 random potential (rms 1), dt = U(10,
    100) times the explicit limit dx^2/(6 eta_max), one step each to `tol`.  Instance q's fields
    use seeds derived from (seed, q) only, so any prefix of the list is reproducible alone."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(edges), size=count)
    hiers = {}
    out = []
    for q, n in enumerate(int(v) for v in ns):
        dx = 1.0 / n
        h = hiers.setdefault(n, uniform(n, n, n, dx))
        base = 1_000_003 * seed + 7 * q
        B = random_potential_field((n, n, n), dx, base + 1, 1.0)
        eta = smooth_lognormal_eta(n, base + 2)
        f = float(np.random.default_rng(base + 3).uniform(10.0, 100.0))
        out.append(Instance(n, h, dense_to_blocks(h, B), dense_to_blocks(h, eta), f * dx * dx / (6.0 * float(eta.max()))))
    return out
