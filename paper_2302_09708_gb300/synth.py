"""Seeded synthetic inputs for one CheFSI step (problem set-up only).

This module builds the inputs that both the CUDA library and the CPU oracle
consume: the finite-difference grid, a synthetic effective potential Veff, the
Kleinman-Bylander projector tables, and a starting orbital block X0.  It holds
none of the CheFSI arithmetic (no Hamiltonian application, filtering,
projection, eigensolve or rotation); it is shared by the tests, the benchmark
and the oracle checks so that both sides see byte-identical inputs.

The paper (Sec. IV) runs bulk Mo and TiO2 slabs with ONCV pseudopotentials.
Those data are not available, so the workloads are stood in for by synthetic
systems with the same grid shapes, boundary conditions, spacing and orbital
counts:

* Veff(r) = sum_J -D_J exp(-|r - R_J|^2 / (2 w_J^2)), D_J ~ U(1,3) Ha,
  w_J ~ U(0.8,1.5) bohr, minimum image along periodic axes.
* per atom, l = 0 and l = 1 projectors chi_{J,lm}(r) = g_l(r) Y_lm(r_hat) for
  |r - R_J| <= 3 bohr, g_0 = exp(-r^2/2), g_1 = r exp(-r^2/2) (sigma = 1 bohr),
  real Y_1m ordered (y, z, x); each chi is normalised on the grid so that
  h^3 sum chi^2 = 1; the energies gamma_{J,l} ~ U(-1,1) Ha are shared by the m
  components of one l.
* X0: i.i.d. N(0,1) entries, orthonormalised (X0^T X0 = I) by Cholesky-QR
  applied twice.

Grid convention: point (i, j, k) sits at (i h, j h, k h), 0 <= i < N, with the
linear index i + nx (j + ny k) (x fastest).  Along a periodic axis neighbours
wrap modulo N; along a Dirichlet axis values outside [0, N) are zero and atoms
have no periodic images.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PERIODIC = 0
DIRICHLET = 1

SEED_BASE = 230209708

# Projector cut-off radius (bohr) and radial width sigma (bohr).
RC = 3.0
SIGMA = 1.0


@dataclasses.dataclass
class System:
    """A synthetic Kohn-Sham Hamiltonian: grid, Veff and KB projector tables.

    The nonlocal tables are per atom, in the layout of the C ABI:
    ``supp_ptr[A+1]`` (int64) delimits each atom's support points in
    ``supp_idx`` (int32 linear grid indices, ascending); ``chi_ptr[A+1]``
    (int64) delimits each atom's column-major ``n_supp x nproj`` block of
    projector values in ``chi``; ``gamma`` holds one energy per projector
    (``proj_ptr[A+1]`` delimits each atom's projectors).
    """

    nx: int
    ny: int
    nz: int
    h: float
    bc: tuple
    veff: np.ndarray
    positions: np.ndarray
    supp_ptr: np.ndarray
    supp_idx: np.ndarray
    nproj: np.ndarray
    chi_ptr: np.ndarray
    chi: np.ndarray
    proj_ptr: np.ndarray
    gamma: np.ndarray
    name: str = ""

    @property
    def nd(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def natoms(self) -> int:
        return int(self.positions.shape[0])

    @property
    def shape(self):
        return (self.nx, self.ny, self.nz)


def _axis_delta(coord: np.ndarray, center: float, n: int, h: float, bc: int) -> np.ndarray:
    """Signed displacement coord - center along one axis (minimum image if periodic)."""
    d = coord - center
    if bc == PERIODIC:
        length = n * h
        d = d - length * np.round(d / length)
    return d


def _veff(shape, h, bc, positions, depth, width):
    nx, ny, nz = shape
    x = np.arange(nx) * h
    y = np.arange(ny) * h
    z = np.arange(nz) * h
    v = np.zeros((nz, ny, nx))
    for (px, py, pz), dj, wj in zip(positions, depth, width):
        dx = _axis_delta(x, px, nx, h, bc[0])
        dy = _axis_delta(y, py, ny, h, bc[1])
        dz = _axis_delta(z, pz, nz, h, bc[2])
        r2 = dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2
        v -= dj * np.exp(-r2 / (2.0 * wj * wj))
    return v.reshape(-1)


def _atom_support(shape, h, bc, pos):
    """Grid points within RC of one atom (minimum image): indices and displacements."""
    nx, ny, nz = shape
    r = int(math.ceil(RC / h))
    axes = []
    for n, p, b in zip((nx, ny, nz), pos, bc):
        c = int(round(p / h))
        idx = np.arange(c - r, c + r + 1)
        if b == PERIODIC:
            idx = np.unique(np.mod(idx, n))
        else:
            idx = idx[(idx >= 0) & (idx < n)]
        d = _axis_delta(idx * h, p, n, h, b)
        axes.append((idx, d))
    (ix, dx), (iy, dy), (iz, dz) = axes
    DZ, DY, DX = np.meshgrid(dz, dy, dx, indexing="ij")
    IZ, IY, IX = np.meshgrid(iz, iy, ix, indexing="ij")
    r2 = DX ** 2 + DY ** 2 + DZ ** 2
    mask = r2 <= RC * RC
    lin = (IX + nx * (IY + ny * IZ))[mask]
    order = np.argsort(lin, kind="stable")
    return (lin[order].astype(np.int32), DX[mask][order], DY[mask][order], DZ[mask][order])


def _projectors(shape, h, bc, positions, energies_l0, energies_l1):
    supp_ptr = [0]
    chi_ptr = [0]
    proj_ptr = [0]
    idx_all, chi_all, gam_all, nproj = [], [], [], []
    for J, pos in enumerate(positions):
        lin, dx, dy, dz = _atom_support(shape, h, bc, pos)
        r2 = dx * dx + dy * dy + dz * dz
        g = np.exp(-r2 / (2.0 * SIGMA * SIGMA))
        y00 = 0.5 / math.sqrt(math.pi)
        y1 = math.sqrt(3.0 / (4.0 * math.pi))
        # g_0 Y_00 and g_1 Y_1m with g_1 = r exp(-r^2/2): r * (x_m / r) = x_m
        cols = [g * y00, g * y1 * dy, g * y1 * dz, g * y1 * dx]
        block = np.stack(cols, axis=1)  # n_supp x 4
        norms = np.sqrt(h ** 3 * np.sum(block * block, axis=0))
        block = block / norms[None, :]
        idx_all.append(lin)
        chi_all.append(np.asfortranarray(block).reshape(-1, order="F"))
        gam_all.append(np.array([energies_l0[J]] + [energies_l1[J]] * 3))
        nproj.append(4)
        supp_ptr.append(supp_ptr[-1] + lin.size)
        chi_ptr.append(chi_ptr[-1] + block.size)
        proj_ptr.append(proj_ptr[-1] + 4)
    if not idx_all:
        return (np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32),
                np.zeros(1, np.int64), np.zeros(0), np.zeros(1, np.int64), np.zeros(0))
    return (np.array(supp_ptr, np.int64), np.concatenate(idx_all).astype(np.int32),
            np.array(nproj, np.int32), np.array(chi_ptr, np.int64),
            np.concatenate(chi_all).astype(np.float64), np.array(proj_ptr, np.int64),
            np.concatenate(gam_all).astype(np.float64))


def build_system(shape, h, bc, positions, depth, width, e_l0, e_l1, name="") -> System:
    """Assemble a System from explicit atom data (positions in bohr)."""
    positions = np.asarray(positions, dtype=np.float64).reshape(-1, 3)
    veff = _veff(shape, h, bc, positions, depth, width)
    sp, si, npj, cp, chi, pp, gam = _projectors(shape, h, bc, positions, e_l0, e_l1)
    return System(shape[0], shape[1], shape[2], float(h), tuple(int(b) for b in bc),
                  veff, positions, sp, si, npj, cp, chi, pp, gam, name)


def random_system(shape, h, bc, natoms, seed, positions=None, name="") -> System:
    """Seeded system: atoms uniform in the box (or given), Gaussian Veff, KB projectors."""
    rng = np.random.default_rng(seed)
    lengths = np.array(shape, dtype=np.float64) * h
    if positions is None:
        positions = rng.uniform(0.0, 1.0, size=(natoms, 3)) * lengths
    positions = np.asarray(positions, dtype=np.float64).reshape(-1, 3)
    a = positions.shape[0]
    depth = rng.uniform(1.0, 3.0, size=a)
    width = rng.uniform(0.8, 1.5, size=a)
    e_l0 = rng.uniform(-1.0, 1.0, size=a)
    e_l1 = rng.uniform(-1.0, 1.0, size=a)
    return build_system(shape, h, bc, positions, depth, width, e_l0, e_l1, name)


def free_system(shape, h, bc, v0=0.0) -> System:
    """No atoms and a constant Veff = v0: the free-electron Hamiltonian on the grid."""
    nd = shape[0] * shape[1] * shape[2]
    sp, si, npj, cp, chi, pp, gam = _projectors(shape, h, bc, np.zeros((0, 3)), [], [])
    return System(shape[0], shape[1], shape[2], float(h), tuple(int(b) for b in bc),
                  np.full(nd, float(v0)), np.zeros((0, 3)), sp, si, npj, cp, chi, pp, gam,
                  "free")


def jittered_lattice(counts, spacing, origin, jitter, rng):
    """Simple-cubic lattice of counts[0] x counts[1] x counts[2] sites with U(-j, j) jitter."""
    cx, cy, cz = counts
    g = np.stack(np.meshgrid(np.arange(cx), np.arange(cy), np.arange(cz), indexing="ij"), -1)
    pts = g.reshape(-1, 3).astype(np.float64) * np.asarray(spacing) + np.asarray(origin)
    return pts + rng.uniform(-jitter, jitter, size=pts.shape)


def random_orbitals(nd: int, ns: int, seed: int, ld: int | None = None) -> np.ndarray:
    """X0 with X0^T X0 = I: N(0,1) entries orthonormalised by Cholesky-QR twice.

    Returned as a C-contiguous (ns, ld) array, i.e. the column-major Nd x Ns
    block with leading dimension ld (rows nd..ld-1 of each column are zero).
    """
    import scipy.linalg

    ld = nd if ld is None else ld
    rng = np.random.default_rng(seed)
    x = np.zeros((ns, ld))
    x[:, :nd] = rng.standard_normal((ns, nd))
    for _ in range(2):
        g = x @ x.T
        r = np.linalg.cholesky(g)  # g = r r^T with r lower: X <- X r^-T
        x = scipy.linalg.solve_triangular(r, x, lower=True, overwrite_b=True, check_finite=False)
    return np.ascontiguousarray(x)


def electrons_for(ns: int) -> int:
    """Electron count Ne = 2 round((Ns - 5) / 1.2) (inverts Ns = 1.2 Ne/2 + 5, Sec. IV)."""
    return 2 * int(round((ns - 5) / 1.2))


# ---------------------------------------------------------------------------
# Named workloads.  Each has its own seed block: seed = SEED_BASE + offset +
# system index.
# ---------------------------------------------------------------------------
WORKLOADS = {
    "bulk24": dict(name="24^3 periodic, h=0.5, 8 random atoms, Ns=40, m=20", seed_offset=1000,
                   shape=(24, 24, 24), h=0.5, bc=(PERIODIC,) * 3, ns=40, degree=20, steps=1,
                   natoms=8),
    # one system of the batched set's size range (N^3 with N not a multiple of
    # 16, so the generic slab stencil runs): a single-handle profiling case
    "member36": dict(name="36^3 periodic, h=0.5, 24 random atoms, Ns=150, m=20",
                     seed_offset=1500, shape=(36, 36, 36), h=0.5, bc=(PERIODIC,) * 3, ns=150,
                     degree=20, steps=1, natoms=24),
    "bulk96": dict(name="96^3 periodic bulk, h=0.4, 216 atoms (6^3 jittered SC), Ns=1300, m=20",
                   seed_offset=2000, shape=(96, 96, 96), h=0.4, bc=(PERIODIC,) * 3, ns=1300,
                   degree=20, steps=3),
    "slab64x64x160": dict(name="64x64x160 slab (periodic xy, Dirichlet z), h=0.35, 600 atoms, "
                               "Ns=4800, m=24", seed_offset=4000, shape=(64, 64, 160), h=0.35,
                          bc=(PERIODIC, PERIODIC, DIRICHLET), ns=4800, degree=24, steps=1,
                          lattice=(10, 10, 6)),
    # the same slab recipe at half the lateral size and half the depth: the
    # reduced slab the oracle can step in seconds
    "slab32x32x80": dict(name="32x32x80 slab (periodic xy, Dirichlet z), h=0.35, 75 atoms, "
                              "Ns=600, m=24", seed_offset=4100, shape=(32, 32, 80), h=0.35,
                         bc=(PERIODIC, PERIODIC, DIRICHLET), ns=600, degree=24, steps=1,
                         lattice=(5, 5, 3)),
}
BATCH_SEED_OFFSET = 5000  # the 64 uneven systems of the batched form


def workload_seed(workload: str, index: int = 0) -> int:
    return SEED_BASE + WORKLOADS[workload]["seed_offset"] + index


def make_workload_system(workload: str) -> System:
    """The synthetic system of a named workload: the 24^3 bulk with 8 random
    atoms, the 36^3 batch-member case with 24 random atoms, the 96^3 bulk with 216 atoms on a jittered simple-cubic lattice, the
    64 x 64 x 160 slab with 600 atoms in the central 60 % of z, or the reduced
    32 x 32 x 80 slab (75 atoms) built the same way."""
    c = WORKLOADS[workload]
    seed = workload_seed(workload)
    shape, h, bc = c["shape"], c["h"], c["bc"]
    if workload in ("bulk24", "member36"):
        return random_system(shape, h, bc, c["natoms"], seed, name=c["name"])
    rng = np.random.default_rng(seed + 500)
    if workload == "bulk96":
        pos = jittered_lattice((6, 6, 6), 6.4, (3.2, 3.2, 3.2), 0.5, rng)
    else:  # slab: cx x cy x cz lattice in x, y and z in [0.2, 0.8] Lz
        cx, cy, cz = c["lattice"]
        lx, lz = shape[0] * h, (shape[2] - 1) * h
        zs = np.linspace(0.2 * lz, 0.8 * lz, cz)
        sx = lx / cx
        base = jittered_lattice((cx, cy, 1), (sx, sx, 1.0), (sx / 2, sx / 2, 0.0), 0.0, rng)
        pos = np.concatenate([base + np.array([0.0, 0.0, z]) for z in zs])
        pos += rng.uniform(-0.5, 0.5, size=pos.shape)
    return random_system(shape, h, bc, pos.shape[0], seed, positions=pos, name=c["name"])


def batch_members(count: int = 64, seed: int | None = None):
    """Uneven small systems for the batched form: N^3 grids, N ~ U{24..48}, h = 0.5,
    periodic, 4..40 atoms, Ns ~ U{40..300}, degree ~ U{16..24}."""
    rng = np.random.default_rng(SEED_BASE + BATCH_SEED_OFFSET if seed is None else seed)
    out = []
    for i in range(count):
        n = int(rng.integers(24, 49))
        a = int(rng.integers(4, 41))
        ns = int(rng.integers(40, 301))
        ns = min(ns, n ** 3 // 4)
        m = int(rng.integers(16, 25))
        out.append(dict(shape=(n, n, n), h=0.5, bc=(PERIODIC,) * 3, natoms=a, ns=ns, degree=m,
                        seed=SEED_BASE + BATCH_SEED_OFFSET + i + 1))
    return out
