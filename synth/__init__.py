"""Seeded synthetic inputs for the mass-spring workloads.

This module only *describes* systems: geometry, connectivity, per-element
parameters and random designs drawn from fixed seeds.  It holds none of the
step's arithmetic (no forces, no integration, no spring merging), so both the
CPU oracle and the GPU library can consume its output without sharing any
part of the method.

A "system" is a plain dict of numpy arrays in the caller's index order:

    x      (N,3) float32   initial positions [m]
    v      (N,3) float32   initial velocities [m/s]
    m      (N,)  float32   mass per node [kg]
    fixed  (N,)  uint8     1 = anchored (position frozen, velocity zero)
    fext   (N,3) float32   external force [N], or absent
    ij     (S,2) int32     spring endpoints
    k      (S,)  float32   Hooke stiffness [N/m]
    c      (S,)  float32   axial dashpot coefficient [N s/m]
    L0     (S,)  float32   rest length [m]
    A      (S,)  float32   actuation amplitude (0 = passive), or absent
    phi    (S,)  float32   actuation phase [rad], or absent
    freq   float           actuation frequency [Hz]

and "params" is a dict: dt, g (3-tuple), k_c, mu, vel_damping, contact.

The lattices follow the voxel construction of the paper's lattice section
(Generating a Lattice, Fig. figure1): nodes on a cubic grid, linked along
edges, face diagonals and long (body) diagonals, i.e. the 26-neighbourhood
with each pair linked once.  Workload sizes are those of the benchmark
workloads: a 10^3 soft cube and 40x4x4 cantilever, a 256^3 throughput
lattice, and populations of voxel robots.
"""
from __future__ import annotations

import numpy as np

# The 13 "forward" neighbour offsets (dx, dy, dz) of the 26-neighbourhood:
# those whose (dz, dy, dx) is lexicographically positive, so that with the
# x-fastest node numbering the partner index is always larger.
FORWARD_OFFSETS = np.array(
    [(dx, dy, dz)
     for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
     if (dz, dy, dx) > (0, 0, 0)], dtype=np.int64)
assert FORWARD_OFFSETS.shape == (13, 3)

DEFAULT_PARAMS = dict(dt=1e-4, g=(0.0, 0.0, -9.81), k_c=1e5, mu=0.0,
                      vel_damping=0.0, contact=False)


def params(**kw):
    p = dict(DEFAULT_PARAMS)
    p.update(kw)
    return p


def box_lattice(nx: int, ny: int, nz: int, a: float, origin=(0.0, 0.0, 0.0)):
    """Cubic node grid with 26-neighbourhood springs, each pair once.

    Node (ix, iy, iz) has index ix + nx*(iy + ny*iz).  Springs are listed
    node-major (all forward springs of node 0, then node 1, ...), in the
    order of FORWARD_OFFSETS.  Rest lengths are the nominal lattice lengths
    a, a*sqrt(2), a*sqrt(3) rounded to float32.
    Returns (x[N,3] f32, ij[S,2] i32, L0[S] f32).
    """
    N = nx * ny * nz
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ix = ix.ravel(); iy = iy.ravel(); iz = iz.ravel()
    x = np.empty((N, 3), dtype=np.float32)
    x[:, 0] = (origin[0] + ix * a)
    x[:, 1] = (origin[1] + iy * a)
    x[:, 2] = (origin[2] + iz * a)
    if N >= 2 ** 31 // 16:
        raise ValueError("lattice too large for int32 indexing")
    off = FORWARD_OFFSETS
    # validity of each forward offset per node, shape (N, 13)
    valid = np.ones((N, 13), dtype=bool)
    for d in range(13):
        dx, dy, dz = off[d]
        v = valid[:, d]
        if dx > 0: v &= ix < nx - 1
        if dx < 0: v &= ix > 0
        if dy > 0: v &= iy < ny - 1
        if dy < 0: v &= iy > 0
        if dz > 0: v &= iz < nz - 1
        if dz < 0: v &= iz > 0
    del ix, iy, iz
    step = (off[:, 0] + nx * (off[:, 1] + ny * off[:, 2])).astype(np.int32)
    nodes = np.arange(N, dtype=np.int32)
    cnt = valid.sum(axis=1)
    S = int(cnt.sum())
    ij = np.empty((S, 2), dtype=np.int32)
    ij[:, 0] = np.repeat(nodes, cnt)
    dsel = np.broadcast_to(np.arange(13, dtype=np.int8), (N, 13))[valid]
    ij[:, 1] = ij[:, 0] + step[dsel]
    nominal = (a * np.sqrt((off ** 2).sum(axis=1).astype(np.float64))).astype(np.float32)
    L0 = nominal[dsel]
    return x, ij, L0


def lattice_spring_count(nx: int, ny: int, nz: int) -> int:
    """Number of 26-neighbourhood pairs in an nx*ny*nz node grid (closed form)."""
    def n(a, d):  # pairs along one axis with offset |d|
        return max(a - abs(d), 0)
    tot = 0
    for dx, dy, dz in FORWARD_OFFSETS:
        tot += n(nx, dx) * n(ny, dy) * n(nz, dz)
    return int(tot)


def _system(x, ij, L0, m, k, c, v=None, fixed=None, fext=None):
    N = x.shape[0]; S = ij.shape[0]
    sysd = dict(
        x=np.ascontiguousarray(x, np.float32),
        v=np.zeros((N, 3), np.float32) if v is None else np.ascontiguousarray(v, np.float32),
        m=np.full(N, m, np.float32) if np.isscalar(m) else np.ascontiguousarray(m, np.float32),
        fixed=np.zeros(N, np.uint8) if fixed is None else np.ascontiguousarray(fixed, np.uint8),
        ij=np.ascontiguousarray(ij, np.int32),
        k=np.full(S, k, np.float32) if np.isscalar(k) else np.ascontiguousarray(k, np.float32),
        c=np.full(S, c, np.float32) if np.isscalar(c) else np.ascontiguousarray(c, np.float32),
        L0=np.ascontiguousarray(L0, np.float32),
        freq=0.0,
    )
    if fext is not None:
        sysd["fext"] = np.ascontiguousarray(fext, np.float32)
    return sysd


def soft_cube(n: int = 10, a: float = 0.01, m: float = 1e-3, k: float = 1e4,
              c: float = 0.1, z0: float = 0.05):
    """Plain soft cube: n^3 nodes, spacing a, bottom face at height z0."""
    x, ij, L0 = box_lattice(n, n, n, a, origin=(0.0, 0.0, z0))
    return _system(x, ij, L0, m, k, c)


def soft_cube_params(contact: bool = True, **kw):
    p = params(dt=1e-4, k_c=1e5, mu=0.5 if contact else 0.0, contact=contact)
    p.update(kw)
    return p


def cantilever(nx: int = 40, ny: int = 4, nz: int = 4, a: float = 0.01,
               m: float = 1e-3, k: float = 1e4, c: float = 0.0,
               tip_load: float = 0.01):
    """Cantilever beam along +x, clamped (anchored) at the x=0 layer.

    The tip load [N] acts in -z, split evenly over the nodes of the x=max
    layer.  Gravity is expected to be off for this workload.
    """
    x, ij, L0 = box_lattice(nx, ny, nz, a)
    N = x.shape[0]
    ixs = np.arange(N) % nx
    fixed = (ixs == 0).astype(np.uint8)
    tip = ixs == nx - 1
    fext = np.zeros((N, 3), np.float32)
    fext[tip, 2] = np.float32(-tip_load / tip.sum())
    return _system(x, ij, L0, m, k, c, fixed=fixed, fext=fext)


def throughput_lattice(n: int = 256, a: float = 1e-3, m: float = 1e-3,
                       k_range=(5e3, 5e4), c: float = 0.05,
                       v_sigma: float = 1e-3, seed_k: int = 0, seed_v: int = 1):
    """Plain throughput lattice: n^3 nodes, per-spring k ~ U[k_range] (seed_k),
    uniform damping c, bottom (z=0) layer anchored, free-node velocities
    ~ N(0, v_sigma) per component (seed_v)."""
    x, ij, L0 = box_lattice(n, n, n, a)
    N = x.shape[0]; S = ij.shape[0]
    rk = np.random.default_rng(seed_k)
    k = rk.random(S, dtype=np.float32)
    k *= np.float32(k_range[1] - k_range[0]); k += np.float32(k_range[0])
    fixed = (np.arange(N) < n * n).astype(np.uint8)
    rv = np.random.default_rng(seed_v)
    v = rv.standard_normal((N, 3), dtype=np.float32) * np.float32(v_sigma)
    v[fixed.astype(bool)] = 0.0
    sysd = _system(x, ij, L0, m, k, np.float32(c), v=v, fixed=fixed)
    sysd["c_uniform"] = float(np.float32(c))
    return sysd


def throughput_params(**kw):
    p = params(dt=5e-5, contact=False)
    p.update(kw)
    return p


# ---------------------------------------------------------------------------
# Voxel robots (batched population, differentiable walkers, surrogate designs)
# ---------------------------------------------------------------------------

# Material table for voxel robots: index -> (k [N/m], c [N s/m], actuation amplitude)
# 0 = empty voxel.  Actuated voxels oscillate their springs' rest length by
# factor (1 + 0.2 sin(2 pi 2Hz t + phi)).
VOXEL_MATERIALS = np.array([
    (0.0, 0.0, 0.0),      # empty
    (1e3, 0.1, 0.0),      # soft
    (1e5, 0.1, 0.0),      # stiff
    (5e3, 0.1, 0.2),      # actuated
], dtype=np.float64)
VOXEL_FREQ = 2.0          # Hz
VOXEL_EDGE = 0.01         # m
VOXEL_MASS = 0.03         # kg per voxel, 1/8 to each corner


def voxel_params(**kw):
    p = params(dt=1e-4, k_c=1e5, mu=0.7, contact=True)
    p.update(kw)
    return p


def _largest_component(occ: np.ndarray) -> np.ndarray:
    """Largest 6-face-connected component of a boolean voxel grid; ties go to
    the component containing the lowest linear voxel index (scipy numbers
    components in raster order of their first voxel)."""
    from scipy import ndimage
    lab, n = ndimage.label(occ, structure=ndimage.generate_binary_structure(3, 1))
    if n == 0:
        return np.zeros(occ.shape, bool)
    sizes = np.bincount(lab.ravel())[1:]
    best = int(np.argmax(sizes)) + 1
    return lab == best


def largest_components(mats: np.ndarray, chunk: int = 32768) -> np.ndarray:
    """Each design of a batch [n, nz, ny, nx] of material ids reduced to its
    largest 6-face-connected component of non-empty voxels (the rest set to
    0), ties to the component met first in raster order -- the rule of
    _largest_component, applied to many designs at once (one labelling per
    chunk, with no connectivity across designs)."""
    from scipy import ndimage
    mats = np.asarray(mats, np.uint8)
    out = np.zeros_like(mats)
    face = np.zeros((3, 3, 3, 3), bool)
    face[1] = ndimage.generate_binary_structure(3, 1)       # neighbours within one design only
    per = int(np.prod(mats.shape[1:]))
    for s0 in range(0, len(mats), chunk):
        part = mats[s0:s0 + chunk]
        lab, n = ndimage.label(part > 0, structure=face)
        if n == 0:
            continue
        flat = lab.reshape(len(part), per)
        sizes = np.bincount(flat.ravel(), minlength=n + 1)
        # labels are numbered in raster order and designs are the outermost
        # axis, so each design holds a contiguous range of labels
        top = np.maximum.accumulate(flat.max(axis=1))
        owner = np.searchsorted(top, np.arange(1, n + 1), side="left")
        # per design the label of most voxels, the lowest label on ties
        order = np.lexsort((np.arange(1, n + 1), -sizes[1:], owner))
        od = owner[order]
        head = np.flatnonzero(np.r_[True, od[1:] != od[:-1]])   # first entry per design after the sort
        best = np.zeros(len(part), np.int64)
        best[od[head]] = order[head] + 1
        keep = flat == best[:, None]
        out[s0:s0 + chunk] = np.where(keep.reshape(part.shape), part, 0)
    return out


def random_voxel_design(rng, dims):
    """One design: materials (nz,ny,nx) uint8 i.i.d. over {0,1,2,3} restricted
    to its largest connected component (resampled if empty), and phases
    uniform in [0, 2 pi)."""
    nx, ny, nz = dims
    while True:
        mat = rng.integers(0, 4, size=(nz, ny, nx)).astype(np.uint8)
        keep = _largest_component(mat > 0)
        if keep.any():
            break
    mat = np.where(keep, mat, 0).astype(np.uint8)
    phase = rng.uniform(0.0, 2 * np.pi, size=(nz, ny, nx)).astype(np.float32)
    return mat, phase


def voxel_population(n_robots: int = 4096, seed: int = 2, side_range=(3, 12)):
    """Batched design population: side lengths uniform in side_range (inclusive)
    independently per axis."""
    rng = np.random.default_rng(seed)
    designs = []
    for _ in range(n_robots):
        dims = tuple(int(s) for s in rng.integers(side_range[0], side_range[1] + 1, size=3))
        designs.append(random_voxel_design(rng, dims))
    return designs


def walker_designs(n_robots: int = 256, seed: int = 3, side: int = 8):
    rng = np.random.default_rng(seed)
    return [random_voxel_design(rng, (side, side, side)) for _ in range(n_robots)]


def surrogate_phase_field(side: int = 8):
    """Fixed travelling-wave phase field phi(x) = 2 pi x / side shared by all
    surrogate designs, so that a design's label is a function of its
    materials alone."""
    xs = (2 * np.pi * np.arange(side) / side).astype(np.float32)
    return np.broadcast_to(xs[None, None, :], (side, side, side)).copy()


def surrogate_designs(n: int, seed: int = 4, side: int = 8):
    """Surrogate training/screening designs: materials only (phase field fixed)."""
    rng = np.random.default_rng(seed)
    out = np.empty((n, side, side, side), np.uint8)
    for r in range(n):
        mat, _ = random_voxel_design(rng, (side, side, side))
        out[r] = mat
    return out


# ---------------------------------------------------------------------------
# Quasi-uniform lattice (Generating a Lattice: Mitchell's best-candidate
# sampling -- each new vertex is the best of `candidates` random points, the
# one whose k nearest existing vertices are farthest away)
# ---------------------------------------------------------------------------

def best_candidate_points(n: int, box=(1.0, 1.0, 1.0), candidates: int = 100, k_nearest: int = 1,
                          seed: int = 0):
    """n points in the box [0, box) by best-candidate sampling.  The score of
    a candidate is the distance to its k-th nearest accepted point."""
    rng = np.random.default_rng(seed)
    box = np.asarray(box, np.float64)
    pts = np.empty((n, 3))
    pts[0] = rng.random(3) * box
    for q in range(1, n):
        cand = rng.random((candidates, 3)) * box
        d = np.sqrt(((cand[:, None, :] - pts[None, :q, :]) ** 2).sum(axis=2))
        kk = min(k_nearest, q)
        score = np.partition(d, kk - 1, axis=1)[:, kk - 1]
        pts[q] = cand[int(np.argmax(score))]
    return pts


def quasi_uniform_lattice(n: int = 2000, box=(0.1, 0.1, 0.1), cutoff_factor: float = 1.6,
                          max_degree: int = 26, seed: int = 0, m: float = 1e-3, k: float = 1e4,
                          c: float = 0.05, candidates: int = 100):
    """Irregular spring network on best-candidate points: every pair closer than
    cutoff_factor x (the mean nearest-neighbour distance) is linked, keeping at
    most max_degree shortest springs per node.  Rest lengths are the initial
    distances (rounded to float32)."""
    pts = best_candidate_points(n, box, candidates=candidates, seed=seed)
    d = np.sqrt(((pts[:, None, :] - pts[None, :, :]) ** 2).sum(axis=2))
    np.fill_diagonal(d, np.inf)
    nn = d.min(axis=1).mean()
    cutoff = cutoff_factor * nn
    keep = np.zeros_like(d, dtype=bool)
    for i in range(n):
        cand = np.flatnonzero(d[i] < cutoff)
        cand = cand[np.argsort(d[i, cand])][:max_degree]
        keep[i, cand] = True
    keep &= keep.T                                   # mutual: both ends within their degree cap
    iu, ju = np.nonzero(np.triu(keep, 1))
    ij = np.stack([iu, ju], axis=1).astype(np.int32)
    x = pts.astype(np.float32)
    L0 = np.sqrt(((x[ij[:, 1]].astype(np.float64) - x[ij[:, 0]]) ** 2).sum(axis=1)).astype(np.float32)
    return _system(x, ij, L0, m, k, c)
