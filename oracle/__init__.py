"""CPU oracle for the mass-spring step (FP64).  TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline / reference
legs may import this package.  The GPU library never does, and this package
never imports the library: the two share no code.  The numerical work lives
in ``ms_oracle.c`` (plain C, FP64, springs summed in index order); this file
builds it with gcc, marshals numpy arrays into it and adds the small plain
definitions that sit around the step: energies, the centre of mass and the
voxel-robot lattice.  ``oracle/mlp.py`` holds the MLP of the surrogate.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ms_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libms_oracle.so")
_lock = threading.Lock()
_lib = None

INTEGRATORS = {"symplectic_euler": 0, "forward_euler": 1, "verlet": 2, "rk4": 3}


class OraParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("g", C.c_double * 3), ("k_c", C.c_double),
                ("mu", C.c_double), ("vel_damping", C.c_double), ("freq", C.c_double),
                ("contact_on", C.c_int32), ("integrator", C.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                "-o", tmp, _SRC, "-lm"]
        try:        # OpenMP only serves ora_run_threads (timing on all host cores)
            subprocess.check_call(base + ["-fopenmp"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            l.ora_run.restype = C.c_int
            l.ora_run.argtypes = [C.POINTER(OraParams), C.c_int64, dp, dp, dp, C.c_void_p, C.c_void_p,
                                  C.c_int64, C.c_void_p, dp, dp, dp, C.c_void_p, C.c_void_p,
                                  C.c_int64, C.c_int64]
            l.ora_run_threads.restype = C.c_int
            l.ora_run_threads.argtypes = l.ora_run.argtypes + [C.c_int32, C.POINTER(C.c_int32)]
            _lib = l
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(params: dict, freq: float = 0.0, integrator="symplectic_euler") -> OraParams:
    p = OraParams()
    p.dt = float(params["dt"])
    for a in range(3):
        p.g[a] = float(params["g"][a])
    p.k_c = float(params.get("k_c", 0.0))
    p.mu = float(params.get("mu", 0.0))
    p.vel_damping = float(params.get("vel_damping", 0.0))
    p.freq = float(freq)
    p.contact_on = 1 if params.get("contact", False) else 0
    p.integrator = INTEGRATORS[integrator] if isinstance(integrator, str) else int(integrator)
    return p


class _Arrays:
    """FP64 copies of a system's constant arrays, kept alive for the C calls."""

    def __init__(self, system: dict):
        N = system["x"].shape[0]; S = system["ij"].shape[0]
        self.N, self.S = N, S
        self.m = _f64(system["m"])
        self.fixed = np.ascontiguousarray(system["fixed"], np.uint8)
        self.fext = _f64(system["fext"], (N, 3)) if system.get("fext") is not None else None
        self.ij = np.ascontiguousarray(system["ij"], np.int32).reshape(S, 2)
        self.k = _f64(system["k"])
        c = system["c"]
        self.c = _f64(np.broadcast_to(np.asarray(c, np.float64), (S,)))
        self.L0 = _f64(system["L0"])
        if system.get("A") is not None:
            self.A = _f64(system["A"]); self.phi = _f64(system["phi"])
        else:
            self.A = self.phi = None
        self.freq = float(system.get("freq", 0.0))


def run(system: dict, params: dict, nsteps: int, n0: int = 0, x=None, v=None,
        integrator="symplectic_euler", arrays: _Arrays | None = None):
    """Advance a system nsteps steps from step index n0; returns (x, v) FP64.

    The start state defaults to the system's (float32) x, v widened to FP64.
    """
    ar = arrays or _Arrays(system)
    N = ar.N
    x = _f64(system["x"] if x is None else x, (N, 3)).copy()
    v = _f64(system["v"] if v is None else v, (N, 3)).copy()
    p = make_params(params, ar.freq, integrator)
    rc = lib().ora_run(C.byref(p), N, _dptr(x), _dptr(v), _dptr(ar.m), _ptr(ar.fixed), _ptr(ar.fext),
                       ar.S, _ptr(ar.ij), _dptr(ar.k), _dptr(ar.c), _dptr(ar.L0), _ptr(ar.A), _ptr(ar.phi),
                       int(n0), int(nsteps))
    if rc != 0:
        raise RuntimeError(f"ora_run failed with code {rc}")
    return x, v


def run_threads(system: dict, params: dict, nsteps: int, threads: int, n0: int = 0, x=None, v=None,
                arrays: _Arrays | None = None):
    """run() on `threads` host threads (symplectic Euler only), for timing the
    oracle on all cores.  Each thread owns a block of masses and sums their
    springs in spring-index order, so the result equals run() bit for bit.
    Returns (x, v, threads actually used)."""
    ar = arrays or _Arrays(system)
    N = ar.N
    x = _f64(system["x"] if x is None else x, (N, 3)).copy()
    v = _f64(system["v"] if v is None else v, (N, 3)).copy()
    p = make_params(params, ar.freq)
    used = C.c_int32(0)
    rc = lib().ora_run_threads(C.byref(p), N, _dptr(x), _dptr(v), _dptr(ar.m), _ptr(ar.fixed), _ptr(ar.fext),
                               ar.S, _ptr(ar.ij), _dptr(ar.k), _dptr(ar.c), _dptr(ar.L0), _ptr(ar.A),
                               _ptr(ar.phi), int(n0), int(nsteps), int(threads), C.byref(used))
    if rc != 0:
        raise RuntimeError(f"ora_run_threads failed with code {rc}")
    return x, v, int(used.value)


# ---------------------------------------------------------------------------
# Energies (Energy Conservation Tests section: elastic, gravitational and
# kinetic energy), centre of mass
# ---------------------------------------------------------------------------

def energy(system: dict, params: dict, x, v, t: float = 0.0):
    """(kinetic, elastic, gravitational, ground-penalty) energy, FP64."""
    x = _f64(x); v = _f64(v)
    m = _f64(system["m"])
    ij = np.asarray(system["ij"])
    ke = 0.5 * float(np.sum(m[:, None] * v * v))
    d = x[ij[:, 1]] - x[ij[:, 0]]
    l = np.sqrt(np.sum(d * d, axis=1))
    L = _f64(system["L0"])
    if system.get("A") is not None:
        L = L * (1.0 + _f64(system["A"]) * np.sin(2 * np.pi * system.get("freq", 0.0) * t + _f64(system["phi"])))
    pe = 0.5 * float(np.sum(_f64(system["k"]) * (l - L) ** 2))
    g = np.asarray(params["g"], np.float64)
    gpe = -float(np.sum(m[:, None] * x * g[None, :]))
    cpe = 0.0
    if params.get("contact", False):
        z = x[:, 2]
        cpe = 0.5 * float(params["k_c"]) * float(np.sum(np.where(z < 0, z * z, 0.0)))
    return ke, pe, gpe, cpe


def centre_of_mass(m, x):
    m = _f64(m); x = _f64(x)
    return (m[:, None] * x).sum(axis=0) / m.sum()


# ---------------------------------------------------------------------------
# Voxel robots: the voxel lattice of the "Generating a Lattice" section, one
# spring per pair of corners of every non-empty voxel (12 edges, 12 face
# diagonals, 4 body diagonals = all 28 corner pairs), springs of neighbouring
# voxels kept as separate parallel springs.
# ---------------------------------------------------------------------------

def voxel_system(mat, phase, materials, freq: float, a: float, voxel_mass: float,
                 logk=None):
    """Expand one voxel design into an unmerged mass-spring system.

    mat (nz,ny,nx) uint8 material ids (0 = empty); phase (nz,ny,nx) phases;
    materials[id] = (k, c, amplitude).  logk, if given, overrides each
    voxel's stiffness as k = exp(logk[voxel]).  Corner masses are numbered in
    raster order (x fastest) of the (nx+1)(ny+1)(nz+1) corner grid, keeping
    only corners of non-empty voxels.  Each corner receives voxel_mass / 8
    from every non-empty voxel it touches.  Positions start at ix*a etc. so
    that the lowest corners sit on z = 0.
    Returns the system dict plus 'spring_voxel' (S,) = flat voxel index of
    each spring and 'corner_of' (used corner raster ids).
    """
    mat = np.asarray(mat)
    nz, ny, nx = mat.shape
    cx, cy, cz = nx + 1, ny + 1, nz + 1
    used = np.zeros(cx * cy * cz, bool)
    cmass = np.zeros(cx * cy * cz)
    corners = [(dx, dy, dz) for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]
    pairs = [(p, q) for p in range(8) for q in range(p + 1, 8)]
    assert len(pairs) == 28
    vox = [(iz, iy, ix) for iz in range(nz) for iy in range(ny) for ix in range(nx) if mat[iz, iy, ix] > 0]
    for iz, iy, ix in vox:
        for dx, dy, dz in corners:
            cid = (ix + dx) + cx * ((iy + dy) + cy * (iz + dz))
            used[cid] = True
            cmass[cid] += voxel_mass / 8.0
    cid_used = np.flatnonzero(used)
    remap = -np.ones(cx * cy * cz, np.int64)
    remap[cid_used] = np.arange(cid_used.size)
    N = cid_used.size
    cz_, rem = np.divmod(cid_used, cx * cy)
    cy_, cx_ = np.divmod(rem, cx)
    x = np.stack([cx_ * a, cy_ * a, cz_ * a], axis=1).astype(np.float32)
    ij, k, c, L0, A, ph, sv = [], [], [], [], [], [], []
    for iz, iy, ix in vox:
        mid = int(mat[iz, iy, ix])
        kv, cv, av = materials[mid]
        vflat = ix + nx * (iy + ny * iz)
        if logk is not None:
            kv = float(np.exp(np.asarray(logk).ravel()[vflat]))
        for p, q in pairs:
            P, Q = corners[p], corners[q]
            ci = (ix + P[0]) + cx * ((iy + P[1]) + cy * (iz + P[2]))
            cj = (ix + Q[0]) + cx * ((iy + Q[1]) + cy * (iz + Q[2]))
            ij.append((remap[ci], remap[cj]))
            nsq = sum((P[t] - Q[t]) ** 2 for t in range(3))
            L0.append(np.float32(a * np.sqrt(float(nsq))))
            k.append(kv); c.append(cv); A.append(av)
            ph.append(float(np.asarray(phase).ravel()[vflat]))
            sv.append(vflat)
    sysd = dict(
        x=x, v=np.zeros((N, 3), np.float32), m=cmass[cid_used].astype(np.float64),
        fixed=np.zeros(N, np.uint8), ij=np.asarray(ij, np.int32).reshape(-1, 2),
        k=np.asarray(k, np.float64), c=np.asarray(c, np.float64),
        L0=np.asarray(L0, np.float32), A=np.asarray(A, np.float64),
        phi=np.asarray(ph, np.float64), freq=float(freq),
        spring_voxel=np.asarray(sv, np.int64), corner_of=cid_used,
    )
    return sysd
