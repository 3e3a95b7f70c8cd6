"""FP64 CPU oracle for the D3Q19 + immersed-boundary step (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is a plain, slow, double-precision
restatement of the method of Gusenbauer et al. (arXiv:1110.0995), Sec. 2.1-2.4,
compiled from ``lbibm_oracle.cpp`` with g++ (no CUDA, nothing shared with the
GPU library).  See the header of ``lbibm_oracle.cpp`` for the readings taken
where the paper prints no formula.

Parity status per function (what pins it, in ``tests/test_oracle_*.py``):

* equilibrium, Guo source       : exact moment identities (rational arithmetic)
* lb_step (stream/collide/walls): rest state, mass and momentum bookkeeping,
                                  exact discrete plane-Poiseuille solution,
                                  Couette, duct Fourier series (2nd order)
* rasterise                     : brute-force sphere membership
* stencil / spread / interpolate: partition of unity, first moment, adjointness,
                                  exact interpolation of linear fields
* area_volume                   : sphere area/volume limits, translation invariance
* force_stretch                 : Hookean limit kappa(1) = 1, hand-computed values,
                                  momentum / angular momentum, rest state
* force_bend                    : central finite differences of an independently
                                  computed bending energy (arccos form)
* force_area (local / global)   : exact gradient on equilateral triangles, finite
                                  differences of the global energy on a sphere
                                  under homocentric scaling, invariants
* force_volume                  : finite differences of the volume energy
* system_step (coupled cycle)   : a cell in uniform flow translates rigidly
* DiffProblem (differentiable   : dual-number derivatives vs central finite
  variant, Brinkman beads)        differences; phi = 0 reproduces the plain cycle;
                                  phi = 1 with alpha = 2 holds u at g / 2
* repulsion (Sec. 2.4)          : forces are minus the gradient of the pair
                                  potential (finite differences), cell-cell sums
                                  conserve momentum, cut-off and periodic image
* drag_coefficients,            : p1 and e^-a against 40-digit values; one step in
  system_step_massive             uniform flow against the closed form; total
  (IB points with mass)           momentum conserved; gamma = 0 leaves the fluid at
                                  rest; the massless limit's first cycle
* dipole_force, bead_forces,    : axial attraction / transverse repulsion of two
  bead_relax (Sec. 2.5)           dipoles, minus the gradient of the dipole energy,
                                  third law, minimum image, a pair relaxing to its
                                  force balance
* coupled-cycle stability       : the explicit coupling amplifies perturbations
                                  of a stiff membrane and damps a soft one
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbibm_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (portable flags, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           _SRC, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        P = ctypes.c_void_p
        L.or_sys_create.restype = vp
        L.or_sys_create.argtypes = [i, i, i, d, P, P, P]
        L.or_sys_destroy.argtypes = [vp]
        L.or_sys_set_solid.argtypes = [vp, P]
        L.or_sys_set_extra_force.argtypes = [vp, P]
        L.or_sys_set_repulsion.argtypes = [vp, d, d, P, i]
        L.or_sys_init_equilibrium.argtypes = [vp, d, P]
        L.or_sys_get_f.argtypes = [vp, P]
        L.or_sys_set_f.argtypes = [vp, P]
        L.or_sys_get_fields.argtypes = [vp, P, P]
        L.or_sys_add_mesh.restype = i
        L.or_sys_add_mesh.argtypes = [vp, P, i, P, i, P]
        L.or_sys_set_nodes.argtypes = [vp, i, P]
        L.or_sys_get_nodes.argtypes = [vp, i, P]
        L.or_sys_get_forces.argtypes = [vp, i, P]
        L.or_sys_set_dynamics.restype = i
        L.or_sys_set_dynamics.argtypes = [vp, d, d]
        L.or_sys_get_velocities.argtypes = [vp, i, P]
        L.or_drag_coefficients.argtypes = [d, d, P]
        L.or_dipole_force.argtypes = [P, P, P, d, P]
        L.or_dipole_energy.restype = d
        L.or_dipole_energy.argtypes = [P, P, P, d]
        L.or_bead_forces.argtypes = [P, P, i, P, P, P]
        L.or_bead_relax.argtypes = [P, P, i, P, P, i]
        L.or_sys_step.argtypes = [vp, i]
        L.or_constants.argtypes = [P, P, P]
        L.or_equilibrium.argtypes = [d, P, P]
        L.or_guo_source.argtypes = [d, P, P, P]
        L.or_rasterise_spheres.argtypes = [P, i, i, i, i, P]
        L.or_mesh_area_volume.restype = i
        L.or_mesh_area_volume.argtypes = [P, i, P, i, P, P]
        L.or_mesh_edges.restype = i
        L.or_mesh_edges.argtypes = [P, i, i, P, P]
        L.or_mesh_forces.restype = i
        L.or_mesh_forces.argtypes = [P, P, i, P, i, P, i, P]
        L.or_dihedral.restype = d
        L.or_dihedral.argtypes = [P, P, P, P]
        L.or_spread.argtypes = [vp, P, P, i, P]
        L.or_interpolate.argtypes = [vp, P, i, P, P]
        L.or_diff_create.restype = vp
        L.or_diff_create.argtypes = [i, i, i, d, P, P, i, P, d, d]
        L.or_diff_destroy.argtypes = [vp]
        L.or_diff_add_mesh.restype = i
        L.or_diff_add_mesh.argtypes = [vp, P, i, P, i, P]
        L.or_diff_run.restype = d
        L.or_diff_run.argtypes = [vp, i, i, i, i, P]
        L.or_diff_state.restype = d
        L.or_diff_state.argtypes = [vp, i, i, P, P]
        L.or_diff_phi.argtypes = [vp, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


TERM_STRETCH, TERM_BEND, TERM_AREA_LOCAL, TERM_AREA_GLOBAL, TERM_VOLUME = 1, 2, 4, 8, 16
TERM_ALL = 31


def constants():
    e = np.zeros((19, 3), np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, np.int32)
    lib().or_constants(_p(e), _p(w), _p(opp))
    return e, w, opp


def equilibrium(rho: float, u) -> np.ndarray:
    out = np.zeros(19)
    lib().or_equilibrium(float(rho), _p(_f64(u)), _p(out))
    return out


def guo_source(tau: float, u, g) -> np.ndarray:
    out = np.zeros(19)
    lib().or_guo_source(float(tau), _p(_f64(u)), _p(_f64(g)), _p(out))
    return out


def drag_coefficients(m: float, gamma: float):
    """(a, p1, E) of the exact drag drift of IB points with mass (a = gamma / m,
    p1 = (1 - e^-a) / a, E = e^-a)."""
    out = np.zeros(3)
    lib().or_drag_coefficients(float(m), float(gamma), _p(out))
    return tuple(out)


def dipole_force(m1, m2, r, c: float) -> np.ndarray:
    """Force on bead 2 from bead 1 (Sec. 2.5), r = x2 - x1, c = mu0 / (4 pi)."""
    F = np.zeros(3)
    lib().or_dipole_force(_p(_f64(m1)), _p(_f64(m2)), _p(_f64(r)), float(c), _p(F))
    return F


def dipole_energy(m1, m2, r, c: float) -> float:
    return float(lib().or_dipole_energy(_p(_f64(m1)), _p(_f64(m2)), _p(_f64(r)), float(c)))


def _bead_params(c, radius, k, mobility, dt, box, periodic):
    pr = _f64([c, radius, k, mobility, dt, *box])
    per = np.ascontiguousarray(periodic, dtype=np.int32)
    return pr, per


def bead_forces(x, m, c, radius, k, box=(1, 1, 1), periodic=(0, 0, 0)) -> np.ndarray:
    """Dipole + contact forces on every bead (n x 3)."""
    xx, mm = _f64(x), _f64(m)
    pr, per = _bead_params(c, radius, k, 0.0, 0.0, box, periodic)
    F = np.zeros_like(xx)
    lib().or_bead_forces(_p(xx), _p(mm), int(xx.shape[0]), _p(pr), _p(per), _p(F))
    return F


def bead_relax(x, m, c, radius, k, mobility, dt, steps, box=(1, 1, 1), periodic=(0, 0, 0)) -> np.ndarray:
    """Overdamped bead assembly: positions after `steps` steps."""
    xx = _f64(x).copy()
    mm = _f64(m)
    pr, per = _bead_params(c, radius, k, mobility, dt, box, periodic)
    lib().or_bead_relax(_p(xx), _p(mm), int(xx.shape[0]), _p(pr), _p(per), int(steps))
    return xx


def rasterise(spheres: np.ndarray, dims) -> np.ndarray:
    nx, ny, nz = dims
    sph = np.ascontiguousarray(spheres, dtype=np.float32).reshape(-1, 4)
    out = np.zeros(nx * ny * nz, np.uint8)
    lib().or_rasterise_spheres(_p(sph), int(sph.shape[0]), nx, ny, nz, _p(out))
    return out


def mesh_area_volume(x: np.ndarray, tris: np.ndarray):
    S = ctypes.c_double()
    V = ctypes.c_double()
    xx = _f64(x)
    tt = np.ascontiguousarray(tris, dtype=np.int32)
    rc = lib().or_mesh_area_volume(_p(xx), int(xx.shape[0]), _p(tt), int(tt.shape[0]),
                                   ctypes.byref(S), ctypes.byref(V))
    if rc != 0:
        raise ValueError("mesh is not a closed oriented manifold")
    return S.value, V.value


def mesh_edges(tris: np.ndarray, n: int) -> np.ndarray:
    tt = np.ascontiguousarray(tris, dtype=np.int32)
    ne = ctypes.c_int()
    rc = lib().or_mesh_edges(_p(tt), int(tt.shape[0]), int(n), None, ctypes.byref(ne))
    if rc != 0:
        raise ValueError("mesh is not a closed oriented manifold")
    out = np.zeros((ne.value, 4), np.int32)
    lib().or_mesh_edges(_p(tt), int(tt.shape[0]), int(n), _p(out), ctypes.byref(ne))
    return out


def mesh_forces(x: np.ndarray, x0: np.ndarray, tris: np.ndarray, moduli, terms: int = TERM_ALL) -> np.ndarray:
    xx, x00 = _f64(x), _f64(x0)
    tt = np.ascontiguousarray(tris, dtype=np.int32)
    F = np.zeros_like(xx)
    rc = lib().or_mesh_forces(_p(xx), _p(x00), int(xx.shape[0]), _p(tt), int(tt.shape[0]),
                              _p(_f64(moduli)), int(terms), _p(F))
    if rc != 0:
        raise ValueError("mesh is not a closed oriented manifold")
    return F


def dihedral(xa, xb, xc, xd) -> float:
    return lib().or_dihedral(_p(_f64(xa)), _p(_f64(xb)), _p(_f64(xc)), _p(_f64(xd)))


class System:
    """FP64 lattice + cells; one ``step`` is one immersed-boundary cycle."""

    def __init__(self, dims, tau=1.0, body_force=(0, 0, 0), periodic=(1, 0, 0),
                 wall_velocity=((0, 0, 0), (0, 0, 0)), solid: Optional[np.ndarray] = None):
        self.dims = tuple(int(v) for v in dims)
        self.N = self.dims[0] * self.dims[1] * self.dims[2]
        self._G = _f64(body_force)
        self._per = np.ascontiguousarray(periodic, dtype=np.int32)
        self._uw = _f64(np.asarray(wall_velocity, dtype=np.float64).reshape(6))
        h = lib().or_sys_create(*self.dims, float(tau), _p(self._G), _p(self._per), _p(self._uw))
        if not h:
            raise ValueError("invalid lattice parameters")
        self._h = h
        self.n_nodes = []
        if solid is not None:
            self.set_solid(solid)

    @classmethod
    def from_scene(cls, scene) -> "System":
        s = cls(scene.dims, scene.tau, scene.body_force, scene.periodic, scene.wall_velocity)
        if len(scene.spheres):
            s.set_solid(rasterise(scene.spheres, scene.dims))
        for m in scene.meshes:
            s.add_mesh(m.rest, m.tris, m.moduli)
        rep = getattr(scene, "repulsion", None)
        if rep is not None:
            s.set_repulsion(rep[0], rep[1], scene.spheres)
        dyn = getattr(scene, "ib_dynamics", None)
        if dyn is not None:
            s.set_dynamics(dyn[0], dyn[1])
        return s

    def set_repulsion(self, k: float, dc: float, spheres=None):
        """Soft-sphere collisions (Sec. 2.4 reading): force k (dc - d) below separation dc."""
        sph = _f64(np.zeros((0, 4)) if spheres is None else spheres).reshape(-1, 4)
        self._sph = sph
        lib().or_sys_set_repulsion(self._h, float(k), float(dc), _p(sph), int(sph.shape[0]))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_sys_destroy(h)
            self._h = None

    def set_solid(self, solid: np.ndarray):
        s = np.ascontiguousarray(solid, dtype=np.uint8).reshape(self.N)
        self.solid = s.copy()
        lib().or_sys_set_solid(self._h, _p(s))

    def set_extra_force(self, g: Optional[np.ndarray]):
        if g is None:
            lib().or_sys_set_extra_force(self._h, None)
        else:
            gg = _f64(g).reshape(3 * self.N)
            lib().or_sys_set_extra_force(self._h, _p(gg))

    def init_equilibrium(self, rho=1.0, u=(0, 0, 0)):
        lib().or_sys_init_equilibrium(self._h, float(rho), _p(_f64(u)))

    def get_f(self) -> np.ndarray:
        f = np.zeros((19, self.N))
        lib().or_sys_get_f(self._h, _p(f))
        return f

    def set_f(self, f: np.ndarray):
        ff = _f64(f).reshape(19 * self.N)
        lib().or_sys_set_f(self._h, _p(ff))

    def fields(self):
        rho = np.zeros(self.N)
        u = np.zeros((3, self.N))
        lib().or_sys_get_fields(self._h, _p(rho), _p(u))
        return rho, u

    def add_mesh(self, x0, tris, moduli) -> int:
        xx = _f64(x0)
        tt = np.ascontiguousarray(tris, dtype=np.int32)
        m = lib().or_sys_add_mesh(self._h, _p(xx), int(xx.shape[0]), _p(tt), int(tt.shape[0]), _p(_f64(moduli)))
        if m < 0:
            raise ValueError("mesh rejected (not closed/oriented or non-positive volume)")
        self.n_nodes.append(int(xx.shape[0]))
        return m

    def set_nodes(self, m: int, x):
        lib().or_sys_set_nodes(self._h, m, _p(_f64(x)))

    def nodes(self, m: int) -> np.ndarray:
        x = np.zeros((self.n_nodes[m], 3))
        lib().or_sys_get_nodes(self._h, m, _p(x))
        return x

    def forces(self, m: int) -> np.ndarray:
        F = np.zeros((self.n_nodes[m], 3))
        lib().or_sys_get_forces(self._h, m, _p(F))
        return F

    def set_dynamics(self, m: float, gamma: float):
        """IB points with mass m and drag gamma (Sec. 2.2 reading B); m = 0: massless."""
        if lib().or_sys_set_dynamics(self._h, float(m), float(gamma)) != 0:
            raise ValueError("mass and drag must be finite and >= 0")

    def velocities(self, m: int) -> np.ndarray:
        """Point velocities after the last step's drift (W)."""
        v = np.zeros((self.n_nodes[m], 3))
        lib().or_sys_get_velocities(self._h, m, _p(v))
        return v

    def step(self, n: int = 1):
        lib().or_sys_step(self._h, int(n))

    def spread(self, X, Fn) -> np.ndarray:
        XX, FF = _f64(X), _f64(Fn)
        g = np.zeros(3 * self.N)
        lib().or_spread(self._h, _p(XX), _p(FF), int(XX.shape[0]), _p(g))
        return g.reshape(3, self.N)

    def interpolate(self, X, u) -> np.ndarray:
        XX = _f64(X)
        uu = _f64(u).reshape(3 * self.N)
        U = np.zeros_like(XX)
        lib().or_interpolate(self._h, _p(XX), int(XX.shape[0]), _p(uu), _p(U))
        return U


SEED = {"bead": 1, "ks": 2, "kb": 3}


class DiffProblem:
    """The differentiable variant (Brinkman beads, see ``diff_run`` in
    lbibm_oracle.cpp): J = mean x displacement of the objective cell after T
    cycles from rest, and forward-mode derivatives of J (FP64 dual numbers)
    with respect to one bead coordinate, or the objective cell's ks or kb."""

    def __init__(self, dims, tau, body_force, periodic, beads, alpha=2.0, delta=0.5):
        self.dims = tuple(int(v) for v in dims)
        self.N = self.dims[0] * self.dims[1] * self.dims[2]
        self.beads = _f64(beads).reshape(-1, 4).copy()
        G = _f64(body_force)
        per = np.ascontiguousarray(periodic, dtype=np.int32)
        h = lib().or_diff_create(*self.dims, float(tau), _p(G), _p(per), int(self.beads.shape[0]),
                                 _p(self.beads), float(alpha), float(delta))
        if not h:
            raise ValueError("invalid problem")
        self._h = h
        self.n_nodes = []

    @classmethod
    def from_scene(cls, scene, alpha=2.0, delta=0.5, moduli=None) -> "DiffProblem":
        p = cls(scene.dims, scene.tau, scene.body_force, scene.periodic, np.asarray(scene.spheres, np.float64),
                alpha, delta)
        for k, m in enumerate(scene.meshes):
            p.add_mesh(m.rest, m.tris, m.moduli if moduli is None else moduli[k])
        return p

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_diff_destroy(h)
            self._h = None

    def add_mesh(self, x0, tris, moduli) -> int:
        xx = _f64(x0)
        tt = np.ascontiguousarray(tris, dtype=np.int32)
        m = lib().or_diff_add_mesh(self._h, _p(xx), int(xx.shape[0]), _p(tt), int(tt.shape[0]), _p(_f64(moduli)))
        if m < 0:
            raise ValueError("mesh rejected")
        self.n_nodes.append(int(xx.shape[0]))
        return m

    def run(self, steps: int, obj: int, seed=None):
        """J, or (J, dJ/dp) for seed = ("bead", 3 k + axis) / ("ks",) / ("kb",)."""
        if seed is None:
            return lib().or_diff_run(self._h, int(steps), int(obj), 0, 0, None)
        dJ = ctypes.c_double()
        J = lib().or_diff_run(self._h, int(steps), int(obj), SEED[seed[0]], int(seed[1]) if len(seed) > 1 else 0,
                              ctypes.byref(dJ))
        return J, dJ.value

    def state(self, steps: int, obj: int = 0):
        """(J, last velocity field 3 x N, every mesh's final positions concatenated)."""
        u = np.zeros(3 * self.N)
        x = np.zeros((sum(self.n_nodes), 3))
        J = lib().or_diff_state(self._h, int(steps), int(obj), _p(u), _p(x))
        return J, u.reshape(3, self.N), x

    def phi(self) -> np.ndarray:
        out = np.zeros(self.N)
        lib().or_diff_phi(self._h, _p(out))
        return out
