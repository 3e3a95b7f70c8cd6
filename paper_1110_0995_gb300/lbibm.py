"""Thin Python binding of the C ABI in ``include/lbibm.h`` (ctypes).

Argument marshalling only: every step of the method runs in the CUDA library
``_build/liblbibm.so``.  There is no CPU fallback; importing this module on a
machine without the compiled library raises.  PyTorch, when used, only
provides device buffers (``data_ptr``) and the CUDA stream handle.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import _build

LB_OK, LB_ERR_ARG, LB_ERR_STATE, LB_ERR_CUDA, LB_ERR_OOM, LB_ERR_NUMERIC, LB_ERR_TIMEOUT = range(7)
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}

# Every entry point that include/lbibm.h declares.
EXPORTS = (
    "lb_create", "lb_create_batch", "lb_select_channel", "lb_destroy", "lb_set_obstacles", "lb_set_brinkman", "lb_adjoint", "lb_set_repulsion", "lb_set_ib_dynamics", "lb_set_deterministic",
    "ibm_get_velocities", "ibm_add_mesh",
    "ibm_set_nodes", "lb_step", "lb_synchronize", "lb_get_fields", "lb_get_populations", "lb_set_populations",
    "ibm_get_nodes", "ibm_get_all_nodes", "ibm_get_forces", "ibm_get_area_volume", "lb_diagnostics", "lb_get_step", "lb_save_state",
    "lb_load_state", "lb_set_schedule", "lb_get_schedule", "lb_set_timing", "lb_kernel_times", "lb_last_error", "lb_version", "lb_get_mask",
    "lb_set_kernel_config", "lb_get_kernel_config", "lb_set_prefetch", "lb_get_prefetch", "lb_autotune",
    "ibm_area_volume_noalloc",
    "bead_forces", "bead_relax", "ibm_get_all_nodes_async", "lb_readback_wait", "ibm_check_mesh",
    "lb_set_guard_zones", "lb_check_guard_zones",
)


class LbParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("tau", ctypes.c_double),
                ("body_force", ctypes.c_double * 3), ("periodic", ctypes.c_int * 3),
                ("wall_velocity", (ctypes.c_double * 3) * 2), ("storage", ctypes.c_int),
                ("reserved", ctypes.c_int * 4)]


class IbmModuli(ctypes.Structure):
    _fields_ = [("ks", ctypes.c_double), ("kb", ctypes.c_double), ("kal", ctypes.c_double),
                ("kag", ctypes.c_double), ("kv", ctypes.c_double)]


class BeadParams(ctypes.Structure):
    _fields_ = [("mu0_4pi", ctypes.c_double), ("radius", ctypes.c_double), ("k_contact", ctypes.c_double),
                ("mobility", ctypes.c_double), ("dt", ctypes.c_double), ("box", ctypes.c_double * 3),
                ("periodic", ctypes.c_int * 3), ("reserved", ctypes.c_int * 5)]


class LbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lbibm status {status}: {msg}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load the compiled library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise ImportError(f"CUDA library not built: {_build.LIB} (run __graft_entry__.build())")
        L = ctypes.CDLL(_build.LIB)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        sig = {
            "lb_create": ([ctypes.POINTER(LbParams), P, ctypes.POINTER(P)], I),
            "lb_create_batch": ([ctypes.POINTER(LbParams), I, P, ctypes.POINTER(P)], I),
            "lb_select_channel": ([P, I], I),
            "lb_destroy": ([P], I),
            "lb_set_obstacles": ([P, P, I, P], I),
            "ibm_add_mesh": ([P, P, I, P, I, ctypes.POINTER(IbmModuli), ctypes.POINTER(I)], I),
            "ibm_set_nodes": ([P, I, P], I),
            "lb_step": ([P, I], I),
            "lb_synchronize": ([P], I),
            "lb_get_fields": ([P, P, P, I], I),
            "lb_get_populations": ([P, P], I),
            "lb_set_populations": ([P, P], I),
            "ibm_get_nodes": ([P, I, P], I),
            "ibm_get_all_nodes": ([P, P], I),
            "ibm_get_forces": ([P, I, P], I),
            "ibm_get_area_volume": ([P, P, P], I),
            "lb_diagnostics": ([P, D, P], I),
            "lb_get_step": ([P, ctypes.POINTER(ctypes.c_int64)], I),
            "lb_save_state": ([P, P, ctypes.POINTER(ctypes.c_size_t)], I),
            "lb_load_state": ([P, P, ctypes.c_size_t], I),
            "lb_set_timing": ([P, I], I),
            "lb_set_brinkman": ([P, P, I, D, D], I),
            "lb_set_repulsion": ([P, D, D], I),
            "lb_set_ib_dynamics": ([P, D, D], I),
            "lb_set_deterministic": ([P, I], I),
            "ibm_get_velocities": ([P, I, P], I),
            "lb_adjoint": ([P, I, I, I, P, P, P, P], I),
            "lb_set_schedule": ([P, I], I),
            "lb_get_schedule": ([P, P], I),
            "lb_kernel_times": ([P, P, P], I),
            "lb_last_error": ([P], ctypes.c_char_p),
            "lb_version": ([], I),
            "lb_get_mask": ([P, P], I),
            "lb_set_kernel_config": ([P, I, I], I),
            "lb_get_kernel_config": ([P, ctypes.POINTER(I), ctypes.POINTER(I)], I),
            "lb_set_prefetch": ([P, I], I),
            "lb_set_guard_zones": ([ctypes.c_size_t], I),
            "lb_check_guard_zones": ([P, I, ctypes.POINTER(ctypes.c_int64)], I),
            "lb_get_prefetch": ([P, ctypes.POINTER(I)], I),
            "lb_autotune": ([P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D)], I),
            "ibm_area_volume_noalloc": ([P, P, P, P, I, P, P, P], I),
            "bead_forces": ([P, P, I, P, P, P], I),
            "ibm_get_all_nodes_async": ([P, P, I], I),
            "lb_readback_wait": ([P, I], I),
            "bead_relax": ([P, P, I, P, I, P], I),
            "ibm_check_mesh": ([P, I, P, I, ctypes.c_char_p, I], I),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def last_error() -> str:
    """Message of this thread's last failed call that has no context."""
    return lib().lb_last_error(None).decode()


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64_out(out: np.ndarray, n_points: int) -> np.ndarray:
    """Check a caller's output buffer for n_points x 3 doubles before the
    library writes into it: float64, C-contiguous, writable and large enough."""
    if not isinstance(out, np.ndarray) or out.dtype != np.float64 or not out.flags.c_contiguous \
            or not out.flags.writeable:
        raise ValueError("output buffer must be a writable C-contiguous float64 array")
    if out.size < 3 * n_points:
        raise ValueError(f"output buffer holds {out.size} doubles, {3 * n_points} needed")
    return out


def _f64_in(xyz, n_points: int) -> np.ndarray:
    """n_points x 3 doubles, C-contiguous; raises on any other size."""
    x = np.ascontiguousarray(xyz, dtype=np.float64)
    if x.size != 3 * n_points:
        raise ValueError(f"expected {n_points} x 3 coordinates, got {x.shape}")
    return x


def make_params(dims, tau=1.0, body_force=(0.0, 0.0, 0.0), periodic=(1, 0, 0),
                wall_velocity=((0, 0, 0), (0, 0, 0)), storage="f32") -> LbParams:
    p = LbParams()
    p.nx, p.ny, p.nz = (int(v) for v in dims)
    p.tau = float(tau)
    for d in range(3):
        p.body_force[d] = float(body_force[d])
        p.periodic[d] = int(periodic[d])
        for w in range(2):
            p.wall_velocity[w][d] = float(wall_velocity[w][d])
    p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    return p


class Simulation:
    """One context: a channel (or a batch of channels) plus its cell meshes."""

    def __init__(self, params: Sequence[LbParams], stream: Optional[int] = None):
        self._L = lib()
        self._h = ctypes.c_void_p()
        arr = (LbParams * len(params))(*params)
        st = self._L.lb_create_batch(arr, len(params), ctypes.c_void_p(stream or 0), ctypes.byref(self._h))
        if st != LB_OK:
            raise LbError(st, "lb_create_batch: " + last_error())
        self.dims = [(p.nx, p.ny, p.nz) for p in params]
        self.n_mesh_nodes = [[] for _ in params]
        self.channel = 0
        self._n_beads = 0

    # -- construction ------------------------------------------------------
    @classmethod
    def from_scene(cls, scene, storage="f32", stream=None) -> "Simulation":
        return cls.from_scenes([scene], storage, stream)

    @classmethod
    def from_scenes(cls, scenes, storage="f32", stream=None) -> "Simulation":
        """One context with a channel per scene.  Collisions and the point
        dynamics are settings of the whole context: every scene must agree."""
        for attr in ("repulsion", "ib_dynamics"):
            vals = {None if getattr(s, attr, None) is None else tuple(getattr(s, attr)) for s in scenes}
            if len(vals) > 1:
                raise ValueError(f"scenes of one batch differ in {attr}: {sorted(map(str, vals))}")
        params = [make_params(s.dims, s.tau, s.body_force, s.periodic, s.wall_velocity, storage) for s in scenes]
        sim = cls(params, stream)
        rep = getattr(scenes[0], "repulsion", None)
        if rep is not None:
            sim.set_repulsion(*rep)
        dyn = getattr(scenes[0], "ib_dynamics", None)
        if dyn is not None:
            sim.set_ib_dynamics(*dyn)
        for k, s in enumerate(scenes):
            sim.select(k)
            if len(s.spheres):
                sim.set_obstacles(s.spheres)
            for m in s.meshes:
                sim.add_mesh(m.rest, m.tris, m.moduli)
        sim.select(0)
        return sim

    def _check(self, st: int):
        if st != LB_OK:
            raise LbError(st, self._L.lb_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.lb_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> int:
        return self._h.value

    def select(self, channel: int):
        self._check(self._L.lb_select_channel(self._h, int(channel)))
        self.channel = int(channel)

    @property
    def N(self) -> int:
        nx, ny, nz = self.dims[self.channel]
        return nx * ny * nz

    def set_obstacles(self, spheres: np.ndarray, extra_mask: Optional[np.ndarray] = None):
        sph = np.ascontiguousarray(spheres, dtype=np.float32).reshape(-1, 4)
        ext = None if extra_mask is None else np.ascontiguousarray(extra_mask, dtype=np.uint8).reshape(self.N)
        self._check(self._L.lb_set_obstacles(self._h, _ptr(sph) if len(sph) else None, int(sph.shape[0]),
                                             None if ext is None else _ptr(ext)))

    def solid_mask(self) -> np.ndarray:
        m = np.zeros(self.N, np.uint8)
        self._check(self._L.lb_get_mask(self._h, _ptr(m)))
        return m

    def add_mesh(self, rest: np.ndarray, tris: np.ndarray, moduli) -> int:
        x = np.ascontiguousarray(rest, dtype=np.float64)
        t = np.ascontiguousarray(tris, dtype=np.int32)
        m = IbmModuli(*[float(v) for v in moduli])
        mid = ctypes.c_int(-1)
        self._check(self._L.ibm_add_mesh(self._h, _ptr(x), int(x.shape[0]), _ptr(t), int(t.shape[0]),
                                         ctypes.byref(m), ctypes.byref(mid)))
        self.n_mesh_nodes[self.channel].append(int(x.shape[0]))
        return mid.value

    def _mesh_nodes(self, mesh: int) -> int:
        meshes = self.n_mesh_nodes[self.channel]
        if not 0 <= int(mesh) < len(meshes):
            raise IndexError(f"mesh {mesh} out of range (channel {self.channel} has {len(meshes)})")
        return meshes[int(mesh)]

    def set_nodes(self, mesh: int, xyz: np.ndarray):
        x = _f64_in(xyz, self._mesh_nodes(mesh))
        self._check(self._L.ibm_set_nodes(self._h, int(mesh), _ptr(x)))

    # -- stepping ----------------------------------------------------------
    def step(self, n: int = 1):
        self._check(self._L.lb_step(self._h, int(n)))

    def synchronize(self):
        self._check(self._L.lb_synchronize(self._h))

    @property
    def steps_done(self) -> int:
        v = ctypes.c_int64()
        self._check(self._L.lb_get_step(self._h, ctypes.byref(v)))
        return v.value

    # -- outputs -----------------------------------------------------------
    def fields(self):
        rho = np.empty(self.N, np.float32)
        u = np.empty((3, self.N), np.float32)
        self._check(self._L.lb_get_fields(self._h, _ptr(rho), _ptr(u), 0))
        return rho, u

    def fields_into(self, rho: np.ndarray, u: np.ndarray):
        """The fields of the selected channel into caller buffers (float32,
        contiguous, N and 3 x N values; page-locked buffers copy fastest)."""
        for a, n in ((rho, self.N), (u, 3 * self.N)):
            if a.dtype != np.float32 or not a.flags.c_contiguous or a.size != n:
                raise ValueError(f"expected a contiguous float32 array of {n} values")
        self._check(self._L.lb_get_fields(self._h, _ptr(rho), _ptr(u), 0))

    def fields_to_device(self, rho_ptr: int, u_ptr: int):
        self._check(self._L.lb_get_fields(self._h, ctypes.c_void_p(rho_ptr), ctypes.c_void_p(u_ptr), 1))

    def populations(self) -> np.ndarray:
        f = np.zeros((19, self.N))
        self._check(self._L.lb_get_populations(self._h, _ptr(f)))
        return f

    def set_populations(self, f: np.ndarray):
        ff = np.ascontiguousarray(f, dtype=np.float64).reshape(19 * self.N)
        self._check(self._L.lb_set_populations(self._h, _ptr(ff)))

    def nodes(self, mesh: int) -> np.ndarray:
        x = np.zeros((self._mesh_nodes(mesh), 3))
        self._check(self._L.ibm_get_nodes(self._h, int(mesh), _ptr(x)))
        return x

    def nodes_into(self, mesh: int, out: np.ndarray):
        out = _f64_out(out, self._mesh_nodes(mesh))
        self._check(self._L.ibm_get_nodes(self._h, int(mesh), _ptr(out)))

    def all_nodes_into(self, out: np.ndarray):
        """Positions of every mesh of the selected channel, concatenated (one transfer)."""
        out = _f64_out(out, sum(self.n_mesh_nodes[self.channel]))
        self._check(self._L.ibm_get_all_nodes(self._h, _ptr(out)))

    def all_nodes_into_async(self, out: np.ndarray, slot: int):
        """Enqueue the readback of every mesh's positions of the selected channel into
        `out` (page-locked for overlap); complete after wait_readback(slot).  `out`
        must stay alive until then."""
        out = _f64_out(out, sum(self.n_mesh_nodes[self.channel]))
        self._check(self._L.ibm_get_all_nodes_async(self._h, _ptr(out), int(slot)))

    def wait_readback(self, slot: int):
        self._check(self._L.lb_readback_wait(self._h, int(slot)))

    def forces(self, mesh: int) -> np.ndarray:
        f = np.zeros((self._mesh_nodes(mesh), 3))
        self._check(self._L.ibm_get_forces(self._h, int(mesh), _ptr(f)))
        return f

    def area_volume(self):
        n = len(self.n_mesh_nodes[self.channel])
        S = np.zeros(n)
        V = np.zeros(n)
        self._check(self._L.ibm_get_area_volume(self._h, _ptr(S), _ptr(V)))
        return S, V

    def diagnostics(self, u_max: float = 0.0) -> np.ndarray:
        out = np.zeros(6)
        st = self._L.lb_diagnostics(self._h, float(u_max), _ptr(out))
        if st not in (LB_OK, LB_ERR_NUMERIC):
            self._check(st)
        return out

    def save_state(self) -> bytes:
        n = ctypes.c_size_t(0)
        self._check(self._L.lb_save_state(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._check(self._L.lb_save_state(self._h, buf, ctypes.byref(n)))
        return buf.raw[: n.value]

    def load_state(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        self._check(self._L.lb_load_state(self._h, buf, len(data)))

    def set_kernel_config(self, nodes_per_thread: int, block_size: int):
        self._check(self._L.lb_set_kernel_config(self._h, int(nodes_per_thread), int(block_size)))

    def kernel_config(self):
        n, b = ctypes.c_int(), ctypes.c_int()
        self._check(self._L.lb_get_kernel_config(self._h, ctypes.byref(n), ctypes.byref(b)))
        return n.value, b.value

    def set_prefetch(self, nodes_ahead: int):
        """L2 prefetch distance of the stream-collide kernel in lattice nodes (0 = off)."""
        self._check(self._L.lb_set_prefetch(self._h, int(nodes_ahead)))

    def prefetch(self) -> int:
        n = ctypes.c_int()
        self._check(self._L.lb_get_prefetch(self._h, ctypes.byref(n)))
        return n.value

    def guard_damage(self, self_test: bool = False) -> int:
        """Bytes of the debug guard zones a kernel overwrote (see set_guard_zones)."""
        n = ctypes.c_int64()
        self._check(self._L.lb_check_guard_zones(self._h, int(self_test), ctypes.byref(n)))
        return n.value

    def autotune(self, repeats: int = 20):
        """Time every stream-collide variant (before the first step) and keep the fastest."""
        n, b, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._check(self._L.lb_autotune(self._h, int(repeats), ctypes.byref(n), ctypes.byref(b), ctypes.byref(ms)))
        return n.value, b.value, ms.value

    def set_repulsion(self, k: float, dc: float):
        """Soft-sphere collisions (cells, beads, walls): force k (dc - d) below separation dc."""
        self._check(self._L.lb_set_repulsion(self._h, float(k), float(dc)))

    def set_ib_dynamics(self, mass: float, gamma: float):
        """IB points with mass and drag (kick + exact drag drift); mass 0: massless points."""
        self._check(self._L.lb_set_ib_dynamics(self._h, float(mass), float(gamma)))

    def set_deterministic(self, on: bool = True):
        """Fixed-point spreading: bit-identical results from run to run."""
        self._check(self._L.lb_set_deterministic(self._h, int(bool(on))))

    def velocities(self, mesh: int) -> np.ndarray:
        """Point velocities after the last step (zeros for massless points)."""
        v = np.zeros((self._mesh_nodes(mesh), 3))
        self._check(self._L.ibm_get_velocities(self._h, int(mesh), _ptr(v)))
        return v

    def set_brinkman(self, beads, alpha: float = 2.0, delta: float = 0.5):
        """Differentiable variant: beads (n x 4: cx, cy, cz, r) as a smooth Brinkman solid fraction."""
        b = np.ascontiguousarray(beads, dtype=np.float64).reshape(-1, 4)
        self._check(self._L.lb_set_brinkman(self._h, _ptr(b), int(b.shape[0]), float(alpha), float(delta)))
        self._n_beads = int(b.shape[0])

    def adjoint(self, n_steps: int, ckpt_every: int = 50, objective_mesh: int = 0) -> dict:
        """J and its gradient (bead centres, ks, kb of the objective cell) by the discrete adjoint
        (after set_brinkman)."""
        nb = self._n_beads
        J = ctypes.c_double()
        gks = ctypes.c_double()
        gkb = ctypes.c_double()
        gb = np.zeros((max(nb, 1), 3))
        self._check(self._L.lb_adjoint(self._h, int(n_steps), int(ckpt_every), int(objective_mesh), ctypes.byref(J),
                                       _ptr(gb), ctypes.byref(gks), ctypes.byref(gkb)))
        return {"J": J.value, "beads": gb[:nb].copy(), "ks": gks.value, "kb": gkb.value}

    SEQUENTIAL, OVERLAPPED, SEQUENTIAL_PLAIN = 0, 1, 2

    def set_schedule(self, schedule):
        """0 (or False): sequential cycle with programmatic dependent launches;
        1 (or True): IB chain concurrent with the bulk stream-collide;
        2: sequential cycle with ordinary launches."""
        self._check(self._L.lb_set_schedule(self._h, int(schedule)))

    def schedule(self) -> int:
        v = ctypes.c_int(0)
        self._check(self._L.lb_get_schedule(self._h, ctypes.byref(v)))
        return v.value

    def set_timing(self, on=True):
        """True: time every kernel class; an int: bit mask of classes; False: off."""
        mask = 15 if on is True else (0 if on is False else int(on))
        self._check(self._L.lb_set_timing(self._h, mask))

    def kernel_times(self):
        ms = np.zeros(4)
        n = np.zeros(4, np.int64)
        self._check(self._L.lb_kernel_times(self._h, _ptr(ms), _ptr(n)))
        return ms, n


def set_guard_zones(nbytes: int):
    """Debug guard zones of nbytes around every device allocation of the
    contexts created afterwards (0: off); Simulation.guard_damage counts the
    bytes a kernel overwrote."""
    L = lib()
    st = L.lb_set_guard_zones(int(nbytes))
    if st != LB_OK:
        raise LbError(st, last_error())


def check_mesh(rest: np.ndarray, tris: np.ndarray) -> str:
    """'' when ibm_add_mesh would accept the mesh, else the reason it refuses
    it (host code of the library; needs no GPU)."""
    x = np.ascontiguousarray(rest, dtype=np.float64).reshape(-1, 3)
    t = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 3)
    why = ctypes.create_string_buffer(256)
    st = lib().ibm_check_mesh(_ptr(x), int(x.shape[0]), _ptr(t), int(t.shape[0]), why, len(why))
    msg = why.value.decode()
    if (st == LB_OK) != (msg == ""):
        raise LbError(st, f"ibm_check_mesh: status and reason disagree ({msg!r})")
    return msg


# ---- magnetic bead assembly (context-free) ----------------------------------
def _bead_params(c, radius, k, mobility=0.0, dt=0.0, box=(1.0, 1.0, 1.0), periodic=(0, 0, 0)) -> BeadParams:
    p = BeadParams()
    p.mu0_4pi, p.radius, p.k_contact, p.mobility, p.dt = float(c), float(radius), float(k), float(mobility), float(dt)
    for d in range(3):
        p.box[d] = float(box[d])
        p.periodic[d] = int(periodic[d])
    return p


def bead_forces(xyz, moments, c, radius, k, box=(1.0, 1.0, 1.0), periodic=(0, 0, 0), stream=None) -> np.ndarray:
    """Dipole + contact forces on every bead (n x 3), computed on the GPU."""
    x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    m = np.ascontiguousarray(moments, dtype=np.float64).reshape(-1, 3)
    F = np.zeros_like(x)
    p = _bead_params(c, radius, k, box=box, periodic=periodic)
    st = lib().bead_forces(_ptr(x), _ptr(m), int(x.shape[0]), ctypes.byref(p), _ptr(F), stream)
    if st != 0:
        raise LbError(st, "bead_forces: " + last_error())
    return F


def bead_relax(xyz, moments, c, radius, k, mobility, dt, steps, box=(1.0, 1.0, 1.0), periodic=(0, 0, 0),
               stream=None) -> np.ndarray:
    """Overdamped bead assembly on the GPU: positions after `steps` steps."""
    x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3).copy()
    m = np.ascontiguousarray(moments, dtype=np.float64).reshape(-1, 3)
    p = _bead_params(c, radius, k, mobility, dt, box, periodic)
    st = lib().bead_relax(_ptr(x), _ptr(m), int(x.shape[0]), ctypes.byref(p), int(steps), stream)
    if st != 0:
        raise LbError(st, "bead_relax: " + last_error())
    return x
