"""Seeded synthetic scenes for the D3Q19 + immersed-boundary blood-flow step.

This module only *builds inputs*: lattice dimensions, obstacle spheres (bead
chains / microposts), closed triangulated cell meshes at their rest shape, and
the scalar parameters of a run.  It contains none of the method's arithmetic
(no lattice-Boltzmann update, no membrane force, no interpolation kernel), so
both the FP64 oracle and the CUDA library consume its output without sharing
any computation.

What the inputs stand for (Gusenbauer et al., "A tunable cancer cell filter
using magnetic beads", arXiv:1110.0995):

* Sec. 2.3.1 / Table 1: red blood cells are biconcave discs (8 um diameter),
  tumor cells spheres (16 um diameter).  With 1 lattice unit = 1 um the red
  cell radius is 4 lu and the tumor cell radius 8 lu.  The meshes here are
  icospheres (level 3: 642 nodes / 1280 triangles; level 4: 2562 / 5120),
  the red cell mapped onto the Evans-Fung biconcave profile.
* Sec. 2.5: bead chains are fixed in space after the magnetic stage and act
  as no-slip obstacles; here they are vertical chains of touching beads
  (radius 3 lu) placed in a staggered post array with seeded gaps.
* Sec. 3.1: the gap-size sweep motivates the batched channel workload.

All random draws come from ``numpy.random.default_rng(seed)`` (PCG64), which
is bit-reproducible across platforms.  Node positions are rounded to
multiples of 2**-32 lu and sphere data to multiples of 2**-8 lu so that both
consumers start from identical, exactly representable values.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

POS_QUANTUM = 2.0 ** -32      # node positions are multiples of this (lu)
SPHERE_QUANTUM = 2.0 ** -8    # sphere centres / radii are multiples of this (lu)

# Membrane moduli (ks, kb, kal, kag, kv).  Red-cell values are the ones the
# plain-channel workload states; the tumor cell is stiffer in stretching
# (ks = 0.5) and reuses the red-cell values for the other four moduli.
RBC_MODULI = (0.05, 0.01, 0.01, 0.5, 0.9)
CTC_MODULI = (0.5, 0.01, 0.01, 0.5, 0.9)

# The massless, explicitly coupled immersed-boundary cycle has a stiffness
# limit.  Over a few hundred steps, with these meshes (edges 0.3-0.7 lu) and
# tau = 1, a stretching modulus above ~0.035 makes small perturbations grow
# (ks = 0.05 by ~3x per 100 steps, ks = 0.5 diverges within ~50 steps).  Over
# thousands of steps slower modes grow as well: the 2562-node tumor-cell mesh
# at ks = 0.03, kb = kal = 0.01 by x5 per 500 steps even at rest, and the
# 256x128x64 filter with red cells at ks = 0.02 ends near 14500 steps.  The
# workloads therefore use ks = kb = kal = 0.01 for red cells and 0.003 for
# tumor cells (whose finer mesh has the lower limit, so the paper's stiffer
# cell is the softer one here), with which the filter completes its 20000
# steps (measured on GB300); kag and kv are unchanged.
STABLE_RBC_MODULI = (0.01, 0.01, 0.01, 0.5, 0.9)
STABLE_CTC_MODULI = (0.003, 0.003, 0.003, 0.5, 0.9)
STABLE = {"rbc": STABLE_RBC_MODULI, "ctc": STABLE_CTC_MODULI}
SPEC = {"rbc": RBC_MODULI, "ctc": CTC_MODULI}

RBC_RADIUS = 4.0
CTC_RADIUS = 8.0
BEAD_RADIUS = 3.0
WALL_CLEARANCE = 1.5          # min distance of any mesh node from walls / solids


@dataclass
class Mesh:
    """One closed, outward-oriented triangle mesh at its rest shape."""
    kind: str                      # "rbc" or "ctc"
    rest: np.ndarray               # (n, 3) float64, lattice units, placed
    tris: np.ndarray               # (t, 3) int32, counter-clockwise seen from outside
    moduli: Tuple[float, float, float, float, float]   # ks, kb, kal, kag, kv

    @property
    def n_nodes(self) -> int:
        return int(self.rest.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])


@dataclass
class Scene:
    """Everything one channel run needs, in lattice units."""
    name: str
    dims: Tuple[int, int, int]                 # (nx, ny, nz), x fastest in memory
    tau: float = 1.0
    body_force: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    periodic: Tuple[int, int, int] = (1, 0, 0)
    wall_velocity: Tuple[Tuple[float, float, float], Tuple[float, float, float]] = (
        (0.0, 0.0, 0.0), (0.0, 0.0, 0.0))      # y-low wall, y-high wall
    spheres: np.ndarray = field(default_factory=lambda: np.zeros((0, 4), np.float32))
    meshes: List[Mesh] = field(default_factory=list)
    steps: int = 0
    seed: int = 0
    # soft-sphere collisions (k, d_c), or None for none (Sec. 2.4 reading)
    repulsion: Optional[Tuple[float, float]] = None
    # IB points with mass and drag (m, gamma), or None for massless points (Sec. 2.2)
    ib_dynamics: Optional[Tuple[float, float]] = None

    @property
    def n_nodes(self) -> int:
        nx, ny, nz = self.dims
        return nx * ny * nz

    @property
    def n_ib_nodes(self) -> int:
        return sum(m.n_nodes for m in self.meshes)


# ---------------------------------------------------------------------------
# mesh geometry (input construction only)
# ---------------------------------------------------------------------------

def _icosahedron() -> Tuple[np.ndarray, np.ndarray]:
    phi = (1.0 + 5.0 ** 0.5) / 2.0
    v = []
    for a in (-1.0, 1.0):
        for b in (-phi, phi):
            v.append((a, b, 0.0))
            v.append((0.0, a, b))
            v.append((b, 0.0, a))
    v = np.array(v, dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    # faces = triples of mutually nearest vertices (edge length is the minimum)
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=2)
    emin = np.min(d[d > 1e-9])
    adj = np.abs(d - emin) < 1e-9
    faces = []
    n = len(v)
    for i in range(n):
        for j in range(i + 1, n):
            if not adj[i, j]:
                continue
            for k in range(j + 1, n):
                if adj[i, k] and adj[j, k]:
                    a, b, c = i, j, k
                    if np.dot(np.cross(v[b] - v[a], v[c] - v[a]), v[a] + v[b] + v[c]) < 0:
                        b, c = c, b
                    faces.append((a, b, c))
    return v, np.array(faces, dtype=np.int32)


def icosphere(level: int) -> Tuple[np.ndarray, np.ndarray]:
    """Unit icosphere: 10*4**level + 2 vertices, 20*4**level outward CCW triangles."""
    v, f = _icosahedron()
    verts = [tuple(p) for p in v]
    for _ in range(level):
        cache = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                p = np.add(verts[a], verts[b])
                p = p / np.linalg.norm(p)
                verts.append(tuple(p))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = np.array(nf, dtype=np.int32)
    return np.array(verts, dtype=np.float64), f


def biconcave(unit: np.ndarray, radius: float) -> np.ndarray:
    """Evans-Fung biconcave disc from unit-sphere points (rest shape of a red cell)."""
    sx, sy, sz = unit[:, 0], unit[:, 1], unit[:, 2]
    r2 = np.clip(sx * sx + sy * sy, 0.0, 1.0)
    z = np.sign(sz) * (radius / 2.0) * np.sqrt(1.0 - r2) * (0.2072 + 2.0026 * r2 - 1.1228 * r2 * r2)
    return np.stack([radius * sx, radius * sy, z], axis=1)


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniformly distributed rotation matrix (unit quaternion from four normals)."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def quantize(x: np.ndarray, quantum: float) -> np.ndarray:
    return np.round(np.asarray(x, dtype=np.float64) / quantum) * quantum


_TEMPLATES = {}


def cell_template(kind: str) -> Tuple[np.ndarray, np.ndarray]:
    """Rest shape centred at the origin: red cell (level 3) or tumor cell (level 4)."""
    if kind not in _TEMPLATES:
        if kind == "rbc":
            u, t = icosphere(3)
            _TEMPLATES[kind] = (biconcave(u, RBC_RADIUS), t)
        elif kind == "ctc":
            u, t = icosphere(4)
            _TEMPLATES[kind] = (CTC_RADIUS * u, t)
        else:
            raise ValueError(kind)
    v, t = _TEMPLATES[kind]
    return v.copy(), t.copy()


# ---------------------------------------------------------------------------
# obstacles
# ---------------------------------------------------------------------------

def post_array(dims, n_cols: int, n_rows: int, n_beads: int, gaps: Sequence[float],
               radius: float = BEAD_RADIUS, x_span: Optional[Tuple[float, float]] = None) -> np.ndarray:
    """Staggered array of vertical bead chains.

    Columns sit at evenly spaced x; each column holds ``n_rows`` posts along y
    separated by the column's surface-to-surface gap, every other column
    shifted by half a pitch.  A post is a chain of ``n_beads`` touching beads
    stacked in z (centres 2.5 + 2*r*m for r = 3).
    """
    nx, ny, nz = dims
    x0, x1 = x_span if x_span is not None else (0.0, float(nx))
    out = []
    for c in range(n_cols):
        xc = x0 + (x1 - x0) * (c + 0.5) / n_cols
        pitch = 2.0 * radius + float(gaps[c])
        y_mid = (ny - 1) / 2.0 + (0.5 * pitch if c % 2 else 0.0)
        for r in range(n_rows):
            yc = y_mid + (r - (n_rows - 1) / 2.0) * pitch
            if yc - radius < -0.5 or yc + radius > ny - 0.5:
                continue
            for m in range(n_beads):
                out.append((xc, yc, 2.5 + 2.0 * radius * m, radius))
    a = quantize(np.array(out, dtype=np.float64).reshape(-1, 4), SPHERE_QUANTUM)
    return a.astype(np.float32)


# ---------------------------------------------------------------------------
# cell placement
# ---------------------------------------------------------------------------

def _periodic_delta(d: np.ndarray, dims, periodic) -> np.ndarray:
    d = d.copy()
    for ax in range(3):
        if periodic[ax]:
            L = dims[ax]
            d[..., ax] -= L * np.round(d[..., ax] / L)
    return d


def place_cells(rng: np.random.Generator, dims, periodic, spheres: np.ndarray,
                kinds: Sequence[str], moduli: dict, max_tries: int = 20000,
                x_range: Optional[Tuple[float, float]] = None) -> List[Mesh]:
    """Seeded uniform placement with rejection.

    Every node keeps ``WALL_CLEARANCE`` lu from the halfway walls of the
    non-periodic axes and from every sphere surface; bounding spheres of two
    cells do not overlap (1 lu margin).  Larger cells are placed first.
    """
    nx, ny, nz = dims
    order = sorted(range(len(kinds)), key=lambda i: 0 if kinds[i] == "ctc" else 1)
    placed: List[Tuple[np.ndarray, float]] = []
    meshes: List[Optional[Mesh]] = [None] * len(kinds)
    sph = spheres.astype(np.float64)
    for idx in order:
        kind = kinds[idx]
        tmpl, tris = cell_template(kind)
        rb = float(np.max(np.linalg.norm(tmpl, axis=1)))
        for _ in range(max_tries):
            R = random_rotation(rng)
            lo = np.array([0.0, 0.0, 0.0])
            hi = np.array([float(nx), float(ny), float(nz)])
            if x_range is not None:
                lo[0], hi[0] = x_range
            c = lo + rng.random(3) * (hi - lo)
            pts = tmpl @ R.T + c
            ok = True
            for ax in range(3):
                if periodic[ax]:
                    continue
                if pts[:, ax].min() < -0.5 + WALL_CLEARANCE or pts[:, ax].max() > dims[ax] - 0.5 - WALL_CLEARANCE:
                    ok = False
                    break
            if not ok:
                continue
            if len(sph):
                d = _periodic_delta(c[None, :] - sph[:, :3], dims, periodic)
                near = np.linalg.norm(d, axis=1) < rb + sph[:, 3] + WALL_CLEARANCE
                if np.any(near):
                    dd = _periodic_delta(pts[:, None, :] - sph[None, near, :3], dims, periodic)
                    if np.any(np.linalg.norm(dd, axis=2) < sph[None, near, 3] + WALL_CLEARANCE):
                        continue
            clash = False
            for (c2, r2) in placed:
                d = _periodic_delta(c - c2, dims, periodic)
                if np.linalg.norm(d) < rb + r2 + 1.0:
                    clash = True
                    break
            if clash:
                continue
            placed.append((c, rb))
            meshes[idx] = Mesh(kind=kind, rest=quantize(pts, POS_QUANTUM), tris=tris.astype(np.int32),
                               moduli=tuple(moduli[kind]))
            break
        else:
            raise RuntimeError(f"could not place {kind} cell after {max_tries} tries")
    return [m for m in meshes if m is not None]


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------

def channel_plain(seed: int = 1, steps: int = 1000, dims=(32, 16, 64), n_rbc: int = 1,
                  body_force: float = 1e-5, moduli: Optional[dict] = None) -> Scene:
    """Plain channel 32x16x64: periodic x, walls in y and z, one red cell
    (moduli as stated for the plain-method workload unless given)."""
    rng = np.random.default_rng(seed)
    per = (1, 0, 0)
    meshes = place_cells(rng, dims, per, np.zeros((0, 4), np.float32), ["rbc"] * n_rbc, moduli or SPEC)
    return Scene(name=f"channel_{dims[0]}x{dims[1]}x{dims[2]}_{n_rbc}rbc", dims=tuple(dims), tau=1.0,
                 body_force=(body_force, 0.0, 0.0), periodic=per, meshes=meshes, steps=steps, seed=seed)


def micropost_filter(seed: int = 11, dims=(256, 128, 64), cols: int = 4, rows: int = 3,
                     n_rbc: int = 60, n_ctc: int = 2, gap_range=(8.0, 14.0), body_force: float = 2e-5,
                     steps: int = 20000, moduli: Optional[dict] = None) -> Scene:
    """Micropost filter: staggered bead-chain posts, red cells and tumor cells."""
    rng = np.random.default_rng(seed)
    per = (1, 0, 0)
    nz = dims[2]
    n_beads = int((nz - 0.5 - 2.5 - BEAD_RADIUS) // (2 * BEAD_RADIUS)) + 1
    gaps = rng.uniform(gap_range[0], gap_range[1], size=cols)
    spheres = post_array(dims, cols, rows, n_beads, gaps)
    kinds = ["ctc"] * n_ctc + ["rbc"] * n_rbc
    meshes = place_cells(rng, dims, per, spheres, kinds, moduli or STABLE)
    return Scene(name=f"micropost_filter_{dims[0]}x{dims[1]}x{dims[2]}", dims=tuple(dims), tau=1.0,
                 body_force=(body_force, 0.0, 0.0), periodic=per, spheres=spheres, meshes=meshes,
                 steps=steps, seed=seed)


def micropost_filter_large(seed: int = 31, steps: int = 10000) -> Scene:
    """512x256x128 filter: 8x4 posts of 21 beads, 400 red cells + 4 tumor cells."""
    return micropost_filter(seed=seed, dims=(512, 256, 128), cols=8, rows=4, n_rbc=400, n_ctc=4,
                            gap_range=(8.0, 14.0), body_force=2e-6, steps=steps)


def gap_sweep(seed: int = 21, n_channels: int = 24, steps: int = 5000) -> List[Scene]:
    """Gap-size sweep: independent channels of uneven size, one post row each."""
    rng = np.random.default_rng(seed)
    out = []
    for ch in range(n_channels):
        nx = int(rng.integers(8, 33)) * 8        # 64..256
        ny = int(rng.integers(4, 17)) * 8        # 32..128
        nz = int(rng.integers(4, 9)) * 8         # 32..64
        gap = float(rng.uniform(6.0, 16.0))
        n_rbc = int(rng.integers(10, 41))
        dims = (nx, ny, nz)
        n_beads = int((nz - 0.5 - 2.5 - BEAD_RADIUS) // (2 * BEAD_RADIUS)) + 1
        rows = max(1, int((ny - 1) // (2 * BEAD_RADIUS + gap)))
        spheres = post_array(dims, 1, rows, n_beads, [gap], x_span=(0.0, float(nx)))
        sub = np.random.default_rng(int(rng.integers(0, 2 ** 31)))
        try:
            meshes = place_cells(sub, dims, (1, 0, 0), spheres, ["rbc"] * n_rbc, STABLE, max_tries=4000)
        except RuntimeError:
            # very small channels cannot hold 40 cells: keep as many as fit
            meshes = []
            for k in range(n_rbc, 0, -1):
                try:
                    meshes = place_cells(np.random.default_rng(int(sub.integers(0, 2 ** 31))), dims, (1, 0, 0),
                                         spheres, ["rbc"] * k, STABLE, max_tries=2000)
                    break
                except RuntimeError:
                    continue
        out.append(Scene(name=f"gap_sweep_ch{ch}_{nx}x{ny}x{nz}_gap{gap:.2f}", dims=dims, tau=1.0,
                         body_force=(1e-5, 0.0, 0.0), periodic=(1, 0, 0), spheres=spheres, meshes=meshes,
                         steps=steps, seed=seed))
    return out


# The paper's cell models (Table 1): 400-node red cell and 306-node tumor
# cell (796 and 608 triangles, i.e. closed triangulations of the sphere),
# diameters 8 and 16 um (lu here).  Moduli as printed, except the red cell's
# K^V = 10, which the explicit massless cycle does not hold (the oracle
# diverges within 500 steps; 0.9 is stable).
TABLE1_MODULI = {"rbc": (0.008, 0.0016, 0.01, 1.0, 0.9), "ctc": (0.0023, 0.000464, 0.0029, 0.29, 2.9)}
TABLE1_NODES = {"rbc": 400, "ctc": 306}


def fibonacci_sphere_mesh(n: int) -> Tuple[np.ndarray, np.ndarray]:
    """n near-uniform unit-sphere points (Fibonacci lattice) and their convex
    hull as outward counter-clockwise triangles (2n - 4 of them)."""
    from scipy.spatial import ConvexHull

    i = np.arange(n) + 0.5
    phi = np.arccos(1.0 - 2.0 * i / n)
    th = np.pi * (1.0 + 5.0 ** 0.5) * i
    u = np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], axis=1)
    t = ConvexHull(u).simplices.astype(np.int32)
    c = u[t].mean(axis=1)
    nrm = np.cross(u[t[:, 1]] - u[t[:, 0]], u[t[:, 2]] - u[t[:, 0]])
    flip = (nrm * c).sum(axis=1) < 0
    t[flip] = t[flip][:, [0, 2, 1]]
    return u, t


def table1_template(kind: str) -> Tuple[np.ndarray, np.ndarray]:
    """Rest shape of the paper's cell model centred at the origin."""
    u, t = fibonacci_sphere_mesh(TABLE1_NODES[kind])
    v = biconcave(u, RBC_RADIUS) if kind == "rbc" else CTC_RADIUS * u
    return v, t


def slit_barrier(dims, gap: float, x0: float, radius: float = 2.2, spacing: float = 3.0) -> np.ndarray:
    """A plate of overlapping beads across the channel at x = x0 with a slit of
    surface-to-surface width ``gap`` along z, centred in y.  Beads of radius
    2.2 at a 3.0 pitch leave no fluid node between four neighbours (the
    square's centre lies 2.12 from each), so the fluid and the cells cross
    the plate only through the slit."""
    nx, ny, nz = dims
    yc = (ny - 1) / 2.0
    out = []
    for y in np.arange(-0.5, ny - 0.5 + spacing, spacing):
        if abs(y - yc) < gap / 2.0 + radius:
            continue
        for z in np.arange(-0.5, nz - 0.5 + spacing, spacing):
            out.append((x0, float(y), float(z), radius))
    # the beads closest to the slit, on its two edges, at every z
    for sgn in (-1.0, 1.0):
        y = yc + sgn * (gap / 2.0 + radius)
        for z in np.arange(-0.5, nz - 0.5 + spacing, spacing):
            out.append((x0, float(y), float(z), radius))
    a = quantize(np.array(out, dtype=np.float64).reshape(-1, 4), SPHERE_QUANTUM)
    return a.astype(np.float32)


def gap_cell(kind: str, gap: float, dims=(96, 40, 32), steps: int = 10000, body_force: float = 2e-5,
             moduli=None, table1: bool = False) -> Scene:
    """One cell upstream of a slit of width ``gap`` (Sec. 3 gap experiment):
    a red cell edge-on to the slit (its disc in the x-z plane) or a tumor cell,
    the stable moduli, collisions on so that the cell cannot enter the beads."""
    nx, ny, nz = dims
    x0 = nx / 2.0
    spheres = slit_barrier(dims, gap, x0)
    v, t = table1_template(kind) if table1 else cell_template(kind)
    if kind == "rbc":
        v = v[:, [0, 2, 1]]          # disc axis along y: edge-on to a slit narrow in y
        t = t[:, [0, 2, 1]]          # keep the outward orientation after the swap
    r_cell = RBC_RADIUS if kind == "rbc" else CTC_RADIUS
    centre = np.array([x0 - 2.2 - r_cell - 6.0, (ny - 1) / 2.0, (nz - 1) / 2.0])
    rest = quantize(v + centre, POS_QUANTUM)
    if moduli is None:
        moduli = TABLE1_MODULI[kind] if table1 else STABLE[kind]
    mesh = Mesh(kind, rest, np.ascontiguousarray(t, dtype=np.int32), moduli)
    return Scene(name=f"gap_{kind}_{gap:g}", dims=dims, tau=1.0, body_force=(body_force, 0.0, 0.0),
                 periodic=(1, 0, 0), spheres=spheres, meshes=[mesh], steps=steps, seed=0,
                 repulsion=(0.01, 1.0))


def adjoint_channel(seed: int = 41, steps: int = 400) -> Scene:
    """128x64x64 channel with two 6-bead posts, 8 red cells and 1 tumor cell."""
    rng = np.random.default_rng(seed)
    dims = (128, 64, 64)
    gap = float(rng.uniform(8.0, 14.0))
    spheres = post_array(dims, 1, 2, 6, [gap], x_span=(64.0, 128.0))
    kinds = ["ctc"] + ["rbc"] * 8
    meshes = place_cells(rng, dims, (1, 0, 0), spheres, kinds, STABLE, x_range=(0.0, 60.0))
    return Scene(name="adjoint_128x64x64", dims=dims, tau=1.0, body_force=(1e-5, 0.0, 0.0),
                 periodic=(1, 0, 0), spheres=spheres, meshes=meshes, steps=steps, seed=seed)


def adjoint_channel_small(seed: int = 43, steps: int = 100) -> Scene:
    """64x48x32 channel with two 3-bead posts, 2 red cells and 1 tumor cell (mesh 0)."""
    rng = np.random.default_rng(seed)
    dims = (64, 48, 32)
    gap = float(rng.uniform(8.0, 12.0))
    spheres = post_array(dims, 1, 2, 3, [gap], x_span=(36.0, 64.0))
    kinds = ["ctc", "rbc", "rbc"]
    meshes = place_cells(rng, dims, (1, 0, 0), spheres, kinds, STABLE, x_range=(0.0, 34.0))
    return Scene(name="adjoint_small_64x48x32", dims=dims, tau=1.0, body_force=(1e-5, 0.0, 0.0),
                 periodic=(1, 0, 0), spheres=spheres, meshes=meshes, steps=steps, seed=seed)


def small_filter(seed: int = 5, dims=(96, 48, 32), n_rbc: int = 4, n_ctc: int = 1, steps: int = 100) -> Scene:
    """Small filter (several tiles, ragged nothing) used for fast parity runs."""
    return micropost_filter(seed=seed, dims=dims, cols=2, rows=2, n_rbc=n_rbc, n_ctc=n_ctc,
                            gap_range=(8.0, 14.0), body_force=2e-5, steps=steps)


def random_field(seed: int, shape, scale: float = 1.0) -> np.ndarray:
    """Seeded standard-normal array (used for test force fields and perturbations)."""
    return np.random.default_rng(seed).standard_normal(shape) * scale
