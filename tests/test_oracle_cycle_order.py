"""Which fluid velocity the advance of the coupled cycle uses (reading 10 of
Sec. 2.2: forces at X^t -> spread -> collision gives u^t -> X^{t+1} = X^t +
interp(u^t, X^t)).

One cycle from a state whose answer is known in closed form: populations at
equilibrium with density 1 and a linear velocity field u0(x), a cell at its
rest shape (every membrane force is zero, so nothing is spread), and a uniform
body force G.  The collision then sees rho = 1 and momentum u0 (the
equilibrium's zeroth and first moments), so its velocity is u0 + G/2
everywhere, and trilinear interpolation of a linear field is exact: every
node must move by u0(X) + G/2.  An advance with the previous cycle's velocity
(u0 or nothing), with the velocity after streaming (which carries the whole
source G of the collision, u0 + 3G/2), or before the half-force correction
(u0) misses this by G/2 or more, far above the FP64 tolerance."""
import numpy as np
import pytest

import oracle
from paper_1110_0995_gb300 import scene

A, B, C = 1.0e-3, -8.0e-4, 5.0e-4            # u0 = (A (y - 12), B (z - 12), C (x - 12))
G = (2.0e-5, -1.0e-5, 5.0e-6)
DIMS = (24, 24, 24)


def u0(x, y, z):
    return np.array([A * (y - 12.0), B * (z - 12.0), C * (x - 12.0)])


def linear_shear_state(dims=DIMS):
    nx, ny, nz = dims
    f = np.zeros((19, nx * ny * nz))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                f[:, x + nx * (y + ny * z)] = oracle.equilibrium(1.0, u0(x, y, z))
    return f


def rest_cell():
    v, t = scene.cell_template("rbc")
    rng = np.random.default_rng(4)
    R = scene.random_rotation(rng)
    rest = scene.quantize(v @ R.T + np.array([12.3, 11.7, 12.1]), scene.POS_QUANTUM)
    return scene.Mesh(kind="rbc", rest=rest, tris=t, moduli=scene.SPEC["rbc"])


def cycle_scene():
    return scene.Scene(name="shear_one_cycle", dims=DIMS, tau=0.8, body_force=G, periodic=(1, 0, 0),
                       meshes=[rest_cell()], steps=1)


def expected_positions(x0):
    return x0 + np.array([u0(*p) for p in x0]) + np.array(G) / 2


def test_advance_uses_the_velocity_of_the_same_collision():
    sc = cycle_scene()
    ref = oracle.System.from_scene(sc)
    ref.set_f(linear_shear_state())
    x0 = ref.nodes(0)
    ref.step(1)
    x1 = ref.nodes(0)
    np.testing.assert_allclose(x1, expected_positions(x0), rtol=0, atol=1e-12)
    # the collision's velocity field itself: u0 + G/2 at every node
    _, u = ref.fields()
    nx, ny, nz = DIMS
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    want = np.stack([A * (yy - 12.0), B * (zz - 12.0), C * (xx - 12.0)]).reshape(3, -1) + np.array(G)[:, None] / 2
    np.testing.assert_allclose(u, want, rtol=0, atol=1e-15)


def test_a_misordered_cycle_fails_the_pin():
    """The pin separates the candidate orderings: the displacement of the
    reading differs from each alternative's by at least |G|/2 per node."""
    sc = cycle_scene()
    ref = oracle.System.from_scene(sc)
    ref.set_f(linear_shear_state())
    x0 = ref.nodes(0)
    good = expected_positions(x0) - x0
    previous = np.array([u0(*p) for p in x0])            # last cycle's (initial) field, no G/2
    after_streaming = previous + 1.5 * np.array(G)       # the post-collision momentum, streamed
    for alt in (previous, after_streaming, np.zeros_like(previous)):
        assert np.abs(alt - good).max() >= 0.5 * np.abs(G).max() - 1e-15
