"""Small hand-built models with textbook closed forms (test fixtures)."""
import numpy as np

from paper_2603_29332_b300.modelgen import make_model

G = 9.81


def pendulum(mass=2.0, lc=0.3, iyy=0.05, height=1.0):
    """One body on a hinge about +y at (0, 0, height); COM at (lc, 0, 0); gravity -z."""
    return make_model("pendulum", [-1], [1], [[0, 0, height]], [mass], [[lc, 0, 0]],
                      [[0.01, iyy, 0.02, 0, 0, 0]], [[0, 1, 0]])


def two_link(m1=1.5, m2=0.8, l1=0.6, lc1=0.25, lc2=0.2, i1=0.03, i2=0.02):
    """Planar two-link arm: hinges about +z, links along +x at q = 0, gravity -y."""
    return make_model("two_link", [-1, 0], [1, 1], [[0, 0, 0], [l1, 0, 0]], [m1, m2],
                      [[lc1, 0, 0], [lc2, 0, 0]], [[0.001, 0.001, i1, 0, 0, 0], [0.001, 0.001, i2, 0, 0, 0]],
                      [[0, 0, 1], [0, 0, 1]], gravity=[0.0, -G, 0.0])


def rod_on_ground(mass=1.2, lc=0.25, length=0.5, radius=0.03, iyy=0.03, **scalars):
    """Rod on a hinge about +y at height r; contact sphere of radius r at its tip (x = length).
    At q = 0 the sphere touches z = 0; positive q presses it into the ground."""
    return make_model("rod", [-1], [1], [[0, 0, radius]], [mass], [[lc, 0, 0]], [[0.005, iyy, 0.03, 0, 0, 0]],
                      [[0, 1, 0]], spheres=[(0, (length, 0, 0), radius)], **scalars)


def hinge_muscle(a=0.1, b=0.12, h0=0.05, h1=0.04):
    """Two bodies along +x, joint of body 1 about +z at x = 0.3; one two-point muscle from
    (0.3 - a, h0, 0) on body 0 to (b, h1, 0) on body 1.  Zero gravity."""
    return make_model("hinge_muscle", [-1, 0], [1, 1], [[0, 0, 0], [0.3, 0, 0]], [1.0, 1.0],
                      [[0.15, 0, 0], [0.1, 0, 0]], [[0.001, 0.01, 0.01, 0, 0, 0]] * 2, [[0, 0, 1], [0, 0, 1]],
                      muscle_points=[[(0, (0.3 - a, h0, 0.0)), (1, (b, h1, 0.0))]], muscle_fmax=[1000.0],
                      muscle_lopt=[0.1], gravity=[0.0, 0.0, 0.0])


def chain(n_links=3, seed=0, gravity=True, root_axis=(0, 1, 0)):
    """A chain of capsule-like links with random hinge axes (no muscles, no contact)."""
    rng = np.random.default_rng(seed)
    axes = [root_axis] + [tuple(v / np.linalg.norm(v)) for v in rng.normal(size=(n_links - 1, 3))]
    offs = [[0, 0, 1.0]] + [[0.3, 0.05 * k, 0] for k in range(1, n_links)]
    masses = rng.uniform(1, 3, size=n_links)
    coms = [[0.15, 0.01, -0.02]] * n_links
    inert = [[0.02, 0.03, 0.025, 0.001, -0.002, 0.0015]] * n_links
    return make_model("chain", list(range(-1, n_links - 1)), [1] * n_links, offs, masses, coms, inert, axes,
                      gravity=[0, 0, -G] if gravity else [0, 0, 0])


def free_ball(mass=2.0, radius=0.05, inertia=0.002, height=None, **scalars):
    """A free-floating ball: body 0 on a free root, COM at its origin, one contact sphere of the
    ball's radius centred there.  With q = 0 its origin is at ``height`` (default: resting on
    z = 0, sphere touching the ground)."""
    from paper_2603_29332_b300.modelgen import with_free_root
    h = radius if height is None else height
    base = make_model("ball", [-1], [1], [[0, 0, h]], [mass], [[0, 0, 0]], [[inertia, inertia, inertia, 0, 0, 0]],
                      [[0, 0, 1]], spheres=[(0, (0.0, 0.0, 0.0), radius)], **scalars)
    return with_free_root(base)
