"""Seeded synthetic musculoskeletal models, initial states and excitation signals.

This module only *draws inputs*: skeleton trees, body and muscle parameters,
via-point tables, contact spheres, initial states and excitation signals.  It
holds none of the arithmetic of the forward-dynamics step (no kinematics, no
muscle geometry, no force law, no dynamics).  Both the CUDA path and the FP64
oracle consume what it produces, each with its own code.

The MS-Human-700 model the paper simulates (Methods, "Whole-body
musculoskeletal model") is not available, so the workloads are synthetic
stand-ins with the sizes of the whole-body model: ~700 Hill-type muscle-tendon
units with via-point paths on a tree of hinge joints, foot contact geometry
(Methods, "Contact modeling") and the activation constants of Eq. (2).

Conventions shared by every consumer of a :class:`Model`:

* Bodies are listed parents-first (``body_parent[b] < b``; ``-1`` is the fixed
  world).  Body ``b`` owns ``body_ndof[b]`` (1..3) consecutive hinge DoFs
  starting at ``body_dof_start[b]``; DoFs are numbered in body order.
* Body ``b``'s frame = parent frame * translate(``body_offset[b]``) *
  Rot(axis_0, q_0) * ... * Rot(axis_{k-1}, q_{k-1}).  Each ``dof_axis`` is a
  unit vector in the frame just before its hinge (intrinsic sequence).  At
  q = 0 every body frame is aligned with the world.
* ``body_com`` / ``body_inertia`` (xx, yy, zz, xy, xz, yz about the COM) and
  ``point_pos`` / ``sphere_pos`` are given in the body frame.
* Muscle ``k`` is the polyline through points
  ``muscle_point_start[k] .. muscle_point_start[k+1]-1`` (origin first,
  insertion last); consecutive points lie on the same body or on a body
  further down the one ancestor chain the muscle spans.
* All floating-point parameters are rounded to FP32 values (stored as
  float64) so that the FP32 GPU path and the FP64 oracle see identical
  numbers.
"""
from __future__ import annotations

from dataclasses import dataclass, field, asdict
import numpy as np

# Activation and deactivation time constants of Eq. (2): 10 ms and 40 ms.
TAU_ACT = 0.010
TAU_DEACT = 0.040


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


@dataclass
class Model:
    name: str
    body_parent: np.ndarray          # int32 [B]
    body_dof_start: np.ndarray       # int32 [B]
    body_ndof: np.ndarray            # int32 [B]
    body_offset: np.ndarray          # [B,3]
    body_mass: np.ndarray            # [B]
    body_com: np.ndarray             # [B,3]
    body_inertia: np.ndarray         # [B,6]
    dof_axis: np.ndarray             # [n,3]
    dof_limit: np.ndarray            # [n,2]  lo >= hi disables the limit
    dof_damping: np.ndarray          # [n]
    muscle_point_start: np.ndarray   # int32 [m+1]
    muscle_fmax: np.ndarray          # [m]
    muscle_lopt: np.ndarray          # [m]
    muscle_lslack: np.ndarray        # [m]
    point_body: np.ndarray           # int32 [P]
    point_pos: np.ndarray            # [P,3]
    sphere_body: np.ndarray          # int32 [S]
    sphere_pos: np.ndarray           # [S,3]
    sphere_radius: np.ndarray        # [S]
    gravity: np.ndarray = field(default_factory=lambda: _f32([0.0, 0.0, -9.81]))
    contact_k: float = 1.0e5
    contact_c: float = 1.0e3
    contact_mu: float = 0.9
    contact_eps: float = 0.1
    # joint-limit penalty: stiffness k_l, damping c_l, onset width (see the limit reading)
    limit_k: float = 1.0e5
    limit_c: float = 1.0e3
    limit_delta: float = 0.0
    tau_act: float = TAU_ACT
    tau_deact: float = TAU_DEACT
    vmax_per_lopt: float = 10.0
    # free root: body 0 joined to the world by six DoFs 0-5, translations of its origin along
    # world x, y, z, then rotations about world x, y, z through it (q: position and rotation
    # vector, qd: velocity and world angular velocity); dof_axis rows 0-5 are e_x e_y e_z e_x e_y e_z
    free_root: bool = False
    # wrapping cylinders (at most one per muscle): the segment ending at the muscle's point
    # number wrap_segment wraps around an infinite cylinder fixed to body wrap_body
    wrap_muscle: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    wrap_segment: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    wrap_body: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    wrap_center: np.ndarray = field(default_factory=lambda: np.zeros((0, 3), np.float32))   # body frame
    wrap_axis: np.ndarray = field(default_factory=lambda: np.zeros((0, 3), np.float32))     # unit, body frame
    wrap_radius: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float32))
    wrap_kind: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))   # 0 cylinder, 1 sphere
    # per muscle: tendon strain at F_max; > 0 makes the tendon compliant (its slack length is the
    # muscle's length at q = 0 less l_opt), 0 keeps it rigid.  Empty: every tendon rigid.
    muscle_tendon_strain: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float32))

    def __post_init__(self):
        # scalar parameters are FP32 values too, like every array
        for k in ("contact_k", "contact_c", "contact_mu", "contact_eps", "limit_k", "limit_c", "limit_delta",
                  "tau_act", "tau_deact", "vmax_per_lopt"):
            setattr(self, k, float(np.float32(getattr(self, k))))
        self.gravity = _f32(self.gravity)
        for k in ("wrap_muscle", "wrap_segment", "wrap_body", "wrap_kind"):
            setattr(self, k, np.asarray(getattr(self, k), dtype=np.int32).reshape(-1))
        if self.wrap_kind.shape[0] == 0 and self.wrap_muscle.shape[0] > 0:
            self.wrap_kind = np.zeros(self.wrap_muscle.shape[0], np.int32)   # cylinders
        self.wrap_center = _f32(np.asarray(self.wrap_center, dtype=np.float64).reshape(-1, 3))
        self.wrap_axis = _f32(np.asarray(self.wrap_axis, dtype=np.float64).reshape(-1, 3))
        self.wrap_radius = _f32(np.asarray(self.wrap_radius, dtype=np.float64).reshape(-1))
        ts = np.asarray(self.muscle_tendon_strain, dtype=np.float64).reshape(-1)
        self.muscle_tendon_strain = _f32(ts if ts.shape[0] else np.zeros(self.muscle_fmax.shape[0]))

    @property
    def n_bodies(self):
        return int(self.body_parent.shape[0])

    @property
    def n_dofs(self):
        return int(self.dof_axis.shape[0])

    @property
    def n_muscles(self):
        return int(self.muscle_fmax.shape[0])

    @property
    def n_points(self):
        return int(self.point_body.shape[0])

    @property
    def n_spheres(self):
        return int(self.sphere_body.shape[0])

    def scalars(self):
        return dict(contact_k=self.contact_k, contact_c=self.contact_c, contact_mu=self.contact_mu,
                    contact_eps=self.contact_eps, limit_k=self.limit_k, limit_c=self.limit_c,
                    limit_delta=self.limit_delta,
                    tau_act=self.tau_act, tau_deact=self.tau_deact, vmax_per_lopt=self.vmax_per_lopt)

    def validate(self):
        B, n = self.n_bodies, self.n_dofs
        assert np.all(self.body_parent < np.arange(B))
        nd = self.body_ndof
        if self.free_root:
            assert self.body_parent[0] == -1 and nd[0] == 6
            assert np.array_equal(self.dof_axis[:6], np.vstack([np.eye(3), np.eye(3)]))
            assert np.all(self.dof_limit[:6, 0] >= self.dof_limit[:6, 1])   # no limits on the root
            nd = nd[1:]
        assert np.all((nd >= 1) & (nd <= 3))
        assert self.body_dof_start[0] == 0
        assert np.all(self.body_dof_start[1:] == np.cumsum(self.body_ndof)[:-1])
        assert int(self.body_ndof.sum()) == n
        assert np.allclose(np.linalg.norm(self.dof_axis, axis=1), 1.0, atol=1e-6)
        assert self.muscle_point_start[0] == 0 and self.muscle_point_start[-1] == self.n_points
        assert np.all(np.diff(self.muscle_point_start) >= 2)
        W = self.wrap_muscle.shape[0]
        assert all(a.shape[0] == W for a in (self.wrap_segment, self.wrap_body, self.wrap_center, self.wrap_axis,
                                            self.wrap_radius, self.wrap_kind))
        assert np.all((self.wrap_kind == 0) | (self.wrap_kind == 1))
        assert len(set(self.wrap_muscle.tolist())) == W          # at most one cylinder per muscle
        if W:
            npts = np.diff(self.muscle_point_start)[self.wrap_muscle]
            assert np.all((self.wrap_segment >= 1) & (self.wrap_segment < npts))
            assert np.all(self.wrap_radius > 0)
        return self


# ----------------------------------------------------------------------------------------------
# building blocks


def _unit(v):
    return v / np.linalg.norm(v)


def _perp(rng, d):
    """A random unit vector perpendicular to unit vector d."""
    while True:
        v = rng.normal(size=3)
        v -= d * (v @ d)
        nv = np.linalg.norm(v)
        if nv > 1e-3:
            return v / nv


def _random_rotation(rng):
    a = rng.normal(size=(3, 3))
    qm, r = np.linalg.qr(a)
    qm = qm * np.sign(np.diag(r))
    if np.linalg.det(qm) < 0:
        qm[:, 0] = -qm[:, 0]
    return qm


def capsule_inertia(mass, length, radius, direction):
    """Inertia (xx, yy, zz, xy, xz, yz) about the COM of a solid capsule of uniform density.

    The capsule is a cylinder of the given length with hemispherical caps, its axis along
    ``direction``.  Closed form: cylinder plus two hemispheres shifted by the parallel-axis
    theorem (hemisphere COM at 3r/8 from its flat face).  This is a model parameter, not
    part of the dynamics.
    """
    r, h = radius, length
    v_cyl = np.pi * r * r * h
    v_hs = 2.0 / 3.0 * np.pi * r ** 3
    rho = mass / (v_cyl + 2 * v_hs)
    m_c, m_h = rho * v_cyl, rho * v_hs
    i_axial = m_c * r * r / 2 + 2 * (2.0 / 5.0 * m_h * r * r)
    i_hs_own = (83.0 / 320.0) * m_h * r * r          # about the hemisphere's own COM, transverse
    dist = h / 2 + 3.0 * r / 8.0
    i_trans = m_c * (3 * r * r + h * h) / 12 + 2 * (i_hs_own + m_h * dist * dist)
    d = _unit(np.asarray(direction, dtype=np.float64))
    inertia = i_trans * np.eye(3) + (i_axial - i_trans) * np.outer(d, d)
    return np.array([inertia[0, 0], inertia[1, 1], inertia[2, 2],
                     inertia[0, 1], inertia[0, 2], inertia[1, 2]])


def make_model(name, body_parent, body_ndof, body_offset, body_mass, body_com, body_inertia,
               dof_axis, muscle_points=(), muscle_fmax=(), muscle_lopt=(), muscle_lslack=None,
               dof_limit=None, dof_damping=None, spheres=(), wraps=(), **scalars):
    """Assemble a :class:`Model` from explicit arrays (used for hand-built test models).

    ``muscle_points`` is a list (one entry per muscle) of lists of (body, (x, y, z)).
    ``spheres`` is a list of (body, (x, y, z), radius).
    ``wraps`` is a list of (muscle, segment end point index, body, centre, axis, radius[, kind]):
    kind 0 = cylinder (default), 1 = sphere (the axis is then unused).
    """
    body_parent = np.asarray(body_parent, dtype=np.int32)
    body_ndof = np.asarray(body_ndof, dtype=np.int32)
    B = body_parent.shape[0]
    n = int(body_ndof.sum())
    starts = np.zeros(B, dtype=np.int32)
    starts[1:] = np.cumsum(body_ndof)[:-1]
    pstart = [0]
    pbody, ppos = [], []
    for pts in muscle_points:
        for b, x in pts:
            pbody.append(b)
            ppos.append(x)
        pstart.append(len(pbody))
    m = len(muscle_points)
    if muscle_lslack is None:
        muscle_lslack = np.asarray(muscle_lopt, dtype=np.float64) * 1.0
    sb = np.asarray([s[0] for s in spheres], dtype=np.int32)
    sp = np.asarray([s[1] for s in spheres], dtype=np.float64).reshape(-1, 3)
    sr = np.asarray([s[2] for s in spheres], dtype=np.float64)
    mdl = Model(
        name=name,
        body_parent=body_parent,
        body_dof_start=starts,
        body_ndof=body_ndof,
        body_offset=_f32(np.asarray(body_offset, dtype=np.float64).reshape(B, 3)),
        body_mass=_f32(np.asarray(body_mass, dtype=np.float64).reshape(B)),
        body_com=_f32(np.asarray(body_com, dtype=np.float64).reshape(B, 3)),
        body_inertia=_f32(np.asarray(body_inertia, dtype=np.float64).reshape(B, 6)),
        dof_axis=_f32(np.asarray(dof_axis, dtype=np.float64).reshape(n, 3)),
        dof_limit=_f32(np.zeros((n, 2)) if dof_limit is None else np.asarray(dof_limit).reshape(n, 2)),
        dof_damping=_f32(np.zeros(n) if dof_damping is None else np.asarray(dof_damping).reshape(n)),
        muscle_point_start=np.asarray(pstart, dtype=np.int32),
        muscle_fmax=_f32(np.asarray(muscle_fmax, dtype=np.float64).reshape(m)),
        muscle_lopt=_f32(np.asarray(muscle_lopt, dtype=np.float64).reshape(m)),
        muscle_lslack=_f32(np.asarray(muscle_lslack, dtype=np.float64).reshape(m)),
        point_body=np.asarray(pbody, dtype=np.int32),
        point_pos=_f32(np.asarray(ppos, dtype=np.float64).reshape(-1, 3)),
        sphere_body=sb, sphere_pos=_f32(sp), sphere_radius=_f32(sr),
        wrap_muscle=[w[0] for w in wraps], wrap_segment=[w[1] for w in wraps], wrap_body=[w[2] for w in wraps],
        wrap_center=[w[3] for w in wraps], wrap_axis=[_unit(np.asarray(w[4], dtype=np.float64)) for w in wraps],
        wrap_radius=[w[5] for w in wraps], wrap_kind=[w[6] if len(w) > 6 else 0 for w in wraps],
    )
    for k, v in scalars.items():
        if k == "gravity":
            mdl.gravity = _f32(v)
        else:
            setattr(mdl, k, float(np.float32(v)))
    return mdl.validate()


def with_free_root(model, name=None):
    """The same model with body 0 (a root) joined to the world by a free joint: its hinges are
    replaced by the six free-root DoFs (no limits, no damping); everything else is unchanged."""
    assert model.body_parent[0] == -1 and not model.free_root
    k = int(model.body_ndof[0])
    ndof = model.body_ndof.copy()
    ndof[0] = 6
    starts = np.zeros_like(ndof)
    starts[1:] = np.cumsum(ndof)[:-1]
    axis = np.vstack([np.eye(3), np.eye(3), model.dof_axis[k:]])
    lim = np.vstack([np.zeros((6, 2)), model.dof_limit[k:]])
    damp = np.concatenate([np.zeros(6), model.dof_damping[k:]])
    kw = {f: getattr(model, f) for f in model.__dataclass_fields__}
    kw.update(name=name or model.name + "_float", body_ndof=ndof.astype(np.int32), body_dof_start=starts.astype(np.int32),
              dof_axis=_f32(axis), dof_limit=_f32(lim), dof_damping=_f32(damp), free_root=True)
    return Model(**kw).validate()


def with_tendons(model, rest_lengths, frac=1.0, strain=(0.033, 0.06), min_ratio=0.6, seed=0, name=None):
    """The same model with compliant tendons: each muscle whose slack length (its length at q = 0,
    ``rest_lengths``, less l_opt) is at least ``min_ratio`` l_opt gets, with probability ``frac``, a
    tendon strain at F_max drawn from U(strain).  The rest lengths are the caller's (the path
    geometry is not this module's)."""
    L0 = np.asarray(rest_lengths, dtype=np.float64).reshape(model.n_muscles)
    ratio = (L0 - model.muscle_lopt) / model.muscle_lopt
    rng = np.random.default_rng(seed + 7000)
    pick = (ratio >= min_ratio) & (rng.uniform(size=model.n_muscles) < frac)
    eps0 = np.where(pick, rng.uniform(strain[0], strain[1], size=model.n_muscles), 0.0)
    kw = {f: getattr(model, f) for f in model.__dataclass_fields__}
    kw.update(name=name or model.name + "_tendon", muscle_tendon_strain=_f32(eps0))
    return Model(**kw).validate()


# ----------------------------------------------------------------------------------------------
# synthetic whole-body-like models

# name -> generator parameters.  C0 and C1 are the tiny arm-leg chain and the whole-body
# model; "upper" and "lower" are the two extra skeletons of the mixed-size batch.
CONFIGS = {
    "c0_tiny": dict(n_bodies=8, n_dofs=14, n_muscles=40, max_points=4, max_span=2, limits=False,
                    contact=False, seed=0, max_dof_per_body=2),
    "c1_whole": dict(n_bodies=60, n_dofs=90, n_muscles=700, max_points=6, max_span=3, limits=True,
                     contact=True, seed=1),
    "c2_upper": dict(n_bodies=20, n_dofs=30, n_muscles=250, max_points=6, max_span=3, limits=True,
                     contact=False, seed=21),
    "c2_lower": dict(n_bodies=27, n_dofs=40, n_muscles=300, max_points=6, max_span=3, limits=True,
                     contact=True, seed=22),
    # the whole body with a quarter of its muscles wrapping a cylinder at a joint
    "c1_wrap": dict(n_bodies=60, n_dofs=90, n_muscles=700, max_points=6, max_span=3, limits=True,
                    contact=True, seed=1, wrap_frac=0.25),
    # the wrapped body with half of its surfaces spheres instead of cylinders
    "c1_wrap_mix": dict(n_bodies=60, n_dofs=90, n_muscles=700, max_points=6, max_span=3, limits=True,
                        contact=True, seed=1, wrap_frac=0.25, sphere_frac=0.5),
    # the whole body on a free (floating) root instead of its root hinges
    "c1_float": dict(n_bodies=60, n_dofs=90, n_muscles=700, max_points=6, max_span=3, limits=True,
                     contact=True, seed=1, free_root=True),
}


def generate(name=None, *, n_bodies, n_dofs, n_muscles, max_points, max_span, limits, contact, seed,
             n_legs=2, spheres_per_foot=4, sphere_radius=0.03, max_dof_per_body=3, wrap_frac=0.0,
             sphere_frac=0.0, free_root=False):
    """Draw one synthetic skeleton + muscle model.

    Tree: a root body, then limb chains of U{3..8} bodies each, the parent of each chain drawn
    uniformly over existing bodies (with contact, the first two chains hang down from the root
    as legs).  Link length U(0.2, 0.5) m, mass U(1, 8) kg, capsule inertia with radius 0.1 x
    length.  DoFs: one per body, then incremented at random (max ``max_dof_per_body``) up to
    ``n_dofs``; a 3-DoF body is a ball joint as three hinges with orthonormal axes.
    Muscles: U{2..max_points} path points; insertion body B, origin body A = the ancestor
    ``span`` joints up (span U{1..min(max_span, points-1)}); one point on each body of the A..B
    chain (origin at U(0.6, 0.95) of A's length, insertion at U(0.05, 0.4) of B's, the others at
    U(0.1, 0.9)), extra points on random chain bodies; radial offset U(0.02, 0.06) m; redrawn if a
    segment is shorter than 1 cm at q = 0.
    F_max U(100, 3000) N, l_opt U(0.05, 0.3) m, l_slack = U(1.0, 1.5) x l_opt.
    Limits (if enabled) lo = -U(0.5, 2), hi = U(0.5, 2) rad, except the middle hinge of a ball
    joint: +-U(0.5, 1.0) rad, which keeps it away from gimbal lock at 90 deg (where the three
    hinge axes span only two directions and M(q) is singular).  Contact: 4 spheres of radius
    3 cm on the last body of each leg; the root is lifted so that the lowest sphere touches
    z = 0 at q = 0.
    """
    rng = np.random.default_rng(seed)
    B = n_bodies
    parent = np.full(B, -1, dtype=np.int32)
    link = np.zeros((B, 3))
    chain_of = np.full(B, -1)
    legs_end = []
    # root body (pelvis-like), pointing up
    link[0] = _unit(np.array([0.0, 0.0, 1.0]) + 0.1 * rng.normal(size=3)) * rng.uniform(0.2, 0.5)
    nb = 1
    chain_id = 0
    while nb < B:
        clen = int(rng.integers(3, 9))
        clen = min(clen, B - nb)
        if contact and chain_id < n_legs:
            p = 0
            side = 1.0 if chain_id == 0 else -1.0
            cdir = _unit(np.array([0.0, 0.25 * side, -1.0]))
        else:
            p = int(rng.integers(0, nb))
            cdir = _unit(rng.normal(size=3))
        prev = p
        for j in range(clen):
            b = nb
            parent[b] = prev
            d = _unit(cdir + (0.15 if (contact and chain_id < n_legs) else 0.35) * rng.normal(size=3))
            if contact and chain_id < n_legs:
                d[2] = -abs(d[2])
                d = _unit(d)
            link[b] = d * rng.uniform(0.2, 0.5)
            chain_of[b] = chain_id
            prev = b
            nb += 1
        if contact and chain_id < n_legs:
            legs_end.append(prev)
        chain_id += 1

    # DoF allocation
    ndof = np.ones(B, dtype=np.int32)
    assert n_dofs <= max_dof_per_body * B
    while ndof.sum() < n_dofs:
        cand = np.nonzero(ndof < max_dof_per_body)[0]
        ndof[rng.choice(cand)] += 1
    assert ndof.sum() == n_dofs
    axes = []
    for b in range(B):
        rot = _random_rotation(rng)
        for k in range(ndof[b]):
            axes.append(rot[:, k])
    axes = np.asarray(axes)

    mass = rng.uniform(1.0, 8.0, size=B)
    lengths = np.linalg.norm(link, axis=1)
    com = 0.5 * link
    inertia = np.stack([capsule_inertia(mass[b], lengths[b], 0.1 * lengths[b], link[b]) for b in range(B)])

    # joint offsets: a child attaches at its parent's distal end
    offset = np.zeros((B, 3))
    for b in range(1, B):
        offset[b] = link[parent[b]]
    # world position of each body origin at q = 0 (all frames world aligned there), before lift
    origin0 = np.zeros((B, 3))
    for b in range(1, B):
        origin0[b] = origin0[parent[b]] + offset[b]

    # contact spheres
    spheres = []
    if contact:
        for fb in legs_end:
            d = _unit(link[fb])
            lat = _perp(rng, d)
            for frac, side in ((0.7, 1.0), (0.7, -1.0), (1.0, 1.0), (1.0, -1.0)):
                spheres.append((fb, frac * link[fb] + side * 0.04 * lat, sphere_radius))
        spheres = spheres[: n_legs * spheres_per_foot]
        low = min(origin0[b][2] + pos[2] - r for b, pos, r in spheres)
        root = np.array([0.0, 0.0, -low])
    else:
        root = np.array([0.0, 0.0, 1.5])
    offset[0] = root
    origin0 = origin0 + root

    # depth of each body (joints from the world)
    depth = np.zeros(B, dtype=np.int32)
    for b in range(1, B):
        depth[b] = depth[parent[b]] + 1

    # muscles: one path point on every body of the spanned chain, each placed next to the joint
    # it leads to or comes from (origin near the distal end of its body, insertion near the
    # proximal end of its body), extra points anywhere along a chain body.  Points sit
    # U(0.02, 0.06) m off the link axis, so moment arms have anatomical size (cm).
    def point_at(b, lo, hi):
        d = _unit(link[b])
        t = rng.uniform(lo, hi)
        r = rng.uniform(0.02, 0.06)
        return t, t * link[b] + r * _perp(rng, d)

    muscle_points = []
    while len(muscle_points) < n_muscles:
        ins = int(rng.integers(1, B))
        npts = int(rng.integers(2, max_points + 1))
        span = int(rng.integers(1, min(max_span, npts - 1) + 1))
        span = min(span, int(depth[ins]))
        chain = [ins]
        for _ in range(span):
            chain.append(int(parent[chain[-1]]))
        chain = chain[::-1]            # origin body first
        J = len(chain) - 1
        pts = [(0, ) + point_at(chain[0], 0.6, 0.95)]
        for ci in range(1, J):
            pts.append((ci, ) + point_at(chain[ci], 0.1, 0.9))
        pts.append((J, ) + point_at(chain[J], 0.05, 0.4))
        for _ in range(npts - len(pts)):
            ci = int(rng.integers(0, J + 1))
            lo, hi = (0.6, 0.95) if ci == 0 else ((0.05, 0.4) if ci == J else (0.1, 0.9))
            pts.append((ci, ) + point_at(chain[ci], lo, hi))
        ordered = sorted(pts, key=lambda x: (x[0], x[1]))
        world = np.array([origin0[chain[ci]] + x for ci, _, x in ordered])
        seg = np.linalg.norm(np.diff(world, axis=0), axis=1)
        if np.any(seg < 0.01):
            continue
        muscle_points.append([(chain[ci], x) for ci, _, x in ordered])
    fmax = rng.uniform(100.0, 3000.0, size=n_muscles)
    lopt = rng.uniform(0.05, 0.3, size=n_muscles)
    lslack = lopt * rng.uniform(1.0, 1.5, size=n_muscles)

    if limits:
        lim = np.stack([-rng.uniform(0.5, 2.0, size=n_dofs), rng.uniform(0.5, 2.0, size=n_dofs)], axis=1)
        starts = np.concatenate([[0], np.cumsum(ndof)[:-1]])
        for b in range(B):
            if ndof[b] == 3:
                mid = starts[b] + 1
                lim[mid] = [-rng.uniform(0.5, 1.0), rng.uniform(0.5, 1.0)]
    else:
        lim = np.zeros((n_dofs, 2))

    # wrapping cylinders (after every other draw, from their own stream, so the rest of the model
    # does not depend on wrap_frac): on a fraction of the muscles, the first segment that crosses
    # a joint wraps a cylinder at that joint, fixed to the distal body, its axis along the
    # joint's first hinge, radius 0.7 x the nearer point's distance from that axis at q = 0
    # (at most 5 cm)
    wraps = []
    if wrap_frac > 0:
        wr = np.random.default_rng(seed + 5000)
        starts = np.concatenate([[0], np.cumsum(ndof)[:-1]])
        for k in np.flatnonzero(wr.uniform(size=n_muscles) < wrap_frac):
            pts = muscle_points[k]
            for j in range(1, len(pts)):
                bp, bs = pts[j - 1][0], pts[j][0]
                if bp == bs:
                    continue
                a = _unit(np.asarray(axes[starts[bs]], dtype=np.float64))
                P = origin0[bp] + np.asarray(pts[j - 1][1])
                S = origin0[bs] + np.asarray(pts[j][1])
                dist = [np.linalg.norm((X - origin0[bs]) - ((X - origin0[bs]) @ a) * a) for X in (P, S)]
                r = min(0.7 * min(dist), 0.05)
                if r >= 0.005:
                    wraps.append((int(k), j, int(bs), (0.0, 0.0, 0.0), a, r, 0))
                break
        # a fraction of the surfaces become spheres centred at the joint, same radius (own
        # stream, so the cylinders' parameters do not depend on sphere_frac)
        sr = np.random.default_rng(seed + 6000)
        kinds = (sr.uniform(size=len(wraps)) < sphere_frac).astype(int)
        wraps = [w[:6] + (int(kd),) for w, kd in zip(wraps, kinds)]
    mdl = make_model(name or "synthetic", parent, ndof, offset, mass, com, inertia, axes,
                     muscle_points, fmax, lopt, lslack, dof_limit=lim, spheres=spheres, wraps=wraps)
    return with_free_root(mdl, name) if free_root else mdl


def config_model(name):
    """The synthetic model of a named workload (see :data:`CONFIGS`)."""
    return generate(name, **CONFIGS[name])


def tree_stats(model):
    """Depth statistics of the DoF tree (for reports): max DoF depth, sum of DoF depths."""
    n = model.n_dofs
    dparent = np.full(n, -1)
    for b in range(model.n_bodies):
        s, k = model.body_dof_start[b], model.body_ndof[b]
        pb = model.body_parent[b]
        dparent[s] = -1 if pb < 0 else model.body_dof_start[pb] + model.body_ndof[pb] - 1
        for j in range(1, k):
            dparent[s + j] = s + j - 1
    depth = np.zeros(n, dtype=np.int64)
    for i in range(n):
        depth[i] = 0 if dparent[i] < 0 else depth[dparent[i]] + 1
    bdepth = np.zeros(model.n_bodies, dtype=np.int64)
    for b in range(1, model.n_bodies):
        bdepth[b] = bdepth[model.body_parent[b]] + 1 if model.body_parent[b] >= 0 else 0
    return dict(max_dof_depth=int(depth.max()), sum_dof_depth1=int((depth + 1).sum()),
                max_body_depth=int(bdepth.max()), n_points=model.n_points)


# ----------------------------------------------------------------------------------------------
# states and excitations


def initial_state(model, n_envs, seed):
    """q0 ~ U(-0.3, 0.3) rad (clipped into enabled joint limits), qd0 = 0, act0 = 0; a free
    root starts at its model pose (q = 0: position offset, world-aligned)."""
    rng = np.random.default_rng(seed + 1000)
    n, m = model.n_dofs, model.n_muscles
    q = rng.uniform(-0.3, 0.3, size=(n_envs, n))
    lo, hi = model.dof_limit[:, 0], model.dof_limit[:, 1]
    on = lo < hi
    q[:, on] = np.clip(q[:, on], lo[on], hi[on])
    if model.free_root:
        q[:, :6] = 0.0
    return (q.astype(np.float32), np.zeros((n_envs, n), np.float32), np.zeros((n_envs, m), np.float32))


def uniform_excitations(model, n_envs, n_steps, seed):
    """Excitations drawn i.i.d. U(0, 1) per step and muscle: array [n_steps, n_envs, m]."""
    rng = np.random.default_rng(seed + 2000)
    return rng.uniform(0.0, 1.0, size=(n_steps, n_envs, model.n_muscles)).astype(np.float32)


def smooth_excitations(model, n_envs, n_steps, seed, dt=1e-3, t_filter=0.05, sigma=2.5):
    """Smooth random excitations: Gaussian noise N(0.5, sigma^2) per step, first-order low-pass
    with time constant ``t_filter`` (50 ms), clipped to [0, 1].  Array [n_steps, n_envs, m].
    """
    rng = np.random.default_rng(seed + 3000)
    m = model.n_muscles
    y = np.full((n_envs, m), 0.5)
    out = np.empty((n_steps, n_envs, m), np.float32)
    g = dt / t_filter
    for t in range(n_steps):
        x = rng.normal(0.5, sigma, size=(n_envs, m))
        y = y + g * (x - y)
        out[t] = np.clip(y, 0.0, 1.0)
    return out
