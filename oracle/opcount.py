"""Instrumented count of the floating-point operations of one substep of one environment.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): the tests may call it; the product never
does.  Shares no code with the CUDA path.

The roofline of the step kernel divides the method's arithmetic by the kernel's time.  This
module counts that arithmetic by *running* the method's algorithms, stage by stage, on numbers
that count every operation applied to them: +, -, *, / and sqrt, sin, cos, exp each count one
(an FMA is two: its multiply and its add); comparisons, negations, clamps and branch tests count
nothing.  The algorithms are the ones the method needs for a tree of hinges (written from their
definitions, not from the CUDA source), and every stage's values are checked against the FP64
oracle's independent formulations by the tests, so the count is of a working implementation:

  kinematics       body frames and joint axes: R_b, origin p_b = p_parent + R_parent offset_b,
                   world axis s_d = R a_d, R <- R Rot(a_d, q_d) (Rodrigues)
  velocities       spatial body velocities V_b = V_parent + sum_d S_d qd_d and velocity-product
                   accelerations A_b = A_parent + V x S_d qd_d, world frame at the origin, with
                   S_d = (s_d, o_d x s_d) and the base acceleration -g (gravity)
  body_forces      world-frame spatial inertia (m, h = m c, J about the origin) of every body
                   and its Newton-Euler force f_b = I_b A_b + V_b x* (I_b V_b)
  bias_rnea        subtree force sums f_sub and the bias C_d = S_d . f_sub(body of d)
  crba             composite inertias I^c_b and M_{d,a} = S_a . (I^c_{body d} S_d) over the
                   ancestors a of d (the packed tree pattern)
  muscle_geometry  world via points x = R_b p + p_b, segment lengths, unit directions, moment arms
                   R_kd = -s_d . ((x_distal - o_d) x u) of the DoFs each segment crosses, and
                   dL/dt = -sum_d R_kd qd_d
  hill_activation  l_m, v_m, f_l, f_v, f_p, F (Eq. 1), dF/dLdot, and the activation update (Eq. 2)
  tau_muscle       tau = R^T F over the non-zeros
  implicit_damping dF/dLdot R_k R_k^T over each muscle's crossed DoFs (lower triangle) into D
  contact_detect   world sphere centres and penetration depths (the force and torque work of the
                   spheres in contact depends on the state and is not counted)
  limits           joint damping torque and diagonal (the penalty of a DoF past its limit depends
                   on the state and is not counted)
  assemble         A = M + dt D over the packed pattern and rhs = tau_m + tau_l - C
  factor           tree-sparse A = L^T L eliminating leaves first (pivot, row scaling, Schur
                   updates over pairs of ancestors) with the right-hand side as one more column
  solves           the rest of L^T y = b (updates of the ancestors' right-hand sides) and the
                   root-first L x = y
  integrate        qd += dt qdd, q += dt qd

count_substep(model, dt, q, qd, act, exc) returns (counts per stage, values) where values holds
L, R, M, A, bias, rhs, qdd, force for the tests to compare with the oracle.
"""
from __future__ import annotations

import math

import numpy as np


class Tally:
    def __init__(self):
        self.stage = None
        self.counts = {}

    def add(self, k=1):
        self.counts[self.stage] = self.counts.get(self.stage, 0) + k


_T = Tally()


def _v(x):
    return x.v if isinstance(x, N) else float(x)


class N:
    """A float that counts the arithmetic applied to it (into the current stage)."""
    __slots__ = ("v",)

    def __init__(self, v):
        self.v = float(v)

    def __add__(self, o):
        _T.add()
        return N(self.v + _v(o))

    __radd__ = __add__

    def __sub__(self, o):
        _T.add()
        return N(self.v - _v(o))

    def __rsub__(self, o):
        _T.add()
        return N(_v(o) - self.v)

    def __mul__(self, o):
        _T.add()
        return N(self.v * _v(o))

    __rmul__ = __mul__

    def __truediv__(self, o):
        _T.add()
        return N(self.v / _v(o))

    def __rtruediv__(self, o):
        _T.add()
        return N(_v(o) / self.v)

    def __neg__(self):
        return N(-self.v)

    def __gt__(self, o):
        return self.v > _v(o)

    def __lt__(self, o):
        return self.v < _v(o)

    def __ge__(self, o):
        return self.v >= _v(o)

    def __le__(self, o):
        return self.v <= _v(o)


def sqrt(x):
    _T.add()
    return N(math.sqrt(_v(x)))


def exp(x):
    _T.add()
    return N(math.exp(_v(x)))


def sincos(x):
    _T.add(2)
    return N(math.sin(_v(x))), N(math.cos(_v(x)))


def clamp(x, lo, hi):
    return N(min(max(_v(x), lo), hi))


# ------------------------------------------------------------------ 3-vectors of counted numbers
def cross(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def add(a, b):
    return [a[0] + b[0], a[1] + b[1], a[2] + b[2]]


def sub(a, b):
    return [a[0] - b[0], a[1] - b[1], a[2] - b[2]]


def scale(a, s):
    return [a[0] * s, a[1] * s, a[2] * s]


def matvec(R, x):   # R row-major 3 x 3
    return [R[0] * x[0] + R[1] * x[1] + R[2] * x[2], R[3] * x[0] + R[4] * x[1] + R[5] * x[2],
            R[6] * x[0] + R[7] * x[1] + R[8] * x[2]]


def matmul(A, B):
    return [A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j] for i in range(3) for j in range(3)]


def rodrigues(a, sn, cs):
    """Rotation by angle (sin, cos) about the constant unit axis a: c I + s [a]x + (1 - c) a a^T."""
    k = 1.0 - cs
    ka = [a[0] * k, a[1] * k, a[2] * k]
    sa = [a[0] * sn, a[1] * sn, a[2] * sn]
    xy, xz, yz = ka[0] * a[1], ka[0] * a[2], ka[1] * a[2]
    return [ka[0] * a[0] + cs, xy - sa[2], xz + sa[1],
            xy + sa[2], ka[1] * a[1] + cs, yz - sa[0],
            xz - sa[1], yz + sa[0], ka[2] * a[2] + cs]


# ------------------------------------------------------------------ spatial (world frame, origin)
def inertia_apply(I, V):
    """I = (m, h, J): (n, F) = (J w + h x v, m v - h x w) for V = (w, v)."""
    m, h, J = I
    w, v = V
    Jw = [J[0] * w[0] + J[3] * w[1] + J[4] * w[2], J[3] * w[0] + J[1] * w[1] + J[5] * w[2],
          J[4] * w[0] + J[5] * w[1] + J[2] * w[2]]
    return (add(Jw, cross(h, v)), sub(scale(v, m), cross(h, w)))


def cross_force(V, f):
    """V x* f = (w x n + v x F, w x F)."""
    w, v = V
    n, F = f
    return (add(cross(w, n), cross(v, F)), cross(w, F))


def cross_motion(V, S):
    """V x S = (w x w', w x v' + v x w')."""
    w, v = V
    w2, v2 = S
    return (cross(w, w2), add(cross(w, v2), cross(v, w2)))


def fl(l):
    d = l - 1.0
    return exp(d * d * (-1.0 / 0.45))


def fp(l):
    if l <= 1.0:
        return N(0.0)
    e4 = math.exp(4.0)
    if l <= 1.6:
        return (exp((l - 1.0) * (4.0 / 0.6)) - 1.0) * (1.0 / (e4 - 1.0))
    return (l - 1.6) * ((4.0 / 0.6) * e4 / (e4 - 1.0)) + 1.0


def fv(v):
    if v < -1.0:
        return N(0.0)
    if v <= 0.0:
        return (v + 1.0) / (1.0 - v * 4.0)
    return v * 0.4 / (v + 0.08) + 1.0


def dfv(v):
    if v < -1.0:
        return N(0.0)
    if v <= 0.0:
        d = 1.0 - v * 4.0
        return 5.0 / (d * d)
    d = v + 0.08
    return 0.032 / (d * d)


# ------------------------------------------------------------------ the substep
def _tree(model):
    n, nb = model.n_dofs, model.n_bodies
    dbody = np.zeros(n, dtype=int)
    par = np.full(n, -1)
    for b in range(nb):
        s0, k, pb = model.body_dof_start[b], model.body_ndof[b], model.body_parent[b]
        dbody[s0:s0 + k] = b
        par[s0] = -1 if pb < 0 else model.body_dof_start[pb] + model.body_ndof[pb] - 1
        for j in range(1, k):
            par[s0 + j] = s0 + j - 1
    anc = []
    for d in range(n):
        a, chain = d, []
        while a >= 0:
            chain.append(a)
            a = par[a]
        anc.append(chain)   # d first, root last
    return dbody, par, anc


STAGES = ("kinematics", "velocities", "body_forces", "bias_rnea", "crba", "muscle_geometry", "hill_activation",
          "tau_muscle", "implicit_damping", "contact_detect", "limits", "assemble", "factor", "solves", "integrate")


def count_substep(model, dt, q, qd, act, exc, L0):
    """Counts per stage and the values (see the module docstring).  Fixed-base hinge models
    without wrapping surfaces or compliant tendons."""
    assert not getattr(model, "free_root", False) and model.wrap_muscle.shape[0] == 0
    assert not np.any(np.asarray(model.muscle_tendon_strain) > 0)
    _T.counts = {k: 0 for k in STAGES}
    n, nb, m = model.n_dofs, model.n_bodies, model.n_muscles
    dbody, par, anc = _tree(model)
    qN = [N(x) for x in q]
    qdN = [N(x) for x in qd]

    # kinematics
    _T.stage = "kinematics"
    Rb, pb = [None] * nb, [None] * nb
    s, o = [None] * n, [None] * n
    for b in range(nb):
        pa = model.body_parent[b]
        off = [float(x) for x in model.body_offset[b]]
        if pa < 0:
            R = [N(1.0), N(0.0), N(0.0), N(0.0), N(1.0), N(0.0), N(0.0), N(0.0), N(1.0)]
            p = [N(x) for x in off]
        else:
            R = list(Rb[pa])
            p = add(pb[pa], matvec(R, off))
        for j in range(model.body_ndof[b]):
            d = model.body_dof_start[b] + j
            a = [float(x) for x in model.dof_axis[d]]
            s[d] = matvec(R, a)
            o[d] = p
            sn, cs = sincos(qN[d])
            R = matmul(R, rodrigues(a, sn, cs))
        Rb[b], pb[b] = R, p

    # velocities and velocity-product accelerations
    _T.stage = "velocities"
    S = [(s[d], cross(o[d], s[d])) for d in range(n)]
    V, A = [None] * nb, [None] * nb
    g = [float(x) for x in model.gravity]
    for b in range(nb):
        pa = model.body_parent[b]
        if pa < 0:
            Vb = ([N(0.0)] * 3, [N(0.0)] * 3)
            Ab = ([N(0.0)] * 3, [N(-g[0]), N(-g[1]), N(-g[2])])
        else:
            Vb, Ab = V[pa], A[pa]
        for j in range(model.body_ndof[b]):
            d = model.body_dof_start[b] + j
            Sq = (scale(S[d][0], qdN[d]), scale(S[d][1], qdN[d]))
            c = cross_motion(Vb, Sq)
            Ab = (add(Ab[0], c[0]), add(Ab[1], c[1]))
            Vb = (add(Vb[0], Sq[0]), add(Vb[1], Sq[1]))
        V[b], A[b] = Vb, Ab

    # body inertias in the world frame and Newton-Euler body forces
    _T.stage = "body_forces"
    Ib, fb = [None] * nb, [None] * nb
    for b in range(nb):
        mass = float(model.body_mass[b])
        R = Rb[b]
        ii = [float(x) for x in model.body_inertia[b]]
        Ic = [ii[0], ii[3], ii[4], ii[3], ii[1], ii[5], ii[4], ii[5], ii[2]]
        RI = matmul(R, Ic)
        # J_c = R I R^T (symmetric: 6 entries, each a 3-term dot product)
        Jc = [RI[0] * R[0] + RI[1] * R[1] + RI[2] * R[2], RI[3] * R[3] + RI[4] * R[4] + RI[5] * R[5],
              RI[6] * R[6] + RI[7] * R[7] + RI[8] * R[8], RI[0] * R[3] + RI[1] * R[4] + RI[2] * R[5],
              RI[0] * R[6] + RI[1] * R[7] + RI[2] * R[8], RI[3] * R[6] + RI[4] * R[7] + RI[5] * R[8]]
        c = add(pb[b], matvec(R, [float(x) for x in model.body_com[b]]))
        h = scale(c, mass)
        # J about the origin = J_c + m (|c|^2 I - c c^T) = J_c + |c|^2 m I - h c^T
        cc = dot(c, c) * mass
        J = [Jc[0] + cc - h[0] * c[0], Jc[1] + cc - h[1] * c[1], Jc[2] + cc - h[2] * c[2],
             Jc[3] - h[0] * c[1], Jc[4] - h[0] * c[2], Jc[5] - h[1] * c[2]]
        Ib[b] = (N(mass), h, J)
        IA = inertia_apply(Ib[b], A[b])
        IV = inertia_apply(Ib[b], V[b])
        x = cross_force(V[b], IV)
        fb[b] = (add(IA[0], x[0]), add(IA[1], x[1]))

    # subtree sums and the bias
    _T.stage = "bias_rnea"
    fsub = [list(f) for f in fb]
    for b in range(nb - 1, 0, -1):
        pa = model.body_parent[b]
        if pa >= 0:
            fsub[pa] = [add(fsub[pa][0], fsub[b][0]), add(fsub[pa][1], fsub[b][1])]
    C = [dot(S[d][0], fsub[dbody[d]][0]) + dot(S[d][1], fsub[dbody[d]][1]) for d in range(n)]

    # composite inertias and the packed mass matrix
    _T.stage = "crba"
    Icb = [(Ib[b][0], list(Ib[b][1]), list(Ib[b][2])) for b in range(nb)]
    for b in range(nb - 1, 0, -1):
        pa = model.body_parent[b]
        if pa >= 0:
            mp, hp, Jp = Icb[pa]
            mc, hc, Jc = Icb[b]
            Icb[pa] = (mp + mc, add(hp, hc), [Jp[i] + Jc[i] for i in range(6)])
    M = {}
    for d in range(n):
        F = inertia_apply(Icb[dbody[d]], S[d])
        for a in anc[d]:
            M[(d, a)] = dot(S[a][0], F[0]) + dot(S[a][1], F[1])

    # muscle geometry
    _T.stage = "muscle_geometry"
    Lm, Rm, ldot = [], [], []
    for k in range(m):
        j0, j1 = model.muscle_point_start[k], model.muscle_point_start[k + 1]
        origin = model.point_body[j0]
        chain = []
        b = model.point_body[j1 - 1]
        while b != origin:
            chain.append(b)
            b = model.body_parent[b]
        chain = chain[::-1]
        pos = {origin: 0}
        for t, bb in enumerate(chain):
            pos[bb] = t + 1
        crossed = [[] for _ in range(len(chain) + 1)]   # DoFs entered at chain position t
        for t, bb in enumerate(chain):
            s0 = model.body_dof_start[bb]
            crossed[t + 1] = list(range(s0, s0 + model.body_ndof[bb]))
        row, length, ld = {}, N(0.0), N(0.0)
        x0 = None
        for j in range(j0, j1):
            bb = model.point_body[j]
            x = add(matvec(Rb[bb], [float(v) for v in model.point_pos[j]]), pb[bb])
            if x0 is not None:
                dv = sub(x, x0)
                l2 = dot(dv, dv)
                ln = sqrt(l2)
                length = length + ln
                inv = 1.0 / ln
                u = scale(dv, inv)
                for t in range(pos[model.point_body[j - 1]] + 1, pos[bb] + 1):
                    for d in crossed[t]:
                        r = sub(x, o[d])
                        Rv = -dot(s[d], cross(r, u))
                        row[d] = Rv
                        ld = ld - Rv * qdN[d]
            x0 = x
        Lm.append(length)
        Rm.append(row)
        ldot.append(ld)

    # Hill force (Eq. 1) and activation (Eq. 2)
    _T.stage = "hill_activation"
    Fm, dF, act_next = [], [], []
    for k in range(m):
        inv_lopt = 1.0 / float(model.muscle_lopt[k])
        inv_vmax = 1.0 / (model.vmax_per_lopt * float(model.muscle_lopt[k]))
        lm = (Lm[k] - float(L0[k])) * inv_lopt + 1.0
        vm = ldot[k] * inv_vmax
        a = N(act[k])
        fll = fl(lm)
        fvv = fv(vm)
        afl = a * fll
        F = (afl * fvv + fp(lm)) * float(model.muscle_fmax[k])
        Fm.append(F)
        dF.append(afl * dfv(vm) * (float(model.muscle_fmax[k]) * inv_vmax))
        u = clamp(N(exc[k]), 0.0, 1.0)
        sh = a * 1.5 + 0.5
        tau = model.tau_act * sh if u > a else model.tau_deact / sh
        act_next.append(clamp(a + (u - a) / tau * dt, 0.0, 1.0))

    _T.stage = "tau_muscle"
    tau_m = [N(0.0) for _ in range(n)]
    for k in range(m):
        for d, Rv in Rm[k].items():
            tau_m[d] = tau_m[d] + Rv * Fm[k]

    _T.stage = "implicit_damping"
    D = {}
    for k in range(m):
        ds = sorted(Rm[k].keys())
        for i, da in enumerate(ds):
            gi = dF[k] * Rm[k][da]
            for db in ds[:i + 1]:       # db <= da: db is an ancestor of da on the muscle's chain
                D[(da, db)] = D.get((da, db), N(0.0)) + gi * Rm[k][db]

    _T.stage = "contact_detect"
    depth = []
    for i in range(model.n_spheres):
        bb = model.sphere_body[i]
        x = add(matvec(Rb[bb], [float(v) for v in model.sphere_pos[i]]), pb[bb])
        depth.append(float(model.sphere_radius[i]) - x[2])
    if any(dd.v > 0.0 for dd in depth):
        raise ValueError("count_substep: a sphere is in contact (its force work is not counted)")

    _T.stage = "limits"
    tl, diag = [None] * n, [None] * n
    for d in range(n):
        lo, hi = model.dof_limit[d]
        if lo < hi and not (lo <= q[d] <= hi):
            raise ValueError("count_substep: a DoF is past its limit (its penalty work is not counted)")
        b = N(model.dof_damping[d])
        tl[d] = -(qdN[d] * b)
        diag[d] = b * dt

    # A = M + dt D in the packed pattern, rhs = tau - C
    _T.stage = "assemble"
    Amat = {}
    rhs = [None] * n
    for d in range(n):
        for a in anc[d]:
            Amat[(d, a)] = M[(d, a)] + D[(d, a)] * dt if (d, a) in D else M[(d, a)]
        Amat[(d, d)] = Amat[(d, d)] + diag[d]
        rhs[d] = tau_m[d] + tl[d] - C[d]

    # tree-sparse A = L^T L, leaves first; the right-hand side rides along as one more column
    _T.stage = "factor"
    Lf = dict(Amat)
    y = list(rhs)
    for k in range(n - 1, -1, -1):        # children have larger indices than their parents
        lkk = sqrt(Lf[(k, k)])
        inv = 1.0 / lkk
        Lf[(k, k)] = lkk
        for a in anc[k][1:]:
            Lf[(k, a)] = Lf[(k, a)] * inv
        y[k] = y[k] * inv
        ak = anc[k][1:]
        for i, a in enumerate(ak):
            for b in ak[i:]:              # b ancestor-or-self of a
                Lf[(a, b)] = Lf[(a, b)] - Lf[(k, a)] * Lf[(k, b)]
        _T.stage = "solves"
        for a in ak:
            y[a] = y[a] - Lf[(k, a)] * y[k]
        _T.stage = "factor"
    _T.stage = "solves"
    x = [None] * n
    for k in range(n):                    # root first
        acc = y[k]
        for a in anc[k][1:]:
            acc = acc - Lf[(k, a)] * x[a]
        x[k] = acc / Lf[(k, k)]

    _T.stage = "integrate"
    qd1 = [qdN[d] + x[d] * dt for d in range(n)]
    q1 = [qN[d] + qd1[d] * dt for d in range(n)]

    counts = dict(_T.counts)
    counts["total"] = int(sum(counts.values()))
    Rd = np.zeros((m, n))
    for k in range(m):
        for d, v in Rm[k].items():
            Rd[k, d] = v.v
    full = lambda P: np.array([[P[(i, j)].v if (i, j) in P else (P[(j, i)].v if (j, i) in P else 0.0)
                                for j in range(n)] for i in range(n)])
    values = dict(L=np.array([v.v for v in Lm]), R=Rd, M=full(M), A=full(Amat), bias=np.array([v.v for v in C]),
                  rhs=np.array([v.v for v in rhs]), qdd=np.array([v.v for v in x]),
                  force=np.array([v.v for v in Fm]), act_next=np.array([v.v for v in act_next]),
                  tau_m=np.array([v.v for v in tau_m]), q_next=np.array([v.v for v in q1]))
    return counts, values
