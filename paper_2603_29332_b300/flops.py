"""Algorithmic FP32 operation counts of one substep of one environment (the roofline numerator).

The count is of the method's arithmetic, stage by stage, as the algorithm needs it (an FMA is 2
FLOPs; sin/cos/exp/sqrt/rsqrt/division count as 1 each, i.e. not inflated by their instruction
cost): forward kinematics, the Newton-Euler bias, the composite-rigid-body mass matrix, via-point
muscle geometry and moment arms, the Hill force (Eq. 1) and activation update (Eq. 2), R^T F,
the implicit-damping terms, contact detection, joint limits, the assembly of the system, the
tree-sparse L^T L factorisation, the two triangular solves and the integration.
Extended-precision overhead (the float-float words used for the mass matrix) is implementation
cost and is not counted.  The per-element costs are those of an instrumented run of the same
algorithms (the tests compare this formula with that count, stage by stage).
"""
import numpy as np


def tree(model):
    """DoF parents and depths of a model (host-side structure only)."""
    n = model.n_dofs
    par = np.full(n, -1)
    for b in range(model.n_bodies):
        s, c, pb = model.body_dof_start[b], model.body_ndof[b], model.body_parent[b]
        par[s] = -1 if pb < 0 else model.body_dof_start[pb] + model.body_ndof[pb] - 1
        for j in range(1, c):
            par[s + j] = s + j - 1
    depth = np.zeros(n, dtype=np.int64)
    for i in range(n):
        depth[i] = 0 if par[i] < 0 else depth[par[i]] + 1
    return par, depth


def crossed_dofs(model):
    """Number of DoFs each muscle crosses (the non-zeros of its row of R)."""
    out = np.zeros(model.n_muscles, dtype=np.int64)
    for k in range(model.n_muscles):
        j0, j1 = model.muscle_point_start[k], model.muscle_point_start[k + 1]
        origin, b = model.point_body[j0], model.point_body[j1 - 1]
        cnt = 0
        while b != origin:
            cnt += model.body_ndof[b]
            b = model.body_parent[b]
        out[k] = cnt
    return out


def damping_pairs(model):
    """Distinct (DoF, ancestor DoF) pairs that some muscle couples in the implicit damping (both
    among the DoFs it crosses): the entries of the packed matrix that receive dt D."""
    pairs = set()
    for k in range(model.n_muscles):
        j0, j1 = model.muscle_point_start[k], model.muscle_point_start[k + 1]
        origin, b = model.point_body[j0], model.point_body[j1 - 1]
        ds = []
        while b != origin:
            s0 = model.body_dof_start[b]
            ds.extend(range(s0, s0 + model.body_ndof[b]))
            b = model.body_parent[b]
        ds.sort()
        for i, da in enumerate(ds):
            for db in ds[:i + 1]:
                pairs.add((da, db))
    return len(pairs)


# per-element operation costs of the stages (see flops_per_env_substep)
HILL_PER_MUSCLE = 31   # l_m, v_m, f_l, f_v, F, dF/dLdot, Eq. 2; f_p's exponential branch adds 5


def flops_per_env_substep(model):
    """Dict stage -> FLOPs for one environment and one substep, plus 'total'.

    Per structural element: a child body's origin 18 (3 x 3 product and sum); a hinge's
    kinematics 84 (world axis 15, sine and cosine 2, Rodrigues rotation 22, frame product 45);
    its velocity and velocity-product acceleration 57; a body's world inertia and Newton-Euler
    force 237; a child body's subtree force sum 6 and composite inertia 10; a DoF's bias
    projection 11 and composite-inertia product 42; a packed mass-matrix entry 11; a via point
    18; a straight segment 14 (difference, length, direction); a crossed DoF's moment arm and
    dL/dt term 19, its torque term 2; per muscle and crossed DoF pair (lower triangle) of the
    implicit damping 2, plus 1 per crossed DoF; a sphere's centre and depth 19; a DoF's joint
    damping 2; assembly 2 per damped packed entry and 3 per DoF; the tree factorisation 3 per
    node plus its row length plus twice its Schur updates; the solves 4 per ancestor entry plus 1
    per node; integration 4 per DoF.  The Hill and activation stage depends on the branch of the
    curves (HILL_PER_MUSCLE is its common case: no passive force, either fibre-velocity branch).
    The instrumented counter of the test infrastructure reproduces every structural stage
    exactly."""
    n, nb, m, P, S = model.n_dofs, model.n_bodies, model.n_muscles, model.n_points, model.n_spheres
    _, depth = tree(model)
    nx = crossed_dofs(model)
    nnz = int(nx.sum())
    n_packed = int((depth + 1).sum())
    child_bodies = int((model.body_parent >= 0).sum())
    f = {}
    f["kinematics"] = child_bodies * 18 + n * 84
    f["velocities"] = n * 57
    f["body_forces"] = nb * 237
    f["bias_rnea"] = child_bodies * 6 + n * 11
    f["crba"] = child_bodies * 10 + n * 42 + n_packed * 11
    f["muscle_geometry"] = P * 18 + (P - m) * 14 + nnz * 19
    f["hill_activation"] = m * HILL_PER_MUSCLE
    f["tau_muscle"] = nnz * 2
    f["implicit_damping"] = nnz + int((nx * (nx + 1)).sum())
    f["contact_detect"] = S * 19
    f["limits"] = n * 2
    f["assemble"] = 2 * damping_pairs(model) + 3 * n
    f["factor"] = n * 3 + int(depth.sum()) + int((depth * (depth + 1)).sum())
    f["solves"] = 4 * int(depth.sum()) + n
    f["integrate"] = 4 * n
    f["total"] = int(sum(f.values()))
    return f
