"""Algorithmic FP32 operation counts of one substep of one environment (the roofline numerator).

The count is of the method's arithmetic, stage by stage, as the algorithm needs it (an FMA is 2
FLOPs; sin/cos/exp/sqrt/rsqrt/division count as 1 each, i.e. not inflated by their instruction
cost): forward kinematics, the Newton-Euler bias, the composite-rigid-body mass matrix, via-point
muscle geometry and moment arms, the Hill force (Eq. 1) and activation update (Eq. 2), R^T F,
the implicit-damping terms, contact detection, joint limits, the tree-sparse L^T L
factorisation, the two triangular solves and the integration.  Extended-precision overhead
(the float-float words used for the mass matrix) is implementation cost and is not counted.
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


def flops_per_env_substep(model):
    """Dict stage -> FLOPs for one environment and one substep, plus 'total'."""
    n, nb, m, P, S = model.n_dofs, model.n_bodies, model.n_muscles, model.n_points, model.n_spheres
    _, depth = tree(model)
    nx = crossed_dofs(model)
    nnz = int(nx.sum())
    n_packed = int((depth + 1).sum())
    f = {}
    f["kinematics"] = n * (15 + 6 + 2 + 48) + nb * 18             # axis, p x s, sincos, R update; offsets
    f["velocities"] = n * 36                                         # v, bias acceleration per hinge
    f["body_forces"] = nb * (45 + 27 + 24 + 2 * 30 + 36)             # R I R^T, parallel axis, I v, I a, cross terms
    f["bias_rnea"] = nb * 6 + n * 11                                 # subtree force sums, S^T f
    f["crba"] = nb * 10 + n * 36 + n_packed * 11                     # composite inertia, F = Ic S, S_a^T F
    f["muscle_geometry"] = P * 18 + (P - m) * 16 + nnz * 21          # points, segments, moment arms, dL/dt
    f["hill_activation"] = m * 45                                     # f_l, f_v, f_p, dF/dLdot, Eq. 2
    f["tau_muscle"] = nnz * 2
    f["implicit_damping"] = int((nx * (nx + 1) // 2).sum()) * 3 + m * 3
    f["contact_detect"] = S * 60
    f["limits"] = n * 10
    f["factor"] = n * 3 + int(depth.sum()) + int((depth * (depth + 1) // 2).sum()) * 2
    f["solves"] = 4 * int(depth.sum()) + 2 * n
    f["integrate"] = 4 * n
    f["total"] = int(sum(f.values()))
    return f
