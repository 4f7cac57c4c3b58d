/*
 * msim_model.h -- model description consumed by msim_create (host memory, caller-owned).
 *
 * A musculoskeletal model in the sense of the paper's Methods ("Whole-body musculoskeletal
 * model", "Muscle-tendon dynamics", "Contact modeling"): a tree of rigid bodies joined by
 * hinge DoFs, Hill-type muscle-tendon units routed through via points, and contact spheres
 * against the ground plane z = 0.
 *
 * Geometry conventions:
 *   - Bodies are listed parents first: body_parent[b] < b, -1 = the fixed world.
 *   - Body b owns body_ndof[b] in {1,2,3} hinge DoFs, numbered consecutively in body order
 *     (6 free DoFs for body 0 with free_root, below).
 *   - Frame of body b = frame of its parent * translate(body_offset[b]) * Rot(a_0, q_0) * ...
 *     * Rot(a_{k-1}, q_{k-1}), each axis a_j (dof_axis, unit) given in the frame just before
 *     its hinge.  The body origin is the joint origin.
 *   - body_com, body_inertia (xx, yy, zz, xy, xz, yz about the COM), point_pos, sphere_pos
 *     are in the body frame.  Units: m, kg, s, N.
 *   - Muscle k runs through points muscle_point_start[k] .. muscle_point_start[k+1]-1
 *     (origin first).  Consecutive points must lie on the same body or on a descendant of
 *     it, all on the one ancestor chain from the origin body to the insertion body.
 *   - dof_limit[2d], dof_limit[2d+1] = lo, hi [rad]; lo >= hi disables the limit.
 *
 * Limits of this build: n_dofs <= 255, n_bodies <= 255, max DoF depth <= 63, points per
 * muscle <= 8, DoFs crossed per muscle <= 12, n_spheres <= 32, n_muscles <= 4096,
 * n_wraps <= 255.
 */
#ifndef MSIM_MODEL_H
#define MSIM_MODEL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t n_bodies, n_dofs, n_muscles, n_points, n_spheres;
    const int32_t* body_parent;        /* [n_bodies] */
    const int32_t* body_ndof;          /* [n_bodies] */
    const float* body_offset;          /* [n_bodies][3] */
    const float* body_mass;            /* [n_bodies] */
    const float* body_com;             /* [n_bodies][3] */
    const float* body_inertia;         /* [n_bodies][6] */
    const float* dof_axis;             /* [n_dofs][3] */
    const float* dof_limit;            /* [n_dofs][2] */
    const float* dof_damping;          /* [n_dofs], N m s / rad */
    const int32_t* muscle_point_start; /* [n_muscles + 1] */
    const float* muscle_fmax;          /* [n_muscles] maximum isometric force F_max (Eq. 1) */
    const float* muscle_lopt;          /* [n_muscles] optimal fibre length */
    const float* muscle_lslack;        /* [n_muscles] tendon slack length (recorded, unused: a
                                        * compliant tendon's slack length follows from L0 below) */
    const int32_t* point_body;         /* [n_points] */
    const float* point_pos;            /* [n_points][3] */
    const int32_t* sphere_body;        /* [n_spheres] */
    const float* sphere_pos;           /* [n_spheres][3] */
    const float* sphere_radius;        /* [n_spheres] */
    float gravity[3];                  /* m / s^2 */
    float contact_k, contact_c;        /* penalty stiffness N/m and damping N s/m */
    float contact_mu, contact_eps;     /* Coulomb coefficient, friction smoothing velocity m/s */
    float limit_k, limit_c;            /* joint-limit stiffness N m/rad, damping N m s/rad */
    float tau_act, tau_deact;          /* activation / deactivation time constants (Eq. 2) */
    float vmax_per_lopt;               /* maximum contraction velocity in l_opt per second */
    /* wrapping surfaces (may be 0 / NULL): the segment of muscle wrap_muscle[w] that ends at
     * its point number wrap_segment[w] (1 .. points - 1) takes the shortest way around an
     * infinite cylinder (or a sphere, wrap_kind below) fixed to body wrap_body[w] (on the muscle's chain between that segment's
     * two bodies), centre and axis in that body's frame; at most one cylinder per muscle */
    int32_t n_wraps;
    const int32_t* wrap_muscle;        /* [n_wraps] */
    const int32_t* wrap_segment;       /* [n_wraps] */
    const int32_t* wrap_body;          /* [n_wraps] */
    const float* wrap_center;          /* [n_wraps][3] */
    const float* wrap_axis;            /* [n_wraps][3] (normalised by the library) */
    const float* wrap_radius;          /* [n_wraps], > 0 */
    /* free (floating) root: 0 = every root body is fixed to the world.  1 = body 0 (a root) is
     * joined to the world by six DoFs 0-5 (body_ndof[0] = 6; its dof_axis rows are ignored and
     * its dof_limit rows must be disabled): DoFs 0-2 translate its origin along world x, y, z
     * (q = position offset from body_offset[0] in m, qd = velocity), DoFs 3-5 turn it about
     * world x, y, z through its origin (qd = angular velocity in the world frame, rad/s; q =
     * the rotation vector of its orientation, rad, advanced by R <- exp(dt w) R each substep and
     * kept at angle <= pi).  The paper's skeleton has such a root ("Observation space"). */
    int32_t free_root;
    /* kind of each wrapping surface: 0 = cylinder, 1 = sphere (centre wrap_center, radius
     * wrap_radius; wrap_axis unused): the wrapped segment follows the great circle in the plane
     * through its two points and the centre.  NULL = all cylinders. */
    const int32_t* wrap_kind;          /* [n_wraps] or NULL */
    /* compliant tendons (NULL = every tendon rigid, the paper's model): per muscle, the tendon
     * strain at F_max, eps0 in (0, 0.5] for a compliant tendon, 0 for a rigid one.  A compliant
     * tendon's slack length is l_s = L0 - l_opt (L0 the length at q = 0), which must be at least
     * 0.5 l_opt (checked at create); its strain eps is a state (msim_tendon_strain, zero after a
     * reset).  Per substep: fibre length l_m = (L - l_s (1 + eps)) / l_opt; tendon force
     * F_max f_t(eps / eps0) with f_t(x) = (e^{3x} - 1 - 3x)/(e^3 - 4) on [0, 1], linear (C1)
     * beyond, 0 when slack (C1 at slack too); the fibre velocity v_m solves act f_l f_v(v_m) + f_p + 0.1 v_m = f_t (a
     * damped fibre, Millard 2013); eps advances linearly implicitly by
     * d eps/dt = (dL/dt - v_max v_m) / l_s, and the skeleton receives the tendon force at the
     * new strain, its dL/dt derivative taken into the implicit damping. */
    const float* muscle_tendon_strain; /* [n_muscles] or NULL */
    /* onset width of the joint-limit penalty, rad (>= 0): over the first limit_delta of the
     * excess x past a limit the spring torque grows as limit_k x^2 / (2 limit_delta) and the
     * damper as limit_c x / limit_delta; beyond, limit_k (x - limit_delta / 2) and limit_c.  The
     * torque and its derivatives in q and qd are then continuous at the limit, so the linearly
     * implicit step has no jump there.  0 = the plain penalty limit_k x, limit_c.  Stability: the
     * implicit coefficient (limit_k dt + limit_c) x / limit_delta then depends on the excess, and a
     * joint entering the onset at speed qd meets an explicit stiffness
     * (limit_k dt + limit_c) |qd| / limit_delta, which must stay well below I / dt^2 (I the joint's
     * effective inertia); the plain penalty has no such term. */
    float limit_delta;
} msim_model_desc;

#ifdef __cplusplus
}
#endif
#endif /* MSIM_MODEL_H */
