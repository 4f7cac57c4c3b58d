/*
 * msim_oracle.c -- plain, slow FP64 CPU oracle of the batched muscle-driven forward-dynamics step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call it: only the tests, the
 * package's smoke check and the benchmark's CPU-baseline leg load this library.  It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * What it computes (per environment, per substep of length dt), following the paper's Methods:
 *   1. activation rate  d act/dt = (u - act) / tau(u, act)                          [Eq. 2]
 *      tau = tau_act (0.5 + 1.5 act) if u > act, tau_deact / (0.5 + 1.5 act) if u <= act
 *   2. forward kinematics of the hinge tree (Rodrigues rotations, world frames)
 *   3. muscle-tendon lengths L(q) of via-point polylines and the moment-arm matrix
 *      R = -dL/dq, written out from the point Jacobians                          [EoM, J_m(q)]
 *   4. normalised fibre length / velocity: l_m = 1 + (L - L0)/l_opt, v_m = (dL/dt)/(10 l_opt)
 *   5. Hill force  F = F_max [act f_l(l_m) f_v(v_m) + f_p(l_m)]                    [Eq. 1]
 *   6. joint torques tau_m = R^T F, penalty ground contact (tau_ext), joint-limit penalty
 *   7. bias C(q, qd) by world-frame Newton-Euler, M(q) column by column from the same
 *      Newton-Euler routine (q_dd = e_i, no gravity, qd = 0)                       [EoM]
 *   8. M q_dd + C = R^T F + tau_ext solved by dense Cholesky; velocity-dependent forces
 *      (muscle force-velocity, contact damping and friction, joint damping) and the
 *      joint-limit penalty are taken linearly implicit: (M + dt D) q_dd = rhs
 *   9. semi-implicit Euler: qd += dt q_dd, q += dt qd, act = clamp(act + dt act_dot, 0, 1)
 *
 * Compliant tendon (optional, per muscle; the paper's model keeps the tendon rigid): the fibre
 * and an elastic tendon in series, the tendon strain a state (ora_tendon below).
 *
 * Free root (optional, the paper's skeleton has a floating pelvis): body 0 joined to the world
 * by six DoFs.  DoFs 0-2 translate its origin along world x, y, z (q = position, qd = velocity);
 * DoFs 3-5 turn it about world x, y, z through its origin (qd = world angular velocity, q = the
 * rotation vector of its orientation, advanced by the exponential map: R <- exp(dt w) R).
 *
 * The paper does not print f_l, f_v, f_p (it cites Millard 2013), the tendon model, the contact
 * solver details or the integrator; the readings used here are the named functions below and
 * are listed with their reasons in the design notes of the repository.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nb, n, m, np, ns;
    const int *body_parent, *body_dof_start, *body_ndof;
    const double *body_offset, *body_mass, *body_com, *body_inertia;
    const double *dof_axis, *dof_limit, *dof_damping;
    const int *muscle_point_start;
    const double *fmax, *lopt, *lslack;
    const int *point_body;
    const double *point_pos;
    const int *sphere_body;
    const double *sphere_pos, *sphere_radius;
    double gravity[3];
    double contact_k, contact_c, contact_mu, contact_eps;
    double limit_k, limit_c, tau_act, tau_deact, vmax_per_lopt;
    int implicit_damping;
    /* wrapping surfaces (cylinders or spheres): at most one per muscle, on the segment that ends
     * at the muscle's point number wrap_segment (1 .. points - 1), fixed to body wrap_body */
    int nw;
    const int *wrap_muscle, *wrap_segment, *wrap_body;
    const double *wrap_center, *wrap_axis, *wrap_radius;
    int free_root;   /* 1: body 0 has the six free DoFs 0-5 described above */
    const int* wrap_kind;   /* per wrap: 0 cylinder, 1 sphere (wrap_axis unused); NULL: cylinders */
    /* per muscle: tendon strain at F_max (> 0: compliant tendon, below; 0: rigid); NULL: all rigid */
    const double* tendon_strain;
    double limit_delta;   /* onset width of the joint-limit penalty (ora_joint_limits) */
} ora_model;

int ora_abi_version(void) { return 9; }

/* DoF kinds: a translation of the free root (its point Jacobian is the axis itself), else a
 * rotation about the axis s_d through o_d (point Jacobian s_d x (x - o_d)). */
static int is_slide(const ora_model* M, int d) { return M->free_root && d < 3; }
static int is_free_rot(const ora_model* M, int d) { return M->free_root && d >= 3 && d < 6; }

/* ---------------------------------------------------------------- small 3-vector helpers */
static void cross3(const double a[3], const double b[3], double c[3]) {
    double x = a[1] * b[2] - a[2] * b[1];
    double y = a[2] * b[0] - a[0] * b[2];
    double z = a[0] * b[1] - a[1] * b[0];
    c[0] = x; c[1] = y; c[2] = z;
}
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void matvec3(const double R[9], const double v[3], double out[3]) {
    double x = R[0] * v[0] + R[1] * v[1] + R[2] * v[2];
    double y = R[3] * v[0] + R[4] * v[1] + R[5] * v[2];
    double z = R[6] * v[0] + R[7] * v[1] + R[8] * v[2];
    out[0] = x; out[1] = y; out[2] = z;
}
static void matmul3(const double A[9], const double B[9], double C[9]) {
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
    memcpy(C, T, sizeof(T));
}

/* Rotation by angle th about unit axis a (Rodrigues): R = cos I + sin [a]x + (1 - cos) a a^T. */
static void rodrigues(const double a[3], double th, double R[9]) {
    double c = cos(th), s = sin(th), t = 1.0 - c;
    R[0] = c + t * a[0] * a[0];        R[1] = t * a[0] * a[1] - s * a[2]; R[2] = t * a[0] * a[2] + s * a[1];
    R[3] = t * a[1] * a[0] + s * a[2]; R[4] = c + t * a[1] * a[1];        R[5] = t * a[1] * a[2] - s * a[0];
    R[6] = t * a[2] * a[0] - s * a[1]; R[7] = t * a[2] * a[1] + s * a[0]; R[8] = c + t * a[2] * a[2];
}

/* World inertia about the COM: Rb I Rb^T, I given as xx yy zz xy xz yz in the body frame. */
static void world_inertia(const double Rb[9], const double I6[6], double Iw[9]) {
    double I[9] = {I6[0], I6[3], I6[4], I6[3], I6[1], I6[5], I6[4], I6[5], I6[2]};
    double T[9];
    matmul3(Rb, I, T);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Iw[3 * i + j] = T[3 * i] * Rb[3 * j] + T[3 * i + 1] * Rb[3 * j + 1] + T[3 * i + 2] * Rb[3 * j + 2];
}

/* ---------------------------------------------------------------- forward kinematics
 * Rb[b]: world rotation of body b's frame, pb[b]: world position of its origin (the joint
 * origin).  s[d]: world axis of hinge d, o[d]: world point on that axis (the joint origin). */
void ora_fk(const ora_model* M, const double* q, double* Rb, double* pb, double* s, double* o) {
    for (int b = 0; b < M->nb; ++b) {
        int pa = M->body_parent[b];
        double R[9], p[3];
        const double* off = M->body_offset + 3 * b;
        if (pa < 0) {
            double I[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
            memcpy(R, I, sizeof(R));
            p[0] = off[0]; p[1] = off[1]; p[2] = off[2];
        } else {
            memcpy(R, Rb + 9 * pa, sizeof(R));
            matvec3(R, off, p);
            p[0] += pb[3 * pa]; p[1] += pb[3 * pa + 1]; p[2] += pb[3 * pa + 2];
        }
        if (b == 0 && M->free_root) {
            /* origin at offset + q[0..2]; orientation exp(q[3..5]); world axes x, y, z */
            double th = sqrt(q[3] * q[3] + q[4] * q[4] + q[5] * q[5]);
            if (th > 0.0) {
                double a[3] = {q[3] / th, q[4] / th, q[5] / th};
                rodrigues(a, th, R);
            }
            for (int i = 0; i < 3; ++i) p[i] += q[i];
            for (int d = 0; d < 6; ++d) {
                for (int i = 0; i < 3; ++i) { s[3 * d + i] = (i == d % 3) ? 1.0 : 0.0; o[3 * d + i] = p[i]; }
            }
            memcpy(Rb, R, sizeof(R));
            memcpy(pb, p, sizeof(p));
            continue;
        }
        for (int j = 0; j < M->body_ndof[b]; ++j) {
            int d = M->body_dof_start[b] + j;
            const double* a = M->dof_axis + 3 * d;
            matvec3(R, a, s + 3 * d);
            o[3 * d] = p[0]; o[3 * d + 1] = p[1]; o[3 * d + 2] = p[2];
            double Rj[9];
            rodrigues(a, q[d], Rj);
            matmul3(R, Rj, R);
        }
        memcpy(Rb + 9 * b, R, sizeof(R));
        memcpy(pb + 3 * b, p, sizeof(p));
    }
}

/* g[d] += scale * w . (s_d x (x - o_d)) for every hinge d that moves body `body`
 * (its own hinges and those of all its ancestors): the row w^T J_x of a point Jacobian. */
static void add_wJ(const ora_model* M, const double* s, const double* o, int body, const double x[3],
                   const double w[3], double scale, double* g) {
    for (int b = body; b >= 0; b = M->body_parent[b]) {
        for (int j = 0; j < M->body_ndof[b]; ++j) {
            int d = M->body_dof_start[b] + j;
            double r[3] = {x[0] - o[3 * d], x[1] - o[3 * d + 1], x[2] - o[3 * d + 2]}, c[3];
            if (is_slide(M, d)) memcpy(c, s + 3 * d, sizeof(c));
            else cross3(s + 3 * d, r, c);
            g[d] += scale * dot3(w, c);
        }
    }
}

/* Full 3 x n point Jacobian (row-major, zeroed here). */
static void point_jac(const ora_model* M, const double* s, const double* o, int body, const double x[3],
                      double* J) {
    memset(J, 0, sizeof(double) * 3 * M->n);
    for (int b = body; b >= 0; b = M->body_parent[b]) {
        for (int j = 0; j < M->body_ndof[b]; ++j) {
            int d = M->body_dof_start[b] + j;
            double r[3] = {x[0] - o[3 * d], x[1] - o[3 * d + 1], x[2] - o[3 * d + 2]}, c[3];
            if (is_slide(M, d)) memcpy(c, s + 3 * d, sizeof(c));
            else cross3(s + 3 * d, r, c);
            J[d] = c[0]; J[M->n + d] = c[1]; J[2 * M->n + d] = c[2];
        }
    }
}

/* ---------------------------------------------------------------- muscle geometry
 * L[k] = sum over segments of |x_{j+1} - x_j|; R[k][d] = -dL_k/dq_d (dense m x n, or NULL). */
/* Shortest path from P to S around an infinite cylinder (centre c, unit axis a, radius r;
 * world frame).  In the plane normal to the axis the path is the tangent from P, the arc, and
 * the tangent to S, taken around the side with the shorter arc; along the axis the path is a
 * straight line once the cylinder is unrolled, so the length is sqrt(l_plane^2 + dz^2).  The
 * path wraps when both points lie outside the cylinder and the straight segment passes within
 * r of the axis (in the normal plane); otherwise it is the straight segment (*active = 0).
 * Q and T receive the two tangent points. */
double ora_wrap_cylinder(const double P[3], const double S[3], const double c[3], const double a[3], double r,
                            int* active, double Q[3], double T[3]) {
    double e1[3], e2[3];
    const double ref[3] = {fabs(a[0]) < 0.9 ? 1.0 : 0.0, fabs(a[0]) < 0.9 ? 0.0 : 1.0, 0.0};
    cross3(a, ref, e1);
    double nrm = sqrt(dot3(e1, e1));
    e1[0] /= nrm; e1[1] /= nrm; e1[2] /= nrm;
    cross3(a, e1, e2);
    double p[3] = {P[0] - c[0], P[1] - c[1], P[2] - c[2]}, q[3] = {S[0] - c[0], S[1] - c[1], S[2] - c[2]};
    double px = dot3(p, e1), py = dot3(p, e2), pz = dot3(p, a);
    double sx = dot3(q, e1), sy = dot3(q, e2), sz = dot3(q, a);
    double rp = sqrt(px * px + py * py), rs = sqrt(sx * sx + sy * sy);
    double dv[3] = {S[0] - P[0], S[1] - P[1], S[2] - P[2]};
    double straight = sqrt(dot3(dv, dv));
    *active = 0;
    if (rp <= r || rs <= r) return straight;
    double ex = sx - px, ey = sy - py, ee = ex * ex + ey * ey;
    double t = ee > 0.0 ? -(px * ex + py * ey) / ee : 0.0;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    double cx = px + t * ex, cy = py + t * ey;
    if (cx * cx + cy * cy >= r * r) return straight;
    double thp = atan2(py, px), ths = atan2(sy, sx), alp = acos(r / rp), als = acos(r / rs);
    const double two_pi = 6.283185307179586476925286766559;
    double arc_ccw = fmod(fmod((ths - als) - (thp + alp), two_pi) + two_pi, two_pi);
    double arc_cw = fmod(fmod((thp - alp) - (ths + als), two_pi) + two_pi, two_pi);
    double phq, pht, arc;
    if (arc_ccw <= arc_cw) { phq = thp + alp; pht = ths - als; arc = arc_ccw; }
    else { phq = thp - alp; pht = ths + als; arc = arc_cw; }
    double lp = sqrt(rp * rp - r * r), ls = sqrt(rs * rs - r * r);
    double lplane = lp + r * arc + ls, dz = sz - pz;
    double zq = pz + dz * lp / lplane, zt = pz + dz * (lp + r * arc) / lplane;
    for (int i = 0; i < 3; ++i) {
        Q[i] = c[i] + r * cos(phq) * e1[i] + r * sin(phq) * e2[i] + zq * a[i];
        T[i] = c[i] + r * cos(pht) * e1[i] + r * sin(pht) * e2[i] + zt * a[i];
    }
    *active = 1;
    return sqrt(lplane * lplane + dz * dz);
}

/* Shortest path from P to S over a sphere (centre c, radius r): the great-circle route in the
 * plane through P, S and c, i.e. the cylinder case with the axis normal to that plane (both
 * points then have the same axial coordinate).  When P, c and S are collinear every plane
 * through them is shortest; the one normal to a fixed vector perpendicular to S - P is taken. */
double ora_wrap_sphere(const double P[3], const double S[3], const double c[3], double r, int* active, double Q[3],
                       double T[3]) {
    double p[3] = {P[0] - c[0], P[1] - c[1], P[2] - c[2]}, q[3] = {S[0] - c[0], S[1] - c[1], S[2] - c[2]}, n[3];
    cross3(p, q, n);
    double nn = sqrt(dot3(n, n));
    if (!(nn > 1e-12 * sqrt(dot3(p, p) * dot3(q, q)))) {
        double d[3] = {S[0] - P[0], S[1] - P[1], S[2] - P[2]};
        const double ref[3] = {fabs(d[0]) <= fabs(d[1]) && fabs(d[0]) <= fabs(d[2]) ? 1.0 : 0.0,
                               fabs(d[0]) > fabs(d[1]) && fabs(d[1]) <= fabs(d[2]) ? 1.0 : 0.0,
                               fabs(d[2]) < fabs(d[0]) && fabs(d[2]) < fabs(d[1]) ? 1.0 : 0.0};
        cross3(d, ref, n);
        nn = sqrt(dot3(n, n));
    }
    n[0] /= nn; n[1] /= nn; n[2] /= nn;
    return ora_wrap_cylinder(P, S, c, n, r, active, Q, T);
}

void ora_muscle_geometry(const ora_model* M, const double* Rb, const double* pb, const double* s,
                         const double* o, double* L, double* R) {
    for (int k = 0; k < M->m; ++k) {
        int p0 = M->muscle_point_start[k], p1 = M->muscle_point_start[k + 1];
        double len = 0.0;
        double* row = R ? R + (size_t)k * M->n : NULL;
        if (row) memset(row, 0, sizeof(double) * M->n);
        int w = -1;
        for (int i = 0; i < M->nw; ++i)
            if (M->wrap_muscle[i] == k) w = i;
        double xprev[3];
        int bprev = -1;
        for (int j = p0; j < p1; ++j) {
            int b = M->point_body[j];
            double x[3];
            matvec3(Rb + 9 * b, M->point_pos + 3 * j, x);
            x[0] += pb[3 * b]; x[1] += pb[3 * b + 1]; x[2] += pb[3 * b + 2];
            int wrapped = 0;
            if (j > p0 && w >= 0 && j - p0 == M->wrap_segment[w]) {
                /* the segment from the previous point to this one may wrap the cylinder: lengths
                 * by wrap_cylinder, moment arms from the two straight parts with the tangent
                 * points held fixed on the cylinder's body (they slide along the surface, which
                 * changes the length only to second order) */
                int bw = M->wrap_body[w];
                double cw[3], aw[3], Q[3], T[3];
                matvec3(Rb + 9 * bw, M->wrap_center + 3 * w, cw);
                cw[0] += pb[3 * bw]; cw[1] += pb[3 * bw + 1]; cw[2] += pb[3 * bw + 2];
                double lw;
                if (M->wrap_kind && M->wrap_kind[w] == 1) {
                    lw = ora_wrap_sphere(xprev, x, cw, M->wrap_radius[w], &wrapped, Q, T);
                } else {
                    matvec3(Rb + 9 * bw, M->wrap_axis + 3 * w, aw);
                    double an = sqrt(dot3(aw, aw));
                    aw[0] /= an; aw[1] /= an; aw[2] /= an;
                    lw = ora_wrap_cylinder(xprev, x, cw, aw, M->wrap_radius[w], &wrapped, Q, T);
                }
                if (wrapped) {
                    len += lw;
                    if (row) {
                        double d1[3] = {Q[0] - xprev[0], Q[1] - xprev[1], Q[2] - xprev[2]};
                        double d2[3] = {x[0] - T[0], x[1] - T[1], x[2] - T[2]};
                        double l1 = sqrt(dot3(d1, d1)), l2 = sqrt(dot3(d2, d2));
                        double u1[3] = {d1[0] / l1, d1[1] / l1, d1[2] / l1};
                        double u2[3] = {d2[0] / l2, d2[1] / l2, d2[2] / l2};
                        add_wJ(M, s, o, bw, Q, u1, -1.0, row);
                        add_wJ(M, s, o, bprev, xprev, u1, +1.0, row);
                        add_wJ(M, s, o, b, x, u2, -1.0, row);
                        add_wJ(M, s, o, bw, T, u2, +1.0, row);
                    }
                }
            }
            if (j > p0 && !wrapped) {
                double dv[3] = {x[0] - xprev[0], x[1] - xprev[1], x[2] - xprev[2]};
                double sl = sqrt(dot3(dv, dv));
                len += sl;
                if (row) {
                    double u[3] = {dv[0] / sl, dv[1] / sl, dv[2] / sl};
                    add_wJ(M, s, o, b, x, u, -1.0, row);
                    add_wJ(M, s, o, bprev, xprev, u, +1.0, row);
                }
            }
            memcpy(xprev, x, sizeof(x));
            bprev = b;
        }
        L[k] = len;
    }
}

/* ---------------------------------------------------------------- activation and Hill curves */
double ora_act_rate(double u, double act, double tau_act, double tau_deact) {
    double tau = (u > act) ? tau_act * (0.5 + 1.5 * act) : tau_deact / (0.5 + 1.5 * act);
    return (u - act) / tau;
}

/* active force-length: Gaussian of width 0.45 about the optimal length */
double ora_fl(double l) { return exp(-(l - 1.0) * (l - 1.0) / 0.45); }

/* passive force-length: exponential rise from l = 1 to f_p(1.6) = 1, linear (C1) beyond */
double ora_fp(double l) {
    const double kpe = 4.0, e0 = 0.6;
    if (l <= 1.0) return 0.0;
    if (l <= 1.0 + e0) return (exp(kpe * (l - 1.0) / e0) - 1.0) / (exp(kpe) - 1.0);
    double slope = (kpe / e0) * exp(kpe) / (exp(kpe) - 1.0);
    return 1.0 + slope * (l - 1.0 - e0);
}

/* force-velocity: Hill hyperbola when shortening (v < 0), saturating to 1.4 when lengthening */
double ora_fv(double v) {
    if (v < -1.0) return 0.0;
    if (v <= 0.0) return (1.0 + v) / (1.0 - v / 0.25);
    return 1.0 + 0.4 * v / (v + 0.08);
}
double ora_dfv(double v) {
    if (v < -1.0) return 0.0;
    if (v <= 0.0) { double den = 1.0 - 4.0 * v; return 5.0 / (den * den); }
    return 0.4 * 0.08 / ((v + 0.08) * (v + 0.08));
}

double ora_dfl(double l) { return -2.0 * (l - 1.0) / 0.45 * ora_fl(l); }
double ora_dfp(double l) {
    const double kpe = 4.0, e0 = 0.6;
    if (l <= 1.0) return 0.0;
    if (l <= 1.0 + e0) return (kpe / e0) * exp(kpe * (l - 1.0) / e0) / (exp(kpe) - 1.0);
    return (kpe / e0) * exp(kpe) / (exp(kpe) - 1.0);
}

/* ---------------------------------------------------------------- compliant tendon
 * Reading (not in the paper, whose tendon is rigid): the Hill model's series elastic tendon in
 * the damped-equilibrium form of Millard 2013.
 *   slack length   l_s = L0 - l_opt, so that l_m = 1 at q = 0 with the tendon unstretched and
 *                  the rigid tendon is the stiff limit;
 *   state          the tendon strain eps (0 after a reset: tendon at its slack length);
 *   fibre length   l_m = (L - l_s (1 + eps)) / l_opt;
 *   tendon force   F_max f_t(eps / eps0), eps0 the strain at F_max: f_t(x) = (e^{3x} - 1 - 3x)/(e^3 - 4)
 *                  on [0, 1] (toe region, starting with zero slope at slack), linear with the same
 *                  slope beyond, 0 when slack: C1 everywhere, so the linearly implicit update below
 *                  is continuous in the strain (an inactive muscle with an unstretched fibre rests
 *                  at eps = 0);
 *   fibre          carries the tendon's force with a parallel damper beta = 0.1:
 *                  act f_l(l_m) f_v(v_m) + f_p(l_m) + beta v_m = f_t, which fixes v_m (the left side
 *                  increases strictly with v_m);
 *   strain rate    d eps/dt = (dL/dt - v_max v_m) / l_s, taken linearly implicit in eps (with the
 *                  non-negative part of d v_m / d eps): eps_next = eps + dt rate / (1 + dt v_max J / l_s);
 *   skeleton       receives F = F_max f_t(eps_next / eps0); dF/d(dL/dt) joins the implicit damping. */
#define ORA_TENDON_BETA 0.1
double ora_ft(double x) {
    if (x <= 0.0) return 0.0;
    if (x <= 1.0) return (expm1(3.0 * x) - 3.0 * x) / (exp(3.0) - 4.0);
    return 1.0 + 3.0 * (exp(3.0) - 1.0) / (exp(3.0) - 4.0) * (x - 1.0);
}
double ora_dft(double x) {
    if (x <= 0.0) return 0.0;
    if (x <= 1.0) return 3.0 * expm1(3.0 * x) / (exp(3.0) - 4.0);
    return 3.0 * (exp(3.0) - 1.0) / (exp(3.0) - 4.0);
}

/* root of A f_v(v) + beta v + c0 = 0 (A >= 0, beta > 0) by bisection: the left side is below zero
 * at v = (-c0 - 1.4 A)/beta - 1 and above it at v = -c0/beta + 1 (0 <= f_v <= 1.4) */
double ora_fibre_velocity(double A, double c0, double beta) {
    double lo = (-c0 - 1.4 * A) / beta - 1.0, hi = -c0 / beta + 1.0;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (A * ora_fv(mid) + beta * mid + c0 < 0.0) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* One substep of a compliant muscle at length L, dL/dt = Ldot, activation act and strain eps.
 * out[0] l_m, [1] v_m, [2] eps_next, [3] F / F_max, [4] d(F / F_max)/d(dL/dt), [5] J. */
void ora_tendon(double eps0, double lopt, double ls, double vmax, double act, double L, double Ldot, double eps,
                double dt, double* out) {
    const double beta = ORA_TENDON_BETA;
    double lm = (L - ls * (1.0 + eps)) / lopt;
    double ft = ora_ft(eps / eps0);
    double A = act * ora_fl(lm);
    double vm = ora_fibre_velocity(A, ora_fp(lm) - ft, beta);
    /* d v_m / d eps from the fibre equation: d l_m / d eps = -l_s / l_opt */
    double num = ora_dft(eps / eps0) / eps0 + (act * ora_dfl(lm) * ora_fv(vm) + ora_dfp(lm)) * ls / lopt;
    double J = num / (A * ora_dfv(vm) + beta);
    if (J < 0.0) J = 0.0;
    double g = 1.0 + dt * vmax * J / ls;
    double en = eps + dt * (Ldot - vmax * vm) / ls / g;
    out[0] = lm;
    out[1] = vm;
    out[2] = en;
    out[3] = ora_ft(en / eps0);
    out[4] = ora_dft(en / eps0) / eps0 * dt / (ls * g);
    out[5] = J;
}

/* ---------------------------------------------------------------- Newton-Euler (world frame)
 * tau = M(q) qdd + C(q, qd) [+ gravity term if grav]. */
void ora_rnea(const ora_model* M, const double* q, const double* qd, const double* qdd, int grav,
              double* tau) {
    int nb = M->nb, n = M->n;
    double* Rb = malloc(sizeof(double) * 9 * nb);
    double* pb = malloc(sizeof(double) * 3 * nb);
    double* s = malloc(sizeof(double) * 3 * n);
    double* o = malloc(sizeof(double) * 3 * n);
    double* w = malloc(sizeof(double) * 3 * nb);
    double* dw = malloc(sizeof(double) * 3 * nb);
    double* ao = malloc(sizeof(double) * 3 * nb);
    double* f = malloc(sizeof(double) * 3 * nb);
    double* nm = malloc(sizeof(double) * 3 * nb);
    ora_fk(M, q, Rb, pb, s, o);
    double abase[3] = {0, 0, 0};
    if (grav) { abase[0] = -M->gravity[0]; abase[1] = -M->gravity[1]; abase[2] = -M->gravity[2]; }
    for (int b = 0; b < nb; ++b) {
        int pa = M->body_parent[b];
        double wv[3] = {0, 0, 0}, dwv[3] = {0, 0, 0}, a[3];
        const double* ob = pb + 3 * b;
        if (pa < 0) {
            a[0] = abase[0]; a[1] = abase[1]; a[2] = abase[2];
        } else {
            double r[3] = {ob[0] - pb[3 * pa], ob[1] - pb[3 * pa + 1], ob[2] - pb[3 * pa + 2]}, t1[3], t2[3];
            memcpy(wv, w + 3 * pa, sizeof(wv));
            memcpy(dwv, dw + 3 * pa, sizeof(dwv));
            cross3(dwv, r, t1);
            cross3(wv, r, t2);
            cross3(wv, t2, t2);
            for (int i = 0; i < 3; ++i) a[i] = ao[3 * pa + i] + t1[i] + t2[i];
        }
        for (int j = 0; j < M->body_ndof[b]; ++j) {
            int d = M->body_dof_start[b] + j;
            const double* sd = s + 3 * d;
            if (is_slide(M, d)) {          /* the origin's acceleration is q_dd itself */
                for (int i = 0; i < 3; ++i) a[i] += sd[i] * qdd[d];
                continue;
            }
            double c[3];
            cross3(wv, sd, c);
            if (is_free_rot(M, d)) c[0] = c[1] = c[2] = 0.0;   /* world-fixed axes */
            for (int i = 0; i < 3; ++i) dwv[i] += c[i] * qd[d] + sd[i] * qdd[d];
            for (int i = 0; i < 3; ++i) wv[i] += sd[i] * qd[d];
        }
        memcpy(w + 3 * b, wv, sizeof(wv));
        memcpy(dw + 3 * b, dwv, sizeof(dwv));
        memcpy(ao + 3 * b, a, sizeof(a));
        /* body wrench about its origin */
        double r[3], ac[3], t1[3], t2[3], Iw[9], Iwv[3], Ida[3];
        matvec3(Rb + 9 * b, M->body_com + 3 * b, r);
        cross3(dwv, r, t1);
        cross3(wv, r, t2);
        cross3(wv, t2, t2);
        for (int i = 0; i < 3; ++i) ac[i] = a[i] + t1[i] + t2[i];
        double mb = M->body_mass[b];
        double F[3] = {mb * ac[0], mb * ac[1], mb * ac[2]};
        world_inertia(Rb + 9 * b, M->body_inertia + 6 * b, Iw);
        matvec3(Iw, dwv, Ida);
        matvec3(Iw, wv, Iwv);
        cross3(wv, Iwv, t1);
        double rF[3];
        cross3(r, F, rF);
        for (int i = 0; i < 3; ++i) {
            f[3 * b + i] = F[i];
            nm[3 * b + i] = Ida[i] + t1[i] + rF[i];
        }
    }
    for (int b = nb - 1; b >= 0; --b) {
        for (int j = 0; j < M->body_ndof[b]; ++j) {
            int d = M->body_dof_start[b] + j;
            tau[d] = dot3(s + 3 * d, is_slide(M, d) ? f + 3 * b : nm + 3 * b);   /* force or moment */
        }
        int pa = M->body_parent[b];
        if (pa >= 0) {
            double r[3] = {pb[3 * b] - pb[3 * pa], pb[3 * b + 1] - pb[3 * pa + 1], pb[3 * b + 2] - pb[3 * pa + 2]}, c[3];
            cross3(r, f + 3 * b, c);
            for (int i = 0; i < 3; ++i) {
                f[3 * pa + i] += f[3 * b + i];
                nm[3 * pa + i] += nm[3 * b + i] + c[i];
            }
        }
    }
    free(Rb); free(pb); free(s); free(o); free(w); free(dw); free(ao); free(f); free(nm);
}

/* M(q) column by column: M e_i = RNEA(q, 0, e_i) without gravity. Row-major n x n. */
void ora_mass_matrix(const ora_model* M, const double* q, double* Mout) {
    int n = M->n;
    double* z = calloc(n, sizeof(double));
    double* e = calloc(n, sizeof(double));
    double* col = malloc(sizeof(double) * n);
    for (int i = 0; i < n; ++i) {
        e[i] = 1.0;
        ora_rnea(M, q, z, e, 0, col);
        e[i] = 0.0;
        for (int r = 0; r < n; ++r) Mout[(size_t)r * n + i] = col[r];
    }
    free(z); free(e); free(col);
}

/* Independent second formulation: M = sum_b m_b Jc^T Jc + Jw^T Iw Jw (body Jacobians). */
void ora_mass_matrix_jac(const ora_model* M, const double* q, double* Mout) {
    int nb = M->nb, n = M->n;
    double* Rb = malloc(sizeof(double) * 9 * nb);
    double* pb = malloc(sizeof(double) * 3 * nb);
    double* s = malloc(sizeof(double) * 3 * n);
    double* o = malloc(sizeof(double) * 3 * n);
    double* J = malloc(sizeof(double) * 3 * n);
    double* Jw = malloc(sizeof(double) * 3 * n);
    ora_fk(M, q, Rb, pb, s, o);
    memset(Mout, 0, sizeof(double) * n * n);
    for (int b = 0; b < nb; ++b) {
        double c[3], Iw[9];
        matvec3(Rb + 9 * b, M->body_com + 3 * b, c);
        for (int i = 0; i < 3; ++i) c[i] += pb[3 * b + i];
        point_jac(M, s, o, b, c, J);
        memset(Jw, 0, sizeof(double) * 3 * n);
        for (int a = b; a >= 0; a = M->body_parent[a])
            for (int j = 0; j < M->body_ndof[a]; ++j) {
                int d = M->body_dof_start[a] + j;
                if (is_slide(M, d)) continue;   /* translations do not turn the body */
                Jw[d] = s[3 * d]; Jw[n + d] = s[3 * d + 1]; Jw[2 * n + d] = s[3 * d + 2];
            }
        world_inertia(Rb + 9 * b, M->body_inertia + 6 * b, Iw);
        double mb = M->body_mass[b];
        for (int r = 0; r < n; ++r)
            for (int cc = 0; cc < n; ++cc) {
                double v = mb * (J[r] * J[cc] + J[n + r] * J[n + cc] + J[2 * n + r] * J[2 * n + cc]);
                for (int i = 0; i < 3; ++i)
                    for (int k = 0; k < 3; ++k) v += Jw[i * n + r] * Iw[3 * i + k] * Jw[k * n + cc];
                Mout[(size_t)r * n + cc] += v;
            }
    }
    free(Rb); free(pb); free(s); free(o); free(J); free(Jw);
}

/* ---------------------------------------------------------------- contact
 * Penalty ground contact at the lowest point y of each sphere (plane z = 0):
 *   depth = r - z_center; f_n = max(0, k depth - c v_n); f_t = -mu f_n v_t / sqrt(|v_t|^2 + eps^2);
 *   tau_c += J_y^T F.  With implicit damping, Dc += J_y^T diag(mu f_n / s, mu f_n / s, c) J_y
 *   (normal: d f_n / d v_n = -c; friction: its coefficient mu f_n / s held, velocity implicit).
 * fs (optional, S x 3) receives the world contact force of each sphere. */
void ora_contact(const ora_model* M, const double* Rb, const double* pb, const double* s, const double* o,
                 const double* qd, double* tau_c, double* Dc, double* fs) {
    int n = M->n;
    double* J = malloc(sizeof(double) * 3 * n);
    for (int i = 0; i < M->ns; ++i) {
        int b = M->sphere_body[i];
        double x[3];
        matvec3(Rb + 9 * b, M->sphere_pos + 3 * i, x);
        for (int c = 0; c < 3; ++c) x[c] += pb[3 * b + c];
        double r = M->sphere_radius[i];
        double y[3] = {x[0], x[1], x[2] - r};
        double depth = r - x[2];
        if (fs) fs[3 * i] = fs[3 * i + 1] = fs[3 * i + 2] = 0.0;
        if (depth <= 0.0) continue;
        point_jac(M, s, o, b, y, J);
        double v[3] = {0, 0, 0};
        for (int c = 0; c < 3; ++c)
            for (int d = 0; d < n; ++d) v[c] += J[c * n + d] * qd[d];
        double fn = M->contact_k * depth - M->contact_c * v[2];
        if (fn <= 0.0) continue;
        double sm = sqrt(v[0] * v[0] + v[1] * v[1] + M->contact_eps * M->contact_eps);
        double F[3] = {-M->contact_mu * fn * v[0] / sm, -M->contact_mu * fn * v[1] / sm, fn};
        if (fs) { fs[3 * i] = F[0]; fs[3 * i + 1] = F[1]; fs[3 * i + 2] = F[2]; }
        for (int d = 0; d < n; ++d) tau_c[d] += J[d] * F[0] + J[n + d] * F[1] + J[2 * n + d] * F[2];
        if (Dc) {
            double dd[3] = {M->contact_mu * fn / sm, M->contact_mu * fn / sm, M->contact_c};
            for (int a = 0; a < n; ++a)
                for (int bb = 0; bb < n; ++bb)
                    Dc[(size_t)a * n + bb] += J[a] * dd[0] * J[bb] + J[n + a] * dd[1] * J[n + bb] +
                                              J[2 * n + a] * dd[2] * J[2 * n + bb];
        }
    }
    free(J);
}

/* ---------------------------------------------------------------- joint limits and damping
 * Outside [lo, hi] (enabled when lo < hi) a penalty spring-damper acts on the excess x past the
 * limit.  Spring torque k_l phi(x), damper c_l psi(x) qd, with a smooth onset of width delta:
 *   phi(x) = x^2 / (2 delta), psi(x) = x / delta     for 0 < x < delta,
 *   phi(x) = x - delta / 2,   psi(x) = 1             for x >= delta,
 * so phi' = psi, and torque, phi' and psi are continuous in x (delta = 0: the plain penalty k_l x,
 * c_l).  Linearly implicit in position and velocity: the spring is taken at the end-of-step excess
 * x' = x + dt qd' (above hi; x - dt qd' below lo) to first order, phi(x') = phi(x) + psi(x) dt qd',
 * and the damper at the new velocity qd' = qd + dt qdd, so above hi
 *   tau = -k_l phi(x) - (k_l dt + c_l) psi(x) qd'
 * (below lo the spring term changes sign).  The explicit part goes to tau_l, the coefficient of
 * qd' to Dj (the system matrix receives dt * Dj).  Joint damping: tau -= b qd, Dj += b. */
void ora_joint_limits(const ora_model* M, double dt, const double* q, const double* qd, double* tau_l, double* Dj) {
    for (int d = 0; d < M->n; ++d) {
        double lo = M->dof_limit[2 * d], hi = M->dof_limit[2 * d + 1];
        double t = -M->dof_damping[d] * qd[d], dd = M->dof_damping[d];
        double kk = M->limit_k, cc = M->limit_c, del = M->limit_delta;
        if (lo < hi && (q[d] > hi || q[d] < lo)) {
            double x = q[d] > hi ? q[d] - hi : lo - q[d];
            double phi, psi;
            if (del > 0.0 && x < del) { phi = 0.5 * x * x / del; psi = x / del; }
            else { phi = x - 0.5 * del; psi = 1.0; }
            double spring = kk * phi, kd = (kk * dt + cc) * psi;
            t += (q[d] > hi ? -spring : spring) - kd * qd[d];
            dd += kd;
        }
        tau_l[d] = t;
        if (Dj) Dj[d] = dd;
    }
}

/* ---------------------------------------------------------------- dense Cholesky solve
 * A (n x n, row-major, SPD) = L L^T; solves A x = b.  Returns 0, or 1 if a pivot is not positive. */
int ora_cholesky_solve(int n, const double* A, const double* b, double* x) {
    double* Lm = malloc(sizeof(double) * n * n);
    memcpy(Lm, A, sizeof(double) * n * n);
    int bad = 0;
    for (int j = 0; j < n && !bad; ++j) {
        double sdiag = Lm[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) sdiag -= Lm[(size_t)j * n + k] * Lm[(size_t)j * n + k];
        if (!(sdiag > 0.0)) { bad = 1; break; }
        double ljj = sqrt(sdiag);
        Lm[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double v = Lm[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) v -= Lm[(size_t)i * n + k] * Lm[(size_t)j * n + k];
            Lm[(size_t)i * n + j] = v / ljj;
        }
    }
    if (!bad) {
        for (int i = 0; i < n; ++i) {           /* L y = b */
            double v = b[i];
            for (int k = 0; k < i; ++k) v -= Lm[(size_t)i * n + k] * x[k];
            x[i] = v / Lm[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {      /* L^T x = y */
            double v = x[i];
            for (int k = i + 1; k < n; ++k) v -= Lm[(size_t)k * n + i] * x[k];
            x[i] = v / Lm[(size_t)i * n + i];
        }
    }
    free(Lm);
    return bad;
}

/* Muscle-tendon lengths at q = 0: the reference lengths L0 used to normalise fibre length. */
void ora_rest_lengths(const ora_model* M, double* L0) {
    int nb = M->nb, n = M->n;
    double* q = calloc(n, sizeof(double));
    double* Rb = malloc(sizeof(double) * 9 * nb);
    double* pb = malloc(sizeof(double) * 3 * nb);
    double* s = malloc(sizeof(double) * 3 * n);
    double* o = malloc(sizeof(double) * 3 * n);
    ora_fk(M, q, Rb, pb, s, o);
    ora_muscle_geometry(M, Rb, pb, s, o, L0, NULL);
    free(q); free(Rb); free(pb); free(s); free(o);
}

/* Every intermediate of one substep at state (q, qd, act) with excitation exc.
 * Any output pointer may be NULL.  Returns 0, or 1 if the system matrix was not SPD. */
typedef struct {
    double *qdd, *force, *L, *R, *lm, *vm, *dFdv, *tau_m, *tau_c, *tau_l, *bias, *M, *A, *rhs, *act_next,
        *sphere_force, *eps_next;
} ora_eval_out;

/* eps: tendon strains [m] (NULL: zero); only compliant muscles read theirs.
 * L_in [m], R_in [m][n] (either may be NULL): muscle-tendon lengths and moment arms to use in
 * place of the via-point geometry at q, for a substep driven by an approximation of J_m(q) (a
 * learned geometry); everything downstream of the geometry (fibre state, Eq. 1, R^T F, the
 * implicit damping R^T diag(dF/dLdot) R over the non-zero entries of each row, contact, limits,
 * Newton-Euler, Cholesky) is the same as for the exact geometry. */
int ora_eval_geom(const ora_model* M, const double* L0, double dt, const double* q, const double* qd,
                  const double* act, const double* exc, const double* eps, const double* L_in,
                  const double* R_in, const ora_eval_out* out);

int ora_eval(const ora_model* M, const double* L0, double dt, const double* q, const double* qd,
             const double* act, const double* exc, const double* eps, const ora_eval_out* out) {
    return ora_eval_geom(M, L0, dt, q, qd, act, exc, eps, NULL, NULL, out);
}

int ora_eval_geom(const ora_model* M, const double* L0, double dt, const double* q, const double* qd,
                  const double* act, const double* exc, const double* eps, const double* L_in,
                  const double* R_in, const ora_eval_out* out) {
    int nb = M->nb, n = M->n, m = M->m;
    double* Rb = malloc(sizeof(double) * 9 * nb);
    double* pb = malloc(sizeof(double) * 3 * nb);
    double* s = malloc(sizeof(double) * 3 * n);
    double* o = malloc(sizeof(double) * 3 * n);
    double* L = malloc(sizeof(double) * m);
    double* R = malloc(sizeof(double) * (size_t)m * n);
    double* F = malloc(sizeof(double) * m);
    double* dF = malloc(sizeof(double) * m);
    double* lm = malloc(sizeof(double) * m);
    double* vm = malloc(sizeof(double) * m);
    double* en = malloc(sizeof(double) * m);
    double* tau_m = calloc(n, sizeof(double));
    double* tau_c = calloc(n, sizeof(double));
    double* tau_l = calloc(n, sizeof(double));
    double* Dj = calloc(n, sizeof(double));
    double* C = malloc(sizeof(double) * n);
    double* Mm = malloc(sizeof(double) * n * n);
    double* A = malloc(sizeof(double) * n * n);
    double* D = calloc((size_t)n * n, sizeof(double));
    double* rhs = malloc(sizeof(double) * n);
    double* qdd = malloc(sizeof(double) * n);
    double* zero = calloc(n, sizeof(double));
    int* nz = malloc(sizeof(int) * n);

    ora_fk(M, q, Rb, pb, s, o);
    ora_muscle_geometry(M, Rb, pb, s, o, L, R);
    if (L_in) memcpy(L, L_in, sizeof(double) * m);
    if (R_in) memcpy(R, R_in, sizeof(double) * (size_t)m * n);
    for (int k = 0; k < m; ++k) {
        const double* row = R + (size_t)k * n;
        double ldot = 0.0;
        for (int d = 0; d < n; ++d) ldot -= row[d] * qd[d];       /* dL/dt = (dL/dq) qd = -R qd */
        double vmax = M->vmax_per_lopt * M->lopt[k];
        double a = act[k];
        en[k] = eps ? eps[k] : 0.0;
        if (M->tendon_strain && M->tendon_strain[k] > 0.0) {
            double t[6];
            ora_tendon(M->tendon_strain[k], M->lopt[k], L0[k] - M->lopt[k], vmax, a, L[k], ldot, en[k], dt, t);
            lm[k] = t[0];
            vm[k] = t[1];
            en[k] = t[2];
            F[k] = M->fmax[k] * t[3];
            dF[k] = M->fmax[k] * t[4];
        } else {
            lm[k] = 1.0 + (L[k] - L0[k]) / M->lopt[k];
            vm[k] = ldot / vmax;
            F[k] = M->fmax[k] * (a * ora_fl(lm[k]) * ora_fv(vm[k]) + ora_fp(lm[k]));
            dF[k] = M->fmax[k] * a * ora_fl(lm[k]) * ora_dfv(vm[k]) / vmax;
        }
        for (int d = 0; d < n; ++d) tau_m[d] += row[d] * F[k];
        if (M->implicit_damping) {
            /* d tau_m / d qd = -R^T diag(dF/dLdot) R; only the non-zeros of the row matter */
            int c = 0;
            for (int d = 0; d < n; ++d) if (row[d] != 0.0) nz[c++] = d;
            for (int i = 0; i < c; ++i)
                for (int j = 0; j < c; ++j) D[(size_t)nz[i] * n + nz[j]] += dF[k] * row[nz[i]] * row[nz[j]];
        }
    }
    ora_contact(M, Rb, pb, s, o, qd, tau_c, M->implicit_damping ? D : NULL, out ? out->sphere_force : NULL);
    ora_joint_limits(M, dt, q, qd, tau_l, Dj);
    ora_rnea(M, q, qd, zero, 1, C);
    ora_mass_matrix(M, q, Mm);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = Mm[(size_t)i * n + j];
        if (M->implicit_damping) {
            for (int j = 0; j < n; ++j) A[(size_t)i * n + j] += dt * D[(size_t)i * n + j];
            A[(size_t)i * n + i] += dt * Dj[i];
        }
        rhs[i] = tau_m[i] + tau_c[i] + tau_l[i] - C[i];
    }
    int bad = ora_cholesky_solve(n, A, rhs, qdd);
    if (bad) for (int i = 0; i < n; ++i) qdd[i] = NAN;

    if (out) {
        if (out->qdd) memcpy(out->qdd, qdd, sizeof(double) * n);
        if (out->force) memcpy(out->force, F, sizeof(double) * m);
        if (out->L) memcpy(out->L, L, sizeof(double) * m);
        if (out->R) memcpy(out->R, R, sizeof(double) * (size_t)m * n);
        if (out->lm) memcpy(out->lm, lm, sizeof(double) * m);
        if (out->vm) memcpy(out->vm, vm, sizeof(double) * m);
        if (out->eps_next) memcpy(out->eps_next, en, sizeof(double) * m);
        if (out->dFdv) memcpy(out->dFdv, dF, sizeof(double) * m);
        if (out->tau_m) memcpy(out->tau_m, tau_m, sizeof(double) * n);
        if (out->tau_c) memcpy(out->tau_c, tau_c, sizeof(double) * n);
        if (out->tau_l) memcpy(out->tau_l, tau_l, sizeof(double) * n);
        if (out->bias) memcpy(out->bias, C, sizeof(double) * n);
        if (out->M) memcpy(out->M, Mm, sizeof(double) * n * n);
        if (out->A) memcpy(out->A, A, sizeof(double) * n * n);
        if (out->rhs) memcpy(out->rhs, rhs, sizeof(double) * n);
        if (out->act_next)
            for (int k = 0; k < m; ++k) {
                double u = exc[k] < 0.0 ? 0.0 : (exc[k] > 1.0 ? 1.0 : exc[k]);   /* action space [0,1] */
                double a = act[k] + dt * ora_act_rate(u, act[k], M->tau_act, M->tau_deact);
                out->act_next[k] = a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
            }
    }
    free(Rb); free(pb); free(s); free(o); free(L); free(R); free(F); free(dF); free(lm); free(vm); free(en);
    free(tau_m); free(tau_c); free(tau_l); free(Dj); free(C); free(Mm); free(A); free(D); free(rhs);
    free(qdd); free(zero); free(nz);
    return bad;
}

/* Position update of semi-implicit Euler from the new velocities: q += dt qd, except the free
 * root's rotation vector, which follows R <- exp(dt w) R (unit quaternions: the product of the
 * step's rotation and the current one, returned as the rotation vector of angle in [0, pi]). */
void ora_integrate_q(const ora_model* M, double dt, double* q, const double* qd) {
    for (int d = 0; d < M->n; ++d)
        if (!is_free_rot(M, d)) q[d] += dt * qd[d];
    if (!M->free_root) return;
    double qa[4], qb[4], qc[4];
    double th = sqrt(q[3] * q[3] + q[4] * q[4] + q[5] * q[5]);
    qa[0] = cos(0.5 * th);
    for (int i = 0; i < 3; ++i) qa[1 + i] = th > 0.0 ? sin(0.5 * th) * q[3 + i] / th : 0.0;
    double w[3] = {dt * qd[3], dt * qd[4], dt * qd[5]};
    double ph = sqrt(dot3(w, w));
    qb[0] = cos(0.5 * ph);
    for (int i = 0; i < 3; ++i) qb[1 + i] = ph > 0.0 ? sin(0.5 * ph) * w[i] / ph : 0.0;
    /* qc = qb * qa (Hamilton product) */
    qc[0] = qb[0] * qa[0] - qb[1] * qa[1] - qb[2] * qa[2] - qb[3] * qa[3];
    qc[1] = qb[0] * qa[1] + qb[1] * qa[0] + qb[2] * qa[3] - qb[3] * qa[2];
    qc[2] = qb[0] * qa[2] - qb[1] * qa[3] + qb[2] * qa[0] + qb[3] * qa[1];
    qc[3] = qb[0] * qa[3] + qb[1] * qa[2] - qb[2] * qa[1] + qb[3] * qa[0];
    if (qc[0] < 0.0) for (int i = 0; i < 4; ++i) qc[i] = -qc[i];
    double vn = sqrt(qc[1] * qc[1] + qc[2] * qc[2] + qc[3] * qc[3]);
    double ang = 2.0 * atan2(vn, qc[0]);
    for (int i = 0; i < 3; ++i) q[3 + i] = vn > 0.0 ? ang * qc[1 + i] / vn : 0.0;
}

/* n_sub substeps for each of n_envs environments, states updated in place (rows [E][n], [E][m]);
 * exc [E][m] is held over the substeps.  eps (optional, [E][m]): tendon strains, updated in place
 * (NULL: zero at every substep, for models without compliant tendons).  qdd_out / force_out
 * (optional) receive the last substep's accelerations and muscle forces.  status (optional, [E])
 * gets 1 where a solve failed.  Environments run in parallel on n_threads host threads (<= 0:
 * the OpenMP default). */
void ora_step(const ora_model* M, const double* L0, double dt, int n_envs, int n_sub, double* q, double* qd,
              double* act, const double* exc, double* eps, double* qdd_out, double* force_out, int* status,
              int n_threads) {
    int n = M->n, m = M->m;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int e = 0; e < n_envs; ++e) {
        double* qe = q + (size_t)e * n;
        double* qde = qd + (size_t)e * n;
        double* ae = act + (size_t)e * m;
        const double* ue = exc + (size_t)e * m;
        double* qdd = malloc(sizeof(double) * n);
        double* F = malloc(sizeof(double) * m);
        double* anext = malloc(sizeof(double) * m);
        double* ee = eps ? eps + (size_t)e * m : NULL;
        double* enext = malloc(sizeof(double) * (m > 0 ? m : 1));
        int bad = 0;
        for (int t = 0; t < n_sub; ++t) {
            ora_eval_out out;
            memset(&out, 0, sizeof(out));
            out.qdd = qdd; out.force = F; out.act_next = anext; out.eps_next = enext;
            bad |= ora_eval(M, L0, dt, qe, qde, ae, ue, ee, &out);
            for (int d = 0; d < n; ++d) qde[d] += dt * qdd[d];
            ora_integrate_q(M, dt, qe, qde);
            memcpy(ae, anext, sizeof(double) * m);
            if (ee) memcpy(ee, enext, sizeof(double) * m);
        }
        free(enext);
        if (qdd_out) memcpy(qdd_out + (size_t)e * n, qdd, sizeof(double) * n);
        if (force_out) memcpy(force_out + (size_t)e * m, F, sizeof(double) * m);
        if (status) status[e] = bad;
        free(qdd); free(F); free(anext);
    }
}

int ora_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
