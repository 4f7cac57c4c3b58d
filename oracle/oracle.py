"""Python wrapper of the FP64 CPU oracle (``msim_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's CPU-baseline
leg may use it; the product path never does.  It shares no code with the CUDA path: it reads the
synthetic :class:`Model` arrays produced by the input generator and marshals them into its own
C struct.

Every function here follows the paper's Methods section (Eq. 1 Hill force, Eq. 2 activation
dynamics, the generalised-coordinate equations of motion M q_dd + C = J_m^T F + tau_ext, and the
penalty reading of the ground contact).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msim_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class _OraModel(C.Structure):
    _fields_ = [("nb", C.c_int), ("n", C.c_int), ("m", C.c_int), ("np", C.c_int), ("ns", C.c_int),
                ("body_parent", _ip), ("body_dof_start", _ip), ("body_ndof", _ip),
                ("body_offset", _dp), ("body_mass", _dp), ("body_com", _dp), ("body_inertia", _dp),
                ("dof_axis", _dp), ("dof_limit", _dp), ("dof_damping", _dp),
                ("muscle_point_start", _ip), ("fmax", _dp), ("lopt", _dp), ("lslack", _dp),
                ("point_body", _ip), ("point_pos", _dp),
                ("sphere_body", _ip), ("sphere_pos", _dp), ("sphere_radius", _dp),
                ("gravity", C.c_double * 3),
                ("contact_k", C.c_double), ("contact_c", C.c_double), ("contact_mu", C.c_double),
                ("contact_eps", C.c_double), ("limit_k", C.c_double), ("limit_c", C.c_double),
                ("tau_act", C.c_double), ("tau_deact", C.c_double), ("vmax_per_lopt", C.c_double),
                ("implicit_damping", C.c_int),
                ("nw", C.c_int), ("wrap_muscle", _ip), ("wrap_segment", _ip), ("wrap_body", _ip),
                ("wrap_center", _dp), ("wrap_axis", _dp), ("wrap_radius", _dp),
                ("free_root", C.c_int), ("wrap_kind", _ip), ("tendon_strain", _dp), ("limit_delta", C.c_double)]


class _EvalOut(C.Structure):
    _fields_ = [(k, _dp) for k in ("qdd", "force", "L", "R", "lm", "vm", "dFdv", "tau_m", "tau_c", "tau_l",
                                   "bias", "M", "A", "rhs", "act_next", "sphere_force", "eps_next")]


def build(force=False):
    """Compile the oracle with gcc (plain C99 + OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu99", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_LIB)
        _lib.ora_abi_version.restype = C.c_int
        if _lib.ora_abi_version() != 9:
            raise RuntimeError("stale oracle library: rebuild with oracle.build(force=True)")
        for name in ("ora_fl", "ora_fp", "ora_fv", "ora_dfv", "ora_dfl", "ora_dfp", "ora_ft", "ora_dft"):
            getattr(_lib, name).restype = C.c_double
            getattr(_lib, name).argtypes = [C.c_double]
        _lib.ora_act_rate.restype = C.c_double
        _lib.ora_act_rate.argtypes = [C.c_double] * 4
        _lib.ora_eval.restype = C.c_int
        _lib.ora_eval_geom.restype = C.c_int
        _lib.ora_cholesky_solve.restype = C.c_int
        _lib.ora_max_threads.restype = C.c_int
        _lib.ora_wrap_cylinder.restype = C.c_double
        _lib.ora_wrap_sphere.restype = C.c_double
        _lib.ora_fibre_velocity.restype = C.c_double
        _lib.ora_fibre_velocity.argtypes = [C.c_double] * 3
        _lib.ora_tendon.argtypes = [C.c_double] * 9 + [_dp]
    return _lib


def tendon_strains(model):
    """Per-muscle tendon strain at F_max (0: rigid tendon); None when every tendon is rigid."""
    t = getattr(model, "muscle_tendon_strain", None)
    if t is None:
        return None
    t = np.asarray(t, dtype=np.float64).reshape(-1)
    return t if t.shape[0] == model.n_muscles and np.any(t > 0) else None


def _wrap_kinds(model, nw):
    """Per-wrap surface kind (0 cylinder, 1 sphere); a model without the field has cylinders."""
    k = np.asarray(getattr(model, "wrap_kind", np.zeros(0)), dtype=np.int32).reshape(-1)
    return k if (nw and k.shape[0] == nw) else np.zeros(max(nw, 1), np.int32)


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


class OracleModel:
    """A :class:`Model` marshalled into the oracle's own C struct (keeps its arrays alive)."""

    def __init__(self, model, implicit_damping=True):
        self.model = model
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        i = lambda a: np.ascontiguousarray(a, dtype=np.int32)
        self._keep = dict(
            body_parent=i(model.body_parent), body_dof_start=i(model.body_dof_start), body_ndof=i(model.body_ndof),
            body_offset=f(model.body_offset), body_mass=f(model.body_mass), body_com=f(model.body_com),
            body_inertia=f(model.body_inertia), dof_axis=f(model.dof_axis), dof_limit=f(model.dof_limit),
            dof_damping=f(model.dof_damping), muscle_point_start=i(model.muscle_point_start),
            fmax=f(model.muscle_fmax), lopt=f(model.muscle_lopt), lslack=f(model.muscle_lslack),
            point_body=i(model.point_body), point_pos=f(model.point_pos),
            sphere_body=i(model.sphere_body if model.n_spheres else np.zeros(1)),
            sphere_pos=f(model.sphere_pos if model.n_spheres else np.zeros((1, 3))),
            sphere_radius=f(model.sphere_radius if model.n_spheres else np.zeros(1)))
        nw = int(np.asarray(model.wrap_muscle).shape[0])
        self._keep.update(
            wrap_muscle=i(model.wrap_muscle if nw else np.zeros(1)),
            wrap_segment=i(model.wrap_segment if nw else np.zeros(1)),
            wrap_body=i(model.wrap_body if nw else np.zeros(1)),
            wrap_center=f(model.wrap_center if nw else np.zeros((1, 3))),
            wrap_axis=f(model.wrap_axis if nw else np.zeros((1, 3))),
            wrap_radius=f(model.wrap_radius if nw else np.zeros(1)),
            wrap_kind=i(_wrap_kinds(model, nw)))
        s = _OraModel()
        s.nb, s.n, s.m, s.np, s.ns = model.n_bodies, model.n_dofs, model.n_muscles, model.n_points, model.n_spheres
        for k, v in self._keep.items():
            setattr(s, k, _ptr(v, _ip if v.dtype == np.int32 else _dp))
        s.gravity = (C.c_double * 3)(*[float(x) for x in model.gravity])
        for k, v in model.scalars().items():
            setattr(s, k, float(v))
        s.implicit_damping = 1 if implicit_damping else 0
        s.nw = nw
        s.free_root = 1 if getattr(model, "free_root", False) else 0
        ts = tendon_strains(model)
        if ts is not None:
            self._keep["tendon_strain"] = np.ascontiguousarray(ts)
            s.tendon_strain = _ptr(self._keep["tendon_strain"])
        self.compliant = ts is not None
        self.s = s
        self.n, self.m, self.nb = model.n_dofs, model.n_muscles, model.n_bodies
        self.L0 = np.zeros(self.m)
        lib().ora_rest_lengths(C.byref(self.s), _ptr(self.L0))

    @property
    def ref(self):
        return C.byref(self.s)


def _as(model, implicit_damping=True):
    return model if isinstance(model, OracleModel) else OracleModel(model, implicit_damping)


# ------------------------------------------------------------------------------ scalar curves
def fl(l):
    return lib().ora_fl(float(l))


def fp(l):
    return lib().ora_fp(float(l))


def fv(v):
    return lib().ora_fv(float(v))


def dfv(v):
    return lib().ora_dfv(float(v))


def dfl(l):
    return lib().ora_dfl(float(l))


def dfp(l):
    return lib().ora_dfp(float(l))


def ft(x):
    """Normalised tendon force at x = strain / strain at F_max."""
    return lib().ora_ft(float(x))


def dft(x):
    return lib().ora_dft(float(x))


TENDON_BETA = 0.1


def fibre_velocity(A, c0, beta=TENDON_BETA):
    """Root v of A f_v(v) + beta v + c0 = 0 (bisection)."""
    return lib().ora_fibre_velocity(float(A), float(c0), float(beta))


def tendon(eps0, lopt, ls, vmax, act, L, Ldot, eps, dt):
    """One substep of a compliant muscle: dict l_m, v_m, eps_next, F (normalised by F_max),
    dF (its derivative by dL/dt), J (the implicit part of d v_m / d eps)."""
    out = np.zeros(6)
    lib().ora_tendon(*(float(x) for x in (eps0, lopt, ls, vmax, act, L, Ldot, eps, dt)), _ptr(out))
    return dict(zip(("lm", "vm", "eps_next", "F", "dF", "J"), out))


def act_rate(u, a, tau_act=0.010, tau_deact=0.040):
    return lib().ora_act_rate(float(u), float(a), float(tau_act), float(tau_deact))


# ------------------------------------------------------------------------------ kinematics / dynamics
def fk(model, q):
    om = _as(model)
    q = np.ascontiguousarray(q, dtype=np.float64)
    Rb = np.zeros((om.nb, 3, 3)); pb = np.zeros((om.nb, 3)); s = np.zeros((om.n, 3)); o = np.zeros((om.n, 3))
    lib().ora_fk(om.ref, _ptr(q), _ptr(Rb), _ptr(pb), _ptr(s), _ptr(o))
    return Rb, pb, s, o


def wrap_cylinder(P, S, c, a, r):
    """Shortest path P -> S around an infinite cylinder (centre c, unit axis a, radius r):
    (length, wraps, tangent point Q, tangent point T)."""
    P, S, c, a = (np.ascontiguousarray(v, dtype=np.float64) for v in (P, S, c, a))
    Q, T = np.zeros(3), np.zeros(3)
    act = C.c_int(0)
    L = lib().ora_wrap_cylinder(_ptr(P), _ptr(S), _ptr(c), _ptr(a), C.c_double(r), C.byref(act), _ptr(Q), _ptr(T))
    return L, bool(act.value), Q, T


def wrap_sphere(P, S, c, r):
    """Shortest path P -> S over a sphere (centre c, radius r): (length, wraps, Q, T)."""
    P, S, c = (np.ascontiguousarray(v, dtype=np.float64) for v in (P, S, c))
    Q, T = np.zeros(3), np.zeros(3)
    act = C.c_int(0)
    L = lib().ora_wrap_sphere(_ptr(P), _ptr(S), _ptr(c), C.c_double(r), C.byref(act), _ptr(Q), _ptr(T))
    return L, bool(act.value), Q, T


def muscle_geometry(model, q):
    """(L [m], R [m, n] = -dL/dq) at q."""
    om = _as(model)
    Rb, pb, s, o = fk(om, q)
    L = np.zeros(om.m); R = np.zeros((om.m, om.n))
    lib().ora_muscle_geometry(om.ref, _ptr(Rb), _ptr(pb), _ptr(s), _ptr(o), _ptr(L), _ptr(R))
    return L, R


def rnea(model, q, qd, qdd, gravity=True):
    om = _as(model)
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (q, qd, qdd)]
    tau = np.zeros(om.n)
    lib().ora_rnea(om.ref, _ptr(a[0]), _ptr(a[1]), _ptr(a[2]), C.c_int(1 if gravity else 0), _ptr(tau))
    return tau


def mass_matrix(model, q):
    om = _as(model)
    q = np.ascontiguousarray(q, dtype=np.float64)
    Mm = np.zeros((om.n, om.n))
    lib().ora_mass_matrix(om.ref, _ptr(q), _ptr(Mm))
    return Mm


def mass_matrix_jac(model, q):
    om = _as(model)
    q = np.ascontiguousarray(q, dtype=np.float64)
    Mm = np.zeros((om.n, om.n))
    lib().ora_mass_matrix_jac(om.ref, _ptr(q), _ptr(Mm))
    return Mm


def contact(model, q, qd):
    """(tau_c [n], D_c [n, n], sphere forces [S, 3]) at (q, qd)."""
    om = _as(model)
    Rb, pb, s, o = fk(om, q)
    qd = np.ascontiguousarray(qd, dtype=np.float64)
    tau = np.zeros(om.n); D = np.zeros((om.n, om.n)); fs = np.zeros((max(om.model.n_spheres, 1), 3))
    lib().ora_contact(om.ref, _ptr(Rb), _ptr(pb), _ptr(s), _ptr(o), _ptr(qd), _ptr(tau), _ptr(D), _ptr(fs))
    return tau, D, fs[: om.model.n_spheres]


def integrate_q(model, dt, q, qd):
    """Position update of semi-implicit Euler from the new velocities (a copy of q): q + dt qd,
    except a free root's rotation vector, advanced by R <- exp(dt w) R."""
    om = _as(model)
    q = np.array(q, dtype=np.float64, order="C")
    qd = np.ascontiguousarray(qd, dtype=np.float64)
    lib().ora_integrate_q(om.ref, C.c_double(dt), _ptr(q), _ptr(qd))
    return q


def cholesky_solve(A, b):
    A = np.ascontiguousarray(A, dtype=np.float64); b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    bad = lib().ora_cholesky_solve(C.c_int(A.shape[0]), _ptr(A), _ptr(b), _ptr(x))
    return x, bad


_EVAL_KEYS = ("qdd", "force", "L", "R", "lm", "vm", "dFdv", "tau_m", "tau_c", "tau_l", "bias", "M", "A", "rhs",
              "act_next", "sphere_force", "eps_next")


def evaluate(model, dt, q, qd, act, exc, eps=None, L=None, R=None):
    """All intermediates of one substep at one state (dict of float64 arrays, plus 'status').
    eps: tendon strains [m] (None: zero).  L [m] and R [m, n] (optional): muscle-tendon lengths
    and moment arms used in place of the via-point geometry at q (a substep driven by a learned
    geometry); the output's L and R are then these."""
    om = _as(model)
    n, m, S = om.n, om.m, om.model.n_spheres
    shapes = dict(qdd=(n,), force=(m,), L=(m,), R=(m, n), lm=(m,), vm=(m,), dFdv=(m,), tau_m=(n,), tau_c=(n,),
                  tau_l=(n,), bias=(n,), M=(n, n), A=(n, n), rhs=(n,), act_next=(m,), sphere_force=(max(S, 1), 3),
                  eps_next=(max(m, 1),))
    res = {k: np.zeros(shapes[k]) for k in _EVAL_KEYS}
    out = _EvalOut(**{k: _ptr(v) for k, v in res.items()})
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (q, qd, act, exc)]
    e = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64)
    Lg = None if L is None else np.ascontiguousarray(L, dtype=np.float64).reshape(m)
    Rg = None if R is None else np.ascontiguousarray(R, dtype=np.float64).reshape(m, n)
    st = lib().ora_eval_geom(om.ref, _ptr(om.L0), C.c_double(dt), _ptr(a[0]), _ptr(a[1]), _ptr(a[2]), _ptr(a[3]),
                             _ptr(e) if e is not None else None, _ptr(Lg) if Lg is not None else None,
                             _ptr(Rg) if Rg is not None else None, C.byref(out))
    res["eps_next"] = res["eps_next"][:m]
    res["sphere_force"] = res["sphere_force"][:S]
    res["status"] = st
    return res


def step(model, dt, q, qd, act, exc, n_sub=1, n_threads=0, eps=None):
    """Advance E environments by n_sub substeps (exc [E, m] held).  eps [E, m]: tendon strains
    (None: zero, the state after a reset).  Returns new (q, qd, act, qdd, force, status, eps);
    inputs are not modified."""
    om = _as(model)
    q = np.array(q, dtype=np.float64, order="C"); qd = np.array(qd, dtype=np.float64, order="C")
    act = np.array(act, dtype=np.float64, order="C"); exc = np.ascontiguousarray(exc, dtype=np.float64)
    E = q.shape[0]
    eps = np.zeros((E, om.m)) if eps is None else np.array(eps, dtype=np.float64, order="C").reshape(E, om.m)
    qdd = np.zeros((E, om.n)); F = np.zeros((E, om.m)); status = np.zeros(E, dtype=np.int32)
    lib().ora_step(om.ref, _ptr(om.L0), C.c_double(dt), C.c_int(E), C.c_int(n_sub), _ptr(q), _ptr(qd), _ptr(act),
                   _ptr(exc), _ptr(eps), _ptr(qdd), _ptr(F), _ptr(status, _ip), C.c_int(n_threads))
    return q, qd, act, qdd, F, status, eps


def max_threads():
    return lib().ora_max_threads()
