"""Python binding of the C ABI in ``include/msim.h`` (ctypes; argument marshalling only).

Every step of the simulation runs in the CUDA library ``libmsim.so`` built in-tree next to this
file; PyTorch provides device memory and streams.  There is no CPU fallback: if the library or
a CUDA device is missing, constructing :class:`Sim` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmsim.so")

MSIM_OK = 0
STATUS_NAMES = {0: "MSIM_OK", 1: "MSIM_ERR_ARG", 2: "MSIM_ERR_CUDA", 3: "MSIM_ERR_OOM", 4: "MSIM_ERR_MODEL",
                5: "MSIM_ERR_TIMEOUT", 6: "MSIM_ERR_STATE", 7: "MSIM_ERR_UNSUPPORTED"}
ENV_NONFINITE = 0x1
ENV_NOT_SPD = 0x2
FLAG_TIMEOUT = 0x100

_i32p = C.POINTER(C.c_int32)
_f32p = C.POINTER(C.c_float)


class ModelDesc(C.Structure):
    _fields_ = [("n_bodies", C.c_int32), ("n_dofs", C.c_int32), ("n_muscles", C.c_int32), ("n_points", C.c_int32),
                ("n_spheres", C.c_int32),
                ("body_parent", _i32p), ("body_ndof", _i32p), ("body_offset", _f32p), ("body_mass", _f32p),
                ("body_com", _f32p), ("body_inertia", _f32p), ("dof_axis", _f32p), ("dof_limit", _f32p),
                ("dof_damping", _f32p), ("muscle_point_start", _i32p), ("muscle_fmax", _f32p),
                ("muscle_lopt", _f32p), ("muscle_lslack", _f32p), ("point_body", _i32p), ("point_pos", _f32p),
                ("sphere_body", _i32p), ("sphere_pos", _f32p), ("sphere_radius", _f32p),
                ("gravity", C.c_float * 3), ("contact_k", C.c_float), ("contact_c", C.c_float),
                ("contact_mu", C.c_float), ("contact_eps", C.c_float), ("limit_k", C.c_float),
                ("limit_c", C.c_float), ("tau_act", C.c_float), ("tau_deact", C.c_float),
                ("vmax_per_lopt", C.c_float)]


class CreateArgs(C.Structure):
    _fields_ = [("n_models", C.c_int32), ("models", C.POINTER(ModelDesc)), ("envs_per_model", _i32p),
                ("geometry_mode", C.c_int32), ("dt", C.c_float), ("seed", C.c_uint64), ("device", C.c_int32)]


class Dims(C.Structure):
    _fields_ = [("n_envs", C.c_int32), ("n_models", C.c_int32), ("pitch_n", C.c_int32), ("pitch_m", C.c_int32),
                ("env_begin", C.c_int32 * 9), ("n_dofs", C.c_int32 * 8), ("n_muscles", C.c_int32 * 8),
                ("n_bodies", C.c_int32 * 8), ("nnz", C.c_int32 * 8), ("n_packed", C.c_int32 * 8),
                ("envs_per_block", C.c_int32 * 8), ("image_bytes", C.c_int32 * 8),
                ("workspace_bytes_per_env", C.c_int32 * 8), ("points_in_smem", C.c_int32 * 8),
                ("warps_per_env", C.c_int32 * 8)]


_EVAL_FIELDS = ("L", "lm", "vm", "force", "act_next", "R", "tau_m", "tau_c", "tau_l", "bias", "rhs", "qdd", "M", "A")


class EvalOut(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in _EVAL_FIELDS] + [("nnz_pitch", C.c_int32), ("packed_pitch", C.c_int32)]


EXPORTS = ("msim_create", "msim_destroy", "msim_get_dims", "msim_reset", "msim_step", "msim_step_host",
           "msim_get_state", "msim_get_status", "msim_clear_status", "msim_eval", "msim_get_layout",
           "msim_set_launch", "msim_gemm_bf16", "msim_last_error", "msim_version")

_lib = None


def load_library(path=LIB_PATH):
    """Load ``libmsim.so`` (raises OSError if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libmsim.so not found at %s: build it with python -m paper_2603_29332_b300.build" % path)
    lib = C.CDLL(path)
    vp = C.c_void_p
    lib.msim_create.argtypes = [C.POINTER(CreateArgs), C.POINTER(vp)]
    lib.msim_destroy.argtypes = [vp]
    lib.msim_get_dims.argtypes = [vp, C.POINTER(Dims)]
    lib.msim_reset.argtypes = [vp, vp, vp, vp, vp, C.c_int32, vp]
    lib.msim_step.argtypes = [vp, vp, C.c_int32, vp]
    lib.msim_step_host.argtypes = [vp, vp, C.c_int32, vp, vp, vp]
    lib.msim_get_state.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.msim_get_status.argtypes = [vp, C.POINTER(C.c_uint32)]
    lib.msim_clear_status.argtypes = [vp, vp]
    lib.msim_eval.argtypes = [vp, vp, vp, vp, vp, C.POINTER(EvalOut), vp]
    lib.msim_get_layout.argtypes = [vp, C.c_int32, vp, vp, vp, vp, vp]
    lib.msim_set_launch.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
    lib.msim_gemm_bf16.argtypes = [vp, C.c_int32, vp, C.c_int32, vp, vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                   C.c_int32, C.c_int32, vp, C.c_int32, vp, vp]
    lib.msim_last_error.argtypes = [vp]
    lib.msim_last_error.restype = C.c_char_p
    lib.msim_version.restype = C.c_int32
    for name in EXPORTS:
        if name not in ("msim_last_error", "msim_version"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


class MsimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, str(code)), msg))
        self.code = code


def _ptr(t):
    """Device (or host) address of a torch tensor / numpy array, or None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def model_desc(model):
    """Marshal a :class:`modelgen.Model` into the C struct; returns (desc, keep-alive arrays)."""
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    i = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    keep = dict(body_parent=i(model.body_parent), body_ndof=i(model.body_ndof), body_offset=f(model.body_offset),
                body_mass=f(model.body_mass), body_com=f(model.body_com), body_inertia=f(model.body_inertia),
                dof_axis=f(model.dof_axis), dof_limit=f(model.dof_limit), dof_damping=f(model.dof_damping),
                muscle_point_start=i(model.muscle_point_start), muscle_fmax=f(model.muscle_fmax),
                muscle_lopt=f(model.muscle_lopt), muscle_lslack=f(model.muscle_lslack),
                point_body=i(model.point_body), point_pos=f(model.point_pos), sphere_body=i(model.sphere_body),
                sphere_pos=f(model.sphere_pos), sphere_radius=f(model.sphere_radius))
    d = ModelDesc()
    d.n_bodies, d.n_dofs, d.n_muscles = model.n_bodies, model.n_dofs, model.n_muscles
    d.n_points, d.n_spheres = model.n_points, model.n_spheres
    for k, v in keep.items():
        setattr(d, k, v.ctypes.data_as(_i32p if v.dtype == np.int32 else _f32p) if v.size else None)
    d.gravity = (C.c_float * 3)(*[float(x) for x in model.gravity])
    for k, v in model.scalars().items():
        setattr(d, k, float(v))
    return d, keep


class Sim:
    """A batch of environments of one or more models on one CUDA device (``msim_create``)."""

    def __init__(self, models, envs_per_model, dt=1e-3, device=0, geometry_mode=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2603_29332_b300.Sim needs a CUDA device (no CPU fallback)")
        self.lib = load_library()
        if not isinstance(models, (list, tuple)):
            models, envs_per_model = [models], [envs_per_model]
        self.models = list(models)
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        descs, self._keep = [], []
        for m in self.models:
            d, k = model_desc(m)
            descs.append(d)
            self._keep.append(k)
        arr = (ModelDesc * len(descs))(*descs)
        epm = np.ascontiguousarray(envs_per_model, dtype=np.int32)
        args = CreateArgs(len(descs), arr, epm.ctypes.data_as(_i32p), geometry_mode, float(dt), 0, device)
        h = C.c_void_p()
        st = self.lib.msim_create(C.byref(args), C.byref(h))
        if st != MSIM_OK:
            raise MsimError(st, self.lib.msim_last_error(None).decode())
        self.h = h
        self.dt = float(dt)
        self.dims = Dims()
        self._check(self.lib.msim_get_dims(self.h, C.byref(self.dims)))
        self.n_envs = self.dims.n_envs
        self.pitch_n = self.dims.pitch_n
        self.pitch_m = self.dims.pitch_m
        self.env_begin = list(self.dims.env_begin[: len(self.models) + 1])

    # ------------------------------------------------------------------ helpers
    def _check(self, st):
        if st != MSIM_OK:
            raise MsimError(st, self.lib.msim_last_error(self.h).decode())

    def zeros(self, cols, rows=None, dtype=None):
        import torch
        return torch.zeros((self.n_envs if rows is None else rows, cols), device=self.device,
                           dtype=dtype or torch.float32)

    def pad_n(self, x):
        """[E, n] (any float array) -> device float32 [E, pitch_n], zero padded."""
        return self._pad(x, self.pitch_n)

    def pad_m(self, x):
        return self._pad(x, self.pitch_m)

    def _pad(self, x, pitch):
        import torch
        x = torch.as_tensor(np.asarray(x) if not isinstance(x, torch.Tensor) else x, dtype=torch.float32)
        out = torch.zeros((x.shape[0], pitch), dtype=torch.float32, device=self.device)
        out[:, : x.shape[1]] = x.to(self.device)
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.msim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ API
    def reset(self, q0=None, qd0=None, act0=None, env_ids=None, stream=None):
        n_ids = 0 if env_ids is None else int(env_ids.numel())
        self._check(self.lib.msim_reset(self.h, _ptr(q0), _ptr(qd0), _ptr(act0), _ptr(env_ids), n_ids,
                                        _stream_ptr(stream)))

    def step(self, exc, n_sub=1, stream=None):
        self._check(self.lib.msim_step(self.h, _ptr(exc), int(n_sub), _stream_ptr(stream)))

    def step_host(self, exc_host, n_sub=1, q_host=None, qd_host=None, stream=None):
        self._check(self.lib.msim_step_host(self.h, _ptr(exc_host), int(n_sub), _ptr(q_host), _ptr(qd_host),
                                            _stream_ptr(stream)))

    def state(self, stream=None):
        import torch
        out = dict(q=self.zeros(self.pitch_n), qd=self.zeros(self.pitch_n), qdd=self.zeros(self.pitch_n),
                   act=self.zeros(self.pitch_m), force=self.zeros(self.pitch_m),
                   status=torch.zeros(self.n_envs, dtype=torch.int32, device=self.device))
        self._check(self.lib.msim_get_state(self.h, _ptr(out["q"]), _ptr(out["qd"]), _ptr(out["act"]),
                                            _ptr(out["qdd"]), _ptr(out["force"]), _ptr(out["status"]),
                                            _stream_ptr(stream)))
        return out

    def status(self):
        flags = C.c_uint32(0)
        st = self.lib.msim_get_status(self.h, C.byref(flags))
        return st, flags.value

    def clear_status(self, stream=None):
        self._check(self.lib.msim_clear_status(self.h, _stream_ptr(stream)))

    def set_launch(self, model, envs_per_block=0, stage_points=-1, warps_per_env=0):
        self._check(self.lib.msim_set_launch(self.h, int(model), int(envs_per_block), int(stage_points),
                                             int(warps_per_env)))
        self._check(self.lib.msim_get_dims(self.h, C.byref(self.dims)))

    def eval(self, q, qd, act, exc, stream=None):
        """All intermediates of one substep (dict of device tensors, padded rows)."""
        nnz_p = max(4, (max(self.dims.nnz[: len(self.models)]) + 3) // 4 * 4)
        pk_p = max(4, (max(self.dims.n_packed[: len(self.models)]) + 3) // 4 * 4)
        cols = dict(L=self.pitch_m, lm=self.pitch_m, vm=self.pitch_m, force=self.pitch_m, act_next=self.pitch_m,
                    R=nnz_p, tau_m=self.pitch_n, tau_c=self.pitch_n, tau_l=self.pitch_n, bias=self.pitch_n,
                    rhs=self.pitch_n, qdd=self.pitch_n, M=pk_p, A=pk_p)
        res = {k: self.zeros(c) for k, c in cols.items()}
        out = EvalOut(*[_ptr(res[k]) for k in _EVAL_FIELDS], nnz_p, pk_p)
        self._check(self.lib.msim_eval(self.h, _ptr(q), _ptr(qd), _ptr(act), _ptr(exc), C.byref(out),
                                       _stream_ptr(stream)))
        return res

    def layout(self, model=0):
        n, m, nnz = self.dims.n_dofs[model], self.dims.n_muscles[model], self.dims.nnz[model]
        a = dict(dof_parent=np.zeros(n, np.int32), dof_depth=np.zeros(n, np.int32), packed_row=np.zeros(n, np.int32),
                 muscle_dof_ptr=np.zeros(m + 1, np.int32), muscle_dof=np.zeros(max(nnz, 1), np.int32))
        self._check(self.lib.msim_get_layout(self.h, model, *[a[k].ctypes.data for k in
                                                             ("dof_parent", "dof_depth", "packed_row",
                                                              "muscle_dof_ptr", "muscle_dof")]))
        a["muscle_dof"] = a["muscle_dof"][:nnz]
        return a


def gemm_bf16(A, B, bias=None, act=0, out_bf16=False, Z=None, err=None, stream=None):
    """C = act(A B^T + bias) on the tensor cores (msim_gemm_bf16).  A [M, K], B [N, K]: BF16 CUDA
    tensors with unit column stride and row pitches multiple of 8."""
    import torch
    lib = load_library()
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), device=A.device, dtype=torch.bfloat16 if out_bf16 else torch.float32)
    st = lib.msim_gemm_bf16(A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                            None if bias is None else bias.data_ptr(), C.data_ptr(), C.stride(0), M, N, K,
                            1 if out_bf16 else 0, act, None if Z is None else Z.data_ptr(),
                            0 if Z is None else Z.stride(0), None if err is None else err.data_ptr(),
                            _stream_ptr(stream))
    if st != MSIM_OK:
        raise MsimError(st, lib.msim_last_error(None).decode())
    return C


def unpack_packed(packed, layout):
    """Tree-packed lower triangle (one env row) -> dense symmetric numpy matrix."""
    packed = np.asarray(packed, dtype=np.float64)
    par, dep, row = layout["dof_parent"], layout["dof_depth"], layout["packed_row"]
    n = par.shape[0]
    M = np.zeros((n, n))
    for d in range(n):
        a = d
        while a >= 0:
            v = packed[row[d] + dep[a]]
            M[d, a] = v
            M[a, d] = v
            a = par[a]
    return M


def unpack_R(values, layout, n):
    """Sparse moment arms (one env row) -> dense numpy [m, n]."""
    ptr, dof = layout["muscle_dof_ptr"], layout["muscle_dof"]
    m = ptr.shape[0] - 1
    R = np.zeros((m, n))
    values = np.asarray(values, dtype=np.float64)
    for k in range(m):
        for t in range(ptr[k], ptr[k + 1]):
            R[k, dof[t]] = values[t]
    return R
