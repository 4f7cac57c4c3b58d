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
                ("vmax_per_lopt", C.c_float),
                ("n_wraps", C.c_int32), ("wrap_muscle", _i32p), ("wrap_segment", _i32p), ("wrap_body", _i32p),
                ("wrap_center", _f32p), ("wrap_axis", _f32p), ("wrap_radius", _f32p), ("free_root", C.c_int32),
                ("wrap_kind", _i32p), ("muscle_tendon_strain", _f32p), ("limit_delta", C.c_float)]


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


class SurrogateInfo(C.Structure):
    _fields_ = [("env_substeps", C.c_uint64), ("learned", C.c_uint64), ("out_of_box", C.c_uint64),
                ("flagged", C.c_uint64), ("checked", C.c_uint64), ("check_failed", C.c_uint64),
                ("max_check_error", C.c_float), ("train_loss", C.c_float), ("flagged_envs", C.c_int32),
                ("trained", C.c_int32), ("structured", C.c_int32), ("hidden", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneResult(C.Structure):
    _fields_ = [("mixed", C.c_int32), ("mixed_warps_per_env", C.c_int32), ("mixed_slots", C.c_int32),
                ("mixed_stage_points_mask", C.c_int32), ("warps_per_env", C.c_int32 * 8),
                ("envs_per_block", C.c_int32 * 8), ("stage_points", C.c_int32 * 8), ("ms_per_model", C.c_float),
                ("ms_mixed", C.c_float), ("candidates", C.c_int32), ("from_cache", C.c_int32)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if isinstance(v, C.Array) else v
        return out


class EvalOut(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in _EVAL_FIELDS] + [("nnz_pitch", C.c_int32), ("packed_pitch", C.c_int32),
                                                           ("tendon_strain", C.c_void_p),
                                                           ("tendon_strain_next", C.c_void_p)]


EXPORTS = ("msim_create", "msim_destroy", "msim_get_dims", "msim_reset", "msim_step", "msim_step_host",
           "msim_step_host_async", "msim_host_wait",
           "msim_get_state", "msim_get_status", "msim_clear_status", "msim_eval", "msim_get_layout",
           "msim_set_launch", "msim_gemm_bf16", "msim_gemm_bf16_mn", "msim_mlp_create", "msim_mlp_destroy", "msim_mlp_layout",
           "msim_mlp_get", "msim_mlp_set", "msim_mlp_forward", "msim_mlp_backward", "msim_mlp_adam",
           "msim_surrogate_train", "msim_set_geometry_mode", "msim_surrogate_set_check", "msim_surrogate_stats",
           "msim_surrogate_network", "msim_geometry", "msim_surrogate_predict", "msim_mlp_forward_noalloc",
           "msim_set_mixed_launch", "msim_autotune", "msim_surrogate_set_box", "msim_surrogate_set_width",
           "msim_surrogate_set_structure", "msim_policy_attach",
           "msim_policy_step", "msim_policy_excitations", "msim_measure_fp32_peak", "msim_flow_attach",
           "msim_flow_actions", "msim_reward_attach", "msim_reward", "msim_body_positions", "msim_tendon_strain",
           "msim_last_error", "msim_version")

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
    lib.msim_step_host_async.argtypes = [vp, vp, C.c_int32, vp, vp, vp]
    lib.msim_host_wait.argtypes = [vp]
    lib.msim_get_state.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.msim_get_status.argtypes = [vp, C.POINTER(C.c_uint32)]
    lib.msim_clear_status.argtypes = [vp, vp]
    lib.msim_eval.argtypes = [vp, vp, vp, vp, vp, C.POINTER(EvalOut), vp]
    lib.msim_tendon_strain.argtypes = [vp, vp, vp, vp]
    lib.msim_get_layout.argtypes = [vp, C.c_int32, vp, vp, vp, vp, vp]
    lib.msim_set_launch.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
    lib.msim_gemm_bf16.argtypes = [vp, C.c_int32, vp, C.c_int32, vp, vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                   C.c_int32, C.c_int32, vp, C.c_int32, vp, vp]
    lib.msim_gemm_bf16_mn.argtypes = [vp, C.c_int32, C.c_int32, vp, C.c_int32, C.c_int32, vp, vp, C.c_int32, vp,
                                      C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, vp,
                                      C.c_int32, vp, vp]
    lib.msim_mlp_create.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.c_float,
                                    C.POINTER(vp)]
    lib.msim_mlp_destroy.argtypes = [vp]
    lib.msim_mlp_layout.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_int32)]
    lib.msim_mlp_get.argtypes = [vp, C.c_int32, vp, C.c_int64]
    lib.msim_mlp_set.argtypes = [vp, C.c_int32, vp, C.c_int64, C.c_int32]
    lib.msim_mlp_forward.argtypes = [vp, vp, C.c_int32, C.c_int32, vp, C.c_int32, vp]
    lib.msim_mlp_backward.argtypes = [vp, vp, C.c_int32, vp, C.c_int32, C.c_int32, C.POINTER(C.c_float), vp]
    lib.msim_mlp_adam.argtypes = [vp, C.c_float, C.c_float, C.c_float, C.c_float, vp]
    lib.msim_surrogate_train.argtypes = [vp, C.c_int64, C.c_int32, C.c_int32, C.c_float, vp]
    lib.msim_set_geometry_mode.argtypes = [vp, C.c_int32]
    lib.msim_surrogate_set_check.argtypes = [vp, C.c_float, C.c_float]
    lib.msim_surrogate_set_box.argtypes = [vp, C.c_float]
    lib.msim_surrogate_set_width.argtypes = [vp, C.c_int32]
    lib.msim_surrogate_set_structure.argtypes = [vp, C.c_int32]
    lib.msim_surrogate_stats.argtypes = [vp, C.POINTER(SurrogateInfo), C.c_int32]
    lib.msim_surrogate_network.argtypes = [vp, C.POINTER(vp)]
    lib.msim_geometry.argtypes = [vp, C.c_int32, vp, C.c_int32, C.c_int32, vp, C.c_int32, vp]
    lib.msim_surrogate_predict.argtypes = [vp, vp, C.c_int32, C.c_int32, vp, C.c_int32, vp]
    lib.msim_mlp_forward_noalloc.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, vp, C.c_int32, vp, vp, vp,
                                             vp, vp, vp, C.c_int32, C.c_int32, vp, C.c_int32, vp, vp]
    lib.msim_set_mixed_launch.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
    lib.msim_autotune.argtypes = [vp, C.c_char_p, C.c_int32, C.POINTER(TuneResult)]
    lib.msim_policy_attach.argtypes = [vp, vp]
    lib.msim_policy_step.argtypes = [vp, C.c_int32, C.c_int32, vp]
    lib.msim_policy_excitations.argtypes = [vp, vp, vp]
    lib.msim_measure_fp32_peak.argtypes = [C.c_int32, C.POINTER(C.c_double)]
    lib.msim_flow_attach.argtypes = [vp, vp, C.c_int32, C.c_float, C.c_float]
    lib.msim_flow_actions.argtypes = [vp, vp, vp, vp]
    lib.msim_reward_attach.argtypes = [vp, vp, C.c_float]
    lib.msim_reward.argtypes = [vp, vp, vp, vp, vp, C.c_int32, vp]
    lib.msim_body_positions.argtypes = [vp, vp, C.c_int32, C.c_int32, vp, vp]
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
                sphere_pos=f(model.sphere_pos), sphere_radius=f(model.sphere_radius),
                wrap_muscle=i(model.wrap_muscle), wrap_segment=i(model.wrap_segment), wrap_body=i(model.wrap_body),
                wrap_center=f(model.wrap_center), wrap_axis=f(model.wrap_axis), wrap_radius=f(model.wrap_radius),
                wrap_kind=i(getattr(model, "wrap_kind", np.zeros(0))))
    ts = np.asarray(getattr(model, "muscle_tendon_strain", np.zeros(0)), dtype=np.float32).reshape(-1)
    if ts.shape[0] == model.n_muscles and np.any(ts > 0):
        keep["muscle_tendon_strain"] = f(ts)
    d = ModelDesc()
    d.n_bodies, d.n_dofs, d.n_muscles = model.n_bodies, model.n_dofs, model.n_muscles
    d.n_points, d.n_spheres = model.n_points, model.n_spheres
    d.n_wraps = int(model.wrap_muscle.shape[0])
    d.free_root = 1 if getattr(model, "free_root", False) else 0
    for k, v in keep.items():
        setattr(d, k, v.ctypes.data_as(_i32p if v.dtype == np.int32 else _f32p) if v.size else None)
    d.gravity = (C.c_float * 3)(*[float(x) for x in model.gravity])
    for k, v in model.scalars().items():
        setattr(d, k, float(v))
    return d, keep


class Sim:
    """A batch of environments of one or more models on one CUDA device (``msim_create``)."""

    def __init__(self, models, envs_per_model, dt=1e-3, device=0, geometry_mode=0, seed=0):
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
        args = CreateArgs(len(descs), arr, epm.ctypes.data_as(_i32p), geometry_mode, float(dt), seed, device)
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

    def step_host_async(self, exc_host, n_sub=1, q_host=None, qd_host=None, stream=None):
        """Pipelined host stepping: queue the upload, the step and the download and return; the
        pinned host buffers must stay untouched until :meth:`host_wait`."""
        self._check(self.lib.msim_step_host_async(self.h, _ptr(exc_host), int(n_sub), _ptr(q_host), _ptr(qd_host),
                                                  _stream_ptr(stream)))

    def host_wait(self):
        self._check(self.lib.msim_host_wait(self.h))

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

    def tendon_strain(self, set=None, stream=None):
        """The tendon strains of compliant tendons ([n_envs, pitch_m] device tensor); ``set``
        (same shape) replaces them first."""
        out = self.zeros(self.pitch_m)
        self._check(self.lib.msim_tendon_strain(self.h, _ptr(set), _ptr(out), _stream_ptr(stream)))
        return out

    def eval(self, q, qd, act, exc, stream=None, eps=None):
        """All intermediates of one substep (dict of device tensors, padded rows); ``eps``: the
        tendon strains of the evaluated states (None: zero), their update in 'eps_next'."""
        nnz_p = max(4, (max(self.dims.nnz[: len(self.models)]) + 3) // 4 * 4)
        pk_p = max(4, (max(self.dims.n_packed[: len(self.models)]) + 3) // 4 * 4)
        cols = dict(L=self.pitch_m, lm=self.pitch_m, vm=self.pitch_m, force=self.pitch_m, act_next=self.pitch_m,
                    R=nnz_p, tau_m=self.pitch_n, tau_c=self.pitch_n, tau_l=self.pitch_n, bias=self.pitch_n,
                    rhs=self.pitch_n, qdd=self.pitch_n, M=pk_p, A=pk_p)
        res = {k: self.zeros(c) for k, c in cols.items()}
        res["eps_next"] = self.zeros(self.pitch_m)
        out = EvalOut(*[_ptr(res[k]) for k in _EVAL_FIELDS], nnz_p, pk_p, _ptr(eps), _ptr(res["eps_next"]))
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


    def set_mixed_launch(self, enable=True, warps_per_env=0, slots_per_block=0, stage_points_mask=-1):
        """One persistent launch for all models (msim_set_mixed_launch)."""
        self._check(self.lib.msim_set_mixed_launch(self.h, 1 if enable else 0, warps_per_env, slots_per_block,
                                                   stage_points_mask))

    def autotune(self, cache_path=None, n_sub=10):
        """Launch-shape autotuner (msim_autotune); returns the chosen shapes and timings."""
        r = TuneResult()
        path = cache_path.encode() if cache_path else None
        self._check(self.lib.msim_autotune(self.h, path, int(n_sub), C.byref(r)))
        self._check(self.lib.msim_get_dims(self.h, C.byref(self.dims)))
        return r.as_dict()

    # ------------------------------------------------------------------ policy in the loop
    def policy_attach(self, net):
        """Bind an MLP (in >= 2n + 2m, out = m, sigmoid) as the policy; None detaches."""
        self._policy = net
        self._check(self.lib.msim_policy_attach(self.h, net.h if net is not None else None))

    def policy_step(self, n_sub_per_act=2, n_acts=1, stream=None):
        self._check(self.lib.msim_policy_step(self.h, int(n_sub_per_act), int(n_acts), _stream_ptr(stream)))

    def flow_attach(self, net, n_steps=20, dt=0.05, sigma=0.0):
        """Refine the policy's action with a flow network (in = policy in + m + 1, out = m)."""
        self._flow = net
        self._check(self.lib.msim_flow_attach(self.h, net.h if net is not None else None, int(n_steps), float(dt),
                                              float(sigma)))

    def flow_actions(self, stream=None):
        """(sampler mean, last refined action), [n_envs, pitch_m] each."""
        mu, a = self.zeros(self.pitch_m), self.zeros(self.pitch_m)
        self._check(self.lib.msim_flow_actions(self.h, _ptr(mu), _ptr(a), _stream_ptr(stream)))
        return mu, a

    def reward_attach(self, disc, w_power=0.0):
        """Bind the discriminator (in = n + 3 nb, out = 1, sigmoid) of the imitation reward."""
        self._disc = disc
        self._check(self.lib.msim_reward_attach(self.h, disc.h if disc is not None else None, float(w_power)))

    def reward(self, q_ref, stream=None, with_parts=False, with_delta=False):
        """Imitation reward of every environment against q_ref [n_envs, pitch_n] (CUDA)."""
        import torch
        r = torch.zeros(self.n_envs, device=self.device)
        parts = torch.zeros((self.n_envs, 2), device=self.device) if with_parts else None
        nd = self.dims.n_dofs[0] + 3 * self.dims.n_bodies[0]
        delta = torch.zeros((self.n_envs, nd), device=self.device) if with_delta else None
        self._check(self.lib.msim_reward(self.h, _ptr(q_ref), _ptr(r), _ptr(parts) if parts is not None else None,
                                         _ptr(delta) if delta is not None else None, nd, _stream_ptr(stream)))
        return r, parts, delta

    def body_positions(self, q, stream=None):
        """Body origins [rows, 3 nb] at configurations q [rows, >= n] (CUDA FP32)."""
        import torch
        q = q.contiguous()
        out = torch.zeros((q.shape[0], 3 * self.dims.n_bodies[0]), device=self.device)
        self._check(self.lib.msim_body_positions(self.h, q.data_ptr(), q.stride(0), q.shape[0], out.data_ptr(),
                                                 _stream_ptr(stream)))
        return out

    def policy_excitations(self, stream=None):
        out = self.zeros(self.pitch_m)
        self._check(self.lib.msim_policy_excitations(self.h, _ptr(out), _stream_ptr(stream)))
        return out

    # ------------------------------------------------------------------ learned geometry
    def geometry(self, q, model=0, stream=None):
        """Exact geometry rows [L | R (sparse order)] at configurations q [rows, >= n] (CUDA FP32)."""
        import torch
        q = q.contiguous()
        nm = self.dims.n_muscles[model] + self.dims.nnz[model]
        out = torch.zeros((q.shape[0], nm), device=self.device)
        self._check(self.lib.msim_geometry(self.h, model, q.data_ptr(), q.stride(0), q.shape[0], out.data_ptr(),
                                           out.stride(0), _stream_ptr(stream)))
        return out

    def train_surrogate(self, n_samples, epochs, batch=4096, lr=1e-3, stream=None):
        self._check(self.lib.msim_surrogate_train(self.h, int(n_samples), int(epochs), int(batch), float(lr),
                                                  _stream_ptr(stream)))

    def surrogate_set_box(self, margin):
        self._check(self.lib.msim_surrogate_set_box(self.h, float(margin)))

    def surrogate_set_width(self, hidden):
        self._check(self.lib.msim_surrogate_set_width(self.h, int(hidden)))

    def surrogate_set_structure(self, structured):
        self._check(self.lib.msim_surrogate_set_structure(self.h, 1 if structured else 0))

    def set_geometry_mode(self, mode):
        self._check(self.lib.msim_set_geometry_mode(self.h, int(mode)))

    def surrogate_set_check(self, check_frac, tol=1e-3):
        self._check(self.lib.msim_surrogate_set_check(self.h, float(check_frac), float(tol)))

    def surrogate_stats(self, reset=False):
        info = SurrogateInfo()
        self._check(self.lib.msim_surrogate_stats(self.h, C.byref(info), 1 if reset else 0))
        return info.as_dict()

    def surrogate_predict(self, q, stream=None):
        import torch
        q = q.contiguous()
        nm = self.dims.n_muscles[0] + self.dims.nnz[0]
        out = torch.zeros((q.shape[0], nm), device=self.device)
        self._check(self.lib.msim_surrogate_predict(self.h, q.data_ptr(), q.stride(0), q.shape[0], out.data_ptr(),
                                                    out.stride(0), _stream_ptr(stream)))
        return out

    def surrogate_network(self):
        """The trained network as a borrowed MLP (parameters readable and replaceable)."""
        h = C.c_void_p()
        self._check(self.lib.msim_surrogate_network(self.h, C.byref(h)))
        d_in = self.dims.n_dofs[0]
        off = (C.c_int64 * 6)()
        ip = C.c_int32()
        self.lib.msim_mlp_layout(h, off, None, C.byref(ip), None)
        hidden = (off[1] - off[0]) // ip.value
        return MLP.borrowed(h, d_in, hidden, self.dims.n_muscles[0] + self.dims.nnz[0])


def measure_fp32_peak(device=0):
    """FP32 FMA throughput of the device in TFLOP/s (msim_measure_fp32_peak)."""
    lib = load_library()
    v = C.c_double()
    st = lib.msim_measure_fp32_peak(int(device), C.byref(v))
    if st != MSIM_OK:
        raise MsimError(st, "msim_measure_fp32_peak failed")
    return v.value


def gemm_bf16(A, B, bias=None, act=0, out_bf16=False, Z=None, err=None, stream=None, a_mn=False, b_mn=False,
              addend=None):
    """C = act(A B^T + bias + addend) on the tensor cores (msim_gemm_bf16_mn).  A [M, K] (or, with
    a_mn, its transpose [K, M] as stored), B [N, K] (with b_mn [K, N]): BF16 CUDA tensors with unit
    column stride and row pitches multiple of 8; addend (optional) FP32 [M, N] with unit column
    stride."""
    import torch
    lib = load_library()
    M, K = (A.shape[1], A.shape[0]) if a_mn else A.shape
    N = B.shape[1] if b_mn else B.shape[0]
    if (B.shape[0] if b_mn else B.shape[1]) != K:
        raise ValueError("gemm_bf16: inner dimensions differ")
    C = torch.empty((M, N), device=A.device, dtype=torch.bfloat16 if out_bf16 else torch.float32)
    st = lib.msim_gemm_bf16_mn(A.data_ptr(), A.stride(0), 1 if a_mn else 0, B.data_ptr(), B.stride(0),
                               1 if b_mn else 0, None if bias is None else bias.data_ptr(),
                               None if addend is None else addend.data_ptr(), 0 if addend is None else addend.stride(0),
                               C.data_ptr(), C.stride(0),
                               M, N, K, 1 if out_bf16 else 0, act, None if Z is None else Z.data_ptr(),
                               0 if Z is None else Z.stride(0), None if err is None else err.data_ptr(),
                               _stream_ptr(stream))
    if st != MSIM_OK:
        raise MsimError(st, lib.msim_last_error(None).decode())
    return C


class MLP:
    """3-layer MLP on the tensor cores (msim_mlp_*): BF16 weights/activations, FP32 accumulation."""

    def __init__(self, d_in, hidden, d_out, out_sigmoid=False, max_batch=4096, seed=0, out_scale=1.0):
        self.lib = load_library()
        h = C.c_void_p()
        st = self.lib.msim_mlp_create(d_in, hidden, d_out, 2 if out_sigmoid else 0, max_batch, seed, out_scale,
                                      C.byref(h))
        if st != MSIM_OK:
            raise MsimError(st, self.lib.msim_last_error(None).decode())
        self.h = h
        self._layout(d_in, hidden, d_out, max_batch)

    @classmethod
    def borrowed(cls, h, d_in, hidden, d_out):
        """A view of a network owned elsewhere (a simulator's surrogate); close() leaves it alone."""
        self = cls.__new__(cls)
        self.lib = load_library()
        self.h = h
        self._borrowed = True
        self._layout(d_in, hidden, d_out, 0)
        return self

    def _layout(self, d_in, hidden, d_out, max_batch):
        off = (C.c_int64 * 6)()
        n = C.c_int64()
        ip, op = C.c_int32(), C.c_int32()
        self.lib.msim_mlp_layout(self.h, off, C.byref(n), C.byref(ip), C.byref(op))
        self.offsets = list(off)
        self.n_params = n.value
        self.in_pitch, self.out_pitch = ip.value, op.value
        self.d_in, self.hidden, self.d_out, self.max_batch = d_in, hidden, d_out, max_batch

    def _check(self, st):
        if st != MSIM_OK:
            raise MsimError(st, self.lib.msim_last_error(None).decode())

    def close(self):
        if getattr(self, "h", None) and not getattr(self, "_borrowed", False):
            self.lib.msim_mlp_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # flat <-> (W1, b1, W2, b2, W3, b3)
    def unflatten(self, flat):
        o, h = self.offsets, self.hidden
        W1 = flat[o[0]:o[0] + h * self.in_pitch].reshape(h, self.in_pitch)[:, : self.d_in]
        W3 = flat[o[4]:o[4] + self.out_pitch * h].reshape(self.out_pitch, h)[: self.d_out]
        return [W1, flat[o[1]:o[1] + h], flat[o[2]:o[2] + h * h].reshape(h, h), flat[o[3]:o[3] + h], W3,
                flat[o[5]:o[5] + self.d_out]]

    def flatten(self, params):
        flat = np.zeros(self.n_params, np.float32)
        o, h = self.offsets, self.hidden
        W1 = np.zeros((h, self.in_pitch), np.float32)
        W1[:, : self.d_in] = params[0]
        flat[o[0]:o[0] + W1.size] = W1.ravel()
        flat[o[1]:o[1] + h] = params[1]
        flat[o[2]:o[2] + h * h] = np.asarray(params[2], np.float32).ravel()
        flat[o[3]:o[3] + h] = params[3]
        W3 = np.zeros((self.out_pitch, h), np.float32)
        W3[: self.d_out] = params[4]
        flat[o[4]:o[4] + W3.size] = W3.ravel()
        flat[o[5]:o[5] + self.d_out] = params[5]
        return flat

    def get(self, which=0):
        flat = np.zeros(self.n_params, np.float32)
        self._check(self.lib.msim_mlp_get(self.h, which, flat.ctypes.data, self.n_params))
        return flat

    def set(self, flat, which=0, adam_step=0):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        self._check(self.lib.msim_mlp_set(self.h, which, flat.ctypes.data, self.n_params, adam_step))

    def pad_input(self, X):
        """[B, d_in] -> BF16 CUDA tensor [B, in_pitch]."""
        import torch
        X = torch.as_tensor(X).float()
        out = torch.zeros((X.shape[0], self.in_pitch), dtype=torch.bfloat16, device="cuda")
        out[:, : self.d_in] = X.cuda().bfloat16()
        return out

    def forward(self, Xb, Y=None, stream=None):
        import torch
        B = Xb.shape[0]
        if Y is None:
            Y = torch.empty((B, self.out_pitch), dtype=torch.float32, device="cuda")
        self._check(self.lib.msim_mlp_forward(self.h, Xb.data_ptr(), Xb.stride(0), B, Y.data_ptr(), Y.stride(0),
                                              _stream_ptr(stream)))
        return Y

    def backward(self, Xb, T, stream=None):
        loss = C.c_float()
        self._check(self.lib.msim_mlp_backward(self.h, Xb.data_ptr(), Xb.stride(0), T.data_ptr(), T.stride(0),
                                               Xb.shape[0], C.byref(loss), _stream_ptr(stream)))
        return loss.value

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        self._check(self.lib.msim_mlp_adam(self.h, lr, beta1, beta2, eps, _stream_ptr(stream)))


NOALLOC_MAX_ACT_ELEMS = 8 * 1024 * 1024   # MSIM_NOALLOC_MAX_ACT_ELEMS: B * hidden limit


def mlp_forward_noalloc(W1, b1, W2, b2, W3, b3, X, d_in, out_sigmoid=False, Y=None, status=None, stream=None):
    """msim_mlp_forward_noalloc: the MLP forward at caller-held CUDA weights (BF16 W, FP32 b), no
    device allocation inside the call.  W1 [hidden, >= d_in] (pitch = its row stride), W2 [hidden,
    hidden], W3 [out, hidden], X [B, >= d_in] BF16.  Returns Y [B, out] FP32 (allocated here by torch
    unless given)."""
    import torch
    lib = load_library()
    hidden, out, B = W2.shape[0], W3.shape[0], X.shape[0]
    dev = X.device
    if dev.type != "cuda":
        raise ValueError("mlp_forward_noalloc: X must be a CUDA tensor")
    if Y is None:
        Y = torch.empty((B, out), dtype=torch.float32, device=dev)
    want = dict(W1=(W1, torch.bfloat16), W2=(W2, torch.bfloat16), W3=(W3, torch.bfloat16), X=(X, torch.bfloat16),
                b1=(b1, torch.float32), b2=(b2, torch.float32), b3=(b3, torch.float32), Y=(Y, torch.float32))
    if status is not None:
        want["status"] = (status, status.dtype if status.dtype in (torch.int32, torch.uint32) else torch.int32)
    for name, (t, dt) in want.items():
        # the scratch array and the stream are those of the current device: every operand must
        # live there (a peer device's memory is not reachable by the GEMMs' tensor maps)
        if t.device != dev or t.dtype != dt or (t.dim() > 0 and t.stride(-1) != 1):
            raise ValueError("mlp_forward_noalloc: %s must be %s on %s with unit inner stride" % (name, dt, dev))
    if W2.stride(0) != hidden or W3.stride(0) != hidden or W1.stride(0) < d_in or X.stride(0) < d_in:
        raise ValueError("mlp_forward_noalloc: W2 and W3 rows must be contiguous, W1 and X pitches >= d_in")
    with torch.cuda.device(dev):
        st = lib.msim_mlp_forward_noalloc(d_in, hidden, out, 2 if out_sigmoid else 0, W1.data_ptr(), W1.stride(0),
                                          b1.data_ptr(), W2.data_ptr(), b2.data_ptr(), W3.data_ptr(), b3.data_ptr(),
                                          X.data_ptr(), X.stride(0), B, Y.data_ptr(), Y.stride(0),
                                          status.data_ptr() if status is not None else None, _stream_ptr(stream))
    if st != MSIM_OK:
        raise MsimError(st, lib.msim_last_error(None).decode())
    return Y


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
