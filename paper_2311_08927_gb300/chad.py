"""Python binding of the C ABI in include/chad.h (ctypes; marshalling only).

Every function here forwards to libchad.so, the CUDA library built in-tree by
``paper_2311_08927_gb300.build``.  There is no fallback: if the library is not
built, or no GPU is present, the calls fail loudly.  Buffers may be numpy
arrays (host) or torch CUDA tensors (device; their data_ptr is passed).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import inputs as I

_HERE = os.path.dirname(os.path.abspath(__file__))
# CHAD_LIB selects another build of the library (the bounds-check build,
# libchad_debug.so); by default the in-tree libchad.so
LIB_PATH = os.environ.get("CHAD_LIB") or os.path.join(_HERE, "libchad.so")
_lock = threading.Lock()
_lib = None

NS = 29
MEM_HOST, MEM_DEVICE = 0, 1
PREC_FP64, PREC_MIXED, PREC_MIXED_F32RATES = 0, 1, 2
HEADSPACE_PARTICLE, HEADSPACE_SHARED = 0, 1
STATUS = {0: "CHAD_OK", 1: "CHAD_E_INVALID", 2: "CHAD_E_NOMEM", 3: "CHAD_E_CUDA",
          4: "CHAD_E_STATE", 5: "CHAD_E_PARTICLE"}
P_NEWTON, P_STEPS, P_HMIN, P_NEG, P_NAN = 1, 2, 4, 8, 16

_i64p = C.POINTER(C.c_int64)
_dp = C.POINTER(C.c_double)


class chad_config(C.Structure):
    _fields_ = [("n_digesters", C.c_int), ("n_particles", _i64p), ("V_liq", _dp),
                ("V_gas", _dp), ("params", _dp), ("D_uniform", _dp), ("y_in", _dp),
                ("precision", C.c_int), ("learned", C.c_int), ("headspace", C.c_int),
                ("rtol", C.c_double), ("atol", _dp), ("max_steps_per_interval", C.c_int),
                ("max_newton_iters", C.c_int), ("fixed_substeps", C.c_int),
                ("cuda_stream", C.c_void_p), ("h2_algebraic", C.c_int)]


class chad_flow(C.Structure):
    _fields_ = [("has_flow", C.c_int), ("U", C.c_double), ("R", C.c_double), ("H", C.c_double),
                ("sigma", C.c_double), ("slab_zmin", C.c_double), ("q_in", C.c_double),
                ("y_in", _dp), ("seed", C.c_uint64)]


class chad_stats(C.Structure):
    _fields_ = [("accepted_steps", C.c_int64), ("rejected_steps", C.c_int64),
                ("newton_iters", C.c_int64), ("newton_fallbacks", C.c_int64),
                ("min_steps", C.c_int64), ("max_steps", C.c_int64),
                ("failed_particles", C.c_int64), ("mlp_redo", C.c_int64),
                ("pivot_rejects", C.c_int64),
                ("intervals", C.c_int64), ("sim_days", C.c_double),
                ("h2_newton_iters", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ChadError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def lib():
    """Load libchad.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it with "
                                  "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(LIB_PATH)
            L.chad_abi_version.restype = C.c_int
            L.chad_n_params.restype = C.c_int
            L.chad_param_name.restype = C.c_char_p
            L.chad_param_name.argtypes = [C.c_int]
            L.chad_last_error.restype = C.c_char_p
            L.chad_last_error.argtypes = [C.c_void_p]
            L.chad_create.restype = C.c_int
            L.chad_create.argtypes = [C.POINTER(chad_config), C.POINTER(C.c_void_p)]
            L.chad_destroy.restype = None
            L.chad_destroy.argtypes = [C.c_void_p]
            L.chad_load_particles.restype = C.c_int
            L.chad_load_particles.argtypes = [C.c_void_p, C.c_int, C.c_int64, C.c_void_p,
                                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_int]
            L.chad_set_flow.restype = C.c_int
            L.chad_set_flow.argtypes = [C.c_void_p, C.c_int, C.POINTER(chad_flow)]
            L.chad_step.restype = C.c_int
            L.chad_step.argtypes = [C.c_void_p, C.c_double, C.c_int]
            L.chad_synchronize.restype = C.c_int
            L.chad_synchronize.argtypes = [C.c_void_p]
            L.chad_read_states.restype = C.c_int
            L.chad_read_states.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.POINTER(chad_stats), C.c_int]
            L.chad_set_mlp.restype = C.c_int
            L.chad_set_mlp.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.chad_mlp_features.restype = C.c_int
            L.chad_mlp_features.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                            C.c_void_p, C.c_void_p, C.c_void_p]
            L.chad_mlp_forward.restype = C.c_int
            L.chad_mlp_forward.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                           C.c_void_p]
            L.chad_mlp_grad_scratch_bytes.restype = C.c_size_t
            L.chad_mlp_grad_scratch_bytes.argtypes = [C.c_int64]
            L.chad_mlp_grad.restype = C.c_int
            L.chad_mlp_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
            L.chad_mlp_grad_async.restype = C.c_int
            L.chad_mlp_grad_async.argtypes = L.chad_mlp_grad.argtypes
            L.chad_mlp_wait.restype = C.c_int
            L.chad_mlp_wait.argtypes = [C.c_void_p]
            L.chad_mlp_prep_scratch_bytes.restype = C.c_size_t
            L.chad_mlp_prep_scratch_bytes.argtypes = []
            L.chad_mlp_feature_norm.restype = C.c_int
            L.chad_mlp_feature_norm.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                                C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
            L.chad_mlp_targets.restype = C.c_int
            L.chad_mlp_targets.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
            L.chad_mlp_gather.restype = C.c_int
            L.chad_mlp_gather.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_uint64, C.c_int64,
                                          C.c_int64, C.c_uint64, C.c_int64, C.c_int64, C.c_void_p,
                                          C.c_void_p, C.c_void_p]
            L.chad_mlp_adam.restype = C.c_int
            L.chad_mlp_adam.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                        C.c_float, C.c_float, C.c_float, C.c_float, C.c_void_p]
            L.chad_headspace_mean_noalloc.restype = C.c_int
            L.chad_headspace_mean_noalloc.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_void_p,
                                                      C.c_void_p, C.c_void_p]
            L.chad_flop_counts.restype = C.c_int
            L.chad_flop_counts.argtypes = [C.c_void_p, C.c_int]
            L.chad_autotune.restype = C.c_int
            L.chad_autotune.argtypes = [C.c_void_p, C.c_double, C.POINTER(C.c_int32), C.c_void_p]
            L.chad_set_kernel_variant.restype = C.c_int
            L.chad_set_kernel_variant.argtypes = [C.c_void_p, C.c_int]
            L.chad_kernel_variant.restype = C.c_int
            L.chad_kernel_variant.argtypes = [C.c_int, C.c_int, C.c_int] + [C.POINTER(C.c_int32)] * 3
            L.chad_eval_model.restype = C.c_int
            L.chad_eval_model.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double,
                                          C.c_void_p, C.c_double, C.c_void_p, C.c_double,
                                          C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_int]
            L.chad_eval_model_split.restype = C.c_int
            L.chad_eval_model_split.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double,
                                                C.c_void_p, C.c_double, C.c_void_p, C.c_double,
                                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                                C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                                C.c_int]
            L.chad_set_diffusion.restype = C.c_int
            L.chad_set_diffusion.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double]
            L.chad_set_positions_by_id.restype = C.c_int
            L.chad_set_positions_by_id.argtypes = [C.c_void_p, C.c_int, C.c_int64, C.c_void_p,
                                                   C.c_void_p, C.c_int]
            L.chad_load_frame.restype = C.c_int
            L.chad_load_frame.argtypes = [C.c_void_p, C.c_int, C.c_char_p,
                                          C.POINTER(C.c_uint64), C.POINTER(C.c_double)]
            L.chad_read_frame.restype = C.c_int
            L.chad_read_frame.argtypes = [C.c_char_p, C.c_int64, C.c_void_p, C.c_void_p,
                                          C.POINTER(C.c_int64), C.POINTER(C.c_uint64),
                                          C.POINTER(C.c_double), C.POINTER(C.c_int32)]
            L.chad_debug_bounds.restype = C.c_int
            L.chad_debug_bounds.argtypes = [C.POINTER(C.c_int32), C.POINTER(C.c_uint32), C.c_int]
            L.chad_get_interval.restype = C.c_int
            L.chad_get_interval.argtypes = [C.c_void_p, C.POINTER(C.c_uint64)]
            L.chad_set_interval.restype = C.c_int
            L.chad_set_interval.argtypes = [C.c_void_p, C.c_uint64]
            L.chad_set_positions.restype = C.c_int
            L.chad_set_positions.argtypes = [C.c_void_p, C.c_int, C.c_int64, C.c_void_p, C.c_int]
            L.chad_diffusion_kernel_times.restype = C.c_int
            L.chad_diffusion_kernel_times.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_double),
                                                      C.POINTER(C.c_double)]
            L.chad_diffusion_info.restype = C.c_int
            L.chad_diffusion_info.argtypes = [C.c_void_p, C.POINTER(C.c_int64),
                                              C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                              C.POINTER(C.c_double)]
            L.chad_probe_numerics.restype = C.c_int
            L.chad_probe_numerics.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                              C.c_void_p]
            L.chad_probe_alu_peak.restype = C.c_int
            L.chad_probe_alu_peak.argtypes = [C.c_int, C.POINTER(C.c_double)]
            _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return ["chad_abi_version", "chad_n_params", "chad_param_name", "chad_last_error",
            "chad_create", "chad_destroy", "chad_load_particles", "chad_set_flow",
            "chad_step", "chad_synchronize", "chad_read_states", "chad_probe_alu_peak",
            "chad_eval_model", "chad_eval_model_split", "chad_probe_numerics", "chad_autotune",
            "chad_flop_counts", "chad_set_diffusion", "chad_diffusion_info",
            "chad_diffusion_kernel_times", "chad_set_positions",
            "chad_set_positions_by_id", "chad_load_frame", "chad_read_frame",
            "chad_get_interval", "chad_set_interval", "chad_debug_bounds",
            "chad_headspace_mean_noalloc", "chad_set_mlp", "chad_mlp_features",
            "chad_mlp_forward", "chad_mlp_grad_scratch_bytes", "chad_mlp_grad", "chad_mlp_adam",
            "chad_kernel_variant", "chad_mlp_grad_async", "chad_mlp_wait",
            "chad_mlp_prep_scratch_bytes", "chad_mlp_feature_norm", "chad_mlp_targets",
            "chad_mlp_gather", "chad_set_kernel_variant"]

MLP_IN, MLP_HID, MLP_OUT = 32, 64, 2
MLP_NPARAM = MLP_HID * MLP_IN + MLP_HID + MLP_HID * MLP_HID + MLP_HID + MLP_OUT * MLP_HID + MLP_OUT


def chad_set_mlp(ctx, params, feat_norm, out_norm):
    L = lib()
    p = np.ascontiguousarray(params, dtype=np.float32)
    fn = np.ascontiguousarray(feat_norm, dtype=np.float32)
    on = np.ascontiguousarray(out_norm, dtype=np.float32)
    assert p.size == MLP_NPARAM and fn.size == 2 * MLP_IN and on.size == 4
    _check(L, ctx, L.chad_set_mlp(ctx, p.ctypes.data, fn.ctypes.data, on.ctypes.data))


def _dev(t):
    """Device pointer of a contiguous torch CUDA tensor."""
    if not (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def chad_mlp_features(y, T, feat_norm, X, stream=None):
    """y [29][ld] f64, T [n] f64, feat_norm [64] f32 -> X [n][32] (int16 holding BF16)."""
    L = lib()
    n = T.shape[0]
    _check(L, None, L.chad_mlp_features(_dev(y), y.shape[1], _dev(T), n, _dev(feat_norm), _dev(X),
                                        stream))


def chad_mlp_forward(X, params, out, stream=None):
    L = lib()
    _check(L, None, L.chad_mlp_forward(_dev(X), X.shape[0], _dev(params), _dev(out), stream))


def chad_mlp_grad(X, Y, params, grad, loss, scratch, stream=None):
    L = lib()
    _check(L, None, L.chad_mlp_grad(_dev(X), _dev(Y), X.shape[0], _dev(params), _dev(grad),
                                    _dev(loss), _dev(scratch), scratch.numel() * scratch.element_size(),
                                    stream))


def chad_mlp_grad_async(X, Y, params, grad, loss, scratch, stream=None):
    L = lib()
    _check(L, None, L.chad_mlp_grad_async(_dev(X), _dev(Y), X.shape[0], _dev(params), _dev(grad),
                                          _dev(loss), _dev(scratch),
                                          scratch.numel() * scratch.element_size(), stream))


def chad_mlp_wait(stream=None):
    L = lib()
    _check(L, None, L.chad_mlp_wait(stream))


def mlp_prep_scratch_bytes():
    return lib().chad_mlp_prep_scratch_bytes()


def chad_mlp_feature_norm(y, T, norm, scratch, stream=None):
    L = lib()
    _check(L, None, L.chad_mlp_feature_norm(_dev(y), y.shape[1], _dev(T), T.shape[0], _dev(norm),
                                            _dev(scratch), scratch.numel() * scratch.element_size(),
                                            stream))


def chad_mlp_targets(S_H, h, Y, out_norm, scratch, stream=None):
    L = lib()
    _check(L, None, L.chad_mlp_targets(_dev(S_H), _dev(h), S_H.shape[0], _dev(Y), _dev(out_norm),
                                       _dev(scratch), scratch.numel() * scratch.element_size(),
                                       stream))


def chad_mlp_gather(X, Y, split_key, offset, n_part, epoch_key, start, count, Xb, Yb, stream=None):
    L = lib()
    _check(L, None, L.chad_mlp_gather(_dev(X), _dev(Y), X.shape[0], int(split_key), int(offset),
                                      int(n_part), int(epoch_key), int(start), int(count),
                                      _dev(Xb), _dev(Yb), stream))


def mlp_grad_scratch_bytes(n):
    return lib().chad_mlp_grad_scratch_bytes(int(n))


def chad_mlp_adam(params, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    L = lib()
    _check(L, None, L.chad_mlp_adam(_dev(params), _dev(grad), _dev(m), _dev(v), int(t), float(lr),
                                    float(beta1), float(beta2), float(eps), stream))


FLOP_KEYS = ["rates_f", "rates_fj", "charge_E", "form_w", "factor", "solve", "jx", "stage",
             "refine", "sm_setup", "sm_update", "sh_final", "scale_j", "jx_twofloat",
             "h2_coeffs", "h2_iter", "mx_fp32_extra", "mx_fp64_extra", "rates_partials",
             "form_w_h2a", "factor_h2a", "solve_h2a"]


def flop_counts() -> dict:
    """Algorithmic operation counts of the integrator's building blocks."""
    L = lib()
    out = np.zeros(len(FLOP_KEYS), dtype=np.int64)
    _check(L, None, L.chad_flop_counts(out.ctypes.data, len(FLOP_KEYS)))
    return dict(zip(FLOP_KEYS, (int(x) for x in out)))


def attempt_flops_h2_mixed() -> dict:
    """FP64 and FP32 operations of one step attempt of the mixed form with
    S_h2 algebraic (kernel form 4), without the Newton iterations of Eq. 7
    (FP64) and Eq. 8 (FP32), which are counted per iteration: FP32 rates with
    J_d and u at the step's start and rates at the two stage points, the
    sparse LU, two sparse solves for q and p2 and two per stage, the
    Sherman-Morrison updates, three Eq. 8 coefficient sets, the rate
    partials recomputed for each of the three refinement residuals and
    their two-float J x, and the two-float stage arithmetic;
    FP64 for the evaluation points and the S_H guesses.  The LU is the one
    without S_h2's row and column (spa)."""
    f = flop_counts()
    f32 = (f["rates_fj"] + 2 * f["rates_f"] + f["form_w_h2a"] + f["factor_h2a"] +
           8 * f["solve_h2a"] +
           f["sm_setup"] + 7 * f["sm_update"] + 3 * f["h2_coeffs"] + 3 * f["jx_twofloat"] +
           3 * f["rates_partials"] + f["mx_fp32_extra"])
    return {"fp64": f["mx_fp64_extra"], "fp32": f32, "fp32_per_h2_iter": f["h2_iter"]}


def attempt_flops(precision: int, h2_algebraic: bool = False) -> dict:
    """FP64 and FP32 operations of one W-method step attempt, without the
    Eq. 7 Newton iterations (counted separately per iteration).  The linear
    algebra is the Sherman-Morrison form: one LU of I - g J_d, one solve for
    q = (I - g J_d)^-1 g u, and per stage one solve plus the rank-1 update;
    the mixed form adds one FP64 residual (J x from the rate partials) and a
    second FP32 solve per stage.  With h2_algebraic (FP64 form only; the
    mixed form's count is attempt_flops_h2_mixed): the LU without S_h2 (spa),
    a fifth solve for the second Sherman-Morrison vector p2 and its update
    of each stage, the Eq. 8 coefficients at the three evaluation points and
    the S_h2 tangent guesses (its Newton iterations counted per iteration,
    h2_iter)."""
    f = flop_counts()
    if precision == PREC_FP64 and h2_algebraic:
        # W_d as in the FP64 form over the 28 states of spa; p2: solve, first
        # level, zh^T p2 and 1 - s (59); zh from the S_h2 row (29 + 24 + 1);
        # per stage the second level (2 x 29 + 1 + 2 x 29); two tangent
        # guesses of the Eq. 8 root (2 x 29 each)
        f64 = (f["rates_fj"] + 2 * f["rates_f"] + f["scale_j"] + (NS - 1) + f["factor_h2a"] +
               5 * f["solve_h2a"] + f["sm_setup"] + 4 * f["sm_update"] + f["stage"] +
               3 * f["h2_coeffs"] + 59 + 54 + 3 * 117 + 2 * 58)
        return {"fp64": f64, "fp32": 0, "fp64_per_h2_iter": f["h2_iter"]}
    if precision == PREC_FP64:
        # W_d: the rate partials scaled by -g before the scatter, plus the diagonal ones
        f64 = (f["rates_fj"] + 2 * f["rates_f"] + f["scale_j"] + NS + f["factor"] +
               4 * f["solve"] + f["sm_setup"] + 3 * f["sm_update"] + f["stage"])
        return {"fp64": f64, "fp32": 0}
    f32_rates = precision == PREC_MIXED_F32RATES
    f64 = 3 * (f["jx"] + f["refine"]) + f["stage"] + (0 if f32_rates else 3 * f["rates_f"])
    f32 = (f["rates_fj"] + f["form_w"] + f["factor"] + 7 * f["solve"] + f["sm_setup"] +
           6 * f["sm_update"] + (2 * f["rates_f"] if f32_rates else 0))
    return {"fp64": f64, "fp32": f32}


def newton_flops() -> int:
    """FP64 operations of one Eq. 7 Newton iteration (evaluation + update)."""
    return flop_counts()["charge_E"] + 2


NUM_VARIANTS = 7  # CHAD_NUM_VARIANTS


def chad_autotune(ctx, dt_coupling_s):
    """Returns (chosen variant, ms per variant)."""
    L = lib()
    ch = C.c_int32(-1)
    ms = np.zeros(NUM_VARIANTS)
    _check(L, ctx, L.chad_autotune(ctx, float(dt_coupling_s), C.byref(ch), ms.ctypes.data))
    return ch.value, ms


def chad_set_kernel_variant(ctx, v) -> None:
    L = lib()
    _check(L, ctx, L.chad_set_kernel_variant(ctx, int(v)))


def kernel_variant(precision, h2_algebraic, v) -> dict:
    """Launch shape of integrator kernel variant v (chad_kernel_variant)."""
    L = lib()
    t, m, w = C.c_int32(), C.c_int32(), C.c_int32()
    _check(L, None, L.chad_kernel_variant(int(precision), int(bool(h2_algebraic)), int(v),
                                          C.byref(t), C.byref(m), C.byref(w)))
    return {"threads": t.value, "min_blocks": m.value, "w_shared": bool(w.value),
            "registers_max": min(255, 65536 // (t.value * m.value))}


def eval_model(params, T, y, y_in=None, D=0.0, V_liq=3400.0, V_gas=300.0, SH_guess=1e-7,
               on_device=False):
    """(f, J, S_H) of the library's model for one particle (host or GPU)."""
    L = lib()
    p = np.ascontiguousarray(params, dtype=np.float64)
    yy = np.ascontiguousarray(y, dtype=np.float64)
    yi = None if y_in is None else np.ascontiguousarray(y_in, dtype=np.float64)
    f = np.zeros(NS)
    J = np.zeros((NS, NS))
    SH = C.c_double(0.0)
    code = L.chad_eval_model(p.ctypes.data, float(V_liq), float(V_gas), float(D),
                             None if yi is None else yi.ctypes.data, float(T), yy.ctypes.data,
                             float(SH_guess), f.ctypes.data, J.ctypes.data, C.byref(SH),
                             1 if on_device else 0)
    if code not in (0, 5):
        raise ChadError(code, "chad_eval_model failed")
    return f, J, SH.value


def eval_model_split(params, T, y, y_in=None, D=0.0, V_liq=3400.0, V_gas=300.0, SH_guess=1e-7,
                     on_device=False, x=None):
    """(f, J_d, u, v, S_H) of the library's model for one particle: the
    Jacobian split as J = J_d + u v^T (S_H held fixed in J_d, u = df/dS_H,
    v = dS_H/dy).  With a direction x, returns (f, J_d, u, v, S_H, Jx) where
    Jx = J x is formed from the rate partials as in the mixed refinement."""
    L = lib()
    p = np.ascontiguousarray(params, dtype=np.float64)
    yy = np.ascontiguousarray(y, dtype=np.float64)
    yi = None if y_in is None else np.ascontiguousarray(y_in, dtype=np.float64)
    f = np.zeros(NS)
    Jd = np.zeros((NS, NS))
    u = np.zeros(NS)
    v = np.zeros(NS)
    SH = C.c_double(0.0)
    xx = None if x is None else np.ascontiguousarray(x, dtype=np.float64)
    Jx = None if x is None else np.zeros(NS)
    code = L.chad_eval_model_split(p.ctypes.data, float(V_liq), float(V_gas), float(D),
                                   None if yi is None else yi.ctypes.data, float(T),
                                   yy.ctypes.data, float(SH_guess),
                                   None if xx is None else xx.ctypes.data, f.ctypes.data,
                                   Jd.ctypes.data, u.ctypes.data, v.ctypes.data,
                                   None if Jx is None else Jx.ctypes.data, C.byref(SH),
                                   1 if on_device else 0)
    if code not in (0, 5):
        raise ChadError(code, "chad_eval_model_split failed")
    if x is None:
        return f, Jd, u, v, SH.value
    return f, Jd, u, v, SH.value, Jx


def probe_numerics(x):
    """(narrow, widen, recip) of the kernels' conversion and reciprocal
    helpers applied to x on the current GPU."""
    L = lib()
    xx = np.ascontiguousarray(x, dtype=np.float64)
    n = xx.size
    nar = np.zeros(n, dtype=np.float32)
    wid = np.zeros(n)
    rec = np.zeros(n)
    _check(L, None, L.chad_probe_numerics(xx.ctypes.data, n, nar.ctypes.data, wid.ctypes.data,
                                          rec.ctypes.data))
    return nar, wid, rec


def probe_alu_peak(fp64: bool) -> float:
    """Measured FMA throughput (TFLOP/s) of the current GPU."""
    L = lib()
    v = C.c_double(0.0)
    _check(L, None, L.chad_probe_alu_peak(1 if fp64 else 0, C.byref(v)))
    return v.value


def param_names() -> list[str]:
    L = lib()
    return [L.chad_param_name(i).decode() for i in range(L.chad_n_params())]


def _ptr(a):
    """(pointer, mem) of a numpy array or a torch CUDA tensor (or (None, None))."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data, MEM_HOST
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), (MEM_DEVICE if a.is_cuda else MEM_HOST)
    raise TypeError(f"unsupported buffer type {type(a)}")


def _check(L, ctx, code):
    if code != 0:
        raise ChadError(code, L.chad_last_error(ctx).decode())


# ---------------------------------------------------------------- raw ABI calls
def chad_create(cfg: chad_config) -> C.c_void_p:
    L = lib()
    ctx = C.c_void_p()
    _check(L, None, L.chad_create(C.byref(cfg), C.byref(ctx)))
    return ctx


def chad_destroy(ctx) -> None:
    lib().chad_destroy(ctx)


def chad_load_particles(ctx, digester, n, pos, y, T=None, S_H=None, h=None) -> None:
    L = lib()
    ptrs = [_ptr(a) for a in (pos, y, T, S_H, h)]
    mems = {m for _, m in ptrs if m is not None}
    if len(mems) > 1:
        raise ValueError("all buffers of one call must be host or all device")
    mem = mems.pop() if mems else MEM_HOST
    _check(L, ctx, L.chad_load_particles(ctx, int(digester), int(n), *[p for p, _ in ptrs], mem))


def chad_debug_bounds(reset=False):
    """(enabled, status bits) of the bounds-check build; (0, 0) in the normal one."""
    L = lib()
    en, st = C.c_int32(), C.c_uint32()
    code = L.chad_debug_bounds(C.byref(en), C.byref(st), int(bool(reset)))
    if code != 0:
        raise ChadError(code, "reading the bounds-check status failed")
    return en.value, st.value


def chad_get_interval(ctx) -> int:
    """The coupling-interval index that keys the advection noise."""
    L = lib()
    v = C.c_uint64()
    _check(L, ctx, L.chad_get_interval(ctx, C.byref(v)))
    return v.value


def chad_set_interval(ctx, interval) -> None:
    L = lib()
    _check(L, ctx, L.chad_set_interval(ctx, int(interval)))


def chad_set_positions(ctx, digester, n, pos) -> None:
    """Replace one digester's positions ([3][n], numpy or CUDA tensor), keeping its states."""
    L = lib()
    p, mem = _ptr(pos)
    _check(L, ctx, L.chad_set_positions(ctx, int(digester), int(n), p, MEM_HOST if mem is None else mem))


def chad_set_positions_by_id(ctx, digester, n, pos, ids) -> None:
    """Positions [3][n] in frame order with the particle id [n] (int64) of each entry."""
    L = lib()
    ptrs = [_ptr(a) for a in (pos, ids)]
    mems = {m for _, m in ptrs if m is not None}
    if len(mems) > 1:
        raise ValueError("pos and ids must both be host or both device")
    mem = mems.pop() if mems else MEM_HOST
    _check(L, ctx, L.chad_set_positions_by_id(ctx, int(digester), int(n), ptrs[0][0], ptrs[1][0], mem))


def chad_load_frame(ctx, digester, path):
    """Load a frame file into one digester's positions; returns (step, time_s)."""
    L = lib()
    st, t = C.c_uint64(), C.c_double()
    _check(L, ctx, L.chad_load_frame(ctx, int(digester), os.fsencode(path), C.byref(st), C.byref(t)))
    return st.value, t.value


def chad_read_frame(path):
    """Host read of a frame file through the library (no GPU): dict with n,
    step, time_s, pos [3][n] and id [n] (None without ids)."""
    L = lib()
    n, st, t, hid = C.c_int64(), C.c_uint64(), C.c_double(), C.c_int32()
    fp = os.fsencode(path)
    if L.chad_read_frame(fp, 0, None, None, C.byref(n), C.byref(st), C.byref(t), C.byref(hid)) != 0:
        raise ChadError(1, f"cannot read frame {path}")
    pos = np.empty((3, n.value))
    ids = np.empty(n.value, dtype=np.int64) if hid.value else None
    code = L.chad_read_frame(fp, n.value, pos.ctypes.data, None if ids is None else ids.ctypes.data,
                             None, None, None, None)
    if code != 0:
        raise ChadError(code, f"cannot read frame {path}")
    return dict(n=n.value, step=st.value, time_s=t.value, pos=pos, id=ids)


def chad_set_flow(ctx, digester, flow: chad_flow) -> None:
    L = lib()
    _check(L, ctx, L.chad_set_flow(ctx, int(digester), C.byref(flow)))


def chad_set_diffusion(ctx, digester, D, h) -> None:
    L = lib()
    _check(L, ctx, L.chad_set_diffusion(ctx, int(digester), float(D), float(h)))


def chad_diffusion_info(ctx) -> dict:
    """The last interval's diffusion plan: reserved entries, substeps, capped, S_max."""
    L = lib()
    e, n, c, s = C.c_int64(), C.c_int32(), C.c_int32(), C.c_double()
    _check(L, ctx, L.chad_diffusion_info(ctx, C.byref(e), C.byref(n), C.byref(c), C.byref(s)))
    return dict(entries=e.value, n_sub=n.value, capped=c.value, s_max=s.value)


def chad_diffusion_kernel_times(ctx, reps=1):
    """Mean ms per launch of the diffusion rows and substep kernels (re-run on scratch)."""
    L = lib()
    r, s = C.c_double(), C.c_double()
    _check(L, ctx, L.chad_diffusion_kernel_times(ctx, int(reps), C.byref(r), C.byref(s)))
    return r.value, s.value


def chad_step(ctx, dt_coupling_s, n_intervals) -> None:
    L = lib()
    _check(L, ctx, L.chad_step(ctx, float(dt_coupling_s), int(n_intervals)))


def chad_synchronize(ctx) -> int:
    return lib().chad_synchronize(ctx)


def chad_read_states(ctx, digester, y=None, pos=None, S_H=None, h=None, status=None,
                     stats: chad_stats | None = None) -> int:
    """Returns the chad_status code (CHAD_E_PARTICLE is not raised)."""
    L = lib()
    ptrs = [_ptr(a) for a in (y, pos, S_H, h, status)]
    mems = {m for _, m in ptrs if m is not None}
    if len(mems) > 1:
        raise ValueError("all buffers of one call must be host or all device")
    mem = mems.pop() if mems else MEM_HOST
    code = L.chad_read_states(ctx, int(digester), *[p for p, _ in ptrs],
                              C.byref(stats) if stats is not None else None, mem)
    if code not in (0, 5):
        _check(L, ctx, code)
    return code


# ---------------------------------------------------------------- population helper
class Simulator:
    """Owns one context for a seeded Population (inputs.Population)."""

    def __init__(self, pop: I.Population, precision=PREC_FP64, rtol=1e-6, atol=None,
                 max_steps=100000, max_newton=50, fixed_substeps=0, stream=None,
                 headspace=None, learned=0, h2_algebraic=False, diffusion=None):
        self.pop = pop
        nd = len(pop.digesters)
        self._keep = []
        self._T = None

        def arr(x, dt=np.float64):
            a = np.ascontiguousarray(x, dtype=dt)
            self._keep.append(a)
            return a

        counts = arr([d.n for d in pop.digesters], np.int64)
        V_liq = arr([d.V_liq for d in pop.digesters])
        V_gas = arr([d.V_gas for d in pop.digesters])
        params = arr(np.stack([d.params for d in pop.digesters]))
        D_u = arr([d.D for d in pop.digesters])
        y_in = arr(np.stack([d.y_in for d in pop.digesters]))
        atol = arr(I.atol_vector() if atol is None else atol)
        if headspace is None:
            headspace = HEADSPACE_SHARED if pop.shared_headspace else HEADSPACE_PARTICLE
        cfg = chad_config()
        cfg.n_digesters = nd
        cfg.n_particles = counts.ctypes.data_as(_i64p)
        cfg.V_liq = V_liq.ctypes.data_as(_dp)
        cfg.V_gas = V_gas.ctypes.data_as(_dp)
        cfg.params = params.ctypes.data_as(_dp)
        cfg.D_uniform = D_u.ctypes.data_as(_dp)
        cfg.y_in = y_in.ctypes.data_as(_dp)
        cfg.precision = precision
        cfg.learned = int(learned)
        cfg.headspace = headspace
        cfg.rtol = rtol
        cfg.atol = atol.ctypes.data_as(_dp)
        cfg.max_steps_per_interval = max_steps
        cfg.max_newton_iters = max_newton
        cfg.fixed_substeps = fixed_substeps
        cfg.cuda_stream = stream
        cfg.h2_algebraic = int(bool(h2_algebraic))
        self.ctx = chad_create(cfg)
        self.offsets = pop.offsets
        for d, dg in enumerate(pop.digesters):
            if dg.flow is not None:
                f = dg.flow
                yin = arr(f["y_in"])
                fl = chad_flow(1, f["U"], f["R"], f["H"], f["sigma"], f["slab_zmin"], f["q_in"],
                               yin.ctypes.data_as(_dp), f["seed"])
                chad_set_flow(self.ctx, d, fl)
        if diffusion is not None:  # (D m^2/s, h m) for every digester with flow, or one per digester
            per = diffusion if isinstance(diffusion, list) else [diffusion] * nd
            for d, dg in enumerate(pop.digesters):
                if dg.flow is not None and per[d] is not None:
                    chad_set_diffusion(self.ctx, d, per[d][0], per[d][1])

    def load(self, y=None, pos=None, T=None, S_H=None, h=None):
        """Load every digester from host arrays (SoA over the whole population)."""
        pop = self.pop
        y = pop.y if y is None else y
        pos = pop.pos if pos is None else pos
        T = pop.T if T is None else T
        self._T = np.asarray(T)
        for d, dg in enumerate(pop.digesters):
            a, b = self.offsets[d], self.offsets[d + 1]
            sl = lambda x: None if x is None else np.ascontiguousarray(x[..., a:b])
            chad_load_particles(self.ctx, d, b - a, sl(pos), sl(y), sl(T), sl(S_H), sl(h))

    @classmethod
    def from_config(cls, path, particles=None, **overrides):
        """(Simulator, coupling interval in s, intervals) for a run
        configuration (runconfig; the bundled ones are configs/c1 .. c5.json).
        A learned configuration still needs chad_set_mlp before chad_step."""
        from . import runconfig as RC
        pop, kw, dt, k = RC.load(path, particles)
        kw.update(overrides)
        return cls(pop, **kw), dt, k

    def checkpoint(self, path):
        """Save what a bitwise resume needs: y, pos, S_H, h (every digester),
        the temperatures and the interval index, as one .npz file."""
        out = self.read()
        T = np.ascontiguousarray(self.pop.T if self._T is None else self._T)
        np.savez(path, y=out["y"], pos=out["pos"], S_H=out["S_H"], h=out["h"], T=T,
                 interval=np.uint64(chad_get_interval(self.ctx)))

    def restore(self, path):
        """Load a checkpoint written by checkpoint() into this context."""
        with np.load(path) as z:
            self.load(y=z["y"], pos=z["pos"], T=z["T"], S_H=z["S_H"], h=z["h"])
            chad_set_interval(self.ctx, int(z["interval"]))

    def set_positions(self, pos):
        """New positions [3][N] for every digester (an external CFD's coupling step)."""
        for d in range(len(self.pop.digesters)):
            a, b = self.offsets[d], self.offsets[d + 1]
            chad_set_positions(self.ctx, d, b - a, np.ascontiguousarray(pos[:, a:b], dtype=np.float64))

    def step(self, dt_coupling_s, n_intervals):
        chad_step(self.ctx, dt_coupling_s, n_intervals)

    def read(self):
        """Host copies of y, pos, S_H, h, status and the counters (dict)."""
        N = self.pop.n
        out = dict(y=np.zeros((NS, N)), pos=np.zeros((3, N)), S_H=np.zeros(N), h=np.zeros(N),
                   status=np.zeros(N, dtype=np.int32))
        total = None
        for d in range(len(self.pop.digesters)):
            a, b = self.offsets[d], self.offsets[d + 1]
            n = b - a
            yy, pp = np.zeros((NS, n)), np.zeros((3, n))
            sh, hh, st = np.zeros(n), np.zeros(n), np.zeros(n, dtype=np.int32)
            stats = chad_stats()
            chad_read_states(self.ctx, d, yy, pp, sh, hh, st, stats if d == 0 else None)
            if d == 0:
                total = stats.as_dict()
            out["y"][:, a:b], out["pos"][:, a:b] = yy, pp
            out["S_H"][a:b], out["h"][a:b], out["status"][a:b] = sh, hh, st
        out["stats"] = total
        return out

    def close(self):
        if self.ctx:
            chad_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
