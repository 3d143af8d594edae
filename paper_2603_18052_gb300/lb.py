"""ctypes binding of liblb (the C ABI declared in include/lb.h).

Argument marshalling only: every function takes torch tensors that already
live on the context's CUDA device, checks dtype, shape and contiguity, and
passes their data pointers and the current CUDA stream to the C function of
the same name.  All arithmetic runs in the library's kernels; there is no
fallback path, and a missing or unloadable library raises immediately.
"""

import ctypes
import os

import torch

from . import _build

LB_FP64, LB_FP32, LB_BF16X3, LB_FP64_HERMITIAN, LB_FP32_HERMITIAN, LB_FP64_SLICED = 0, 1, 2, 3, 4, 5
PRECISIONS = {"fp64": LB_FP64, "fp32": LB_FP32, "bf16x3": LB_BF16X3, "fp64_hermitian": LB_FP64_HERMITIAN,
              "fp32_hermitian": LB_FP32_HERMITIAN, "fp64_sliced": LB_FP64_SLICED}

_STATUS = {
    0: "LB_OK",
    1: "LB_EINVAL",
    2: "LB_ENODEV",
    3: "LB_ENOMEM",
    4: "LB_ECUDA",
    5: "LB_ENONFINITE",
    6: "LB_ESINGULAR",
    7: "LB_ETIMEOUT",
    8: "LB_EUNSUPPORTED",
}

EXPORTED = (
    "lb_version",
    "lb_status_str",
    "lb_create",
    "lb_destroy",
    "lb_sync_status",
    "lb_workspace_bytes",
    "lb_launch_count",
    "lb_set_max_squarings",
    "lb_autotune",
    "lb_set_stage_timing",
    "lb_stage_times",
    "lb_kernel_times",
    "lb_assemble",
    "lb_expm_pade",
    "lb_propagate_batch",
    "lb_gemm_f64_sliced",
    "lb_grape_grad",
    "lb_grape_grad_batch",
    "lb_propagate_batch_static",
    "lb_run_instances",
    "lb_mlp_forward",
    "lb_mlp_backward",
    "lb_mse_loss_grad",
    "lb_adam_step",
    "lb_adam_step_f64",
    "lb_selftest_wait_timeout",
    "lb_expm_frechet",
    "lb_control_update",
    "lb_expmv",
    "lb_expmv_hermitian",
    "lb_fixed_quantize",
    "lb_fixed_dequantize",
    "lb_propagate_fixed",
    "lb_propagate_resident",
    "lb_propagate_host",
    "lb_probe_launch",
    "lb_probe_copy",
    "lb_probe_read",
    "lb_probe_alloc",
    "lb_probe_dfma",
    "lb_probe_ffma",
    "lb_probe_dmma",
    "lb_probe_bf16_tc",
)


class Instance(ctypes.Structure):
    """lb_instance: one problem of lb_run_instances (device pointers)."""

    _fields_ = [("d", ctypes.c_int), ("nslices", ctypes.c_int), ("steps_per_slice", ctypes.c_int),
                ("B", ctypes.c_int), ("Lbase", ctypes.c_void_p), ("Ldrv", ctypes.c_void_p),
                ("u", ctypes.c_void_p), ("states", ctypes.c_void_p)]


class LBError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        self.name = _STATUS.get(status, "?")
        super().__init__("%s failed: %s" % (what, lib().lb_status_str(status).decode()))


_lib = None


def lib_path():
    return _build.LIB


def lib():
    """Load liblb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError("liblb.so is not built (%s); run __graft_entry__.build()" % path)
    L = ctypes.CDLL(path)
    vp, ip, dp, i32, f64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.lb_version.restype = i32
    L.lb_version.argtypes = []
    L.lb_status_str.restype = ctypes.c_char_p
    L.lb_status_str.argtypes = [i32]
    L.lb_create.restype = i32
    L.lb_create.argtypes = [ctypes.POINTER(vp), i32, i32, i32, i32]
    L.lb_destroy.restype = i32
    L.lb_destroy.argtypes = [vp]
    L.lb_sync_status.restype = i32
    L.lb_sync_status.argtypes = [vp, vp]
    L.lb_workspace_bytes.restype = ctypes.c_ulonglong
    L.lb_workspace_bytes.argtypes = [vp]
    L.lb_autotune.restype = i32
    L.lb_autotune.argtypes = [vp, i32, i32, i32, ctypes.POINTER(ctypes.c_int), vp]
    L.lb_set_max_squarings.restype = i32
    L.lb_set_max_squarings.argtypes = [vp, i32]
    L.lb_launch_count.restype = ctypes.c_ulonglong
    L.lb_launch_count.argtypes = []
    L.lb_set_stage_timing.restype = i32
    L.lb_set_stage_timing.argtypes = [vp, i32]
    L.lb_stage_times.restype = i32
    L.lb_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
    L.lb_kernel_times.restype = i32
    L.lb_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_longlong)]
    L.lb_assemble.restype = i32
    L.lb_assemble.argtypes = [vp, i32, vp, i32, vp, vp, vp]
    L.lb_expm_pade.restype = i32
    L.lb_expm_pade.argtypes = [vp, i32, i32, vp, vp, vp, f64, i32, vp, vp, vp]
    L.lb_propagate_batch.restype = i32
    L.lb_propagate_batch.argtypes = [vp, i32, i32, vp, i32, i32, vp, i32, i32, vp]
    L.lb_gemm_f64_sliced.restype = i32
    i64 = ctypes.c_longlong
    L.lb_gemm_f64_sliced.argtypes = [vp, i32, i32, i32, i32, vp, i64, i64, vp, i64, i64, vp, i64, i64, f64, f64, vp]
    L.lb_propagate_batch_static.restype = i32
    L.lb_propagate_batch_static.argtypes = [i32, i32, vp, i32, i32, vp, vp]
    L.lb_expm_frechet.restype = i32
    L.lb_expm_frechet.argtypes = [vp, i32, i32, vp, vp, vp, f64, vp, vp, vp]
    L.lb_control_update.restype = i32
    L.lb_control_update.argtypes = [i32, i32, vp, vp, vp, vp, vp]
    L.lb_selftest_wait_timeout.restype = i32
    L.lb_selftest_wait_timeout.argtypes = [vp, ctypes.c_longlong, vp]
    L.lb_run_instances.restype = i32
    L.lb_run_instances.argtypes = [vp, ctypes.POINTER(Instance), i32, f64, i32, i32, vp]
    f32 = ctypes.c_float
    ll = ctypes.c_longlong
    L.lb_mlp_forward.restype = i32
    L.lb_mlp_forward.argtypes = [i32, ctypes.POINTER(ctypes.c_int), i32, vp, vp, vp, vp, vp]
    L.lb_mlp_backward.restype = i32
    L.lb_mlp_backward.argtypes = [i32, ctypes.POINTER(ctypes.c_int), i32, vp, vp, vp, vp, vp, vp, vp, vp]
    L.lb_mse_loss_grad.restype = i32
    L.lb_mse_loss_grad.argtypes = [ll, vp, vp, vp, vp, vp]
    L.lb_adam_step.restype = i32
    L.lb_adam_step.argtypes = [ll, vp, vp, vp, vp, vp, f32, f32, f32, f32, i32, vp]
    L.lb_adam_step_f64.restype = i32
    L.lb_adam_step_f64.argtypes = [ll, vp, vp, vp, vp, f64, f64, f64, f64, i32, i32, vp]
    L.lb_grape_grad.restype = i32
    L.lb_grape_grad.argtypes = [vp, i32, i32, vp, vp, vp, f64, i32, i32, vp, vp, vp, vp, vp]
    L.lb_grape_grad_batch.restype = i32
    L.lb_grape_grad_batch.argtypes = [vp, i32, i32, i32, vp, ll, vp, vp, f64, i32, i32, vp, vp, i32, vp, vp, vp]
    L.lb_expmv.restype = i32
    L.lb_expmv.argtypes = [vp, i32, i32, vp, vp, vp, f64, i32, vp, ctypes.POINTER(ctypes.c_int), vp]
    L.lb_expmv_hermitian.restype = i32
    L.lb_expmv_hermitian.argtypes = [vp, i32, i32, vp, vp, vp, f64, i32, vp, ctypes.POINTER(ctypes.c_int), vp]
    L.lb_fixed_quantize.restype = i32
    L.lb_fixed_quantize.argtypes = [i32, ll, vp, vp, vp]
    L.lb_fixed_dequantize.restype = i32
    L.lb_fixed_dequantize.argtypes = [i32, ll, vp, vp, vp]
    L.lb_propagate_fixed.restype = i32
    L.lb_propagate_fixed.argtypes = [i32, i32, vp, i32, i32, vp, vp]
    L.lb_propagate_resident.restype = i32
    L.lb_propagate_resident.argtypes = [vp, i32, vp, i32, vp, vp]
    L.lb_propagate_host.restype = i32
    L.lb_propagate_host.argtypes = [vp, i32, vp, i32, vp, vp]
    L.lb_probe_launch.restype = i32
    L.lb_probe_launch.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_double), vp]
    L.lb_probe_copy.restype = i32
    L.lb_probe_copy.argtypes = [vp, vp, ll, i32, i32, ctypes.POINTER(ctypes.c_double), vp]
    L.lb_probe_alloc.restype = i32
    L.lb_probe_alloc.argtypes = [ll, i32, ctypes.POINTER(ctypes.c_double)]
    L.lb_probe_read.restype = i32
    L.lb_probe_read.argtypes = [vp, ll, i32, vp, vp]
    for name in ("lb_probe_dfma", "lb_probe_ffma", "lb_probe_dmma", "lb_probe_bf16_tc"):
        getattr(L, name).restype = i32
        getattr(L, name).argtypes = [ctypes.POINTER(ctypes.c_double), vp]
    del ip, dp
    _lib = L
    return L


def _check(status, what):
    if status != 0:
        raise LBError(status, what)


# The raw handle of the current stream without building a Stream object
# (a few microseconds per call otherwise, which shows in one-step calls).
_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream(stream):
    if stream is None:
        if _raw_stream is not None:
            return _raw_stream(torch.cuda.current_device())
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t, dtype, what, shape=None, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError("%s must not be None" % what)
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_cuda or not t.is_contiguous():
        raise ValueError("%s must be a contiguous CUDA %s tensor" % (what, dtype))
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (what, tuple(t.shape), tuple(shape)))
    return t.data_ptr()


class Context:
    """An lb_ctx bound to one CUDA device, owning the library's scratch."""

    def __init__(self, device=0, max_n=729, max_batch=1024, max_slices=200):
        L = lib()
        h = ctypes.c_void_p()
        if isinstance(device, torch.device):
            device = device.index or 0
        _check(L.lb_create(ctypes.byref(h), int(device), int(max_n), int(max_batch), int(max_slices)),
               "lb_create")
        self.handle = h
        self.device = int(device)
        self.max_n, self.max_batch, self.max_slices = int(max_n), int(max_batch), int(max_slices)

    def close(self):
        if getattr(self, "handle", None):
            lib().lb_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def workspace_bytes(self):
        return int(lib().lb_workspace_bytes(self.handle))


def lb_autotune(ctx, n, nslices, B, stream=None):
    """Tune GEMM tiles for the launch shapes of an n-sized build over nslices
    slices and a B-state propagation step; returns the number of tuned shapes."""
    k = ctypes.c_int(0)
    _check(lib().lb_autotune(ctx.handle, int(n), int(nslices), int(B), ctypes.byref(k), _stream(stream)),
           "lb_autotune")
    return int(k.value)


def lb_set_max_squarings(ctx, bound):
    """Fixed number of squaring rounds (>= 0) so that builds can be captured
    in a CUDA graph; -1 restores the host read of the squaring count."""
    _check(lib().lb_set_max_squarings(ctx.handle, int(bound)), "lb_set_max_squarings")


def lb_launch_count():
    """Kernel launches issued by the library so far in this process."""
    return int(lib().lb_launch_count())


def lb_set_stage_timing(ctx, enable=True):
    """Clear the stage totals and switch the per-stage CUDA events of
    lb_expm_pade on or off."""
    _check(lib().lb_set_stage_timing(ctx.handle, int(bool(enable))), "lb_set_stage_timing")


STAGES = ("prepare", "pade_products", "lu_solve", "squarings", "check")


def lb_kernel_times(ctx):
    """Summed time (ms), digit-product FLOPs and launches of the sliced
    FP64 product kernel since the last lb_set_stage_timing."""
    ms = ctypes.c_double(0.0)
    fl = ctypes.c_double(0.0)
    nl = ctypes.c_longlong(0)
    _check(lib().lb_kernel_times(ctx.handle, ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(nl)), "lb_kernel_times")
    return ms.value, fl.value, int(nl.value)


def lb_stage_times(ctx):
    """Stage totals (ms) since the last lb_set_stage_timing, and the number
    of slice chunks they cover."""
    out = (ctypes.c_double * 5)()
    chunks = ctypes.c_longlong(0)
    _check(lib().lb_stage_times(ctx.handle, out, ctypes.byref(chunks)), "lb_stage_times")
    return dict(zip(STAGES, list(out))), int(chunks.value)


def lb_sync_status(ctx, stream=None):
    """Synchronise the stream and raise on a device-side error."""
    _check(lib().lb_sync_status(ctx.handle, _stream(stream)), "lb_sync_status")


def lb_assemble(ctx, H, Ls, L_out, stream=None):
    """L_out (n x n) = vectorised Lindbladian of H (d x d) and the jump
    operators Ls (K x d x d, or None)."""
    d = H.shape[0]
    K = 0 if Ls is None else Ls.shape[0]
    c128 = torch.complex128
    _check(lib().lb_assemble(ctx.handle, d, _ptr(H, c128, "H", (d, d)), K,
                             _ptr(Ls, c128, "Ls", (K, d, d)) if K else None,
                             _ptr(L_out, c128, "L_out", (d * d, d * d)), _stream(stream)),
           "lb_assemble")


def lb_expm_pade(ctx, Lbase, Ldrv, u, dt, P_out, prec="fp64", s_out=None, stream=None):
    """P_out[s] = exp((Lbase + u[s] Ldrv) dt); with Ldrv None, Lbase holds
    one generator per slice."""
    c128 = torch.complex128
    S, n = P_out.shape[0], P_out.shape[1]
    if Ldrv is None:
        pb = _ptr(Lbase, c128, "Lbase", (S, n, n))
        pd, pu = None, None
    else:
        pb = _ptr(Lbase, c128, "Lbase", (n, n))
        pd = _ptr(Ldrv, c128, "Ldrv", (n, n))
        pu = _ptr(u, torch.float64, "u", (S,))
    ps = _ptr(s_out, torch.int32, "s_out", (S,), allow_none=True)
    _check(lib().lb_expm_pade(ctx.handle, n, S, pb, pd, pu, float(dt), PRECISIONS.get(prec, prec),
                              _ptr(P_out, c128, "P_out", (S, n, n)), ps, _stream(stream)),
           "lb_expm_pade")


def lb_propagate_batch(ctx, P, states, steps_per_slice=1, prec="fp64", renorm_trace=False, stream=None):
    """states (B x n) <- chain of P[t // steps_per_slice] applied to every row."""
    c128 = torch.complex128
    S, n = P.shape[0], P.shape[1]
    B = states.shape[0]
    _check(lib().lb_propagate_batch(ctx.handle, n, S, _ptr(P, c128, "P", (S, n, n)), int(steps_per_slice), B,
                                    _ptr(states, c128, "states", (B, n)), PRECISIONS.get(prec, prec),
                                    int(bool(renorm_trace)), _stream(stream)),
           "lb_propagate_batch")


def lb_gemm_f64_sliced(ctx, A, B, C, alpha=1.0, beta=0.0, stream=None):
    """C = alpha A B + beta C for float64 (batch, M, K) x (batch, K, N) ->
    (batch, M, N) (or 2-D), row-major contiguous, via exact BF16 slices."""
    f = torch.float64
    A3, B3, C3 = (x if x.dim() == 3 else x.unsqueeze(0) for x in (A, B, C))
    nb, M, K = A3.shape
    N = B3.shape[2]
    _check(lib().lb_gemm_f64_sliced(ctx.handle, M, N, K, nb, _ptr(A3, f, "A", (nb, M, K)), K, M * K,
                                    _ptr(B3, f, "B", (nb, K, N)), N, K * N, _ptr(C3, f, "C", (nb, M, N)), N, M * N,
                                    float(alpha), float(beta), _stream(stream)),
           "lb_gemm_f64_sliced")


def lb_grape_grad(ctx, Lbase, Ldrv, u, dt, steps_per_slice, X0, Xtarget, fidelity_out, grad_out, stream=None):
    """Fidelity and gradient of a piecewise-constant control."""
    c128 = torch.complex128
    n = Lbase.shape[0]
    S = u.shape[0]
    B = X0.shape[0]
    _check(lib().lb_grape_grad(ctx.handle, n, S, _ptr(Lbase, c128, "Lbase", (n, n)),
                               _ptr(Ldrv, c128, "Ldrv", (n, n)), _ptr(u, torch.float64, "u", (S,)), float(dt),
                               int(steps_per_slice), B, _ptr(X0, c128, "X0", (B, n)),
                               _ptr(Xtarget, c128, "Xtarget", (B, n)),
                               _ptr(fidelity_out, torch.float64, "fidelity_out", (1,)),
                               _ptr(grad_out, torch.float64, "grad_out", (S,)), _stream(stream)),
           "lb_grape_grad")


def lb_grape_grad_batch(ctx, Lbase, Ldrv, u, dt, steps_per_slice, X0, Xtarget, fidelity_out, grad_out, prec="fp64",
                        stream=None):
    """K problems at once: Lbase (n, n) shared or (K, n, n) per problem, Ldrv
    (n, n) shared, u (K, S), X0 / Xtarget (K, B, n); fidelity_out (K,),
    grad_out (K, S)."""
    c128 = torch.complex128
    K, S = u.shape
    n = Ldrv.shape[0]
    B = X0.shape[1]
    if Lbase.dim() == 2:
        lbp, stride = _ptr(Lbase, c128, "Lbase", (n, n)), 0
    else:
        lbp, stride = _ptr(Lbase, c128, "Lbase", (K, n, n)), n * n
    _check(lib().lb_grape_grad_batch(ctx.handle, n, K, S, lbp, stride, _ptr(Ldrv, c128, "Ldrv", (n, n)),
                                     _ptr(u, torch.float64, "u", (K, S)), float(dt), int(steps_per_slice), B,
                                     _ptr(X0, c128, "X0", (K, B, n)), _ptr(Xtarget, c128, "Xtarget", (K, B, n)),
                                     PRECISIONS.get(prec, prec),
                                     _ptr(fidelity_out, torch.float64, "fidelity_out", (K,)),
                                     _ptr(grad_out, torch.float64, "grad_out", (K, S)), _stream(stream)),
           "lb_grape_grad_batch")


def lb_expm_frechet(ctx, Lbase, Ldrv, u, dt, P_out, dP_out, stream=None):
    """P_out[s] = exp((Lbase + u[s] Ldrv) dt) and dP_out[s] = its derivative
    with respect to u[s] (FP64; contexts with max_n <= 81)."""
    c128 = torch.complex128
    n = Lbase.shape[0]
    S = u.shape[0]
    _check(lib().lb_expm_frechet(ctx.handle, n, S, _ptr(Lbase, c128, "Lbase", (n, n)), _ptr(Ldrv, c128, "Ldrv", (n, n)),
                                 _ptr(u, torch.float64, "u", (S,)), float(dt), _ptr(P_out, c128, "P_out", (S, n, n)),
                                 _ptr(dP_out, c128, "dP_out", (S, n, n)), _stream(stream)), "lb_expm_frechet")


def lb_control_update(P, dP, delta, P_out, stream=None):
    """P_out[s] = P[s] + delta[s] dP[s]: propagators for nearby controls."""
    c128 = torch.complex128
    S, n = P.shape[0], P.shape[1]
    _check(lib().lb_control_update(n, S, _ptr(P, c128, "P", (S, n, n)), _ptr(dP, c128, "dP", (S, n, n)),
                                   _ptr(delta, torch.float64, "delta", (S,)), _ptr(P_out, c128, "P_out", (S, n, n)),
                                   _stream(stream)), "lb_control_update")


def lb_selftest_wait_timeout(ctx, cycles=2_000_000, stream=None):
    """Queue a bounded wait that runs out; the next lb_sync_status raises
    LBError with name LB_ETIMEOUT."""
    _check(lib().lb_selftest_wait_timeout(ctx.handle, int(cycles), _stream(stream)), "lb_selftest_wait_timeout")


def lb_propagate_batch_static(P, states, steps_per_slice=1, stream=None):
    """FP64 propagation with no context and no device allocation (the
    intermediate states use a 4 MiB array reserved by the library; calls
    must not overlap on the GPU).  Runs on the current CUDA device."""
    c128 = torch.complex128
    S, n = P.shape[0], P.shape[1]
    B = states.shape[0]
    cur = torch.cuda.current_device()
    for t, what in ((P, "P"), (states, "states")):
        if t.is_cuda and t.device.index != cur:
            raise ValueError("%s is on cuda:%d, the current device is cuda:%d" % (what, t.device.index, cur))
    _check(lib().lb_propagate_batch_static(n, S, _ptr(P, c128, "P", (S, n, n)), int(steps_per_slice), B,
                                           _ptr(states, c128, "states", (B, n)), _stream(stream)),
           "lb_propagate_batch_static")


def lb_expmv(ctx, Lbase, Ldrv, u, dt, states, stream=None, hermitian=False):
    """states (B x n, overwritten) <- exp((Lbase + u[s] Ldrv) dt) states for
    every slice s, without forming the propagators (truncated Taylor series
    with scaling, FP64).  Ldrv None: Lbase is (S, n, n) and u is ignored.
    hermitian: the states are density matrices, propagated on their real
    coordinates (lb_expmv_hermitian).  Returns the Taylor degree m and the
    number of sub-steps per slice."""
    c128 = torch.complex128
    B, n = states.shape
    if Ldrv is None:
        S = Lbase.shape[0]
        lbp = _ptr(Lbase, c128, "Lbase", (S, n, n))
        ldp = up = None
    else:
        S = u.shape[0]
        lbp = _ptr(Lbase, c128, "Lbase", (n, n))
        ldp = _ptr(Ldrv, c128, "Ldrv", (n, n))
        up = _ptr(u, torch.float64, "u", (S,))
    ms = (ctypes.c_int * 2)()
    fn = lib().lb_expmv_hermitian if hermitian else lib().lb_expmv
    _check(fn(ctx.handle, n, S, lbp, ldp, up, float(dt), B, _ptr(states, c128, "states", (B, n)), ms, _stream(stream)),
           "lb_expmv_hermitian" if hermitian else "lb_expmv")
    return int(ms[0]), int(ms[1])


_CODE_DTYPES = {15: torch.int16, 31: torch.int32}


def _code_ptr(t, frac_bits, what, count=None):
    """A contiguous CUDA tensor of code pairs: int16 (Q1.15) or int32 (Q1.31),
    last dimension 2 (re, im).  Returns (pointer, number of complex values)."""
    dt = _CODE_DTYPES.get(frac_bits)
    if dt is None:
        raise ValueError("frac_bits must be 15 or 31")
    if not isinstance(t, torch.Tensor) or t.dtype != dt or not t.is_cuda or not t.is_contiguous() \
            or t.dim() < 1 or t.shape[-1] != 2:
        raise ValueError("%s must be a contiguous CUDA %s tensor of shape (..., 2)" % (what, dt))
    m = t.numel() // 2
    if count is not None and m != count:
        raise ValueError("%s holds %d complex values, expected %d" % (what, m, count))
    return ctypes.c_void_p(t.data_ptr()), m


def lb_fixed_quantize(x, q, frac_bits=15, stream=None):
    """q = Q1.f codes of the complex128 tensor x (nearest, ties to even,
    saturated); q has x's shape plus a last dimension 2."""
    qp, m = _code_ptr(q, frac_bits, "q", x.numel())
    _check(lib().lb_fixed_quantize(int(frac_bits), m, _ptr(x, torch.complex128, "x"), qp, _stream(stream)),
           "lb_fixed_quantize")


def lb_fixed_dequantize(q, x, frac_bits=15, stream=None):
    """x = q / 2^f as complex128."""
    qp, m = _code_ptr(q, frac_bits, "q", x.numel())
    _check(lib().lb_fixed_dequantize(int(frac_bits), m, qp, _ptr(x, torch.complex128, "x"), _stream(stream)),
           "lb_fixed_dequantize")


def lb_propagate_fixed(P_q, states_q, nsteps, frac_bits=15, stream=None):
    """nsteps fixed-point steps (Algorithm alg:fpga) of the B states in
    states_q (B x n x 2 codes, overwritten) with the propagator P_q
    (n x n x 2 codes)."""
    n = P_q.shape[0]
    pp, _ = _code_ptr(P_q, frac_bits, "P_q", n * n)
    B = states_q.shape[0]
    sp, _ = _code_ptr(states_q, frac_bits, "states_q", B * n)
    _check(lib().lb_propagate_fixed(int(frac_bits), n, pp, int(nsteps), B, sp, _stream(stream)),
           "lb_propagate_fixed")


def _host_ptr(t, what, shape):
    if not isinstance(t, torch.Tensor) or t.dtype != torch.complex128 or t.is_cuda or not t.is_contiguous():
        raise ValueError("%s must be a contiguous CPU complex128 tensor" % what)
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (what, tuple(t.shape), tuple(shape)))
    return ctypes.c_void_p(t.data_ptr())


def lb_propagate_resident(ctx, P, states_host, stream=None):
    """One FP64 step of the host-memory states (B x n CPU tensor, overwritten)
    with the device propagator P (n x n): the resident-P model (Eq. 8)."""
    n = P.shape[0]
    B = states_host.shape[0]
    _check(lib().lb_propagate_resident(ctx.handle, n, _ptr(P, torch.complex128, "P", (n, n)), B,
                                       _host_ptr(states_host, "states_host", (B, n)), _stream(stream)),
           "lb_propagate_resident")


def lb_propagate_host(ctx, P_host, states_host, stream=None):
    """As lb_propagate_resident with P in host memory too, device buffers
    allocated and freed inside the call: the host-visible model (Eq. 9)."""
    n = P_host.shape[0]
    B = states_host.shape[0]
    _check(lib().lb_propagate_host(ctx.handle, n, _host_ptr(P_host, "P_host", (n, n)), B,
                                   _host_ptr(states_host, "states_host", (B, n)), _stream(stream)),
           "lb_propagate_host")


def lb_probe_launch(reps=1000, sync_each=False, stream=None):
    """Host microseconds per empty-kernel launch (sync_each: launch + sync)."""
    us = ctypes.c_double(0.0)
    _check(lib().lb_probe_launch(int(reps), int(bool(sync_each)), ctypes.byref(us), _stream(stream)),
           "lb_probe_launch")
    return us.value


def lb_probe_copy(host, device, to_device, reps=20, stream=None):
    """Host microseconds per synchronous copy between the CPU tensor `host`
    and the CUDA tensor `device` (same byte size)."""
    nb = host.numel() * host.element_size()
    if host.is_cuda or not device.is_cuda or device.numel() * device.element_size() != nb:
        raise ValueError("host must be a CPU tensor and device a CUDA tensor of the same byte size")
    us = ctypes.c_double(0.0)
    _check(lib().lb_probe_copy(ctypes.c_void_p(host.data_ptr()), ctypes.c_void_p(device.data_ptr()), nb,
                               int(bool(to_device)), int(reps), ctypes.byref(us), _stream(stream)), "lb_probe_copy")
    return us.value


def _peak(name, stream):
    tf = ctypes.c_double(0.0)
    _check(getattr(lib(), name)(ctypes.byref(tf), _stream(stream)), name)
    return tf.value


def lb_probe_dfma(stream=None):
    """Measured FP64 FMA rate of the current device, TFLOP/s."""
    return _peak("lb_probe_dfma", stream)


def lb_probe_ffma(stream=None):
    """Measured FP32 FMA rate of the current device, TFLOP/s."""
    return _peak("lb_probe_ffma", stream)


def lb_probe_dmma(stream=None):
    """Measured FP64 tensor-core (mma.sync m8n8k4) rate, TFLOP/s."""
    return _peak("lb_probe_dmma", stream)


def lb_probe_bf16_tc(stream=None):
    """Measured BF16 tcgen05 MMA rate (dense, FP32 accumulation), TFLOP/s."""
    return _peak("lb_probe_bf16_tc", stream)


def lb_probe_alloc(nbytes, reps=20):
    """Host microseconds per cudaMalloc + cudaFree pair of nbytes bytes."""
    us = ctypes.c_double(0.0)
    _check(lib().lb_probe_alloc(int(nbytes), int(reps), ctypes.byref(us)), "lb_probe_alloc")
    return us.value


def lb_probe_read(buf, n, sink, stream=None):
    """One read pass over the complex128 CUDA tensor buf: n = 0 coalesced
    stream, n >= 1 stride-n gather (Algorithm alg:gpu's access pattern)."""
    _check(lib().lb_probe_read(_ptr(buf, torch.complex128, "buf"), buf.numel(), int(n),
                               _ptr(sink, torch.int64, "sink"), _stream(stream)), "lb_probe_read")


def lb_run_instances(ctx, instances, dt, prec="fp64", renorm_trace=False, stream=None):
    """Run many independent problems: ``instances`` is a list of dicts with
    keys Lbase, Ldrv (n x n), u (nslices,), states (B x n, overwritten) and
    optional steps_per_slice (default 1).  Tensors stay alive during the call."""
    c128 = torch.complex128
    arr = (Instance * len(instances))()
    for i, x in enumerate(instances):
        n = x["Lbase"].shape[0]
        d = int(round(n ** 0.5))
        S = x["u"].shape[0]
        B = x["states"].shape[0]
        arr[i] = Instance(d, S, int(x.get("steps_per_slice", 1)), B,
                          _ptr(x["Lbase"], c128, "Lbase", (n, n)), _ptr(x["Ldrv"], c128, "Ldrv", (n, n)),
                          _ptr(x["u"], torch.float64, "u", (S,)), _ptr(x["states"], c128, "states", (B, n)))
    _check(lib().lb_run_instances(ctx.handle, arr, len(instances), float(dt), PRECISIONS.get(prec, prec),
                                  int(bool(renorm_trace)), _stream(stream)), "lb_run_instances")


def _dims(dims):
    return (ctypes.c_int * len(dims))(*[int(x) for x in dims])


def lb_mlp_forward(dims, W_bf16, b, x, acts, stream=None):
    """acts <- outputs of every layer (see include/lb.h)."""
    nl = len(dims) - 1
    batch = x.shape[0]
    _check(lib().lb_mlp_forward(nl, _dims(dims), batch, _ptr(W_bf16, torch.bfloat16, "W"),
                                _ptr(b, torch.float32, "b"), _ptr(x, torch.float32, "x"),
                                _ptr(acts, torch.float32, "acts"), _stream(stream)), "lb_mlp_forward")


def lb_mlp_backward(dims, W_bf16, x, acts, dy, gW, gb, scratch, stream=None):
    nl = len(dims) - 1
    batch = x.shape[0]
    _check(lib().lb_mlp_backward(nl, _dims(dims), batch, _ptr(W_bf16, torch.bfloat16, "W"),
                                 _ptr(x, torch.float32, "x"), _ptr(acts, torch.float32, "acts"),
                                 _ptr(dy, torch.float32, "dy"), _ptr(gW, torch.float32, "gW"),
                                 _ptr(gb, torch.float32, "gb"), _ptr(scratch, torch.float32, "scratch"),
                                 _stream(stream)), "lb_mlp_backward")


def lb_mse_loss_grad(y, t, dy, loss=None, stream=None):
    _check(lib().lb_mse_loss_grad(y.numel(), _ptr(y, torch.float32, "y"), _ptr(t, torch.float32, "t"),
                                  _ptr(dy, torch.float32, "dy"), _ptr(loss, torch.float32, "loss", allow_none=True),
                                  _stream(stream)), "lb_mse_loss_grad")


def lb_adam_step(p, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, p_bf16=None, stream=None):
    _check(lib().lb_adam_step(p.numel(), _ptr(p, torch.float32, "p"), _ptr(g, torch.float32, "g"),
                              _ptr(m, torch.float32, "m"), _ptr(v, torch.float32, "v"),
                              _ptr(p_bf16, torch.bfloat16, "p_bf16", allow_none=True), float(lr), float(beta1),
                              float(beta2), float(eps), int(step), _stream(stream)), "lb_adam_step")


def lb_adam_step_f64(p, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, ascend=False, stream=None):
    _check(lib().lb_adam_step_f64(p.numel(), _ptr(p, torch.float64, "p"), _ptr(g, torch.float64, "g"),
                                  _ptr(m, torch.float64, "m"), _ptr(v, torch.float64, "v"), float(lr), float(beta1),
                                  float(beta2), float(eps), int(step), int(bool(ascend)), _stream(stream)),
           "lb_adam_step_f64")
