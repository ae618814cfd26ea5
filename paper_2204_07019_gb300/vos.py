"""ctypes binding of the C ABI in include/vos.h (argument marshalling only).

Every step of the computation runs in ``libvos.so``; this module only
converts arguments.  Importing it loads the library and raises if it is
missing: there is no CPU fallback.  Device memory can come from PyTorch's
caching allocator (``allocator="torch"``, the default when torch with CUDA
is importable) and the work is enqueued on the caller's CUDA stream.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import inputs as _inputs

__all__ = [
    "VosError", "load_library", "vos_create", "vos_step", "vos_fields", "vos_set_fields",
    "vos_device_fields_get", "vos_get_stats", "vos_suggest_dt", "vos_upscaled", "vos_last_error", "vos_destroy",
    "vos_device_bytes", "vos_kernel_launches", "vos_set_launch_mode", "vos_set_coarse_cycle", "vos_set_vector_sweeps",
    "vos_set_fused_pcg", "vos_prof_enable", "vos_prof_report", "vos_prof_reset",
    "vos_suggest_dt_noalloc", "vos_batch_create", "vos_batch_step", "vos_batch_handle", "vos_batch_destroy",
    "vos_unet_create", "vos_unet_num_params", "vos_unet_set_params", "vos_unet_get_params", "vos_unet_get_grads",
    "vos_unet_forward", "vos_unet_backward", "vos_unet_train_step", "vos_unet_eval_loss", "vos_unet_destroy",
    "vos_floating_clusters", "vos_tile_config", "vos_fp64_div_check", "vos_conv3d_bf16", "UNet", "vos_set_unet_preconditioner",
    "vos_unet_solve_stats", "vos_pressure_snapshots", "Simulation", "LIB_PATH", "EXPORTED_SYMBOLS", "PRECOND_NO_DEFLATION",
    "PRECOND_MOM_DIAG", "PRECOND_MOM_MG", "PRECOND_P_WARM", "PRECOND_U_EXTRAP", "FUSED_DIAG_PCG", "FUSED_MG_PCG", "FUSED_DF_RESIDUAL", "FUSED_ALL",
]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libvos.so")

VOS_OK, VOS_EINVAL, VOS_ENOMEM, VOS_ECUDA, VOS_ENOCONV, VOS_ETIMEOUT = 0, -1, -2, -3, -4, -5
F_EPS, F_C, F_U, F_V, F_W, F_P, F_R, F_RF = 1, 2, 4, 8, 16, 32, 64, 128
F_ALL = 255
PRECOND_NO_DEFLATION = 1
PRECOND_MOM_DIAG = 2
PRECOND_MOM_MG = 4
PRECOND_P_WARM = 8
PRECOND_U_EXTRAP = 16
FUSED_DIAG_PCG = 1
FUSED_MG_PCG = 2
FUSED_DF_RESIDUAL = 4
FUSED_ALL = 7

EXPORTED_SYMBOLS = [
    "vos_create", "vos_step", "vos_fields", "vos_set_fields", "vos_device_fields_get",
    "vos_get_stats", "vos_suggest_dt", "vos_upscaled", "vos_last_error", "vos_destroy", "vos_device_bytes",
    "vos_kernel_launches", "vos_set_launch_mode", "vos_set_coarse_cycle", "vos_set_vector_sweeps", "vos_set_fused_pcg",
    "vos_prof_enable", "vos_prof_report",
    "vos_prof_reset", "vos_suggest_dt_noalloc", "vos_batch_create", "vos_batch_step", "vos_batch_handle",
    "vos_batch_destroy",
    "vos_floating_clusters", "vos_tile_config", "vos_fp64_div_check", "vos_conv3d_bf16",
    "vos_unet_create", "vos_unet_num_params", "vos_unet_set_params", "vos_unet_get_params", "vos_unet_get_grads",
    "vos_unet_forward", "vos_unet_backward", "vos_unet_train_step", "vos_unet_eval_loss", "vos_unet_destroy",
    "vos_set_unet_preconditioner", "vos_unet_solve_stats", "vos_pressure_snapshots",
]


class VosError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class VosParams(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("dx", ctypes.c_double), ("nu", ctypes.c_double), ("D", ctypes.c_double), ("kc", ctypes.c_double),
        ("k0", ctypes.c_double), ("Vm", ctypes.c_double), ("zeta", ctypes.c_double),
        ("rho_ratio", ctypes.c_double), ("c_in", ctypes.c_double), ("u_in", ctypes.c_double),
        ("eps_min", ctypes.c_double), ("lambda_", ctypes.c_double),
        ("method", ctypes.c_int32), ("precision", ctypes.c_int32), ("precond", ctypes.c_int32),
        ("p_rtol", ctypes.c_double), ("u_rtol", ctypes.c_double), ("c_rtol", ctypes.c_double),
        ("max_iter", ctypes.c_int32), ("flow_subiters", ctypes.c_int32), ("wall_mask", ctypes.c_uint32),
        ("qs_rtol", ctypes.c_double), ("qs_dtau", ctypes.c_double), ("inertia", ctypes.c_int32),
    ]


class VosStats(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("t", ctypes.c_double),
        ("iters_u", ctypes.c_int32 * 3), ("iters_p", ctypes.c_int32), ("iters_c", ctypes.c_int32),
        ("outer_u", ctypes.c_int32 * 3), ("outer_p", ctypes.c_int32), ("outer_c", ctypes.c_int32),
        ("res_u", ctypes.c_double * 3), ("res_p", ctypes.c_double), ("res_c", ctypes.c_double),
        ("lambda_", ctypes.c_double), ("porosity", ctypes.c_double), ("clamp_excess", ctypes.c_double),
        ("sum_R", ctypes.c_double), ("sum_Rf", ctypes.c_double), ("reactant", ctypes.c_double),
        ("status", ctypes.c_int32),
        ("q_in", ctypes.c_double), ("q_out", ctypes.c_double), ("flux_in", ctypes.c_double),
        ("flux_out", ctypes.c_double), ("umax", ctypes.c_double), ("rmax", ctypes.c_double),
        ("qs_iters", ctypes.c_int32), ("qs_du", ctypes.c_double), ("qs_dp", ctypes.c_double),
        ("qs_dc", ctypes.c_double),
    ]


class VosUpscaled(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("phi", "Q_in", "A_in", "U_D", "dP", "L_D", "K", "a", "alpha",
                                                "L_ref", "U_ref", "Pe", "Da", "Ki")]


class VosDeviceFields(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("eps", "c", "p", "u", "v", "w", "R", "Rf")]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class VosAllocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


_lib = None


def load_library(path=None):
    """Load libvos.so (raises OSError if it is missing or does not load)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"libvos.so not found at {p}: build it with paper_2204_07019_gb300.build_lib.build()")
    lib = ctypes.CDLL(p)
    H = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    lib.vos_create.argtypes = [dp, ctypes.POINTER(VosParams), ctypes.c_void_p, ctypes.POINTER(VosAllocator),
                               ctypes.POINTER(H)]
    lib.vos_create.restype = ctypes.c_int
    lib.vos_step.argtypes = [H, ctypes.c_double]
    lib.vos_step.restype = ctypes.c_int
    lib.vos_fields.argtypes = [H, ctypes.c_uint32] + [dp] * 8
    lib.vos_fields.restype = ctypes.c_int
    lib.vos_set_fields.argtypes = [H, ctypes.c_uint32] + [dp] * 8
    lib.vos_set_fields.restype = ctypes.c_int
    lib.vos_device_fields_get.argtypes = [H, ctypes.POINTER(VosDeviceFields)]
    lib.vos_device_fields_get.restype = ctypes.c_int
    lib.vos_get_stats.argtypes = [H, ctypes.POINTER(VosStats)]
    lib.vos_get_stats.restype = ctypes.c_int
    lib.vos_upscaled.argtypes = [H, ctypes.POINTER(VosUpscaled)]
    lib.vos_upscaled.restype = ctypes.c_int
    lib.vos_suggest_dt.argtypes = [H, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    lib.vos_suggest_dt.restype = ctypes.c_int
    lib.vos_last_error.argtypes = [H]
    lib.vos_last_error.restype = ctypes.c_char_p
    lib.vos_destroy.argtypes = [H]
    lib.vos_destroy.restype = None
    lib.vos_device_bytes.argtypes = [H]
    lib.vos_device_bytes.restype = ctypes.c_size_t
    lib.vos_kernel_launches.argtypes = []
    lib.vos_kernel_launches.restype = ctypes.c_uint64
    lib.vos_set_launch_mode.argtypes = [ctypes.c_int]
    lib.vos_set_launch_mode.restype = ctypes.c_int
    lib.vos_set_coarse_cycle.argtypes = [ctypes.c_int]
    lib.vos_set_coarse_cycle.restype = ctypes.c_int
    lib.vos_set_vector_sweeps.argtypes = [ctypes.c_int]
    lib.vos_set_vector_sweeps.restype = ctypes.c_int
    lib.vos_set_fused_pcg.argtypes = [ctypes.c_int]
    lib.vos_set_fused_pcg.restype = ctypes.c_int
    lib.vos_prof_enable.argtypes = [ctypes.c_char_p]
    lib.vos_prof_enable.restype = ctypes.c_int
    lib.vos_prof_report.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    lib.vos_prof_report.restype = ctypes.c_int
    lib.vos_prof_reset.argtypes = []
    lib.vos_prof_reset.restype = None
    lib.vos_suggest_dt_noalloc.argtypes = [ctypes.POINTER(VosParams)] + [ctypes.c_void_p] * 5 + [
        ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    lib.vos_suggest_dt_noalloc.restype = ctypes.c_int
    lib.vos_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(dp), ctypes.POINTER(VosParams), ctypes.c_void_p,
                                     ctypes.c_int, ctypes.POINTER(VosAllocator), ctypes.POINTER(ctypes.c_void_p)]
    lib.vos_batch_create.restype = ctypes.c_int
    lib.vos_batch_step.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    lib.vos_batch_step.restype = ctypes.c_int
    lib.vos_batch_handle.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    lib.vos_batch_handle.restype = ctypes.c_int
    lib.vos_batch_destroy.argtypes = [ctypes.c_void_p]
    lib.vos_batch_destroy.restype = None
    lib.vos_floating_clusters.argtypes = [dp, ctypes.POINTER(VosParams), ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]
    lib.vos_floating_clusters.restype = ctypes.c_int
    lib.vos_tile_config.argtypes = [H, ctypes.c_int32, ctypes.c_int32] + [ctypes.POINTER(ctypes.c_int32)] * 4
    lib.vos_tile_config.restype = ctypes.c_int
    lib.vos_fp64_div_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                       ctypes.c_void_p]
    lib.vos_fp64_div_check.restype = ctypes.c_int
    lib.vos_conv3d_bf16.argtypes = [ctypes.c_void_p] + [ctypes.c_int32] * 4 + [ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.vos_conv3d_bf16.restype = ctypes.c_int
    vp, fp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)
    lib.vos_unet_create.argtypes = [ctypes.c_int32] * 4 + [vp, ctypes.POINTER(vp)]
    lib.vos_unet_create.restype = ctypes.c_int
    lib.vos_unet_num_params.argtypes = []
    lib.vos_unet_num_params.restype = ctypes.c_int64
    for name in ("vos_unet_set_params", "vos_unet_get_params", "vos_unet_get_grads"):
        getattr(lib, name).argtypes = [vp, vp, ctypes.c_int64]
        getattr(lib, name).restype = ctypes.c_int
    lib.vos_unet_forward.argtypes = [vp, vp, vp, vp]
    lib.vos_unet_forward.restype = ctypes.c_int
    lib.vos_unet_backward.argtypes = [vp, vp]
    lib.vos_unet_backward.restype = ctypes.c_int
    lib.vos_unet_train_step.argtypes = [vp, vp, vp, ctypes.c_float, fp]
    lib.vos_unet_train_step.restype = ctypes.c_int
    lib.vos_unet_eval_loss.argtypes = [vp, vp, vp, fp]
    lib.vos_unet_eval_loss.restype = ctypes.c_int
    lib.vos_unet_destroy.argtypes = [vp]
    lib.vos_unet_destroy.restype = None
    lib.vos_set_unet_preconditioner.argtypes = [vp, vp]
    lib.vos_set_unet_preconditioner.restype = ctypes.c_int
    lib.vos_unet_solve_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    lib.vos_unet_solve_stats.restype = ctypes.c_int
    lib.vos_pressure_snapshots.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), vp]
    lib.vos_pressure_snapshots.restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def _params_struct(prm):
    p = VosParams()
    full = dict(_inputs.PARAM_DEFAULTS)
    full.update(prm)
    for name, _ in VosParams._fields_:
        key = "lam" if name == "lambda_" else name
        setattr(p, name, type(getattr(p, name))(full[key]))
    return p


class _Handle:
    """Owns a vos_handle* and keeps the allocator callbacks alive."""

    def __init__(self, ptr, prm, keep):
        self.ptr = ptr
        self.prm = dict(prm)
        self._keep = keep

    @property
    def shape(self):
        return (int(self.prm["nz"]), int(self.prm["ny"]), int(self.prm["nx"]))


def _check(lib, h, rc, allow_noconv=False):
    if rc == VOS_OK or (allow_noconv and rc == VOS_ENOCONV):
        return rc
    msg = lib.vos_last_error(h).decode()
    raise VosError(rc, msg)


def _torch_allocator():
    import torch
    dev = torch.cuda.current_device()

    def alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev)
        except Exception:  # noqa: BLE001 - report as NULL to the library
            return None

    def free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    fa, ff = ALLOC_FN(alloc), FREE_FN(free)
    return VosAllocator(fa, ff, None), (fa, ff)


def vos_create(eps_s, prm, stream=None, allocator="auto"):
    """vos_create: eps_s (nz, ny, nx) float64 host array, parameter dict.

    ``stream``: a torch.cuda.Stream, an int cudaStream_t or None (torch's
    current stream if torch is available, else the legacy default stream).
    ``allocator``: "torch", "cuda" or "auto".
    """
    lib = load_library()
    es = np.ascontiguousarray(eps_s, dtype=np.float64)
    ps = _params_struct(prm)
    if es.size != ps.nx * ps.ny * ps.nz:
        raise VosError(VOS_EINVAL, f"eps_s has {es.size} values, grid has {ps.nx * ps.ny * ps.nz}")
    st = None
    keep = []
    alloc_ptr = None
    use_torch = allocator == "torch"
    if allocator == "auto":
        try:
            import torch
            use_torch = torch.cuda.is_available()
        except ImportError:
            use_torch = False
    if stream is None and use_torch:
        import torch
        st = torch.cuda.current_stream().cuda_stream
    elif stream is not None:
        st = int(getattr(stream, "cuda_stream", stream))
    if use_torch:
        a, cbs = _torch_allocator()
        keep += [a, cbs]
        alloc_ptr = ctypes.byref(a)
    out = ctypes.c_void_p()
    rc = lib.vos_create(es.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(ps),
                        ctypes.c_void_p(st), alloc_ptr, ctypes.byref(out))
    if rc != VOS_OK:
        raise VosError(rc, lib.vos_last_error(None).decode())
    return _Handle(out, prm, keep)


def vos_step(h, dt):
    """vos_step: one time step; returns VOS_OK or VOS_ENOCONV."""
    lib = load_library()
    return _check(lib, h.ptr, lib.vos_step(h.ptr, float(dt)), allow_noconv=True)


def _field_shapes(h):
    nz, ny, nx = h.shape
    return {"eps": (nz, ny, nx), "c": (nz, ny, nx), "u": (nz, ny, nx + 1), "v": (nz, ny + 1, nx),
            "w": (nz + 1, ny, nx), "p": (nz, ny, nx), "R": (nz, ny, nx), "Rf": (nz, ny, nx)}


_ORDER = ("eps", "c", "u", "v", "w", "p", "R", "Rf")
_BITS = dict(zip(_ORDER, (F_EPS, F_C, F_U, F_V, F_W, F_P, F_R, F_RF)))


def vos_fields(h, names=_ORDER):
    """vos_fields: copy fields to new host arrays; returns a dict."""
    lib = load_library()
    shp = _field_shapes(h)
    dim = int(h.prm["dim"])
    out, ptrs, mask = {}, [], 0
    for n in _ORDER:
        if n in names and not (n == "w" and dim == 2):
            a = np.empty(shp[n], dtype=np.float64)
            out[n] = a
            mask |= _BITS[n]
            ptrs.append(a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        else:
            ptrs.append(None)
    _check(lib, h.ptr, lib.vos_fields(h.ptr, mask, *ptrs))
    return out


def vos_set_fields(h, **arrays):
    """vos_set_fields: overwrite the given fields from host arrays."""
    lib = load_library()
    shp = _field_shapes(h)
    ptrs, mask, keep = [], 0, []
    for n in _ORDER:
        if n in arrays:
            a = np.ascontiguousarray(arrays[n], dtype=np.float64)
            if a.size != int(np.prod(shp[n])):
                raise VosError(VOS_EINVAL, f"{n}: {a.size} values, expected {shp[n]}")
            keep.append(a)
            mask |= _BITS[n]
            ptrs.append(a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        else:
            ptrs.append(None)
    _check(lib, h.ptr, lib.vos_set_fields(h.ptr, mask, *ptrs))


def vos_device_fields_get(h):
    """vos_device_fields_get: dict of device pointers (ints)."""
    lib = load_library()
    f = VosDeviceFields()
    _check(lib, h.ptr, lib.vos_device_fields_get(h.ptr, ctypes.byref(f)))
    return {n: getattr(f, n) for n, _ in VosDeviceFields._fields_}


def vos_get_stats(h):
    """vos_get_stats: statistics of the last step as a dict."""
    lib = load_library()
    s = VosStats()
    _check(lib, h.ptr, lib.vos_get_stats(h.ptr, ctypes.byref(s)))
    d = {}
    for n, _ in VosStats._fields_:
        v = getattr(s, n)
        d["lambda" if n == "lambda_" else n] = list(v) if hasattr(v, "__len__") else v
    return d


def vos_upscaled(h):
    """vos_upscaled: Darcy-scale properties (phi, U_D, K, a, alpha, ...) as a dict."""
    lib = load_library()
    r = VosUpscaled()
    _check(lib, h.ptr, lib.vos_upscaled(h.ptr, ctypes.byref(r)))
    return {n: getattr(r, n) for n, _ in VosUpscaled._fields_}


def vos_suggest_dt(h, cfl=0.5, deps_max=0.005):
    """vos_suggest_dt: min(cfl dx / max|u|/eps, deps_max / max|Vm R|)."""
    lib = load_library()
    dt = ctypes.c_double()
    _check(lib, h.ptr, lib.vos_suggest_dt(h.ptr, float(cfl), float(deps_max), ctypes.byref(dt)))
    return dt.value


def vos_suggest_dt_noalloc(prm, eps, u, v, w, R, cfl=0.5, deps_max=0.005, stream=None):
    """vos_suggest_dt_noalloc: the time-step limit from caller-owned device
    fields (int device pointers) without any device allocation; see vos.h."""
    lib = load_library()
    ps = _params_struct(prm)
    dt = ctypes.c_double()
    st = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    rc = lib.vos_suggest_dt_noalloc(ctypes.byref(ps), eps, u, v, w, R, float(cfl), float(deps_max),
                                    ctypes.c_void_p(st), ctypes.byref(dt))
    if rc != VOS_OK:
        raise VosError(rc, lib.vos_last_error(None).decode())
    return dt.value


def _ptr(t):
    """Device pointer of a torch tensor (or an int / None)."""
    if t is None:
        return None
    return int(t.data_ptr()) if hasattr(t, "data_ptr") else int(t)


def vos_fp64_div_check(a, d):
    """vos_fp64_div_check on host arrays: returns (q_fast, q_ieee), the
    physics kernels' FP64 quotient a/d and the IEEE one, computed on the
    device (torch provides the device buffers)."""
    import torch
    lib = load_library()
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    d = np.ascontiguousarray(d, dtype=np.float64).ravel()
    if a.shape != d.shape:
        raise ValueError("a and d differ in size")
    torch.cuda.synchronize()
    ad = torch.from_numpy(a).cuda()
    dd = torch.from_numpy(d).cuda()
    qf = torch.empty_like(ad)
    qi = torch.empty_like(ad)
    torch.cuda.synchronize()
    rc = lib.vos_fp64_div_check(_ptr(ad), _ptr(dd), int(a.size), _ptr(qf), _ptr(qi))
    _check(lib, None, rc)
    return qf.cpu().numpy(), qi.cpu().numpy()


def vos_conv3d_bf16(x, shape, cin, w, bias, cout, relu=False, y_f32=None, y_bf16=None, stream=None):
    """vos_conv3d_bf16 on device tensors: x BF16 [V, cin] for a box of
    ``shape`` = (nz, ny, nx), w BF16 [cout, 27, cin], bias FP32 [cout] or
    None; writes y_f32 [V, cout] FP32 and/or y_bf16 [V, cout] BF16."""
    lib = load_library()
    nz, ny, nx = shape
    st = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    rc = lib.vos_conv3d_bf16(_ptr(x), int(nx), int(ny), int(nz), int(cin), _ptr(w), _ptr(bias), int(cout),
                             1 if relu else 0, _ptr(y_f32), _ptr(y_bf16), st)
    if rc != VOS_OK:
        raise VosError(rc, lib.vos_last_error(None).decode())


def _raise(lib, rc, h=None):
    if rc != VOS_OK:
        raise VosError(rc, lib.vos_last_error(h).decode())


class UNet:
    """The learned pressure preconditioner (vos_unet_*): a network for one
    grid shape (nz, ny, nx).  Device vectors are torch CUDA tensors."""

    def __init__(self, shape, train=True, stream=None):
        lib = load_library()
        nz, ny, nx = shape
        self.shape = tuple(shape)
        st = None if stream is None else int(getattr(stream, "cuda_stream", stream))
        ptr = ctypes.c_void_p()
        _raise(lib, lib.vos_unet_create(int(nx), int(ny), int(nz), 1 if train else 0, st, ctypes.byref(ptr)))
        self.ptr = ptr

    @staticmethod
    def num_params():
        return int(load_library().vos_unet_num_params())

    # (C_in, C_out) of the ten 3x3x3 convs in parameter order
    CONVS = ((2, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (96, 32), (32, 32), (48, 16), (16, 16))

    @classmethod
    def he_init(cls, seed):
        """Seeded He-normal weights and zero biases as a flat parameter vector."""
        g = np.random.default_rng(seed)
        parts = []
        for ci, co in cls.CONVS:
            parts.append(g.standard_normal(co * 27 * ci) * np.sqrt(2.0 / (27 * ci)))
            parts.append(np.zeros(co))
        parts.append(g.standard_normal(16) * np.sqrt(1.0 / 16))
        parts.append(np.zeros(1))
        return np.concatenate(parts).astype(np.float32)

    def set_params(self, flat):
        lib = load_library()
        a = np.ascontiguousarray(flat, dtype=np.float32)
        _raise(lib, lib.vos_unet_set_params(self.ptr, a.ctypes.data, a.size))

    def _get(self, name):
        lib = load_library()
        a = np.empty(self.num_params(), dtype=np.float32)
        _raise(lib, getattr(lib, name)(self.ptr, a.ctypes.data, a.size))
        return a

    def get_params(self):
        return self._get("vos_unet_get_params")

    def get_grads(self):
        return self._get("vos_unet_get_grads")

    def forward(self, r, eps, z):
        lib = load_library()
        _raise(lib, lib.vos_unet_forward(self.ptr, _ptr(r), _ptr(eps), _ptr(z)))

    def backward(self, dz):
        lib = load_library()
        _raise(lib, lib.vos_unet_backward(self.ptr, _ptr(dz)))

    def train_step(self, h, r, lr):
        lib = load_library()
        loss = ctypes.c_float()
        _raise(lib, lib.vos_unet_train_step(self.ptr, h.ptr, _ptr(r), float(lr), ctypes.byref(loss)))
        return loss.value

    def eval_loss(self, h, r):
        lib = load_library()
        loss = ctypes.c_float()
        _raise(lib, lib.vos_unet_eval_loss(self.ptr, h.ptr, _ptr(r), ctypes.byref(loss)))
        return loss.value

    def close(self):
        if self.ptr:
            load_library().vos_unet_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# The vos_unet_* calls under their C names (the UNet class carries the
# marshalling; a network is a UNet object).
def vos_unet_create(shape, train=True, stream=None):
    """vos_unet_create: a network for grids of shape (nz, ny, nx)."""
    return UNet(shape, train=train, stream=stream)


def vos_unet_num_params():
    return UNet.num_params()


def vos_unet_set_params(net, flat):
    net.set_params(flat)


def vos_unet_get_params(net):
    return net.get_params()


def vos_unet_get_grads(net):
    return net.get_grads()


def vos_unet_forward(net, r, eps, z):
    net.forward(r, eps, z)


def vos_unet_backward(net, dz):
    net.backward(dz)


def vos_unet_train_step(net, h, r, lr):
    return net.train_step(h, r, lr)


def vos_unet_eval_loss(net, h, r):
    return net.eval_loss(h, r)


def vos_unet_destroy(net):
    if net is not None:
        net.close()


def vos_set_unet_preconditioner(h, net):
    lib = load_library()
    _raise(lib, lib.vos_set_unet_preconditioner(h.ptr, net.ptr if net is not None else None), h.ptr)


def vos_unet_solve_stats(h):
    lib = load_library()
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _raise(lib, lib.vos_unet_solve_stats(h.ptr, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def vos_pressure_snapshots(h, iters, out):
    """Residual snapshots of the last pressure solve into ``out`` (a CUDA
    float32 tensor of len(iters) x cells)."""
    lib = load_library()
    arr = (ctypes.c_int32 * len(iters))(*[int(i) for i in iters])
    _raise(lib, lib.vos_pressure_snapshots(h.ptr, len(iters), arr, _ptr(out)), h.ptr)


def vos_tile_config(h, sys, level):
    """vos_tile_config: (tx, ty, zc, tuned) of the stencil tile used on one
    multigrid level of one system (0-2 momentum, 3 pressure, 4 transport)."""
    lib = load_library()
    v = [ctypes.c_int32() for _ in range(4)]
    rc = lib.vos_tile_config(h.ptr, int(sys), int(level), *[ctypes.byref(x) for x in v])
    if rc != VOS_OK:
        raise VosError(rc, lib.vos_last_error(None).decode())
    return tuple(x.value for x in v)


def vos_floating_clusters(eps, prm):
    """vos_floating_clusters (host only): labels of the floating pore clusters
    that the pressure solve deflates, for a fluid-fraction array eps of the
    grid's shape.  Returns (labels int32 array of eps's shape, -1 outside
    clusters; number of clusters; cells in clusters)."""
    lib = load_library()
    ps = _params_struct(prm)
    e = np.ascontiguousarray(eps, dtype=np.float64)
    if e.size != int(ps.nx) * int(ps.ny) * int(ps.nz):
        raise ValueError("eps has %d cells, the grid %d" % (e.size, int(ps.nx) * int(ps.ny) * int(ps.nz)))
    lab = np.empty(e.shape, dtype=np.int32)
    k = ctypes.c_int32()
    m = ctypes.c_int64()
    rc = lib.vos_floating_clusters(e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(ps),
                                   ctypes.c_void_p(lab.ctypes.data), ctypes.byref(k), ctypes.byref(m))
    if rc != VOS_OK:
        raise VosError(rc, lib.vos_last_error(None).decode())
    return lab, k.value, m.value


class _Batch:
    def __init__(self, ptr, prms, keep):
        self.ptr = ptr
        self.prms = prms
        self._keep = keep
        self.handles = []


def vos_batch_create(eps_list, prm_list, stream=None, nthreads=8, allocator="auto"):
    """vos_batch_create: n instances (lists of eps_s arrays and parameter
    dicts); returns a batch whose ``handles`` are instance handles."""
    lib = load_library()
    n = len(eps_list)
    arrs = [np.ascontiguousarray(e, dtype=np.float64) for e in eps_list]
    ptrs = (ctypes.POINTER(ctypes.c_double) * n)(*[a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in arrs])
    prms = (VosParams * n)(*[_params_struct(p) for p in prm_list])
    keep = [arrs, ptrs, prms]
    use_torch = allocator == "torch"
    if allocator == "auto":
        try:
            import torch
            use_torch = torch.cuda.is_available()
        except ImportError:
            use_torch = False
    st = None
    if stream is None and use_torch:
        import torch
        st = torch.cuda.current_stream().cuda_stream
    elif stream is not None:
        st = int(getattr(stream, "cuda_stream", stream))
    alloc_ptr = None
    if use_torch:
        a, cbs = _torch_allocator()
        keep += [a, cbs]
        alloc_ptr = ctypes.byref(a)
    out = ctypes.c_void_p()
    rc = lib.vos_batch_create(n, ptrs, prms, ctypes.c_void_p(st), int(nthreads), alloc_ptr, ctypes.byref(out))
    if rc != VOS_OK:
        raise VosError(rc, lib.vos_last_error(None).decode())
    b = _Batch(out, [dict(p) for p in prm_list], keep)
    for i in range(n):
        hp = ctypes.c_void_p()
        rc = lib.vos_batch_handle(out, i, ctypes.byref(hp))
        if rc != VOS_OK:
            msg = lib.vos_last_error(None).decode()
            lib.vos_batch_destroy(out)
            raise VosError(rc, msg)
        b.handles.append(_Handle(hp, prm_list[i], []))
    return b


def vos_batch_handle(b, i):
    """vos_batch_handle: instance i's handle, owned by the batch (do not
    destroy it, nor use it while a batch step runs)."""
    if b is None or not b.ptr or not 0 <= int(i) < len(b.handles):
        raise VosError(VOS_EINVAL, "vos_batch_handle: bad argument")
    return b.handles[int(i)]


def vos_batch_step(b, dts):
    """vos_batch_step: advance instance i by dts[i]; returns VOS_OK or VOS_ENOCONV."""
    lib = load_library()
    arr = (ctypes.c_double * len(dts))(*[float(x) for x in dts])
    rc = lib.vos_batch_step(b.ptr, arr)
    if rc not in (VOS_OK, VOS_ENOCONV):
        raise VosError(rc, lib.vos_last_error(None).decode())
    return rc


def vos_batch_destroy(b):
    """vos_batch_destroy: free every instance (idempotent)."""
    if b is not None and b.ptr:
        load_library().vos_batch_destroy(b.ptr)
        b.ptr = None
        for h in b.handles:
            h.ptr = None


def vos_last_error(h=None):
    lib = load_library()
    return lib.vos_last_error(h.ptr if h is not None else None).decode()


def vos_device_bytes(h):
    return int(load_library().vos_device_bytes(h.ptr))


def vos_kernel_launches():
    """Kernels launched by the library so far (process-wide)."""
    return int(load_library().vos_kernel_launches())


def vos_set_launch_mode(graphs):
    """1: replay each step as a CUDA graph with device-side loops (default);
    0: launch the same kernels one by one."""
    load_library().vos_set_launch_mode(1 if graphs else 0)


def vos_set_vector_sweeps(on):
    """1 (default): four-cells-per-thread matrix-free pressure sweeps when nx
    is a multiple of 4 and fused residual-restriction / prolongation-sweep
    passes in the multigrid cycles; 0: one cell per thread and separate
    passes (identical results)."""
    load_library().vos_set_vector_sweeps(1 if on else 0)


def vos_set_fused_pcg(mask):
    """Fused forms of the mixed path's solves, a bit mask (default FUSED_ALL =
    7): FUSED_DIAG_PCG (1) two-kernel diagonal PCG on constant-link operators
    (results identical to the separate kernels), FUSED_MG_PCG (2) MG-PCG on
    the matrix-free pressure level with the x/r update and r.z fused into the
    V-cycle's first and last fine sweeps (iterates equal up to rounding),
    FUSED_DF_RESIDUAL (4) the refinement residual after the first pass in
    double-FP32 for symmetric solves to 1e-9 or looser.  Set before the
    handle's first step (a captured step graph keeps its form)."""
    rc = load_library().vos_set_fused_pcg(int(mask))
    if rc != VOS_OK:
        raise VosError(rc, f"vos_set_fused_pcg: mask {mask} outside 0..7")


def vos_set_coarse_cycle(on):
    """1: the coarse multigrid levels of hierarchies set up afterwards run as
    one cluster launch per V-cycle; 0 (default): one launch per operation."""
    load_library().vos_set_coarse_cycle(1 if on else 0)


def vos_prof_enable(filt):
    """Time launches of kernels whose name contains one of the comma-separated
    substrings ("*" all, None or "" off)."""
    load_library().vos_prof_enable(filt.encode() if filt else None)


def vos_prof_report():
    """{name: (launches, total_ms, algorithmic_bytes)} of the timed kernels."""
    lib = load_library()
    n = lib.vos_prof_report(None, 0)
    buf = ctypes.create_string_buffer(max(int(n), 1) + 1024)
    lib.vos_prof_report(buf, len(buf))
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms, by = line.split("\t")
        out[name] = (int(cnt), float(ms), float(by))
    return out


def vos_prof_reset():
    load_library().vos_prof_reset()


def vos_destroy(h):
    """vos_destroy: free the handle's device memory (idempotent)."""
    if h is not None and h.ptr:
        load_library().vos_destroy(h.ptr)
        h.ptr = None


class Simulation:
    """Convenience wrapper: ``with Simulation(eps_s, prm) as sim: sim.step(dt)``."""

    def __init__(self, eps_s, prm, stream=None, allocator="auto"):
        self.h = vos_create(eps_s, prm, stream=stream, allocator=allocator)

    def step(self, dt):
        return vos_step(self.h, dt)

    def fields(self, names=_ORDER):
        return vos_fields(self.h, names)

    def set_fields(self, **arrays):
        vos_set_fields(self.h, **arrays)

    def stats(self):
        return vos_get_stats(self.h)

    def suggest_dt(self, cfl=0.5, deps_max=0.005):
        return vos_suggest_dt(self.h, cfl, deps_max)

    def close(self):
        vos_destroy(self.h)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
