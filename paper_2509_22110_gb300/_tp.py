"""ctypes binding of ``libtp.so`` (argument marshalling only).

Every function here has the name of the C entry point it calls (see
``include/tp.h``) and does nothing but convert arguments: all arithmetic
runs in the library's CUDA kernels.  A missing library is an error, never a
fallback.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# the library this binding loads: libtp.so, or the build named by TP_LIB (for
# instance the checked build libtp_debug.so)
LIB_PATH = os.environ.get("TP_LIB") or os.path.join(_HERE, "libtp.so")
_lib = None

TP_OK, TP_E_ARG, TP_E_CUDA, TP_E_STATE, TP_E_NONFINITE, TP_E_TIMEOUT, TP_E_OOM, TP_E_MODEL = range(8)
TP_DIRECT, TP_BH, TP_LEARNED, TP_BH_DUAL = 0, 1, 2, 3
TP_F32_F64ACC, TP_F32_KAHAN, TP_F64 = 0, 1, 2
TP_DTYPE_F32, TP_DTYPE_F64 = 0, 1
TP_DEVICE_PTR = 0x1
TP_POSITIONS_ONLY = 0x2
TP_EXCLUDE_EDGE = 0x4
TP_LEARNED_ENERGY = 0x8

STATUS_NAMES = {
    0: "TP_OK", 1: "TP_E_ARG", 2: "TP_E_CUDA", 3: "TP_E_STATE", 4: "TP_E_NONFINITE",
    5: "TP_E_TIMEOUT", 6: "TP_E_OOM", 7: "TP_E_MODEL",
}


class TPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class tp_params(C.Structure):
    _fields_ = [("q", C.c_int32), ("p", C.c_int32), ("scale", C.c_double), ("mode", C.c_int32),
                ("theta", C.c_double), ("prec", C.c_int32), ("flags", C.c_uint32)]


class tp_stats(C.Structure):
    _fields_ = [("nt", C.c_int64), ("nv", C.c_int64), ("pairs_exact", C.c_int64), ("far_terms", C.c_int64),
                ("far_pairs", C.c_int64), ("learned_terms", C.c_int64), ("tile_pairs", C.c_int64),
                ("tile_pairs_masked", C.c_int64), ("tile_pairs_precise", C.c_int64), ("ms_kernel", C.c_float),
                ("ms_total", C.c_float), ("kernel_launches", C.c_int64),
                ("kernel_pairs", C.c_int64), ("far_rows", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def lib():
    """Load ``libtp.so``; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2509_22110_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, i64, i32, u32 = C.c_void_p, C.c_int64, C.c_int, C.c_uint32
    L.tp_params_default.argtypes = [C.POINTER(tp_params)]
    L.tp_version.restype = C.c_char_p
    L.tp_create.argtypes = [C.POINTER(vp), i32, vp]
    L.tp_create.restype = i32
    L.tp_destroy.argtypes = [vp]
    L.tp_last_error.argtypes = [vp]
    L.tp_last_error.restype = C.c_char_p
    L.tp_mesh_upload.argtypes = [vp, vp, i64, i32, vp, i64, u32]
    L.tp_mesh_upload.restype = i32
    L.tp_tree_build.argtypes = [vp, i32, i32]
    L.tp_tree_build.restype = i32
    L.tp_energy.argtypes = [vp, C.POINTER(tp_params), C.POINTER(C.c_double)]
    L.tp_energy.restype = i32
    L.tp_gradient.argtypes = [vp, C.POINTER(tp_params), C.POINTER(C.c_double), vp, i32, u32]
    L.tp_gradient.restype = i32
    L.tp_fields.argtypes = [vp, C.POINTER(tp_params), C.POINTER(C.c_double), vp, vp, vp, u32]
    L.tp_fields.restype = i32
    L.tp_set_quadrature.argtypes = [vp, i32]
    L.tp_set_quadrature.restype = i32
    L.tp_conf_upload.argtypes = [vp, vp, i64, i32, vp, i64, u32]
    L.tp_conf_upload.restype = i32
    L.tp_conf_gradient.argtypes = [vp, C.POINTER(tp_params), C.POINTER(C.c_double), vp, i32, u32]
    L.tp_conf_gradient.restype = i32
    L.tp_far_model_load.argtypes = [vp, C.c_char_p]
    L.tp_far_model_load.restype = i32
    L.tp_get_stats.argtypes = [vp, C.POINTER(tp_stats)]
    L.tp_get_stats.restype = i32
    L.tp_debug_tri_data.argtypes = [vp, vp, vp, vp, vp]
    L.tp_debug_tri_data.restype = i32
    L.tp_debug_accum.argtypes = [vp, vp, vp, vp]
    L.tp_debug_accum.restype = i32
    L.tp_debug_tree.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, C.POINTER(C.c_int64), vp, vp]
    L.tp_set_learned_window.argtypes = [vp, C.c_int64]
    L.tp_set_learned_window.restype = i32
    L.tp_debug_tree.restype = i32
    L.tp_far_model_init.argtypes = [vp, C.c_uint64]
    L.tp_far_model_save.argtypes = [vp, C.c_char_p]
    L.tp_far_set_params.argtypes = [vp, vp, vp]
    L.tp_far_get_params.argtypes = [vp, vp, vp]
    L.tp_far_dataset_reset.argtypes = [vp]
    L.tp_far_dataset_size.argtypes = [vp, C.POINTER(C.c_int64)]
    L.tp_far_sample_pairs.argtypes = [vp, C.c_double, C.c_double, C.c_uint64, i64, C.POINTER(C.c_int64)]
    L.tp_far_dataset_get.argtypes = [vp, i64, i64, vp, vp, vp, vp]
    L.tp_far_fit_normalisation.argtypes = [vp]
    L.tp_far_train.argtypes = [vp, i64, i64, C.c_double, C.c_double, C.c_uint64, C.POINTER(C.c_double)]
    L.tp_far_eval.argtypes = [vp, vp, i64, i32, vp, vp, vp, vp, C.POINTER(C.c_double)]
    L.tp_far_adamw_step.argtypes = [vp, vp, C.c_double, C.c_double]
    for n in ("tp_far_model_init", "tp_far_model_save", "tp_far_set_params", "tp_far_get_params",
              "tp_far_dataset_reset", "tp_far_dataset_size", "tp_far_sample_pairs", "tp_far_dataset_get",
              "tp_far_fit_normalisation", "tp_far_train", "tp_far_eval", "tp_far_adamw_step"):
        getattr(L, n).restype = i32
    L.tp_gradient_direct_noalloc.argtypes = [vp, i64, vp, i64, C.POINTER(tp_params), vp, vp, vp, C.c_char_p, i64]
    L.tp_gradient_direct_noalloc.restype = i32
    L.tp_debug_wait_timeout.argtypes = [vp, C.c_double]
    L.tp_debug_wait_timeout.restype = i32
    L.tp_debug_sort.argtypes = [vp, vp, i64, i32, vp, vp, vp, vp]
    L.tp_debug_sort.restype = i32
    L.tp_debug_fail_alloc.argtypes = [vp, i64]
    L.tp_debug_fail_alloc.restype = i32
    L.tp_debug_tc_gemm.argtypes = [i32, vp, i32, vp, i32, vp]
    L.tp_debug_tc_gemm.restype = i32
    L.tp_measure_fp32_peak.argtypes = [i32, vp, i32, i32, i32, C.POINTER(C.c_double)]
    L.tp_measure_fp32_peak.restype = i32
    _lib = L
    return L


def _check(ctx, st):
    if st != TP_OK:
        msg = lib().tp_last_error(ctx)
        raise TPError(st, msg.decode() if msg else "")


def _ptr(a):
    """(address, is_device) of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None, False
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, False
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), a.is_cuda
    raise TypeError(type(a))


def tp_version():
    return lib().tp_version().decode()


def tp_debug_tc_gemm(A_bits, B_bits, device=0):
    """D = A B^T through the tensor-core path: A [128,K], B [N,K] uint16 BF16 bit patterns."""
    A = np.ascontiguousarray(A_bits, dtype=np.uint16)
    B = np.ascontiguousarray(B_bits, dtype=np.uint16)
    K, N = A.shape[1], B.shape[0]
    D = np.zeros((128, N), np.float32)
    st = lib().tp_debug_tc_gemm(int(device), A.ctypes.data, K, B.ctypes.data, N, D.ctypes.data)
    if st != TP_OK:
        raise TPError(st, "tp_debug_tc_gemm failed")
    return D


def tp_measure_fp32_peak(device=0, stream=None, packed=True, warps_per_sm=64, chains=8):
    """Measured FP32 FMA throughput in TFLOP/s (see ``tp_measure_fp32_peak`` in tp.h)."""
    out = C.c_double(0.0)
    st = lib().tp_measure_fp32_peak(int(device), stream, int(bool(packed)), int(warps_per_sm), int(chains),
                                    C.byref(out))
    if st != TP_OK:
        raise TPError(st, "tp_measure_fp32_peak failed")
    return out.value


def tp_params_default(**kw):
    p = tp_params()
    lib().tp_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def tp_create(device=0, stream=None):
    """Context handle on ``device`` ordered on ``stream`` (a cudaStream_t integer or None)."""
    h = C.c_void_p()
    st = lib().tp_create(C.byref(h), int(device), C.c_void_p(stream or 0))
    if st != TP_OK:
        raise TPError(st, "tp_create failed")
    return h


def tp_destroy(ctx):
    if ctx:
        lib().tp_destroy(ctx)


def tp_last_error(ctx):
    return lib().tp_last_error(ctx).decode()


def tp_mesh_upload(ctx, V, F, flags=0):
    """V [nv,3] float32/float64, F [nt,3] int32; numpy (host) or CUDA tensors (device)."""
    pv, dv = _ptr(V)
    pf, df = _ptr(F) if F is not None else (None, dv)
    dtype = str(V.dtype)
    if dtype.endswith("float64"):
        vd = TP_DTYPE_F64
    elif dtype.endswith("float32"):
        vd = TP_DTYPE_F32
    else:
        raise TypeError(f"V must be float32 or float64, got {V.dtype}")
    if F is not None and not str(F.dtype).endswith("int32"):
        raise TypeError("F must be int32")
    if F is not None and dv != df:
        raise ValueError("V and F must both be host or both be device")
    if dv:
        flags |= TP_DEVICE_PTR
    nv = V.shape[0]
    nt = F.shape[0] if F is not None else 0
    _check(ctx, lib().tp_mesh_upload(ctx, pv, nv, vd, pf, nt, flags))


def tp_tree_build(ctx, leaf_size=16, morton_bits=30):
    _check(ctx, lib().tp_tree_build(ctx, leaf_size, morton_bits))


def tp_energy(ctx, params=None):
    p = params or tp_params_default()
    e = C.c_double(0.0)
    _check(ctx, lib().tp_energy(ctx, C.byref(p), C.byref(e)))
    return e.value


def tp_gradient(ctx, grad_out, params=None, want_energy=True):
    """Fill ``grad_out`` ([nv,3] float32/float64, host numpy or CUDA tensor); return the energy."""
    p = params or tp_params_default()
    pg, dg = _ptr(grad_out)
    gd = TP_DTYPE_F64 if str(grad_out.dtype).endswith("float64") else TP_DTYPE_F32
    e = C.c_double(0.0)
    _check(ctx, lib().tp_gradient(ctx, C.byref(p), C.byref(e) if want_energy else None, pg, gd,
                                  TP_DEVICE_PTR if dg else 0))
    return e.value if want_energy else None


def tp_fields(ctx, nt, params=None, fw=None, fnu=None, fx=None):
    """Per-triangle dPhi/dw [nt], dPhi/dnu [nt,3], dPhi/dx [nt,3] (float64, caller's
    triangle order).  Outputs may be given (all host numpy or all CUDA tensors);
    missing ones are allocated on the host.  Returns (energy, fw, fnu, fx)."""
    p = params or tp_params_default()
    given = [a for a in (fw, fnu, fx) if a is not None]
    dev = bool(given) and _ptr(given[0])[1]
    if not dev:
        fw = np.zeros(nt) if fw is None else fw
        fnu = np.zeros((nt, 3)) if fnu is None else fnu
        fx = np.zeros((nt, 3)) if fx is None else fx
    for a in (fw, fnu, fx):
        if a is not None and (not str(a.dtype).endswith("float64") or _ptr(a)[1] != dev):
            raise ValueError("outputs must be float64 and all on the host or all on the device")
    e = C.c_double(0.0)
    _check(ctx, lib().tp_fields(ctx, C.byref(p), C.byref(e), _ptr(fw)[0], _ptr(fnu)[0], _ptr(fx)[0],
                                TP_DEVICE_PTR if dev else 0))
    return e.value, fw, fnu, fx


def tp_set_quadrature(ctx, npoints):
    """Quadrature points per triangle (1, 3 or 6) for the next full mesh upload."""
    _check(ctx, lib().tp_set_quadrature(ctx, int(npoints)))


def tp_conf_upload(ctx, V, F):
    """Upload the fixed confining surface (numpy arrays or CUDA tensors; V f32/f64 [nv,3], F int32 [nt,3])."""
    pv, dv = _ptr(V)
    pf, df = _ptr(F)
    if dv != df:
        raise ValueError("V and F must both be on the host or both on the device")
    vd = TP_DTYPE_F64 if str(V.dtype).endswith("float64") else TP_DTYPE_F32
    _check(ctx, lib().tp_conf_upload(ctx, pv, V.shape[0], vd, pf, F.shape[0], TP_DEVICE_PTR if dv else 0))


def tp_conf_gradient(ctx, grad_out=None, params=None):
    """Confinement energy of the uploaded mesh against the confining surface; fills
    ``grad_out`` ([nv,3] float32/float64, host numpy or CUDA tensor) when given."""
    p = params or tp_params_default()
    e = C.c_double(0.0)
    if grad_out is None:
        _check(ctx, lib().tp_conf_gradient(ctx, C.byref(p), C.byref(e), None, TP_DTYPE_F64, 0))
    else:
        pg, dg = _ptr(grad_out)
        gd = TP_DTYPE_F64 if str(grad_out.dtype).endswith("float64") else TP_DTYPE_F32
        _check(ctx, lib().tp_conf_gradient(ctx, C.byref(p), C.byref(e), pg, gd, TP_DEVICE_PTR if dg else 0))
    return e.value


def tp_far_model_load(ctx, path):
    _check(ctx, lib().tp_far_model_load(ctx, os.fsencode(path)))


def tp_get_stats(ctx):
    s = tp_stats()
    _check(ctx, lib().tp_get_stats(ctx, C.byref(s)))
    return s.as_dict()


def tp_debug_tri_data(ctx, nt):
    perm = np.zeros(nt, dtype=np.int32)
    x = np.zeros((nt, 3))
    nu = np.zeros((nt, 3))
    w = np.zeros(nt)
    _check(ctx, lib().tp_debug_tri_data(ctx, perm.ctypes.data, x.ctypes.data, nu.ctypes.data, w.ctypes.data))
    return perm, x, nu, w


def tp_debug_accum(ctx, nt):
    gw = np.zeros(nt)
    gnu = np.zeros((nt, 3))
    gx = np.zeros((nt, 3))
    _check(ctx, lib().tp_debug_accum(ctx, gw.ctypes.data, gnu.ctypes.data, gx.ctypes.data))
    return gw, gnu, gx


def tp_set_learned_window(ctx, rows=0):
    """Listed far pairs per window of the learned passes (0: the default, 32 Mi rows)."""
    _check(ctx, lib().tp_set_learned_window(ctx, int(rows)))


def tp_debug_tree(ctx, nt):
    nn = 2 * nt - 1
    out = dict(codes=np.zeros(nt, np.uint32), perm=np.zeros(nt, np.int32), left=np.zeros(max(nt - 1, 1), np.int32),
               right=np.zeros(max(nt - 1, 1), np.int32), first=np.zeros(nn, np.int32), last=np.zeros(nn, np.int32),
               leaves=np.zeros(nt, np.int32), mom=np.zeros((nn, 13)), box=np.zeros((nn, 6)))
    nl = C.c_int64(0)
    _check(ctx, lib().tp_debug_tree(ctx, out["codes"].ctypes.data, out["perm"].ctypes.data, out["left"].ctypes.data,
                                    out["right"].ctypes.data, out["first"].ctypes.data, out["last"].ctypes.data,
                                    out["leaves"].ctypes.data, C.byref(nl), out["mom"].ctypes.data,
                                    out["box"].ctypes.data))
    out["leaves"] = out["leaves"][: nl.value]
    out["left"] = out["left"][: nt - 1]
    out["right"] = out["right"][: nt - 1]
    return out


def tp_debug_wait_timeout(ctx, limit_ms):
    """Make a device-side bounded wait run out (raises TPError with TP_E_TIMEOUT)."""
    _check(ctx, lib().tp_debug_wait_timeout(ctx, float(limit_ms)))


def tp_debug_sort(ctx, keys, bits=32, compact=False):
    """Stable sort of uint32 keys by their low ``bits`` bits with the library's own kernels:
    (sorted keys, input positions) and, with ``compact``, the entries >= 0 of the keys
    read as int32, in order."""
    k = np.ascontiguousarray(keys, dtype=np.uint32)
    n = k.shape[0]
    ko = np.zeros(n, dtype=np.uint32)
    po = np.zeros(n, dtype=np.int32)
    co = np.zeros(max(n, 1), dtype=np.int32)
    nc = C.c_int32(0)
    _check(ctx, lib().tp_debug_sort(ctx, k.ctypes.data, n, bits, ko.ctypes.data, po.ctypes.data,
                                    co.ctypes.data if compact else None, C.byref(nc) if compact else None))
    return (ko, po, co[: nc.value]) if compact else (ko, po)


def tp_debug_fail_alloc(ctx, after):
    """Fail the allocation after ``after`` more successful ones (negative: disarm)."""
    _check(ctx, lib().tp_debug_fail_alloc(ctx, int(after)))


def tp_gradient_direct_noalloc(V, F, energy_out, grad_out, params=None, stream=None):
    """Allocation-free direct energy + gradient: V [nv,3] f64, F [nt,3] int32,
    energy_out [1] f64 and grad_out [nv,3] f64, all CUDA tensors on the
    current device; ``stream`` a cudaStream_t integer (None: legacy default)."""
    import torch

    p = params or tp_params_default()
    for name, a in (("V", V), ("F", F), ("energy_out", energy_out), ("grad_out", grad_out)):
        if not isinstance(a, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
    if V.dtype != torch.float64 or energy_out.dtype != torch.float64 or grad_out.dtype != torch.float64:
        raise TypeError("V, energy_out and grad_out must be float64")
    if F.dtype != torch.int32:
        raise TypeError("F must be int32")
    if V.dim() != 2 or V.shape[1] != 3 or F.dim() != 2 or F.shape[1] != 3:
        raise ValueError("V must be [nv, 3] and F [nt, 3]")
    if tuple(grad_out.shape) != tuple(V.shape) or energy_out.numel() < 1:
        raise ValueError("grad_out must have V's shape and energy_out at least one element")
    for a in (V, F, energy_out, grad_out):
        if not (a.is_cuda and a.is_contiguous()):
            raise ValueError("all arguments must be contiguous CUDA tensors")
        if a.device.index != torch.cuda.current_device():
            raise ValueError("all arguments must be on the current CUDA device")
    buf = C.create_string_buffer(256)
    st = lib().tp_gradient_direct_noalloc(V.data_ptr(), V.shape[0], F.data_ptr(), F.shape[0], C.byref(p),
                                          energy_out.data_ptr(), grad_out.data_ptr(), C.c_void_p(stream or 0),
                                          buf, 256)
    if st != TP_OK:
        raise TPError(st, buf.value.decode())


# ---------------------------------------------------------------- learned far field
FAR_NPARAM = 10375


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None:
        a = a.reshape(shape)
    return a


def tp_far_model_init(ctx, seed=0):
    _check(ctx, lib().tp_far_model_init(ctx, seed))


def tp_far_model_save(ctx, path):
    _check(ctx, lib().tp_far_model_save(ctx, os.fsencode(path)))


def tp_far_set_params(ctx, params, norm=None):
    p = _f32(params, (FAR_NPARAM,))
    n = _f32(norm, (4, 24)) if norm is not None else None
    _check(ctx, lib().tp_far_set_params(ctx, p.ctypes.data, n.ctypes.data if n is not None else None))


def tp_far_get_params(ctx):
    p = np.zeros(FAR_NPARAM, np.float32)
    n = np.zeros((4, 24), np.float32)
    _check(ctx, lib().tp_far_get_params(ctx, p.ctypes.data, n.ctypes.data))
    return p, n


def tp_far_dataset_reset(ctx):
    _check(ctx, lib().tp_far_dataset_reset(ctx))


def tp_far_dataset_size(ctx):
    n = C.c_int64(0)
    _check(ctx, lib().tp_far_dataset_size(ctx, C.byref(n)))
    return n.value


def tp_far_sample_pairs(ctx, theta, keep, seed, max_pairs):
    n = C.c_int64(0)
    _check(ctx, lib().tp_far_sample_pairs(ctx, theta, keep, seed, max_pairs, C.byref(n)))
    return n.value


def tp_far_dataset_get(ctx, i0, n):
    f = np.zeros((n, 24), np.float32)
    lab = np.zeros((n, 8), np.float32)
    m = np.zeros((n, 8), np.float32)
    pr = np.zeros((n, 2), np.int32)
    _check(ctx, lib().tp_far_dataset_get(ctx, i0, n, f.ctypes.data, lab.ctypes.data, m.ctypes.data, pr.ctypes.data))
    return f, lab, m, pr


def tp_far_fit_normalisation(ctx):
    _check(ctx, lib().tp_far_fit_normalisation(ctx))


def tp_far_train(ctx, steps, batch, lr, wd=0.0, seed=0):
    loss = C.c_double(0.0)
    _check(ctx, lib().tp_far_train(ctx, steps, batch, lr, wd, seed, C.byref(loss)))
    return loss.value


def tp_far_eval(ctx, X, normalised=False, tgt=None, mask=None, mma_sync=False):
    X = _f32(X)
    n = X.shape[0]
    Y = np.zeros((n, 7), np.float32)
    g = np.zeros(FAR_NPARAM, np.float32)
    t = _f32(tgt) if tgt is not None else None
    m = _f32(mask) if mask is not None else None
    loss = C.c_double(0.0)
    _check(ctx, lib().tp_far_eval(ctx, X.ctypes.data, n, int(bool(normalised)) | (2 if mma_sync else 0),
                                  t.ctypes.data if t is not None else None,
                                  m.ctypes.data if m is not None else None, Y.ctypes.data, g.ctypes.data,
                                  C.byref(loss)))
    return Y, g, loss.value


def tp_far_adamw_step(ctx, grad, lr, wd=0.0):
    g = _f32(grad, (FAR_NPARAM,))
    _check(ctx, lib().tp_far_adamw_step(ctx, g.ctypes.data, lr, wd))
