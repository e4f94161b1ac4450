"""Thin Python binding of the C ABI in include/lbm.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing but
convert arguments (numpy arrays, torch tensors, Python numbers) into pointers and sizes,
call the library, and turn a non-zero status into an ``LbmError``.  All computation runs
in the CUDA kernels of ``liblbm.so``; there is no fallback: if the library is missing the
first call raises.

PyTorch is used only for device memory and streams: a CUDA tensor is passed by its
``data_ptr()`` with ``on_device = 1``, and the default stream of a handle is torch's
current stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY may name another build of the library (the bounds-checked liblbm_check.so)
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(_HERE, "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ESTATE, LBM_EUNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6
PRECISION = {"f32": 0, "f16": 1, "bf16": 2}
STREAMING = {"aa": 0, "pull": 1}
PIPELINE = {"tma": 0, "direct": 1, "prefetch": 2, "async": 3}
COLLISION = {"trt": 0, "mrt": 1, "reg": 2}
CLOSURE = {"none": 0, "smag": 1, "mlp": 2}
FACE = {"periodic": 0, "wall": 1, "freeslip": 2, "inflow": 3, "outflow": 4, "halo": 5}
CELL = {"fluid": 0, "solid": 1, "inflow": 2}
MLP_NPARAM = 1345
STATS_K = 10

_STATUS_NAMES = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA",
                 -4: "LBM_EUNSTABLE", -5: "LBM_ESTATE", -6: "LBM_EUNSUPPORTED"}


class LbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("precision", ctypes.c_int32),
        ("streaming", ctypes.c_int32),
        ("closure", ctypes.c_int32),
        ("magic_lambda", ctypes.c_double),
        ("cs_smag", ctypes.c_double),
        ("face_bc", ctypes.c_int32 * 6),
        ("u_inflow", ctypes.c_double * 3),
        ("rho_inflow", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("pipeline", ctypes.c_int32),
        ("collision", ctypes.c_int32),
        ("mrt_rates", ctypes.c_double * 5),
    ]


_lock = threading.Lock()
_lib = None


def load():
    """Loads liblbm.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(the CUDA library is required; there is no CPU path)")
        L = ctypes.CDLL(LIB_PATH)
        H, P, I, D = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        sig = {
            "lbm_params_default": (None, [ctypes.POINTER(lbm_params)]),
            "lbm_stencil": (I, [I, P, P]),
            "lbm_create": (I, [I, I, I, I, D, ctypes.POINTER(lbm_params), ctypes.POINTER(H)]),
            "lbm_destroy": (I, [H]),
            "lbm_set_flags": (I, [H, P, I]),
            "lbm_set_force": (I, [H, D, D, D]),
            "lbm_init_equilibrium": (I, [H, P, P, I]),
            "lbm_step": (I, [H, ctypes.c_int64]),
            "lbm_sync": (I, [H]),
            "lbm_debug_set_wait_polls": (I, [H, ctypes.c_int64]),
            "lbm_moments": (I, [H, P, P, I]),
            "lbm_get_populations": (I, [H, P, I]),
            "lbm_set_populations": (I, [H, P, I]),
            "lbm_reduce": (I, [H, P]),
            "lbm_stats_reset": (I, [H]),
            "lbm_stats_sample": (I, [H]),
            "lbm_step_stats": (I, [H, ctypes.c_int64, ctypes.c_int64]),
            "lbm_stats_get": (I, [H, P, ctypes.POINTER(ctypes.c_int64)]),
            "lbm_set_closure": (I, [H, P, I, D, D]),
            "lbm_info": (I, [H, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D)]),
            "lbm_last_error": (ctypes.c_char_p, [H]),
            "lbm_halo_bytes": (ctypes.c_size_t, [H, I]),
            "lbm_halo_pack": (I, [H, I, P]),
            "lbm_halo_unpack": (I, [H, I, P]),
            "lbm_refine_explode": (I, [H, I, H, I, I]),
            "lbm_refine_coalesce": (I, [H, I, H, I]),
            "lbm_get_post_collision": (I, [H, P, I]),
            "lbm_reduce_noalloc": (I, [P, P, I, I, I, I, P, P, P]),
            "lbm_set_closure_f32": (I, [H, P, I, D, D]),
            "lbm_set_closure_floor": (I, [H, D]),
            "lbm_closure_samples": (I, [H, D, D, P, P, P, P, P]),
            "lbm_mlp_forward": (I, [P, P, ctypes.c_int64, P, P]),
            "lbm_filter2": (I, [H, P, P]),
            "lbm_mlp_backward": (I, [P, P, P, ctypes.c_int64, P, P]),
            "lbm_closure_loss_grad": (I, [P, P, P, P, P, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int64, D, P, P, P]),
            "lbm_adam_step": (I, [P, P, P, P, I, D, D, D, D, ctypes.c_int64, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _check(status: int, h=None):
    if status != LBM_OK:
        msg = load().lbm_last_error(h)
        raise LbmError(status, msg.decode() if msg else "")


def _buf(a, dtype, writable=False):
    """(pointer, on_device) of a numpy array or torch tensor of the given numpy dtype."""
    if a is None:
        return None, 0
    mod = type(a).__module__
    if mod.startswith("torch"):
        import torch

        tdt = {np.float32: torch.float32, np.uint8: torch.uint8, np.uint16: torch.uint16
               if hasattr(torch, "uint16") else torch.int16, np.float64: torch.float64}[dtype]
        if a.dtype != tdt and not (dtype is np.uint16 and a.dtype == torch.int16):
            raise TypeError(f"expected a {tdt} tensor, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda)
    if not isinstance(a, np.ndarray):
        raise TypeError("expected a numpy array or a torch tensor")
    if a.dtype != dtype:
        raise TypeError(f"expected dtype {np.dtype(dtype)}, got {a.dtype}")
    if not a.flags.c_contiguous:
        raise ValueError("array must be C-contiguous")
    if writable and not a.flags.writeable:
        raise ValueError("array must be writable")
    return a.ctypes.data_as(ctypes.c_void_p), 0


def _current_stream():
    try:
        import torch

        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


# ---- entry points (same names as the C ABI) ------------------------------------------------

def lbm_params_default(precision="f32", streaming="aa", closure="none", magic_lambda=3.0 / 16.0,
                       cs_smag=0.1, faces=("periodic",) * 6, u_inflow=(0.0, 0.0, 0.0),
                       rho_inflow=1.0, stream=None, pipeline="direct", collision="trt",
                       mrt_rates=None) -> lbm_params:
    p = lbm_params()
    load().lbm_params_default(ctypes.byref(p))
    p.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    p.streaming = STREAMING[streaming] if isinstance(streaming, str) else int(streaming)
    p.closure = CLOSURE[closure] if isinstance(closure, str) else int(closure)
    p.magic_lambda = float(magic_lambda)
    p.cs_smag = float(cs_smag)
    for k in range(6):
        p.face_bc[k] = FACE[faces[k]] if isinstance(faces[k], str) else int(faces[k])
    for a in range(3):
        p.u_inflow[a] = float(u_inflow[a])
    p.rho_inflow = float(rho_inflow)
    p.stream = stream if stream is not None else _current_stream()
    p.pipeline = PIPELINE[pipeline] if isinstance(pipeline, str) else int(pipeline)
    p.collision = COLLISION[collision] if isinstance(collision, str) else int(collision)
    if mrt_rates is not None:
        for k in range(5):
            p.mrt_rates[k] = float(mrt_rates[k])
    return p


def lbm_stencil(q: int):
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q, dtype=np.float64)
    if load().lbm_stencil(q, c.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p)) != q:
        raise ValueError(f"unsupported stencil {q}")
    return c, w


def lbm_create(nx, ny, nz, stencil, tau, params: lbm_params | None = None):
    h = ctypes.c_void_p()
    st = load().lbm_create(int(nx), int(ny), int(nz), int(stencil), float(tau),
                           ctypes.byref(params) if params is not None else None, ctypes.byref(h))
    _check(st, None)
    return h


def lbm_destroy(h):
    _check(load().lbm_destroy(h), h)


def lbm_set_flags(h, flags):
    p, dev = _buf(flags, np.uint8)
    _check(load().lbm_set_flags(h, p, dev), h)


def lbm_set_force(h, fx, fy, fz):
    _check(load().lbm_set_force(h, float(fx), float(fy), float(fz)), h)


def lbm_init_equilibrium(h, rho=None, u=None):
    pr, dr = _buf(rho, np.float32)
    pu, du = _buf(u, np.float32)
    if rho is not None and u is not None and dr != du:
        raise ValueError("rho and u must both be host or both be device buffers")
    _check(load().lbm_init_equilibrium(h, pr, pu, dr or du), h)


def lbm_step(h, n: int):
    _check(load().lbm_step(h, int(n)), h)


def lbm_sync(h):
    _check(load().lbm_sync(h), h)


def lbm_debug_set_wait_polls(h, polls: int):
    _check(load().lbm_debug_set_wait_polls(h, int(polls)), h)


def lbm_moments(h, rho=None, u=None):
    pr, dr = _buf(rho, np.float32, True)
    pu, du = _buf(u, np.float32, True)
    if rho is not None and u is not None and dr != du:
        raise ValueError("rho and u must both be host or both be device buffers")
    _check(load().lbm_moments(h, pr, pu, dr or du), h)


def lbm_get_populations(h, df):
    p, dev = _buf(df, np.float32, True)
    _check(load().lbm_get_populations(h, p, dev), h)


def lbm_get_post_collision(h, df):
    p, dev = _buf(df, np.float32, True)
    _check(load().lbm_get_post_collision(h, p, dev), h)


def lbm_refine_explode(coarse, coarse_face: int, fine, fine_face: int, substep: int):
    _check(load().lbm_refine_explode(coarse, int(coarse_face), fine, int(fine_face), int(substep)), fine)


def lbm_refine_coalesce(fine, fine_face: int, coarse, coarse_face: int):
    _check(load().lbm_refine_coalesce(fine, int(fine_face), coarse, int(coarse_face)), coarse)


def lbm_set_populations(h, df):
    p, dev = _buf(df, np.float32)
    _check(load().lbm_set_populations(h, p, dev), h)


def lbm_reduce(h) -> np.ndarray:
    out = np.zeros(4, dtype=np.float64)
    _check(load().lbm_reduce(h, out.ctypes.data_as(ctypes.c_void_p)), h)
    return out


def lbm_stats_reset(h):
    _check(load().lbm_stats_reset(h), h)


def lbm_stats_sample(h):
    _check(load().lbm_stats_sample(h), h)


def lbm_halo_bytes(h, face: int) -> int:
    return int(load().lbm_halo_bytes(h, int(face)))


def _raw_ptr(buf):
    """Address of a contiguous torch tensor or numpy array (any dtype: the halo buffers hold
    storage-precision values as raw bytes)."""
    if type(buf).__module__.startswith("torch"):
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size()
    if not isinstance(buf, np.ndarray) or not buf.flags.c_contiguous:
        raise TypeError("expected a contiguous numpy array or torch tensor")
    return ctypes.c_void_p(buf.ctypes.data), buf.nbytes


def lbm_halo_pack(h, face: int, buf):
    ptr, nbytes = _raw_ptr(buf)
    if nbytes < lbm_halo_bytes(h, face):
        raise ValueError("halo buffer too small")
    _check(load().lbm_halo_pack(h, int(face), ptr), h)


def lbm_halo_unpack(h, face: int, buf):
    ptr, nbytes = _raw_ptr(buf)
    if nbytes < lbm_halo_bytes(h, face):
        raise ValueError("halo buffer too small")
    _check(load().lbm_halo_unpack(h, int(face), ptr), h)


def lbm_step_stats(h, n: int, every: int):
    _check(load().lbm_step_stats(h, int(n), int(every)), h)


def lbm_stats_get(h, ny: int):
    out = np.zeros((ny, STATS_K), dtype=np.float64)
    n = ctypes.c_int64(0)
    _check(load().lbm_stats_get(h, out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)), h)
    return out, int(n.value)


def lbm_set_closure(h, bf16_params: np.ndarray, scale_pi: float, scale_rho: float):
    a = np.ascontiguousarray(bf16_params, dtype=np.uint16)
    _check(load().lbm_set_closure(h, a.ctypes.data_as(ctypes.c_void_p), int(a.size),
                                  float(scale_pi), float(scale_rho)), h)


def lbm_info(h):
    nxp, bpp, bpu = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    _check(load().lbm_info(h, ctypes.byref(nxp), ctypes.byref(bpp), ctypes.byref(bpu)), h)
    return nxp.value, bpp.value, bpu.value


def lbm_reduce_noalloc(df, flags, nx, ny, nz, stencil, force=(0.0, 0.0, 0.0), stream=None):
    """FP64 sums of a caller-held population array without any allocation by the library
    (out is a host array owned here).  df (q*nx*ny*nz float32) and flags (nx*ny*nz uint8, or
    None) must be CUDA tensors on the current device; sizes and devices are checked here,
    since the C call can only trust the pointers it is given."""
    import torch

    pd, dd = _buf(df, np.float32)
    pf, df_ = _buf(flags, np.uint8) if flags is not None else (None, 1)
    if not dd or not df_:
        raise ValueError("df and flags must be device buffers")
    n = int(nx) * int(ny) * int(nz)
    if n > 0 and df.numel() < int(stencil) * n:
        raise ValueError(f"df holds {df.numel()} values, {int(stencil) * n} needed")
    if flags is not None and n > 0 and flags.numel() < n:
        raise ValueError(f"flags holds {flags.numel()} values, {n} needed")
    dev = torch.cuda.current_device()
    for name, t in (("df", df), ("flags", flags)):
        if t is not None and t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")
    fv = np.ascontiguousarray(force, dtype=np.float64)
    out = np.zeros(4, dtype=np.float64)
    st = stream if stream is not None else _current_stream()
    _check(load().lbm_reduce_noalloc(pd, pf, int(nx), int(ny), int(nz), int(stencil),
                                     fv.ctypes.data_as(ctypes.c_void_p),
                                     out.ctypes.data_as(ctypes.c_void_p), st), None)
    return out


def _dev(a, dtype=np.float32):
    p, dev = _buf(a, dtype)
    if not dev:
        raise ValueError("expected a CUDA tensor")
    return p


def lbm_set_closure_f32(h, params, scale_pi: float, scale_rho: float):
    p, dev = _buf(params, np.float32)
    _check(load().lbm_set_closure_f32(h, p, dev, float(scale_pi), float(scale_rho)), h)


def lbm_set_closure_floor(h, cs_min: float):
    _check(load().lbm_set_closure_floor(h, float(cs_min)), h)


def lbm_closure_samples(h, tau0_c, cs0, scale, x, target, smag, weight):
    sc = np.ascontiguousarray(scale, dtype=np.float64)
    _check(load().lbm_closure_samples(h, float(tau0_c), float(cs0), sc.ctypes.data_as(ctypes.c_void_p),
                                      _dev(x), _dev(target), _dev(smag), _dev(weight)), h)


def lbm_filter2(h, rho_bar, u_bar):
    _check(load().lbm_filter2(h, _dev(rho_bar), _dev(u_bar)), h)


def lbm_mlp_forward(params, x, n, y, stream=None):
    st = stream if stream is not None else _current_stream()
    _check(load().lbm_mlp_forward(_dev(params), _dev(x), int(n), _dev(y), st), None)


def lbm_mlp_backward(params, x, dy, n, grad, stream=None):
    st = stream if stream is not None else _current_stream()
    _check(load().lbm_mlp_backward(_dev(params), _dev(x), _dev(dy), int(n), _dev(grad), st), None)


def lbm_closure_loss_grad(params, x, target, smag, weight, n, offset, stride, cs0, grad, stream=None):
    st = stream if stream is not None else _current_stream()
    loss = ctypes.c_double(0.0)
    _check(load().lbm_closure_loss_grad(_dev(params), _dev(x), _dev(target), _dev(smag), _dev(weight),
                                        int(n), int(offset), int(stride), float(cs0), _dev(grad),
                                        ctypes.byref(loss), st), None)
    return loss.value


def lbm_adam_step(params, grad, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    st = stream if stream is not None else _current_stream()
    n = params.numel() if hasattr(params, "numel") else params.size
    _check(load().lbm_adam_step(_dev(params), _dev(grad), _dev(m), _dev(v), int(n), float(lr),
                                float(beta1), float(beta2), float(eps), int(t), st), None)


def lbm_last_error(h=None) -> str:
    m = load().lbm_last_error(h)
    return m.decode() if m else ""


# ---- convenience wrapper ---------------------------------------------------------------------

class Lattice:
    """Owns one handle; arrays use the (q|3, nz, ny, nx) shapes of the C ABI."""

    def __init__(self, nx, ny, nz, stencil=19, tau=0.8, **params):
        self.nx, self.ny, self.nz, self.q = int(nx), int(ny), int(nz), int(stencil)
        self.params = lbm_params_default(**params)
        self.h = lbm_create(nx, ny, nz, stencil, tau, self.params)
        self.nxp, self.bytes_per_pop, self.bytes_per_update = lbm_info(self.h)

    @property
    def ncell(self):
        return self.nx * self.ny * self.nz

    def close(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_flags(self, flags):
        lbm_set_flags(self.h, flags)

    def set_force(self, fx, fy=0.0, fz=0.0):
        lbm_set_force(self.h, fx, fy, fz)

    def init_equilibrium(self, rho=None, u=None):
        lbm_init_equilibrium(self.h, rho, u)

    def step(self, n=1):
        lbm_step(self.h, n)

    def sync(self):
        lbm_sync(self.h)

    def moments(self):
        rho = np.zeros((self.nz, self.ny, self.nx), dtype=np.float32)
        u = np.zeros((3, self.nz, self.ny, self.nx), dtype=np.float32)
        lbm_moments(self.h, rho, u)
        return rho, u

    def get_populations(self):
        df = np.zeros((self.q, self.nz, self.ny, self.nx), dtype=np.float32)
        lbm_get_populations(self.h, df)
        return df

    def get_post_collision(self):
        df = np.zeros((self.q, self.nz, self.ny, self.nx), dtype=np.float32)
        lbm_get_post_collision(self.h, df)
        return df

    def set_populations(self, df):
        lbm_set_populations(self.h, np.ascontiguousarray(df, dtype=np.float32))

    def reduce(self):
        return lbm_reduce(self.h)
