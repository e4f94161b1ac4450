"""FP64 CPU oracle of the lattice Boltzmann stream-and-collide update.

TEST INFRASTRUCTURE ONLY: this package is the plain, slow reference the CUDA library is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA path.

The arithmetic lives in ``lbm_oracle.c`` (plain C, double precision, loops in the order
of the paper's Eq. LBCollision then Eq. LBStreaming, Sec. 2); this module compiles it
with gcc and exposes it on numpy arrays.

Array conventions: populations ``f`` have shape (q, nz, ny, nx), x fastest, holding the
plain (unshifted) pre-collision values; velocities have shape (3, nz, ny, nx).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FACE = {"periodic": 0, "wall": 1, "freeslip": 2, "inflow": 3, "outflow": 4}
CELL = {"fluid": 0, "solid": 1, "inflow": 2}
CLOSURE = {"none": 0, "smag": 1, "mlp": 2}
MLP_NPARAM = 32 * 7 + 32 + 32 * 32 + 32 + 32 + 1
CFLAGS = ["-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-D_GNU_SOURCE"]


def build(force: bool = False) -> str:
    """Compiles liboracle.so with gcc (OpenMP, no FMA contraction)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lbm_oracle.h"))):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def mrt_matrix():
    """The oracle's 19 x 19 D3Q19 MRT moment basis M[k][i]."""
    return np.array([[lib().ora_mrt_row(k, i) for i in range(19)] for k in range(19)])


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("q", ctypes.c_int),
        ("tau", ctypes.c_double), ("lam", ctypes.c_double),
        ("closure", ctypes.c_int),
        ("cs", ctypes.c_double),
        ("face", ctypes.c_int * 6),
        ("u_w", ctypes.c_double * 3),
        ("rho_w", ctypes.c_double),
        ("force", ctypes.c_double * 3),
        ("flags", ctypes.c_void_p),
        ("mlp", ctypes.c_void_p),
        ("mlp_scale", ctypes.c_double * 2),
        ("mlp_cs_min", ctypes.c_double),
        ("collision", ctypes.c_int),
        ("mrt_s", ctypes.c_double * 5),
    ]


def load(path: str):
    """Loads a compiled copy of the oracle from ``path`` and declares its functions."""
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    L.ora_stencil.argtypes = [ctypes.c_int, P, P, P]
    L.ora_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, P, P]
    L.ora_smag_tau.argtypes = [ctypes.c_double] * 4
    L.ora_smag_tau.restype = ctypes.c_double
    L.ora_collide.argtypes = [P, P, P, P]
    L.ora_mrt_row.argtypes = [ctypes.c_int, ctypes.c_int]
    L.ora_mrt_row.restype = ctypes.c_double
    L.ora_moments_cell.argtypes = [P, P, P, P]
    L.ora_check.argtypes = [P]
    L.ora_step.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int]
    L.ora_stream.argtypes = [P, P, P, ctypes.c_int]
    L.ora_collide_all.argtypes = [P, P, P, ctypes.c_int]
    L.ora_init_equilibrium.argtypes = [P, P, P, P]
    L.ora_moments.argtypes = [P, P, P, P]
    L.ora_mass_momentum.argtypes = [P, P, P]
    L.ora_step_sampled.argtypes = [P, P, P, P, ctypes.c_int64, P]
    L.ora_step_sampled_pop.argtypes = [P, P, P, ctypes.c_int64, P]
    L.ora_stats_sample.argtypes = [P, P, P]
    L.ora_mlp_forward.argtypes = [P, P, P, P, P, P]
    L.ora_mlp_forward.restype = ctypes.c_double
    L.ora_mlp_backward.argtypes = [P, P, ctypes.c_double, P]
    L.ora_mlp_features.argtypes = [P, P, P]
    L.ora_closure_samples.argtypes = [P, P, ctypes.c_double, ctypes.c_double, P, P, P, P, P]
    L.ora_closure_loss.argtypes = [P, P, P, P, P, ctypes.c_int64, ctypes.c_double, P]
    L.ora_closure_loss.restype = ctypes.c_double
    L.ora_filter2.argtypes = [P, P, P, P]
    L.ora_adam.argtypes = [P, P, P, P, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                           ctypes.c_double, ctypes.c_double, ctypes.c_int64]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = load(_SO)
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def stencil(q: int):
    """(c[q,3] int, w[q] float64, opp[q] int) in the published direction order."""
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q, dtype=np.float64)
    o = np.zeros(q, dtype=np.int32)
    if lib().ora_stencil(q, _ptr(c), _ptr(w), _ptr(o)) != q:
        raise ValueError(f"unsupported stencil {q}")
    return c, w, o


def equilibrium(q: int, rho: float, u) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(q, dtype=np.float64)
    lib().ora_equilibrium(q, float(rho), _ptr(u), _ptr(out))
    return out


def smag_tau(tau0: float, cs2: float, qn: float, rho: float) -> float:
    return lib().ora_smag_tau(tau0, cs2, qn, rho)


def mlp_forward(params: np.ndarray, x: np.ndarray) -> float:
    params = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().ora_mlp_forward(_ptr(params), _ptr(x), None, None, None, None)


def mlp_backward(params: np.ndarray, x: np.ndarray, dy: float) -> np.ndarray:
    params = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.zeros(MLP_NPARAM, dtype=np.float64)
    lib().ora_mlp_backward(_ptr(params), _ptr(x), float(dy), _ptr(g))
    return g


def closure_loss(params, x, target, smag, weight, cs0):
    """(L, dL/dparams) of the weighted eddy-viscosity MSE (FP64)."""
    params = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    t = np.ascontiguousarray(target, dtype=np.float64)
    sm = np.ascontiguousarray(smag, dtype=np.float64)
    w = np.ascontiguousarray(weight, dtype=np.float64)
    g = np.zeros(MLP_NPARAM, dtype=np.float64)
    loss = lib().ora_closure_loss(_ptr(params), _ptr(x), _ptr(t), _ptr(sm), _ptr(w), t.size,
                                  float(cs0), _ptr(g))
    return loss, g


def adam(p, g, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step in place on float64 arrays p, m, v (t is 1-based)."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = np.ascontiguousarray(g, dtype=np.float64)
    lib().ora_adam(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.size, float(lr), float(beta1),
                   float(beta2), float(eps), int(t))


class Oracle:
    """One lattice held on the host in FP64 (plain populations, shape (q, nz, ny, nx))."""

    def __init__(self, nx, ny, nz, q=19, tau=0.8, lam=3.0 / 16.0, closure="none", cs=0.0,
                 faces=("periodic",) * 6, u_w=(0.0, 0.0, 0.0), rho_w=1.0,
                 force=(0.0, 0.0, 0.0), flags=None, mlp=None, mlp_scale=(1.0, 1.0), mlp_cs_min=0.0,
                 collision="trt", mrt_s=(1.19, 1.4, 1.2, 1.4, 1.98)):
        self.nx, self.ny, self.nz, self.q = int(nx), int(ny), int(nz), int(q)
        self.N = self.nx * self.ny * self.nz
        self._flags = None
        if flags is not None:
            fl = np.ascontiguousarray(flags, dtype=np.uint8).reshape(self.nz, self.ny, self.nx)
            if fl.max(initial=0) > 2:
                raise ValueError("unknown cell flag")
            self._flags = fl
        self._mlp = None if mlp is None else np.ascontiguousarray(mlp, dtype=np.float64)
        if self._mlp is not None and self._mlp.size != MLP_NPARAM:
            raise ValueError("MLP parameter count")
        c = _Cfg()
        c.nx, c.ny, c.nz, c.q = self.nx, self.ny, self.nz, self.q
        c.tau, c.lam = float(tau), float(lam)
        c.closure = CLOSURE[closure]
        c.cs = float(cs)
        for k in range(6):
            c.face[k] = FACE[faces[k]]
        for a in range(3):
            c.u_w[a] = float(u_w[a])
            c.force[a] = float(force[a])
        c.rho_w = float(rho_w)
        c.flags = None if self._flags is None else self._flags.ctypes.data
        c.mlp = None if self._mlp is None else self._mlp.ctypes.data
        c.mlp_scale[0], c.mlp_scale[1] = float(mlp_scale[0]), float(mlp_scale[1])
        c.mlp_cs_min = float(mlp_cs_min)
        c.collision = {"trt": 0, "mrt": 1, "reg": 2}[collision]
        for k in range(5):
            c.mrt_s[k] = float(mrt_s[k])
        self.cfg = c
        rc = lib().ora_check(ctypes.byref(c))
        if rc != 0:
            raise ValueError(f"invalid oracle configuration ({rc})")
        _, w, _ = stencil(self.q)
        self.w = w
        self.f = np.empty((self.q, self.nz, self.ny, self.nx), dtype=np.float64)
        self.f[:] = w[:, None, None, None]
        self._work = None

    @property
    def flags(self):
        if self._flags is None:
            return np.zeros((self.nz, self.ny, self.nx), dtype=np.uint8)
        return self._flags

    def init_equilibrium(self, rho, u):
        rho = np.ascontiguousarray(np.broadcast_to(rho, (self.nz, self.ny, self.nx)), dtype=np.float64)
        u = np.asarray(u, dtype=np.float64)
        if u.ndim == 1:
            u = u.reshape(3, 1, 1, 1)
        u = np.ascontiguousarray(np.broadcast_to(u, (3, self.nz, self.ny, self.nx)), dtype=np.float64)
        lib().ora_init_equilibrium(ctypes.byref(self.cfg), _ptr(rho), _ptr(u), _ptr(self.f))

    def set_shifted(self, df):
        """Sets f = w + df (df shaped like f, e.g. the FP32 values a GPU state holds)."""
        self.f[:] = self.w[:, None, None, None] + np.asarray(df, dtype=np.float64)

    def shifted(self):
        return self.f - self.w[:, None, None, None]

    def step(self, n=1, threads=None):
        if self._work is None:
            self._work = np.empty_like(self.f)
        if threads is None:
            threads = os.cpu_count() or 1
        rc = lib().ora_step(ctypes.byref(self.cfg), _ptr(self.f), _ptr(self._work), int(n), int(threads))
        if rc != 0:
            raise RuntimeError("oracle step failed")

    def stream(self, fstar, threads=1):
        """Eq. LBStreaming alone applied to a post-collision array shaped like f."""
        fstar = np.ascontiguousarray(fstar, dtype=np.float64).reshape(self.f.shape)
        if lib().ora_stream(ctypes.byref(self.cfg), _ptr(fstar), _ptr(self.f), int(threads)) != 0:
            raise RuntimeError("oracle stream failed")

    def collide_all(self, f=None, threads=1):
        """Eq. LBCollision alone on every fluid cell of f (default: the state); returns f*."""
        f = self.f if f is None else np.ascontiguousarray(f, dtype=np.float64).reshape(self.f.shape)
        out = np.empty_like(f)
        if lib().ora_collide_all(ctypes.byref(self.cfg), _ptr(f), _ptr(out), int(threads)) != 0:
            raise RuntimeError("oracle collision failed")
        return out

    def moments(self):
        rho = np.empty((self.nz, self.ny, self.nx), dtype=np.float64)
        u = np.empty((3, self.nz, self.ny, self.nx), dtype=np.float64)
        lib().ora_moments(ctypes.byref(self.cfg), _ptr(self.f), _ptr(rho), _ptr(u))
        return rho, u

    def mass_momentum(self):
        out = np.zeros(4, dtype=np.float64)
        lib().ora_mass_momentum(ctypes.byref(self.cfg), _ptr(self.f), _ptr(out))
        return out

    def stats_sample(self, acc=None):
        if acc is None:
            acc = np.zeros((self.ny, 10), dtype=np.float64)
        lib().ora_stats_sample(ctypes.byref(self.cfg), _ptr(self.f), _ptr(acc))
        return acc

    def collide_cell(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros(self.q, dtype=np.float64)
        tau = ctypes.c_double(0.0)
        lib().ora_collide(ctypes.byref(self.cfg), _ptr(f), _ptr(out), ctypes.byref(tau))
        return out, tau.value

    def features_cell(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        x = np.zeros(7, dtype=np.float64)
        lib().ora_mlp_features(ctypes.byref(self.cfg), _ptr(f), _ptr(x))
        return x

    def closure_samples(self, tau0_c, cs0, scale=(1.0, 1.0)):
        """Box-filter-2 training samples for the coarse grid from the current state.

        Returns x (nc, 7), target nu*, |S_c|, weight, with nc = (nx/2)(ny/2)(nz/2)."""
        nc = (self.nx // 2) * (self.ny // 2) * (self.nz // 2)
        x = np.zeros((nc, 7))
        t, sm, w = np.zeros(nc), np.zeros(nc), np.zeros(nc)
        sc = np.ascontiguousarray(scale, dtype=np.float64)
        lib().ora_closure_samples(ctypes.byref(self.cfg), _ptr(self.f), float(tau0_c), float(cs0),
                                  _ptr(sc), _ptr(x), _ptr(t), _ptr(sm), _ptr(w))
        return x, t, sm, w

    def filter2(self):
        """Box-filter-2 density (nzc, nyc, nxc) and Favre velocity (3, nzc, nyc, nxc)."""
        shp = (self.nz // 2, self.ny // 2, self.nx // 2)
        rb = np.zeros(shp)
        ub = np.zeros((3,) + shp)
        lib().ora_filter2(ctypes.byref(self.cfg), _ptr(self.f), _ptr(rb), _ptr(ub))
        return rb, ub

    def step_sampled(self, rho_in, u_in, cells):
        """One step from f = f^eq(rho_in, u_in) (float32 fields), at the listed linear cells.

        Returns an array (len(cells), q) of plain populations f_i(x, t+1)."""
        rho_in = np.ascontiguousarray(rho_in, dtype=np.float32)
        u_in = np.ascontiguousarray(u_in, dtype=np.float32)
        assert rho_in.size == self.N and u_in.size == 3 * self.N
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.zeros((cells.size, self.q), dtype=np.float64)
        lib().ora_step_sampled(ctypes.byref(self.cfg), _ptr(rho_in), _ptr(u_in), _ptr(cells),
                               cells.size, _ptr(out))
        return out

    def step_sampled_pop(self, df, cells):
        """One step from f = w + df (df: shifted float32 populations of every cell, shaped like
        f), at the listed linear cells.  Returns an array (len(cells), q) of plain f_i(x, t+1)."""
        df = np.ascontiguousarray(df, dtype=np.float32)
        assert df.size == self.q * self.N
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.zeros((cells.size, self.q), dtype=np.float64)
        lib().ora_step_sampled_pop(ctypes.byref(self.cfg), _ptr(df), _ptr(cells), cells.size, _ptr(out))
        return out
