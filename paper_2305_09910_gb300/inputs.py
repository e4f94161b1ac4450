"""Seeded synthetic inputs shaped like the paper's benchmark cases (Sec. 5.1, Sec. 5.2).

This module holds input generation only -- no lattice Boltzmann arithmetic -- and serves
both the CUDA library and the FP64 oracle, which receive identical arrays from it.  The
paper's channel data (Hoyas DNS) and the LAGOON landing-gear geometry are not available,
so synthetic stand-ins with the shapes of those cases are generated here:

* turbulent channel (Sec. 5.1): laminar parabola + seeded sinusoidal perturbation +
  uniform noise of +/-5 % of the bulk velocity, walls at the +/-y faces;
* landing-gear-like bluff body (Sec. 5.2): strut, axle, two wheels and 3-6 seeded boxes
  voxelised into a uint8 flag field.

Random numbers come from a counter-based generator (the splitmix64 finaliser of
Steele, Lea and Flood 2014 applied to seed + (counter + 1) * golden-ratio increment), so
any cell's value can be regenerated from (seed, stream, index) alone.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
DEFAULT_SEED = 20230509


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, stream: int, index) -> np.ndarray:
    """Uniform doubles in [0, 1) for counter values ``index`` of a (seed, stream) pair."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(stream & 0xFFFF) << np.uint64(48))
        z = _mix(base + (idx + np.uint64(1)) * GOLDEN)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_field(seed: int, stream: int, shape, lo: float, hi: float, dtype=np.float64):
    n = int(np.prod(shape))
    return (lo + (hi - lo) * uniform01(seed, stream, np.arange(n, dtype=np.uint64))).reshape(shape).astype(dtype)


# ---- cases --------------------------------------------------------------------------------

def poiseuille_flags(nx: int, ny: int, nz: int) -> np.ndarray:
    """Channel with solid rows at y = 0 and y = ny - 1 (walls halfway, H = ny - 2)."""
    f = np.zeros((nz, ny, nx), dtype=np.uint8)
    f[:, 0, :] = 1
    f[:, ny - 1, :] = 1
    return f


def channel_parameters(ny: int, re_tau: float = 180.0, u_bulk: float = 0.05):
    """tau and body force for a channel of half-height delta = ny/2 (walls at the y faces).

    The bulk Reynolds number follows from Re_tau through Dean's correlation
    Re_tau = 0.09 Re_b^0.88 (Re_b = 2 delta u_b / nu); u_tau = Re_tau nu / delta and the
    driving force per unit mass balances the wall stress, g = u_tau^2 / delta."""
    delta = ny / 2.0
    re_b = (re_tau / 0.09) ** (1.0 / 0.88)
    nu = 2.0 * delta * u_bulk / re_b
    u_tau = re_tau * nu / delta
    return {"tau": 3.0 * nu + 0.5, "nu": nu, "force": u_tau * u_tau / delta, "u_tau": u_tau,
            "re_b": re_b, "delta": delta}


def channel_init(nx: int, ny: int, nz: int, u_bulk: float = 0.05, seed: int = DEFAULT_SEED,
                 z_range=None, dtype=np.float32, amp: float = 0.1):
    """(rho, u) of the perturbed laminar channel, shapes (nz', ny, nx) and (3, nz', ny, nx).

    Walls are at the -y and +y faces (y = -1/2 and y = ny - 1/2).  u_x is the parabola of
    bulk velocity u_bulk; u_y and u_z carry a sinusoid of amplitude amp * u_bulk (0.1 by
    default) with seeded phases (4 periods in x, 2 in z, vanishing at the walls); every
    component gets uniform noise in [-0.05, 0.05] u_bulk.  z_range = (z0, z1) generates a
    slab of the full field."""
    z0, z1 = (0, nz) if z_range is None else z_range
    ph = 2 * math.pi * uniform01(seed, 1, np.arange(4, dtype=np.uint64))
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    yc = (np.arange(ny, dtype=np.float64) + 0.5)[None, :, None] / ny
    z = np.arange(z0, z1, dtype=np.float64)[:, None, None]
    shape = (z1 - z0, ny, nx)
    u = np.zeros((3,) + shape, dtype=np.float64)
    u[0] = 6.0 * u_bulk * yc * (1.0 - yc)
    amp = amp * u_bulk
    env = np.sin(math.pi * yc)
    u[1] = amp * np.sin(2 * math.pi * 4 * x / nx + ph[0]) * env * np.cos(2 * math.pi * 2 * z / nz + ph[1])
    u[2] = amp * np.cos(2 * math.pi * 4 * x / nx + ph[2]) * env * np.sin(2 * math.pi * 2 * z / nz + ph[3])
    ncell = nx * ny * nz
    first = z0 * ny * nx
    idx = np.arange(first, first + int(np.prod(shape)), dtype=np.uint64)
    for a in range(3):
        noise = uniform01(seed, 2 + a, idx + np.uint64(a * ncell)).reshape(shape)
        u[a] += (noise - 0.5) * 0.1 * u_bulk
    rho = np.ones(shape, dtype=dtype)
    return rho, u.astype(dtype)


def landing_gear_flags(nx: int, ny: int, nz: int, scale: float = 1.0, seed: int = DEFAULT_SEED):
    """uint8 flags (nz, ny, nx) of a landing-gear-shaped bluff body (x streamwise, z up).

    Centre (nx/4, ny/2, nz/2).  Strut: cylinder of radius 12 along z from the axle to the +z
    face.  Axle: cylinder of radius 6 along y across both wheels.  Wheels: cylinders of
    radius 40 and width 30 along y centred at y = ny/2 +/- 35.  Plus 3-6 seeded boxes of
    edge 5-20 within +/-60 cells of the centre.  Lengths are multiplied by ``scale``; a cell
    is solid when its centre lies inside (boundaries included)."""
    s = float(scale)
    cxg, cyg, czg = nx / 4.0, ny / 2.0, nz / 2.0
    X = (np.arange(nx, dtype=np.float64) + 0.5)[None, None, :]
    Y = (np.arange(ny, dtype=np.float64) + 0.5)[None, :, None]
    Z = (np.arange(nz, dtype=np.float64) + 0.5)[:, None, None]
    solid = np.zeros((nz, ny, nx), dtype=bool)
    # strut (vertical), from the axle height to the top face
    solid |= ((X - cxg) ** 2 + (Y - cyg) ** 2 <= (12 * s) ** 2) & (Z >= czg)
    # axle (horizontal, along y), spanning both wheels
    solid |= ((X - cxg) ** 2 + (Z - czg) ** 2 <= (6 * s) ** 2) & (np.abs(Y - cyg) <= (35 + 15) * s)
    # wheels
    for side in (-1.0, 1.0):
        yw = cyg + side * 35 * s
        solid |= ((X - cxg) ** 2 + (Z - czg) ** 2 <= (40 * s) ** 2) & (np.abs(Y - yw) <= 15 * s)
    # seeded boxes
    r = uniform01(seed, 10, np.arange(64, dtype=np.uint64))
    nbox = 3 + int(r[0] * 4)
    for b in range(nbox):
        e = [(5 + 15 * r[1 + 6 * b + k]) * s for k in range(3)]
        c = [g + (2 * r[4 + 6 * b + k] - 1) * 60 * s for k, g in enumerate((cxg, cyg, czg))]
        solid |= ((np.abs(X - c[0]) <= e[0] / 2) & (np.abs(Y - c[1]) <= e[1] / 2)
                  & (np.abs(Z - c[2]) <= e[2] / 2))
    return solid.astype(np.uint8)


def sample_cells(ncell: int, k: int, seed: int = DEFAULT_SEED, stream: int = 20) -> np.ndarray:
    """k distinct linear cell indices drawn with the counter-based generator."""
    k = min(k, ncell)
    picks = (uniform01(seed, stream, np.arange(4 * k, dtype=np.uint64)) * ncell).astype(np.int64)
    _, first = np.unique(picks, return_index=True)
    out = picks[np.sort(first)][:k]
    return np.sort(out)
