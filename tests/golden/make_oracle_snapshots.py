"""Writes tests/golden/oracle_snapshots.txt: outputs of the FP64 oracle on small fixed cases
(seeded inputs), a regression guard for the oracle's arithmetic.  Calls only oracle/ and the
seeded input generator; a change of these values is a change of the oracle and needs the
paper passage (or its reading) that justifies it.

    python tests/golden/make_oracle_snapshots.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle.refine import RefinedOracle  # noqa: E402
from paper_2305_09910_gb300 import inputs  # noqa: E402

CELLS = [0, 37, 101, 250, 511]


def cases():
    """(name, values) of every snapshot."""
    nx, ny, nz = 16, 8, 6
    faces = ("periodic", "periodic", "wall", "wall", "periodic", "periodic")
    flags = np.zeros((nz, ny, nx), np.uint8)
    flags[2:4, 3:5, 5:8] = 1
    rho, u = inputs.channel_init(nx, ny, nz, u_bulk=0.05, seed=2)
    for coll in ("trt", "mrt", "reg"):
        o = oracle.Oracle(nx, ny, nz, q=19, tau=0.6, closure="smag", cs=0.12, faces=faces, force=(1e-5, 0, 0),
                          flags=flags, collision=coll)
        o.init_equilibrium(rho.astype(np.float64), u.astype(np.float64))
        o.step(10, threads=1)
        r, v = o.moments()
        yield f"channel16_q19_{coll}_mass_momentum", o.mass_momentum()
        yield f"channel16_q19_{coll}_ux_cells", v[0].reshape(-1)[CELLS]
    o = oracle.Oracle(12, 6, 6, q=27, tau=0.7, closure="smag", cs=0.1,
                      faces=("inflow", "outflow", "freeslip", "freeslip", "freeslip", "freeslip"),
                      u_w=(0.04, 0, 0))
    o.init_equilibrium(1.0, np.array([0.04, 0.0, 0.0]))
    o.step(8, threads=1)
    yield "tunnel12_q27_mass_momentum", o.mass_momentum()
    r = RefinedOracle(4, 2, 8, q=19, tau=0.7, walls=True, force=(1e-5, 0, 0), slabs=[(0, 2), (5, 8)])
    rc = 1.0 + inputs.uniform_field(3, 1, (8, 2, 4), -0.01, 0.01)
    uc = inputs.uniform_field(3, 2, (3, 8, 2, 4), -0.02, 0.02)
    rf = [1.0 + inputs.uniform_field(3, 3 + k, (2 * (b - a), 4, 8), -0.01, 0.01) for k, (a, b) in
          enumerate([(0, 2), (5, 8)])]
    uf = [inputs.uniform_field(3, 5 + k, (3, 2 * (b - a), 4, 8), -0.02, 0.02) for k, (a, b) in
          enumerate([(0, 2), (5, 8)])]
    r.init_equilibrium(rc, uc, rf, uf)
    r.step(4)
    yield "refined_walls_mass", np.array([r.mass()])
    yield "refined_walls_fine0_f", r.ffs[0][:, 1, 2, 3]


def main():
    path = os.path.join(HERE, "oracle_snapshots.txt")
    with open(path, "w") as fh:
        fh.write("# FP64 oracle outputs on small seeded cases, written by make_oracle_snapshots.py\n")
        fh.write("# (calls only oracle/); a regression guard for the oracle's arithmetic.\n")
        for name, vals in cases():
            fh.write(name + " " + " ".join(repr(float(v)) for v in np.ravel(vals)) + "\n")
    print(path)


if __name__ == "__main__":
    main()
