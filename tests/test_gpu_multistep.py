"""lbm_step(n) with several steps per launch: cooperative multi-step launches on lattices up to
2^17 (pull) or 2^15 (AA) padded cells, CUDA graph replays above.  Both give the bits of n single launches
(lbm_step(1) n times) for every stencil, storage precision, streaming pattern and collision
operator, with the boundary rules of the test cases."""
import numpy as np
import pytest

from tests.test_gpu_parity import CASES

pytestmark = pytest.mark.gpu


def _pair(case, streaming, precision, collision, size=None):
    from paper_2305_09910_gb300 import lbm

    case = dict(case)
    flags = case.pop("flags", None)
    nx, ny, nz = size or (case["nx"], case["ny"], case["nz"])
    lats = []
    for _ in range(2):
        lat = lbm.Lattice(nx, ny, nz, stencil=case.get("q", 19), tau=case["tau"], precision=precision,
                          closure=case.get("closure", "none"), cs_smag=case.get("cs", 0.1),
                          faces=case.get("faces", ("periodic",) * 6), u_inflow=case.get("u_w", (0, 0, 0)),
                          streaming=streaming, collision=collision)
        if flags is not None and size is None:
            lat.set_flags(flags)
        lat.set_force(*case.get("force", (0.0, 0.0, 0.0)))
        lat.init_equilibrium()
        lats.append(lat)
    return lats


@pytest.mark.parametrize("name,streaming,precision,collision", [
    ("tunnel19", "aa", "f32", "trt"), ("tunnel27", "aa", "f32", "reg"), ("channel19", "pull", "f16", "mrt"),
    ("mixed27", "pull", "bf16", "trt"), ("periodic19", "aa", "f32", "reg"), ("mixed19", "aa", "f16", "trt"),
    ("tunnel19", "pull", "f32", "mrt"), ("channel27", "pull", "f32", "trt")])
def test_multi_step_launches_match_single_launches(name, streaming, precision, collision):
    a, b = _pair(CASES[name], streaming, precision, collision)
    try:
        for n in (2, 33, 5):
            a.step(n)
            for _ in range(n):
                b.step(1)
            assert np.array_equal(a.get_populations(), b.get_populations()), n
        a.sync()
        b.sync()
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("name,streaming,precision", [("channel19", "pull", "f32"), ("channel19", "aa", "f16"),
                                                     ("channel19", "pull", "f16"), ("tunnel27", "pull", "f16")])
def test_graph_replays_on_a_larger_lattice_match_single_launches(name, streaming, precision):
    # 160 x 128 x 128 = 2.6 M cells: above the multi-step limits, below the graph limit, so
    # lbm_step replays graphs (for the half-storage pull steps, graphs of the x-pair and the
    # boundary-list kernels)
    a, b = _pair(CASES[name], streaming, precision, "trt", size=(160, 128, 128))
    try:
        for n in (24, 9):
            a.step(n)
            for _ in range(n):
                b.step(1)
            assert np.array_equal(a.get_populations(), b.get_populations()), n
    finally:
        a.close()
        b.close()
