"""The D3Q19 MRT collision on the GPU against the FP64 oracle's (both from d'Humieres et al.
2002, written independently): single steps of developed states within 1e-6 per population
(AA and pull, boundary cases), the laminar Poiseuille run within 1e-5 relative, AA and pull
giving the same bits, and the argument checks."""
import numpy as np
import pytest

from tests.cases import developed_state, make_pair, max_abs_pop_error
from tests.test_gpu_parity import CASES, _start

pytestmark = pytest.mark.gpu

MRT_CASES = ["channel19", "tunnel19", "mixed19", "periodic19", "channel19_plain"]


@pytest.mark.parametrize("name", MRT_CASES)
@pytest.mark.parametrize("streaming", ["aa", "pull"])
@pytest.mark.parametrize("steps", [1, 3])
def test_mrt_single_steps_match_oracle(name, streaming, steps):
    case = dict(CASES[name])
    lat, ora = make_pair(collision="mrt", streaming=streaming, **case)
    _start(lat, ora, case, seed=200 + steps)
    lat.step(steps)
    ora.step(steps)
    lat.sync()
    err = max_abs_pop_error(lat, ora)
    assert err <= 1e-6, f"{name}/{streaming}: {err}"


def test_mrt_poiseuille_1000_steps_matches_oracle():
    from paper_2305_09910_gb300 import inputs

    nx, ny, nz = 64, 32, 32
    flags = inputs.poiseuille_flags(nx, ny, nz)
    lat, ora = make_pair(nx, ny, nz, q=19, tau=0.8, force=(1e-6, 0, 0), flags=flags, collision="mrt")
    lat.init_equilibrium()
    ora.init_equilibrium(1.0, np.zeros(3))
    m0 = lat.reduce()[0]
    lat.step(1000)
    ora.step(1000)
    lat.sync()
    _, u = lat.moments()
    _, ur = ora.moments()
    assert np.abs(u - ur).max() / np.abs(ur).max() <= 1e-5
    assert abs(lat.reduce()[0] - m0) / m0 <= 1e-7


@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_mrt_pull_and_aa_agree_bit_for_bit(precision):
    from paper_2305_09910_gb300 import lbm

    case = dict(CASES["tunnel19"])
    flags = case.pop("flags")
    common = dict(stencil=19, tau=case["tau"], closure="smag", cs_smag=case["cs"], faces=case["faces"],
                  u_inflow=case["u_w"], precision=precision, collision="mrt")
    a = lbm.Lattice(case["nx"], case["ny"], case["nz"], streaming="aa", **common)
    b = lbm.Lattice(case["nx"], case["ny"], case["nz"], streaming="pull", **common)
    _, ora = make_pair(flags=flags, **case)
    for lat in (a, b):
        lat.set_flags(flags)
    df = _start(a, ora, dict(CASES["tunnel19"]), seed=24)
    b.set_populations(df)
    for n in (1, 2, 3):
        a.step(n)
        b.step(n)
        assert np.array_equal(a.get_populations(), b.get_populations())


def test_mrt_argument_checks():
    from paper_2305_09910_gb300 import lbm

    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice(32, 8, 8, stencil=27, collision="mrt")
    assert e.value.status == lbm.LBM_EUNSUPPORTED
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice(32, 8, 8, closure="mlp", collision="mrt")
    assert e.value.status == lbm.LBM_EUNSUPPORTED
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice(32, 8, 8, collision="mrt", mrt_rates=(1.2, 1.4, 2.0, 1.4, 1.9))
    assert e.value.status == lbm.LBM_EINVAL
