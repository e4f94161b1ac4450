"""The regularised collision (projected regularisation, Latt & Chopard 2006) on the GPU against
the FP64 oracle's (written independently from the same definition): single steps of developed
states within 1e-6 per population (D3Q19 and D3Q27, AA and pull, every boundary case), FP16
storage within its rounding, the laminar Poiseuille run within 1e-5 relative, AA and pull
giving the same bits, and the argument checks."""
import numpy as np
import pytest

from tests.cases import make_pair, max_abs_pop_error
from tests.test_gpu_parity import CASES, _start

pytestmark = pytest.mark.gpu

REG_CASES = ["channel19", "channel27", "tunnel19", "tunnel27", "mixed19", "mixed27", "periodic19",
             "periodic27", "channel19_plain"]


@pytest.mark.parametrize("name", REG_CASES)
@pytest.mark.parametrize("streaming", ["aa", "pull"])
@pytest.mark.parametrize("steps", [1, 3])
def test_reg_steps_match_oracle(name, streaming, steps):
    case = dict(CASES[name])
    lat, ora = make_pair(collision="reg", streaming=streaming, **case)
    _start(lat, ora, case, seed=300 + steps)
    lat.step(steps)
    ora.step(steps)
    lat.sync()
    err = max_abs_pop_error(lat, ora)
    assert err <= 1e-6, f"{name}/{streaming}: {err}"


@pytest.mark.parametrize("name", ["channel19", "tunnel27"])
def test_reg_half_storage_within_rounding(name):
    case = dict(CASES[name])
    lat, ora = make_pair(collision="reg", streaming="pull", precision="f16", **case)
    df = _start(lat, ora, case, seed=17)
    lat.step(1)
    ora.step(1)
    lat.sync()
    # one FP16 rounding of the shifted post-collision value (|df| below 2 max|df0|): 2^-11 relative
    assert max_abs_pop_error(lat, ora) <= 2.0 * np.abs(df).max() * 2.0 ** -11 + 1e-6


def test_reg_poiseuille_1000_steps_matches_oracle():
    from paper_2305_09910_gb300 import inputs

    nx, ny, nz = 64, 32, 32
    flags = inputs.poiseuille_flags(nx, ny, nz)
    lat, ora = make_pair(nx, ny, nz, q=19, tau=0.8, force=(1e-6, 0, 0), flags=flags, collision="reg")
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


@pytest.mark.parametrize("precision", ["f32", "bf16"])
def test_reg_pull_and_aa_agree_bit_for_bit(precision):
    from paper_2305_09910_gb300 import lbm

    case = dict(CASES["tunnel27"])
    flags = case.pop("flags")
    common = dict(stencil=27, tau=case["tau"], closure="smag", cs_smag=case["cs"], faces=case["faces"],
                  u_inflow=case["u_w"], precision=precision, collision="reg")
    a = lbm.Lattice(case["nx"], case["ny"], case["nz"], streaming="aa", **common)
    b = lbm.Lattice(case["nx"], case["ny"], case["nz"], streaming="pull", **common)
    _, ora = make_pair(flags=flags, **case)
    for lat in (a, b):
        lat.set_flags(flags)
    df = _start(a, ora, dict(CASES["tunnel27"]), seed=25)
    b.set_populations(df)
    for n in (1, 2, 3):
        a.step(n)
        b.step(n)
        assert np.array_equal(a.get_populations(), b.get_populations())


def test_reg_argument_checks():
    from paper_2305_09910_gb300 import lbm

    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice(32, 8, 8, closure="mlp", collision="reg")
    assert e.value.status == lbm.LBM_EUNSUPPORTED
    lat = lbm.Lattice(32, 8, 8, stencil=27, collision="reg")  # every stencil
    lat.close()
