"""CPU-side checks of the CUDA library and the input generators (no GPU calls).

* liblbm.so builds for sm_103a, loads, and exports every entry point include/lbm.h declares;
* its host-only velocity-set table equals the oracle's (same published order);
* the seeded generators are deterministic, counter-based and shaped like the paper's cases.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2305_09910_gb300 import build, lbm

    build.build()
    return lbm.load()


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_symbols()
    assert "lbm_create" in names and "lbm_step" in names and "lbm_moments" in names
    for name in names:
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


@pytest.mark.parametrize("q", [19, 27])
def test_library_stencil_equals_oracle(lib, oracle_mod, q):
    from paper_2305_09910_gb300 import lbm

    c, w = lbm.lbm_stencil(q)
    co, wo, _ = oracle_mod.stencil(q)
    assert np.array_equal(c, co)
    assert np.array_equal(w, wo)


def test_params_default(lib):
    from paper_2305_09910_gb300 import lbm

    p = lbm.lbm_params()
    lib.lbm_params_default(ctypes.byref(p))
    assert p.struct_size == ctypes.sizeof(lbm.lbm_params)
    assert p.magic_lambda == 3.0 / 16.0 and p.cs_smag == 0.1 and p.rho_inflow == 1.0
    assert list(p.face_bc) == [0] * 6 and p.precision == 0 and p.streaming == 0
    assert p.pipeline == 1  # direct loads


def test_create_rejects_bad_arguments_before_touching_the_device(lib):
    from paper_2305_09910_gb300 import lbm

    for args in [(0, 4, 4, 19, 0.8), (4, 4, 4, 15, 0.8), (4, 4, 4, 19, 0.5)]:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_create(*args, lbm.lbm_params_default(stream=ctypes.c_void_p(0)))
        assert e.value.status == lbm.LBM_EINVAL
    p = lbm.lbm_params_default(stream=ctypes.c_void_p(0))
    p.struct_size = 8
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create(4, 4, 4, 19, 0.8, p)


def test_create_refuses_the_staged_pipelines_before_touching_the_device(lib):
    """Only the direct-load pipeline is built; the reserved values are refused, unknown ones
    are invalid."""
    from paper_2305_09910_gb300 import lbm

    for pipe, status in ((0, lbm.LBM_EUNSUPPORTED), (2, lbm.LBM_EUNSUPPORTED), (3, lbm.LBM_EUNSUPPORTED),
                         (7, lbm.LBM_EINVAL)):
        p = lbm.lbm_params_default(stream=ctypes.c_void_p(0))
        p.pipeline = pipe
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_create(8, 4, 4, 19, 0.8, p)
        assert e.value.status == status, (pipe, e.value)


def test_wait_limit_entry_rejects_bad_arguments(lib):
    assert lib.lbm_debug_set_wait_polls(None, 0) == -1  # LBM_EINVAL: no handle


def test_uniform01_counter_based():
    from paper_2305_09910_gb300 import inputs

    a = inputs.uniform01(1, 2, np.arange(1000, dtype=np.uint64))
    b = inputs.uniform01(1, 2, np.arange(500, 1000, dtype=np.uint64))
    assert np.array_equal(a[500:], b)
    assert 0.0 <= a.min() and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.03
    assert not np.array_equal(a, inputs.uniform01(1, 3, np.arange(1000, dtype=np.uint64)))
    # splitmix64 finaliser on a known state: mix(0x9E3779B97F4A7C15) of seed 0, counter 0
    z = inputs._mix(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF  # first output of splitmix64 seeded with 0


def test_channel_init_shape_and_statistics():
    from paper_2305_09910_gb300 import inputs

    rho, u = inputs.channel_init(64, 32, 16, u_bulk=0.05, seed=9)
    assert rho.shape == (16, 32, 64) and u.shape == (3, 16, 32, 64)
    assert rho.dtype == np.float32 and (rho == 1).all()
    assert abs(u[0].mean() - 0.05) < 0.002
    assert np.abs(u[1]).max() <= 0.1 * 0.05 + 0.0025 + 1e-7
    # a slab equals the same rows of the full field (counter-based)
    _, us = inputs.channel_init(64, 32, 16, u_bulk=0.05, seed=9, z_range=(5, 9))
    assert np.array_equal(us, u[:, 5:9])


def test_channel_parameters_re_tau_180():
    from paper_2305_09910_gb300 import inputs

    p = inputs.channel_parameters(256)
    assert 5500 < p["re_b"] < 5700
    assert abs(p["u_tau"] * p["delta"] / p["nu"] - 180) < 1e-9
    assert 0.5068 < p["tau"] < 0.5069


def test_landing_gear_geometry():
    from paper_2305_09910_gb300 import inputs

    f = inputs.landing_gear_flags(768, 384, 384)
    assert f.dtype == np.uint8 and f.shape == (384, 384, 768)
    frac = f.mean()
    assert 0.001 < frac < 0.05
    # nothing touches the inflow face, the outflow face or the y faces
    assert f[:, :, 0].sum() == 0 and f[:, :, -1].sum() == 0
    assert f[:, 0, :].sum() == 0 and f[:, -1, :].sum() == 0
    # the wheel hub at the gear centre is solid, the far field is not
    assert f[192, 192 + 35, 192] == 1 and f[10, 10, 600] == 0
    small = inputs.landing_gear_flags(96, 48, 48, scale=1 / 8)
    assert small.sum() > 0


def test_sample_cells_distinct_sorted():
    from paper_2305_09910_gb300 import inputs

    c = inputs.sample_cells(10 ** 6, 300)
    assert c.size == 300 and np.all(np.diff(c) > 0) and c.min() >= 0 and c.max() < 10 ** 6


def test_kernel_digest_ignores_comments_and_sees_code(tmp_path, monkeypatch):
    """The digest that gates the committed ncu summaries: unchanged by comment and blank-line
    edits of the kernel sources, changed by any change of their code."""
    from paper_2305_09910_gb300 import build

    assert build._code_only("a = 1; // note\n\n/* block\n comment */ b = 2;  \n") == "a = 1;\n  b = 2;"
    src = tmp_path / "k.cuh"
    monkeypatch.setattr(build, "_kernel_sources", lambda: [str(src)])
    src.write_text("int f(int x) {\n  return x + 1;  // add one\n}\n")
    d0 = build.kernel_digest()
    src.write_text("// a header comment\nint f(int x) {\n\n  return x + 1;  /* add one */\n}\n")
    assert build.kernel_digest() == d0
    src.write_text("int f(int x) {\n  return x + 2;\n}\n")
    assert build.kernel_digest() != d0
    assert build.kernel_digest(extra=("-DX",)) != build.kernel_digest()
