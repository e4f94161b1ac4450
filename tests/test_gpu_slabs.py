"""z slabs with halo exchange (two-grid pull) against the undivided lattice on one GPU: the same
bits after every step, for a channel (periodic z) and the bluff body (free-slip z faces, the
gear crossing the slab boundaries)."""
import numpy as np
import pytest

from tests.cases import FACES_CHANNEL, FACES_TUNNEL

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["f32", "f16"])
@pytest.mark.parametrize("nslab", [2, 3])
def test_channel_slabs_match_whole_lattice(precision, nslab):
    from paper_2305_09910_gb300 import inputs, lbm, slabs

    nx, ny, nz = 100, 18, 21
    kw = dict(stencil=19, tau=0.56, precision=precision, closure="smag", cs_smag=0.12)
    whole = lbm.Lattice(nx, ny, nz, faces=FACES_CHANNEL, streaming="pull", **kw)
    parts = slabs.ZSlabs(nx, ny, nz, nslab, faces=FACES_CHANNEL, **kw)
    rho, u = inputs.channel_init(nx, ny, nz, u_bulk=0.05, seed=41)
    for lat in (whole, parts):
        lat.set_force(3e-6)
        lat.init_equilibrium(rho, u)
    for n in (1, 1, 3):
        whole.step(n)
        parts.step(n)
        assert np.array_equal(whole.get_populations(), parts.get_populations())
    whole.sync()
    parts.sync()
    assert np.allclose(whole.reduce(), parts.reduce(), rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_bluff_body_slabs_match_whole_lattice(precision):
    from paper_2305_09910_gb300 import inputs, lbm, slabs

    nx, ny, nz = 96, 48, 48
    flags = inputs.landing_gear_flags(nx, ny, nz, scale=1 / 8)
    assert flags[20:28].any()  # the geometry crosses the slab boundary at z = 24
    kw = dict(stencil=27, tau=0.515, precision=precision, closure="smag", cs_smag=0.1, u_inflow=(0.05, 0, 0))
    whole = lbm.Lattice(nx, ny, nz, faces=FACES_TUNNEL, streaming="pull", **kw)
    parts = slabs.ZSlabs(nx, ny, nz, 2, faces=FACES_TUNNEL, **kw)
    u0 = np.zeros((3, nz, ny, nx), np.float32)
    u0[0] = 0.05
    for lat in (whole, parts):
        lat.set_flags(flags)
        lat.init_equilibrium(None, u0)
    for n in (1, 2, 4):
        whole.step(n)
        parts.step(n)
        assert np.array_equal(whole.get_populations(), parts.get_populations())


def test_halo_faces_errors():
    from paper_2305_09910_gb300 import lbm

    for faces, streaming in ((("halo", "halo") + ("periodic",) * 4, "pull"),
                             (("periodic",) * 4 + ("halo", "halo"), "aa"),
                             (("periodic",) * 4 + ("halo", "periodic"), "pull")):
        with pytest.raises(lbm.LbmError) as e:
            lbm.Lattice(40, 6, 8, faces=faces, streaming=streaming)
        assert e.value.status in (lbm.LBM_EUNSUPPORTED, lbm.LBM_EINVAL)
    import torch

    lat = lbm.Lattice(40, 6, 8, faces=("periodic",) * 4 + ("halo", "halo"), streaming="pull")
    lat.set_flags(np.zeros((10, 6, 40), np.uint8))
    lat.init_equilibrium()
    nbytes = lbm.lbm_halo_bytes(lat.h, 5)
    assert nbytes == 5 * 6 * 64 * 4
    buf = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_halo_pack(lat.h, 5, buf)  # no post-collision state yet
    assert e.value.status == lbm.LBM_ESTATE
    lat.step(1)
    lbm.lbm_halo_pack(lat.h, 5, buf)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_halo_pack(lat.h, 3, buf)
    assert e.value.status == lbm.LBM_EINVAL
    # pageable host memory is refused before any launch; pinned host memory is served
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_halo_pack(lat.h, 5, np.zeros(nbytes, np.uint8))
    assert e.value.status == lbm.LBM_EINVAL
    pinned = torch.zeros(nbytes, dtype=torch.uint8).pin_memory()
    lbm.lbm_halo_pack(lat.h, 5, pinned)
    lat.sync()
    assert torch.equal(pinned, buf.cpu())
