"""Host inputs of lbm_init_equilibrium: pinned host arrays are read by the kernel in place,
pageable ones staged through a device copy, device arrays read directly.  Every path gives the
same state, bit for bit, before and after steps, and solid cells export zeros (a lattice with
solid cells; D3Q19 FP32 and FP16, D3Q27 FP32, pull and AA)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("q,precision,streaming", [(19, "f32", "pull"), (19, "f16", "pull"), (27, "f32", "pull"),
                                                   (19, "f32", "aa")])
def test_host_and_device_inputs_give_the_same_state(q, precision, streaming):
    import torch

    from paper_2305_09910_gb300 import inputs, lbm

    nx, ny, nz = 64, 32, 24
    flags = inputs.poiseuille_flags(nx, ny, nz)
    flags[5:9, 10:14, 20:30] = 1  # a solid block
    rho, u = inputs.channel_init(nx, ny, nz, u_bulk=0.05, seed=11)
    dev = (torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    pinned = (torch.from_numpy(rho).pin_memory(), torch.from_numpy(u).pin_memory())
    states = []
    for src in (dev, pinned, (rho, u)):
        lat = lbm.Lattice(nx, ny, nz, stencil=q, tau=0.7, precision=precision, closure="smag", cs_smag=0.1,
                          faces=("periodic", "periodic", "periodic", "periodic", "periodic", "periodic"),
                          streaming=streaming)
        lat.set_flags(flags)
        lat.set_force(1e-5)
        lat.init_equilibrium(*src)
        first = lat.get_populations()
        lat.step(3)
        lat.sync()
        states.append((first, lat.get_populations(), np.asarray(lat.reduce())))
        lat.close()
    for first, after, sums in states[1:]:
        assert np.array_equal(first, states[0][0])
        assert np.array_equal(after, states[0][1])
        assert np.array_equal(sums, states[0][2])
    solid = np.broadcast_to(flags != 0, states[0][1].shape)
    assert np.all(states[0][1][solid] == 0.0)
