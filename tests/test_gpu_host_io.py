"""Host arrays through the C ABI: pinned host memory is read and written by the kernels in
place, pageable memory is staged through device copies; both give the same bits."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_pinned_and_pageable_host_arrays_give_the_same_bits():
    import torch

    from paper_2305_09910_gb300 import inputs, lbm

    nx, ny, nz = 70, 12, 9
    rho, u = inputs.channel_init(nx, ny, nz, u_bulk=0.05, seed=4)
    faces = ("periodic", "periodic", "wall", "wall", "periodic", "periodic")
    a = lbm.Lattice(nx, ny, nz, tau=0.7, closure="smag", faces=faces, streaming="pull")
    b = lbm.Lattice(nx, ny, nz, tau=0.7, closure="smag", faces=faces, streaming="pull")
    try:
        a.set_force(1e-5)
        b.set_force(1e-5)
        lbm.lbm_init_equilibrium(a.h, rho, u)  # pageable numpy
        lbm.lbm_init_equilibrium(b.h, torch.from_numpy(rho).pin_memory(), torch.from_numpy(u).pin_memory())
        a.step(5)
        b.step(5)
        pa = a.get_populations()
        pb = torch.zeros((19, nz, ny, nx), dtype=torch.float32).pin_memory()
        lbm.lbm_get_populations(b.h, pb)
        assert np.array_equal(pa, pb.numpy())
        ra, ua = a.moments()
        rb = torch.zeros((nz, ny, nx), dtype=torch.float32).pin_memory()
        ub = torch.zeros((3, nz, ny, nx), dtype=torch.float32).pin_memory()
        lbm.lbm_moments(b.h, rb, ub)
        assert np.array_equal(ra, rb.numpy()) and np.array_equal(ua, ub.numpy())
        # in-place import from pinned memory, then continue
        lbm.lbm_set_populations(b.h, pb)
        a.set_populations(pa)
        a.step(2)
        b.step(2)
        assert np.array_equal(a.get_populations(), b.get_populations())
    finally:
        a.close()
        b.close()
