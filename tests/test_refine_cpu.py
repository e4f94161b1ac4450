"""Host logic of the refined slab (no GPU): the coarse pieces and interfaces of a refined z
range, and the acoustic scaling of the relaxation time."""
from __future__ import annotations

import pytest

from paper_2305_09910_gb300 import refine


def test_plan_periodic_wraps_one_coarse_piece():
    pieces, inter = refine.plan(10, 3, 7, walls=False)
    assert pieces == [([7, 8, 9, 0, 1, 2], ("halo", "halo"))]
    # the piece's -z face (global plane 7) meets the slab's +z face, its +z face (plane 2) the slab's -z face
    assert inter == [(0, 4, 5), (0, 5, 4)]


def test_plan_walls_two_coarse_pieces():
    pieces, inter = refine.plan(9, 2, 6, walls=True)
    assert pieces == [([0, 1], ("wall", "halo")), ([6, 7, 8], ("halo", "wall"))]
    assert inter == [(0, 5, 4), (1, 4, 5)]


@pytest.mark.parametrize("args", [(8, 3, 3, False), (8, 0, 7, False), (8, 0, 4, True), (8, 2, 8, True),
                                  (8, 5, 3, False)])
def test_plan_rejects_bad_ranges(args):
    with pytest.raises(ValueError):
        refine.plan(*args)


def test_fine_tau_doubles_the_lattice_viscosity():
    for tau in (0.51, 0.8, 1.3):
        assert (refine.fine_tau(tau) - 0.5) / 3 == pytest.approx(2 * (tau - 0.5) / 3)
