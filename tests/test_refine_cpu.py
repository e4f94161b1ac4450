"""Host logic of the refined slab (no GPU): the coarse pieces and interfaces of a refined z
range, and the acoustic scaling of the relaxation time."""
from __future__ import annotations

import pytest

from paper_2305_09910_gb300 import refine


def test_plan_periodic_wraps_one_coarse_piece():
    coarse, fine, inter = refine.plan(10, [(3, 7)], walls=False)
    assert coarse == [([7, 8, 9, 0, 1, 2], ("halo", "halo"))]
    assert fine == [((3, 7), ("halo", "halo"))]
    # the slab's -z face meets the piece's +z face (plane 2), its +z face the piece's -z face (plane 7)
    assert sorted(inter) == [(0, 4, 0, 5), (0, 5, 0, 4)]


def test_plan_walls_two_coarse_pieces():
    coarse, fine, inter = refine.plan(9, [(2, 6)], walls=True)
    assert coarse == [([0, 1], ("wall", "halo")), ([6, 7, 8], ("halo", "wall"))]
    assert inter == [(0, 5, 0, 4), (1, 4, 0, 5)]


def test_plan_refined_walls_of_a_channel():
    coarse, fine, inter = refine.plan(16, [(12, 16), (0, 4)], walls=True)
    assert coarse == [(list(range(4, 12)), ("halo", "halo"))]
    assert fine == [((0, 4), ("wall", "halo")), ((12, 16), ("halo", "wall"))]
    assert inter == [(0, 4, 0, 5), (0, 5, 1, 4)]


def test_plan_two_periodic_slabs():
    coarse, fine, inter = refine.plan(12, [(1, 3), (6, 9)], walls=False)
    assert coarse == [([9, 10, 11, 0], ("halo", "halo")), ([3, 4, 5], ("halo", "halo"))]
    assert sorted(inter) == [(0, 4, 1, 5), (0, 5, 0, 4), (1, 4, 0, 5), (1, 5, 1, 4)]


@pytest.mark.parametrize("args", [(8, [(3, 3)], False), (8, [(0, 7)], False), (8, [(2, 9)], True),
                                  (8, [(5, 3)], False), (8, [(1, 3), (3, 5)], True), (8, [(0, 2), (6, 8)], False),
                                  (8, [(0, 8)], True), (8, [], True)])
def test_plan_rejects_bad_ranges(args):
    with pytest.raises(ValueError):
        refine.plan(*args)


def test_fine_tau_doubles_the_lattice_viscosity():
    for tau in (0.51, 0.8, 1.3):
        assert (refine.fine_tau(tau) - 0.5) / 3 == pytest.approx(2 * (tau - 0.5) / 3)


def test_per_slab_arrays_must_match_the_slabs():
    rs = refine.RefinedSlab.__new__(refine.RefinedSlab)  # host logic only, no lattices
    rs.fines = [object(), object()]
    assert rs._per_slab(None) == [None, None]
    assert rs._per_slab([1, 2]) == [1, 2]
    with pytest.raises(ValueError):
        rs._per_slab([1])
    with pytest.raises(ValueError):
        rs._per_slab(1)
    rs.fines = [object()]
    assert rs._per_slab(3) == [3]
