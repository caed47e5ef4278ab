"""Geometry of the H study's set-ups, on CPU: the corner octant of the whole
box is the whole box's octant voxel for voxel, so the mirror argument that
lets rollers stand for the cut planes holds for the rasterised spheroid."""
import numpy as np
import pytest

from paper_2410_20441_gb300 import contribution


@pytest.mark.parametrize("L,alpha", [(64, 0.5), (48, 1.0), (64, 4.0), (40, 0.1)])
def test_octant_is_the_whole_box_octant(L, alpha):
    Kf, Gf, phif = contribution.image(L, alpha, 0.2, octant=False)
    Ko, Go, phio = contribution.image(L, alpha, 0.2, octant=True)
    h = L // 2
    assert Ko.shape == (h, h, h)
    assert np.array_equal(Ko, Kf[h:, h:, h:]) and np.array_equal(Go, Gf[h:, h:, h:])
    # the whole box is the octant mirrored across the three planes
    for ax in range(3):
        assert np.array_equal(Kf, np.flip(Kf, axis=ax))
    assert phio == pytest.approx(phif, rel=0, abs=1e-15)


def test_semi_axes_keep_the_larger_one_at_size():
    for alpha in (0.1, 1.0, 10.0):
        a, c = contribution.semi_axes(192, alpha, 0.2)
        assert max(a, c) == pytest.approx(0.2 * 192) and c == pytest.approx(alpha * a)
