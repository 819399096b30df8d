"""Pins of the oracle's orthographic camera: which image axis each world axis
lands on, and with which sign.

The paper's ring test (Section 3, Fig. 1) views the ring face-on along x and
shows the (y, z) plane: with rays along +x and up = +z, image u runs along +y
and image v along +z. The other views follow the same basis rule,
u = normalize(up x dir), v = dir x u, e.g. (u, v) = (x, y) for rays along +z
with up = +y. Each case below lights one half-space or one quadrant of a
16^3 grid and checks, from the expected pixel set written out by hand, that
exactly those pixels of an 8 x 8 image see emission. A swapped or negated
image axis, or a wrong default `up`, lights a different set.
"""
import numpy as np
import pytest

import oracle
import scenes

N = 16          # cells per axis on [-1, 1]^3
RES = 8         # image pixels per axis, H = 1: pixel k has centre -1 + (k + 1/2) / 4
LIT_HI = {6, 7}   # pixel centres 0.625, 0.875: the half-space coordinate > 0.5
LIT_LO = {0, 1}   # pixel centres -0.875, -0.625: coordinate < -0.5


def _field(cond):
    c = -1.0 + (np.arange(N) + 0.5) * (2.0 / N)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return np.where(cond(x, y, z), 1.0, 0.0)


def _lit(view, cond):
    sc = scenes.uniform_from_array(_field(cond), kappa=0.0)
    f = oracle.Oracle(sc).fixed(view, RES)
    img = f["inten"][:, 0]
    lit = {(int(i), int(j)) for i, j, v in zip(f["i"], f["j"], img) if v > 0.0}
    # every lit ray crosses the whole box inside the lit region: I = rho^2 x 2
    assert np.allclose(img[img > 0.0], 2.0, rtol=1e-12)
    return lit


def _set(I, J):
    return {(i, j) for i in I for j in J}


ALL = set(range(RES))

# (view, field condition, expected lit pixels (i, j))
CASES = [
    # ring view (Section 3): (u, v) = (y, z)
    ("ring y>0.5", scenes.View(dir=(1, 0, 0), up=(0, 0, 1)), lambda x, y, z: y > 0.5, _set(LIT_HI, ALL)),
    ("ring z>0.5", scenes.View(dir=(1, 0, 0), up=(0, 0, 1)), lambda x, y, z: z > 0.5, _set(ALL, LIT_HI)),
    ("ring y>0.5,z<-0.5", scenes.View(dir=(1, 0, 0), up=(0, 0, 1)),
     lambda x, y, z: (y > 0.5) & (z < -0.5), _set(LIT_HI, LIT_LO)),
    # +z view, up +y: (u, v) = (x, y)
    ("+z x>0.5", scenes.axis_view("+z"), lambda x, y, z: x > 0.5, _set(LIT_HI, ALL)),
    ("+z y>0.5", scenes.axis_view("+z"), lambda x, y, z: y > 0.5, _set(ALL, LIT_HI)),
    ("+z x>0.5,y<-0.5", scenes.axis_view("+z"), lambda x, y, z: (x > 0.5) & (y < -0.5),
     _set(LIT_HI, LIT_LO)),
    # -z view, up +y: u = y x (-z) = -x, v = (-z) x (-x) = y
    ("-z x>0.5", scenes.axis_view("-z"), lambda x, y, z: x > 0.5, _set(LIT_LO, ALL)),
    ("-z y>0.5", scenes.axis_view("-z"), lambda x, y, z: y > 0.5, _set(ALL, LIT_HI)),
    # +x view with the library's default up +y: u = y x x = -z, v = x x (-z) = y
    ("+x z>0.5", scenes.axis_view("+x"), lambda x, y, z: z > 0.5, _set(LIT_LO, ALL)),
    ("+x y<-0.5", scenes.axis_view("+x"), lambda x, y, z: y < -0.5, _set(ALL, LIT_LO)),
    # +y view, up +x: u = x x y = z, v = y x z = x
    ("+y z>0.5", scenes.axis_view("+y"), lambda x, y, z: z > 0.5, _set(LIT_HI, ALL)),
    ("+y x<-0.5", scenes.axis_view("+y"), lambda x, y, z: x < -0.5, _set(ALL, LIT_LO)),
]


@pytest.mark.parametrize("name,view,cond,expect", CASES, ids=[c[0] for c in CASES])
def test_camera_axes(name, view, cond, expect):
    assert _lit(view, cond) == expect


def test_image_centre_offset_moves_the_image():
    """A +z view centred at (0.5, 0, 0) sees the x > 0.5 slab at u = x - 0.5 > 0,
    pixels i >= 4, but pixels 6 and 7 (x = 1.125, 1.375) miss the box."""
    v = scenes.View(dir=(0, 0, 1), center=(0.5, 0.0, 0.0))
    lit = _lit(v, lambda x, y, z: x > 0.5)
    assert lit == _set({4, 5}, ALL)


def test_ring_scene_view_is_the_face_on_yz_view():
    """scenes.ring_view() (the paper's Section 3 view) is rays along +x with
    up = +z, i.e. the (u, v) = (y, z) mapping pinned above."""
    v = scenes.ring_view()
    d = np.asarray(v.dir, float)
    assert np.allclose(d / np.linalg.norm(d), (1, 0, 0)) and tuple(v.up) == (0.0, 0.0, 1.0)
