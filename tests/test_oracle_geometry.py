"""Pins of the oracle's cut-cell geometry against closed forms (Sec. 2.2).

Each check is independent of the oracle's own formulas: exact volumes, areas
and second moments of spheres/ellipsoids, Gauss' theorem for the boundary
normals, and the fluid area of a grid plane cut by a sphere.
"""
import math

import numpy as np
import pytest

from oracle.geometry import MONO_INDEX, CellGeometry, face_area

R = 0.25
C = np.array([0.5, 0.5, 0.5])


@pytest.fixture(scope="module")
def sphere16():
    return CellGeometry(16, [(C, np.array([R] * 3))])


@pytest.fixture(scope="module")
def ellipsoid32():
    c = np.array([0.47, 0.52, 0.55])
    a = np.array([0.21, 0.17, 0.26])
    return CellGeometry(32, [(c, a)]), c, a


def _global_moment(g, f):
    """sum over cells of f applied to each cell's (moments, centre)."""
    tot = 0.0
    h = g.h
    for idx in range(g.n ** 3):
        if g.kind[idx] == 0:
            continue
        i, j, k = g.coords(idx)
        centre = np.array([(i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h])
        tot += f(g, idx, centre)
    return tot


def test_sphere_volume_and_area(sphere16):
    g = sphere16
    vol = g.vol.sum() * g.h ** 3
    assert abs(vol - (1.0 - 4.0 / 3.0 * math.pi * R ** 3)) < 1e-13
    area = sum(m["srf"][0] for m in g.mom.values()) * g.h ** 2
    assert abs(area - 4.0 * math.pi * R ** 2) < 1e-11


def test_ellipsoid_volume_and_second_moment(ellipsoid32):
    g, c, a = ellipsoid32
    h = g.h
    vol = g.vol.sum() * h ** 3
    assert abs(vol - (1.0 - 4.0 / 3.0 * math.pi * a.prod())) < 1e-11

    # int over the fluid of (x - c_x)^2 = int_box - int_ellipsoid (4 pi/15) a^3 b c
    def xx(g, idx, centre):
        if g.kind[idx] == 1:
            m2, m1, m0 = 1.0 / 12.0, 0.0, 1.0
        else:
            m = g.mom[idx]["vol"]
            m2, m1, m0 = m[MONO_INDEX[(2, 0, 0)]], m[MONO_INDEX[(1, 0, 0)]], m[0]
        d = (centre[0] - c[0]) / h
        return (m2 + 2 * d * m1 + d * d * m0) * h ** 5

    got = _global_moment(g, xx)
    box = ((1 - c[0]) ** 3 + c[0] ** 3) / 3.0
    ell = 4.0 * math.pi / 15.0 * a[0] ** 3 * a[1] * a[2]
    assert abs(got - (box - ell)) < 1e-11


def test_boundary_normals_gauss(ellipsoid32):
    """Closed surface: int n dS = 0 and int x_d n_d dS = -|E| (n points out of the fluid)."""
    g, c, a = ellipsoid32
    h = g.h
    vE = 4.0 / 3.0 * math.pi * a.prod()
    for d in range(3):
        tot_n = 0.0
        tot_xn = 0.0
        e1 = [0, 0, 0]
        e1[d] = 1
        for idx, m in g.mom.items():
            i, j, k = g.coords(idx)
            centre = np.array([(i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h])
            sn = m["srfn"][d]
            tot_n += sn[0] * h ** 2
            tot_xn += (sn[MONO_INDEX[tuple(e1)]] * h + centre[d] * sn[0]) * h ** 2
        assert abs(tot_n) < 1e-11
        assert abs(tot_xn + vE) < 1e-11


def test_face_area_disc():
    """Fluid area of a whole grid plane cut by a sphere = 1 - pi (r^2 - dz^2)."""
    n = 16
    h = 1.0 / n
    shapes = [(C, np.array([R] * 3))]
    for plane in (5, 7, 8):
        X = plane * h
        tot = 0.0
        for i in range(n):
            for j in range(n):
                tot += face_area(2, X, [i * h, j * h], [(i + 1) * h, (j + 1) * h], [0], shapes)
        assert abs(tot - (1.0 - math.pi * (R * R - (X - 0.5) ** 2))) < 1e-13


def test_classes(sphere16):
    g = sphere16
    n = g.n
    # the cell containing the centre is exterior, corner cells are full
    assert g.kind[g.index(8, 8, 8)] == 0
    assert g.kind[g.index(0, 0, 0)] == 1
    # cut cells are exactly those whose box meets the sphere surface
    h = g.h
    for idx in np.nonzero(g.kind == 2)[0][:50]:
        i, j, k = g.coords(int(idx))
        lo = np.array([i, j, k]) * h
        hi = lo + h
        near = np.clip(C, lo, hi)
        far = np.where(np.abs(lo - C) > np.abs(hi - C), lo, hi)
        assert np.linalg.norm(near - C) < R < np.linalg.norm(far - C)
