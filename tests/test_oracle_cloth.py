"""Pins of the cloth plane, its anchors and the incision (Sec. 4: a soft-body cloth plane
with definable anchor points; a scalpel's incision in a soft body), in the FP64 oracle.

Against mathematics: anchors do not move however long the cloth hangs; a blade spanning
the cloth in the plane between two particle columns cuts exactly the springs crossing that
plane (lattice counting: ny structural, 2 (ny - 1) shear, 2 ny bending) and splits the
cloth in two unconnected halves; the segment-triangle test agrees with a linear solve.
"""
import numpy as np
import pytest

import oracle
from paper_2511_15908_gb300 import scenes


def _cloth_only(nx=10, ny=8, anchors="corners"):
    s = 0.02
    p = scenes.make_params(s, 5e-4, (-0.2, -0.2, -0.3), (0.4, 0.4, 0.2))
    sheet = scenes.cloth_plane(nx, ny, s, (0.0, 0.0, 0.0), anchors=anchors)
    return scenes.Scene("cloth", p, np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), s,
                        [sheet]), sheet


def test_anchors_stay_put_while_the_cloth_sags():
    sc, sheet = _cloth_only()
    sysm = oracle.System(sc, mode=0)
    x0 = sysm.by_id(sysm.x).copy()
    for _ in range(200):
        sysm.substep()
    x = sysm.by_id(sysm.x)
    anc = sheet.anchors
    assert np.array_equal(x[anc], x0[anc])
    free = np.setdiff1d(np.arange(len(x)), anc)
    assert (x0[free, 2] - x[free, 2]).max() > 1e-3          # the rest falls under gravity


def _components(n, pairs, active):
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a
    for (a, b), on in zip(pairs, active):
        if on:
            parent[find(a)] = find(b)
    return len({find(i) for i in range(n)})


@pytest.mark.parametrize("column", [2, 4, 6])
def test_blade_between_columns_cuts_5ny_minus_2_springs(column):
    nx, ny = 10, 8
    sc, sheet = _cloth_only(nx, ny, anchors="none")
    sysm = oracle.System(sc, mode=0)
    xc = (column + 0.5) * 0.02                      # between columns `column` and column + 1
    blade = [[xc, -1.0, -1.0], [xc, 3.0, -1.0], [xc, -1.0, 3.0]]
    n_cut, per_body = sysm.cut_springs(blade)
    assert n_cut == 5 * ny - 2
    cut, near = per_body[0]
    assert not near.any()
    assert _components(nx * ny, sheet.springs, ~cut) == 2
    # the same blade again finds nothing left to cut
    assert sysm.cut_springs(blade)[0] == 0


def test_segment_triangle_test_matches_a_linear_solve():
    rng = np.random.default_rng(4)
    sc, sheet = _cloth_only(12, 12, anchors="none")
    sysm = oracle.System(sc, mode=0)
    tri = np.array([[0.03, 0.02, -0.05], [0.2, 0.05, 0.06], [0.05, 0.21, 0.04]])
    x = sysm.by_id(sysm.x).astype(np.float64)
    pairs = sheet.springs
    n_cut, per_body = sysm.cut_springs(tri)
    cut, near = per_body[0]
    want = np.zeros(len(pairs), bool)
    for k, (a, b) in enumerate(pairs):
        lo, hi = min(a, b), max(a, b)
        A = np.stack([tri[1] - tri[0], tri[2] - tri[0], x[lo] - x[hi]], 1)
        u, v, s = np.linalg.solve(A, x[lo] - tri[0])
        want[k] = u >= 0 and v >= 0 and u + v <= 1 and 0 <= s <= 1
    assert want.sum() > 5 and n_cut == int(cut.sum())
    assert np.array_equal(cut[~near], want[~near])
