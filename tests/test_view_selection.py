"""View selection for continual refinement (Section 4.2, Eq. 1; delta_pos =
0.05, theta_view = 5 degrees): the oracle pinned to hand-constructed cases on
both sides of each threshold, and the library's host call against the oracle
on random cases (no GPU needed)."""
import numpy as np
import pytest

import oracle
import scenes


def _rot_z(v, deg):
    a = np.deg2rad(deg)
    c, s = np.cos(a), np.sin(a)
    return np.array([c * v[0] - s * v[1], s * v[0] + c * v[1], v[2]])


P0 = np.array([0.3, -0.2, 2.5])
D0 = np.array([1.0, 0.0, 0.0])


@pytest.mark.parametrize("pos,dirn,novel", [
    (P0, D0, False),                                   # the same view
    (P0 + [0.06, 0, 0], D0, True),                     # moved past delta_pos
    (P0 + [0.04, 0, 0], D0, False),                    # moved, not far enough, same direction
    (P0 + [0.0, 0.03, 0.039], D0, False),              # |move| = 0.0492, just inside delta_pos
    (P0, _rot_z(D0, 6.0), True),                       # turned past theta
    (P0, _rot_z(D0, 4.0), False),                      # turned less than theta
    (P0 + [0.04, 0, 0], _rot_z(D0, 4.0), False),       # close in both
    (P0 + [0.04, 0, 0], _rot_z(D0, 7.0), True),        # close in position, turned enough
    (P0, 3.0 * D0, False),                             # direction length does not matter
])
def test_oracle_pins_single_view(pos, dirn, novel):
    assert oracle.view_is_novel(pos, dirn, [P0], [D0]) is novel


def test_oracle_pins_sets():
    assert oracle.view_is_novel(P0, D0, np.zeros((0, 3)), np.zeros((0, 3))) is True  # empty set
    far = [P0 + [1.0, 0, 0], P0 + [0, 1.0, 0]]
    dirs = [D0, D0]
    assert oracle.view_is_novel(P0, D0, far, dirs) is True
    # novel w.r.t. two views, redundant w.r.t. a third: not added
    assert oracle.view_is_novel(P0, D0, far + [P0 + [0.01, 0, 0]], dirs + [_rot_z(D0, 1.0)]) is False


def test_library_matches_oracle():
    from paper_2601_22026_gb300 import gsfit as G
    g = scenes.rng(91)
    agree = 0
    for _ in range(400):
        m = int(g.integers(0, 6))
        ps = P0 + g.normal(0, 0.05, (m, 3))
        ds = D0 + g.normal(0, 0.08, (m, 3))
        pn = P0 + g.normal(0, 0.05, 3)
        dn = D0 + g.normal(0, 0.08, 3)
        # skip cases within float32 rounding of a threshold
        dist = np.linalg.norm(ps - pn, axis=1)
        cosang = (ds / np.linalg.norm(ds, axis=1, keepdims=True)) @ (dn / np.linalg.norm(dn))
        if np.any(np.abs(dist - 0.05) < 1e-5) or np.any(np.abs(cosang - np.cos(np.deg2rad(5.0))) < 1e-6):
            continue
        got = G.gsfit_view_is_novel(pn.astype(np.float32), dn.astype(np.float32), ps.astype(np.float32),
                                    ds.astype(np.float32))
        assert got == oracle.view_is_novel(pn.astype(np.float32), dn.astype(np.float32), ps.astype(np.float32),
                                           ds.astype(np.float32))
        agree += 1
    assert agree > 350


def test_library_rejects_bad_arguments():
    from paper_2601_22026_gb300 import gsfit as G
    with pytest.raises(RuntimeError):
        G.gsfit_view_is_novel(P0, np.zeros(3), [P0], [D0])
    with pytest.raises(RuntimeError):
        G.gsfit_view_is_novel(P0, D0, [P0], [np.zeros(3)])
