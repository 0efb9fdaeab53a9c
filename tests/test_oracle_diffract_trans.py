"""Pins of the oracle's first-order diffraction with transmissions on its
legs (or_diffract_trans; Sec. III steps 1-5, with the per-path limits of the
runtime comparisons in Sec. IV: two transmissions and one diffraction).

The invariant: a thin penetrable wall across a leg of a diffraction path
changes neither the diffraction point (Keller's law, the rules) nor the
path's length, only its field, by the wall's Table II penetration loss,
10^(-L/20) per crossing. So every path here is checked against the same
path of the scene without the walls (or_diffract, pinned on its own by the
corner path assembled from the UTD coefficient). Keys list the crossings in
path order around the wedge."""
import json
import os

import numpy as np
import pytest

from paper_2112_07115_gb300 import scenes
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
T0, R0 = (30.0, -20.0, 2.0), (-20.0, 30.0, 2.0)   # Q = (0, 0, 2) on the corner's edge


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def _losses():
    with open(os.path.join(GOLDEN, "paper_parameters.json")) as fh:
        rows = {r["material"]: r for r in json.load(fh)["table2_materials"]["rows"]}
    return rows["wall (indoor)"]["penetration_loss_db"], rows["glass (indoor)"]["penetration_loss_db"]


def _scene(walls, tx=T0, rx=R0):
    """The building corner of the first-order pins (walls y = 0 and x = 0,
    concrete, material 0; its one wedge the vertical edge x = y = 0), plus
    small vertical walls, each (plane axis, plane offset, (u0, u1), material):
    axis 0 a wall x = offset spanning y in (u0, u1), axis 1 a wall y =
    offset spanning x in (u0, u1); z from -5 to 10."""
    tris = scenes._quad((0.0, 0.0, -50.0), (50.0, 0.0, -50.0), (50.0, 0.0, 50.0), (0.0, 0.0, 50.0))
    tris += scenes._quad((0.0, 0.0, -50.0), (0.0, 50.0, -50.0), (0.0, 50.0, 50.0), (0.0, 0.0, 50.0))
    mats = [0, 0, 0, 0]
    for axis, c, (u0, u1), m in walls:
        if axis == 0:
            tris += scenes._quad((c, u0, -5.0), (c, u1, -5.0), (c, u1, 10.0), (c, u0, 10.0))
        else:
            tris += scenes._quad((u0, c, -5.0), (u1, c, -5.0), (u1, c, 10.0), (u0, c, 10.0))
        mats += [m, m]
    materials = np.array([[5.31, 0.0326, 0.0], [1.0, 0.0, 1.0], [6.0, 0.0, 0.0], [4.0, 0.0, 0.0]], np.float32)
    return scenes._static_scene("corner_walls", tris, mats, tx, (rx,), materials=materials)


def _run(fn, sc, prm):
    return fn(sc.tris.reshape(-1, 9), sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[0], prm)


def _prm(max_trans, lw, lg):
    # materials: 0 concrete (opaque), 1 metal (opaque), 2 an indoor wall, 3 glass
    return O.OracleParams(freq_hz=28e9, max_refl=1, max_trans=max_trans, trans_db=(-1.0, -1.0, lw, lg))


def _amp(p):
    return complex(p["amp_re"], p["amp_im"])


def test_glass_on_the_first_leg():
    """Glass across the leg from the transmitter: the same Q and length as
    without it, the amplitude times 10^(-L_glass/20), the key (glass, wedge);
    the plain diffraction is blocked by it."""
    lw, lg = _losses()
    base_k, base_p = _run(O.diffract, _scene([]), O.OracleParams(freq_hz=28e9, max_refl=1))
    assert base_k.shape[0] == 1
    sc = _scene([(0, 15.0, (-15.0, -5.0), 3)])
    assert _run(O.diffract, sc, _prm(2, lw, lg))[0].shape[0] == 0
    k, p = _run(O.diffract_trans, sc, _prm(2, lw, lg))
    assert k.shape[0] == 1
    assert k[0, 1] == 2 and (k[0, 2] & O.TRANS) and (k[0, 2] & ~O.TRANS) in (4, 5)
    assert k[0, 3] == base_k[0, 2] and np.all(k[0, 4:] == -1)
    assert np.allclose(p[0]["pts"][0], [15.0, -10.0, 2.0], atol=1e-9)
    assert np.allclose(p[0]["pts"][1], base_p[0]["pts"][0], atol=1e-12)
    assert abs(p[0]["len_m"] - base_p[0]["len_m"]) <= 1e-12
    a0 = _amp(base_p[0])
    assert abs(_amp(p[0]) - a0 * 10.0 ** (-lg / 20.0)) <= 1e-12 * abs(a0)


def test_walls_on_both_legs_and_the_limits():
    """A wall on each leg: key (glass, wedge, wall), losses multiplied; one
    transmission allowed, or one wall opaque, or no loss table: no path."""
    lw, lg = _losses()
    _, base_p = _run(O.diffract, _scene([]), O.OracleParams(freq_hz=28e9, max_refl=1))
    sc = _scene([(0, 15.0, (-15.0, -5.0), 3), (1, 15.0, (-15.0, -5.0), 2)])
    k, p = _run(O.diffract_trans, sc, _prm(2, lw, lg))
    assert k.shape[0] == 1 and k[0, 1] == 3
    assert (k[0, 2] & ~O.TRANS) in (4, 5) and (k[0, 3] & O.DIFF) and (k[0, 4] & ~O.TRANS) in (6, 7)
    assert (k[0, 2] & O.TRANS) and (k[0, 4] & O.TRANS)
    assert np.allclose(p[0]["pts"][2], [-10.0, 15.0, 2.0], atol=1e-9)
    a0 = _amp(base_p[0])
    assert abs(_amp(p[0]) - a0 * 10.0 ** (-(lw + lg) / 20.0)) <= 1e-12 * abs(a0)
    assert _run(O.diffract_trans, sc, _prm(1, lw, lg))[0].shape[0] == 0
    assert _run(O.diffract_trans, sc, _prm(2, -1.0, lg))[0].shape[0] == 0
    assert _run(O.diffract_trans, sc, O.OracleParams(freq_hz=28e9, max_refl=1))[0].shape[0] == 0


def test_crossings_in_order_along_the_leg():
    """Two walls on the first leg (x = 22.5 nearer the transmitter, then
    x = 15): the key lists them in that order; losses multiply."""
    lw, lg = _losses()
    _, base_p = _run(O.diffract, _scene([]), O.OracleParams(freq_hz=28e9, max_refl=1))
    sc = _scene([(0, 15.0, (-15.0, -5.0), 3), (0, 22.5, (-20.0, -5.0), 2)])
    k, p = _run(O.diffract_trans, sc, _prm(2, lw, lg))
    assert k.shape[0] == 1 and k[0, 1] == 3
    assert (k[0, 2] & ~O.TRANS) in (6, 7) and (k[0, 3] & ~O.TRANS) in (4, 5) and (k[0, 4] & O.DIFF)
    assert np.allclose(p[0]["pts"][0], [22.5, -15.0, 2.0], atol=1e-9)
    assert np.allclose(p[0]["pts"][1], [15.0, -10.0, 2.0], atol=1e-9)
    a0 = _amp(base_p[0])
    assert abs(_amp(p[0]) - a0 * 10.0 ** (-(lw + lg) / 20.0)) <= 1e-12 * abs(a0)


def test_reversed_direction_and_no_crossing():
    """Transmitter and receiver swapped: the crossings in reverse order and
    the amplitude that of the reversed plain diffraction times the same
    losses (the UTD coefficient with Luebbers' face factors is reciprocal
    only in the high-frequency limit, so the two directions are each
    compared with their own plain path); with no wall on a leg the path is
    or_diffract's, not this one's."""
    lw, lg = _losses()
    walls = [(0, 15.0, (-15.0, -5.0), 3), (1, 15.0, (-15.0, -5.0), 2)]
    k1, p1 = _run(O.diffract_trans, _scene(walls), _prm(2, lw, lg))
    k2, p2 = _run(O.diffract_trans, _scene(walls, tx=R0, rx=T0), _prm(2, lw, lg))
    assert k1.shape[0] == k2.shape[0] == 1
    assert (k1[0, 2] & ~O.TRANS) // 2 == (k2[0, 4] & ~O.TRANS) // 2
    assert (k1[0, 4] & ~O.TRANS) // 2 == (k2[0, 2] & ~O.TRANS) // 2
    _, b2 = _run(O.diffract, _scene([], tx=R0, rx=T0), O.OracleParams(freq_hz=28e9, max_refl=1))
    a2 = _amp(b2[0])
    assert abs(_amp(p2[0]) - a2 * 10.0 ** (-(lw + lg) / 20.0)) <= 1e-12 * abs(a2)
    assert abs(p1[0]["len_m"] - p2[0]["len_m"]) <= 1e-12
    assert _run(O.diffract_trans, _scene([(0, 15.0, (10.0, 20.0), 3)]), _prm(2, lw, lg))[0].shape[0] == 0


def _ridges(walls):
    """The two metal ridges of the chain pins (tops along y at x = 0 and
    x = 8, height 10) with _TM and _RM, plus walls as in _scene spanning y
    in (-20, 20) and z in (0, 20)."""
    from tests.test_oracle_pins import _RM, _TM, _ridge
    tris = _ridge(0.0, 2.0, 10.0) + _ridge(8.0, 2.0, 10.0)
    mats = [1] * len(tris)
    for x, m in walls:
        tris += scenes._quad((x, -20.0, 0.0), (x, 20.0, 0.0), (x, 20.0, 20.0), (x, -20.0, 20.0))
        mats += [m, m]
    materials = np.array([[5.31, 0.0326, 0.0], [1.0, 0.0, 1.0], [6.0, 0.0, 0.0], [4.0, 0.0, 0.0]], np.float32)
    return scenes._static_scene("ridges_walls", tris, mats, _TM, (_RM,), materials=materials)


def test_chain_through_walls_before_and_after():
    """The order-2 chain over the two ridges with glass across its first leg
    and an indoor wall across its last: the same Keller points and length as
    without the walls, the amplitude times both losses, the key (glass, w1,
    w2, wall) in path order; blocked for the plain chain, absent with one
    transmission allowed or the wall opaque."""
    lw, lg = _losses()
    n = len(_ridges([]).tris)
    base_k, base_p = O.diffract_multi(*_args(_ridges([]), O.OracleParams(freq_hz=28e9, max_refl=2)), 2)
    assert base_k.shape[0] == 1
    sc = _ridges([(-15.0, 3), (23.0, 2)])
    prm = O.OracleParams(freq_hz=28e9, max_refl=2, max_trans=2, trans_db=(-1.0, -1.0, lw, lg))
    assert O.diffract_multi(*_args(sc, prm), 2)[0].shape[0] == 0
    k, p = O.diffract_multi_trans(*_args(sc, prm), 2)
    assert k.shape[0] == 1 and k[0, 1] == 4
    assert (k[0, 2] & O.TRANS) and (k[0, 2] & ~O.TRANS) in (n, n + 1)
    assert k[0, 3] == base_k[0, 2] and k[0, 4] == base_k[0, 3]
    assert (k[0, 5] & O.TRANS) and (k[0, 5] & ~O.TRANS) in (n + 2, n + 3)
    assert np.allclose(p[0]["pts"][1], base_p[0]["pts"][0], atol=1e-9)
    assert np.allclose(p[0]["pts"][2], base_p[0]["pts"][1], atol=1e-9)
    assert abs(p[0]["pts"][0][0] + 15.0) <= 1e-9 and abs(p[0]["pts"][3][0] - 23.0) <= 1e-9
    assert abs(p[0]["len_m"] - base_p[0]["len_m"]) <= 1e-9
    a0 = _amp(base_p[0])
    assert abs(_amp(p[0]) - a0 * 10.0 ** (-(lw + lg) / 20.0)) <= 1e-9 * abs(a0)
    p1 = O.OracleParams(freq_hz=28e9, max_refl=2, max_trans=1, trans_db=(-1.0, -1.0, lw, lg))
    assert O.diffract_multi_trans(*_args(sc, p1), 2)[0].shape[0] == 0
    p2 = O.OracleParams(freq_hz=28e9, max_refl=2, max_trans=2, trans_db=(-1.0, -1.0, -1.0, lg))
    assert O.diffract_multi_trans(*_args(sc, p2), 2)[0].shape[0] == 0


def _args(sc, prm):
    return (sc.tris.reshape(-1, 9), sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[0], prm)
