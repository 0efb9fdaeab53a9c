"""First-order diffraction with transmissions on its legs on the GPU (the
scene's transmission on, dcem_scene_set_transmission, with diffraction)
against the oracle's or_diffract and or_diffract_trans: the same keys (the
crossings in path order around the wedge), lengths within 1e-6 m and
amplitudes within 1e-6; then the whole frame's paths and power against the
oracle's frame. Decisions the oracle flags as within the FP margins may
differ."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_07115_gb300 import dcem, scenes
from tests import parity as P
from tests.test_oracle_diffract_trans import R0, T0, _losses, _scene

pytestmark = pytest.mark.gpu

FLAGS = O.VAL_PARAM | O.VAL_EDGE | O.OCC_NEAR


@pytest.fixture(scope="module")
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_07115_gb300 import build
    build.build()
    O.build()
    torch.cuda.set_device(0)
    return torch


def _first_order(paths):
    """Records with exactly one diffraction and nothing but transmissions
    besides it."""
    t = paths["tri"]
    used = t >= 0
    d = used & ((t & dcem.TRI_DIFFRACT) != 0)
    tr = used & ((t & dcem.TRI_TRANSMIT) != 0)
    return (d.sum(axis=1) == 1) & ((d | tr).sum(axis=1) == used.sum(axis=1))


def _check(torch, sc, trans_db, max_trans, max_refl=1, n_rays=20_000, least=1):
    rays = scenes.fibonacci_sphere(n_rays)
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(rays)
    s.set_transmission(list(trans_db), max_trans)
    s.set_diffraction(True)
    prm = P.gpu_params(sc, max_refl=max_refl)
    oprm = P.oracle_params(sc, n_rays=n_rays, max_refl=max_refl, max_trans=max_trans, trans_db=tuple(trans_db),
                           diffraction=True)
    fr = s.trace(sc.tx, sc.rx[0], prm)
    wt = sc.tris.reshape(-1, 9)
    args = (wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[0], oprm)
    ref = {}
    for fn in (O.diffract, O.diffract_trans):
        k, p = fn(*args)
        w = oprm.width
        for kk, pp in zip(k.tolist(), p):
            ref[tuple(kk[:2 + w])] = pp
    g = fr.paths[_first_order(fr.paths)]
    gk = {tuple(k): p for k, p in zip(P.path_keys(g, oprm.width), g)}
    flagged = {k for k, p in ref.items() if p["flags"] & FLAGS}
    assert set(gk) ^ set(ref) <= flagged, sorted(set(gk) ^ set(ref))[:4]
    n_trans = 0
    for k in set(gk) & set(ref):
        a, b = gk[k], ref[k]
        assert abs(a["len_m"] - b["len_m"]) <= 1e-6, k
        za, zb = complex(a["amp_re"], a["amp_im"]), complex(b["amp_re"], b["amp_im"])
        assert abs(za - zb) <= 1e-6 * abs(zb), (k, za, zb)
        assert a["ray"] == -1
        n_trans += any(v >= 0 and (v & dcem.TRI_TRANSMIT) for v in k[2:])
    assert n_trans >= least, n_trans
    r = O.frame(sc, 0, rays, oprm)
    res = P.compare_paths(fr, r, oprm.width)
    assert not res["missing"] and not res["extra"] and not res["len"] and not res["amp"], res
    fin = np.isfinite(r.p_coh_dbm) & np.isfinite(fr.p_coh_dbm)
    assert np.array_equal(np.isfinite(r.p_coh_dbm), np.isfinite(fr.p_coh_dbm))
    assert np.all(np.abs(r.p_coh_dbm[fin] - fr.p_coh_dbm[fin]) <= 0.01)
    s.close()
    return n_trans


def test_corner_with_walls_on_both_legs(cuda):
    """The building corner of the oracle's pins with glass across the leg
    from the transmitter and an indoor wall across the leg to the receiver:
    the path through both, and with one transmission allowed, none of it."""
    lw, lg = _losses()
    sc = _scene([(0, 15.0, (-15.0, -5.0), 3), (1, 15.0, (-15.0, -5.0), 2)])
    assert _check(cuda, sc, (-1.0, -1.0, lw, lg), 2) == 1
    _check(cuda, sc, (-1.0, -1.0, lw, lg), 1, least=0)


def test_corner_both_directions(cuda):
    """Transmitter and receiver swapped, glass on one leg only."""
    lw, lg = _losses()
    for tx, rx in ((T0, R0), (R0, T0)):
        sc = _scene([(0, 15.0, (-15.0, -5.0), 3)], tx=tx, rx=rx)
        assert _check(cuda, sc, (-1.0, -1.0, lw, lg), 2) == 1


@pytest.mark.parametrize("seed", [3, 14])
def test_random_penetrable_boxes(cuda, seed):
    """Six random boxes, the concrete ones penetrable (10 dB) and the metal
    ones opaque, 20 receivers: diffraction at box edges seen through other
    boxes, up to two crossings."""
    from tests.test_gpu_diffraction_multi import _boxes
    sc = _boxes(seed)
    _check(cuda, sc, (10.0, -1.0), 2, max_refl=2, least=1)
