"""One reflection before or after a first-order diffraction on the GPU
(dcem_scene_set_diffraction_reflections) against the oracle's
or_diffract_refl: the same (triangle, wedge) sequences in both orders, the
same lengths, reflection and diffraction points and fields, and the frame's
received power with every mechanism summed. Decisions the oracle flags as
within the FP margins (Keller point or reflection point at an end, a point
near a triangle edge, an occlusion near a leg's end) may differ."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_07115_gb300 import dcem, scenes
from tests import parity as P

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


def _combined(paths):
    t = paths["tri"]
    return (paths["depth"] == 2) & (((t[:, 0] & dcem.TRI_DIFFRACT) != 0) | ((t[:, 1] & dcem.TRI_DIFFRACT) != 0))


def _check(torch, sc, n_rays, max_refl, frames, mode=dcem.MODE_FULL, min_paths=1):
    rays = scenes.fibonacci_sphere(n_rays)
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(rays)
    s.set_diffraction(True)
    assert s.set_diffraction_reflections(True) >= 1
    prm = P.gpu_params(sc, max_refl=max_refl, mode=mode)
    oprm = P.oracle_params(sc, n_rays=n_rays, max_refl=max_refl, diffraction=True)
    total = 0
    for f in frames:
        if sc.nobj:
            s.update_transforms(sc.xf[f])
        fr = s.trace(sc.tx, sc.rx[f], prm)
        wt = O.transform(sc.tris, sc.tri_obj, sc.xf[f] if sc.nobj else np.zeros((0, 12)))
        ck, cp = O.diffract_refl(wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[f], oprm)
        ref = {tuple(k): p for k, p in zip(ck.tolist(), cp)}
        g = fr.paths[_combined(fr.paths)]
        gk = {tuple(k): p for k, p in zip(P.path_keys(g, oprm.width), g)}
        flagged = {k for k, p in ref.items() if p["flags"] & FLAGS}
        diff = set(gk) ^ set(ref)
        assert diff <= flagged, (f, sorted(diff - flagged)[:4])
        for k in set(gk) & set(ref):
            a, b = gk[k], ref[k]
            assert abs(a["len_m"] - b["len_m"]) <= 1e-6, (f, k)
            za, zb = complex(a["amp_re"], a["amp_im"]), complex(b["amp_re"], b["amp_im"])
            assert abs(za - zb) <= 1e-6 * abs(zb), (f, k, za, zb)
            assert np.allclose(a["pts"][:2], b["pts"][:2], atol=1e-4)
            assert a["ray"] == -1
        total += len(gk)
        # the whole frame: reflection paths, first-order and combined diffraction
        r = O.frame(sc, f, rays, oprm)
        keys = np.concatenate([r.keys, ck]) if len(ck) else r.keys
        paths = np.concatenate([r.paths, cp]) if len(ck) else r.paths
        order = np.lexsort(keys.T[::-1])
        _, pc, _ = O.reduce(keys[order], paths[order], sc.nrx, oprm.tx_power_w)
        fin = np.isfinite(pc) & np.isfinite(fr.p_coh_dbm)
        assert np.array_equal(np.isfinite(pc), np.isfinite(fr.p_coh_dbm))
        assert np.all(np.abs(pc[fin] - fr.p_coh_dbm[fin]) <= 0.01), f
    s.close()
    assert total >= min_paths
    return total


def _ground_building(ground_mat, tx, rx):
    tris = scenes._quad((-200.0, -200.0, 0.0), (200.0, -200.0, 0.0), (200.0, 200.0, 0.0), (-200.0, 200.0, 0.0))
    mats = [ground_mat] * 2
    b = scenes.box_tris(20.0, 20.0, 15.0)
    return scenes._static_scene("ground_building", tris + b, mats + [scenes.MAT_CONCRETE] * len(b), tx, rx)


@pytest.mark.parametrize("ground", [scenes.MAT_METAL, scenes.MAT_CONCRETE])
def test_ground_and_building(cuda, ground):
    """Both orders around a building's corners, over a metal and a concrete
    ground; several receivers on the far side."""
    rx = ((35.0, 22.0, 10.0), (35.0, 22.0, 2.0), (30.0, -25.0, 6.0), (-25.0, 30.0, 3.0))
    for tx in ((-40.0, -12.0, 2.0), (-40.0, -12.0, 6.0)):
        _check(cuda, _ground_building(ground, tx, rx), 20_000, 2, [0], min_paths=2)


@pytest.mark.parametrize("mode", [dcem.MODE_FULL, dcem.MODE_COHERENT])
def test_toy_street_behind_buildings(cuda, mode):
    """The toy street (moving vehicles' wedges, static ground and walls as
    reflectors) with receivers behind the buildings, frames 0-3."""
    sc = scenes.toy_street()
    behind = np.array([[-30.0, 45.0, 1.5], [30.0, -45.0, 1.5], [-45.0, 30.0, 1.5], [12.0, 12.0, 1.5]], np.float32)
    sc.rx = np.repeat(behind[None], sc.nframes, axis=0)
    _check(cuda, sc, 10_000, 2, range(4), mode=mode, min_paths=4)


def test_highway_reduced(cuda):
    sc = scenes.highway(n_frames=3, n_vehicles=30, length=400.0, n_rays=50_000, max_refl=2)
    _check(cuda, sc, 50_000, 2, [0, 2], min_paths=4)


def test_combined_needs_diffraction(cuda):
    sc = scenes.toy_street()
    s = dcem.Scene.from_scene(sc)
    with pytest.raises(dcem.DcemError):
        s.set_diffraction_reflections(True)
    s.set_diffraction(True)
    assert s.set_diffraction_reflections(True) >= 1
    s.close()
