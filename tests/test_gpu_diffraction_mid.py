"""A reflection between the two wedges of an order-2 diffraction chain on the
GPU (dcem_scene_set_diffraction_reflections with on = 3, diffraction order
2) against the oracle's or_diffract_mid: the same (wedge, triangle, wedge)
paths with the same points, lengths and fields (within 1e-6), then the
frame's received power with every mechanism summed. Decisions the oracle
flags as within the FP margins may differ."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_07115_gb300 import dcem, scenes
from tests import parity as P
from tests.test_gpu_diffraction_multi import _boxes
from tests.test_gpu_diffraction_refl2 import _ground
from tests.test_oracle_pins import _GROUND, _RM, _TM, _ridge

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


def _mid_recs(paths):
    """Records of depth 3: wedge, triangle, wedge."""
    t = paths["tri"][:, :3]
    d = (t >= 0) & ((t & dcem.TRI_DIFFRACT) != 0)
    return (paths["depth"] == 3) & d[:, 0] & ~d[:, 1] & d[:, 2]


def _check(torch, sc, frames, mode=dcem.MODE_FULL, least=1, n_rays=20_000):
    """Per frame: the GPU's wedge-reflection-wedge paths against the
    oracle's, then the whole frame's power against the oracle's reflections,
    diffraction up to order 2 and every combination with reflections."""
    rays = scenes.fibonacci_sphere(n_rays)
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(rays)
    s.set_diffraction(True)
    assert s.set_diffraction_reflections(3) >= 1
    s.set_diffraction_order(2)
    prm = P.gpu_params(sc, max_refl=4, mode=mode)
    oprm = P.oracle_params(sc, n_rays=n_rays, max_refl=4, diffraction=True, diffraction_order=2)
    total = 0
    for f in frames:
        if sc.nobj:
            s.update_transforms(sc.xf[f])
        fr = s.trace(sc.tx, sc.rx[f], prm)
        wt = O.transform(sc.tris, sc.tri_obj, sc.xf[f] if sc.nobj else np.zeros((0, 12)))
        args = (wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[f], oprm)
        ck, cp = O.diffract_mid(*args)
        ref = {tuple(k): p for k, p in zip(ck.tolist(), cp)}
        g = fr.paths[_mid_recs(fr.paths)]
        gk = {tuple(k): p for k, p in zip(P.path_keys(g, oprm.width), g)}
        flagged = {k for k, p in ref.items() if p["flags"] & FLAGS}
        assert set(gk) ^ set(ref) <= flagged, (f, sorted(set(gk) ^ set(ref))[:4])
        for k in set(gk) & set(ref):
            a, b = gk[k], ref[k]
            assert abs(a["len_m"] - b["len_m"]) <= 1e-6, (f, k)
            za, zb = complex(a["amp_re"], a["amp_im"]), complex(b["amp_re"], b["amp_im"])
            assert abs(za - zb) <= 1e-6 * abs(zb), (f, k, za, zb)
            assert np.allclose(a["pts"][:3], b["pts"][:3], atol=1e-4), (f, k)
            assert a["ray"] == -1
        total += len(gk)
        more = [O.diffract_refl(*args), O.diffract_refl2(*args), O.diffract_multi_refl(*args, 2), (ck, cp)]
        r = O.frame(sc, f, rays, oprm)
        keys = np.concatenate([r.keys] + [x[0] for x in more])
        paths = np.concatenate([r.paths] + [x[1] for x in more])
        order = np.lexsort(keys.T[::-1])
        _, pc, _ = O.reduce(keys[order], paths[order], sc.nrx, oprm.tx_power_w)
        fin = np.isfinite(pc) & np.isfinite(fr.p_coh_dbm)
        assert np.array_equal(np.isfinite(pc), np.isfinite(fr.p_coh_dbm)), f
        assert np.all(np.abs(pc[fin] - fr.p_coh_dbm[fin]) <= 0.01), f
    s.close()
    assert total >= least, total
    return total


@pytest.mark.parametrize("mat", [scenes.MAT_METAL, scenes.MAT_CONCRETE])
def test_two_ridges_on_ground(cuda, mat):
    """The two ridges of the oracle's pins on a conducting ground: over the
    first ridge, off the ground and over the second, receivers on the far
    side at several heights and offsets, both directions."""
    tris = _GROUND + _ridge(0.0, 2.0, 10.0) + _ridge(8.0, 2.0, 10.0)
    mats = [scenes.MAT_METAL] * 2 + [mat] * (len(tris) - 2)
    rx = [_RM, (36.0, 0.0, 1.0), (40.0, -6.0, 2.5), (34.0, 8.0, 1.2)]
    for tx, rxs in ((_TM, rx), (_RM, [_TM, (-28.0, 4.0, 1.5)])):
        sc = scenes._static_scene("ridges", tris, mats, tx, rxs)
        _check(cuda, sc, [0], least=1)


@pytest.mark.parametrize("seed", [6, 10])
def test_boxes_on_ground(cuda, seed):
    """Random static boxes on a concrete ground, 20 receivers: roof and
    corner edges of two boxes with the ground or a face between them."""
    _check(cuda, _ground(_boxes(seed)), [0], least=1)


@pytest.mark.parametrize("mode", [dcem.MODE_FULL, dcem.MODE_COHERENT])
def test_moving_boxes_on_ground(cuda, mode):
    """Two of the boxes move (their wedges follow them), frames 0-2."""
    _check(cuda, _ground(_boxes(6, n_moving=2, n_frames=3)), range(3), mode=mode, least=1)


def test_level_three_needs_order_two(cuda):
    """on = 3 with diffraction order 1 adds nothing beyond on = 2; outside
    0..3 is an argument error."""
    torch = cuda
    tris = _GROUND + _ridge(0.0, 2.0, 10.0) + _ridge(8.0, 2.0, 10.0)
    sc = scenes._static_scene("ridges", tris, [scenes.MAT_METAL] * len(tris), _TM, [_RM])
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(scenes.fibonacci_sphere(20_000))
    s.set_diffraction(True)
    prm = P.gpu_params(sc, max_refl=4)
    out = []
    for on in (2, 3):
        s.set_diffraction_reflections(on)
        fr = s.trace(sc.tx, sc.rx[0], prm)
        out.append(fr.paths.tobytes())
    assert out[0] == out[1]
    s.set_diffraction_order(2)
    fr = s.trace(sc.tx, sc.rx[0], prm)
    assert _mid_recs(fr.paths).sum() == 1
    with pytest.raises(dcem.DcemError):
        s.set_diffraction_reflections(4)
    s.close()


def test_links_and_batch_equal_single_frames(cuda):
    """Two transmitters in one frame, and a batch of two scenes, with every
    combination of reflections up to order 2: each link (scene) equals its own
    single frame bit for bit, paths with a reflection between two wedges
    among them."""
    torch = cuda
    st = torch.cuda.current_stream().cuda_stream
    rays = scenes.fibonacci_sphere(20_000)

    def make(sc, sets=1):
        s = dcem.Scene.from_scene(sc, stream=st)
        if sets > 1:
            s.set_ray_sets([rays] * sets)
        else:
            s.set_rays(rays)
        s.set_diffraction(True)
        s.set_diffraction_reflections(3)
        s.set_diffraction_order(2)
        return s
    sc = _ground(_boxes(10))
    prm = P.gpu_params(sc, max_refl=4)
    tx2 = sc.tx + np.array([6.0, -9.0, 1.0], np.float32)
    sl, one = make(sc, 2), make(sc)
    fl = sl.trace_links(np.stack([sc.tx, tx2]), sc.rx[0], prm)
    n = 0
    for t, tx in enumerate((sc.tx, tx2)):
        single = one.trace(tx, sc.rx[0], prm)
        p = fl.paths[fl.paths["tx"] == t].copy()
        p["tx"] = 0
        p["ray"] = np.where(p["ray"] >= 0, p["ray"] - t * rays.shape[0], -1)
        assert p.tobytes() == single.paths.tobytes(), t
        assert np.array_equal(fl.p_coh_dbm[t], single.p_coh_dbm)
        n += int(_mid_recs(single.paths).sum())
    assert n >= 5
    for s in (sl, one):
        s.close()
    wl = [_ground(_boxes(10, n_frames=2)), _ground(_boxes(6, n_moving=2, n_frames=2))]
    batched, alone = [make(w) for w in wl], [make(w) for w in wl]
    b = dcem.Batch(batched, stream=st)
    prm = dcem.default_params(max_refl=4, freq_hz=28e9, mode=dcem.MODE_COHERENT)
    n = 0
    for f in range(2):
        b.update_transforms([w.xf[f] if w.nobj else None for w in wl])
        got = b.trace([w.tx[None] for w in wl], [w.rx[f] for w in wl], prm)
        for w, s, g in zip(wl, alone, got):
            if w.nobj:
                s.update_transforms(w.xf[f])
            ref = s.trace_links(w.tx[None], w.rx[f], prm)
            assert g.paths.tobytes() == ref.paths.tobytes(), (f, w.nobj)
            n += int(_mid_recs(ref.paths).sum())
    assert n >= 10
    b.close()
    for s in batched + alone:
        s.close()
