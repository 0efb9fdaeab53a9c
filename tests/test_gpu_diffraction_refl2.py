"""Two reflections around a first-order diffraction on the GPU
(dcem_scene_set_diffraction_reflections with on = 2) against the oracle's
or_diffract_refl2: the same (reflection, reflection, wedge), (reflection,
wedge, reflection) and (wedge, reflection, reflection) paths with the same
points, lengths and fields (within 1e-6), then the frame's received power with
every mechanism summed. Decisions the oracle flags as within the FP margins
may differ."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_07115_gb300 import dcem, scenes
from tests import parity as P
from tests.test_gpu_diffraction_multi import _boxes
from tests.test_oracle_pins import _R2, _T2, _walls_and_tip

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


def _refl2_recs(paths):
    """Records of depth 3 with exactly one diffraction among their ids."""
    t = paths["tri"][:, :3]
    d = ((t >= 0) & ((t & dcem.TRI_DIFFRACT) != 0)).sum(axis=1)
    return (paths["depth"] == 3) & (d == 1)


def _check(torch, sc, frames, mode=dcem.MODE_FULL, least=1, n_rays=20_000):
    """Per frame: the GPU's two-reflection paths against the oracle's, then
    the whole frame's power against the oracle's reflections, first-order
    diffraction, one reflection around it and two. Returns the kinds seen
    (the position of the wedge in the path)."""
    rays = scenes.fibonacci_sphere(n_rays)
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(rays)
    s.set_diffraction(True)
    assert s.set_diffraction_reflections(2) >= 1
    prm = P.gpu_params(sc, max_refl=4, mode=mode)
    oprm = P.oracle_params(sc, n_rays=n_rays, max_refl=4, diffraction=True)
    total, kinds = 0, set()
    for f in frames:
        if sc.nobj:
            s.update_transforms(sc.xf[f])
        fr = s.trace(sc.tx, sc.rx[f], prm)
        wt = O.transform(sc.tris, sc.tri_obj, sc.xf[f] if sc.nobj else np.zeros((0, 12)))
        ck1, cp1 = O.diffract_refl(wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[f], oprm)
        ck, cp = O.diffract_refl2(wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[f], oprm)
        ref = {tuple(k): p for k, p in zip(ck.tolist(), cp)}
        g = fr.paths[_refl2_recs(fr.paths)]
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
            kinds.add([i for i in range(3) if k[2 + i] & O.DIFF][0])
        total += len(gk)
        r = O.frame(sc, f, rays, oprm)
        keys = np.concatenate([r.keys, ck1, ck])
        paths = np.concatenate([r.paths, cp1, cp])
        order = np.lexsort(keys.T[::-1])
        _, pc, _ = O.reduce(keys[order], paths[order], sc.nrx, oprm.tx_power_w)
        fin = np.isfinite(pc) & np.isfinite(fr.p_coh_dbm)
        assert np.array_equal(np.isfinite(pc), np.isfinite(fr.p_coh_dbm)), f
        assert np.all(np.abs(pc[fin] - fr.p_coh_dbm[fin]) <= 0.01), f
    s.close()
    assert total >= least, total
    return kinds


def _ground(sc):
    """sc with a 400 m x 400 m concrete ground (two static triangles first)."""
    g = np.asarray(scenes._quad((-200.0, -200.0, 0.0), (200.0, -200.0, 0.0), (200.0, 200.0, 0.0),
                                (-200.0, 200.0, 0.0)), np.float32)
    sc.tris = np.concatenate([g, sc.tris])
    sc.tri_obj = np.concatenate([np.full(2, -1, np.int32), sc.tri_obj])
    sc.tri_mat = np.concatenate([np.full(2, scenes.MAT_CONCRETE, np.int32), sc.tri_mat])
    return sc


@pytest.mark.parametrize("mat", [scenes.MAT_METAL, scenes.MAT_CONCRETE])
def test_walls_and_tip(cuda, mat):
    """The two walls at 45 degrees and the prism's tip of the oracle's pins,
    both directions: two reflections before the wedge, one on each side and
    (swapped) two after it."""
    tris = _walls_and_tip()
    mats = [mat] * 4 + [scenes.MAT_METAL] * (len(tris) - 4)
    rx = [_R2, (16.0, -12.0, 1.0), (12.0, -8.0, 2.5), (18.0, -15.0, 4.0)]
    kinds = set()
    for tx, rxs in ((_T2, rx), (_R2, [_T2, (16.0, 12.0, 1.0), (12.0, 8.0, 2.5)])):
        sc = scenes._static_scene("walls_tip", tris, mats, tx, rxs)
        kinds |= _check(cuda, sc, [0], least=1)
    assert kinds == {0, 1, 2}


@pytest.mark.parametrize("seed", [6, 10])
def test_boxes_on_ground(cuda, seed):
    """Random static boxes on a ground, 20 receivers: reflections on the
    ground and the boxes' faces around their wedges."""
    _check(cuda, _ground(_boxes(seed)), [0], least=5)


@pytest.mark.parametrize("mode", [dcem.MODE_FULL, dcem.MODE_COHERENT])
def test_moving_boxes_on_ground(cuda, mode):
    """Two of the boxes move (their wedges follow them, their faces are not
    reflectors), frames 0-2 in full and coherent frames."""
    _check(cuda, _ground(_boxes(6, n_moving=2, n_frames=3)), range(3), mode=mode, least=6)


def test_levels_and_errors(cuda):
    """on = 1 adds no two-reflection path, on = 2 adds them, on = 0 drops both;
    outside 0..3 is an argument error."""
    torch = cuda
    sc = _ground(_boxes(10))
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(scenes.fibonacci_sphere(20_000))
    s.set_diffraction(True)
    prm = P.gpu_params(sc, max_refl=4)
    counts = []
    for on in (1, 2, 0):
        s.set_diffraction_reflections(on)
        fr = s.trace(sc.tx, sc.rx[0], prm)
        counts.append(int(_refl2_recs(fr.paths).sum()))
    assert counts[0] == 0 and counts[1] >= 5 and counts[2] == 0
    for bad in (-1, 4):
        with pytest.raises(dcem.DcemError):
            s.set_diffraction_reflections(bad)
    s.close()


def test_highway_full_size_sampled(cuda):
    """The bench's highway at full size (1M rays, 4 reflections, 200 moving
    receivers, 2400 wedges, the road and barrier faces as 8 reflector
    planes), frame 1 in coherent frames with diffraction up to order 2 and up
    to two reflections around it or one between two wedges: every path of
    four receivers (the three with the most two-reflection paths and receiver
    0) that has a reflection around or between wedges, evaluated by the
    oracle for the same ids
    (or_diffract_path): valid there too, with the same points, length and
    field. The oracle's own search over every pair of the 2000 static
    triangles and every wedge is too slow at this size; the small scenes
    above check that no path is missing."""
    torch = cuda
    hw = scenes.highway(n_frames=3, n_rays=1_000_000, max_refl=4)
    s = dcem.Scene.from_scene(hw, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(scenes.fibonacci_sphere(hw.n_rays))
    assert s.set_diffraction(True) == 2400
    assert s.set_diffraction_reflections(3) == 8
    s.set_diffraction_order(2)
    prm = P.gpu_params(hw, max_refl=4, mode=dcem.MODE_COHERENT)
    for f in (0, 1):
        s.update_transforms(hw.xf[f])
        fr = s.trace(hw.tx, hw.rx[f], prm)
    assert fr.stats["coherent"] == 1
    p = fr.paths
    t = p["tri"][:, :4]
    nd = ((t >= 0) & ((t & dcem.TRI_DIFFRACT) != 0)).sum(axis=1)
    combined = p[(nd >= 1) & (p["depth"] > nd)]
    two = _refl2_recs(p)
    counts = np.bincount(p["rx"][two], minlength=hw.nrx)
    sample = [0] + [int(r) for r in np.argsort(-counts, kind="stable")[:3]]
    assert counts[sample[1]] >= 3
    oprm = P.oracle_params(hw, n_rays=hw.n_rays, max_refl=4)
    wt = O.transform(hw.tris, hw.tri_obj, hw.xf[1])
    checked, kinds = 0, set()
    for rec in combined[np.isin(combined["rx"], sample)]:
        d = int(rec["depth"])
        ids = [int(x) for x in rec["tri"][:d]]
        q = O.diffract_path(wt, hw.tri_mat, hw.tri_obj, hw.materials, hw.tx, hw.rx[1][rec["rx"]], ids, oprm)
        assert q is not None, ids
        assert abs(q["len_m"] - rec["len_m"]) <= 1e-6, ids
        za, zb = complex(rec["amp_re"], rec["amp_im"]), complex(q["amp_re"], q["amp_im"])
        assert abs(za - zb) <= 1e-6 * abs(zb), ids
        assert np.allclose(rec["pts"][:d], q["pts"][:d], atol=1e-4), ids
        kinds.add(tuple(bool(x & dcem.TRI_DIFFRACT) for x in ids))
        checked += 1
    s.close()
    # two reflections (both before, one on each side, both after), one
    # reflection around one and two wedges, one between two
    assert checked >= 10 and len(kinds) >= 5, (checked, kinds)


def test_links_equal_single_transmitter_frames(cuda):
    """Two transmitters in one frame (dcem_trace_links) with diffraction up to
    order 2 and up to two reflections around it: each transmitter's links equal
    its own single-transmitter frame bit for bit (the images of every
    transmitter are formed per link)."""
    torch = cuda
    sc = _ground(_boxes(10))
    rays = scenes.fibonacci_sphere(20_000)
    prm = P.gpu_params(sc, max_refl=4)
    tx2 = sc.tx + np.array([6.0, -9.0, 1.0], np.float32)
    st = torch.cuda.current_stream().cuda_stream

    def make(sets):
        s = dcem.Scene.from_scene(sc, stream=st)
        if sets:
            s.set_ray_sets([rays, rays])
        else:
            s.set_rays(rays)
        s.set_diffraction(True)
        s.set_diffraction_reflections(2)
        s.set_diffraction_order(2)
        return s
    sl, one = make(True), make(False)
    fl = sl.trace_links(np.stack([sc.tx, tx2]), sc.rx[0], prm)
    n2 = 0
    for t, tx in enumerate((sc.tx, tx2)):
        single = one.trace(tx, sc.rx[0], prm)
        p = fl.paths[fl.paths["tx"] == t].copy()
        p["tx"] = 0
        p["ray"] = np.where(p["ray"] >= 0, p["ray"] - t * rays.shape[0], -1)
        assert p.tobytes() == single.paths.tobytes(), t
        assert np.array_equal(fl.p_coh_dbm[t], single.p_coh_dbm)
        n2 += int(_refl2_recs(single.paths).sum())
    assert n2 >= 5
    sl.close()
    one.close()


@pytest.mark.parametrize("mode", [dcem.MODE_FULL, dcem.MODE_COHERENT])
def test_batch_equals_single_scenes(cuda, mode):
    """A batch of scenes (one with moving boxes) with diffraction up to order
    2 and up to two reflections around it: each scene's frame equals its own
    frame bit for bit."""
    torch = cuda
    st = torch.cuda.current_stream().cuda_stream
    wl = [_ground(_boxes(10, n_frames=3)), _ground(_boxes(6, n_moving=2, n_frames=3))]
    rays = scenes.fibonacci_sphere(20_000)

    def make(sc):
        s = dcem.Scene.from_scene(sc, stream=st)
        s.set_rays(rays)
        s.set_diffraction(True)
        s.set_diffraction_reflections(2)
        s.set_diffraction_order(2)
        return s
    batched, alone = [make(sc) for sc in wl], [make(sc) for sc in wl]
    b = dcem.Batch(batched, stream=st)
    prm = dcem.default_params(max_refl=4, freq_hz=28e9, mode=mode)
    n2 = 0
    for f in range(3):
        b.update_transforms([sc.xf[f] if sc.nobj else None for sc in wl])
        got = b.trace([sc.tx[None] for sc in wl], [sc.rx[f] for sc in wl], prm)
        for sc, s, g in zip(wl, alone, got):
            if sc.nobj:
                s.update_transforms(sc.xf[f])
            ref = s.trace_links(sc.tx[None], sc.rx[f], prm)
            assert g.paths.tobytes() == ref.paths.tobytes(), (f, sc.nobj)
            assert np.array_equal(g.p_coh_dbm, ref.p_coh_dbm)
            n2 += int(_refl2_recs(ref.paths).sum())
    assert n2 >= 10
    b.close()
    for s in batched + alone:
        s.close()
