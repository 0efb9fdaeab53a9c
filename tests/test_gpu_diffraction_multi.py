"""Diffraction of order 2 and 3 on the GPU (dcem_scene_set_diffraction_order)
against the oracle's or_diffract_multi: the same wedge sequences, the same
Keller points, lengths and fields (within 1e-6), and the frame's received
power with every mechanism summed. Decisions the oracle flags as within the
FP margins (a Keller point at an edge's end, the shadow rule at its
threshold, an occlusion near a leg's end) may differ."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_07115_gb300 import dcem, scenes
from tests import parity as P
from tests.test_oracle_pins import _prism, _slab

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


def _of_order(paths, m):
    t = paths["tri"]
    sel = paths["depth"] == m
    for i in range(m):
        sel &= (t[:, i] & dcem.TRI_DIFFRACT) != 0
    return sel


def _check(torch, sc, n_rays, max_refl, frames, order, mode=dcem.MODE_FULL, min_paths=(1, 0)):
    """Frames of `sc` with diffraction up to `order` wedges: per order the GPU's
    paths against the oracle's, then the received power of the whole frame."""
    rays = scenes.fibonacci_sphere(n_rays)
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(rays)
    s.set_diffraction(True)
    s.set_diffraction_order(order)
    prm = P.gpu_params(sc, max_refl=max_refl, mode=mode)
    oprm = P.oracle_params(sc, n_rays=n_rays, max_refl=max_refl, diffraction=True, diffraction_order=order)
    totals = [0, 0]
    for f in frames:
        if sc.nobj:
            s.update_transforms(sc.xf[f])
        fr = s.trace(sc.tx, sc.rx[f], prm)
        wt = O.transform(sc.tris, sc.tri_obj, sc.xf[f] if sc.nobj else np.zeros((0, 12)))
        for m in range(2, order + 1):
            ck, cp = O.diffract_multi(wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[f], oprm, m)
            ref = {tuple(k): p for k, p in zip(ck.tolist(), cp)}
            g = fr.paths[_of_order(fr.paths, m)]
            gk = {tuple(k): p for k, p in zip(P.path_keys(g, oprm.width), g)}
            flagged = {k for k, p in ref.items() if p["flags"] & FLAGS}
            diff = set(gk) ^ set(ref)
            assert diff <= flagged, (f, m, sorted(diff - flagged)[:4])
            for k in set(gk) & set(ref):
                a, b = gk[k], ref[k]
                assert abs(a["len_m"] - b["len_m"]) <= 1e-6, (f, k)
                za, zb = complex(a["amp_re"], a["amp_im"]), complex(b["amp_re"], b["amp_im"])
                assert abs(za - zb) <= 1e-6 * abs(zb), (f, k, za, zb)
                assert np.allclose(a["pts"][:m], b["pts"][:m], atol=1e-4)
                assert a["ray"] == -1
            totals[m - 2] += len(gk)
        # the whole frame: reflections and diffraction of every order
        r = O.frame(sc, f, rays, oprm)
        fin = np.isfinite(r.p_coh_dbm) & np.isfinite(fr.p_coh_dbm)
        assert np.array_equal(np.isfinite(r.p_coh_dbm), np.isfinite(fr.p_coh_dbm))
        assert np.all(np.abs(r.p_coh_dbm[fin] - fr.p_coh_dbm[fin]) <= 0.01), f
    s.close()
    assert totals[0] >= min_paths[0] and totals[1] >= min_paths[1], totals
    return totals


@pytest.mark.parametrize("mat", [scenes.MAT_METAL, scenes.MAT_CONCRETE])
def test_two_walls(cuda, mat):
    """The double diffraction around two thin walls' ends (the oracle's
    composition pin), with extra receivers around them."""
    tris = _slab(0.0, 0.5, -50.0, 0.0) + _slab(10.0, 10.5, 5.0, 55.0)
    rx = [(20.0, 20.0, 2.0), (25.0, 10.0, 1.5), (15.0, 30.0, 4.0), (-5.0, 20.0, 2.0)]
    sc = scenes._static_scene("walls", tris, [mat] * len(tris), (-10.0, -20.0, 2.0), rx)
    _check(cuda, sc, 20_000, 3, [0], 3, min_paths=(2, 0))


@pytest.mark.parametrize("mat", [scenes.MAT_METAL, scenes.MAT_CONCRETE])
def test_three_prisms(cuda, mat):
    """The triple diffraction around three prism tips, and receivers beside it."""
    tris = []
    for a in np.deg2rad([60.0, 0.0, -60.0]):
        tris += _prism(a)
    at = lambda deg, r=22.0, z=2.0: (r * np.cos(np.deg2rad(deg)), r * np.sin(np.deg2rad(deg)), z)
    rx = [at(-120.0), at(-110.0, 25.0, 3.0), at(-130.0, 21.0, 1.0), at(-100.0, 30.0, 5.0)]
    sc = scenes._static_scene("prisms", tris, [mat] * len(tris), at(120.0), rx)
    _check(cuda, sc, 20_000, 3, [0], 3, min_paths=(0, 1))


def _boxes(seed, n_boxes=6, nrx=20, n_moving=0, n_frames=1):
    """Random boxes (vertical corners and roof edges in every orientation
    pair), materials metal or concrete, a random Tx and receivers; the first
    n_moving boxes are rigid objects translating by 0.4 m per frame."""
    rng = np.random.default_rng(seed)
    meshes = []
    for _ in range(n_boxes):
        lx, ly, lz = rng.uniform(3, 10), rng.uniform(3, 10), rng.uniform(3, 12)
        meshes.append(scenes.box_tris(lx, ly, lz, center=(rng.uniform(-20, 20), rng.uniform(-20, 20), 0.0)))
    mat_of = [scenes.MAT_METAL if rng.uniform() < 0.5 else scenes.MAT_CONCRETE for _ in range(n_boxes)]
    tx = (rng.uniform(-40, 40), rng.uniform(-40, 40), rng.uniform(1, 6))
    rx = np.array([(rng.uniform(-40, 40), rng.uniform(-40, 40), rng.uniform(1, 6)) for _ in range(nrx)], np.float32)
    static = [t for mesh in meshes[n_moving:] for t in mesh]
    smat = [m for mesh, m in zip(meshes[n_moving:], mat_of[n_moving:]) for _ in mesh]
    tris, tobj, tmat = scenes._assemble(static, smat, meshes[:n_moving], mat_of[:n_moving])
    xf = np.zeros((n_frames, n_moving, 12), np.float32)
    for f in range(n_frames):
        for o in range(n_moving):
            xf[f, o] = scenes._xf_row(0.0, 0.4 * f, 0.2 * f * (o + 1), 0.0)
    return scenes.Scene("boxes", tris, tobj, tmat, scenes.default_materials(), n_moving, xf,
                        np.asarray(tx, np.float32), np.repeat(rx[None], n_frames, axis=0), n_rays=20_000, max_refl=3)


@pytest.mark.parametrize("seed,least", [(1, (10, 0)), (6, (5, 4)), (10, (8, 16)), (14, (3, 12))])
def test_random_boxes(cuda, seed, least):
    """Six random boxes, 20 receivers: many paths of orders 2 and 3."""
    _check(cuda, _boxes(seed), 20_000, 3, [0], 3, min_paths=least)


@pytest.mark.parametrize("mode", [dcem.MODE_FULL, dcem.MODE_COHERENT])
def test_moving_boxes(cuda, mode):
    """Two of the boxes move (their wedges follow them), frames 0-2 in full
    and coherent frames."""
    _check(cuda, _boxes(6, n_moving=2, n_frames=3), 20_000, 3, range(3), 3, mode=mode, min_paths=(20, 8))


def test_order_needs_diffraction_and_range(cuda):
    sc = scenes.toy_street()
    s = dcem.Scene.from_scene(sc)
    with pytest.raises(dcem.DcemError):
        s.set_diffraction_order(2)
    s.set_diffraction(True)
    for bad in (0, 4):
        with pytest.raises(dcem.DcemError):
            s.set_diffraction_order(bad)
    s.set_diffraction_order(3)
    s.set_diffraction_order(1)
    s.close()


def test_order_one_is_unchanged(cuda):
    """max_order 1 after 3 gives the first-order frame bit for bit."""
    sc = scenes.toy_street()
    rays = scenes.fibonacci_sphere(10_000)
    out = []
    for orders in ((1,), (3, 1)):
        s = dcem.Scene.from_scene(sc, stream=cuda.cuda.current_stream().cuda_stream)
        s.set_rays(rays)
        s.set_diffraction(True)
        for o in orders:
            s.set_diffraction_order(o)
        s.update_transforms(sc.xf[1])
        fr = s.trace(sc.tx, sc.rx[1], P.gpu_params(sc, max_refl=3))
        out.append((fr.paths.tobytes(), fr.p_coh_dbm.tobytes()))
        s.close()
    assert out[0] == out[1]


def test_links_equal_single_transmitter_frames(cuda):
    """Two transmitters in one frame (dcem_trace_links): the wedge pairs and
    triples are formed per transmitter, and each transmitter's links equal its
    own single-transmitter frame bit for bit (paths of every order, powers)."""
    torch = cuda
    sc = _boxes(10)
    rays = scenes.fibonacci_sphere(20_000)
    prm = P.gpu_params(sc, max_refl=3)
    tx2 = sc.tx + np.array([6.0, -9.0, 1.0], np.float32)
    st = torch.cuda.current_stream().cuda_stream
    sl = dcem.Scene.from_scene(sc, stream=st)
    sl.set_ray_sets([rays, rays])
    sl.set_diffraction(True)
    sl.set_diffraction_order(3)
    fl = sl.trace_links(np.stack([sc.tx, tx2]), sc.rx[0], prm)
    one = dcem.Scene.from_scene(sc, stream=st)
    one.set_rays(rays)
    one.set_diffraction(True)
    one.set_diffraction_order(3)
    orders = set()
    for t, tx in enumerate((sc.tx, tx2)):
        single = one.trace(tx, sc.rx[0], prm)
        p = fl.paths[fl.paths["tx"] == t].copy()
        p["tx"] = 0
        p["ray"] = np.where(p["ray"] >= 0, p["ray"] - t * rays.shape[0], -1)
        assert p.tobytes() == single.paths.tobytes(), t
        assert np.array_equal(fl.p_coh_dbm[t], single.p_coh_dbm)
        for m in (2, 3):
            if _of_order(single.paths, m).any():
                orders.add(m)
    assert orders == {2, 3}
    sl.close()
    one.close()


@pytest.mark.parametrize("mode", [dcem.MODE_FULL, dcem.MODE_COHERENT])
def test_batch_equals_single_scenes(cuda, mode):
    """A batch of scenes with diffraction up to order 3 (one with moving
    boxes): each scene's frame equals its own frame bit for bit."""
    torch = cuda
    st = torch.cuda.current_stream().cuda_stream
    wl = [_boxes(10, n_frames=3), _boxes(6, n_moving=2, n_frames=3), _boxes(14, n_frames=3)]
    rays = scenes.fibonacci_sphere(20_000)

    def make(sc):
        s = dcem.Scene.from_scene(sc, stream=st)
        s.set_rays(rays)
        s.set_diffraction(True)
        s.set_diffraction_order(3)
        return s
    batched, alone = [make(sc) for sc in wl], [make(sc) for sc in wl]
    b = dcem.Batch(batched, stream=st)
    prm = dcem.default_params(max_refl=3, freq_hz=28e9, mode=mode)
    for f in range(3):
        b.update_transforms([sc.xf[f] if sc.nobj else None for sc in wl])
        got = b.trace([sc.tx[None] for sc in wl], [sc.rx[f] for sc in wl], prm)
        for sc, s, g in zip(wl, alone, got):
            if sc.nobj:
                s.update_transforms(sc.xf[f])
            ref = s.trace_links(sc.tx[None], sc.rx[f], prm)
            assert g.paths.tobytes() == ref.paths.tobytes(), (f, sc.nobj)
            assert np.array_equal(g.p_coh_dbm, ref.p_coh_dbm)
            assert _of_order(ref.paths, 2).any()
    b.close()
    for s in batched + alone:
        s.close()


@pytest.mark.parametrize("seed", [6, 10])
def test_with_transmission(cuda, seed):
    """Transmission (concrete boxes 10 dB per pass, up to two passes: through a
    box) together with diffraction up to order 3: the diffraction paths of each
    order and the whole frame's power against the oracle (transmitting faces
    block diffraction legs on both sides)."""
    torch = cuda
    sc = _boxes(seed)
    rays = scenes.fibonacci_sphere(20_000)
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(rays)
    s.set_transmission([10.0, -1.0], 2)
    s.set_diffraction(True)
    s.set_diffraction_order(3)
    prm = P.gpu_params(sc, max_refl=3)
    oprm = P.oracle_params(sc, n_rays=20_000, max_refl=3, max_trans=2, trans_db=(10.0, -1.0), diffraction=True,
                           diffraction_order=3)
    fr = s.trace(sc.tx, sc.rx[0], prm)
    ref = O.frame(sc, 0, rays, oprm)
    wt = sc.tris.reshape(-1, 9)
    for m in (2, 3):
        ck, cp = O.diffract_multi(wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[0], oprm, m)
        g = fr.paths[_of_order(fr.paths, m)]
        gk = {tuple(k): p for k, p in zip(P.path_keys(g, oprm.width), g)}
        rk = {tuple(k): p for k, p in zip(ck.tolist(), cp)}
        flagged = {k for k, p in rk.items() if p["flags"] & FLAGS}
        assert set(gk) ^ set(rk) <= flagged, m
        for k in set(gk) & set(rk):
            za = complex(gk[k]["amp_re"], gk[k]["amp_im"])
            zb = complex(rk[k]["amp_re"], rk[k]["amp_im"])
            assert abs(za - zb) <= 1e-6 * abs(zb)
    res = P.compare_paths(fr, ref, oprm.width)
    assert not res["missing"] and not res["extra"] and not res["len"] and not res["amp"], res
    gkeys = P.path_keys(fr.paths, oprm.width)
    assert any(any(v >= 0 and (v & dcem.TRI_TRANSMIT) for v in k[2:]) for k in gkeys)
    fin = np.isfinite(ref.p_coh_dbm) & np.isfinite(fr.p_coh_dbm)
    assert np.array_equal(np.isfinite(ref.p_coh_dbm), np.isfinite(fr.p_coh_dbm))
    assert np.all(np.abs(ref.p_coh_dbm[fin] - fr.p_coh_dbm[fin]) <= 0.01)
    s.close()


# ---------------------------------------------------------------------------
# one reflection before or after a chain (dcem_scene_set_diffraction_reflections)
# ---------------------------------------------------------------------------
def _refl_chains(paths, m):
    """Records of m wedges and one reflection (first or last)."""
    t = paths["tri"]
    sel = paths["depth"] == m + 1
    d = np.zeros(len(paths), np.int32)
    for i in range(m + 1):
        d += ((t[:, i] >= 0) & ((t[:, i] & dcem.TRI_DIFFRACT) != 0)).astype(np.int32)
    return sel & (d == m)


def _check_refl(torch, sc, frames, order, mode=dcem.MODE_FULL, least=1, refl_orders=None):
    """GPU chains with one reflection (orders 2..order, or refl_orders) against
    or_diffract_multi_refl, then the whole frame's power against the oracle's
    reflections, diffraction of every order and the combined paths."""
    rays = scenes.fibonacci_sphere(20_000)
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(rays)
    s.set_diffraction(True)
    assert s.set_diffraction_reflections(True) >= 1
    s.set_diffraction_order(order)
    prm = P.gpu_params(sc, max_refl=4, mode=mode)
    oprm = P.oracle_params(sc, n_rays=20_000, max_refl=4, diffraction=True, diffraction_order=order)
    total = 0
    for f in frames:
        if sc.nobj:
            s.update_transforms(sc.xf[f])
        fr = s.trace(sc.tx, sc.rx[f], prm)
        wt = O.transform(sc.tris, sc.tri_obj, sc.xf[f] if sc.nobj else np.zeros((0, 12)))
        extra_k, extra_p = [], []
        ck1, cp1 = O.diffract_refl(wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[f], oprm)
        extra_k.append(ck1)
        extra_p.append(cp1)
        for m in range(2, order + 1):
            ck, cp = O.diffract_multi_refl(wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[f], oprm, m)
            extra_k.append(ck)
            extra_p.append(cp)
            if refl_orders is not None and m not in refl_orders:
                continue
            ref = {tuple(k): p for k, p in zip(ck.tolist(), cp)}
            g = fr.paths[_refl_chains(fr.paths, m)]
            gk = {tuple(k): p for k, p in zip(P.path_keys(g, oprm.width), g)}
            flagged = {k for k, p in ref.items() if p["flags"] & FLAGS}
            assert set(gk) ^ set(ref) <= flagged, (f, m, sorted(set(gk) ^ set(ref))[:4])
            for k in set(gk) & set(ref):
                a, b = gk[k], ref[k]
                assert abs(a["len_m"] - b["len_m"]) <= 1e-6, (f, k)
                za, zb = complex(a["amp_re"], a["amp_im"]), complex(b["amp_re"], b["amp_im"])
                assert abs(za - zb) <= 1e-6 * abs(zb), (f, k, za, zb)
                assert np.allclose(a["pts"][:m + 1], b["pts"][:m + 1], atol=1e-4)
            total += len(gk)
        r = O.frame(sc, f, rays, oprm)
        keys = np.concatenate([r.keys] + extra_k)
        paths = np.concatenate([r.paths] + extra_p)
        order_ = np.lexsort(keys.T[::-1])
        _, pc, _ = O.reduce(keys[order_], paths[order_], sc.nrx, oprm.tx_power_w)
        fin = np.isfinite(pc) & np.isfinite(fr.p_coh_dbm)
        assert np.array_equal(np.isfinite(pc), np.isfinite(fr.p_coh_dbm)), f
        assert np.all(np.abs(pc[fin] - fr.p_coh_dbm[fin]) <= 0.01), f
    s.close()
    assert total >= least, total
    return total


def _on_ground(tris, mats, tx, rx, ground_mat):
    g = scenes._quad((-200.0, -200.0, 0.0), (200.0, -200.0, 0.0), (200.0, 200.0, 0.0), (-200.0, 200.0, 0.0))
    return scenes._static_scene("ground", g + tris, [ground_mat] * 2 + mats, tx, rx)


@pytest.mark.parametrize("ground", [scenes.MAT_METAL, scenes.MAT_CONCRETE])
def test_reflection_and_two_walls(cuda, ground):
    """The two walls on a ground: the ground reflection before and after
    their double diffraction (receivers high and low)."""
    walls = _slab(0.0, 0.5, -50.0, 0.0) + _slab(10.0, 10.5, 5.0, 55.0)
    rx = [(20.0, 20.0, 9.0), (20.0, 20.0, 1.0), (25.0, 12.0, 6.0), (15.0, 30.0, 2.0)]
    for tx in ((-10.0, -20.0, 1.0), (-10.0, -20.0, 9.0)):
        sc = _on_ground(walls, [scenes.MAT_METAL] * len(walls), tx, rx, ground)
        _check_refl(cuda, sc, [0], 2, least=1)


def test_reflection_and_three_prisms(cuda):
    """The three prisms on a concrete ground: order 3 with the reflection."""
    pr = []
    for a in np.deg2rad([60.0, 0.0, -60.0]):
        pr += _prism(a)
    at = lambda deg, z, r=22.0: (r * np.cos(np.deg2rad(deg)), r * np.sin(np.deg2rad(deg)), z)
    rx = [at(-120.0, 9.0), at(-120.0, 1.0), at(-110.0, 5.0, 25.0)]
    for tx in (at(120.0, 1.0), at(120.0, 9.0)):
        sc = _on_ground(pr, [scenes.MAT_CONCRETE] * len(pr), tx, rx, scenes.MAT_CONCRETE)
        _check_refl(cuda, sc, [0], 3, least=1)


@pytest.mark.parametrize("mode", [dcem.MODE_FULL, dcem.MODE_COHERENT])
def test_reflection_and_moving_boxes(cuda, mode):
    """Random boxes on a ground, two of them moving, order 2 with reflections
    on the ground and the static boxes' faces, frames 0-2."""
    sc = _boxes(6, n_moving=2, n_frames=3)
    g = np.asarray(scenes._quad((-200.0, -200.0, 0.0), (200.0, -200.0, 0.0), (200.0, 200.0, 0.0),
                                (-200.0, 200.0, 0.0)), np.float32)
    sc.tris = np.concatenate([g, sc.tris])
    sc.tri_obj = np.concatenate([np.full(2, -1, np.int32), sc.tri_obj])
    sc.tri_mat = np.concatenate([np.full(2, scenes.MAT_CONCRETE, np.int32), sc.tri_mat])
    _check_refl(cuda, sc, range(3), 2, mode=mode, least=3)


def test_highway_full_size_sampled(cuda):
    """The bench's highway at full size (1M rays, 4 reflections, 200 moving
    receivers, 2400 wedges on the barriers and the moving vehicles), frame 1
    with diffraction up to order 2, in the launch configuration the bench
    times: the order-2 paths of four receivers (the three with the most and
    receiver 0) against the oracle's, which enumerates all 5.8M wedge pairs
    for each."""
    torch = cuda
    hw = scenes.highway(n_frames=3, n_rays=1_000_000, max_refl=4)
    s = dcem.Scene.from_scene(hw, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(scenes.fibonacci_sphere(hw.n_rays))
    assert s.set_diffraction(True) == 2400
    s.set_diffraction_order(2)
    prm = P.gpu_params(hw, max_refl=4, mode=dcem.MODE_COHERENT)
    for f in (0, 1):
        s.update_transforms(hw.xf[f])
        fr = s.trace(hw.tx, hw.rx[f], prm)
    assert fr.stats["coherent"] == 1
    g = fr.paths[_of_order(fr.paths, 2)]
    counts = np.bincount(g["rx"], minlength=hw.nrx)
    sample = [0] + [int(r) for r in np.argsort(-counts, kind="stable")[:3]]
    assert counts[sample[1]] >= 2
    oprm = P.oracle_params(hw, n_rays=hw.n_rays, max_refl=4)
    wt = O.transform(hw.tris, hw.tri_obj, hw.xf[1])
    for r in sample:
        ck, cp = O.diffract_multi(wt, hw.tri_mat, hw.tri_obj, hw.materials, hw.tx, hw.rx[1][r:r + 1], oprm, 2)
        ref = {tuple(k[1:]): p for k, p in zip(ck.tolist(), cp)}          # receiver index dropped
        gr = g[g["rx"] == r]
        gk = {tuple(k[1:]): p for k, p in zip(P.path_keys(gr, oprm.width), gr)}
        flagged = {k for k, p in ref.items() if p["flags"] & FLAGS}
        assert set(gk) ^ set(ref) <= flagged, (r, sorted(set(gk) ^ set(ref))[:4])
        for k in set(gk) & set(ref):
            za = complex(gk[k]["amp_re"], gk[k]["amp_im"])
            zb = complex(ref[k]["amp_re"], ref[k]["amp_im"])
            assert abs(za - zb) <= 1e-6 * abs(zb), (r, k)
            assert abs(gk[k]["len_m"] - ref[k]["len_m"]) <= 1e-6
            assert np.allclose(gk[k]["pts"][:2], ref[k]["pts"][:2], atol=1e-4)
    s.close()
