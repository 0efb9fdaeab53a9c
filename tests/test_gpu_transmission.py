"""Transmission (Sec. III "Reflected and transmitted rays", Table II
penetration losses) on the GPU against the oracle.

A ray hitting a transmitting material both reflects and spawns a child that
continues straight through; paths carry transmissions as ids with
DCEM_TRI_TRANSMIT and their field is scaled by 10^(-loss/20) per
transmission. Checked: the closed-form wall cases; primary rays' hits, the
child-ray count and the path sets (validity, length, amplitude) against the
oracle's ray tree; bit-identical results across closest-hit kernels, graph
replay and batched transmitters.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_07115_gb300 import dcem, scenes
from tests import parity as P

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
C0 = 299792458.0


@pytest.fixture(scope="module")
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_07115_gb300 import build
    build.build()
    O.build()
    torch.cuda.set_device(0)
    return torch


def _table2():
    with open(os.path.join(GOLDEN, "paper_parameters.json")) as fh:
        rows = json.load(fh)["table2_materials"]["rows"]
    return {r["material"]: r["penetration_loss_db"] for r in rows if "penetration_loss_db" in r}


def _walls(xs):
    tris, mats = [], []
    for k, x in enumerate(xs):
        tris += scenes._quad((x, -50.0, -50.0), (x, 50.0, -50.0), (x, 50.0, 50.0), (x, -50.0, 50.0))
        mats += [k, k]
    materials = np.array([[5.31, 0.0326, 0.0]] * len(xs), np.float32)
    return scenes._static_scene("walls", tris, mats, (0.0, 3.0, 7.0), ((100.0, 3.0, 7.0),), materials=materials)


def _scene(torch, sc, rays, trans_db, max_trans):
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(rays)
    s.set_transmission(trans_db, max_trans)
    return s


def test_walls_closed_form(cuda):
    """Table II's indoor wall then glass between Tx and Rx (100 m): one path
    through both, at the Friis power minus 25 dB."""
    t2 = _table2()
    lw, lg = t2["wall (indoor)"], t2["glass (indoor)"]
    sc = _walls([30.0, 60.0])
    s = _scene(cuda, sc, scenes.fibonacci_sphere(2000), [lw, lg], 2)
    prm = dcem.default_params(max_refl=1, freq_hz=30e9, tx_power_w=0.5)
    fr = s.trace(sc.tx, sc.rx[0], prm)
    assert fr.paths.shape[0] == 1
    p = fr.paths[0]
    assert p["depth"] == 2 and p["tri"][0] & dcem.TRI_TRANSMIT and p["tri"][1] & dcem.TRI_TRANSMIT
    assert abs(p["len_m"] - 100.0) <= 1e-9
    friis = 10 * np.log10(0.5 * (C0 / 30e9 / (4 * np.pi * 100.0)) ** 2) + 30
    assert abs(fr.p_coh_dbm[0] - (friis - lw - lg)) <= 1e-4
    assert fr.stats["child_rays"] > 0
    # one transmission allowed: no path; glass opaque: no path
    s.set_transmission([lw, lg], 1)
    assert s.trace(sc.tx, sc.rx[0], prm).paths.shape[0] == 0
    s.set_transmission([lw, -1.0], 2)
    assert s.trace(sc.tx, sc.rx[0], prm).paths.shape[0] == 0
    s.close()


def _vs_oracle(torch, sc, n_rays, max_refl, max_trans, trans_db, frames, tx_power=5.0):
    rays = scenes.fibonacci_sphere(n_rays)
    s = _scene(torch, sc, rays, trans_db, max_trans)
    prm = P.gpu_params(sc, max_refl=max_refl, tx_power_w=tx_power)
    oprm = P.oracle_params(sc, n_rays=n_rays, max_refl=max_refl, max_trans=max_trans, trans_db=tuple(trans_db),
                           tx_power_w=tx_power)
    nt_total = 0
    for f in frames:
        if sc.nobj:
            s.update_transforms(sc.xf[f])
        fr = s.trace(sc.tx, sc.rx[f], prm)
        ref = O.frame(sc, f, rays, oprm)
        R = n_rays
        prim = {"flags": ref.tr["flags"][:R], "hit_id": ref.tr["hit_id"][:R], "nseg": ref.tr["nseg"][:R]}
        ids, t, ns = s.ray_log()
        _, _, bad = P.compare_hits(ids, ns, prim)
        assert len(bad) == 0, (f, bad[:5])
        # child rays: equal counts unless flagged instances decide otherwise
        n_child = ref.tr["hit_id"].shape[0] - R
        n_flag = int(((ref.tr["flags"] & P.RAY_FLAGS) != 0).sum())
        assert abs(fr.stats["child_rays"] - n_child) <= n_flag, (f, fr.stats["child_rays"], n_child, n_flag)
        res = P.compare_paths(fr, ref, oprm.width)
        assert res["checked"] > 0
        assert not res["missing"] and not res["extra"], (f, res["missing"][:3], res["extra"][:3])
        assert not res["len"] and not res["amp"], (f, res["len"][:2], res["amp"][:2])
        gk = P.path_keys(fr.paths, oprm.width)
        nt_total += sum(any(v >= 0 and (v & dcem.TRI_TRANSMIT) for v in k[2:]) for k in gk)
    s.close()
    return nt_total


def test_office_vs_oracle(cuda):
    sc = scenes.office(n_frames=3)
    assert _vs_oracle(cuda, sc, 20_000, 2, 2, sc.meta["trans_db"], (0, 2), tx_power=0.5) > 100


@pytest.mark.parametrize("seed", [0, 2, 5])
def test_random_tiny_vs_oracle(cuda, seed):
    sc = scenes.random_tiny(seed, ntri=6, nobj=1, nrx=2)
    mats = np.vstack([sc.materials, sc.materials[:1]])
    tm = sc.tri_mat.copy()
    tm[2:] = mats.shape[0] - 1
    sc.materials, sc.tri_mat = mats, tm
    tdb = [10.0] + [-1.0] * (mats.shape[0] - 2) + [3.0]
    _vs_oracle(cuda, sc, 30_000, 2, 1, tdb, (0, 1))


def test_toy_street_buildings_transmit(cuda):
    """Buildings transmit (Table II indoor wall, 20 dB), ground and vehicles
    opaque; 2 reflections and 2 transmissions."""
    sc = scenes.toy_street()
    mats = np.vstack([sc.materials, sc.materials[:1]])
    tm = sc.tri_mat.copy()
    tm[2:18] = 2          # the two buildings' walls (after the two ground triangles)
    sc.materials, sc.tri_mat = mats, tm
    assert _vs_oracle(cuda, sc, 10_000, 2, 2, [-1.0, -1.0, 20.0], (0, 5)) > 0


def test_kernels_graphs_links_identical(cuda):
    """With transmission: every closest-hit kernel, graph replay and two
    transmitters in one frame give the bits of the default single frames;
    coherent requests are traced in full."""
    torch = cuda
    sc = scenes.office(n_frames=4)
    tdb = sc.meta["trans_db"]
    rays = scenes.fibonacci_sphere(30_000)
    prm = dcem.default_params(max_refl=2, freq_hz=30e9, tx_power_w=0.5, mode=dcem.MODE_COHERENT)
    ref = _scene(torch, sc, rays, tdb, 2)
    ref.set_graph_replay(False)
    outs = []
    for f in range(4):
        ref.update_transforms(sc.xf[f])
        fr = ref.trace(sc.tx, sc.rx[f], prm)
        assert fr.stats["coherent"] == 0
        outs.append((fr, ref.ray_log()))
    for cfg in [(1, 256, 24), (2, 256, 24), (0, 128, 16)]:
        s = _scene(torch, sc, rays, tdb, 2)
        s.set_trace_config(*cfg)
        for f in range(4):
            s.update_transforms(sc.xf[f])
            fr = s.trace(sc.tx, sc.rx[f], prm)
            assert fr.paths.tobytes() == outs[f][0].paths.tobytes(), (cfg, f)
            assert np.array_equal(fr.p_coh_dbm, outs[f][0].p_coh_dbm)
            assert fr.stats["child_rays"] == outs[f][0].stats["child_rays"]
            la, lb = s.ray_log(), outs[f][1]
            assert np.array_equal(la[0], lb[0]) and np.array_equal(la[2], lb[2])
            if f >= 2:
                assert fr.stats["graph_replayed"] == 1
        s.close()
    # two transmitters, the second with its own ray set
    tx2 = sc.tx + np.array([12.0, 5.0, 0.0], np.float32)
    rays2 = scenes.fibonacci_sphere(12_000)
    sl = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    sl.set_ray_sets([rays, rays2])
    sl.set_transmission(tdb, 2)
    s2 = _scene(torch, sc, rays2, tdb, 2)
    for f in range(2):
        sl.update_transforms(sc.xf[f])
        s2.update_transforms(sc.xf[f])
        fl = sl.trace_links(np.stack([sc.tx, tx2]), sc.rx[f], prm)
        f2 = s2.trace(tx2, sc.rx[f], prm)
        for t, single in ((0, outs[f][0]), (1, f2)):
            p = fl.paths[fl.paths["tx"] == t].copy()
            p["tx"] = 0
            if t == 1:
                p["ray"] -= rays.shape[0]
            assert p.tobytes() == single.paths.tobytes(), (f, t)
            assert np.array_equal(fl.p_coh_dbm[t], single.p_coh_dbm)
    sl.close()
    s2.close()
    ref.close()


def test_introspection_and_gradients_with_children(cuda):
    """Captures of child rays are reported with their primary ray; the field
    derivatives refuse transmission records (not differentiated)."""
    torch = cuda
    sc = scenes.office(n_frames=2)
    rays = scenes.fibonacci_sphere(20_000)
    s = _scene(torch, sc, rays, sc.meta["trans_db"], 2)
    prm = dcem.default_params(max_refl=2, freq_hz=30e9, tx_power_w=0.5)
    s.update_transforms(sc.xf[0])
    fr = s.trace(sc.tx, sc.rx[0], prm)
    assert fr.stats["child_rays"] > 0
    c = s.candidates()
    assert c.shape[0] == fr.stats["candidates"]
    assert np.all((c[:, 0] >= 0) & (c[:, 0] < rays.shape[0]))
    tp = fr.paths[np.any((fr.paths["tri"] >= 0) & ((fr.paths["tri"] & dcem.TRI_TRANSMIT) != 0), axis=1)]
    assert tp.shape[0] > 0
    with pytest.raises(dcem.DcemError):
        s.gradients(sc.tx, sc.rx[0], tp[:1], dcem.default_params(max_refl=4, freq_hz=30e9))
    s.close()
