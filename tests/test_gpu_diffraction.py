"""First-order edge diffraction (Sec. III step 5; UTD) on the GPU against
the oracle: the same wedges, the same diffraction paths (Keller point,
shadow rule, unoccluded legs) and their fields (the GPU evaluates the
transition function through the complex error function, the oracle by
quadrature of its integral definition), and the per-receiver power with
the reflection paths."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_07115_gb300 import dcem, scenes
from tests import parity as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_07115_gb300 import build
    build.build()
    O.build()
    torch.cuda.set_device(0)
    return torch


def _check(torch, sc, n_rays, max_refl, frames, mode=dcem.MODE_FULL, min_diff=1):
    rays = scenes.fibonacci_sphere(n_rays)
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(rays)
    nw = s.set_diffraction(True)
    wt0 = O.transform(sc.tris, sc.tri_obj, sc.xf[0] if sc.nobj else np.zeros((0, 12)))
    assert nw == O.count_wedges(wt0, sc.tri_obj)
    prm = P.gpu_params(sc, max_refl=max_refl, mode=mode)
    oprm = P.oracle_params(sc, n_rays=n_rays, max_refl=max_refl, diffraction=True)
    ndiff = 0
    for f in frames:
        if sc.nobj:
            s.update_transforms(sc.xf[f])
        fr = s.trace(sc.tx, sc.rx[f], prm)
        wt = O.transform(sc.tris, sc.tri_obj, sc.xf[f] if sc.nobj else np.zeros((0, 12)))
        dk, dp = O.diffract(wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[f], oprm)
        ref = {tuple(k): p for k, p in zip(dk.tolist(), dp)}
        g = fr.paths[(fr.paths["depth"] == 1) & ((fr.paths["tri"][:, 0] & dcem.TRI_DIFFRACT) != 0)]
        gk = {tuple(k): p for k, p in zip(P.path_keys(g, oprm.width), g)}
        # identical sets except paths the oracle flags as FP-margin decisions
        flagged = {k for k, p in ref.items() if p["flags"] & (O.VAL_PARAM | O.OCC_NEAR)}
        assert set(gk) ^ set(ref) <= flagged, (f, sorted(set(gk) ^ set(ref))[:4])
        for k in set(gk) & set(ref):
            a, b = gk[k], ref[k]
            assert abs(a["len_m"] - b["len_m"]) <= 1e-6, (f, k)
            za, zb = complex(a["amp_re"], a["amp_im"]), complex(b["amp_re"], b["amp_im"])
            assert abs(za - zb) <= 1e-6 * abs(zb), (f, k, za, zb)
            assert np.allclose(a["pts"][0], b["pts"][0], atol=1e-4)
            assert a["ray"] == -1
        ndiff += len(gk)
        # the whole frame (reflections + diffraction) against the oracle's
        r = O.frame(sc, f, rays, oprm)
        res = P.compare_paths(fr, r, oprm.width)
        assert not res["missing"] and not res["extra"] and not res["len"] and not res["amp"]
        fin = np.isfinite(r.p_coh_dbm) & np.isfinite(fr.p_coh_dbm)
        assert np.all(np.abs(r.p_coh_dbm[fin] - fr.p_coh_dbm[fin]) <= 0.01)
    s.close()
    assert ndiff >= min_diff
    return ndiff


def test_corner(cuda):
    tris = scenes._quad((0.0, 0.0, -50.0), (50.0, 0.0, -50.0), (50.0, 0.0, 50.0), (0.0, 0.0, 50.0))
    tris += scenes._quad((0.0, 0.0, -50.0), (0.0, 50.0, -50.0), (0.0, 50.0, 50.0), (0.0, 0.0, 50.0))
    sc = scenes._static_scene("corner", tris, [0, 0, 0, 0], (30.0, -20.0, 2.0),
                              ((-20.0, 30.0, 2.0), (-20.0, -30.0, 2.0), (-5.0, 40.0, 9.0)))
    _check(cuda, sc, 20_000, 2, [0], min_diff=2)


@pytest.mark.parametrize("mode", [dcem.MODE_FULL, dcem.MODE_COHERENT])
def test_toy_street_behind_buildings(cuda, mode):
    sc = scenes.toy_street()
    behind = np.array([[-30.0, 45.0, 1.5], [30.0, -45.0, 1.5], [-45.0, 30.0, 1.5], [12.0, 12.0, 1.5],
                       [45.0, -30.0, 1.5], [-12.0, -36.0, 1.5]], np.float32)
    sc.rx = np.repeat(behind[None], sc.nframes, axis=0)
    _check(cuda, sc, 10_000, 2, range(0, 10, 3), mode=mode, min_diff=4)


def test_urban_grid_reduced(cuda):
    """Extruded buildings: wall-wall and wall-roof wedges of every height."""
    sc = scenes.urban_grid(blocks=2, parcels=2, n_vehicles=12, n_tx=1, n_static_rx=12, n_frames=2, max_refl=2)
    _check(cuda, sc, 20_000, 2, [1], min_diff=1)


def test_diffraction_off_and_links(cuda):
    """Off: no diffraction record and the reflection frame's bits; with two
    transmitters the links equal the single-transmitter frames."""
    torch = cuda
    sc = scenes.toy_street()
    behind = np.array([[-30.0, 45.0, 1.5], [30.0, -45.0, 1.5], [-45.0, 30.0, 1.5]], np.float32)
    rx = behind
    rays = scenes.fibonacci_sphere(10_000)
    prm = P.gpu_params(sc, max_refl=2)
    a = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    b = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    a.set_rays(rays)
    b.set_rays(rays)
    a.set_diffraction(True)
    a.update_transforms(sc.xf[0])
    b.update_transforms(sc.xf[0])
    fa = a.trace(sc.tx, rx, prm)
    a.set_diffraction(False)
    fa0 = a.trace(sc.tx, rx, prm)
    fb = b.trace(sc.tx, rx, prm)
    assert fa0.paths.tobytes() == fb.paths.tobytes()
    d = (fa.paths["tri"][:, 0] & dcem.TRI_DIFFRACT) != 0
    assert d.any() and fa.paths[~d].tobytes() == fb.paths.tobytes()
    tx2 = sc.tx + np.array([5.0, -20.0, 0.0], np.float32)
    sl = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    sl.set_ray_sets([rays, rays])
    sl.set_diffraction(True)
    sl.update_transforms(sc.xf[0])
    fl = sl.trace_links(np.stack([sc.tx, tx2]), rx, prm)
    a.set_diffraction(True)
    for t, tx in enumerate((sc.tx, tx2)):
        single = a.trace(tx, rx, prm)
        p = fl.paths[fl.paths["tx"] == t].copy()
        p["tx"] = 0
        p["ray"] = np.where(p["ray"] >= 0, p["ray"] - t * rays.shape[0], -1)
        assert p.tobytes() == single.paths.tobytes(), t
        assert np.array_equal(fl.p_coh_dbm[t], single.p_coh_dbm)
    for s in (a, b, sl):
        s.close()


def test_highway_vehicle_wedges(cuda):
    """Wedges of the moving vehicle boxes follow their objects frame by
    frame (with the barrier wedges): same paths and fields as the oracle,
    which finds the wedges anew from each frame's world triangles."""
    sc = scenes.highway(n_frames=4, n_vehicles=60, length=600.0)
    _check(cuda, sc, 50_000, 2, range(4), mode=dcem.MODE_COHERENT, min_diff=4)


def test_many_receivers_grow_the_survivor_list(cuda):
    """A street grid of 4096 receivers against every wedge of a reduced urban
    grid: more pairs pass the FP32 pre-test than the survivor list's initial
    1024 slots (there are more diffraction paths than that, and each comes
    from a survivor), so the frame grows the list and is traced again. Its
    diffraction paths must equal, record for record, those of the same frame
    traced in eight batches of 512 receivers."""
    torch = cuda
    sc = scenes.urban_grid(blocks=2, parcels=2, n_vehicles=12, n_tx=1, budgets=(20_000, 20_000), n_static_rx=4,
                           n_frames=2, max_refl=2)
    lo, hi = sc.tris.reshape(-1, 3).min(axis=0), sc.tris.reshape(-1, 3).max(axis=0)
    g = np.stack(np.meshgrid(np.linspace(lo[0] + 1, hi[0] - 1, 64), np.linspace(lo[1] + 1, hi[1] - 1, 64),
                             indexing="ij"), -1).reshape(-1, 2)
    rx = np.concatenate([g, np.full((g.shape[0], 1), 1.5)], 1).astype(np.float32)
    tx = sc.meta["tx"][0]
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(scenes.fibonacci_sphere(20_000))
    s.set_diffraction(True)
    prm = dcem.default_params(max_refl=2, freq_hz=28e9)
    s.update_transforms(sc.xf[1])
    whole = s.trace(tx, rx, prm, max_paths=1 << 20)
    dw = whole.paths[(whole.paths["tri"][:, 0] & dcem.TRI_DIFFRACT) != 0]
    assert dw.shape[0] > 1024
    parts = []
    for k in range(8):
        sl = slice(512 * k, 512 * (k + 1))
        fr = s.trace(tx, rx[sl], prm, max_paths=1 << 18)
        p = fr.paths[(fr.paths["tri"][:, 0] & dcem.TRI_DIFFRACT) != 0].copy()
        p["rx"] += 512 * k
        parts.append(p)
    db = np.concatenate(parts)
    # a first-order diffraction path is its (receiver, wedge); the record key
    # hashes the receiver's index within its call, so it is not compared
    wa, wb = dw["tri"][:, 0], db["tri"][:, 0]
    assert sorted(zip(dw["rx"].tolist(), wa.tolist())) == sorted(zip(db["rx"].tolist(), wb.tolist()))
    oa = np.lexsort((wa, dw["rx"]))
    ob = np.lexsort((wb, db["rx"]))
    for f in ("len_m", "amp_re", "amp_im"):
        assert np.array_equal(dw[f][oa], db[f][ob]), f
    s.close()
