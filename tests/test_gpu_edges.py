"""Edge cases and full-size checks of the CUDA path through the C ABI.

Degenerate scenes (no geometry, one triangle), no rays, no receivers, the
direct path only, deep reflection orders, non-finite inputs, calls out of
order, too-small outputs, internal capacity growth; and the full highway
frame (1M rays) checked on sampled rays and on every path against the
FP64 oracle.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_07115_gb300 import dcem, scenes
from tests import parity as P

pytestmark = pytest.mark.gpu
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


def make(torch, sc, n_rays):
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(scenes.fibonacci_sphere(n_rays))
    return s


def gpu_keys(fr, N):
    return set(P.path_keys(fr.paths, N))


# ------------------------------------------------------------------ degenerate scenes

@pytest.mark.parametrize("freq", [28e9, 5.9e9])
def test_free_space_friis(cuda, freq):
    sc = scenes.free_space(tx=(1.0, -2.0, 3.0), rx=((101.0, -2.0, 3.0), (1.0, 248.0, 3.0)), freq_hz=freq)
    s = make(cuda, sc, 4000)
    fr = s.trace(sc.tx, sc.rx[0], dcem.default_params(max_refl=3, freq_hz=freq))
    assert fr.stats["paths_valid"] == 2 and set(fr.paths["depth"]) == {0}
    fspl1 = 20 * np.log10(4 * np.pi * freq / C0)
    for r, d in ((0, 100.0), (1, 250.0)):
        want = 10 * np.log10(5.0) + 30 - (fspl1 + 20 * np.log10(d))
        assert abs(fr.p_coh_dbm[r] - want) < 1e-6 and abs(fr.p_inc_dbm[r] - want) < 1e-6
        p = fr.paths[fr.paths["rx"] == r][0]
        assert abs(p["len_m"] - d) < 1e-9 and abs(p["delay_s"] - d / C0) < 1e-18
    s.close()


def test_single_triangle_scene(cuda):
    tri = np.array([[[-50, -50, 0], [50, -50, 0], [0, 60, 0]]], np.float32)
    sc = scenes._static_scene("one", tri, [scenes.MAT_CONCRETE], (0, 0, 5), ((20, 0, 2),))
    s = make(cuda, sc, 20000)
    fr = s.trace(sc.tx, sc.rx[0], dcem.default_params(max_refl=2))
    ek, ep = O.exhaustive(tri.reshape(-1, 9), sc.tri_mat, sc.materials, sc.tx, sc.rx[0],
                          O.OracleParams(max_refl=2, n_rays=20000))
    assert gpu_keys(fr, 2) == {tuple(k) for k in ek}
    _, pc, pi = O.reduce(ek, ep, 1, 5.0)
    assert abs(fr.p_coh_dbm[0] - pc[0]) < 1e-3 and abs(fr.p_inc_dbm[0] - pi[0]) < 1e-3
    s.close()


def test_plates_deep_reflections(cuda):
    """Two PEC plates, 10 reflections (the paper's maximum order): every
    exhaustive image path is found and matches the oracle."""
    # the link runs along y = 100, far from the plates' diagonal edges
    sc = scenes.parallel_plates(h=10.0, tx=(0.0, 100.0, 3.0), rx=((40.0, 100.0, 7.0),))
    N = 10
    s = make(cuda, sc, 400_000)
    fr = s.trace(sc.tx, sc.rx[0], dcem.default_params(max_refl=N))
    prm = O.OracleParams(max_refl=N, n_rays=400_000)
    ek, ep = O.exhaustive(sc.tris.reshape(-1, 9), sc.tri_mat, sc.materials, sc.tx, sc.rx[0], prm)
    assert gpu_keys(fr, N) == {tuple(k) for k in ek}
    ref = dict(zip(map(tuple, ek), ep))
    for key, p in zip(P.path_keys(fr.paths, N), fr.paths):
        assert abs(p["len_m"] - ref[key]["len_m"]) < 1e-6
        za, zb = complex(p["amp_re"], p["amp_im"]), complex(ref[key]["amp_re"], ref[key]["amp_im"])
        assert abs(za - zb) <= 1e-4 * abs(zb)
    s.close()


def test_direct_path_only(cuda):
    sc = scenes.toy_street()
    s = make(cuda, sc, 10_000)
    s.update_transforms(sc.xf[0])
    fr = s.trace(sc.tx, sc.rx[0], dcem.default_params(max_refl=0))
    assert set(fr.paths["depth"]) <= {0}
    ids, t, ns = s.ray_log()
    assert ids.shape[1] == 1 and np.all(ns == 1)
    ref = O.frame(sc, 0, scenes.fibonacci_sphere(10_000), O.OracleParams(max_refl=0, n_rays=10_000))
    want = {tuple(k) for k, p in zip(ref.keys, ref.paths) if p["valid"]}
    assert gpu_keys(fr, 0) == want
    s.close()


def test_no_rays_and_no_receivers(cuda):
    sc = scenes.toy_street()
    s = make(cuda, sc, 0)
    fr = s.trace(sc.tx, sc.rx[0], dcem.default_params())
    assert fr.status == dcem.OK and fr.stats["paths_valid"] == 0
    assert np.all(np.isneginf(fr.p_coh_dbm)) and np.all(np.isneginf(fr.p_inc_dbm))
    s.set_rays(scenes.fibonacci_sphere(1000))
    fr = s.trace(sc.tx, np.zeros((0, 3), np.float32), dcem.default_params())
    assert fr.status == dcem.OK and fr.stats["paths_valid"] == 0 and fr.stats["candidates"] == 0
    s.close()


# ------------------------------------------------------------------ errors

def test_status_errors(cuda):
    torch = cuda
    sc = scenes.toy_street()
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    fr = s.trace(sc.tx, sc.rx[0], dcem.default_params(), raise_on_error=False)
    assert fr.status == dcem.ERR_STATE                      # no rays yet
    s.set_rays(scenes.fibonacci_sphere(2000))
    bad = sc.xf[0].copy()
    bad[1, 3] = np.nan
    with pytest.raises(dcem.DcemError) as e:
        s.update_transforms(bad)
    assert e.value.status == dcem.ERR_NONFINITE
    rxb = sc.rx[0].copy()
    rxb[2, 0] = np.inf
    assert s.trace(sc.tx, rxb, dcem.default_params(), raise_on_error=False).status == dcem.ERR_NONFINITE
    # non-finite receivers given on the device are found by the device
    rxd = torch.from_numpy(rxb).cuda()
    assert s.trace(sc.tx, rxd, dcem.default_params(), raise_on_error=False).status == dcem.ERR_NONFINITE
    # non-finite transforms given on the device are reported by the next frame
    s.update_transforms(torch.from_numpy(bad).cuda())
    assert s.trace(sc.tx, sc.rx[0], dcem.default_params(), raise_on_error=False).status == dcem.ERR_NONFINITE
    for kw in ({"max_refl": 11}, {"max_refl": -1}, {"freq_hz": 0.0}, {"rx_radius_scale": 0.0},
               {"eps_occ": 0.6}, {"mode": 7}, {"pol": (0.0, 0.0, 0.0)}):
        assert s.trace(sc.tx, sc.rx[0], dcem.default_params(**kw), raise_on_error=False).status == dcem.ERR_ARG
    # the scene still works after every error
    s.update_transforms(sc.xf[0])
    assert s.trace(sc.tx, sc.rx[0], dcem.default_params()).stats["paths_valid"] > 0
    s.close()


def test_output_capacity(cuda):
    sc = scenes.toy_street()
    s = make(cuda, sc, 10_000)
    s.update_transforms(sc.xf[0])
    full = s.trace(sc.tx, sc.rx[0], dcem.default_params())
    n = len(full.paths)
    assert n > 3
    small = s.trace(sc.tx, sc.rx[0], dcem.default_params(), max_paths=3, raise_on_error=False)
    assert small.status == dcem.ERR_CAPACITY and small.stats["paths_valid"] == n
    assert small.paths.tobytes() == full.paths[:3].tobytes()
    assert np.array_equal(small.p_coh_dbm, full.p_coh_dbm)
    s.close()


def test_internal_capacity_growth(cuda):
    """Thousands of receivers near the transmitter overflow the initial
    capture buffers; the frame is retraced with larger ones and equals a
    frame traced with the grown buffers from the start."""
    g = np.linspace(-40.0, 40.0, 64, dtype=np.float32)
    X, Y = np.meshgrid(g, g)
    rx = np.stack([X.ravel(), Y.ravel(), np.full(X.size, 1.5, np.float32)], 1)
    sc = scenes.ground_plane(tx=(0.0, 0.0, 20.0), rx=rx, half=500.0)
    s = make(cuda, sc, 300_000)
    prm = dcem.default_params(max_refl=1, rx_radius_scale=6.0)
    a = s.trace(sc.tx, sc.rx[0], prm, max_paths=1 << 15)
    assert a.stats["candidates"] > 65536
    b = s.trace(sc.tx, sc.rx[0], prm, max_paths=1 << 15)
    assert a.paths.tobytes() == b.paths.tobytes() and np.array_equal(a.p_coh_dbm, b.p_coh_dbm)
    s.close()


# ------------------------------------------------------------------ full size

def test_highway_full_size_sampled(cuda):
    """1M rays, 4 reflections, 200 vehicles: hit ids and captures of every
    100th ray against the oracle; every path the GPU reports re-validated
    by the oracle; per-receiver power over the same path set within 0.01 dB;
    and the coherent frame equal to the full retrace."""
    torch = cuda
    sc = scenes.highway(n_frames=3)
    rays = scenes.fibonacci_sphere(sc.n_rays)
    a, b = make(torch, sc, sc.n_rays), make(torch, sc, sc.n_rays)
    for f in range(3):
        a.update_transforms(sc.xf[f])
        b.update_transforms(sc.xf[f])
        fa = a.trace(sc.tx, sc.rx[f], P.gpu_params(sc, mode=dcem.MODE_COHERENT))
        fb = b.trace(sc.tx, sc.rx[f], P.gpu_params(sc))
        assert fa.paths.tobytes() == fb.paths.tobytes()
        assert np.array_equal(fa.p_coh_dbm, fb.p_coh_dbm)
    f = 2
    ids, t, ns = b.ray_log()
    sample = np.arange(0, sc.n_rays, 100)
    wt = O.transform(sc.tris, sc.tri_obj, sc.xf[f])
    prm = P.oracle_params(sc)
    tr = O.trace(wt, sc.tri_mat, sc.materials, sc.tx, rays[sample], sc.rx[f], prm)
    flagged = (tr["flags"] & P.RAY_FLAGS) != 0
    same = np.all(ids[sample] == tr["hit_id"], axis=1) & (ns[sample] == tr["nseg"])
    assert np.all(same | flagged), np.nonzero(~(same | flagged))[0][:10]
    assert flagged.mean() < 0.05
    # captures of the sampled rays
    cand = b.candidates()
    pos = {int(r): i for i, r in enumerate(sample)}
    gsel = {(pos[c[0]], c[1], c[2]) for c in cand.tolist() if c[0] in pos and not flagged[pos[c[0]]]}
    osel = {tuple(c) for c in tr["cands"].tolist() if not flagged[c[0]]}
    assert gsel == osel
    # every reported path, re-validated in FP64
    keys = np.array(sorted(P.path_keys(fb.paths, sc.max_refl)), np.int32)
    ref = O.validate(wt, sc.tri_mat, sc.materials, sc.tx, sc.rx[f], keys, prm)
    clean = (ref["flags"] & P.PATH_FLAGS) == 0
    assert np.all(ref["valid"][clean] == 1)
    gp = dict(zip(P.path_keys(fb.paths, sc.max_refl), fb.paths))
    for k, r in zip(map(tuple, keys), ref):
        if r["valid"]:
            assert abs(gp[k]["len_m"] - r["len_m"]) < 1e-6
    _, pc, pi = O.reduce(keys, ref, sc.nrx, 5.0)
    assert np.all(P.power_close(fb.p_coh_dbm, pc)) and np.all(P.power_close(fb.p_inc_dbm, pi))
    a.close()
    b.close()


@pytest.mark.parametrize("freq", [5.9e9, 28e9])
def test_highway_reduced_both_bands(cuda, freq):
    sc = scenes.highway(n_frames=2, n_vehicles=40, length=400.0, n_rays=100_000, freq_hz=freq)
    rays = scenes.fibonacci_sphere(sc.n_rays)
    s = make(cuda, sc, sc.n_rays)
    s.update_transforms(sc.xf[1])
    fr = s.trace(sc.tx, sc.rx[1], P.gpu_params(sc))
    ref = O.frame(sc, 1, rays, P.oracle_params(sc))
    out = P.compare_paths(fr, ref, sc.max_refl)
    assert out["checked"] > 0 and not out["missing"] and not out["extra"] and not out["amp"]
    assert np.all(P.power_close(fr.p_coh_dbm, ref.p_coh_dbm))
    s.close()


@pytest.mark.parametrize("tx", [(600.0, 300.0, 300.0), (5e4, 300.0, 2.5e4)])
def test_far_transmitter(cuda, tx):
    """Rays aimed at the street from outside it. From (600, 300, 300) every
    segment stays within the compact node copy's reach; from 50 km away
    (far beyond 4e6 grid steps of the 200 m street: about 12 km across, 1 km
    vertically) first segments take the full-precision nodes and later ones,
    starting in the street, the compact copy. Hit ids equal the oracle's on
    every unflagged ray."""
    torch = cuda
    sc = scenes.toy_street(n_rays=20_000, max_refl=3)
    f = 3
    sc.tx = np.array(tx, np.float32)
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([7, int(tx[0])])))
    aim = rng.uniform([-100.0, -100.0, 0.0], [100.0, 100.0, 15.0], size=(20_000, 3))
    d = aim - sc.tx.astype(np.float64)
    rays = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    rx = sc.rx[f][:1]
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(rays)
    s.update_transforms(sc.xf[f])
    fr = s.trace(sc.tx, rx, P.gpu_params(sc), max_paths=1 << 16)
    ids, t, ns = s.ray_log()
    s.close()
    wt = O.transform(sc.tris, sc.tri_obj, sc.xf[f])
    ref = O.trace(wt, sc.tri_mat, sc.materials, sc.tx, rays, rx, P.oracle_params(sc, n_rays=20_000))
    n, nflag, bad = P.compare_hits(ids, ns, ref)
    assert len(bad) == 0, (len(bad), bad[:5])
    assert n > 15_000
    # most aimed rays hit the street
    assert (ns > 1).mean() > 0.5
    assert fr.status == dcem.OK
