"""The path cache's retention mode (DCEM_MODE_STICKY) against the oracle.

Sec. III "Propagation path caching" keeps cached paths and updates them until
they are removed: besides the paths its rays capture, a frame reports every
path of the previous frame that is still valid under the current geometry
(re-validated; flag DCEM_PATH_STICKY when no ray captured it). The oracle's
``sticky_frames`` states that rule directly; the GPU must report the same
valid key sets (keys the oracle flags as within FP32 margins excepted), the
same kept-only subset, and lengths and amplitudes within the parity
tolerances.
"""
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


def _uncertain(r):
    """Keys of an oracle frame that FP32 may decide either way: validation
    near a triangle edge or an occluder, or discovered only by rays within
    the FP32 margins."""
    out = {tuple(k) for k, p in zip(r.keys.tolist(), r.paths) if p["flags"] & P.PATH_FLAGS}
    flagged = (r.tr["flags"] & P.RAY_FLAGS) != 0
    ck = O.candidate_keys(r.tr["cands"], r.tr["hit_id"], r.keys.shape[1] - 2)
    by_clean = {tuple(k) for k, c in zip(ck.tolist(), r.tr["cands"].tolist()) if not flagged[c[0]]}
    out |= {tuple(k) for k, c in zip(ck.tolist(), r.tr["cands"].tolist()) if flagged[c[0]]} - by_clean
    return out


def _run_sticky(torch, sc, n_rays, max_refl, frames):
    rays = scenes.fibonacci_sphere(n_rays)
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(rays)
    prm = P.gpu_params(sc, mode=dcem.MODE_STICKY, max_refl=max_refl)
    ref = O.sticky_frames(sc, frames, rays, P.oracle_params(sc, n_rays=n_rays, max_refl=max_refl))
    allowed = set()
    kept_total = 0
    for i, f in enumerate(frames):
        if sc.nobj:
            s.update_transforms(sc.xf[f])
        fr = s.trace(sc.tx, sc.rx[f], prm)
        r = ref[i]
        assert fr.stats["coherent"] == (1 if i else 0)
        allowed |= _uncertain(r)
        gk = P.path_keys(fr.paths, max_refl)
        gpu = dict(zip(gk, fr.paths))
        rv = {tuple(k): p for k, p in zip(r.keys.tolist(), r.paths) if p["valid"]}
        diff = set(gpu) ^ set(rv)
        assert diff <= allowed, (f, sorted(diff - allowed)[:5])
        allowed |= diff          # a difference may persist through the cache
        for k in set(gpu) & set(rv):
            assert abs(gpu[k]["len_m"] - rv[k]["len_m"]) <= 1e-6, (f, k)
            za = complex(gpu[k]["amp_re"], gpu[k]["amp_im"])
            zb = complex(rv[k]["amp_re"], rv[k]["amp_im"])
            assert abs(za - zb) <= 1e-4 * abs(zb), (f, k)
        sticky = {k for k, p in gpu.items() if p["flags"] & dcem.PATH_STICKY}
        kept = {tuple(k) for k in r.extra["kept_only"].tolist()}
        assert (sticky ^ kept) <= allowed, (f, sorted((sticky ^ kept) - allowed)[:5])
        assert fr.stats["paths_sticky"] == len(sticky)
        assert all(gpu[k]["ray"] == -1 for k in sticky)
        kept_total += len(kept)
    s.close()
    return kept_total


def test_sticky_toy_street(cuda):
    sc = scenes.toy_street()
    assert _run_sticky(cuda, sc, 200, 2, range(10)) > 0


def test_sticky_highway_reduced(cuda):
    sc = scenes.highway(n_frames=6, n_vehicles=60, length=600.0)
    assert _run_sticky(cuda, sc, 20_000, 3, range(6)) > 10


def test_sticky_contains_coherent_and_resets(cuda):
    """A sticky frame's paths contain the coherent frame's (the captured ones
    are the same); the first frame and a frame after the transmitter moved
    keep nothing."""
    sc = scenes.highway(n_frames=6, n_vehicles=60, length=600.0)
    rays = scenes.fibonacci_sphere(20_000)
    a = dcem.Scene.from_scene(sc, stream=cuda.cuda.current_stream().cuda_stream)
    b = dcem.Scene.from_scene(sc, stream=cuda.cuda.current_stream().cuda_stream)
    a.set_rays(rays)
    b.set_rays(rays)
    pa = P.gpu_params(sc, mode=dcem.MODE_STICKY)
    pb = P.gpu_params(sc, mode=dcem.MODE_COHERENT)
    for f in range(6):
        tx = sc.tx if f != 4 else sc.tx + np.array([0.5, 0.0, 0.0], np.float32)
        a.update_transforms(sc.xf[f])
        b.update_transforms(sc.xf[f])
        fa = a.trace(tx, sc.rx[f], pa)
        fb = b.trace(tx, sc.rx[f], pb)
        ka = dict(zip(P.path_keys(fa.paths, sc.max_refl), fa.paths))
        kb = dict(zip(P.path_keys(fb.paths, sc.max_refl), fb.paths))
        assert set(kb) <= set(ka)
        for k in kb:
            assert ka[k].tobytes() == kb[k].tobytes()
        if f in (0, 4):
            assert fa.stats["paths_sticky"] == 0 and fa.stats["coherent"] == 0
        assert set(ka) - set(kb) == {k for k, p in ka.items() if p["flags"] & dcem.PATH_STICKY}
    a.close()
    b.close()
