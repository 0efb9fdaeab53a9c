"""Closest-hit kernel configurations (dcem_scene_set_trace_config) and the
autotuner (dcem_scene_autotune).

The closest hit and its lowest-id tie rule are decided by the triangle test
alone, so every kernel (binary nodes from global memory, the 4-wide compact
copy in shared memory or read from global memory), block size and stack
depth must give the same bits: ray logs, path records and power. One
configuration per scene is also checked against the oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_07115_gb300 import dcem, scenes
from tests import parity as P

pytestmark = pytest.mark.gpu

CONFIGS = [(1, 256, 24), (2, 256, 24), (2, 128, 16), (2, 64, 8), (0, 256, 24), (0, 128, 32)]


@pytest.fixture(scope="module")
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_07115_gb300 import build
    build.build()
    O.build()
    torch.cuda.set_device(0)
    return torch


def _run(torch, sc, rays, cfg, frames, mode):
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(rays)
    if cfg is not None:
        s.set_trace_config(*cfg)
    prm = P.gpu_params(sc, mode=mode)
    out = []
    for f in frames:
        if sc.nobj:
            s.update_transforms(sc.xf[f])
        fr = s.trace(sc.tx, sc.rx[f], prm)
        out.append((fr, s.ray_log()))
    s.close()
    return out


@pytest.mark.parametrize("which", ["toy", "highway", "urban"])
@pytest.mark.parametrize("mode", [dcem.MODE_FULL, dcem.MODE_COHERENT])
def test_kernel_configs_identical(cuda, which, mode):
    if which == "toy":
        sc, n = scenes.toy_street(), 10_000
    elif which == "highway":
        sc, n = scenes.highway(n_frames=4, n_vehicles=60, length=600.0), 150_000
    else:
        sc = scenes.urban_grid(blocks=3, parcels=2, n_vehicles=30, n_tx=1, n_static_rx=8, n_frames=4,
                               max_refl=5)
        n = 60_000
    rays = scenes.fibonacci_sphere(n)
    ref = _run(cuda, sc, rays, None, range(4), mode)
    for cfg in CONFIGS:
        got = _run(cuda, sc, rays, cfg, range(4), mode)
        for f, ((fa, la), (fb, lb)) in enumerate(zip(ref, got)):
            assert fb.stats["trace_kernel"] == cfg[0], (cfg, fb.stats["trace_kernel"])
            assert fa.paths.tobytes() == fb.paths.tobytes(), (cfg, f)
            assert np.array_equal(fa.p_coh_dbm, fb.p_coh_dbm), (cfg, f)
            assert np.array_equal(la[0], lb[0]) and np.array_equal(la[2], lb[2]), (cfg, f)
            assert np.array_equal(la[1].view(np.uint32), lb[1].view(np.uint32)), (cfg, f)


def test_global_compact_copy_vs_oracle(cuda):
    """The 4-wide copy read from global memory against the oracle (hits of
    unflagged rays, paths, lengths, amplitudes)."""
    sc = scenes.urban_grid(blocks=2, parcels=2, n_vehicles=12, n_tx=1, n_static_rx=4, n_frames=3, max_refl=5)
    rays = scenes.fibonacci_sphere(30_000)
    s = dcem.Scene.from_scene(sc, stream=cuda.cuda.current_stream().cuda_stream)
    s.set_rays(rays)
    s.set_trace_config(2, 128, 16)
    for f in (0, 2):
        s.update_transforms(sc.xf[f])
        fr = s.trace(sc.tx, sc.rx[f], P.gpu_params(sc))
        assert fr.stats["trace_kernel"] == 2
        ids, t, ns = s.ray_log()
        ref = O.frame(sc, f, rays, P.oracle_params(sc, n_rays=30_000))
        _, _, bad = P.compare_hits(ids, ns, ref.tr)
        assert len(bad) == 0, bad[:5]
        res = P.compare_paths(fr, ref, sc.max_refl)
        assert res["checked"] > 0
        assert not res["missing"] and not res["extra"] and not res["len"] and not res["amp"]
    s.close()


def test_autotune(cuda):
    sc = scenes.highway(n_frames=3, n_vehicles=60, length=600.0)
    rays = scenes.fibonacci_sphere(150_000)
    s = dcem.Scene.from_scene(sc, stream=cuda.cuda.current_stream().cuda_stream)
    s.set_rays(rays)
    s.update_transforms(sc.xf[1])
    prm = P.gpu_params(sc, mode=dcem.MODE_COHERENT)
    k, b, st = s.autotune(sc.tx, sc.rx[1], prm, reps=2)
    assert k in (0, 1, 2) and b in (64, 128, 256, 768) and 8 <= st <= 32
    fr = s.trace(sc.tx, sc.rx[1], prm)
    assert fr.stats["trace_kernel"] == k and fr.stats["coherent"] == 0
    ref = _run(cuda, sc, rays, None, [1], dcem.MODE_FULL)[0][0]
    assert fr.paths.tobytes() == ref.paths.tobytes()
    with pytest.raises(dcem.DcemError):
        s.set_trace_config(3)
    with pytest.raises(dcem.DcemError):
        s.set_trace_config(2, 96, 24)
    with pytest.raises(dcem.DcemError):
        s.set_trace_config(2, 128, 40)
    s.close()


def test_large_tree_compact_copy(cuda):
    """A scene whose 4-wide mapping needs global scratch (over 25,600 internal
    nodes) and whose compact copy does not fit in shared memory: kernel 1 is
    refused, the automatic choice is kernel 2, and kernels 2 and 0 agree
    bit for bit, also after a rebuild of the moving-object tree (which
    remaps the copy)."""
    big = scenes.urban_grid(blocks=8, parcels=4, n_vehicles=60, n_tx=1, n_static_rx=4, n_frames=3, max_refl=4)
    assert big.ntri > 30_000
    rays = scenes.fibonacci_sphere(50_000)
    outs = []
    for cfg in (None, (0, 256, 24)):
        s = dcem.Scene.from_scene(big, stream=cuda.cuda.current_stream().cuda_stream)
        s.set_rays(rays)
        with pytest.raises(dcem.DcemError):
            s.set_trace_config(1)
        if cfg:
            s.set_trace_config(*cfg)
        s.set_rebuild_threshold(1.0001)
        got = []
        for f in range(3):
            s.update_transforms(big.xf[f])
            fr = s.trace(big.tx, big.rx[f], P.gpu_params(big))
            assert fr.stats["trace_kernel"] == (cfg[0] if cfg else 2)
            got.append((fr.paths.tobytes(), fr.p_coh_dbm.copy(), s.ray_log()[0].copy()))
        s.close()
        outs.append(got)
    for (pa, ca, la), (pb, cb, lb) in zip(*outs):
        assert pa == pb and np.array_equal(ca, cb) and np.array_equal(la, lb)
