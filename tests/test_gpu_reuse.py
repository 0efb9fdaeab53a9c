"""Validation reuse in coherent frames (Sec. III "Propagation path caching").

A coherent frame copies the previous frame's validation of a distinct key
when nothing it depends on moved: its receiver, the objects of its triangles,
and (for a path whose geometry was valid) any moved object's old or new box
along its sub-segments. The copies must leave every output bit-identical to
a full retrace, and must be made (keys_reused > 0) where receivers are static.
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


def _scene(torch, sc, rays):
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(rays)
    return s


def _run(torch, sc, n_rays, frames, prm_coh=None, prm_full=None):
    """Coherent and full frames side by side; every output bit-identical.
    Returns the coherent frames' stats."""
    rays = scenes.fibonacci_sphere(n_rays)
    a, b = _scene(torch, sc, rays), _scene(torch, sc, rays)
    out = []
    for i, f in enumerate(frames):
        pa = prm_coh(i) if prm_coh else P.gpu_params(sc, mode=dcem.MODE_COHERENT)
        pb = prm_full(i) if prm_full else P.gpu_params(sc, mode=dcem.MODE_FULL)
        if sc.nobj:
            a.update_transforms(sc.xf[f])
            b.update_transforms(sc.xf[f])
        fa = a.trace(sc.tx, sc.rx[f], pa)
        fb = b.trace(sc.tx, sc.rx[f], pb)
        assert fa.paths.tobytes() == fb.paths.tobytes(), f"frame {f}: path records differ"
        assert np.array_equal(fa.p_coh_dbm, fb.p_coh_dbm) and np.array_equal(fa.p_inc_dbm, fb.p_inc_dbm)
        assert np.array_equal(fa.field, fb.field)
        out.append((fa.stats, fb))
    a.close()
    b.close()
    return out


def test_reuse_toy_street_equals_full(cuda):
    sc = scenes.toy_street()
    st = _run(cuda, sc, sc.n_rays, range(sc.nframes))
    reused = [x["keys_reused"] for x, _ in st]
    assert reused[0] == 0                                  # the first frame is a full trace
    assert all(r > 0 for r in reused[1:])                  # static receivers: copies in every later frame
    # vehicles moved: some keys were validated anew over the run
    assert sum(x["unique_candidates"] - x["keys_reused"] for x, _ in st[1:]) > 0


def _crossing_box(n_frames=7):
    """Ground, a static side wall, a static Tx and Rx with a line of sight
    along x, and one metal box that crosses that line (the middle frame blocks it)."""
    ground = scenes._quad((-200, -200, 0), (200, -200, 0), (200, 200, 0), (-200, 200, 0))
    wall = scenes._quad((-50, 15, 0), (80, 15, 0), (80, 15, 12), (-50, 15, 12))
    box = scenes.box_tris(2.0, 2.0, 4.0)
    tris, tobj, tmat = scenes._assemble(ground + wall, [scenes.MAT_CONCRETE] * 4, [box], [scenes.MAT_METAL])
    ys = np.linspace(-9.0, 9.0, n_frames)
    xf = np.zeros((n_frames, 1, 12), np.float32)
    for f, y in enumerate(ys):
        xf[f, 0] = scenes._xf_row(0.0, 20.0, float(y), 0.0)
    rx = np.broadcast_to(np.array([[40.0, 0.0, 2.0]], np.float32), (n_frames, 1, 3)).copy()
    return scenes.Scene("crossing", tris, tobj, tmat, scenes.default_materials(), 1, xf,
                        np.array([0.0, 0.0, 2.0], np.float32), rx, n_rays=200_000, max_refl=2)


def test_reuse_when_an_occluder_crosses_a_cached_path(cuda):
    sc = _crossing_box()
    st = _run(cuda, sc, sc.n_rays, range(sc.nframes))
    los = []
    for stats, fb in st:
        los.append(any(int(p["depth"]) == 0 for p in fb.paths))
    # the scene does what it is meant to: the box blocks the direct path in the middle frames
    assert los[0] and los[-1] and not all(los)
    assert sum(x["keys_reused"] for x, _ in st[1:]) > 0


def test_no_reuse_across_a_frequency_change(cuda):
    """A coherent frame at another frequency reuses segments but no validation."""
    sc = scenes.toy_street()
    freqs = [28e9, 5.9e9, 5.9e9]
    st = _run(cuda, sc, sc.n_rays, [1, 2, 3],
              prm_coh=lambda i: dcem.default_params(max_refl=sc.max_refl, freq_hz=freqs[i],
                                                    mode=dcem.MODE_COHERENT),
              prm_full=lambda i: dcem.default_params(max_refl=sc.max_refl, freq_hz=freqs[i],
                                                     mode=dcem.MODE_FULL))
    assert st[1][0]["coherent"] == 1 and st[1][0]["keys_reused"] == 0
    assert st[2][0]["keys_reused"] > 0


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_reuse_random_scenes_equal_full(cuda, seed):
    sc = scenes.random_tiny(seed, ntri=24, nobj=3, n_frames=5, nrx=6, n_rays=50_000, max_refl=3)
    st = _run(cuda, sc, sc.n_rays, range(sc.nframes))
    assert st[0][0]["keys_reused"] == 0


def test_reuse_matches_oracle(cuda):
    """Reused records still agree with the FP64 oracle (toy street, last frame)."""
    sc = scenes.toy_street()
    rays = scenes.fibonacci_sphere(sc.n_rays)
    s = _scene(cuda, sc, rays)
    prm = P.gpu_params(sc, mode=dcem.MODE_COHERENT)
    for f in range(4):
        s.update_transforms(sc.xf[f])
        fr = s.trace(sc.tx, sc.rx[f], prm)
    assert fr.stats["keys_reused"] > 0
    ref = O.frame(sc, 3, rays, P.oracle_params(sc))
    res = P.compare_paths(fr, ref, sc.max_refl)
    assert res["checked"] > 0
    assert not res["missing"] and not res["extra"] and not res["len"] and not res["amp"], res
    assert np.all(P.power_close(fr.p_coh_dbm, ref.p_coh_dbm))
    s.close()
