"""CUDA path (through the C ABI) against the FP64 CPU oracle.

Bit-exact: world vertices (fmaf transform), refit bounds (min/max), hit
triangle ids per segment and captures of rays the oracle does not flag as
within the FP32 margin of an edge, tie, self-hit offset or sphere boundary.
Within tolerance: path lengths (1e-6 m), amplitudes (1e-6 relative), and
per-receiver power (0.01 dB). Coherent frames must equal full retraces bit
for bit.
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


def make_scene(torch, sc, rays):
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(rays)
    return s


# ------------------------------------------------------------------ geometry

@pytest.mark.parametrize("which", ["toy", "highway"])
def test_transform_bitexact(cuda, which):
    sc = scenes.toy_street() if which == "toy" else scenes.highway(n_frames=6, n_vehicles=60,
                                                                   length=600.0)
    s = make_scene(cuda, sc, scenes.fibonacci_sphere(16))
    for f in range(sc.nframes):
        s.update_transforms(sc.xf[f])
        w = s.world_tris()
        ref = O.transform(sc.tris, sc.tri_obj, sc.xf[f])
        assert np.array_equal(w.view(np.uint32), ref.view(np.uint32)), f"frame {f}"
    s.close()


def _check_tree(child, bounds, root, world, nodes_range, tri_ids):
    """Every triangle of the tree reached once; every child box is the exact
    min/max of its subtree's vertices."""
    lo_n, hi_n = nodes_range
    seen = []

    def box_of_tri(t):
        v = world[t]
        return np.concatenate([v.min(axis=0), v.max(axis=0)])

    def walk(code):
        if code < 0:
            t = -code - 1
            seen.append(t)
            return box_of_tri(t)
        assert lo_n <= code < hi_n
        b0 = walk(int(child[code, 0]))
        b1 = walk(int(child[code, 1]))
        assert np.array_equal(bounds[code, 0].view(np.uint32), b0.astype(np.float32).view(np.uint32))
        assert np.array_equal(bounds[code, 1].view(np.uint32), b1.astype(np.float32).view(np.uint32))
        return np.concatenate([np.minimum(b0[:3], b1[:3]), np.maximum(b0[3:], b1[3:])])

    if root == np.iinfo(np.int32).min:
        assert len(tri_ids) == 0
        return
    walk(int(root))
    assert sorted(seen) == sorted(tri_ids)


@pytest.mark.parametrize("which", ["toy", "highway", "tiny"])
def test_bvh_structure_and_refit_bounds(cuda, which):
    if which == "toy":
        sc = scenes.toy_street()
    elif which == "highway":
        sc = scenes.highway(n_frames=4, n_vehicles=80, length=800.0)
    else:
        sc = scenes.random_tiny(3, ntri=12, nobj=3, n_frames=4)
    s = make_scene(cuda, sc, scenes.fibonacci_sphere(16))
    for f in range(sc.nframes):
        if sc.nobj:
            s.update_transforms(sc.xf[f])
        child, bounds, roots, info = s.bvh()
        world = s.world_tris()
        ns = info["static_nodes"]
        st_ids = np.nonzero(sc.tri_obj < 0)[0].tolist()
        dy_ids = np.nonzero(sc.tri_obj >= 0)[0].tolist()
        _check_tree(child, bounds, roots[0], world, (0, ns), st_ids)
        _check_tree(child, bounds, roots[1], world, (ns, ns + info["dynamic_nodes"]), dy_ids)
    s.close()


# ------------------------------------------------------------------ frames

def _frame_vs_oracle(torch, sc, frames, n_rays=None, mode=dcem.MODE_FULL, check_paths=True,
                     prec=dcem.PREC_F64):
    n_rays = n_rays or sc.n_rays
    rays = scenes.fibonacci_sphere(n_rays)
    s = make_scene(torch, sc, rays)
    prm = P.gpu_params(sc, mode=mode, prec=prec)
    oprm = P.oracle_params(sc, n_rays=n_rays)
    report = []
    for f in frames:
        if sc.nobj:
            s.update_transforms(sc.xf[f])
        fr = s.trace(sc.tx, sc.rx[f], prm)
        ids, t, ns = s.ray_log()
        ref = O.frame(sc, f, rays, oprm)
        cmp_n, nflag, bad = P.compare_hits(ids, ns, ref.tr)
        assert len(bad) == 0, f"frame {f}: {len(bad)} unflagged rays differ, e.g. {bad[:5]}"
        g, r = P.compare_candidates(s.candidates(), ref.tr)
        assert g == r, f"frame {f}: captures differ {len(g ^ r)}"
        if check_paths:
            out = P.compare_paths(fr, ref, sc.max_refl)
            assert not out["missing"] and not out["extra"], out
            assert not out["len"] and not out["amp"], out
            assert np.all(P.power_close(fr.p_inc_dbm, ref.p_inc_dbm)), (fr.p_inc_dbm, ref.p_inc_dbm)
            assert np.all(P.power_close(fr.p_coh_dbm, ref.p_coh_dbm)), (fr.p_coh_dbm, ref.p_coh_dbm)
        report.append((f, cmp_n, nflag, fr.stats["paths_valid"]))
    s.close()
    return report


def test_toy_street_full_vs_oracle(cuda):
    sc = scenes.toy_street()
    rep = _frame_vs_oracle(cuda, sc, range(sc.nframes))
    assert all(r[3] > 0 for r in rep)


def test_toy_street_more_rays_and_reflections(cuda):
    sc = scenes.toy_street(n_rays=60_000, max_refl=5, seed=3)
    _frame_vs_oracle(cuda, sc, [0, 4, 9])


def test_highway_reduced_vs_oracle(cuda):
    sc = scenes.highway(n_frames=4, n_vehicles=40, length=400.0, n_rays=100_000, max_refl=4)
    _frame_vs_oracle(cuda, sc, range(4))


@pytest.mark.parametrize("which", ["toy", "highway"])
def test_double_float_validation_vs_oracle(cuda, which):
    """Validation geometry and phase in double-float (DCEM_PREC_DF32): the
    same path set, lengths within 1e-6 m, amplitudes within 1e-6 and power
    within 0.01 dB of the FP64 oracle."""
    if which == "toy":
        sc = scenes.toy_street()
        frames = range(sc.nframes)
    else:
        sc = scenes.highway(n_frames=3, n_vehicles=40, length=400.0, n_rays=100_000, max_refl=4)
        frames = range(3)
    _frame_vs_oracle(cuda, sc, frames, prec=dcem.PREC_DF32)


def test_double_float_matches_fp64_paths(cuda):
    """Both precisions give the same path records up to ~1e-10 in length and
    amplitude (the double-float geometry carries about 44 bits)."""
    sc = scenes.highway(n_frames=2, n_vehicles=60, length=600.0, n_rays=200_000, max_refl=4)
    rays = scenes.fibonacci_sphere(sc.n_rays)
    out = []
    for prec in (dcem.PREC_F64, dcem.PREC_DF32):
        s = make_scene(cuda, sc, rays)
        s.update_transforms(sc.xf[1])
        out.append(s.trace(sc.tx, sc.rx[1], P.gpu_params(sc, prec=prec)))
        s.close()
    a, b = out
    assert a.paths.shape == b.paths.shape and a.paths.shape[0] > 20
    assert np.array_equal(a.paths["key"], b.paths["key"])
    assert np.abs(a.paths["len_m"] - b.paths["len_m"]).max() < 1e-6
    amp_a = a.paths["amp_re"] + 1j * a.paths["amp_im"]
    amp_b = b.paths["amp_re"] + 1j * b.paths["amp_im"]
    assert np.abs(amp_a - amp_b).max() <= 1e-6 * np.abs(amp_a).max()
    fin = np.isfinite(a.p_coh_dbm)
    assert np.array_equal(fin, np.isfinite(b.p_coh_dbm))
    assert np.abs(a.p_coh_dbm[fin] - b.p_coh_dbm[fin]).max() < 1e-4


@pytest.mark.parametrize("seed", range(4))
def test_random_tiny_vs_oracle(cuda, seed):
    sc = scenes.random_tiny(seed, ntri=14, nobj=2, n_frames=3, nrx=3, n_rays=50_000, max_refl=3)
    _frame_vs_oracle(cuda, sc, range(3))


# ------------------------------------------------------------------ coherence

def _coherent_vs_full(torch, sc, n_rays, frames):
    rays = scenes.fibonacci_sphere(n_rays)
    a, b = make_scene(torch, sc, rays), make_scene(torch, sc, rays)
    pa = P.gpu_params(sc, mode=dcem.MODE_COHERENT)
    pb = P.gpu_params(sc, mode=dcem.MODE_FULL)
    reused = 0
    for i, f in enumerate(frames):
        if sc.nobj:
            a.update_transforms(sc.xf[f])
            b.update_transforms(sc.xf[f])
        fa = a.trace(sc.tx, sc.rx[f], pa)
        fb = b.trace(sc.tx, sc.rx[f], pb)
        assert fa.stats["coherent"] == (1 if i else 0)
        reused += fa.stats["segments_reused"]
        assert fa.paths.tobytes() == fb.paths.tobytes(), f"frame {f}: path records differ"
        assert np.array_equal(fa.p_coh_dbm, fb.p_coh_dbm) and np.array_equal(fa.p_inc_dbm, fb.p_inc_dbm)
        la, lb = a.ray_log(), b.ray_log()
        assert np.array_equal(la[0], lb[0]) and np.array_equal(la[2], lb[2])
        assert np.array_equal(la[1].view(np.uint32), lb[1].view(np.uint32))
    a.close()
    b.close()
    return reused


def test_coherent_equals_full_toy(cuda):
    sc = scenes.toy_street()
    assert _coherent_vs_full(cuda, sc, sc.n_rays, range(sc.nframes)) > 0


def test_coherent_equals_full_highway_reduced(cuda):
    sc = scenes.highway(n_frames=6, n_vehicles=60, length=600.0)
    assert _coherent_vs_full(cuda, sc, 200_000, range(6)) > 0


def test_coherent_static_rx_carries_captures(cuda):
    """Static receivers: captures of reused segments are carried over."""
    sc = scenes.toy_street()
    rays = scenes.fibonacci_sphere(sc.n_rays)
    s = make_scene(cuda, sc, rays)
    prm = P.gpu_params(sc, mode=dcem.MODE_COHERENT)
    s.update_transforms(sc.xf[0])
    s.trace(sc.tx, sc.rx[0], prm)
    s.update_transforms(sc.xf[1])
    fr = s.trace(sc.tx, sc.rx[1], prm)
    assert fr.stats["coherent"] == 1 and fr.stats["rx_moved"] == 0
    assert fr.stats["candidates_reused"] > 0
    assert fr.stats["rays_retraced"] < sc.n_rays
    s.close()


def test_coherent_nothing_moved(cuda):
    sc = scenes.toy_street()
    rays = scenes.fibonacci_sphere(sc.n_rays)
    s = make_scene(cuda, sc, rays)
    prm = P.gpu_params(sc, mode=dcem.MODE_COHERENT)
    s.update_transforms(sc.xf[2])
    f0 = s.trace(sc.tx, sc.rx[2], prm)
    s.update_transforms(sc.xf[2])
    f1 = s.trace(sc.tx, sc.rx[2], prm)
    assert f1.stats["coherent"] == 1 and f1.stats["segments_traced"] == 0
    assert f1.stats["candidates_reused"] == f0.stats["candidates"]
    assert f1.paths.tobytes() == f0.paths.tobytes()
    s.close()


# ------------------------------------------------------------------ BVH rebuilds

@pytest.mark.parametrize("ratio", [1.0001, 0.0])
def test_coherent_equals_full_with_rebuild_policy(cuda, ratio):
    """Rebuilding the moving-object tree every frame (ratio just above 1) or
    never (ratio 0) changes neither the paths nor the power."""
    sc = scenes.highway(n_frames=5, n_vehicles=60, length=600.0)
    rays = scenes.fibonacci_sphere(100_000)
    a, b = make_scene(cuda, sc, rays), make_scene(cuda, sc, rays)
    a.set_rebuild_threshold(ratio)
    pa = P.gpu_params(sc, mode=dcem.MODE_COHERENT)
    pb = P.gpu_params(sc, mode=dcem.MODE_FULL)
    rebuilt = 0
    for f in range(sc.nframes):
        a.update_transforms(sc.xf[f])
        b.update_transforms(sc.xf[f])
        fa = a.trace(sc.tx, sc.rx[f], pa)
        fb = b.trace(sc.tx, sc.rx[f], pb)
        rebuilt += fa.stats["bvh_rebuilt"]
        assert fa.paths.tobytes() == fb.paths.tobytes()
        assert np.array_equal(fa.p_coh_dbm, fb.p_coh_dbm)
        child, bounds, roots, info = a.bvh()
        world = a.world_tris()
        ns = info["static_nodes"]
        _check_tree(child, bounds, roots[1], world, (ns, ns + info["dynamic_nodes"]),
                    np.nonzero(sc.tri_obj >= 0)[0].tolist())
    if ratio > 1.0:
        # the cost measured by a frame's refit decides the next update, and a
        # rebuild resets the ratio to 1: at least every other frame rebuilds
        assert rebuilt >= sc.nframes // 2
    else:
        assert rebuilt <= 1   # the first update builds over the real positions
    a.close()
    b.close()


def test_coherent_after_trace_at_creation_pose(cuda):
    """A frame traced before any transform update (objects at identity) is a
    valid cache: the next coherent frame must see the objects' old boxes."""
    sc = scenes.toy_street()
    rays = scenes.fibonacci_sphere(sc.n_rays)
    a, b = make_scene(cuda, sc, rays), make_scene(cuda, sc, rays)
    pa = P.gpu_params(sc, mode=dcem.MODE_COHERENT)
    pb = P.gpu_params(sc, mode=dcem.MODE_FULL)
    a.trace(sc.tx, sc.rx[0], pa)
    a.update_transforms(sc.xf[0])
    b.update_transforms(sc.xf[0])
    fa = a.trace(sc.tx, sc.rx[0], pa)
    fb = b.trace(sc.tx, sc.rx[0], pb)
    assert fa.stats["coherent"] == 1
    assert fa.paths.tobytes() == fb.paths.tobytes()
    a.close()
    b.close()
