"""Graph replay of a frame's device work (dcem_scene_set_graph_replay).

A frame whose arguments equal those of the frame two calls earlier is
launched as one CUDA graph captured from that call. Replayed frames must give
the same bits as frames launched operation by operation: path records,
per-receiver field and power, the ray log and every counter.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_07115_gb300 import dcem, scenes
from tests import parity as P

pytestmark = pytest.mark.gpu

COUNTERS = ("segments_traced", "segments_reused", "rays_retraced", "candidates", "candidates_reused",
            "unique_candidates", "paths_valid", "objects_moved", "rx_moved", "node_visits", "tri_tests",
            "stack_overflow", "coherent", "kernel_launches", "bvh_rebuilt", "max_segment_nodes",
            "trace_kernel")


@pytest.fixture(scope="module")
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_07115_gb300 import build
    build.build()
    O.build()
    torch.cuda.set_device(0)
    return torch


def _scene(torch, sc, rays, graphs):
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(rays)
    s.set_graph_replay(graphs)
    return s


def _same(fa, fb, a, b, f):
    assert fa.paths.tobytes() == fb.paths.tobytes(), f"frame {f}: path records differ"
    assert np.array_equal(fa.field, fb.field) and np.array_equal(fa.p_coh_dbm, fb.p_coh_dbm)
    assert np.array_equal(fa.p_inc_dbm, fb.p_inc_dbm)
    for k in COUNTERS:
        assert fa.stats[k] == fb.stats[k], (f, k)
    la, lb = a.ray_log(), b.ray_log()
    assert np.array_equal(la[0], lb[0]) and np.array_equal(la[2], lb[2])
    assert np.array_equal(la[1].view(np.uint32), lb[1].view(np.uint32))


@pytest.mark.parametrize("mode", [dcem.MODE_COHERENT, dcem.MODE_FULL])
def test_graph_replay_equals_direct_launches(cuda, mode):
    sc = scenes.highway(n_frames=8, n_vehicles=60, length=600.0)
    rays = scenes.fibonacci_sphere(100_000)
    a, b = _scene(cuda, sc, rays, True), _scene(cuda, sc, rays, False)
    prm = P.gpu_params(sc, mode=mode)
    replayed = []
    for f in range(sc.nframes):
        a.update_transforms(sc.xf[f])
        b.update_transforms(sc.xf[f])
        fa = a.trace(sc.tx, sc.rx[f], prm)
        fb = b.trace(sc.tx, sc.rx[f], prm)
        assert fb.stats["graph_replayed"] == 0
        replayed.append(fa.stats["graph_replayed"])
        _same(fa, fb, a, b, f)
    # full: frames 0 and 1 launch directly (one plan per candidate-buffer
    # parity), frame 2 on replays; coherent: frame 0 is a full trace, so the
    # coherent plans repeat from frame 3
    first = 3 if mode == dcem.MODE_COHERENT else 2
    assert replayed == [0] * first + [1] * (sc.nframes - first)
    a.close()
    b.close()


def test_graph_replay_follows_argument_changes(cuda):
    """A new receiver count or a full retrace (forced by a new transmitter
    position or a new capture radius) changes the plan: direct launches, then
    replay once the plan repeats. Transmitter positions and capture radii are
    copied in as data, so the coherent frames after such a change may replay
    an earlier coherent graph. Results stay equal to direct launches
    throughout."""
    sc = scenes.toy_street()
    rays = scenes.fibonacci_sphere(sc.n_rays)
    a, b = _scene(cuda, sc, rays, True), _scene(cuda, sc, rays, False)
    prm = P.gpu_params(sc, mode=dcem.MODE_COHERENT)
    prm2 = P.gpu_params(sc, mode=dcem.MODE_COHERENT, rx_radius_scale=1.5)
    tx2 = sc.tx + np.array([1.0, 0.0, 0.0], np.float32)
    plan = [(sc.tx, prm, sc.nrx)] * 5 + [(tx2, prm, sc.nrx)] * 5 + [(tx2, prm2, sc.nrx)] * 4 + \
           [(tx2, prm2, sc.nrx - 3)] * 4
    replayed = []
    for i, (tx, p, nrx) in enumerate(plan):
        f = i % sc.nframes
        a.update_transforms(sc.xf[f])
        b.update_transforms(sc.xf[f])
        fa = a.trace(tx, sc.rx[f][:nrx], p)
        fb = b.trace(tx, sc.rx[f][:nrx], p)
        replayed.append(fa.stats["graph_replayed"])
        _same(fa, fb, a, b, i)
    # one graph per candidate-buffer parity; a slot replays when its last
    # plan repeats (full and coherent frames differ, and so do receiver counts)
    assert replayed == ([0, 0, 0, 1, 1] + [0, 1, 0, 1, 1] + [0, 1, 0, 1] + [0, 0, 0, 1])
    a.close()
    b.close()


def test_graph_replay_device_outputs_and_stage_times(cuda):
    """Device output buffers reused every frame (as a serving loop does), and
    stage timing under replay: the event records are part of the graph."""
    torch = cuda
    sc = scenes.highway(n_frames=6, n_vehicles=60, length=600.0)
    rays = scenes.fibonacci_sphere(100_000)
    a, b = _scene(torch, sc, rays, True), _scene(torch, sc, rays, False)
    nrx, max_paths = sc.nrx, 1 << 14
    field = torch.empty((nrx, 2), dtype=torch.float64, device="cuda")
    pc = torch.empty(nrx, dtype=torch.float64, device="cuda")
    pi = torch.empty(nrx, dtype=torch.float64, device="cuda")
    paths = torch.empty(max_paths * C.sizeof(dcem.Path), dtype=torch.uint8, device="cuda")
    rx_d = torch.from_numpy(sc.rx).cuda()
    for timing in (1, 2):
        prm = P.gpu_params(sc, mode=dcem.MODE_COHERENT, timing=timing)
        for f in range(sc.nframes):
            res = dcem.Result()
            res.ptr_kind = dcem.PTR_DEVICE
            res.max_paths = max_paths
            res.field, res.p_coh_dbm, res.p_inc_dbm = field.data_ptr(), pc.data_ptr(), pi.data_ptr()
            res.paths = paths.data_ptr()
            a.update_transforms(sc.xf[f])
            rc = dcem.dcem_trace_frame(a.h, sc.tx, rx_d[f], prm, res)
            torch.cuda.synchronize()
            assert rc == dcem.OK
            st = dcem.stats_dict(res.stats)
            b.update_transforms(sc.xf[f])
            fb = b.trace(sc.tx, sc.rx[f], prm)
            n = res.n_paths
            assert n == fb.stats["paths_valid"]
            got = np.frombuffer(paths[:n * C.sizeof(dcem.Path)].cpu().numpy().tobytes(), dcem.PATH_DTYPE)
            assert got.tobytes() == fb.paths.tobytes()
            assert np.array_equal(pc.cpu().numpy(), fb.p_coh_dbm)
            assert np.array_equal(pi.cpu().numpy(), fb.p_inc_dbm)
            fl = field.cpu().numpy()
            assert np.array_equal(fl[:, 0] + 1j * fl[:, 1], fb.field)
            ms = st["ms_stage"]
            if f >= 3:
                assert st["graph_replayed"] == 1
            assert ms["trace"] > 0 and np.isfinite(ms["trace"])
            if timing == 1:
                stages = [ms[k] for k in ("prep", "mark", "trace", "capture", "dedupe", "validate", "reduce")]
                if f >= 1:   # coherent frames: every stage runs a kernel
                    assert all(x > 0 and np.isfinite(x) for x in stages), (f, ms)
                assert ms["total"] >= sum(stages) * 0.999 and ms["total"] > 0
            else:
                assert ms["total"] == 0.0
    a.close()
    b.close()


def test_graph_replay_switch_errors(cuda):
    sc = scenes.toy_street()
    s = dcem.Scene.from_scene(sc)
    for bad in (2, -1):
        assert dcem.lib().dcem_scene_set_graph_replay(s.h, bad) == dcem.ERR_ARG
    s.close()
