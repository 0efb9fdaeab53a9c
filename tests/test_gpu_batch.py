"""Several scenes per frame (dcem_batch_*): each scene's results must equal,
bit for bit, the same frames traced on that scene alone; every scene's rays
are traced by one closest-hit launch, and once every scene's frame plan
repeats the whole frame must run as one graph launch."""
import numpy as np
import pytest

from paper_2112_07115_gb300 import dcem, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_07115_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch


def _workloads():
    """(scene, transmitters, ray sets) of four different scene families."""
    toy = scenes.toy_street()
    hw = scenes.highway(n_frames=6, n_vehicles=60, length=600.0)
    ur = scenes.urban_grid(blocks=2, parcels=2, n_vehicles=12, n_tx=3, budgets=(4_000, 24_000), n_static_rx=4,
                           n_frames=6, max_refl=4)
    tiny = scenes.random_tiny(5, ntri=10, nobj=2, n_frames=6, nrx=3)
    hw_tx = np.stack([hw.tx, hw.tx + np.array([40.0, -10.0, 2.0], np.float32)])
    return [
        (toy, toy.tx[None], [scenes.fibonacci_sphere(10_000)]),
        (hw, hw_tx, [scenes.fibonacci_sphere(60_000), scenes.fibonacci_sphere(25_000)]),
        (ur, ur.meta["tx"], [scenes.fibonacci_sphere(n) for n in ur.meta["budgets"]]),
        (tiny, tiny.tx[None], [scenes.fibonacci_sphere(5_000)]),
    ]


def _make(torch, sc, sets):
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_ray_sets(sets)
    return s


@pytest.mark.parametrize("mode", [dcem.MODE_FULL, dcem.MODE_COHERENT, dcem.MODE_STICKY])
def test_batch_equals_single_scenes(cuda, mode):
    torch = cuda
    wl = _workloads()
    batched = [_make(torch, sc, sets) for sc, _, sets in wl]
    alone = [_make(torch, sc, sets) for sc, _, sets in wl]
    b = dcem.Batch(batched, stream=torch.cuda.current_stream().cuda_stream)
    prm = dcem.default_params(max_refl=3, freq_hz=28e9, mode=mode)
    nf = 6
    replayed = []
    for f in range(nf):
        # device transforms for the batch, host ones for the single scenes
        b.update_transforms([torch.from_numpy(sc.xf[f]).cuda() if sc.nobj else None for sc, _, _ in wl])
        got = b.trace([t for _, t, _ in wl], [sc.rx[f] for sc, _, _ in wl], prm)
        replayed.append(min(g.stats["graph_replayed"] for g in got))
        for (sc, txs, _), s, g in zip(wl, alone, got):
            if sc.nobj:
                s.update_transforms(sc.xf[f])
            ref = s.trace_links(txs, sc.rx[f], prm)
            assert g.paths.tobytes() == ref.paths.tobytes(), (sc.name, f)
            assert np.array_equal(g.field, ref.field) and np.array_equal(g.p_coh_dbm, ref.p_coh_dbm), (sc.name, f)
            assert np.array_equal(g.p_inc_dbm, ref.p_inc_dbm), (sc.name, f)
            # (node visits depend on the traversal kernel: the batch launch
            # walks the binary nodes, a single scene its 4-wide copy)
            for k in ("segments_traced", "segments_reused", "candidates", "unique_candidates", "paths_valid",
                      "coherent", "paths_sticky", "keys_reused"):
                assert g.stats[k] == ref.stats[k], (sc.name, f, k)
            assert g.stats["trace_kernel"] == 3    # every scene's rays in one launch
    # one graph for the whole frame once every scene's plan repeats
    first = 2 if mode == dcem.MODE_FULL else 3
    assert replayed == [0] * first + [1] * (nf - first)
    b.close()
    for s in batched + alone:
        s.close()


def test_batch_ray_logs_and_timing_fallback(cuda):
    """Ray logs equal the single scenes'; with stage timing the scenes run one
    after another (no batch graph) with the same results."""
    torch = cuda
    wl = _workloads()[:2]
    batched = [_make(torch, sc, sets) for sc, _, sets in wl]
    alone = [_make(torch, sc, sets) for sc, _, sets in wl]
    b = dcem.Batch(batched, stream=torch.cuda.current_stream().cuda_stream)
    prm = dcem.default_params(max_refl=3, freq_hz=28e9, mode=dcem.MODE_COHERENT, timing=1)
    for f in range(4):
        b.update_transforms([sc.xf[f] for sc, _, _ in wl])
        got = b.trace([t for _, t, _ in wl], [sc.rx[f] for sc, _, _ in wl], prm)
        for i, ((sc, txs, _), s, g) in enumerate(zip(wl, alone, got)):
            s.update_transforms(sc.xf[f])
            ref = s.trace_links(txs, sc.rx[f], prm)
            assert g.stats["graph_replayed"] == 0
            assert g.paths.tobytes() == ref.paths.tobytes()
            la, lb = batched[i].ray_log(), s.ray_log()
            assert np.array_equal(la[0], lb[0]) and np.array_equal(la[2], lb[2])
            assert np.array_equal(la[1].view(np.uint32), lb[1].view(np.uint32))
    b.close()
    for s in batched + alone:
        s.close()


def test_batch_errors(cuda):
    torch = cuda
    wl = _workloads()[:2]
    sa = [_make(torch, sc, sets) for sc, _, sets in wl]
    with pytest.raises(dcem.DcemError):
        dcem.Batch([sa[0], sa[0]])
    b = dcem.Batch(sa, stream=torch.cuda.current_stream().cuda_stream)
    prm = dcem.default_params(max_refl=3, freq_hz=28e9)
    bad = wl[1][0].xf[0].copy()
    bad[0, 3] = np.nan
    with pytest.raises(dcem.DcemError):
        b.update_transforms([wl[0][0].xf[0], bad])
    # the second scene has two ray sets: one transmitter is a state error
    res = [dcem.Result() for _ in sa]
    for r in res:
        r.ptr_kind = dcem.PTR_HOST
    rc, failed = b.trace_raw([wl[0][1], wl[1][1][:1]], [wl[0][0].rx[0], wl[1][0].rx[0]], prm, res)
    assert rc == dcem.ERR_STATE and failed == 1
    b.close()
    for s in sa:
        s.close()
