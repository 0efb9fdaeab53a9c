"""Several transmitters in one frame (dcem_scene_set_ray_sets, dcem_trace_links).

Each transmitter has its own sampled sphere (uneven budgets, so its own
reception-sphere spacing); all of them are traced, captured, deduplicated,
validated and summed in the same launches. Transmitter t's paths and power
must equal, bit for bit, a single-transmitter frame of tx[t] with ray set t
alone (which the parity tests hold to the oracle), and the oracle's own frame
of tx[t] directly.
"""
import copy

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


def _scene(torch, sc):
    return dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)


def _tx_set(sc, k, seed=5):
    """k transmitters: the scene's own and k-1 others spread over the scene
    (heights 2-12 m)."""
    rng = np.random.default_rng(seed)
    lo, hi = sc.tris.reshape(-1, 3).min(axis=0), sc.tris.reshape(-1, 3).max(axis=0)
    out = [np.asarray(sc.tx, np.float32)]
    for _ in range(k - 1):
        x = rng.uniform(lo[0] + 0.2 * (hi[0] - lo[0]), hi[0] - 0.2 * (hi[0] - lo[0]))
        y = rng.uniform(lo[1] + 0.2 * (hi[1] - lo[1]), hi[1] - 0.2 * (hi[1] - lo[1]))
        out.append(np.array([x, y, rng.uniform(2.0, 12.0)], np.float32))
    return np.stack(out).astype(np.float32)


def _per_tx(frame_links, t, nrx, off):
    """Transmitter t's part of a links frame, as a single-transmitter frame
    would report it (tx field dropped, ray index local to the set)."""
    p = frame_links.paths[frame_links.paths["tx"] == t].copy()
    assert np.all(p["rx"] < nrx)
    p["ray"] -= off
    p["tx"] = 0
    return p


def _compare_links_vs_single(torch, sc, txs, sizes, frames, mode=dcem.MODE_FULL, rx=None):
    sets = [scenes.fibonacci_sphere(n) for n in sizes]
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    a = _scene(torch, sc)
    a.set_ray_sets(sets)
    singles = []
    for t in range(len(sizes)):
        b = _scene(torch, sc)
        b.set_rays(sets[t])
        singles.append(b)
    prm = P.gpu_params(sc, mode=mode)
    prm_full = P.gpu_params(sc, mode=dcem.MODE_FULL)
    stats = []
    for f in frames:
        rxf = sc.rx[f] if rx is None else rx
        nrx = rxf.shape[0]
        if sc.nobj:
            a.update_transforms(sc.xf[f])
        fl = a.trace_links(txs, rxf, prm)
        stats.append(fl.stats)
        assert fl.p_coh_dbm.shape == (len(sizes), nrx)
        assert fl.paths.shape[0] == fl.stats["paths_valid"]
        # records ordered by (link, key)
        link = fl.paths["tx"].astype(np.int64) * nrx + fl.paths["rx"]
        assert np.all(np.diff(link) >= 0)
        for t, b in enumerate(singles):
            if sc.nobj:
                b.update_transforms(sc.xf[f])
            fs = b.trace(txs[t], rxf, prm_full)
            got = _per_tx(fl, t, nrx, offs[t])
            assert got.tobytes() == fs.paths.tobytes(), f"frame {f}, tx {t}: path records differ"
            assert np.array_equal(fl.field[t], fs.field), (f, t)
            assert np.array_equal(fl.p_coh_dbm[t], fs.p_coh_dbm) and np.array_equal(fl.p_inc_dbm[t], fs.p_inc_dbm)
    a.close()
    for b in singles:
        b.close()
    return stats


def test_links_equal_single_transmitter_frames_toy(cuda):
    sc = scenes.toy_street()
    txs = _tx_set(sc, 3)
    st = _compare_links_vs_single(cuda, sc, txs, [6_000, 10_000, 3_001], range(0, 10, 3))
    assert all(s["paths_valid"] > 0 for s in st)


def test_links_equal_single_transmitter_frames_highway(cuda):
    sc = scenes.highway(n_frames=4, n_vehicles=60, length=600.0)
    txs = _tx_set(sc, 4, seed=7)
    _compare_links_vs_single(cuda, sc, txs, [120_000, 40_000, 65_536, 20_000], range(4))


def test_links_coherent_equals_full(cuda):
    """Coherent reuse across frames with four transmitters equals full
    retraces of every transmitter's set."""
    sc = scenes.highway(n_frames=5, n_vehicles=60, length=600.0)
    txs = _tx_set(sc, 4, seed=11)
    st = _compare_links_vs_single(cuda, sc, txs, [60_000, 25_000, 90_000, 10_000], range(5),
                                  mode=dcem.MODE_COHERENT)
    assert [s["coherent"] for s in st] == [0, 1, 1, 1, 1]
    assert sum(s["segments_reused"] for s in st) > 0


def test_links_many_links_scanned_offsets(cuda):
    """More links than the per-link offset loop serves (8 x 640 = 5120): the
    scanned output offsets give the same records and sums."""
    sc = scenes.toy_street()
    g = np.stack(np.meshgrid(np.linspace(-40, 40, 32), np.linspace(-9, 9, 20), indexing="ij"), -1).reshape(-1, 2)
    rx = np.concatenate([g, np.full((g.shape[0], 1), 1.5)], 1).astype(np.float32)
    assert rx.shape[0] == 640
    txs = _tx_set(sc, 8, seed=3)
    st = _compare_links_vs_single(cuda, sc, txs, [4_000 + 500 * t for t in range(8)], [2], rx=rx)
    assert st[0]["paths_valid"] > 100


def test_links_vs_oracle(cuda):
    """Each transmitter's paths against the oracle's own frame of that
    transmitter and ray set (hits, captures, validity, length, amplitude)."""
    sc = scenes.toy_street()
    txs = _tx_set(sc, 3, seed=2)
    sizes = [5_000, 12_000, 8_000]
    sets = [scenes.fibonacci_sphere(n) for n in sizes]
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    a = _scene(cuda, sc)
    a.set_ray_sets(sets)
    prm = P.gpu_params(sc)
    for f in (1, 8):
        a.update_transforms(sc.xf[f])
        fl = a.trace_links(txs, sc.rx[f], prm)
        ids, tt, ns = a.ray_log()
        for t in range(3):
            sct = copy.copy(sc)
            sct.tx = txs[t]
            ref = O.frame(sct, f, sets[t], P.oracle_params(sc, n_rays=sizes[t]))
            sl = slice(offs[t], offs[t] + sizes[t])
            n_cmp, n_flag, bad = P.compare_hits(ids[sl], ns[sl], ref.tr)
            assert len(bad) == 0, (f, t, bad[:5])
            got = copy.copy(fl)
            got.paths = _per_tx(fl, t, sc.nrx, offs[t])
            res = P.compare_paths(got, ref, sc.max_refl)
            assert res["checked"] > 0
            assert not res["missing"] and not res["extra"], (f, t, res["missing"][:3], res["extra"][:3])
            assert not res["len"] and not res["amp"], (f, t)
    a.close()


def test_links_errors(cuda):
    sc = scenes.toy_street()
    s = _scene(cuda, sc)
    d = scenes.fibonacci_sphere(100)
    # an empty set among several, and no sets
    with pytest.raises(dcem.DcemError):
        s.set_ray_sets([d, d[:0]])
    with pytest.raises(dcem.DcemError):
        s.set_ray_sets([])
    s.set_ray_sets([d, d, d])
    prm = P.gpu_params(sc)
    # the single-transmitter call needs one set; the links call needs one tx per set
    r = s.trace(sc.tx, sc.rx[0], prm, raise_on_error=False)
    assert r.status == dcem.ERR_STATE
    r = s.trace_links(np.stack([sc.tx, sc.tx]), sc.rx[0], prm, raise_on_error=False)
    assert r.status == dcem.ERR_STATE
    bad = np.stack([sc.tx, sc.tx, sc.tx]).copy()
    bad[1, 2] = np.nan
    r = s.trace_links(bad, sc.rx[0], prm, raise_on_error=False)
    assert r.status == dcem.ERR_NONFINITE
    r = s.trace_links(np.stack([sc.tx, sc.tx, sc.tx]), sc.rx[0], prm)
    assert r.status == dcem.OK and set(np.unique(r.paths["tx"])) <= {0, 1, 2}
    # three identical transmitters with identical sets: identical links
    assert np.array_equal(r.p_coh_dbm[0], r.p_coh_dbm[1]) and np.array_equal(r.p_coh_dbm[0], r.p_coh_dbm[2])
    s.close()


def test_urban_grid_reduced_links(cuda):
    """The batched workload's scene family, reduced to 2 x 2 blocks, 12
    vehicles and 3 transmitters with uneven budgets, 5 reflections: each
    transmitter bit for bit as its own frame, and against the oracle."""
    sc = scenes.urban_grid(blocks=2, parcels=2, n_vehicles=12, n_tx=3, budgets=(4_000, 24_000),
                           n_static_rx=4, n_frames=3, max_refl=5)
    txs = sc.meta["tx"]
    sizes = sc.meta["budgets"]
    st = _compare_links_vs_single(cuda, sc, txs, sizes, range(3), mode=dcem.MODE_COHERENT)
    assert st[-1]["paths_valid"] > 0
    sets = [scenes.fibonacci_sphere(n) for n in sizes]
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    a = _scene(cuda, sc)
    a.set_ray_sets(sets)
    f = 2
    a.update_transforms(sc.xf[f])
    fl = a.trace_links(txs, sc.rx[f], P.gpu_params(sc))
    ids, tt, ns = a.ray_log()
    checked = 0
    for t in range(len(sizes)):
        sct = copy.copy(sc)
        sct.tx = txs[t]
        ref = O.frame(sct, f, sets[t], P.oracle_params(sc, n_rays=sizes[t]))
        sl = slice(offs[t], offs[t] + sizes[t])
        _, _, bad = P.compare_hits(ids[sl], ns[sl], ref.tr)
        assert len(bad) == 0, (t, bad[:5])
        got = copy.copy(fl)
        got.paths = _per_tx(fl, t, sc.nrx, offs[t])
        res = P.compare_paths(got, ref, sc.max_refl)
        checked += res["checked"]
        assert not res["missing"] and not res["extra"] and not res["len"] and not res["amp"], t
    assert checked > 0
    a.close()
