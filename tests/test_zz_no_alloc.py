"""The per-receiver reduction that allocates no device memory.

Callers that cannot allocate device memory (a framework that owns the whole
pool, a real-time loop that must not call cudaMalloc after start-up) use
dcem_reduce_paths_noalloc with their own input and output buffers. Its
results must equal the per-receiver results of dcem_trace_frame for the same
path records, call after call (the fixed scratch it shares between calls must
not leak state from one call into the next), and the FP64 oracle's sums of
the same amplitudes. After the one set-up call per device, calls must not
change the device's free memory. Errors the device finds (a receiver index
out of range, too many paths on one receiver) must be reported, and must not
spoil the next call.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_07115_gb300 import dcem, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_07115_gb300 import build
    build.build()
    O.build()
    torch.cuda.set_device(0)
    st = torch.cuda.current_stream().cuda_stream
    # the set-up call: loads the kernels and reserves the scratch on this device
    assert dcem.dcem_reduce_paths_noalloc(None, 0, 0, 5.0, None, None, None, st) == dcem.OK
    return torch


def _frame_on_device(torch, sc, f, n_rays):
    """One frame through dcem_trace_frame with device outputs."""
    st = torch.cuda.current_stream()
    s = dcem.Scene.from_scene(sc, stream=st.cuda_stream)
    s.set_rays(scenes.fibonacci_sphere(n_rays))
    s.update_transforms(sc.xf[f])
    nrx = sc.nrx
    max_paths = 1 << 14
    dev = torch.device("cuda", 0)
    field = torch.empty((nrx, 2), dtype=torch.float64, device=dev)
    pc = torch.empty(nrx, dtype=torch.float64, device=dev)
    pi = torch.empty(nrx, dtype=torch.float64, device=dev)
    paths = torch.empty(max_paths * C.sizeof(dcem.Path), dtype=torch.uint8, device=dev)
    res = dcem.Result()
    res.ptr_kind = dcem.PTR_DEVICE
    res.max_paths = max_paths
    res.field, res.p_coh_dbm, res.p_inc_dbm, res.paths = (field.data_ptr(), pc.data_ptr(), pi.data_ptr(),
                                                          paths.data_ptr())
    prm = dcem.default_params(max_refl=sc.max_refl, freq_hz=sc.freq_hz)
    rx = torch.from_numpy(sc.rx[f]).to(dev)
    assert dcem.dcem_trace_frame(s.h, sc.tx, rx, prm, res) == dcem.OK
    n = res.n_paths
    s.close()
    return n, paths, field, pc, pi, prm.tx_power_w


def _records(paths, n):
    return np.frombuffer(paths[: n * C.sizeof(dcem.Path)].cpu().numpy().tobytes(), dtype=dcem.PATH_DTYPE)


def _oracle_sums(rec, nrx, ptx, max_refl):
    """The oracle's reduction of the same amplitudes, keys in lexicographic order."""
    keys = np.zeros((len(rec), 2 + max_refl), np.int32)
    keys[:, 0] = rec["rx"]
    keys[:, 1] = rec["depth"]
    keys[:, 2:] = np.where(np.arange(max_refl)[None, :] < rec["depth"][:, None], rec["tri"][:, :max_refl], -1)
    order = np.lexsort(keys.T[::-1])
    p = np.zeros(len(rec), O.PATH_DTYPE)
    p["valid"] = 1
    p["amp_re"] = rec["amp_re"]
    p["amp_im"] = rec["amp_im"]
    return O.reduce(keys[order], p[order], nrx, ptx)


@pytest.mark.parametrize("which", ["toy", "highway"])
def test_noalloc_reduction_matches_trace_frame(cuda, which):
    torch = cuda
    if which == "toy":
        sc, f, n_rays = scenes.toy_street(), 3, 20_000
    else:
        sc, f, n_rays = scenes.highway(n_frames=3, n_vehicles=80, length=800.0), 2, 200_000
    n, paths, field, pc, pi, ptx = _frame_on_device(torch, sc, f, n_rays)
    assert n > 0
    rec = _records(paths, n)
    ofield, opc, opi = _oracle_sums(rec, sc.nrx, ptx, sc.max_refl)
    absum = np.zeros(sc.nrx)
    np.add.at(absum, rec["rx"], np.hypot(rec["amp_re"], rec["amp_im"]))
    st = torch.cuda.current_stream().cuda_stream
    f2 = torch.empty_like(field)
    pc2 = torch.empty_like(pc)
    pi2 = torch.empty_like(pi)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):  # two calls in a row share the same scratch
        for t in (f2, pc2, pi2):
            t.fill_(float("nan"))
        rc = dcem.dcem_reduce_paths_noalloc(paths.data_ptr(), n, sc.nrx, ptx, f2.data_ptr(), pc2.data_ptr(),
                                            pi2.data_ptr(), st)
        assert rc == dcem.OK, dcem.status_string(rc)
        a, b = pc.cpu().numpy(), pc2.cpu().numpy()
        fin = np.isfinite(a)
        assert np.array_equal(np.isfinite(b), fin)
        assert np.max(np.abs(a[fin] - b[fin]), initial=0.0) <= 0.01          # dB, the parity tolerance
        assert np.array_equal(a, b)                                           # same order: same bits
        assert np.array_equal(pi.cpu().numpy(), pi2.cpu().numpy())
        assert np.array_equal(field.cpu().numpy(), f2.cpu().numpy())
        # against the oracle's FP64 sums of the same amplitudes
        got = f2.cpu().numpy()
        gz = got[:, 0] + 1j * got[:, 1]
        # sums in another order: rounding of order 1e-16 times sum |a| per term
        assert np.all(np.abs(gz - ofield) <= 1e-13 * absum + 1e-300)
        fo = np.isfinite(opc)
        assert np.array_equal(np.isfinite(b), fo)
        assert np.max(np.abs(b[fo] - opc[fo]), initial=0.0) <= 1e-6
        assert np.max(np.abs(pi2.cpu().numpy()[fo] - opi[fo]), initial=0.0) <= 1e-9
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0    # no device memory taken by the calls


def _crafted(torch, nrec, rx_of, nrx_amp=1.0):
    """nrec device path records: rx_of(i), distinct keys, amplitudes 1e-6 * (i + 1)."""
    rec = np.zeros(nrec, dcem.PATH_DTYPE)
    rec["rx"] = [rx_of(i) for i in range(nrec)]
    rec["depth"] = 1
    rec["tri"][:, 0] = np.arange(nrec)
    rec["key"] = np.arange(1, nrec + 1, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15 & 0xFFFFFFFF)
    rec["amp_re"] = 1e-6 * nrx_amp * (np.arange(nrec) + 1)
    rec["amp_im"] = -0.5e-6 * (np.arange(nrec) + 1)
    buf = torch.from_numpy(np.frombuffer(rec.tobytes(), np.uint8).copy()).to("cuda")
    return rec, buf


def test_noalloc_device_errors_then_a_good_call(cuda):
    torch = cuda
    st = torch.cuda.current_stream().cuda_stream
    dev = torch.device("cuda", 0)
    nrx = 4
    good, gbuf = _crafted(torch, 64, lambda i: i % nrx)
    pc = torch.empty(nrx, dtype=torch.float64, device=dev)
    fld = torch.empty((nrx, 2), dtype=torch.float64, device=dev)

    def run_good():
        pc.fill_(float("nan"))
        fld.fill_(float("nan"))
        rc = dcem.dcem_reduce_paths_noalloc(gbuf.data_ptr(), len(good), nrx, 5.0, fld.data_ptr(), pc.data_ptr(),
                                            None, st)
        assert rc == dcem.OK, dcem.status_string(rc)
        return fld.cpu().numpy().copy(), pc.cpu().numpy().copy()

    ref_f, ref_p = run_good()
    ofield, opc, _ = _oracle_sums(good, nrx, 5.0, dcem.MAX_REFL)
    assert np.allclose(ref_f[:, 0] + 1j * ref_f[:, 1], ofield, rtol=1e-12)
    assert np.max(np.abs(ref_p - opc)) <= 1e-6
    # a record whose receiver lies outside [0, nrx): found on the device
    bad, bbuf = _crafted(torch, 16, lambda i: nrx if i == 7 else i % nrx)
    assert dcem.dcem_reduce_paths_noalloc(bbuf.data_ptr(), len(bad), nrx, 5.0, None, None, None,
                                          st) == dcem.ERR_ARG
    f1, p1 = run_good()
    assert np.array_equal(f1, ref_f) and np.array_equal(p1, ref_p)
    # 4097 records on one receiver: above the per-receiver limit
    big, bigbuf = _crafted(torch, 4097, lambda i: 1)
    assert dcem.dcem_reduce_paths_noalloc(bigbuf.data_ptr(), len(big), nrx, 5.0, None, pc.data_ptr(), None,
                                          st) == dcem.ERR_CAPACITY
    f2, p2 = run_good()
    assert np.array_equal(f2, ref_f) and np.array_equal(p2, ref_p)
    # records but no receivers
    assert dcem.dcem_reduce_paths_noalloc(gbuf.data_ptr(), len(good), 0, 5.0, None, None, None,
                                          st) == dcem.ERR_ARG


def test_noalloc_equal_keys_sum_in_record_order(cuda):
    """Records with equal keys (one sequence from two transmitters) are summed
    in record-index order: the same bits on every call."""
    torch = cuda
    st = torch.cuda.current_stream().cuda_stream
    nrx = 2
    rec = np.zeros(600, dcem.PATH_DTYPE)
    rec["rx"] = np.arange(600) % nrx
    rec["depth"] = 1
    rec["key"] = np.uint64(12345) + (np.arange(600) % 7).astype(np.uint64)   # many equal keys
    rng = np.random.default_rng(3)
    rec["amp_re"] = rng.standard_normal(600) * 10.0 ** rng.uniform(-9, -3, 600)
    rec["amp_im"] = rng.standard_normal(600) * 10.0 ** rng.uniform(-9, -3, 600)
    buf = torch.from_numpy(np.frombuffer(rec.tobytes(), np.uint8).copy()).to("cuda")
    fld = torch.empty((nrx, 2), dtype=torch.float64, device="cuda")
    outs = []
    for _ in range(4):
        fld.fill_(float("nan"))
        assert dcem.dcem_reduce_paths_noalloc(buf.data_ptr(), len(rec), nrx, 5.0, fld.data_ptr(), None, None,
                                              st) == dcem.OK
        outs.append(fld.cpu().numpy().copy())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_noalloc_rejects_sizes_beyond_the_maximum(cuda):
    torch = cuda
    dev = torch.device("cuda", 0)
    buf = torch.zeros(8 * C.sizeof(dcem.Path), dtype=torch.uint8, device=dev)
    out = torch.zeros(8, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream().cuda_stream
    assert dcem.dcem_reduce_paths_noalloc(buf.data_ptr(), 1 << 20, 4, 5.0, None, out.data_ptr(), None,
                                          st) == dcem.ERR_CAPACITY
    assert dcem.dcem_reduce_paths_noalloc(buf.data_ptr(), 0, 100_000, 5.0, None, None, None,
                                          st) == dcem.ERR_CAPACITY
    assert dcem.dcem_reduce_paths_noalloc(None, 4, 4, 5.0, None, None, None, st) == dcem.ERR_ARG
