"""The per-receiver reduction that allocates no device memory.

Callers that cannot allocate device memory (a framework that owns the whole
pool, a real-time loop that must not call cudaMalloc after start-up) use
dcem_reduce_paths_noalloc with their own input and output buffers. Its
results must equal the per-receiver results of dcem_trace_frame for the same
path records, call after call (the fixed scratch it shares between calls must
not leak state from one call into the next).
"""
import ctypes as C

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


@pytest.mark.parametrize("which", ["toy", "highway"])
def test_noalloc_reduction_matches_trace_frame(cuda, which):
    torch = cuda
    if which == "toy":
        sc, f, n_rays = scenes.toy_street(), 3, 20_000
    else:
        sc, f, n_rays = scenes.highway(n_frames=3, n_vehicles=80, length=800.0), 2, 200_000
    n, paths, field, pc, pi, ptx = _frame_on_device(torch, sc, f, n_rays)
    assert n > 0
    st = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # two calls in a row share the same scratch
        f2 = torch.full_like(field, float("nan"))
        pc2 = torch.full_like(pc, float("nan"))
        pi2 = torch.full_like(pi, float("nan"))
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
