"""Field derivatives over a fixed path topology (dcem_path_gradients) against
the FP64 oracle's central differences.

The oracle finds the frame's valid paths itself (its own trace, dedupe and
validation) and differentiates their field by central differences; the GPU
gets the same triangle sequences and returns forward-mode derivatives. The
field E agrees to 1e-9 relative (both FP64), dE/dtheta to 1e-5 of the
receiver's largest derivative (the differences are accurate to ~1e-7), and
d P_coh[dBm]/dtheta likewise.
"""
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
    return torch


def _paths_of(keys, max_refl):
    p = np.zeros(keys.shape[0], dcem.PATH_DTYPE)
    p["rx"] = keys[:, 0]
    p["depth"] = keys[:, 1]
    for j in range(max_refl):
        p["tri"][:, j] = np.where(j < keys[:, 1], keys[:, 2 + j], -1)
    return p


def _oracle_paths(sc, f, prm, rays):
    fr = O.frame(sc, f, rays, prm)
    return fr.world_tris, fr.keys[fr.paths["valid"] != 0]


def _compare(cuda, sc, f, prm, rays, min_paths=3):
    wt, keys = _oracle_paths(sc, f, prm, rays)
    assert keys.shape[0] >= min_paths
    rx = sc.rx[f]
    e_or, de_or, ok = O.field_gradient(wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, rx, keys, prm,
                                       nobj=sc.nobj)
    keys = keys[ok]
    s = dcem.Scene.from_scene(sc, stream=cuda.cuda.current_stream().cuda_stream)
    s.update_transforms(sc.xf[f])
    assert np.array_equal(s.world_tris(), O.transform(sc.tris, sc.tri_obj, sc.xf[f]))
    prm_g = dcem.default_params(max_refl=prm.max_refl, freq_hz=prm.freq_hz)
    e, de, dp = s.gradients(sc.tx, rx, _paths_of(keys, prm.max_refl), prm_g)
    s.close()
    npar = 2 * sc.materials.shape[0] + 2 * sc.nobj
    assert de.shape == (rx.shape[0], npar)
    for r in range(rx.shape[0]):
        if not (keys[:, 0] == r).any():
            assert e[r] == 0 and not de[r].any() and not dp[r].any()
            continue
        assert abs(e[r] - e_or[r]) <= 1e-9 * abs(e_or[r]) + 1e-18, r
        scale = np.abs(de_or[r]).max()
        assert np.abs(de[r] - de_or[r]).max() <= 1e-5 * scale + 1e-15, (r, de[r], de_or[r])
        dp_or = O.pcoh_dbm_gradient(e_or[r:r + 1], de_or[r:r + 1], prm.tx_power_w)[0]
        assert np.abs(dp[r] - dp_or).max() <= 1e-5 * np.abs(dp_or).max() + 1e-9, r
    return keys, de


@pytest.mark.parametrize("f", [1, 8])
def test_gradients_toy_street(cuda, f):
    """Moving perfectly conducting vehicles (translation derivatives; frame 8
    has a path off a vehicle) and concrete ground and walls (permittivity and
    conductivity derivatives)."""
    sc = scenes.toy_street()
    prm = O.OracleParams(freq_hz=28e9, n_rays=10_000, max_refl=3)
    keys, de = _compare(cuda, sc, f, prm, scenes.fibonacci_sphere(10_000))
    nm = sc.materials.shape[0]
    # the vehicles are metal: no derivative along the metal's parameters
    assert not de[:, 2:4].any()
    veh = [any(sc.tri_obj[i] >= 0 for i in row[2:2 + row[1]]) for row in keys]
    assert (np.abs(de[:, 2 * nm:]).max() > 0) == any(veh)
    if f == 8:
        assert any(veh)


@pytest.mark.parametrize("seed", [16, 37])
def test_gradients_random_tiny_three_materials(cuda, seed):
    """Moving concrete and metal objects, and a third (glass-like) material on
    half of the static triangles; 2 reflections."""
    sc = scenes.random_tiny(seed, ntri=10, nobj=2, n_frames=3, nrx=3)
    sc.materials = np.vstack([sc.materials, np.array([[6.27, 0.3, 0.0]], np.float32)])
    tm = sc.tri_mat.copy()
    stat = np.flatnonzero(sc.tri_obj < 0)
    tm[stat[2::2]] = 2
    sc.tri_mat = tm
    prm = O.OracleParams(freq_hz=5.9e9, n_rays=20_000, max_refl=2)
    keys, de = _compare(cuda, sc, 1, prm, scenes.fibonacci_sphere(20_000), min_paths=4)
    # paths off a moving object and off the third material give non-zero derivatives
    assert np.abs(de[:, 6:]).max() > 0 and np.abs(de[:, 4:6]).max() > 0


def test_gradients_repeatable_and_device_outputs(cuda):
    """Two calls give identical bits; device outputs equal host outputs."""
    torch = cuda
    sc = scenes.toy_street()
    prm = O.OracleParams(freq_hz=28e9, n_rays=10_000, max_refl=3)
    _, keys = _oracle_paths(sc, 2, prm, scenes.fibonacci_sphere(10_000))
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.update_transforms(sc.xf[2])
    prm_g = dcem.default_params(max_refl=3, freq_hz=28e9)
    paths = _paths_of(keys, 3)
    e1, de1, dp1 = s.gradients(sc.tx, sc.rx[2], paths, prm_g)
    e2, de2, dp2 = s.gradients(sc.tx, sc.rx[2], paths, prm_g)
    assert np.array_equal(de1, de2) and np.array_equal(dp1, dp2) and np.array_equal(e1, e2)
    nrx, npar = sc.nrx, dcem.dcem_scene_gradient_size(s.h)
    pd = torch.from_numpy(paths.view(np.uint8)).cuda()
    rxd = torch.from_numpy(sc.rx[2]).cuda()
    fd = torch.zeros((nrx, 2), dtype=torch.float64, device="cuda")
    dfd = torch.zeros((nrx, npar, 2), dtype=torch.float64, device="cuda")
    dpd = torch.zeros((nrx, npar), dtype=torch.float64, device="cuda")
    rc = dcem.dcem_path_gradients(s.h, sc.tx, rxd, pd.data_ptr(), prm_g, dcem.PTR_DEVICE, fd.data_ptr(),
                                  dfd.data_ptr(), dpd.data_ptr(), n_paths=paths.shape[0])
    torch.cuda.synchronize()
    assert rc == dcem.OK
    assert np.array_equal(dfd.cpu().numpy()[..., 0] + 1j * dfd.cpu().numpy()[..., 1], de1)
    assert np.array_equal(dpd.cpu().numpy(), dp1)
    s.close()


def test_gradients_errors(cuda):
    """Paths not grouped by receiver, a depth above max_refl and a triangle id
    out of range are argument errors."""
    sc = scenes.toy_street()
    s = dcem.Scene.from_scene(sc)
    prm_g = dcem.default_params(max_refl=2)
    p = np.zeros(2, dcem.PATH_DTYPE)
    p["rx"] = [1, 0]
    p["tri"] = -1
    npar = dcem.dcem_scene_gradient_size(s.h)
    fld = np.zeros(2 * sc.nrx)
    dfl = np.zeros(2 * sc.nrx * npar)
    for bad in ("order", "depth", "tri"):
        q = p.copy()
        if bad == "depth":
            q["rx"] = [0, 1]
            q["depth"][0] = 3
        if bad == "tri":
            q["rx"] = [0, 1]
            q["depth"][0] = 1
            q["tri"][0, 0] = sc.ntri
        rc = dcem.dcem_path_gradients(s.h, sc.tx, sc.rx[0], q, prm_g, dcem.PTR_HOST, fld.ctypes.data,
                                      dfl.ctypes.data, None)
        assert rc == dcem.ERR_ARG, bad
    s.close()


def test_path_power_autograd(cuda):
    """The received power as a torch autograd function of the scene's
    parameters: forward equals the frame's P_coh, and a weighted loss's
    gradient equals the Jacobian of dcem_path_gradients contracted with the
    weights."""
    torch = cuda
    sc = scenes.toy_street()
    f = 8
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(scenes.fibonacci_sphere(10_000))
    s.update_transforms(sc.xf[f])
    prm = dcem.default_params(max_refl=3, freq_hz=28e9)
    fr = s.trace(sc.tx, sc.rx[f], prm)
    assert fr.paths.shape[0] > 0
    # theta: eps_r, sigma per material, then the x, y translation per object
    xf = sc.xf[f].reshape(sc.nobj, 12)
    th0 = np.concatenate([sc.materials[:, :2].astype(np.float64).ravel(),
                          np.stack([xf[:, 3], xf[:, 7]], 1).astype(np.float64).ravel()])
    theta = torch.tensor(th0, dtype=torch.float64, device="cuda", requires_grad=True)
    p = dcem.path_power(s, theta, sc.tx, sc.rx[f], fr.paths, prm)
    pc = p.detach().cpu().numpy()
    fin = np.isfinite(fr.p_coh_dbm)
    assert np.array_equal(np.isfinite(pc), fin) and fin.any()
    assert np.abs(pc[fin] - fr.p_coh_dbm[fin]).max() <= 1e-9
    w = torch.from_numpy(np.random.default_rng(3).normal(size=sc.nrx)).cuda()
    m = torch.from_numpy(fin).cuda()
    loss = (w * torch.where(m, p, torch.zeros_like(p))).sum()
    loss.backward()
    _, _, dp = s.gradients(sc.tx, sc.rx[f], fr.paths, prm)
    want = (w.cpu().numpy()[fin, None] * dp[fin]).sum(0)
    got = theta.grad.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max())
    assert np.abs(want).max() > 0
    s.close()
