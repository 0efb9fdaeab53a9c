"""The reverse-mode (adjoint) field derivatives (dcem_path_adjoint) and the
received power as a differentiable function of theta (dcem.path_power).

The oracle finds a frame's valid paths itself and differentiates their field
by FP64 central differences at the same parameters; the GPU gets the same
triangle sequences. Per element, a derivative must agree with the oracle's to
1e-4 relative, with an absolute floor of 1e-9 of the receiver's largest
derivative for elements that cancel below the differences' own accuracy
(about 1e-7 relative: steps of 1e-6 m and 1e-6 relative). The adjoint equals
the forward-mode kernel (dcem_path_gradients) to 1e-8 of the receiver's
largest derivative, both being FP64 analytic derivatives of the same
amplitude evaluated in different operation orders.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_07115_gb300 import dcem, scenes

pytestmark = pytest.mark.gpu

RTOL, FLOOR = 1e-4, 1e-9


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


def _theta_inputs(sc, f, wt, dmat=None, dpos=None):
    """theta (GPU layout: materials, then absolute x, y per object) and the
    oracle's FP64 inputs at theta: materials and world triangles."""
    mats = sc.materials.astype(np.float64).copy()
    xf = sc.xf[f].reshape(sc.nobj, 12) if sc.nobj else np.zeros((0, 12), np.float32)
    wt64 = np.asarray(wt, np.float64).reshape(-1, 3, 3).copy()
    if dmat is not None:
        mats[:, :2] *= dmat
    th_obj = np.stack([xf[:, 3], xf[:, 7]], 1).astype(np.float64) if sc.nobj else np.zeros((0, 2))
    if dpos is not None:
        th_obj = th_obj + dpos
        for o in range(sc.nobj):
            sel = sc.tri_obj == o
            wt64[sel, :, 0] += th_obj[o, 0] - np.float64(xf[o, 3])
            wt64[sel, :, 1] += th_obj[o, 1] - np.float64(xf[o, 7])
    theta = np.concatenate([mats[:, :2].ravel(), th_obj.ravel()])
    return theta, mats, wt64


def _check_elementwise(got, ref, what):
    for r in range(ref.shape[0]):
        scale = np.abs(ref[r]).max()
        if scale == 0.0:
            assert not np.any(got[r]), (what, r)
            continue
        err = np.abs(got[r] - ref[r])
        bad = err > RTOL * np.abs(ref[r]) + FLOOR * scale
        assert not bad.any(), (what, r, np.flatnonzero(bad), got[r][bad], ref[r][bad])


def _compare(cuda, sc, f, n_rays, dmat=None, dpos=None, min_paths=3, check_forward=True):
    prm = O.OracleParams(freq_hz=sc.freq_hz, n_rays=n_rays, max_refl=sc.max_refl)
    fr = O.frame(sc, f, scenes.fibonacci_sphere(n_rays), prm)
    keys = fr.keys[fr.paths["valid"] != 0]
    assert keys.shape[0] >= min_paths
    theta, mats, wt64 = _theta_inputs(sc, f, fr.world_tris, dmat, dpos)
    rx = sc.rx[f]
    e_or, de_or, ok = O.field_gradient(wt64, sc.tri_mat, sc.tri_obj, mats, sc.tx, rx, keys, prm, nobj=sc.nobj)
    keys = keys[ok]
    assert keys.shape[0] >= min_paths
    s = dcem.Scene.from_scene(sc, stream=cuda.cuda.current_stream().cuda_stream)
    s.update_transforms(sc.xf[f])
    prm_g = dcem.default_params(max_refl=sc.max_refl, freq_hz=sc.freq_hz)
    paths = _paths_of(keys, sc.max_refl)
    e, pc, de, dp, _ = s.adjoint(sc.tx, rx, paths, prm_g, theta=theta)
    if check_forward and dmat is None and dpos is None:
        e_f, de_f, dp_f = s.gradients(sc.tx, rx, paths, prm_g)
        for r in range(rx.shape[0]):
            sc_r = np.abs(de_f[r]).max()
            # two FP64 evaluations in different operation orders: the phase k L
            # carries their rounding (k dL ~ 1e-10 for dL ~ 1e-13 m)
            assert abs(e[r] - e_f[r]) <= 1e-9 * abs(e_f[r]) + 1e-300
            assert np.abs(de[r] - de_f[r]).max() <= 1e-8 * sc_r + 1e-300, r
    s.close()
    npar = 2 * sc.materials.shape[0] + 2 * sc.nobj
    assert de.shape == (rx.shape[0], npar)
    for r in range(rx.shape[0]):
        assert abs(e[r] - e_or[r]) <= 1e-9 * abs(e_or[r]) + 1e-300, r
    _check_elementwise(de, de_or, "dE")
    dp_or = O.pcoh_dbm_gradient(e_or, de_or, prm.tx_power_w)
    _check_elementwise(dp, dp_or, "dP")
    # P_coh at theta against the oracle's sum of the same amplitudes
    with np.errstate(divide="ignore"):
        pc_or = 10 * np.log10(prm.tx_power_w * np.abs(e_or) ** 2) + 30
    fin = np.isfinite(pc_or)
    assert np.array_equal(np.isfinite(pc), fin)
    assert np.abs(pc[fin] - pc_or[fin]).max(initial=0.0) <= 1e-9
    return keys, de


@pytest.mark.parametrize("f", [1, 8])
def test_adjoint_toy_street(cuda, f):
    sc = scenes.toy_street()
    keys, de = _compare(cuda, sc, f, 10_000)
    nm = sc.materials.shape[0]
    assert not de[:, 2:4].any()                      # metal: no material derivative
    if f == 8:
        assert np.abs(de[:, 2 * nm:]).max() > 0      # a path off a moving vehicle


def test_adjoint_at_other_parameters(cuda):
    """theta away from the scene's values: materials scaled, vehicles moved by
    decimetres (paths whose geometry stays valid)."""
    sc = scenes.toy_street()
    rng = np.random.default_rng(5)
    dmat = rng.uniform(0.7, 1.6, size=(sc.materials.shape[0], 2))
    dpos = rng.uniform(-0.3, 0.3, size=(sc.nobj, 2))
    _compare(cuda, sc, 8, 10_000, dmat=dmat, dpos=dpos)


@pytest.mark.parametrize("seed", [16, 37])
def test_adjoint_random_three_materials(cuda, seed):
    sc = scenes.random_tiny(seed, ntri=10, nobj=2, n_frames=3, nrx=3)
    sc.materials = np.vstack([sc.materials, np.array([[6.27, 0.3, 0.0]], np.float32)])
    tm = sc.tri_mat.copy()
    stat = np.flatnonzero(sc.tri_obj < 0)
    tm[stat[2::2]] = 2
    sc.tri_mat = tm
    sc.freq_hz = 5.9e9
    sc.max_refl = 2
    _, de = _compare(cuda, sc, 1, 20_000, min_paths=4)
    assert np.abs(de[:, 6:]).max() > 0 and np.abs(de[:, 4:6]).max() > 0


def test_adjoint_urban_eight_materials(cuda):
    """The differentiable urban workload, reduced: eight (eps_r, sigma)
    classes, 80 moving metal vehicles, 48 roadside receivers."""
    sc = scenes.urban_gradient(blocks=3, parcels=2, n_vehicles=80, n_rx=48, n_rays=300_000, max_refl=3)
    keys, de = _compare(cuda, sc, 1, sc.n_rays, min_paths=20)
    nm = sc.materials.shape[0]
    assert nm == 9 and np.count_nonzero(np.abs(de[:, :16]).max(0)) >= 8   # several material classes
    assert np.abs(de[:, 2 * nm:]).max() > 0                                # vehicle translations


def test_path_power_is_a_function_of_theta(cuda):
    """path_power(theta): the forward pass follows theta (against the oracle
    at another theta), its gradient is the adjoint's vector-Jacobian product
    and matches central differences of path_power itself."""
    torch = cuda
    sc = scenes.toy_street()
    f = 8
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(scenes.fibonacci_sphere(10_000))
    s.update_transforms(sc.xf[f])
    prm = dcem.default_params(max_refl=3, freq_hz=28e9)
    fr = s.trace(sc.tx, sc.rx[f], prm)
    th0 = s.theta(sc.xf[f])
    theta = torch.tensor(th0, dtype=torch.float64, device="cuda", requires_grad=True)
    p0 = dcem.path_power(s, theta, sc.tx, sc.rx[f], fr.paths, prm).detach().cpu().numpy()
    fin = np.isfinite(fr.p_coh_dbm)
    assert np.array_equal(np.isfinite(p0), fin) and fin.any()
    assert np.abs(p0[fin] - fr.p_coh_dbm[fin]).max() <= 1e-9           # theta = the scene: the frame's power
    # another theta: materials x1.2, vehicles moved by up to 1 cm; against the oracle's field there
    rng = np.random.default_rng(2)
    dmat = np.full((sc.materials.shape[0], 2), 1.2)
    dpos = rng.uniform(-0.01, 0.01, size=(sc.nobj, 2))
    th1, mats1, wt1 = _theta_inputs(sc, f, O.transform(sc.tris, sc.tri_obj, sc.xf[f]), dmat, dpos)
    keys = np.zeros((fr.paths.shape[0], 2 + 3), np.int32)
    keys[:, 0], keys[:, 1] = fr.paths["rx"], fr.paths["depth"]
    keys[:, 2:] = np.where(np.arange(3)[None] < fr.paths["depth"][:, None], fr.paths["tri"][:, :3], -1)
    oprm = O.OracleParams(freq_hz=28e9, n_rays=10_000, max_refl=3)
    amp = O.path_amp_d(wt1, sc.tri_mat, mats1, sc.tx, sc.rx[f], keys, oprm)
    assert np.all(amp["valid"] != 0)
    e1 = O.field_of(keys, amp, sc.nrx)
    with np.errstate(divide="ignore"):
        p1_or = 10 * np.log10(5.0 * np.abs(e1) ** 2) + 30
    t1 = torch.tensor(th1, dtype=torch.float64, device="cuda", requires_grad=True)
    p1 = dcem.path_power(s, t1, sc.tx, sc.rx[f], fr.paths, prm)
    assert np.abs(p1.detach().cpu().numpy()[fin] - p1_or[fin]).max() <= 1e-9
    assert np.abs(p1.detach().cpu().numpy()[fin] - p0[fin]).max() > 1e-3    # it moved with theta
    # gradient of a weighted loss at theta1: the adjoint's product, and central differences
    w = torch.from_numpy(np.random.default_rng(3).normal(size=sc.nrx)).cuda()
    m = torch.from_numpy(fin).cuda()
    loss = (w * torch.where(m, p1, torch.zeros_like(p1))).sum()
    loss.backward()
    g = t1.grad.cpu().numpy()
    _, _, _, dp, tb = s.adjoint(sc.tx, sc.rx[f], fr.paths, prm, theta=th1,
                                pcoh_bar=np.where(fin, w.cpu().numpy(), 0.0))
    assert np.array_equal(g, tb)
    assert np.abs(g - (w.cpu().numpy()[fin, None] * dp[fin]).sum(0)).max() <= 1e-10 * np.abs(g).max()

    def lossf(th):
        with torch.no_grad():
            p = dcem.path_power(s, torch.tensor(th, dtype=torch.float64, device="cuda"), sc.tx, sc.rx[f],
                                fr.paths, prm)
            return float((w * torch.where(m, p, torch.zeros_like(p))).sum())
    for i in np.flatnonzero(np.abs(g) > 1e-6 * np.abs(g).max()):
        h = 1e-6 * max(1.0, abs(th1[i])) if i < 2 * sc.materials.shape[0] else 1e-6
        tp, tm = th1.copy(), th1.copy()
        tp[i] += h
        tm[i] -= h
        fd = (lossf(tp) - lossf(tm)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-4 * abs(g[i]) + 1e-9 * np.abs(g).max(), (i, fd, g[i])
    s.close()


def test_adjoint_errors_and_empty(cuda):
    sc = scenes.toy_street()
    s = dcem.Scene.from_scene(sc)
    prm = dcem.default_params(max_refl=2)
    p = np.zeros(1, dcem.PATH_DTYPE)
    p["tri"] = -1
    np_ = dcem.dcem_scene_gradient_size(s.h)
    th = s.theta(sc.xf[0])
    th_bad = th.copy()
    th_bad[0] = np.nan
    out = np.zeros(np_)
    pb = np.zeros(sc.nrx)
    assert dcem.dcem_path_adjoint(s.h, sc.tx, sc.rx[0], p, prm, dcem.PTR_HOST, th_bad.ctypes.data) == \
        dcem.ERR_NONFINITE
    assert dcem.dcem_path_adjoint(s.h, sc.tx, sc.rx[0], p, prm, dcem.PTR_HOST, th.ctypes.data,
                                  theta_bar_ptr=out.ctypes.data) == dcem.ERR_ARG     # theta_bar without pcoh_bar
    # no paths: zero field and gradient
    e, pc, de, dp, tb = s.adjoint(sc.tx, sc.rx[0], np.zeros(0, dcem.PATH_DTYPE), prm, theta=th, pcoh_bar=pb + 1.0)
    assert not e.any() and not de.any() and not tb.any() and np.all(np.isneginf(pc))
    s.close()
