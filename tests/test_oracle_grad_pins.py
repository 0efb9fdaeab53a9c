"""Pins of the oracle's field derivatives (central differences over a fixed
path topology, FP64) against closed forms: the two-ray ground model's
derivative with respect to the ground's permittivity and conductivity, and
a moving perfectly conducting wall, whose image geometry gives the path
length's derivative and whose translation along its own plane changes
nothing."""
import numpy as np
import pytest

from paper_2112_07115_gb300 import scenes

C0 = 299792458.0
EPS0 = 8.8541878128e-12


def _ground(O, freq, x):
    ht, hr = 6.0, 1.5
    s = scenes.ground_plane(tx=(0.0, 0.0, ht), rx=((x, 0.0, hr),), half=5000.0)
    prm = O.OracleParams(freq_hz=freq, max_refl=1)
    keys, _ = O.exhaustive(s.tris.reshape(-1, 9), s.tri_mat, s.materials, s.tx, s.rx[0], prm)
    return s, prm, keys, ht, hr


@pytest.mark.parametrize("freq,x", [(28e9, 50.0), (5.9e9, 200.0)])
def test_two_ray_material_derivative(oracle_mod, freq, x):
    """E = lam/(4 pi) (e^{-jk d1}/d1 + Gamma_TM e^{-jk d2}/d2) (vertical
    polarisation, pure TM). Differentiating Gamma_TM = (eps c - r)/(eps c + r),
    r = sqrt(eps - 1 + c^2), by hand: dGamma/deps = c (eps - 2 s^2) / (r (eps c + r)^2)
    with s^2 = 1 - c^2; eps = eps_r - j sigma / (2 pi f eps0)."""
    O = oracle_mod
    s, prm, keys, ht, hr = _ground(O, freq, x)
    e, de, ok = O.field_gradient(s.tris, s.tri_mat, s.tri_obj, s.materials, s.tx, s.rx[0], keys, prm, nobj=0)
    assert ok.all()
    m = int(s.tri_mat[keys[keys[:, 1] == 1][0, 2]])
    eps_r, sigma = float(np.float32(s.materials[m, 0])), float(np.float32(s.materials[m, 1]))
    d2 = np.hypot(x, ht + hr)
    c = (ht + hr) / d2
    eps = eps_r - 1j * sigma / (2 * np.pi * freq * EPS0)
    r = np.sqrt(eps - (1 - c * c))
    dg = c * (eps - 2 * (1 - c * c)) / (r * (eps * c + r) ** 2)
    k, lam = 2 * np.pi * freq / C0, C0 / freq
    base = lam / (4 * np.pi) * np.exp(-1j * k * d2) / d2
    want_r = base * dg
    want_s = base * dg * (-1j / (2 * np.pi * freq * EPS0))
    got_r, got_s = de[0, 2 * m], de[0, 2 * m + 1]
    assert abs(got_r - want_r) <= 1e-6 * abs(want_r)
    assert abs(got_s - want_s) <= 1e-6 * abs(want_s)
    # materials that no path touches have zero derivative
    for mm in range(s.materials.shape[0]):
        if mm != m:
            assert de[0, 2 * mm] == 0 and de[0, 2 * mm + 1] == 0


def _wall(xw=10.0):
    """A 40 m x 20 m perfectly conducting wall in the plane x = xw, as rigid
    object 0, facing Tx and Rx on the side x < xw."""
    v = np.array([[xw, -20.0, 0.0], [xw, 20.0, 0.0], [xw, 20.0, 20.0], [xw, -20.0, 20.0]])
    tris = np.array([[v[0], v[1], v[2]], [v[0], v[2], v[3]]], np.float64)
    mats = np.array([[5.31, 0.0326, 0.0], [1.0, 0.0, 1.0]])
    tri_mat = np.array([1, 1], np.int32)
    tri_obj = np.array([0, 0], np.int32)
    tx = np.array([0.0, -3.0, 5.0])
    rx = np.array([[-2.0, 4.0, 2.0]])
    return tris, tri_mat, tri_obj, mats, tx, rx


def test_moving_wall_length_derivative(oracle_mod):
    """Image of Tx in the plane x = xw: x_img = 2 xw - x_tx, so
    dL/dxw = 2 (x_img - x_rx) / L, and L does not depend on y."""
    O = oracle_mod
    tris, tri_mat, tri_obj, mats, tx, rx = _wall()
    prm = O.OracleParams(freq_hz=28e9, max_refl=1)
    keys = np.array([[0, 1, 0], [0, 1, 1]], np.int32)
    base = O.path_amp_d(tris, tri_mat, mats, tx, rx, keys, prm)
    row = int(np.flatnonzero(base["valid"])[0])
    key = keys[row:row + 1]
    xw = 10.0
    x_img = 2 * xw - tx[0]
    L = np.sqrt((x_img - rx[0, 0]) ** 2 + (tx[1] - rx[0, 1]) ** 2 + (tx[2] - rx[0, 2]) ** 2)
    assert abs(base["len_m"][row] - L) < 1e-12 * L
    h = 1e-6
    for c, want in [(0, 2 * (x_img - rx[0, 0]) / L), (1, 0.0)]:
        tp, tm = tris.copy(), tris.copy()
        tp[:, :, c] += h
        tm[:, :, c] -= h
        lp = O.path_amp_d(tp, tri_mat, mats, tx, rx, key, prm)["len_m"][0]
        lm = O.path_amp_d(tm, tri_mat, mats, tx, rx, key, prm)["len_m"][0]
        assert abs((lp - lm) / (2 * h) - want) < 1e-7


def test_moving_wall_field_invariant_along_plane(oracle_mod):
    """Translating the wall within its own plane (y) leaves every reflection
    unchanged: dE/dy = 0; along its normal (x) the derivative is not zero and
    matches d/dxw of the single-bounce amplitude at the image geometry."""
    O = oracle_mod
    tris, tri_mat, tri_obj, mats, tx, rx = _wall()
    prm = O.OracleParams(freq_hz=28e9, max_refl=1)
    keys = np.array([[0, 0, -1], [0, 1, 0], [0, 1, 1]], np.int32)
    e, de, ok = O.field_gradient(tris, tri_mat, tri_obj, mats, tx, rx, keys, prm, nobj=1)
    nm = mats.shape[0]
    assert ok[0] and ok[1:].sum() == 1
    dx, dy = de[0, 2 * nm], de[0, 2 * nm + 1]
    assert abs(dy) < 1e-9 * abs(dx)
    # d/dxw at fixed polarisation factors: the phase term dominates at 28 GHz
    k = 2 * np.pi * 28e9 / C0
    xw = 10.0
    x_img = 2 * xw - tx[0]
    L = np.sqrt((x_img - rx[0, 0]) ** 2 + (tx[1] - rx[0, 1]) ** 2 + (tx[2] - rx[0, 2]) ** 2)
    dl = 2 * (x_img - rx[0, 0]) / L
    p = O.path_amp_d(tris, tri_mat, mats, tx, rx, keys[ok], prm)
    a = complex(p["amp_re"][-1], p["amp_im"][-1])
    approx = a * (-1j * k - 1.0 / L) * dl
    assert abs(dx - approx) < 2e-2 * abs(approx)
