"""Pins of the FP64 CPU oracle against closed forms, invariants and brute force.

Each test checks the oracle against something other than itself:
  * Friis free-space loss (Eq. 3 read with path-loss exponent 2, AT = 0),
  * the two-ray ground-reflection model (scalar closed form),
  * image-method path lengths off one plane and between two parallel plates
    (image heights written in closed form, not by iterating mirrors),
  * Fresnel coefficients against Snell-law textbook forms, Brewster's angle,
    normal incidence and the perfect-conductor limit,
  * Tx/Rx reciprocity of the valid path set and amplitudes,
  * sampled-sphere discovery versus exhaustive enumeration of all sequences,
  * the FP32 rigid transform against exact rational arithmetic.
"""
from fractions import Fraction
import json
import os

import numpy as np
import pytest

from paper_2112_07115_gb300 import scenes

C0 = 299792458.0
EPS0 = 8.8541878128e-12
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def f32(x):
    return float(np.float32(x))


def closed_fresnel_lossless(n, theta):
    """Textbook Fresnel amplitudes via Snell's law (lossless, below critical):
    Gamma_s = -sin(ti - tt)/sin(ti + tt), Gamma_p = tan(ti - tt)/tan(ti + tt)."""
    tt = np.arcsin(np.sin(theta) / n)
    if theta == 0.0:
        r = (1 - n) / (1 + n)
        return r, -r
    return (-np.sin(theta - tt) / np.sin(theta + tt), np.tan(theta - tt) / np.tan(theta + tt))


# ---------------------------------------------------------------- paper data

def test_paper_parameters_fixture():
    """Parameter values printed in the paper (Sec. III and Table II)."""
    with open(os.path.join(GOLDEN, "paper_parameters.json")) as fh:
        g = json.load(fh)
    from oracle.oracle import OracleParams
    p = OracleParams()
    assert p.tx_power_w == g["tx_power_outdoor_w"]["value"]
    assert g["max_reflections"]["value"] == 10
    from oracle.oracle import MAX_REFL
    assert MAX_REFL == g["max_reflections"]["value"]


# ---------------------------------------------------------------- Friis

@pytest.mark.parametrize("freq,d", [(28e9, 100.0), (5.9e9, 100.0), (30e9, 37.5), (28e9, 1000.0)])
def test_friis_free_space(oracle_mod, freq, d):
    O = oracle_mod
    s = scenes.free_space(tx=(0.0, 0.0, 0.0), rx=((d, 0.0, 0.0),))
    prm = O.OracleParams(freq_hz=freq, max_refl=2, n_rays=2000)
    rays = scenes.fibonacci_sphere(2000)
    res = O.frame(s, 0, rays, prm)
    # Eq. 3 with n = 2, AT = 0: PL = FSPL(f, 1 m) + 20 log10(d)
    fspl1 = 20 * np.log10(4 * np.pi * freq / C0)
    want = 10 * np.log10(5.0) + 30 - (fspl1 + 20 * np.log10(f32(d)))
    assert res.keys.shape[0] == 1 and res.paths["valid"][0] == 1
    assert abs(res.p_coh_dbm[0] - want) < 1e-9
    assert abs(res.p_inc_dbm[0] - want) < 1e-9
    assert abs(res.paths["delay_s"][0] - f32(d) / C0) < 1e-18


def test_fspl_at_one_metre_values():
    """FSPL(f, 1 m) = 20 log10(4 pi f / c): 61.39 dB at 28 GHz, 61.99 dB at 30 GHz."""
    assert abs(20 * np.log10(4 * np.pi * 28e9 / C0) - 61.3909) < 1e-4
    assert abs(20 * np.log10(4 * np.pi * 30e9 / C0) - 61.9902) < 1e-4


# ---------------------------------------------------------------- two-ray

@pytest.mark.parametrize("freq", [28e9, 5.9e9])
@pytest.mark.parametrize("x", [50.0, 200.0, 733.0])
def test_two_ray_ground(oracle_mod, freq, x):
    O = oracle_mod
    ht, hr = 6.0, 1.5
    s = scenes.ground_plane(tx=(0.0, 0.0, ht), rx=((x, 0.0, hr),), half=5000.0)
    prm = O.OracleParams(freq_hz=freq, max_refl=2)
    keys, paths = O.exhaustive(s.tris.reshape(-1, 9), s.tri_mat, s.materials, s.tx, s.rx[0], prm)
    assert sorted(keys[:, 1].tolist()) == [0, 1]
    _, pc, pi = O.reduce(keys, paths, 1, 5.0)
    # scalar two-ray model; materials enter as their FP32 values
    d1, d2 = np.hypot(x, ht - hr), np.hypot(x, ht + hr)
    cos = (ht + hr) / d2
    gte, gtm = O.fresnel(5.31, 0.0326, 0, freq, cos)
    k, lam = 2 * np.pi * freq / C0, C0 / freq
    e = lam / (4 * np.pi) * (np.exp(-1j * k * d1) / d1 + gtm * np.exp(-1j * k * d2) / d2)
    inc = (lam / (4 * np.pi)) ** 2 * (1 / d1 ** 2 + abs(gtm) ** 2 / d2 ** 2)
    assert abs(pc[0] - (10 * np.log10(5 * abs(e) ** 2) + 30)) < 1e-6
    assert abs(pi[0] - (10 * np.log10(5 * inc) + 30)) < 1e-6
    # image method off one infinite plane: L = sqrt(x^2 + (ht + hr)^2)
    refl = keys[:, 1] == 1
    assert abs(paths["len_m"][refl][0] - d2) < 1e-9
    assert abs(paths["delay_s"][refl][0] - d2 / C0) < 1e-18
    # the reflection point is where the image line crosses z = 0
    assert abs(paths["pts"][refl][0][0][0] - x * ht / (ht + hr)) < 1e-9


def test_vertical_pol_two_ray_far_field_cancels(oracle_mod):
    """Grazing vertical-polarisation reflection tends to -1: at long range the
    coherent power falls well below the incoherent power (d^-4 regime)."""
    O = oracle_mod
    s = scenes.ground_plane(tx=(0.0, 0.0, 6.0), rx=((20000.0, 0.0, 1.5),), half=40000.0)
    prm = O.OracleParams(freq_hz=5.9e9, max_refl=1, escape_len=1e5)
    keys, paths = O.exhaustive(s.tris.reshape(-1, 9), s.tri_mat, s.materials, s.tx, s.rx[0], prm)
    _, pc, pi = O.reduce(keys, paths, 1, 5.0)
    # k * (d2 - d1) ~ 0.11 rad and Gamma_TM ~ -0.998: |1 + Gamma e^{-jk dd}|^2 / 2 ~ -22 dB
    assert pc[0] < pi[0] - 18


# ---------------------------------------------------------------- Fresnel

@pytest.mark.parametrize("freq", [28e9, 5.9e9])
def test_fresnel_normal_incidence(oracle_mod, freq):
    O = oracle_mod
    ec = 5.31 - 1j * 0.0326 / (2 * np.pi * freq * EPS0)
    r = (1 - np.sqrt(ec)) / (1 + np.sqrt(ec))
    te, tm = O.fresnel(5.31, 0.0326, 0, freq, 1.0, exact=True)
    assert abs(te - r) < 1e-13
    assert abs(tm + r) < 1e-13   # Gamma_TM(0) = -Gamma_TE(0) in the p_in/p_out basis


def test_fresnel_normal_incidence_value_28ghz(oracle_mod):
    te, _ = oracle_mod.fresnel(5.31, 0.0326, 0, 28e9, 1.0, exact=True)
    assert abs(te - (-0.394738 + 0.000832j)) < 2e-6
    assert abs(20 * np.log10(abs(te)) - (-8.0738)) < 1e-3


@pytest.mark.parametrize("theta_deg", [0.0, 10.0, 30.0, 45.0, 60.0, 75.0, 85.0, 89.0])
def test_fresnel_lossless_snell(oracle_mod, theta_deg):
    n2 = 5.31
    th = np.radians(theta_deg)
    te, tm = oracle_mod.fresnel(n2, 0.0, 0, 28e9, np.cos(th), exact=True)
    s, p = closed_fresnel_lossless(np.sqrt(n2), th)
    assert abs(te - s) < 1e-12 and abs(tm - p) < 1e-12


def test_fresnel_brewster(oracle_mod):
    er = 5.31
    tb = np.arctan(np.sqrt(er))
    assert abs(np.degrees(tb) - 66.5409) < 1e-4
    te, tm = oracle_mod.fresnel(er, 0.0, 0, 28e9, np.cos(tb), exact=True)
    assert abs(tm) < 1e-12
    assert abs(te - (1 - er) / (1 + er)) < 1e-12


def test_fresnel_pec_and_limits(oracle_mod):
    O = oracle_mod
    for c in [1.0, 0.5, 0.01]:
        te, tm = O.fresnel(1.0, 0.0, 1, 28e9, c)
        assert te == -1 and tm == 1
    for c in [1.0, 0.5]:
        # a very good conductor approaches the PEC values (away from grazing,
        # where a finite conductor's TM coefficient still tends to -1)
        te2, tm2 = O.fresnel(1.0, 1e9, 0, 28e9, c, exact=True)
        assert abs(te2 + 1) < 1e-3 and abs(tm2 - 1) < 1e-3
    # grazing incidence -> -1 for both
    te, tm = O.fresnel(5.31, 0.0326, 0, 28e9, 1e-9, exact=True)
    assert abs(te + 1) < 1e-6 and abs(tm + 1) < 1e-6


def test_fresnel_passive(oracle_mod):
    rng = np.random.default_rng(5)
    for _ in range(300):
        er = rng.uniform(1.0, 80.0)
        sg = 10 ** rng.uniform(-4, 2)
        c = rng.uniform(0, 1)
        te, tm = oracle_mod.fresnel(er, sg, 0, 10 ** rng.uniform(9, 11), c, exact=True)
        assert abs(te) <= 1 + 1e-12 and abs(tm) <= 1 + 1e-12


# ---------------------------------------------------------------- plates

def _plate_image_z(m, first, h, H):
    """Closed-form image height of a source at height h after m alternating
    reflections between z = 0 and z = H, starting on plate `first`."""
    if first == "bottom":
        return -(m - 1) * H - h if m % 2 else m * H + h
    return (m + 1) * H - h if m % 2 else -m * H + h


@pytest.mark.parametrize("freq", [28e9, 5.9e9])
def test_parallel_pec_plates_multibounce(oracle_mod, freq):
    O = oracle_mod
    H, ht, hr, x = 10.0, 3.0, 7.0, 40.0
    s = scenes.parallel_plates(h=H, tx=(0.0, 0.0, ht), rx=((x, 0.0, hr),))
    N = 4
    prm = O.OracleParams(freq_hz=freq, max_refl=N)
    keys, paths = O.exhaustive(s.tris.reshape(-1, 9), s.tri_mat, s.materials, s.tx, s.rx[0], prm)
    bottom = {0, 1}
    lam, k = C0 / freq, 2 * np.pi * freq / C0
    got = {}
    for kk, p in zip(keys, paths):
        m = int(kk[1])
        first = "bottom" if (m and int(kk[2]) in bottom) else "top"
        got.setdefault(m, []).append((first, p))
    assert len(got[0]) == 1
    for m in range(1, N + 1):
        assert sorted(f for f, _ in got[m]) == ["bottom", "top"]
        for first, p in got[m]:
            L = np.hypot(x, _plate_image_z(m, first, ht, H) - hr)
            assert abs(p["len_m"] - L) < 1e-9
            # |Gamma| = 1 and the vertical polarisation maps onto itself
            a = complex(p["amp_re"], p["amp_im"])
            want = lam / (4 * np.pi) * np.exp(-1j * k * L) / L
            # phase k*L carries the FP64 rounding of L (k ~ 590 rad/m at 28 GHz)
            assert abs(a - want) < 1e-9 * abs(want)


def test_plates_sbr_finds_all(oracle_mod):
    """Sampled-sphere discovery recovers every exhaustive path between plates."""
    O = oracle_mod
    s = scenes.parallel_plates(h=10.0, tx=(0.0, 0.0, 3.0), rx=((40.0, 0.0, 7.0),))
    prm = O.OracleParams(max_refl=4, n_rays=200_000)
    res = O.frame(s, 0, scenes.fibonacci_sphere(200_000), prm)
    ek, _ = O.exhaustive(res.world_tris, s.tri_mat, s.materials, s.tx, s.rx[0], prm)
    sbr = {tuple(k) for k, p in zip(res.keys, res.paths) if p["valid"]}
    assert sbr == {tuple(k) for k in ek}


# ---------------------------------------------------------------- reciprocity

@pytest.mark.parametrize("seed", range(6))
def test_reciprocity(oracle_mod, seed):
    O = oracle_mod
    s = scenes.random_tiny(seed, ntri=10, nobj=0, nrx=1)
    wt = s.tris.reshape(-1, 9)
    prm = O.OracleParams(max_refl=3, pol=(0.3, -0.2, 0.9))
    tx, rx = s.tx, s.rx[0][0]
    k1, p1 = O.exhaustive(wt, s.tri_mat, s.materials, tx, rx[None], prm)
    k2, p2 = O.exhaustive(wt, s.tri_mat, s.materials, rx, tx[None], prm)
    fw = {}
    for k, p in zip(k1, p1):
        fw[tuple(k[2:2 + k[1]])] = p
    bw = {}
    for k, p in zip(k2, p2):
        bw[tuple(k[2:2 + k[1]][::-1])] = p
    assert set(fw) == set(bw) and len(fw) >= 2
    for seq in fw:
        a, b = fw[seq], bw[seq]
        assert abs(a["len_m"] - b["len_m"]) < 1e-9
        za, zb = complex(a["amp_re"], a["amp_im"]), complex(b["amp_re"], b["amp_im"])
        assert abs(za - zb) <= 1e-9 * abs(za) + 1e-18


# ---------------------------------------------------------------- discovery

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sbr_subset_of_exhaustive(oracle_mod, seed):
    """Every path the sampled sphere finds is a valid exhaustive path; with
    many rays the two sets coincide on small scenes."""
    O = oracle_mod
    s = scenes.random_tiny(seed, ntri=8, nobj=2, nrx=2)
    for n_rays in (3000, 400_000):
        prm = O.OracleParams(max_refl=2, n_rays=n_rays)
        res = O.frame(s, 1, scenes.fibonacci_sphere(n_rays), prm)
        ek, _ = O.exhaustive(res.world_tris, s.tri_mat, s.materials, s.tx, s.rx[1], prm)
        ex = {tuple(k) for k in ek}
        sbr = {tuple(k) for k, p in zip(res.keys, res.paths) if p["valid"]}
        assert sbr <= ex
        if n_rays > 100_000:
            assert sbr == ex


def test_toy_street_sbr_equals_exhaustive(oracle_mod):
    O = oracle_mod
    s = scenes.toy_street()
    prm = O.OracleParams(max_refl=3, n_rays=10_000)
    res = O.frame(s, 0, scenes.fibonacci_sphere(10_000), prm)
    ek, ep = O.exhaustive(res.world_tris, s.tri_mat, s.materials, s.tx, s.rx[0], prm)
    sbr = {tuple(k) for k, p in zip(res.keys, res.paths) if p["valid"]}
    assert sbr == {tuple(k) for k in ek}
    _, pc, pi = O.reduce(ek, ep, s.nrx, 5.0)
    assert np.allclose(pc, res.p_coh_dbm, atol=1e-12) and np.allclose(pi, res.p_inc_dbm, atol=1e-12)


# ---------------------------------------------------------------- flags

def test_edge_flag(oracle_mod):
    """A ray aimed at the shared diagonal of the two ground triangles is
    flagged; a ray aimed at a triangle interior is not."""
    O = oracle_mod
    s = scenes.ground_plane(tx=(0.0, 0.0, 6.0), half=100.0)
    d_edge = np.array([[10.0, 10.0, -6.0]]) / np.linalg.norm([10.0, 10.0, -6.0])
    d_in = np.array([[10.0, -4.0, -6.0]]) / np.linalg.norm([10.0, -4.0, -6.0])
    prm = O.OracleParams(max_refl=1)
    for d, want in ((d_edge, True), (d_in, False)):
        tr = O.trace(s.tris.reshape(-1, 9), s.tri_mat, s.materials, s.tx, d.astype(np.float32),
                     s.rx[0], prm)
        assert bool(tr["flags"][0] & O.NEAR_EDGE) == want
        assert tr["hit_id"][0, 0] in (0, 1)


def test_reflection_law(oracle_mod):
    """Two-segment ray off the ground: the second segment's direction is the
    mirror image of the first (angle of incidence = angle of reflection)."""
    O = oracle_mod
    s = scenes.ground_plane(tx=(0.0, 0.0, 6.0), half=100.0)
    d = np.array([[3.0, -4.0, -6.0]], np.float32)
    d /= np.linalg.norm(d)
    tr = O.trace(s.tris.reshape(-1, 9), s.tri_mat, s.materials, s.tx, d, s.rx[0],
                 O.OracleParams(max_refl=1), seg_od=True)
    od = tr["seg_od"][0]
    d0 = d[0].astype(np.float64) / np.linalg.norm(d[0].astype(np.float64))
    assert np.allclose(od[1, 3:6], d0 * [1, 1, -1], atol=1e-15)
    assert abs(tr["hit_t"][0, 0] - 6.0 / -d0[2]) < 1e-12
    assert abs(od[1, 6] - tr["hit_t"][0, 0]) < 1e-12          # unfolded length D
    assert tr["hit_id"][0, 1] == -1 and tr["nseg"][0] == 2


# ---------------------------------------------------------------- transform

def _fmaf_exact(a, b, c):
    """Correctly rounded float32 of a*b + c using exact rationals."""
    v = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    f = np.float32(float(v))
    cands = [f, np.nextafter(f, np.float32(np.inf)), np.nextafter(f, np.float32(-np.inf))]
    best = None
    for x in cands:
        err = abs(Fraction(float(x)) - v)
        if best is None or err < best[0] or (err == best[0] and
                                             (np.float32(x).view(np.uint32) & 1) == 0):
            best = (err, x)
    return np.float32(best[1])


def _random_xf(rng, n):
    """General rigid transforms: random unit quaternion rotations + translations."""
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                  2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                  2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1)
    t = rng.uniform(-1500, 1500, size=(n, 3))
    xf = np.concatenate([R.reshape(n, 3, 3), t[:, :, None]], axis=2).reshape(n, 12)
    return xf.astype(np.float32)


def test_transform_fmaf_order(oracle_mod):
    """x' = fmaf(R0, x, fmaf(R1, y, fmaf(R2, z, t))) with each fmaf correctly
    rounded, checked bit for bit against exact rational arithmetic."""
    O = oracle_mod
    rng = np.random.default_rng(1)
    nobj, ntri = 6, 60
    xf = _random_xf(rng, nobj)
    tris = rng.uniform(-7, 7, size=(ntri, 3, 3)).astype(np.float32)
    tri_obj = rng.integers(-1, nobj, size=ntri).astype(np.int32)
    wt = O.transform(tris, tri_obj, xf)
    for i in range(ntri):
        if tri_obj[i] < 0:
            assert np.array_equal(wt[i].view(np.uint32), tris[i].view(np.uint32))
            continue
        m = xf[tri_obj[i]]
        for k in range(3):
            v = tris[i, k]
            for r in range(3):
                inner = _fmaf_exact(m[4 * r + 2], v[2], m[4 * r + 3])
                mid = _fmaf_exact(m[4 * r + 1], v[1], inner)
                want = _fmaf_exact(m[4 * r + 0], v[0], mid)
                assert wt[i, k, r].view(np.uint32) == want.view(np.uint32)


def test_transform_highway_static_untouched(oracle_mod):
    O = oracle_mod
    s = scenes.highway(n_frames=2, n_vehicles=10, length=400.0)
    wt = O.transform(s.tris, s.tri_obj, s.xf[1])
    st = np.nonzero(s.tri_obj < 0)[0]
    assert np.array_equal(wt[st].view(np.uint32), s.tris[st].view(np.uint32))


def test_transform_exact_cases(oracle_mod):
    """Identity and quarter-turn rotations with integral translations are exact."""
    O = oracle_mod
    tris = np.array([[[1.5, -2.25, 0.5], [3.0, 4.0, 5.0], [-7.0, 0.125, 2.0]]], np.float32)
    ident = np.array([[1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0]], np.float32)
    assert np.array_equal(O.transform(tris, np.array([0]), ident), tris)
    rot = np.array([[0, -1, 0, 10, 1, 0, 0, -20, 0, 0, 1, 3]], np.float32)
    out = O.transform(tris, np.array([0]), rot)
    want = np.stack([10 - tris[0, :, 1], -20 + tris[0, :, 0], 3 + tris[0, :, 2]], axis=1)
    assert np.array_equal(out[0], want.astype(np.float32))


# ---------------------------------------------------------------- path cache

def test_sticky_retention_keeps_true_paths(oracle_mod):
    """The path cache's retention mode (Sec. III "Propagation path caching"):
    with few rays, discovery misses paths from frame to frame, and retention
    keeps paths found earlier. Every path a frame reports (captured or kept)
    is a true path of that frame's geometry: it is in the exhaustive
    enumeration of all sequences, with the same length and amplitude. Kept
    paths were valid in the previous frame, and each frame's set contains the
    plain frame's valid set."""
    O = oracle_mod
    s = scenes.toy_street()
    n = 200
    prm = O.OracleParams(max_refl=2, n_rays=n)
    rays = scenes.fibonacci_sphere(n)
    res = O.sticky_frames(s, range(10), rays, prm)
    kept_total = 0
    prev_valid = set()
    for f, r in enumerate(res):
        ek, ep = O.exhaustive(r.world_tris, s.tri_mat, s.materials, s.tx, s.rx[f], prm)
        ex = {tuple(k): p for k, p in zip(ek.tolist(), ep)}
        valid = {tuple(k): p for k, p in zip(r.keys.tolist(), r.paths) if p["valid"]}
        assert set(valid) <= set(ex)
        for k, p in valid.items():
            assert abs(p["len_m"] - ex[k]["len_m"]) <= 1e-9 and abs(p["amp_re"] - ex[k]["amp_re"]) <= 1e-12
        plain = O.frame(s, f, rays, prm)
        assert {tuple(k) for k, p in zip(plain.keys.tolist(), plain.paths) if p["valid"]} <= set(valid)
        kept = {tuple(k) for k in r.extra["kept_only"].tolist()}
        assert kept <= prev_valid and kept <= set(valid)
        kept_total += len(kept)
        prev_valid = set(valid)
    assert kept_total > 0


# ---------------------------------------------------------------- transmission

def _walls(xs, tx=(0.0, 3.0, 7.0), rx=(100.0, 3.0, 7.0)):
    """Square walls (100 m x 100 m, two triangles each) in the planes x = xs[k],
    wall k of material k; the Tx-Rx line crosses them off their diagonals."""
    tris, mats = [], []
    for k, x in enumerate(xs):
        tris += scenes._quad((x, -50.0, -50.0), (x, 50.0, -50.0), (x, 50.0, 50.0), (x, -50.0, 50.0))
        mats += [k, k]
    materials = np.array([[5.31, 0.0326, 0.0]] * len(xs), np.float32)
    return scenes._static_scene("walls", tris, mats, tx, rx, materials=materials)


def _table2():
    with open(os.path.join(GOLDEN, "paper_parameters.json")) as fh:
        rows = json.load(fh)["table2_materials"]["rows"]
    return {r["material"]: r for r in rows}


def _los_amp(freq, L, loss_db=0.0):
    lam = C0 / freq
    k = 2 * np.pi * freq / C0
    return lam / (4 * np.pi * L) * np.exp(-1j * k * L) * 10.0 ** (-loss_db / 20.0)


def test_transmission_table2_wall_friis_minus_loss(oracle_mod):
    """Table II's indoor wall (20 dB) between Tx and Rx: the only path is the
    direct one through the wall, a = Friis amplitude x 10^(-20/20); the
    sampled sphere (the paper's 2000 rays) finds exactly that path."""
    O = oracle_mod
    loss = _table2()["wall (indoor)"]["penetration_loss_db"]
    s = _walls([50.0])
    prm = O.OracleParams(freq_hz=30e9, n_rays=2000, max_refl=2, max_trans=2, trans_db=(loss,))
    ek, ep = O.exhaustive(s.tris.reshape(-1, 9), s.tri_mat, s.materials, s.tx, s.rx[0], prm)
    assert ek.shape[0] == 1 and ek[0, 1] == 1 and (ek[0, 2] & O.TRANS)
    a = complex(ep[0]["amp_re"], ep[0]["amp_im"])
    assert abs(ep[0]["len_m"] - 100.0) <= 1e-12
    assert abs(a - _los_amp(30e9, 100.0, loss)) <= 1e-12 * abs(a)
    res = O.frame(s, 0, scenes.fibonacci_sphere(2000), prm)
    assert {tuple(k) for k, p in zip(res.keys.tolist(), res.paths) if p["valid"]} == {tuple(ek[0])}
    # received power: Friis minus the penetration loss
    friis = 10 * np.log10(prm.tx_power_w * (C0 / 30e9 / (4 * np.pi * 100.0)) ** 2) + 30
    assert abs(res.p_coh_dbm[0] - (friis - loss)) <= 1e-9


def test_transmission_losses_add_and_limits(oracle_mod):
    """Wall (20 dB) then glass (5 dB): one path through both at Friis - 25 dB;
    with one transmission allowed, or with the glass opaque, no path."""
    O = oracle_mod
    t2 = _table2()
    lw, lg = t2["wall (indoor)"]["penetration_loss_db"], t2["glass (indoor)"]["penetration_loss_db"]
    s = _walls([30.0, 60.0])
    wt = s.tris.reshape(-1, 9)
    prm = O.OracleParams(freq_hz=30e9, max_refl=1, max_trans=2, trans_db=(lw, lg))
    ek, ep = O.exhaustive(wt, s.tri_mat, s.materials, s.tx, s.rx[0], prm)
    assert ek.shape[0] == 1 and ek[0, 1] == 2 and (ek[0, 2] & O.TRANS) and (ek[0, 3] & O.TRANS)
    # the first crossing is the 30 m wall (triangles 0/1), then the glass (2/3)
    assert (ek[0, 2] & ~O.TRANS) in (0, 1) and (ek[0, 3] & ~O.TRANS) in (2, 3)
    a = complex(ep[0]["amp_re"], ep[0]["amp_im"])
    assert abs(a - _los_amp(30e9, 100.0, lw + lg)) <= 1e-12 * abs(a)
    p1 = O.OracleParams(freq_hz=30e9, max_refl=1, max_trans=1, trans_db=(lw, lg))
    assert O.exhaustive(wt, s.tri_mat, s.materials, s.tx, s.rx[0], p1)[0].shape[0] == 0
    p2 = O.OracleParams(freq_hz=30e9, max_refl=1, max_trans=2, trans_db=(lw, -1.0))
    assert O.exhaustive(wt, s.tri_mat, s.materials, s.tx, s.rx[0], p2)[0].shape[0] == 0
    # the same key with the glass reversed in order is not a path
    bad = ek.copy()
    bad[0, 2], bad[0, 3] = ek[0, 3], ek[0, 2]
    assert not O.validate(wt, s.tri_mat, s.materials, s.tx, s.rx[0], bad, prm)["valid"][0]


def test_transmission_zero_loss_is_free_space(oracle_mod):
    """A 0 dB wall changes nothing but the path's interaction list: the
    amplitude equals the free-space line of sight."""
    O = oracle_mod
    s = _walls([40.0])
    prm = O.OracleParams(freq_hz=28e9, max_refl=1, max_trans=1, trans_db=(0.0,))
    ek, ep = O.exhaustive(s.tris.reshape(-1, 9), s.tri_mat, s.materials, s.tx, s.rx[0], prm)
    f = scenes.free_space(tx=tuple(s.tx), rx=tuple(map(tuple, s.rx[0])))
    fk, fp = O.exhaustive(np.zeros((0, 9), np.float32), f.tri_mat, f.materials, f.tx, f.rx[0],
                          O.OracleParams(freq_hz=28e9, max_refl=1))
    assert ek.shape[0] == 1 and fk.shape[0] == 1
    a, b = complex(ep[0]["amp_re"], ep[0]["amp_im"]), complex(fp[0]["amp_re"], fp[0]["amp_im"])
    assert abs(a - b) <= 1e-13 * abs(b)


@pytest.mark.parametrize("seed", [0, 2, 5])
def test_transmission_sbr_subset_of_exhaustive(oracle_mod, seed):
    """With transmitting materials (ground 10 dB, the rest 3 dB), every path
    the ray tree finds is a valid exhaustive path, and with many rays the two
    sets coincide."""
    O = oracle_mod
    s = scenes.random_tiny(seed, ntri=6, nobj=1, nrx=2)
    mats = np.vstack([s.materials, s.materials[:1]])
    tm = s.tri_mat.copy()
    tm[2:] = mats.shape[0] - 1
    s.materials, s.tri_mat = mats, tm
    tdb = (10.0,) + (-1.0,) * (mats.shape[0] - 2) + (3.0,)
    for n_rays in (3000, 200_000):
        prm = O.OracleParams(max_refl=1, max_trans=1, n_rays=n_rays, trans_db=tdb)
        res = O.frame(s, 1, scenes.fibonacci_sphere(n_rays), prm)
        ek, _ = O.exhaustive(res.world_tris, s.tri_mat, s.materials, s.tx, s.rx[1], prm)
        ex = {tuple(k) for k in ek.tolist()}
        sbr = {tuple(k) for k, p in zip(res.keys.tolist(), res.paths) if p["valid"]}
        assert sbr <= ex
        assert any(any(v >= 0 and (v & O.TRANS) for v in k[2:]) for k in ex)
        if n_rays > 100_000:
            assert sbr == ex


# ---------------------------------------------------------------- diffraction

def test_utd_transition_function_vs_fresnel_integrals(oracle_mod):
    """F(x) = 2j sqrt(x) e^{jx} int_{sqrt x}^inf e^{-j t^2} dt (Kouyoumjian &
    Pathak 1974) against the Fresnel integrals of scipy: the tail integral is
    sqrt(pi/2) [(1/2 - C(z)) - j (1/2 - S(z))], z = sqrt(2x/pi)."""
    sp = pytest.importorskip("scipy.special")
    O = oracle_mod
    for x in (1e-6, 1e-3, 0.3, 1.0, 3.0, 10.0, 100.0, 1e4):
        z = np.sqrt(2.0 * x / np.pi)
        S, Cf = sp.fresnel(z)
        ref = 2j * np.sqrt(x) * np.exp(1j * x) * np.sqrt(np.pi / 2) * ((0.5 - Cf) - 1j * (0.5 - S))
        assert abs(O.transition(x) - ref) <= 1e-10 * abs(ref), x


@pytest.mark.parametrize("phi,phip", [(2.0, 0.5), (4.5, 1.0), (5.5, 0.3), (3.0, 2.5)])
def test_utd_half_plane_reduces_to_keller(oracle_mod, phi, phip):
    """Far from the shadow boundaries (F -> 1) the UTD coefficient of a
    perfectly conducting half plane (n = 2) is Keller's:
    -e^{-j pi/4} / (2 sqrt(2 pi k) sin b0) [sec((phi-phi')/2) -/+ sec((phi+phi')/2)]."""
    O = oracle_mod
    k = 2 * np.pi * 28e9 / C0
    for b0 in (np.pi / 2, 1.1):
        for sgn, R in ((-1.0, -1.0), (1.0, 1.0)):
            D = O.utd_coefficient(2.0, phi, phip, b0, 1e10, k, R, R)
            ref = -np.exp(-1j * np.pi / 4) / (2 * np.sqrt(2 * np.pi * k) * np.sin(b0)) * (
                1 / np.cos((phi - phip) / 2) + sgn / np.cos((phi + phip) / 2))
            assert abs(D - ref) <= 1e-8 * abs(ref)


def test_utd_total_field_continuous_at_shadow_boundary(oracle_mod):
    """Plane wave on a conducting half plane: the geometric-optics field
    switches off at the incident shadow boundary phi = phi' + pi, and the
    diffracted field makes up the jump, so the total field is continuous."""
    O = oracle_mod
    k = 2 * np.pi * 28e9 / C0
    phip, s = 0.7, 2.0

    def total(phi):
        go = np.exp(1j * k * s * np.cos(phi - phip)) if phi - phip < np.pi else 0.0
        d = O.utd_coefficient(2.0, phi, phip, np.pi / 2, s, k, -1.0, -1.0)
        return go + d * np.exp(-1j * k * s) / np.sqrt(s)

    for delta, tol in ((1e-5, 1e-3), (1e-7, 1e-5)):
        a, b = total(np.pi + phip - delta), total(np.pi + phip + delta)
        assert abs(a - b) <= tol
        # each part alone jumps by about half the incident field
        assert abs(O.utd_coefficient(2.0, np.pi + phip + delta, phip, np.pi / 2, s, k, -1.0, -1.0) -
                   O.utd_coefficient(2.0, np.pi + phip - delta, phip, np.pi / 2, s, k, -1.0, -1.0)) > 0.5


def _corner(rx=(-20.0, 30.0, 2.0)):
    """A building corner: walls y = 0 (x in [0, 50]) and x = 0 (y in [0, 50])
    meeting at the vertical edge x = y = 0; Tx at (30, -20, 2)."""
    tris = scenes._quad((0.0, 0.0, -50.0), (50.0, 0.0, -50.0), (50.0, 0.0, 50.0), (0.0, 0.0, 50.0))
    tris += scenes._quad((0.0, 0.0, -50.0), (0.0, 50.0, -50.0), (0.0, 50.0, 50.0), (0.0, 0.0, 50.0))
    return scenes._static_scene("corner", tris, [0, 0, 0, 0], (30.0, -20.0, 2.0), (rx,))


def test_diffraction_path_around_a_corner(oracle_mod):
    """Tx and Rx on the two sides of a concrete building corner (no line of
    sight, no reflection path): one diffraction path at Q = (0, 0, 2) (Keller:
    equal angles with the edge), whose field, assembled here from the
    geometry and the UTD coefficient (vertical polarisation along a vertical
    edge: the soft coefficient with Luebbers' TE factors), is the oracle's."""
    O = oracle_mod
    sc = _corner()
    wt = sc.tris.reshape(-1, 9)
    assert O.count_wedges(wt, sc.tri_obj) == 1
    prm = O.OracleParams(freq_hz=28e9, max_refl=2, diffraction=True)
    ek, _ = O.exhaustive(wt, sc.tri_mat, sc.materials, sc.tx, sc.rx[0], prm)
    assert ek.shape[0] == 0
    dk, dp = O.diffract(wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[0], prm)
    assert dk.shape[0] == 1 and dk[0, 1] == 1 and (dk[0, 2] & O.DIFF)
    assert np.allclose(dp[0]["pts"][0], [0.0, 0.0, 2.0], atol=1e-12)
    sp_, s_ = np.hypot(30.0, 20.0), np.hypot(20.0, 30.0)
    assert abs(dp[0]["len_m"] - (sp_ + s_)) <= 1e-9
    k = 2 * np.pi * 28e9 / C0
    n = 1.5
    # angles from one face through the exterior (the result does not depend
    # on which face is face 0: both are concrete)
    phip = np.arctan2(20.0, 30.0)
    phi = 2 * np.pi - np.arctan2(30.0, -20.0)
    L = s_ * sp_ / (s_ + sp_)
    er, sg = float(np.float32(5.31)), float(np.float32(0.0326))   # the scene's FP32 material
    g0, _ = O.fresnel(er, sg, 0, 28e9, abs(np.sin(phip)), exact=True)
    gn, _ = O.fresnel(er, sg, 0, 28e9, abs(np.sin(n * np.pi - phi)), exact=True)
    Ds = O.utd_coefficient(n, phi, phip, np.pi / 2, L, k, g0, gn)
    lam = C0 / 28e9
    a = lam / (4 * np.pi) * Ds * np.exp(-1j * k * (sp_ + s_)) / sp_ * np.sqrt(sp_ / (s_ * (s_ + sp_)))
    got = complex(dp[0]["amp_re"], dp[0]["amp_im"])
    assert abs(got - a) <= 1e-9 * abs(a)
    # a receiver in sight of the transmitter: no diffraction path (the
    # paper's step 5 keeps sources in the receiver's shadow region)
    lit = _corner(rx=(-20.0, -30.0, 2.0))
    assert O.diffract(wt, lit.tri_mat, lit.tri_obj, lit.materials, lit.tx, lit.rx[0], prm)[0].shape[0] == 0


def test_toy_street_wedges_and_diffraction_frame(oracle_mod):
    """The toy street's two buildings have four vertical corner wedges each
    and its four vehicle boxes eight each (four roof edges, four vertical);
    with receivers behind the buildings (seen from the Tx), a diffraction
    frame adds diffraction paths to the reflection paths and sums them."""
    O = oracle_mod
    sc = scenes.toy_street()
    behind = np.array([[-30.0, 45.0, 1.5], [30.0, -45.0, 1.5], [-45.0, 30.0, 1.5], [12.0, 12.0, 1.5]], np.float32)
    sc.rx = np.repeat(behind[None], sc.nframes, axis=0)
    wt = O.transform(sc.tris, sc.tri_obj, sc.xf[0])
    assert O.count_wedges(wt, sc.tri_obj) == 8 + 4 * 8
    static = sc.tri_obj < 0
    assert O.count_wedges(wt[static], sc.tri_obj[static]) == 8
    prm = O.OracleParams(max_refl=2, n_rays=10_000, diffraction=True)
    r = O.frame(sc, 0, scenes.fibonacci_sphere(10_000), prm)
    d = (r.keys[:, 2] >= 0) & ((r.keys[:, 2] & O.DIFF) != 0)
    assert d.any() and r.paths["valid"][d].all()
    plain = O.frame(sc, 0, scenes.fibonacci_sphere(10_000), O.OracleParams(max_refl=2, n_rays=10_000))
    assert set(map(tuple, plain.keys.tolist())) == set(map(tuple, r.keys[~d].tolist()))


def _ground_and_building(ground_mat, building_mat, tx, rx, with_ground=True):
    """A 20 x 20 x 15 m box building centred at the origin on a ground plane
    z = 0 (two triangles, 400 m square), or the building alone."""
    tris = scenes._quad((-200.0, -200.0, 0.0), (200.0, -200.0, 0.0), (200.0, 200.0, 0.0), (-200.0, 200.0, 0.0)) \
        if with_ground else []
    mats = [ground_mat] * len(tris)
    b = scenes.box_tris(20.0, 20.0, 15.0)
    tris += b
    mats += [building_mat] * len(b)
    return scenes._static_scene("ground_building", tris, mats, tx, (rx,))


def _paths_by_point(keys, paths, slot):
    """{rounded diffraction point: (amplitude, length)} of combined paths,
    the diffraction point at pts[slot]."""
    out = {}
    for k, p in zip(keys, paths):
        q = tuple(np.round(p["pts"][slot], 6))
        out[q] = (complex(p["amp_re"], p["amp_im"]), float(p["len_m"]))
    return out


@pytest.mark.parametrize("building_mat", [scenes.MAT_METAL, scenes.MAT_CONCRETE])
@pytest.mark.parametrize("tx,rx", [((-40.0, -12.0, 2.0), (35.0, 22.0, 10.0)),    # reflection first
                                   ((-40.0, -12.0, 6.0), (35.0, 22.0, 2.0))])    # reflection last
def test_reflection_then_diffraction_is_the_image_source_diffracted(oracle_mod, building_mat, tx, rx):
    """Image theory over a perfectly conducting ground, vertical polarisation:
    the ground reflection before a wedge (Tx -> P -> Q -> Rx) equals the
    first-order diffraction of the transmitter's image (no ground), and the
    reflection after it (Tx -> Q -> P -> Rx) the diffraction toward the
    receiver's image -- same diffraction points, lengths and amplitudes (the
    PEC reflection of a vertically polarised field is the image's field)."""
    O = oracle_mod
    a = _ground_and_building(scenes.MAT_METAL, building_mat, tx, rx)
    prm = O.OracleParams(freq_hz=28e9, max_refl=2)
    wa = a.tris.reshape(-1, 9)
    keys, paths = O.diffract_refl(wa, a.tri_mat, a.tri_obj, a.materials, a.tx, a.rx[0], prm)
    first = (keys[:, 3] >= 0) & ((keys[:, 3] & O.DIFF) != 0)          # reflection, then wedge
    last = (keys[:, 2] >= 0) & ((keys[:, 2] & O.DIFF) != 0)           # wedge, then reflection
    ground = lambda col: keys[:, col] < 2                             # the ground's two triangles
    rd = first & ground(2)
    dr = last & ground(3)
    assert rd.sum() + dr.sum() >= 2
    for sel, src, obs, slot in ((rd, (tx[0], tx[1], -tx[2]), rx, 1), (dr, tx, (rx[0], rx[1], -rx[2]), 0)):
        b = _ground_and_building(scenes.MAT_METAL, building_mat, src, obs, with_ground=False)
        bk, bp = O.diffract(b.tris.reshape(-1, 9), b.tri_mat, b.tri_obj, b.materials, b.tx, b.rx[0], prm)
        # the image's diffraction points on the real edges (above the ground)
        want = {q: v for q, v in _paths_by_point(bk, bp, 0).items() if q[2] > 0.0}
        got = _paths_by_point(keys[sel], paths[sel], slot)
        assert set(got) == set(want)
        for q, (amp, length) in got.items():
            wa_, wl = want[q]
            assert abs(length - wl) <= 1e-9 * wl
            assert abs(amp - wa_) <= 1e-9 * abs(wa_)


def test_reflection_diffraction_reciprocity(oracle_mod):
    """Perfect conductors everywhere (reciprocal face factors): swapping Tx and
    Rx turns each reflection-then-wedge path into the wedge-then-reflection
    path with the same triangle, wedge, length and amplitude."""
    O = oracle_mod
    tx, rx = (-40.0, -12.0, 6.0), (35.0, 22.0, 2.0)
    prm = O.OracleParams(freq_hz=28e9, max_refl=2)
    out = []
    for t, r in ((tx, rx), (rx, tx)):
        sc = _ground_and_building(scenes.MAT_METAL, scenes.MAT_METAL, t, r)
        k, p = O.diffract_refl(sc.tris.reshape(-1, 9), sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[0], prm)
        out.append({tuple(kk[2:4].tolist()): (complex(pp["amp_re"], pp["amp_im"]), float(pp["len_m"]))
                    for kk, pp in zip(k, p)})
    fwd, back = out
    assert len(fwd) >= 2 and len(fwd) == len(back)
    for (i0, i1), (amp, length) in fwd.items():
        amp2, len2 = back[(i1, i0)]
        assert abs(length - len2) <= 1e-9 * length
        assert abs(amp - amp2) <= 1e-9 * abs(amp)


# ---------------------------------------------------------------------------
# diffraction of order 2 and 3 (Sec. III step 5, bound 3)
# ---------------------------------------------------------------------------
def _slab(x0, x1, y0, y1, h=10.0):
    """A thin vertical wall (four side faces, no top: only its vertical edges are wedges)."""
    return scenes.box_tris(x1 - x0, y1 - y0, h, center=((x0 + x1) / 2, (y0 + y1) / 2, 0.0),
                           faces=("xm", "xp", "ym", "yp"))


def _prism(theta, r_tip=20.0, r_base=8.0, half=2.0, h=10.0):
    """A thin vertical triangular prism pointing radially outward at angle theta: its tip is a
    sharp vertical wedge (interior angle about 19 degrees)."""
    c, s = np.cos(theta), np.sin(theta)
    tip = np.array([r_tip * c, r_tip * s])
    t = np.array([-s, c])
    b1, b2 = np.array([r_base * c, r_base * s]) + half * t, np.array([r_base * c, r_base * s]) - half * t
    out = []
    for a, b in ((tip, b1), (b1, b2), (b2, tip)):
        out += scenes._quad((a[0], a[1], 0.0), (b[0], b[1], 0.0), (b[0], b[1], h), (a[0], a[1], h))
    return out


def _composition_check(O, sc, m, prm):
    """The one path of order m of a scene whose wedges are parallel vertical edges, with Tx, Rx
    and so every Keller point at one height. For parallel edges the astigmatic spreading of
    successive edge-diffracted waves reduces to a closed form: the wave behind edge i has
    caustics on edge i and at the unfolded distance back to the source, which gives
    a_m = (lam/4pi) D_1 .. D_m e^{-jkS} / sqrt(s_0 s_1 .. s_m S) (S the unfolded length), with
    edge i's distance parameter s_{i-1} s_i / (s_{i-1} + s_i) -- the one of a first-order
    diffraction from Q_{i-1} toward Q_{i+1}. So a_m equals the product of the m first-order
    amplitudes (Q_{i-1} -> wedge i -> Q_{i+1}, each computed by or_diffract on its own) times
    (4pi/lam)^(m-1) e^{jk(s_1 + .. + s_{m-1})} sqrt(s_1 .. s_{m-1} (s_0+s_1) .. (s_{m-1}+s_m) / S).
    The first-order calls also find the same Keller points (Keller's law at each edge). The
    Keller points are exact in FP32 (their x, y are vertices, z the common height), so the
    first-order calls see exactly the same geometry."""
    k, lam = 2.0 * np.pi * prm.freq_hz / C0, C0 / prm.freq_hz
    wt = sc.tris.reshape(-1, 9)
    keys, paths = O.diffract_multi(wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[0], prm, m)
    assert len(keys) == 1, keys
    p = paths[0]
    Q = [p["pts"][i].astype(np.float64) for i in range(m)]
    T, R = sc.tx.astype(np.float64), sc.rx[0][0].astype(np.float64)
    for q in Q:
        assert q[2] == T[2] == R[2]
    X = [T] + Q + [R]
    s = [float(np.linalg.norm(X[i + 1] - X[i])) for i in range(m + 1)]
    S = sum(s)
    assert abs(p["len_m"] - S) <= 1e-12 * S
    ws = [int(x) & ~O.DIFF for x in keys[0][2:2 + m]]
    prod = 1.0 + 0.0j
    for i in range(m):
        kk, pp = O.diffract(wt, sc.tri_mat, sc.tri_obj, sc.materials, X[i].astype(np.float32),
                            X[i + 2].astype(np.float32)[None], prm)
        j = [q for q, key in enumerate(kk) if (key[2] & ~O.DIFF) == ws[i]]
        assert len(j) == 1
        assert np.max(np.abs(pp["pts"][j[0]][0] - Q[i])) <= 1e-9
        prod *= complex(pp["amp_re"][j[0]], pp["amp_im"][j[0]])
    inner = np.prod(s[1:m]) * np.prod([s[i] + s[i + 1] for i in range(m)])
    want = prod * (4.0 * np.pi / lam) ** (m - 1) * np.exp(1j * k * sum(s[1:m])) * np.sqrt(inner / S)
    got = complex(p["amp_re"], p["amp_im"])
    assert abs(got - want) <= 1e-9 * abs(want), (got, want)


@pytest.mark.parametrize("mat", [scenes.MAT_METAL, scenes.MAT_CONCRETE])
def test_double_diffraction_composes_from_first_order(oracle_mod, mat):
    """Two thin walls, one reaching south from y = 0 and one north from y = 5: no direct or
    first-order path, one double diffraction around the walls' ends. The two edges of one wall's
    end face are not a chain (each lies in a face plane of the other: the leg would run along
    that face)."""
    O = oracle_mod
    tris = _slab(0.0, 0.5, -50.0, 0.0) + _slab(10.0, 10.5, 5.0, 55.0)
    sc = scenes._static_scene("walls", tris, [mat] * len(tris), (-10.0, -20.0, 2.0), [(20.0, 20.0, 2.0)])
    prm = O.OracleParams(freq_hz=28e9, max_refl=3)
    k1, _ = O.diffract(sc.tris.reshape(-1, 9), sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[0], prm)
    assert len(k1) == 0
    _composition_check(O, sc, 2, prm)


@pytest.mark.parametrize("mat", [scenes.MAT_METAL, scenes.MAT_CONCRETE])
def test_triple_diffraction_composes_from_first_order(oracle_mod, mat):
    """Three thin prisms at 60, 0 and -60 degrees: the path wraps around their tips, each tip
    hiding the point after the next one."""
    O = oracle_mod
    tris = []
    for a in np.deg2rad([60.0, 0.0, -60.0]):
        tris += _prism(a)
    at = lambda deg: (22.0 * np.cos(np.deg2rad(deg)), 22.0 * np.sin(np.deg2rad(deg)), 2.0)
    sc = scenes._static_scene("prisms", tris, [mat] * len(tris), at(120.0), [at(-120.0)])
    prm = O.OracleParams(freq_hz=28e9, max_refl=3)
    wt = sc.tris.reshape(-1, 9)
    for m in (1, 2):
        fn = (lambda: O.diffract(wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[0], prm)) if m == 1 else \
            (lambda: O.diffract_multi(wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[0], prm, m))
        assert len(fn()[0]) == 0
    _composition_check(O, sc, 3, prm)


def _crossed_edges():
    """Three boxes: an order-2 path over a horizontal roof edge (box 0, x = 2.25, z = 4, along y)
    and then a vertical corner (box 1, x = 7.25, y = 2.75)."""
    boxes = [(4.5, 6.0, 4.0, 4.5, -12.5), (4.5, 8.5, 7.5, 5.0, 7.0), (7.0, 4.5, 9.5, -11.5, -7.0)]
    tris = []
    for lx, ly, lz, cx, cy in boxes:
        tris += scenes.box_tris(lx, ly, lz, center=(cx, cy, 0.0))
    return tris, (-4.0, -31.0, 2.5), (12.0, 19.5, 6.0)


def _crossed_path(O, tris, tx, rx, freq):
    sc = scenes._static_scene("boxes", tris, [scenes.MAT_METAL] * len(tris), tx, [rx])
    prm = O.OracleParams(freq_hz=freq, max_refl=3)
    keys, paths = O.diffract_multi(sc.tris.reshape(-1, 9), sc.tri_mat, sc.tri_obj, sc.materials, sc.tx,
                                   sc.rx[0], prm, 2)
    sel = [i for i, p in enumerate(paths) if abs(p["pts"][0][2] - 4.0) < 1e-9 and abs(p["pts"][1][0] - 7.25) < 1e-9
           and abs(p["pts"][1][1] - 2.75) < 1e-9]
    assert len(sel) == 1
    return keys[sel[0]], paths[sel[0]]


def test_multi_diffraction_keller_law_and_minimum(oracle_mod):
    """Non-parallel edges: at each Keller point the incident and the diffracted leg make the same
    angle with the edge, the points lie on their edges, and moving either along its edge
    lengthens the path (the unfolded length is convex, its stationary point its minimum)."""
    O = oracle_mod
    tris, tx, rx = _crossed_edges()
    _, p = _crossed_path(O, tris, tx, rx, 28e9)
    T, R = np.array(tx, np.float64), np.array(rx, np.float64)
    Q1, Q2 = p["pts"][0].astype(np.float64), p["pts"][1].astype(np.float64)
    e1, e2 = np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0])
    assert abs(Q1[0] - 2.25) < 1e-12 and -15.5 < Q1[1] < -9.5
    assert 0.0 < Q2[2] < 7.5
    u = lambda v: v / np.linalg.norm(v)
    assert abs(u(Q1 - T) @ e1 - u(Q2 - Q1) @ e1) < 1e-10
    assert abs(u(Q2 - Q1) @ e2 - u(R - Q2) @ e2) < 1e-10
    length = lambda a, b: np.linalg.norm(a - T) + np.linalg.norm(b - a) + np.linalg.norm(R - b)
    L0 = length(Q1, Q2)
    assert abs(L0 - p["len_m"]) < 1e-9
    for d1 in (-1e-3, 0.0, 1e-3):
        for d2 in (-1e-3, 0.0, 1e-3):
            if d1 or d2:
                assert length(Q1 + d1 * e1, Q2 + d2 * e2) > L0


def test_multi_diffraction_reciprocal_at_high_frequency(oracle_mod):
    """Perfect conductors, non-parallel edges: swapping Tx and Rx gives the same path; the
    amplitudes differ only through the transition functions' arguments (the distance parameters
    of an astigmatic wave are not symmetric), an O(1/(kL)) effect, while the spreading of the
    astigmatic chain is reciprocal. So the relative difference falls as 1/f and is below 1e-4 at
    280 THz; a wrong caustic or principal direction would leave an O(1) mismatch."""
    O = oracle_mod
    tris, tx, rx = _crossed_edges()
    diffs = []
    for f in (2.8e12, 28e12, 280e12):
        ka, pa = _crossed_path(O, tris, tx, rx, f)
        sc = scenes._static_scene("boxes", tris, [scenes.MAT_METAL] * len(tris), rx, [tx])
        prm = O.OracleParams(freq_hz=f, max_refl=3)
        kb, pb = O.diffract_multi(sc.tris.reshape(-1, 9), sc.tri_mat, sc.tri_obj, sc.materials, sc.tx,
                                  sc.rx[0], prm, 2)
        j = [i for i, k in enumerate(kb) if k[2] == ka[3] and k[3] == ka[2]]
        assert len(j) == 1
        assert abs(pb["len_m"][j[0]] - pa["len_m"]) <= 1e-12 * pa["len_m"]
        a, b = complex(pa["amp_re"], pa["amp_im"]), complex(pb["amp_re"][j[0]], pb["amp_im"][j[0]])
        diffs.append(abs(a - b) / abs(a))
    assert diffs[2] < 1e-4
    assert 5.0 < diffs[0] / diffs[1] < 20.0 and 5.0 < diffs[1] / diffs[2] < 20.0


# ---------------------------------------------------------------------------
# one reflection before or after a chain of 2-3 wedges (image theory)
# ---------------------------------------------------------------------------
_GROUND = scenes._quad((-200.0, -200.0, 0.0), (200.0, -200.0, 0.0), (200.0, 200.0, 0.0), (-200.0, 200.0, 0.0))


def _two_walls():
    return _slab(0.0, 0.5, -50.0, 0.0) + _slab(10.0, 10.5, 5.0, 55.0)


def _prisms():
    out = []
    for a in np.deg2rad([60.0, 0.0, -60.0]):
        out += _prism(a)
    return out


def _at(deg, z):
    return (22.0 * np.cos(np.deg2rad(deg)), 22.0 * np.sin(np.deg2rad(deg)), z)


@pytest.mark.parametrize("mat", [scenes.MAT_METAL, scenes.MAT_CONCRETE])
@pytest.mark.parametrize("case", ["walls_first", "walls_last", "prisms_first", "prisms_last"])
def test_reflection_and_chain_is_the_image_chain(oracle_mod, mat, case):
    """Over a perfectly conducting ground and for vertical polarisation (the
    image of the vertically polarised transmitter is a vertically polarised
    transmitter), a ground reflection before a chain of wedges is the chain
    from the transmitter's image without the ground, and a reflection after it
    the chain toward the receiver's image: the same diffraction points,
    lengths and amplitudes (orders 2 and 3; the two walls and the three prisms
    of the composition pins, raised so the chain clears the ground)."""
    O = oracle_mod
    walls, m = (_two_walls(), 2) if case.startswith("walls") else (_prisms(), 3)
    first = case.endswith("first")
    if m == 2:
        tx, rx = ((-10.0, -20.0, 1.0), (20.0, 20.0, 9.0)) if first else ((-10.0, -20.0, 9.0), (20.0, 20.0, 1.0))
    else:
        tx, rx = (_at(120.0, 1.0), _at(-120.0, 9.0)) if first else (_at(120.0, 9.0), _at(-120.0, 1.0))
    prm = O.OracleParams(freq_hz=28e9, max_refl=3)
    tris = _GROUND + walls
    sc = scenes._static_scene("ground_walls", tris, [scenes.MAT_METAL] * 2 + [mat] * len(walls), tx, [rx])
    k, p = O.diffract_multi_refl(sc.tris.reshape(-1, 9), sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[0],
                                 prm, m)
    on_ground = [i for i, kk in enumerate(k) if (kk[2] if first else kk[2 + m]) < 2]
    src = (tx[0], tx[1], -tx[2]) if first else tx
    obs = rx if first else (rx[0], rx[1], -rx[2])
    b = scenes._static_scene("walls", walls, [mat] * len(walls), src, [obs])
    bk, bp = O.diffract_multi(b.tris.reshape(-1, 9), b.tri_mat, b.tri_obj, b.materials, b.tx, b.rx[0], prm, m)
    assert len(on_ground) == len(bk) == 1
    i = on_ground[0]
    wedges = list(k[i][3:3 + m]) if first else list(k[i][2:2 + m])
    assert wedges == list(bk[0][2:2 + m])
    q = p["pts"][i][1:1 + m] if first else p["pts"][i][0:m]
    assert np.max(np.abs(q - bp["pts"][0][:m])) <= 1e-9
    refl = p["pts"][i][0] if first else p["pts"][i][m]
    assert abs(refl[2]) <= 1e-9                      # the reflection point on the ground
    assert abs(p["len_m"][i] - bp["len_m"][0]) <= 1e-9 * bp["len_m"][0]
    a, b_ = complex(p["amp_re"][i], p["amp_im"][i]), complex(bp["amp_re"][0], bp["amp_im"][0])
    assert abs(a - b_) <= 1e-9 * abs(b_)


def test_reflection_and_chain_reciprocity(oracle_mod):
    """Perfect conductors, parallel edges: swapping Tx and Rx turns the
    reflection-first chain into the reflection-last chain over the same wedges
    in reverse order, with the same length and amplitude."""
    O = oracle_mod
    tx, rx = (-10.0, -20.0, 1.0), (20.0, 20.0, 9.0)
    prm = O.OracleParams(freq_hz=28e9, max_refl=3)
    walls = _two_walls()
    out = []
    for t, r in ((tx, rx), (rx, tx)):
        sc = scenes._static_scene("g", _GROUND + walls, [scenes.MAT_METAL] * (2 + len(walls)), t, [r])
        k, p = O.diffract_multi_refl(sc.tris.reshape(-1, 9), sc.tri_mat, sc.tri_obj, sc.materials, sc.tx,
                                     sc.rx[0], prm, 2)
        out.append({tuple(kk[2:5].tolist()): (complex(pp["amp_re"], pp["amp_im"]), float(pp["len_m"]))
                    for kk, pp in zip(k, p)})
    fwd, back = out
    assert len(fwd) >= 1 and len(fwd) == len(back)
    for (a0, a1, a2), (amp, length) in fwd.items():
        amp2, len2 = back[(a2, a1, a0)]
        assert abs(length - len2) <= 1e-9 * length
        assert abs(amp - amp2) <= 1e-9 * abs(amp)


# ---------------------------------------------------------------------------
# two reflections around a first-order diffraction
# ---------------------------------------------------------------------------
def _vwall(p0, p1, h=20.0):
    (x0, y0), (x1, y1) = p0, p1
    return scenes._quad((x0, y0, 0.0), (x1, y1, 0.0), (x1, y1, h), (x0, y0, h))


def _walls_and_tip():
    """Two vertical walls, along y = 25 (triangles 0-1) and along x + y = -20
    (triangles 2-3): their mirrors do not commute (the planes meet at 45
    degrees), and points whose coordinates are multiples of 0.5 keep that
    property. Then the prism pointing along +x, its tip at (20, 0) a sharp
    vertical wedge (triangles 4-9)."""
    return _vwall((-10.0, 25.0), (40.0, 25.0)) + _vwall((-45.0, 25.0), (5.0, -25.0)) + _prism(0.0)


_T2, _R2 = (14.0, 10.0, 1.5), (14.0, -10.0, 1.0)


def _mirror(x, tri):
    v = np.asarray(tri, np.float64)
    n = np.cross(v[1] - v[0], v[2] - v[0])
    n /= np.linalg.norm(n)
    x = np.asarray(x, np.float64)
    return x - 2.0 * np.dot(n, x - v[0]) * n


def _half(x):
    r = np.round(2.0 * x) / 2.0
    assert np.max(np.abs(r - x)) <= 1e-9
    return r


def _refl2(O, tris, mats, tx, rx):
    sc = scenes._static_scene("r2", tris, mats, tx, [rx])
    prm = O.OracleParams(freq_hz=28e9, max_refl=3)
    return O.diffract_refl2(sc.tris.reshape(-1, 9), sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[0], prm)


@pytest.mark.parametrize("mat", [scenes.MAT_METAL, scenes.MAT_CONCRETE])
def test_two_reflections_and_diffraction_are_the_image_diffraction(oracle_mod, mat):
    """Perfectly conducting vertical walls and vertical polarisation: a
    reflection maps the vertically polarised transmitter (receiver) to a
    vertically polarised image of opposite sign, so two reflections on the
    walls around a diffraction, both before it or one on each side, give the
    first-order diffraction of the prism alone from the transmitter's image
    (in the walls' planes in path order) toward the receiver's image (in the
    planes after the wedge, last first): the same diffraction point, length
    and amplitude. The two walls' mirrors do not commute, so an image built in
    the wrong order lands elsewhere."""
    O = oracle_mod
    tris = _walls_and_tip()
    mats = [scenes.MAT_METAL] * 4 + [mat] * (len(tris) - 4)
    k, p = _refl2(O, tris, mats, _T2, _R2)
    prm = O.OracleParams(freq_hz=28e9, max_refl=3)
    kinds = set()
    for kk, pp in zip(k, p):
        ids = kk[2:5].tolist()
        wi = [i for i, x in enumerate(ids) if x & O.DIFF][0]
        before, after = ids[:wi], ids[wi + 1:]
        if any(x >= 4 for x in before + after):
            continue
        src = np.asarray(_T2, np.float64)
        for j in before:
            src = _mirror(src, tris[j])
        obs = np.asarray(_R2, np.float64)
        for j in reversed(after):
            obs = _mirror(obs, tris[j])
        # exact in FP32: the images' coordinates are multiples of 0.5
        src, obs = _half(src), _half(obs)
        b = scenes._static_scene("tip", _prism(0.0), [mat] * 6, src, [obs])
        bk, bp = O.diffract(b.tris.reshape(-1, 9), b.tri_mat, b.tri_obj, b.materials, b.tx, b.rx[0], prm)
        q = pp["pts"][wi]
        j = [i for i in range(len(bk)) if np.max(np.abs(bp["pts"][i][0] - q)) <= 1e-9]
        assert len(j) == 1, (ids, len(bk))
        assert abs(bp["len_m"][j[0]] - pp["len_m"]) <= 1e-12 * pp["len_m"]
        a, b_ = complex(pp["amp_re"], pp["amp_im"]), complex(bp["amp_re"][j[0]], bp["amp_im"][j[0]])
        assert abs(a - b_) <= 1e-9 * abs(b_), ids
        kinds.add(wi)
    assert kinds == {1, 2}                  # one on each side, and both before


def test_two_reflections_and_diffraction_reciprocity(oracle_mod):
    """Perfect conductors: swapping Tx and Rx turns each path into the one over
    the same triangles and wedge in reverse order (two reflections before the
    wedge become two after it), with the same length and amplitude."""
    O = oracle_mod
    tris = _walls_and_tip()
    mats = [scenes.MAT_METAL] * len(tris)
    out = []
    for t, r in ((_T2, _R2), (_R2, _T2)):
        k, p = _refl2(O, tris, mats, t, r)
        out.append({tuple(kk[2:5].tolist()): (complex(pp["amp_re"], pp["amp_im"]), float(pp["len_m"]))
                    for kk, pp in zip(k, p)})
    fwd, back = out
    assert len(fwd) >= 3 and len(fwd) == len(back)
    assert {sum(1 for x in key[:[i for i, x in enumerate(key) if x & O.DIFF][0]]) for key in back} >= {0, 1}
    for key, (amp, length) in fwd.items():
        amp2, len2 = back[key[::-1]]
        assert abs(length - len2) <= 1e-9 * length
        assert abs(amp - amp2) <= 1e-9 * abs(amp)


@pytest.mark.parametrize("mat", [scenes.MAT_METAL, scenes.MAT_CONCRETE])
def test_two_reflections_and_diffraction_obey_the_laws(oracle_mod, mat):
    """Every path, the prism's faces among the reflectors too, checked point by
    point without image theory: a reflection point lies on its triangle (in
    its plane, inside it) and the outgoing leg is the mirror image of the
    incoming one; the diffraction point lies on an edge of the prism and the
    two legs make equal angles with it (Keller's cone); the length is the sum
    of the legs."""
    O = oracle_mod
    tris = _walls_and_tip()
    mats = [scenes.MAT_METAL] * 4 + [mat] * (len(tris) - 4)
    tv = np.asarray(tris, np.float64)
    edges = [(t[a], t[b]) for t in tv[4:] for a, b in ((0, 1), (1, 2), (2, 0))]
    for tx, rx in ((_T2, _R2), (_R2, _T2)):
        k, p = _refl2(O, tris, mats, tx, rx)
        assert len(k) >= 3
        for kk, pp in zip(k, p):
            ids = kk[2:5].tolist()
            X = [np.asarray(tx, np.float64)] + [pp["pts"][i] for i in range(3)] + [np.asarray(rx, np.float64)]
            legs = [np.linalg.norm(X[i + 1] - X[i]) for i in range(4)]
            assert abs(sum(legs) - pp["len_m"]) <= 1e-9 * pp["len_m"]
            for i, tid in enumerate(ids):
                A, Y, B = X[i], X[i + 1], X[i + 2]
                din, dout = (Y - A) / legs[i], (B - Y) / legs[i + 1]
                if tid & O.DIFF:
                    hit = [(e0, e1) for e0, e1 in edges
                           if np.linalg.norm(np.cross(e1 - e0, Y - e0)) <= 1e-9 * np.linalg.norm(e1 - e0)]
                    assert hit, ids
                    e = (hit[0][1] - hit[0][0]) / np.linalg.norm(hit[0][1] - hit[0][0])
                    assert abs(np.dot(din, e) - np.dot(dout, e)) <= 1e-9
                else:
                    v = tv[tid]
                    n = np.cross(v[1] - v[0], v[2] - v[0])
                    n /= np.linalg.norm(n)
                    assert abs(np.dot(n, Y - v[0])) <= 1e-9
                    for a in range(3):
                        assert np.dot(np.cross(v[(a + 1) % 3] - v[a], Y - v[a]), n) >= -1e-9
                    assert np.max(np.abs(dout - (din - 2.0 * np.dot(din, n) * n))) <= 1e-9


def test_given_path_equals_the_enumerated_one(oracle_mod):
    """or_diffract_path evaluates a given combined path (the check of paths
    found elsewhere): every path the enumerations find, from two reflections
    around a wedge to one reflection around a chain, comes out identical, and
    ids that are not such a path are refused."""
    O = oracle_mod
    tris = _walls_and_tip()
    mats = [scenes.MAT_METAL] * 4 + [scenes.MAT_CONCRETE] * (len(tris) - 4)
    sc = scenes._static_scene("r2", tris, mats, _T2, [_R2])
    prm = O.OracleParams(freq_hz=28e9, max_refl=4)
    wt = sc.tris.reshape(-1, 9)
    found = [O.diffract_refl2(wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[0], prm),
             O.diffract_refl(wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[0], prm)]
    n = 0
    for exact, (k, p) in zip((True, False), found):
        for kk, pp in zip(k, p):
            ids = [int(x) for x in kk[2:2 + kk[1]]]
            q = O.diffract_path(wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[0][0], ids, prm)
            assert q is not None, ids
            if exact:  # the same computation
                assert q.tobytes() == pp.tobytes(), ids
            else:  # or_diffract_refl takes the first-order Keller point in closed form
                assert abs(q["len_m"] - pp["len_m"]) <= 1e-12 * pp["len_m"]
                za, zb = complex(q["amp_re"], q["amp_im"]), complex(pp["amp_re"], pp["amp_im"])
                assert abs(za - zb) <= 1e-9 * abs(zb), ids
            n += 1
    assert n >= 5
    # a reflection between two wedges
    tris2 = _GROUND + _ridge(0.0, 2.0, 10.0) + _ridge(8.0, 2.0, 10.0)
    sc2 = scenes._static_scene("mid", tris2, [scenes.MAT_CONCRETE] * len(tris2), _TM, [_RM])
    km, pm = O.diffract_mid(sc2.tris.reshape(-1, 9), sc2.tri_mat, sc2.tri_obj, sc2.materials, sc2.tx, sc2.rx[0],
                            prm)
    assert len(km) == 1
    q = O.diffract_path(sc2.tris.reshape(-1, 9), sc2.tri_mat, sc2.tri_obj, sc2.materials, sc2.tx, sc2.rx[0][0],
                        [int(x) for x in km[0][2:5]], prm)
    assert q is not None and q.tobytes() == pm[0].tobytes()
    D = O.DIFF
    with pytest.raises(ValueError):
        O.diffract_path(wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[0][0], [0, 2, 3], prm)
    with pytest.raises(ValueError):
        O.diffract_path(wt, sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[0][0], [0, 1 | D, 2, 3], prm)


# ---------------------------------------------------------------------------
# a reflection between two diffractions
# ---------------------------------------------------------------------------
def _ridge(xc, w, h, y0=-20.0, y1=20.0):
    """A horizontal triangular prism along y on the ground: base from xc - w to
    xc + w, its ridge (a wedge of about 23 degrees) at height h."""
    a, b, c = (xc - w, 0.0), (xc, h), (xc + w, 0.0)
    out = scenes._quad((a[0], y0, a[1]), (b[0], y0, b[1]), (b[0], y1, b[1]), (a[0], y1, a[1]))
    out += scenes._quad((b[0], y0, b[1]), (c[0], y0, c[1]), (c[0], y1, c[1]), (b[0], y1, b[1]))
    out += [[(a[0], y0, a[1]), (c[0], y0, c[1]), (b[0], y0, b[1])],
            [(a[0], y1, a[1]), (b[0], y1, b[1]), (c[0], y1, c[1])]]
    return out


_TM, _RM = (-30.0, -3.0, 1.0), (38.0, 5.0, 1.5)


def _mid(O, tris, mats, tx, rx):
    sc = scenes._static_scene("mid", tris, mats, tx, [rx])
    prm = O.OracleParams(freq_hz=28e9, max_refl=3)
    return O.diffract_mid(sc.tris.reshape(-1, 9), sc.tri_mat, sc.tri_obj, sc.materials, sc.tx, sc.rx[0], prm)


@pytest.mark.parametrize("mat", [scenes.MAT_METAL, scenes.MAT_CONCRETE])
def test_reflection_between_wedges_is_the_image_chain(oracle_mod, mat):
    """Two ridges on a perfectly conducting ground, vertical polarisation: the
    path over the first ridge, the ground and the second ridge is, by image
    theory, the order-2 chain over the first ridge and the second ridge's
    image below the ground (with no ground) toward the receiver's image (a
    vertically polarised receiver's image is vertically polarised): the same
    diffraction points (the second mirrored), length and amplitude; the
    reflection point on the ground between the ridges."""
    O = oracle_mod
    r1, r2 = _ridge(0.0, 2.0, 10.0), _ridge(8.0, 2.0, 10.0)
    tris = _GROUND + r1 + r2
    k, p = _mid(O, tris, [scenes.MAT_METAL] * 2 + [mat] * (len(tris) - 2), _TM, _RM)
    assert len(k) == 1 and k[0][3] < 2                     # the reflection on the ground
    q1, pg, q2 = p["pts"][0][:3]
    assert abs(pg[2]) <= 1e-12 and 2.0 < pg[0] < 6.0
    img = r1 + [[(x, y, -z) for (x, y, z) in t] for t in r2]
    rm = (_RM[0], _RM[1], -_RM[2])
    b = scenes._static_scene("image", img, [mat] * len(img), _TM, [rm])
    prm = O.OracleParams(freq_hz=28e9, max_refl=3)
    bk, bp = O.diffract_multi(b.tris.reshape(-1, 9), b.tri_mat, b.tri_obj, b.materials, b.tx, b.rx[0], prm, 2)
    q2m = np.array([q2[0], q2[1], -q2[2]])
    j = [i for i in range(len(bk)) if np.max(np.abs(bp["pts"][i][0] - q1)) <= 1e-9
         and np.max(np.abs(bp["pts"][i][1] - q2m)) <= 1e-9]
    assert len(j) == 1
    assert abs(bp["len_m"][j[0]] - p["len_m"][0]) <= 1e-12 * p["len_m"][0]
    a, b_ = complex(p["amp_re"][0], p["amp_im"][0]), complex(bp["amp_re"][j[0]], bp["amp_im"][j[0]])
    assert abs(a - b_) <= 1e-9 * abs(b_)


def test_reflection_between_wedges_reciprocity(oracle_mod):
    """Perfect conductors: swapping Tx and Rx gives the path over the same
    wedges and triangle in reverse order, with the same length and amplitude."""
    O = oracle_mod
    tris = _GROUND + _ridge(0.0, 2.0, 10.0) + _ridge(8.0, 2.0, 10.0)
    mats = [scenes.MAT_METAL] * len(tris)
    (kf, pf), (kb, pb) = _mid(O, tris, mats, _TM, _RM), _mid(O, tris, mats, _RM, _TM)
    assert len(kf) == len(kb) == 1
    assert list(kf[0][2:5]) == list(kb[0][2:5])[::-1]
    assert abs(pf["len_m"][0] - pb["len_m"][0]) <= 1e-9 * pf["len_m"][0]
    a, b = complex(pf["amp_re"][0], pf["amp_im"][0]), complex(pb["amp_re"][0], pb["amp_im"][0])
    assert abs(a - b) <= 1e-9 * abs(a)


@pytest.mark.parametrize("mat", [scenes.MAT_METAL, scenes.MAT_CONCRETE])
def test_reflection_between_wedges_obeys_the_laws(oracle_mod, mat):
    """Without image theory, on a concrete ground: the reflection point lies on
    the ground and the outgoing leg is the mirror image of the incoming one;
    each diffraction point lies on its ridge and its two legs make equal
    angles with it; the length is the sum of the four legs."""
    O = oracle_mod
    tris = _GROUND + _ridge(0.0, 2.0, 10.0) + _ridge(8.0, 2.0, 10.0)
    k, p = _mid(O, tris, [scenes.MAT_CONCRETE] * 2 + [mat] * (len(tris) - 2), _TM, _RM)
    assert len(k) == 1
    X = [np.asarray(_TM, np.float64)] + [p["pts"][0][i] for i in range(3)] + [np.asarray(_RM, np.float64)]
    legs = [np.linalg.norm(X[i + 1] - X[i]) for i in range(4)]
    assert abs(sum(legs) - p["len_m"][0]) <= 1e-9 * p["len_m"][0]
    e = np.array([0.0, 1.0, 0.0])
    for i in (1, 3):  # the ridges run along y
        din, dout = (X[i] - X[i - 1]) / legs[i - 1], (X[i + 1] - X[i]) / legs[i]
        assert abs(X[i][2] - 10.0) <= 1e-9
        assert abs(np.dot(din, e) - np.dot(dout, e)) <= 1e-9
    din, dout = (X[2] - X[1]) / legs[1], (X[3] - X[2]) / legs[2]
    assert abs(X[2][2]) <= 1e-12
    assert np.max(np.abs(dout - din * np.array([1.0, 1.0, -1.0]))) <= 1e-9
