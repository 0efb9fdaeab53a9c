"""Helpers that compare the CUDA path (through the C ABI) with the oracle."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from paper_2112_07115_gb300 import dcem

RAY_FLAGS = O.RAY_FLAGS
PATH_FLAGS = O.PATH_FLAGS


def oracle_params(sc, n_rays=None, **kw):
    kw.setdefault("max_refl", sc.max_refl)
    return O.OracleParams(freq_hz=sc.freq_hz, n_rays=n_rays or sc.n_rays, **kw)


def gpu_params(sc, **kw):
    kw.setdefault("max_refl", sc.max_refl)
    kw.setdefault("freq_hz", sc.freq_hz)
    return dcem.default_params(**kw)


def path_keys(paths, max_refl):
    """Keys (rx, depth, ids..., -1 padded) of GPU path records."""
    out = []
    for p in paths:
        k = int(p["depth"])
        ids = [int(x) for x in p["tri"][:k]] + [-1] * (max_refl - k)
        out.append((int(p["rx"]), k, *ids))
    return out


def compare_hits(gpu_ids, gpu_nseg, ref_tr):
    """Per-ray hit ids per segment, unflagged rays only. Returns
    (compared, flagged, mismatching ray indices)."""
    flagged = (ref_tr["flags"] & RAY_FLAGS) != 0
    ok = ~flagged
    same = np.all(gpu_ids == ref_tr["hit_id"], axis=1) & (gpu_nseg == ref_tr["nseg"])
    bad = np.nonzero(ok & ~same)[0]
    return int(ok.sum()), int(flagged.sum()), bad


def compare_candidates(gpu_cands, ref_tr):
    """Captures (ray, seg, rx) of unflagged rays must be identical."""
    flagged = (ref_tr["flags"] & RAY_FLAGS) != 0
    def keep(c):
        c = np.asarray(c).reshape(-1, 3)
        return {tuple(x) for x in c.tolist() if not flagged[x[0]]}
    g, r = keep(gpu_cands), keep(ref_tr["cands"])
    return g, r


def compare_paths(frame, ref, max_refl, len_tol=1e-6, amp_rtol=1e-6):
    """GPU valid paths vs the oracle's validated keys. Keys discovered by an
    unflagged ray and not flagged in validation must agree in validity, and
    valid ones in length and amplitude. Returns a dict of findings.
    max_refl: the key width (reflections plus transmissions per path).
    Both sides compute the path geometry, the Fresnel coefficients, the
    polarisation and the phase in FP64 from the same FP32 vertices, so a
    length agrees to rounding (1e-9 m at 1 km) and an amplitude to the phase
    error k * dL (6e-7 rad at 28 GHz for dL = 1e-9 m): amp_rtol = 1e-6."""
    flagged = (ref.tr["flags"] & RAY_FLAGS) != 0
    ckeys = O.candidate_keys(ref.tr["cands"], ref.tr["hit_id"], max_refl)
    clean = {tuple(k) for k, c in zip(ckeys.tolist(), ref.tr["cands"].tolist()) if not flagged[c[0]]}
    ref_rec = {tuple(k): p for k, p in zip(ref.keys.tolist(), ref.paths)}
    gpu = dict(zip(path_keys(frame.paths, max_refl), frame.paths))
    out = {"missing": [], "extra": [], "len": [], "amp": [], "checked": 0}
    for key in clean:
        rp = ref_rec[key]
        if rp["flags"] & PATH_FLAGS:
            continue
        out["checked"] += 1
        gv = key in gpu
        if bool(rp["valid"]) != gv:
            (out["missing"] if rp["valid"] else out["extra"]).append(key)
            continue
        if gv:
            gp = gpu[key]
            if abs(gp["len_m"] - rp["len_m"]) > len_tol:
                out["len"].append((key, gp["len_m"], rp["len_m"]))
            za = complex(gp["amp_re"], gp["amp_im"])
            zb = complex(rp["amp_re"], rp["amp_im"])
            if abs(za - zb) > amp_rtol * abs(zb):
                out["amp"].append((key, za, zb))
    return out


def power_close(a_dbm, b_dbm, tol_db=0.01):
    a, b = np.asarray(a_dbm), np.asarray(b_dbm)
    both_inf = np.isneginf(a) & np.isneginf(b)
    with np.errstate(invalid="ignore"):
        return both_inf | (np.abs(a - b) <= tol_db)
