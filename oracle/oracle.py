"""Python driver of the FP64 CPU oracle (``dcem_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, the smoke check and the
benchmark's CPU-baseline leg, never by the product path. It shares no code
with the CUDA library; both consume the FP32 arrays of the seeded input
generators.

Pipeline of one frame (arXiv 2112.07115, Sec. III):
  transform   -> world-space vertices of moving objects (per-frame update)
  trace       -> step 1-2: sampled-sphere shooting with up to N specular
                 reflections, closest hit by brute force over all triangles,
                 reception-sphere captures
  dedupe      -> step 2: the set of distinct (receiver, depth, triangle
                 sequence) keys ("hash table of visited propagation paths for
                 each depth"), here simply sorted and made unique
  validate    -> steps 3-4, 6: image receivers, back-trace, point-in-triangle,
                 occlusion; length, delay, Fresnel TE/TM, complex amplitude
  reduce      -> received power per receiver: coherent P_t |sum a|^2 and
                 incoherent P_t sum |a|^2 in dBm, summed in sorted key order.
  diffract    -> step 5, first order: edge diffraction paths with the UTD
                 coefficient (Kouyoumjian & Pathak 1974; Luebbers 1984).
  sticky      -> the path cache's literal retention (Sec. III "Propagation
                 path caching", cached paths kept and updated until removed):
                 a frame's keys are the ones its rays capture plus every key
                 valid in the previous frame, all validated anew.
  gradient    -> derivatives of the per-receiver field over a fixed path
                 topology with respect to each material's (eps_r, sigma) and
                 each rigid object's (x, y) translation, by FP64 central
                 differences of the same amplitude computation (without the
                 occlusion test, since the paths are given).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# The mutation test (tests/test_oracle_mutations.py) points these at a copy of
# the source with one planted mistake and at a build folder of its own.
_SRC = os.environ.get("DCEM_ORACLE_SRC") or os.path.join(_HERE, "dcem_oracle.c")
_BUILD = os.environ.get("DCEM_ORACLE_BUILD") or os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libdcem_oracle.so")

MAX_REFL = 10
C0 = 299792458.0

# flag bits (mirror the C definitions of this oracle)
NEAR_EDGE, TIE, NEAR_TMIN, NEAR_SPHERE = 1, 2, 4, 8
VAL_EDGE, VAL_PARAM, OCC_NEAR, POL_DEGEN = 16, 32, 64, 128
RAY_FLAGS = NEAR_EDGE | TIE | NEAR_TMIN | NEAR_SPHERE
PATH_FLAGS = VAL_EDGE | VAL_PARAM | OCC_NEAR


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
                        "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("freq_hz", C.c_double), ("tx_power_w", C.c_double), ("alpha", C.c_double),
                ("rx_radius_scale", C.c_double), ("t_min", C.c_double),
                ("escape_len", C.c_double), ("eps_occ", C.c_double), ("edge_eps", C.c_double),
                ("val_eps", C.c_double), ("pol", C.c_double * 3), ("max_refl", C.c_int32),
                ("nthreads", C.c_int32), ("trans_db", C.c_void_p), ("max_trans", C.c_int32),
                ("pad_", C.c_int32)]


TRANS = 0x40000000   # interaction id flag: transmission through the triangle
DIFF = 0x20000000    # interaction id flag: diffraction at the wedge of that index
MAX_SEG = MAX_REFL + 1
INST_DTYPE = np.dtype([("root", np.int32), ("start", np.int32), ("nseg", np.int32), ("flags", np.uint32),
                       ("hit", np.int32, (MAX_SEG,)), ("t", np.float64, (MAX_SEG,))], align=True)


PATH_DTYPE = np.dtype([("valid", np.int32), ("flags", np.uint32), ("len_m", np.float64),
                       ("delay_s", np.float64), ("amp_re", np.float64), ("amp_im", np.float64),
                       ("pts", np.float64, (MAX_REFL, 3))])

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER
        f32, i32, f64, u32 = P(C.c_float), P(C.c_int32), P(C.c_double), P(C.c_uint32)
        _lib.or_transform.argtypes = [C.c_int32, f32, i32, f32, C.c_int32, f32]
        _lib.or_transform.restype = None
        _lib.or_trace.argtypes = [f32, i32, C.c_int32, f32, C.c_int32, f32, f32, C.c_int32, f32,
                                  C.c_int32, P(_Params), i32, f64, i32, u32, f64,
                                  P(P(C.c_int32)), P(C.c_int64)]
        _lib.or_trace.restype = C.c_int
        _lib.or_validate.argtypes = [f32, i32, C.c_int32, f32, C.c_int32, f32, f32, C.c_int32,
                                     i32, C.c_int64, P(_Params), C.c_void_p]
        _lib.or_validate.restype = C.c_int
        _lib.or_exhaustive.argtypes = [f32, i32, C.c_int32, f32, C.c_int32, f32, f32, C.c_int32,
                                       P(_Params), i32, C.c_void_p, C.c_int64]
        _lib.or_exhaustive.restype = C.c_int64
        _lib.or_path_amp_d.argtypes = [f64, i32, C.c_int32, f64, C.c_int32, f64, f64, C.c_int32,
                                       i32, C.c_int64, P(_Params), C.c_void_p]
        _lib.or_path_amp_d.restype = C.c_int
        _lib.or_fresnel.argtypes = [C.c_double, C.c_double, C.c_int32, C.c_double, C.c_double, f64]
        _lib.or_fresnel64.argtypes = [C.c_double, C.c_double, C.c_int32, C.c_double, C.c_double, f64]
        _lib.or_free.argtypes = [C.c_void_p]
        _lib.or_path_size.restype = C.c_int32
        assert _lib.or_path_size() == PATH_DTYPE.itemsize, "path record layout mismatch"
        _lib.or_trace_tree.argtypes = [f32, i32, C.c_int32, f32, C.c_int32, f32, f32, C.c_int32, f32,
                                       C.c_int32, P(_Params), P(C.c_void_p), P(C.c_int64),
                                       P(P(C.c_int32)), P(C.c_int64)]
        _lib.or_trace_tree.restype = C.c_int
        _lib.or_inst_size.restype = C.c_int32
        assert _lib.or_inst_size() == INST_DTYPE.itemsize, "instance record layout mismatch"
        _lib.or_transition.argtypes = [C.c_double, f64]
        _lib.or_transition.restype = None
        _lib.or_keller_points.argtypes = [C.c_int32, f64, f64, f64, f64]
        _lib.or_keller_points.restype = C.c_int
        _lib.or_utd.argtypes = [C.c_double] * 6 + [f64, f64, f64]
        _lib.or_utd.restype = None
        _lib.or_count_wedges.argtypes = [f32, i32, C.c_int32]
        _lib.or_count_wedges.restype = C.c_int32
        _lib.or_diffract.argtypes = [f32, i32, i32, C.c_int32, f32, C.c_int32, f32, f32, C.c_int32,
                                     P(_Params), C.c_int32, i32, C.c_void_p, C.c_int64]
        _lib.or_diffract.restype = C.c_int64
        _lib.or_diffract_trans.argtypes = [f32, i32, i32, C.c_int32, f32, C.c_int32, f32, f32, C.c_int32,
                                           P(_Params), C.c_int32, i32, C.c_void_p, C.c_int64]
        _lib.or_diffract_trans.restype = C.c_int64
        _lib.or_diffract_multi_trans.argtypes = [f32, i32, i32, C.c_int32, f32, C.c_int32, f32, f32, C.c_int32,
                                                 P(_Params), C.c_int32, C.c_int32, i32, C.c_void_p, C.c_int64]
        _lib.or_diffract_multi_trans.restype = C.c_int64
        _lib.or_diffract_refl.argtypes = [f32, i32, i32, C.c_int32, f32, C.c_int32, f32, f32, C.c_int32,
                                          P(_Params), C.c_int32, i32, C.c_void_p, C.c_int64]
        _lib.or_diffract_refl.restype = C.c_int64
        _lib.or_diffract_multi.argtypes = [f32, i32, i32, C.c_int32, f32, C.c_int32, f32, f32, C.c_int32,
                                           P(_Params), C.c_int32, C.c_int32, i32, C.c_void_p, C.c_int64]
        _lib.or_diffract_multi.restype = C.c_int64
        _lib.or_diffract_multi_refl.argtypes = [f32, i32, i32, C.c_int32, f32, C.c_int32, f32, f32, C.c_int32,
                                                P(_Params), C.c_int32, C.c_int32, i32, C.c_void_p, C.c_int64]
        _lib.or_diffract_multi_refl.restype = C.c_int64
        _lib.or_diffract_refl2.argtypes = [f32, i32, i32, C.c_int32, f32, C.c_int32, f32, f32, C.c_int32,
                                           P(_Params), C.c_int32, i32, C.c_void_p, C.c_int64]
        _lib.or_diffract_refl2.restype = C.c_int64
        _lib.or_diffract_mid.argtypes = [f32, i32, i32, C.c_int32, f32, C.c_int32, f32, f32, C.c_int32,
                                         P(_Params), C.c_int32, i32, C.c_void_p, C.c_int64]
        _lib.or_diffract_mid.restype = C.c_int64
        _lib.or_diffract_path.argtypes = [f32, i32, i32, C.c_int32, f32, C.c_int32, f32, f32, i32, C.c_int32,
                                          P(_Params), C.c_void_p]
        _lib.or_diffract_path.restype = C.c_int32
    return _lib


@dataclass
class OracleParams:
    """Tracer parameters (defaults: Sec. III -- 5 W transmit power, isotropic
    antennas; readings: vertical polarisation reference, capture radius
    1.35 * alpha * (D+s)/sqrt(3), self-hit offset 1e-4 m)."""
    freq_hz: float = 28e9
    tx_power_w: float = 5.0
    n_rays: int = 10_000
    max_refl: int = 3
    rx_radius_scale: float = 1.35
    t_min: float = 1e-4
    escape_len: float = 1e4
    eps_occ: float = 1e-4
    edge_eps: float = 1e-5
    val_eps: float = 1e-9
    pol: tuple = (0.0, 0.0, 1.0)
    nthreads: int = 0
    max_trans: int = 0          # transmissions per path (Table II penetration)
    trans_db: tuple = ()        # per material penetration loss [dB], < 0 opaque
    diffraction: bool = False   # first-order edge diffraction paths (UTD)
    diffraction_order: int = 1  # with diffraction: paths over up to this many wedges (1-3)

    @property
    def width(self) -> int:
        """Most interactions of a path (reflections + transmissions): key width."""
        return self.max_refl + (self.max_trans if self.transmission else 0)

    @property
    def transmission(self) -> bool:
        return self.max_trans > 0 and any(x >= 0 for x in self.trans_db)

    def c(self) -> _Params:
        p = _Params()
        p.freq_hz = self.freq_hz
        p.tx_power_w = self.tx_power_w
        p.alpha = float(np.sqrt(4.0 * np.pi / max(self.n_rays, 1)))
        p.rx_radius_scale = self.rx_radius_scale
        p.t_min = self.t_min
        p.escape_len = self.escape_len
        p.eps_occ = self.eps_occ
        p.edge_eps = self.edge_eps
        p.val_eps = self.val_eps
        for i in range(3):
            p.pol[i] = self.pol[i]
        p.max_refl = self.max_refl
        p.nthreads = self.nthreads
        if self.transmission:
            self._trans = np.ascontiguousarray(self.trans_db, np.float64)
            p.trans_db = self._trans.ctypes.data
            p.max_trans = self.max_trans
        else:
            p.trans_db = None
            p.max_trans = 0
        return p


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def transform(tris: np.ndarray, tri_obj: np.ndarray, xf: np.ndarray) -> np.ndarray:
    """World-space vertices: static triangles copied, object triangles mapped by
    their object's row-major 3x4 transform with fmaf(R0,x,fmaf(R1,y,fmaf(R2,z,t)))."""
    tris = _f32(tris).reshape(-1, 9)
    out = np.empty_like(tris)
    xf = _f32(xf).reshape(-1)
    nobj = xf.size // 12
    lib().or_transform(tris.shape[0], _p(tris, C.c_float), _p(_i32(tri_obj), C.c_int32),
                       _p(xf if xf.size else np.zeros(12, np.float32), C.c_float), nobj,
                       _p(out, C.c_float))
    return out.reshape(-1, 3, 3)


def trace(world_tris, tri_mat, materials, tx, rays, rx, prm: OracleParams, seg_od=False):
    """Step 1-2 over every ray. Returns a dict with per-ray hit ids per segment
    (-1 escaped, -2 not reached), hit distances, segment counts, flag bits and
    the captures (ray, segment, receiver), sorted. With transmission the rows
    are ray instances (the primaries, then their children, see trace_tree)."""
    if prm.transmission:
        return trace_tree(world_tris, tri_mat, materials, tx, rays, rx, prm)
    wt = _f32(world_tris).reshape(-1, 9)
    mats = _f32(materials).reshape(-1, 3)
    rays = _f32(rays).reshape(-1, 3)
    rx = _f32(rx).reshape(-1, 3)
    n, W = rays.shape[0], prm.max_refl + 1
    hit_id = np.empty((n, W), np.int32)
    hit_t = np.empty((n, W), np.float64)
    nseg = np.empty(n, np.int32)
    flags = np.empty(n, np.uint32)
    od = np.empty((n, W, 7), np.float64) if seg_od else None
    cptr = C.POINTER(C.c_int32)()
    ncand = C.c_int64(0)
    prm_c = prm.c()
    rc = lib().or_trace(_p(wt, C.c_float), _p(_i32(tri_mat), C.c_int32), wt.shape[0],
                        _p(mats, C.c_float), mats.shape[0], _p(_f32(tx), C.c_float),
                        _p(rays, C.c_float), n, _p(rx, C.c_float), rx.shape[0], C.byref(prm_c),
                        _p(hit_id, C.c_int32), _p(hit_t, C.c_double), _p(nseg, C.c_int32),
                        _p(flags, C.c_uint32), _p(od, C.c_double) if od is not None else None,
                        C.byref(cptr), C.byref(ncand))
    m = int(ncand.value)
    cands = np.ctypeslib.as_array(cptr, shape=(max(m, 1) * 3,))[:m * 3].reshape(m, 3).copy()
    lib().or_free(C.cast(cptr, C.c_void_p))
    if rc != 0:
        raise RuntimeError(f"or_trace failed: {rc}")
    out = {"hit_id": hit_id, "hit_t": hit_t, "nseg": nseg, "flags": flags, "cands": cands}
    if od is not None:
        out["seg_od"] = od
    return out


def trace_tree(world_tris, tri_mat, materials, tx, rays, rx, prm: OracleParams):
    """Steps 1-2 with transmission (Sec. III "Reflected and transmitted
    rays"): a ray hitting a transmitting material both reflects and spawns a
    child continuing straight through, up to max_refl reflections and
    max_trans transmissions per path. Rows: the n primary instances (row i =
    ray i) then the children by (root ray, spawn order); hit ids carry TRANS
    on transmissions and include each child's inherited prefix. Adds "root"
    (sampled direction of each row) and "start" (first segment it traced)."""
    wt = _f32(world_tris).reshape(-1, 9)
    mats = _f32(materials).reshape(-1, 3)
    rays = _f32(rays).reshape(-1, 3)
    rx = _f32(rx).reshape(-1, 3)
    n, W = rays.shape[0], prm.width + 1
    iptr, ni = C.c_void_p(), C.c_int64(0)
    cptr, ncand = C.POINTER(C.c_int32)(), C.c_int64(0)
    prm_c = prm.c()
    rc = lib().or_trace_tree(_p(wt, C.c_float), _p(_i32(tri_mat), C.c_int32), wt.shape[0],
                             _p(mats, C.c_float), mats.shape[0], _p(_f32(tx), C.c_float),
                             _p(rays, C.c_float), n, _p(rx, C.c_float), rx.shape[0], C.byref(prm_c),
                             C.byref(iptr), C.byref(ni), C.byref(cptr), C.byref(ncand))
    k, m = int(ni.value), int(ncand.value)
    buf = (C.c_char * (max(k, 1) * INST_DTYPE.itemsize)).from_address(iptr.value)
    inst = np.frombuffer(bytes(buf), INST_DTYPE, count=k).copy() if k else np.zeros(0, INST_DTYPE)
    cands = np.ctypeslib.as_array(cptr, shape=(max(m, 1) * 3,))[:m * 3].reshape(m, 3).copy()
    lib().or_free(iptr)
    lib().or_free(C.cast(cptr, C.c_void_p))
    if rc != 0:
        raise RuntimeError(f"or_trace_tree failed: {rc}")
    return {"hit_id": inst["hit"][:, :W].copy(), "hit_t": inst["t"][:, :W].copy(), "nseg": inst["nseg"].copy(),
            "flags": inst["flags"].copy(), "cands": cands, "root": inst["root"].copy(),
            "start": inst["start"].copy()}


def candidate_keys(cands: np.ndarray, hit_id: np.ndarray, max_refl: int) -> np.ndarray:
    """Key rows (rx, depth, tri ids of bounces 1..depth, -1 padding) of each capture."""
    m = cands.shape[0]
    keys = np.full((m, 2 + max_refl), -1, np.int32)
    keys[:, 0] = cands[:, 2]
    keys[:, 1] = cands[:, 1]
    for j in range(max_refl):
        sel = cands[:, 1] > j
        keys[sel, 2 + j] = hit_id[cands[sel, 0], j]
    return keys


def unique_keys(keys: np.ndarray) -> np.ndarray:
    """Distinct key rows in lexicographic (rx, depth, ids...) order."""
    if keys.shape[0] == 0:
        return keys.copy()
    return np.unique(keys, axis=0)


def validate(world_tris, tri_mat, materials, tx, rx, keys, prm: OracleParams) -> np.ndarray:
    """Steps 3-4, 6 for every key row; returns PATH_DTYPE records (valid or not)."""
    wt = _f32(world_tris).reshape(-1, 9)
    mats = _f32(materials).reshape(-1, 3)
    rx = _f32(rx).reshape(-1, 3)
    keys = _i32(keys).reshape(-1, 2 + prm.width)
    out = np.zeros(keys.shape[0], PATH_DTYPE)
    prm_c = prm.c()
    rc = lib().or_validate(_p(wt, C.c_float), _p(_i32(tri_mat), C.c_int32), wt.shape[0],
                           _p(mats, C.c_float), mats.shape[0], _p(_f32(tx), C.c_float),
                           _p(rx, C.c_float), rx.shape[0], _p(keys, C.c_int32), keys.shape[0],
                           C.byref(prm_c), out.ctypes.data_as(C.c_void_p))
    if rc != 0:
        raise RuntimeError(f"or_validate failed: {rc}")
    return out


def exhaustive(world_tris, tri_mat, materials, tx, rx, prm: OracleParams, cap=1 << 20):
    """All valid paths of depth <= N by enumerating every triangle sequence."""
    wt = _f32(world_tris).reshape(-1, 9)
    mats = _f32(materials).reshape(-1, 3)
    rx = _f32(rx).reshape(-1, 3)
    stride = 2 + prm.width
    keys = np.zeros((cap, stride), np.int32)
    paths = np.zeros(cap, PATH_DTYPE)
    prm_c = prm.c()
    n = lib().or_exhaustive(_p(wt, C.c_float), _p(_i32(tri_mat), C.c_int32), wt.shape[0],
                            _p(mats, C.c_float), mats.shape[0], _p(_f32(tx), C.c_float),
                            _p(rx, C.c_float), rx.shape[0], C.byref(prm_c),
                            _p(keys, C.c_int32), paths.ctypes.data_as(C.c_void_p), cap)
    if n < 0:
        raise RuntimeError(f"or_exhaustive failed: {n}")
    if n > cap:
        raise RuntimeError(f"or_exhaustive: {n} paths exceed capacity {cap}")
    return keys[:n].copy(), paths[:n].copy()


def fresnel(eps_r, sigma, pec, freq_hz, cos_t, exact=False):
    """(Gamma_TE, Gamma_TM) as complex numbers."""
    out = np.zeros(4)
    f = lib().or_fresnel64 if exact else lib().or_fresnel
    f(eps_r, sigma, int(pec), freq_hz, cos_t, _p(out, C.c_double))
    return complex(out[0], out[1]), complex(out[2], out[3])


def dbm(p_w):
    with np.errstate(divide="ignore"):
        return 10.0 * np.log10(np.asarray(p_w, np.float64)) + 30.0


def reduce(keys: np.ndarray, paths: np.ndarray, nrx: int, tx_power_w: float):
    """Per receiver: complex field sum a (FP64, in the given key order -- callers
    pass keys sorted lexicographically), P_coh = P_t|sum a|^2 and
    P_inc = P_t sum|a|^2 in dBm."""
    field = np.zeros(nrx, np.complex128)
    inc = np.zeros(nrx, np.float64)
    for i in range(keys.shape[0]):
        if not paths["valid"][i]:
            continue
        r = int(keys[i, 0])
        a = complex(paths["amp_re"][i], paths["amp_im"][i])
        field[r] += a
        inc[r] += abs(a) ** 2
    return field, dbm(tx_power_w * np.abs(field) ** 2), dbm(tx_power_w * inc)


def path_amp_d(tris, tri_mat, materials, tx, rx, keys, prm: OracleParams) -> np.ndarray:
    """Steps 3, 4 and 6 for fixed triangle sequences with FP64 vertices,
    materials, Tx and receivers, without the occlusion test (the topology is
    given): PATH_DTYPE records whose ``valid`` is the geometric validity."""
    wt = np.ascontiguousarray(tris, np.float64).reshape(-1, 9)
    mats = np.ascontiguousarray(materials, np.float64).reshape(-1, 3)
    rx = np.ascontiguousarray(rx, np.float64).reshape(-1, 3)
    keys = _i32(keys).reshape(-1, 2 + prm.max_refl)
    out = np.zeros(keys.shape[0], PATH_DTYPE)
    prm_c = prm.c()
    rc = lib().or_path_amp_d(_p(wt, C.c_double), _p(_i32(tri_mat), C.c_int32), wt.shape[0],
                             _p(mats, C.c_double), mats.shape[0],
                             _p(np.ascontiguousarray(tx, np.float64), C.c_double), _p(rx, C.c_double),
                             rx.shape[0], _p(keys, C.c_int32), keys.shape[0], C.byref(prm_c),
                             out.ctypes.data_as(C.c_void_p))
    if rc != 0:
        raise RuntimeError(f"or_path_amp_d failed: {rc}")
    return out


def field_of(keys, paths, nrx) -> np.ndarray:
    """Per-receiver sum of the amplitudes of the rows marked valid, in key order."""
    e = np.zeros(nrx, np.complex128)
    for i in range(keys.shape[0]):
        if paths["valid"][i]:
            e[int(keys[i, 0])] += complex(paths["amp_re"][i], paths["amp_im"][i])
    return e


def field_gradient(world_tris, tri_mat, tri_obj, materials, tx, rx, keys, prm: OracleParams,
                   nobj: int, h_pos: float = 1e-6, h_mat: float = 1e-6):
    """Derivatives of the per-receiver field E = sum a over a fixed set of
    paths (``keys``) by central differences in FP64, with respect to
    theta = (eps_r, sigma) of every material, then (x, y) translations of
    every rigid object (all its triangles moved together), in that order.

    Returns (E, dE, ok): E (nrx,) complex at theta, dE (nrx, 2 nmat + 2 nobj)
    complex, ok (nkeys,) -- the keys whose geometric validity is the same at
    theta and at every perturbed point (only those enter E and dE)."""
    wt = np.ascontiguousarray(world_tris, np.float64).reshape(-1, 3, 3)
    mats = np.ascontiguousarray(materials, np.float64).reshape(-1, 3)
    tri_obj = np.asarray(tri_obj)
    rx = np.ascontiguousarray(rx, np.float64).reshape(-1, 3)
    nrx, nmat = rx.shape[0], mats.shape[0]
    base = path_amp_d(wt, tri_mat, mats, tx, rx, keys, prm)
    ok = base["valid"] != 0
    evals = []
    for m in range(nmat):
        for c in range(2):
            h = h_mat * max(1.0, abs(mats[m, c]))
            mp, mm = mats.copy(), mats.copy()
            mp[m, c] += h
            mm[m, c] -= h
            evals.append((h, (wt, mp), (wt, mm)))
    for o in range(nobj):
        sel = tri_obj == o
        for c in range(2):
            tp, tm = wt.copy(), wt.copy()
            tp[sel, :, c] += h_pos
            tm[sel, :, c] -= h_pos
            evals.append((h_pos, (tp, mats), (tm, mats)))
    res = []
    for h, (tp, mp), (tm, mm) in evals:
        pp = path_amp_d(tp, tri_mat, mp, tx, rx, keys, prm)
        pm = path_amp_d(tm, tri_mat, mm, tx, rx, keys, prm)
        ok &= (pp["valid"] != 0) & (pm["valid"] != 0)
        res.append((h, pp, pm))
    sel = base.copy()
    sel["valid"] = ok
    e = field_of(keys, sel, nrx)
    de = np.zeros((nrx, len(res)), np.complex128)
    for i, (h, pp, pm) in enumerate(res):
        pp = pp.copy()
        pm = pm.copy()
        pp["valid"] = ok
        pm["valid"] = ok
        de[:, i] = (field_of(keys, pp, nrx) - field_of(keys, pm, nrx)) / (2.0 * h)
    return e, de, ok


def pcoh_dbm_gradient(e, de, tx_power_w):
    """d P_coh[dBm] / d theta from E and dE: P = P_t |E|^2, so dP = 2 P_t
    Re(conj(E) dE) and d(dBm) = 10 / ln 10 * dP / P."""
    p = tx_power_w * np.abs(e) ** 2
    dp = 2.0 * tx_power_w * np.real(np.conj(e)[:, None] * de)
    with np.errstate(divide="ignore", invalid="ignore"):
        return (10.0 / np.log(10.0)) * dp / p[:, None]


@dataclass
class FrameResult:
    world_tris: np.ndarray
    tr: dict
    keys: np.ndarray          # unique candidate keys, sorted
    paths: np.ndarray         # PATH_DTYPE per key
    field: np.ndarray
    p_coh_dbm: np.ndarray
    p_inc_dbm: np.ndarray
    extra: dict = field(default_factory=dict)


def frame(scene, f: int, rays: np.ndarray, prm: OracleParams, seg_od=False) -> FrameResult:
    """The whole oracle pipeline for frame ``f`` of a ``scenes.Scene``
    (with prm.diffraction, the diffraction paths -- first order, chains up to
    prm.diffraction_order, and with transmission first-order paths whose
    legs cross penetrable triangles -- join the validated keys before the
    reduction; chains through penetrable triangles, diffract_multi_trans,
    are not part of the frame)."""
    wt = transform(scene.tris, scene.tri_obj, scene.xf[f] if scene.nobj else np.zeros((0, 12)))
    rx = scene.rx[f]
    tr = trace(wt, scene.tri_mat, scene.materials, scene.tx, rays, rx, prm, seg_od=seg_od)
    keys = unique_keys(candidate_keys(tr["cands"], tr["hit_id"], prm.width))
    paths = validate(wt, scene.tri_mat, scene.materials, scene.tx, rx, keys, prm)
    if prm.diffraction:
        dk, dp = diffract(wt, scene.tri_mat, scene.tri_obj, scene.materials, scene.tx, rx, prm)
        keys = np.concatenate([keys, dk])
        paths = np.concatenate([paths, dp])
        if prm.diffraction_order > prm.width:
            raise ValueError("diffraction_order exceeds the key width (max_refl + max_trans)")
        for m in range(2, prm.diffraction_order + 1):
            mk_, mp_ = diffract_multi(wt, scene.tri_mat, scene.tri_obj, scene.materials, scene.tx, rx, prm, m)
            keys = np.concatenate([keys, mk_])
            paths = np.concatenate([paths, mp_])
        if prm.transmission:  # first-order paths whose legs cross penetrable triangles
            tk, tp = diffract_trans(wt, scene.tri_mat, scene.tri_obj, scene.materials, scene.tx, rx, prm)
            if tk.shape[1] != keys.shape[1]:
                raise ValueError("key widths differ: max_refl must be at least 1 with transmission")
            keys = np.concatenate([keys, tk])
            paths = np.concatenate([paths, tp])
        order = np.lexsort(keys.T[::-1])
        keys, paths = keys[order], paths[order]
    fld, pc, pi = reduce(keys, paths, rx.shape[0], prm.tx_power_w)
    return FrameResult(wt, tr, keys, paths, fld, pc, pi)


def keller_points(edges, T, R):
    """The oracle's Keller points of a chain of 1-3 edges from T to R: edges
    an (m, 7) array of (start, unit direction, length). Returns (converged,
    edge parameters t of shape (m,))."""
    e = np.ascontiguousarray(np.asarray(edges, np.float64).reshape(-1, 7))
    m = e.shape[0]
    T = np.ascontiguousarray(np.asarray(T, np.float64))
    R = np.ascontiguousarray(np.asarray(R, np.float64))
    t = np.zeros(3, np.float64)
    ok = lib().or_keller_points(m, _p(e, C.c_double), _p(T, C.c_double), _p(R, C.c_double),
                                _p(t, C.c_double))
    return bool(ok), t[:m].copy()


def transition(x: float) -> complex:
    """UTD transition function F(x) (Kouyoumjian & Pathak 1974)."""
    out = np.zeros(2)
    lib().or_transition(float(x), _p(out, C.c_double))
    return complex(out[0], out[1])


def utd_coefficient(n, phi, phip, beta0, L, k, r0, rn) -> complex:
    """Wedge diffraction coefficient with face reflection factors r0, rn
    (-1 soft / +1 hard for a perfect conductor; Luebbers' Fresnel factors)."""
    out = np.zeros(2)
    a = np.array([complex(r0).real, complex(r0).imag])
    b = np.array([complex(rn).real, complex(rn).imag])
    lib().or_utd(float(n), float(phi), float(phip), float(beta0), float(L), float(k),
                 _p(a, C.c_double), _p(b, C.c_double), _p(out, C.c_double))
    return complex(out[0], out[1])


def count_wedges(world_tris, tri_obj) -> int:
    wt = _f32(world_tris).reshape(-1, 9)
    return int(lib().or_count_wedges(_p(wt, C.c_float), _p(_i32(tri_obj), C.c_int32), wt.shape[0]))


def diffract(world_tris, tri_mat, tri_obj, materials, tx, rx, prm: OracleParams, cap=1 << 20):
    """Step 5, first order: every (receiver, wedge) diffraction path that is
    valid (Keller point on the edge, receiver in the source's shadow region,
    both legs unoccluded), with its UTD field. Keys (rx, 1, wedge | DIFF)."""
    wt = _f32(world_tris).reshape(-1, 9)
    mats = _f32(materials).reshape(-1, 3)
    rx = _f32(rx).reshape(-1, 3)
    width = prm.width
    keys = np.zeros((cap, 2 + width), np.int32)
    paths = np.zeros(cap, PATH_DTYPE)
    prm_c = prm.c()
    n = lib().or_diffract(_p(wt, C.c_float), _p(_i32(tri_mat), C.c_int32), _p(_i32(tri_obj), C.c_int32),
                          wt.shape[0], _p(mats, C.c_float), mats.shape[0], _p(_f32(tx), C.c_float),
                          _p(rx, C.c_float), rx.shape[0], C.byref(prm_c), width, _p(keys, C.c_int32),
                          paths.ctypes.data_as(C.c_void_p), cap)
    if n < 0:
        raise RuntimeError(f"or_diffract failed: {n}")
    if n > cap:
        raise RuntimeError(f"or_diffract: {n} paths exceed capacity {cap}")
    return keys[:n].copy(), paths[:n].copy()


def diffract_trans(world_tris, tri_mat, tri_obj, materials, tx, rx, prm: OracleParams, cap=1 << 20):
    """Step 5 with transmission: first-order diffraction paths whose legs pass
    straight through penetrable triangles (prm.trans_db >= 0), at least one
    and at most prm.max_trans in all, the field times 10^(-L/20) per
    crossing. Keys (rx, depth, crossings of the first leg | TRANS, wedge |
    DIFF, crossings of the second leg | TRANS), -1 padded to 2 +
    max(prm.width, 1 + prm.max_trans)."""
    wt = _f32(world_tris).reshape(-1, 9)
    mats = _f32(materials).reshape(-1, 3)
    rx = _f32(rx).reshape(-1, 3)
    width = max(prm.width, 1 + prm.max_trans)
    keys = np.zeros((cap, 2 + width), np.int32)
    paths = np.zeros(cap, PATH_DTYPE)
    prm_c = prm.c()
    n = lib().or_diffract_trans(_p(wt, C.c_float), _p(_i32(tri_mat), C.c_int32), _p(_i32(tri_obj), C.c_int32),
                                wt.shape[0], _p(mats, C.c_float), mats.shape[0], _p(_f32(tx), C.c_float),
                                _p(rx, C.c_float), rx.shape[0], C.byref(prm_c), width, _p(keys, C.c_int32),
                                paths.ctypes.data_as(C.c_void_p), cap)
    if n < 0:
        raise RuntimeError(f"or_diffract_trans failed: {n}")
    if n > cap:
        raise RuntimeError(f"or_diffract_trans: {n} paths exceed capacity {cap}")
    return keys[:n].copy(), paths[:n].copy()


def diffract_multi_trans(world_tris, tri_mat, tri_obj, materials, tx, rx, prm: OracleParams, order: int,
                         cap=1 << 20):
    """Chains of ``order`` wedges (as diffract_multi) whose legs cross
    penetrable triangles, at least one and at most prm.max_trans in all, the
    field times 10^(-L/20) per crossing. Keys (rx, depth, then in path order
    each leg's crossings | TRANS and the wedges | DIFF), -1 padded to 2 +
    max(prm.width, order + prm.max_trans)."""
    wt = _f32(world_tris).reshape(-1, 9)
    mats = _f32(materials).reshape(-1, 3)
    rx = _f32(rx).reshape(-1, 3)
    width = max(prm.width, order + prm.max_trans)
    keys = np.zeros((cap, 2 + width), np.int32)
    paths = np.zeros(cap, PATH_DTYPE)
    prm_c = prm.c()
    n = lib().or_diffract_multi_trans(_p(wt, C.c_float), _p(_i32(tri_mat), C.c_int32), _p(_i32(tri_obj), C.c_int32),
                                      wt.shape[0], _p(mats, C.c_float), mats.shape[0], _p(_f32(tx), C.c_float),
                                      _p(rx, C.c_float), rx.shape[0], C.byref(prm_c), int(order), width,
                                      _p(keys, C.c_int32), paths.ctypes.data_as(C.c_void_p), cap)
    if n < 0:
        raise RuntimeError(f"or_diffract_multi_trans failed: {n}")
    if n > cap:
        raise RuntimeError(f"or_diffract_multi_trans: {n} paths exceed capacity {cap}")
    return keys[:n].copy(), paths[:n].copy()


def diffract_multi(world_tris, tri_mat, tri_obj, materials, tx, rx, prm: OracleParams, order: int,
                   cap=1 << 20):
    """Step 5, orders 2 and 3: paths over ``order`` distinct wedges (Keller
    points by minimising the unfolded length, the shadow rule at every wedge,
    every leg unoccluded) with the chained UTD field and the astigmatic
    spreading of edge-diffracted waves. Keys (rx, order, w1 | DIFF, ..),
    -1 padded to 2 + max(prm.width, order)."""
    wt = _f32(world_tris).reshape(-1, 9)
    mats = _f32(materials).reshape(-1, 3)
    rx = _f32(rx).reshape(-1, 3)
    width = max(prm.width, order)
    keys = np.zeros((cap, 2 + width), np.int32)
    paths = np.zeros(cap, PATH_DTYPE)
    prm_c = prm.c()
    n = lib().or_diffract_multi(_p(wt, C.c_float), _p(_i32(tri_mat), C.c_int32), _p(_i32(tri_obj), C.c_int32),
                                wt.shape[0], _p(mats, C.c_float), mats.shape[0], _p(_f32(tx), C.c_float),
                                _p(rx, C.c_float), rx.shape[0], C.byref(prm_c), int(order), width,
                                _p(keys, C.c_int32), paths.ctypes.data_as(C.c_void_p), cap)
    if n < 0:
        raise RuntimeError(f"or_diffract_multi failed: {n}")
    if n > cap:
        raise RuntimeError(f"or_diffract_multi: {n} paths exceed capacity {cap}")
    return keys[:n].copy(), paths[:n].copy()


def diffract_multi_refl(world_tris, tri_mat, tri_obj, materials, tx, rx, prm: OracleParams, order: int,
                        cap=1 << 20):
    """Steps 3-5 combined: one reflection on a static triangle before or after
    a chain of ``order`` (2 or 3) wedges (image theory: the chain from the
    transmitter's image, or toward the receiver's image). Keys (rx, order + 1,
    tri, w1 | DIFF, ..) for the reflection first, (rx, order + 1, w1 | DIFF,
    .., tri) for the reflection last, -1 padded to 2 + max(prm.width, order + 1)."""
    wt = _f32(world_tris).reshape(-1, 9)
    mats = _f32(materials).reshape(-1, 3)
    rx = _f32(rx).reshape(-1, 3)
    width = max(prm.width, order + 1)
    keys = np.zeros((cap, 2 + width), np.int32)
    paths = np.zeros(cap, PATH_DTYPE)
    prm_c = prm.c()
    n = lib().or_diffract_multi_refl(_p(wt, C.c_float), _p(_i32(tri_mat), C.c_int32), _p(_i32(tri_obj), C.c_int32),
                                     wt.shape[0], _p(mats, C.c_float), mats.shape[0], _p(_f32(tx), C.c_float),
                                     _p(rx, C.c_float), rx.shape[0], C.byref(prm_c), int(order), width,
                                     _p(keys, C.c_int32), paths.ctypes.data_as(C.c_void_p), cap)
    if n < 0:
        raise RuntimeError(f"or_diffract_multi_refl failed: {n}")
    if n > cap:
        raise RuntimeError(f"or_diffract_multi_refl: {n} paths exceed capacity {cap}")
    return keys[:n].copy(), paths[:n].copy()


def diffract_refl(world_tris, tri_mat, tri_obj, materials, tx, rx, prm: OracleParams, cap=1 << 20):
    """Steps 3-5 combined: one reflection on a static triangle before or after
    a first-order diffraction (image theory: the diffraction of the
    transmitter's image, or toward the receiver's image, in the triangle's
    plane). Keys (rx, 2, tri, wedge | DIFF) for the reflection first,
    (rx, 2, wedge | DIFF, tri) for the reflection last; paths with the UTD
    field, the Fresnel reflection and the unfolded length."""
    wt = _f32(world_tris).reshape(-1, 9)
    mats = _f32(materials).reshape(-1, 3)
    rx = _f32(rx).reshape(-1, 3)
    width = max(prm.width, 2)
    keys = np.zeros((cap, 2 + width), np.int32)
    paths = np.zeros(cap, PATH_DTYPE)
    prm_c = prm.c()
    n = lib().or_diffract_refl(_p(wt, C.c_float), _p(_i32(tri_mat), C.c_int32), _p(_i32(tri_obj), C.c_int32),
                               wt.shape[0], _p(mats, C.c_float), mats.shape[0], _p(_f32(tx), C.c_float),
                               _p(rx, C.c_float), rx.shape[0], C.byref(prm_c), width, _p(keys, C.c_int32),
                               paths.ctypes.data_as(C.c_void_p), cap)
    if n < 0:
        raise RuntimeError(f"or_diffract_refl failed: {n}")
    if n > cap:
        raise RuntimeError(f"or_diffract_refl: {n} paths exceed capacity {cap}")
    return keys[:n].copy(), paths[:n].copy()


def diffract_refl2(world_tris, tri_mat, tri_obj, materials, tx, rx, prm: OracleParams, cap=1 << 20):
    """Steps 3-5 combined with two reflections on static triangles around a
    first-order diffraction: both before the wedge, one on each side, or both
    after it (image theory over the chain solver). Keys (rx, 3, ids in path
    order, the wedge's with DIFF), -1 padded to 2 + max(prm.width, 3)."""
    wt = _f32(world_tris).reshape(-1, 9)
    mats = _f32(materials).reshape(-1, 3)
    rx = _f32(rx).reshape(-1, 3)
    width = max(prm.width, 3)
    keys = np.zeros((cap, 2 + width), np.int32)
    paths = np.zeros(cap, PATH_DTYPE)
    prm_c = prm.c()
    n = lib().or_diffract_refl2(_p(wt, C.c_float), _p(_i32(tri_mat), C.c_int32), _p(_i32(tri_obj), C.c_int32),
                                wt.shape[0], _p(mats, C.c_float), mats.shape[0], _p(_f32(tx), C.c_float),
                                _p(rx, C.c_float), rx.shape[0], C.byref(prm_c), width, _p(keys, C.c_int32),
                                paths.ctypes.data_as(C.c_void_p), cap)
    if n < 0:
        raise RuntimeError(f"or_diffract_refl2 failed: {n}")
    if n > cap:
        raise RuntimeError(f"or_diffract_refl2: {n} paths exceed capacity {cap}")
    return keys[:n].copy(), paths[:n].copy()


def diffract_mid(world_tris, tri_mat, tri_obj, materials, tx, rx, prm: OracleParams, cap=1 << 20):
    """Steps 3-5 combined: a reflection on a static triangle between two
    diffractions (image theory: the chain over the first wedge and the second
    one's image toward the receiver's image). Keys (rx, 3, w1 | DIFF, tri,
    w2 | DIFF), -1 padded to 2 + max(prm.width, 3)."""
    wt = _f32(world_tris).reshape(-1, 9)
    mats = _f32(materials).reshape(-1, 3)
    rx = _f32(rx).reshape(-1, 3)
    width = max(prm.width, 3)
    keys = np.zeros((cap, 2 + width), np.int32)
    paths = np.zeros(cap, PATH_DTYPE)
    prm_c = prm.c()
    n = lib().or_diffract_mid(_p(wt, C.c_float), _p(_i32(tri_mat), C.c_int32), _p(_i32(tri_obj), C.c_int32),
                              wt.shape[0], _p(mats, C.c_float), mats.shape[0], _p(_f32(tx), C.c_float),
                              _p(rx, C.c_float), rx.shape[0], C.byref(prm_c), width, _p(keys, C.c_int32),
                              paths.ctypes.data_as(C.c_void_p), cap)
    if n < 0:
        raise RuntimeError(f"or_diffract_mid failed: {n}")
    if n > cap:
        raise RuntimeError(f"or_diffract_mid: {n} paths exceed capacity {cap}")
    return keys[:n].copy(), paths[:n].copy()


def diffract_path(world_tris, tri_mat, tri_obj, materials, tx, rx, ids, prm: OracleParams):
    """One given path of the combined mechanisms (ids in path order: up to two
    static-triangle reflections around a run of 1-3 wedge ids marked DIFF),
    evaluated for one receiver rx. Returns the path record, or None when the
    path is not valid."""
    wt = _f32(world_tris).reshape(-1, 9)
    mats = _f32(materials).reshape(-1, 3)
    ids = _i32(ids)
    out = np.zeros(1, PATH_DTYPE)
    prm_c = prm.c()
    r = lib().or_diffract_path(_p(wt, C.c_float), _p(_i32(tri_mat), C.c_int32), _p(_i32(tri_obj), C.c_int32),
                               wt.shape[0], _p(mats, C.c_float), mats.shape[0], _p(_f32(tx), C.c_float),
                               _p(_f32(rx).reshape(3), C.c_float), _p(ids, C.c_int32), ids.shape[0],
                               C.byref(prm_c), out.ctypes.data_as(C.c_void_p))
    if r < 0:
        raise ValueError(f"or_diffract_path: ids {ids.tolist()} are not a combined diffraction path ({r})")
    return out[0] if r == 1 else None


def sticky_frames(scene, frames, rays: np.ndarray, prm: OracleParams):
    """Frames in the path cache's retention mode (Sec. III "Propagation path
    caching": a cached path is kept and updated until it is removed). Frame
    i's keys: the distinct keys its rays capture, plus (from the second frame
    on) every key that was valid in frame i-1; all of them are validated with
    frame i's geometry, so a kept path stays while it is valid and is removed
    when it is not. Returns per frame a FrameResult over that key set, with
    ``extra["kept_only"]``: the valid keys that no ray of the frame captured."""
    out = []
    prev = None
    for f in frames:
        fr = frame(scene, f, rays, prm)
        keys = fr.keys
        if prev is not None and prev.shape[0]:
            keys = unique_keys(np.concatenate([fr.keys, prev]))
        paths = validate(fr.world_tris, scene.tri_mat, scene.materials, scene.tx, scene.rx[f], keys, prm)
        fld, pc, pi = reduce(keys, paths, scene.rx[f].shape[0], prm.tx_power_w)
        disc = {tuple(k) for k in fr.keys.tolist()}
        valid = keys[paths["valid"] != 0]
        kept = np.array([k for k in valid.tolist() if tuple(k) not in disc], np.int32).reshape(-1, keys.shape[1])
        out.append(FrameResult(fr.world_tris, fr.tr, keys, paths, fld, pc, pi, {"kept_only": kept}))
        prev = valid
    return out
