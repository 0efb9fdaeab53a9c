"""ctypes binding of libdcem (include/dcem.h): argument marshalling only.

Every step of a frame runs in the library's CUDA kernels; this module only
converts numpy arrays / torch tensors to pointers and sizes. Module-level
functions carry the C names; ``Scene`` is a small convenience wrapper.
If the library has not been built the import of a function fails loudly:
there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# DCEM_LIB_VARIANT=checks selects the bounds-checked build (build.build(checks=True))
_VARIANT = os.environ.get("DCEM_LIB_VARIANT", "")
LIB_PATH = (os.path.join(_HERE, "_build_checks", "libdcem_checks.so") if _VARIANT == "checks"
            else os.path.join(_HERE, "_build", "libdcem.so"))

MAX_REFL = 10
OK, ERR_ARG, ERR_CUDA, ERR_CAPACITY, ERR_NONFINITE, ERR_STACK, ERR_HASH, ERR_STATE, ERR_NOMEM, ERR_CHECK = \
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9
MODE_FULL, MODE_COHERENT, MODE_STICKY = 0, 1, 2
PREC_F64, PREC_DF32 = 0, 1
PTR_HOST, PTR_DEVICE = 0, 1
PATH_POL_DEGENERATE = 1
PATH_STICKY = 2
TRI_TRANSMIT = 0x40000000
TRI_DIFFRACT = 0x20000000

EXPORTED = ["dcem_params_default", "dcem_scene_create", "dcem_scene_set_rays",
            "dcem_scene_update_transforms", "dcem_trace_frame", "dcem_scene_reset_cache",
            "dcem_scene_set_stream", "dcem_scene_destroy", "dcem_status_string", "dcem_scene_info",
            "dcem_scene_get_world_tris", "dcem_scene_get_bvh", "dcem_scene_get_ray_log",
            "dcem_scene_get_candidates", "dcem_scene_set_rebuild_threshold",
            "dcem_reduce_paths_noalloc", "dcem_scene_gradient_size", "dcem_path_gradients", "dcem_path_adjoint",
            "dcem_scene_set_graph_replay", "dcem_scene_set_ray_sets", "dcem_trace_links",
            "dcem_scene_set_trace_config", "dcem_scene_autotune", "dcem_batch_create",
            "dcem_batch_update_transforms", "dcem_batch_trace", "dcem_batch_destroy",
            "dcem_scene_set_transmission", "dcem_scene_set_diffraction", "dcem_scene_set_diffraction_reflections",
            "dcem_scene_set_diffraction_order"]


class Material(C.Structure):
    _fields_ = [("eps_r", C.c_float), ("sigma", C.c_float), ("pec", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("freq_hz", C.c_double), ("tx_power_w", C.c_double), ("max_refl", C.c_int32),
                ("mode", C.c_int32), ("rx_radius_scale", C.c_float), ("t_min", C.c_float),
                ("escape_len", C.c_float), ("eps_occ", C.c_float), ("pol", C.c_float * 3),
                ("timing", C.c_int32), ("prec", C.c_int32)]


class Path(C.Structure):
    _fields_ = [("rx", C.c_int32), ("depth", C.c_int32), ("tri", C.c_int32 * MAX_REFL),
                ("flags", C.c_uint32), ("ray", C.c_int32), ("tx", C.c_int32),
                ("reserved", C.c_int32), ("key", C.c_uint64), ("len_m", C.c_double), ("delay_s", C.c_double), ("amp_re", C.c_double),
                ("amp_im", C.c_double), ("pts", C.c_float * (3 * MAX_REFL))]


class Stats(C.Structure):
    _fields_ = [("n_rays", C.c_int64), ("segments_traced", C.c_int64),
                ("segments_reused", C.c_int64), ("rays_retraced", C.c_int64),
                ("candidates", C.c_int64), ("candidates_reused", C.c_int64),
                ("unique_candidates", C.c_int64), ("paths_valid", C.c_int64),
                ("objects_moved", C.c_int64), ("rx_moved", C.c_int64),
                ("node_visits", C.c_int64), ("tri_tests", C.c_int64),
                ("stack_overflow", C.c_int32), ("coherent", C.c_int32),
                ("kernel_launches", C.c_int32), ("bvh_rebuilt", C.c_int32),
                ("ms_stage", C.c_float * 10), ("bvh_cost_ratio", C.c_float),
                ("max_segment_nodes", C.c_int32), ("trace_kernel", C.c_int32),
                ("graph_replayed", C.c_int32), ("paths_sticky", C.c_int32), ("child_rays", C.c_int32),
                ("keys_reused", C.c_int32), ("diff_candidates", C.c_int32), ("diff_pairs", C.c_int32),
                ("diff_triples", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("ptr_kind", C.c_int32), ("max_paths", C.c_int32), ("field", C.c_void_p),
                ("p_coh_dbm", C.c_void_p), ("p_inc_dbm", C.c_void_p), ("paths", C.c_void_p),
                ("n_paths", C.c_int32), ("stats", Stats)]


PATH_DTYPE = np.dtype([("rx", np.int32), ("depth", np.int32), ("tri", np.int32, (MAX_REFL,)),
                       ("flags", np.uint32), ("ray", np.int32), ("tx", np.int32),
                       ("reserved", np.int32), ("key", np.uint64),
                       ("len_m", np.float64), ("delay_s", np.float64), ("amp_re", np.float64),
                       ("amp_im", np.float64), ("pts", np.float32, (MAX_REFL, 3))])
assert PATH_DTYPE.itemsize == C.sizeof(Path)

STAGES = ["prep", "mark", "trace", "capture", "dedupe", "validate", "reduce", "copy_out", "total"]

_lib = None


def lib():
    """The loaded library (raises if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libdcem.so is not built ({LIB_PATH}); run "
                               "paper_2112_07115_gb300.build.build() first")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        P = C.POINTER
        L.dcem_params_default.argtypes = [P(Params)]
        L.dcem_params_default.restype = None
        L.dcem_scene_create.argtypes = [vp, i32, vp, vp, i32, vp, i32, vp, P(vp)]
        L.dcem_scene_set_rays.argtypes = [vp, vp, i32]
        L.dcem_scene_update_transforms.argtypes = [vp, vp, i32]
        L.dcem_trace_frame.argtypes = [vp, vp, vp, i32, i32, P(Params), P(Result)]
        L.dcem_scene_set_ray_sets.argtypes = [vp, vp, vp, i32]
        L.dcem_trace_links.argtypes = [vp, vp, i32, vp, i32, i32, P(Params), P(Result)]
        L.dcem_scene_set_trace_config.argtypes = [vp, i32, i32, i32]
        L.dcem_scene_set_transmission.argtypes = [vp, vp, i32, i32]
        L.dcem_scene_set_diffraction.argtypes = [vp, i32, P(i32)]
        L.dcem_scene_set_diffraction_reflections.argtypes = [vp, i32, P(i32)]
        L.dcem_scene_set_diffraction_order.argtypes = [vp, i32]
        L.dcem_batch_create.argtypes = [vp, i32, vp, P(vp)]
        L.dcem_batch_update_transforms.argtypes = [vp, vp, i32]
        L.dcem_batch_trace.argtypes = [vp, vp, vp, vp, vp, i32, P(Params), vp, P(i32)]
        L.dcem_batch_destroy.argtypes = [vp]
        L.dcem_batch_destroy.restype = None
        L.dcem_scene_autotune.argtypes = [vp, vp, i32, vp, i32, i32, P(Params), i32, P(i32), P(i32), P(i32)]
        L.dcem_scene_reset_cache.argtypes = [vp]
        L.dcem_scene_set_stream.argtypes = [vp, vp]
        L.dcem_scene_destroy.argtypes = [vp]
        L.dcem_scene_destroy.restype = None
        L.dcem_status_string.argtypes = [C.c_int]
        L.dcem_status_string.restype = C.c_char_p
        L.dcem_scene_info.argtypes = [vp, P(i32), P(i32), P(i32), P(i32), P(i32)]
        L.dcem_scene_get_world_tris.argtypes = [vp, vp]
        L.dcem_scene_get_bvh.argtypes = [vp, vp, vp, vp]
        L.dcem_scene_get_ray_log.argtypes = [vp, vp, vp, vp]
        L.dcem_scene_get_candidates.argtypes = [vp, vp, i64, P(i64)]
        L.dcem_scene_set_rebuild_threshold.argtypes = [vp, C.c_float]
        L.dcem_scene_set_graph_replay.argtypes = [vp, i32]
        L.dcem_reduce_paths_noalloc.argtypes = [vp, i32, i32, C.c_double, vp, vp, vp, vp]
        L.dcem_scene_gradient_size.argtypes = [vp, P(i32)]
        L.dcem_path_adjoint.argtypes = [vp, vp, vp, i32, i32, vp, i32, P(Params), vp, vp, i32, vp, vp, vp, vp, vp]
        L.dcem_path_gradients.argtypes = [vp, vp, vp, i32, i32, vp, i32, P(Params), i32, vp, vp, vp]
        for name in EXPORTED:
            if name not in ("dcem_params_default", "dcem_scene_destroy", "dcem_status_string",
                            "dcem_batch_destroy"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


class DcemError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


def status_string(status: int) -> str:
    return lib().dcem_status_string(int(status)).decode()


def _check(rc: int, where: str):
    if rc != OK:
        raise DcemError(rc, where)


# --------------------------------------------------------------------------
# pointer marshalling
# --------------------------------------------------------------------------
def _is_cuda_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and bool(getattr(x, "is_cuda"))


def _ptr(x, dtype):
    """(pointer, kind, keepalive) of a numpy array (host) or torch tensor."""
    if x is None:
        return None, PTR_HOST, None
    if hasattr(x, "data_ptr"):  # torch tensor
        if not x.is_contiguous():
            x = x.contiguous()
        return x.data_ptr(), (PTR_DEVICE if x.is_cuda else PTR_HOST), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, PTR_HOST, a


def default_params(**kw) -> Params:
    p = Params()
    lib().dcem_params_default(C.byref(p))
    for k, v in kw.items():
        if k == "pol":
            for i in range(3):
                p.pol[i] = float(v[i])
        else:
            setattr(p, k, v)
    return p


# --------------------------------------------------------------------------
# C names
# --------------------------------------------------------------------------
def dcem_scene_create(tris, tri_mat, materials, tri_obj=None, nobj=0, stream=None) -> int:
    """Returns an opaque handle (int). materials: (M,3) rows (eps_r, sigma, pec)."""
    tris = np.ascontiguousarray(tris, np.float32).reshape(-1, 9)
    tri_mat = np.ascontiguousarray(tri_mat, np.int32)
    mats = np.asarray(materials, np.float64).reshape(-1, 3)
    marr = (Material * max(len(mats), 1))()
    for i, (e, s, p) in enumerate(mats):
        marr[i].eps_r, marr[i].sigma, marr[i].pec = float(e), float(s), int(p)
    to = None if tri_obj is None else np.ascontiguousarray(tri_obj, np.int32)
    h = C.c_void_p()
    rc = lib().dcem_scene_create(tris.ctypes.data if tris.size else None, tris.shape[0],
                                 tri_mat.ctypes.data if tri_mat.size else None, marr, len(mats),
                                 to.ctypes.data if to is not None and to.size else None, int(nobj),
                                 stream, C.byref(h))
    _check(rc, "dcem_scene_create")
    return h.value


def dcem_scene_set_rays(h, dirs):
    d = np.ascontiguousarray(dirs, np.float32).reshape(-1, 3)
    _check(lib().dcem_scene_set_rays(h, d.ctypes.data if d.size else None, d.shape[0]),
           "dcem_scene_set_rays")


def dcem_scene_set_ray_sets(h, sets):
    """One ray set per transmitter: `sets` is a list of (n_t, 3) direction arrays."""
    d = [np.ascontiguousarray(x, np.float32).reshape(-1, 3) for x in sets]
    n = np.array([x.shape[0] for x in d], np.int32)
    cat = np.ascontiguousarray(np.concatenate(d) if d else np.zeros((0, 3), np.float32))
    _check(lib().dcem_scene_set_ray_sets(h, cat.ctypes.data if cat.size else None, n.ctypes.data, len(d)),
           "dcem_scene_set_ray_sets")


def dcem_trace_links(h, tx, rx, params: Params, result: Result) -> int:
    """Raw call for ntx transmitters (tx: (ntx, 3)); returns the status."""
    txa = np.ascontiguousarray(tx, np.float32).reshape(-1, 3)
    rp, kind, keep = _ptr(rx, np.float32)
    nrx = (rx.numel() if hasattr(rx, "numel") else np.asarray(rx).size) // 3
    return lib().dcem_trace_links(h, txa.ctypes.data, txa.shape[0], rp, nrx, kind, C.byref(params),
                                  C.byref(result))


def dcem_scene_set_transmission(h, loss_db, max_trans: int):
    a = np.ascontiguousarray(loss_db, np.float32).reshape(-1)
    _check(lib().dcem_scene_set_transmission(h, a.ctypes.data if a.size else None, a.size, int(max_trans)),
           "dcem_scene_set_transmission")


def dcem_scene_set_diffraction(h, on: bool) -> int:
    n = C.c_int32(0)
    _check(lib().dcem_scene_set_diffraction(h, int(bool(on)), C.byref(n)), "dcem_scene_set_diffraction")
    return n.value


def dcem_scene_set_trace_config(h, kernel: int, block: int = 256, stack: int = 24):
    _check(lib().dcem_scene_set_trace_config(h, int(kernel), int(block), int(stack)),
           "dcem_scene_set_trace_config")


def dcem_scene_autotune(h, tx, rx, params: Params, reps: int = 2):
    """Times the closest-hit kernel under each configuration on this frame
    and keeps the fastest; returns (kernel, block, stack)."""
    txa = np.ascontiguousarray(tx, np.float32).reshape(-1, 3)
    rp, kind, keep = _ptr(rx, np.float32)
    nrx = (rx.numel() if hasattr(rx, "numel") else np.asarray(rx).size) // 3
    k, b, s = C.c_int32(0), C.c_int32(0), C.c_int32(0)
    _check(lib().dcem_scene_autotune(h, txa.ctypes.data, txa.shape[0], rp, nrx, kind, C.byref(params), int(reps),
                                     C.byref(k), C.byref(b), C.byref(s)), "dcem_scene_autotune")
    return k.value, b.value, s.value


def dcem_scene_update_transforms(h, xf):
    p, kind, keep = _ptr(xf, np.float32)
    _check(lib().dcem_scene_update_transforms(h, p, kind), "dcem_scene_update_transforms")


def dcem_trace_frame(h, tx, rx, params: Params, result: Result) -> int:
    """Raw call; returns the status (the caller owns `result`'s arrays)."""
    txa = np.ascontiguousarray(tx, np.float32).reshape(3)
    rp, kind, keep = _ptr(rx, np.float32)
    nrx = (rx.numel() if hasattr(rx, "numel") else np.asarray(rx).size) // 3
    return lib().dcem_trace_frame(h, txa.ctypes.data, rp, nrx, kind, C.byref(params),
                                  C.byref(result))


def dcem_scene_set_rebuild_threshold(h, ratio: float):
    _check(lib().dcem_scene_set_rebuild_threshold(h, float(ratio)), "dcem_scene_set_rebuild_threshold")


def dcem_scene_set_graph_replay(h, on: bool):
    _check(lib().dcem_scene_set_graph_replay(h, int(bool(on))), "dcem_scene_set_graph_replay")


def dcem_reduce_paths_noalloc(paths_ptr, n_paths, nrx, tx_power_w, field_ptr, p_coh_ptr, p_inc_ptr,
                              stream=None) -> int:
    """Per-receiver sums of device path records without device allocation
    (device pointers as ints); returns the status."""
    return lib().dcem_reduce_paths_noalloc(paths_ptr, int(n_paths), int(nrx), float(tx_power_w), field_ptr,
                                           p_coh_ptr, p_inc_ptr, stream)


def dcem_scene_gradient_size(h) -> int:
    n = C.c_int32(0)
    _check(lib().dcem_scene_gradient_size(h, C.byref(n)), "dcem_scene_gradient_size")
    return int(n.value)


def dcem_path_gradients(h, tx, rx, paths, params: Params, ptr_kind: int, field_ptr, dfield_ptr,
                        dpcoh_ptr, n_paths: int | None = None) -> int:
    """Raw call; returns the status. ``rx`` is an array or tensor (its kind
    decides rx_ptr_kind); ``paths`` and the outputs are host or device
    pointers as ints per ``ptr_kind`` (or a PATH_DTYPE array for host paths)."""
    txa = np.ascontiguousarray(tx, np.float32).reshape(3)
    rp, rkind, keep = _ptr(rx, np.float32)
    nrx = (rx.numel() if hasattr(rx, "numel") else np.asarray(rx).size) // 3
    if isinstance(paths, np.ndarray):
        n_paths = paths.shape[0] if n_paths is None else n_paths
        pp = paths.ctypes.data if n_paths else None
    else:
        pp = paths
    return lib().dcem_path_gradients(h, txa.ctypes.data, rp, nrx, rkind, pp, int(n_paths or 0),
                                     C.byref(params), ptr_kind, field_ptr, dfield_ptr, dpcoh_ptr)


def dcem_path_adjoint(h, tx, rx, paths, params: Params, ptr_kind: int, theta_ptr=None, pcoh_bar_ptr=None,
                      field_ptr=None, pcoh_ptr=None, dfield_ptr=None, dpcoh_ptr=None, theta_bar_ptr=None,
                      n_paths: int | None = None) -> int:
    """Raw call of the adjoint; returns the status. ``rx`` as in
    dcem_path_gradients; ``paths``, theta, pcoh_bar and the outputs are host
    or device pointers as ints per ``ptr_kind`` (None = NULL)."""
    txa = np.ascontiguousarray(tx, np.float32).reshape(3)
    rp, rkind, keep = _ptr(rx, np.float32)
    nrx = (rx.numel() if hasattr(rx, "numel") else np.asarray(rx).size) // 3
    if isinstance(paths, np.ndarray):
        n_paths = paths.shape[0] if n_paths is None else n_paths
        pp = paths.ctypes.data if n_paths else None
    else:
        pp = paths
    return lib().dcem_path_adjoint(h, txa.ctypes.data, rp, nrx, rkind, pp, int(n_paths or 0), C.byref(params),
                                   theta_ptr, pcoh_bar_ptr, ptr_kind, field_ptr, pcoh_ptr, dfield_ptr, dpcoh_ptr,
                                   theta_bar_ptr)


def dcem_scene_reset_cache(h):
    _check(lib().dcem_scene_reset_cache(h), "dcem_scene_reset_cache")


def dcem_scene_set_stream(h, stream):
    _check(lib().dcem_scene_set_stream(h, stream), "dcem_scene_set_stream")


def dcem_scene_destroy(h):
    lib().dcem_scene_destroy(h)


def dcem_scene_info(h) -> dict:
    v = [C.c_int32() for _ in range(5)]
    _check(lib().dcem_scene_info(h, *[C.byref(x) for x in v]), "dcem_scene_info")
    return dict(zip(["ntri", "nobj", "n_rays", "static_nodes", "dynamic_nodes"], [x.value for x in v]))


def dcem_scene_get_world_tris(h, ntri) -> np.ndarray:
    out = np.empty((ntri, 3, 3), np.float32)
    _check(lib().dcem_scene_get_world_tris(h, out.ctypes.data if ntri else None),
           "dcem_scene_get_world_tris")
    return out


def dcem_scene_get_bvh(h):
    info = dcem_scene_info(h)
    nn = info["static_nodes"] + info["dynamic_nodes"]
    child = np.empty((max(nn, 1), 2), np.int32)
    bounds = np.empty((max(nn, 1), 2, 6), np.float32)
    roots = np.empty(2, np.int32)
    _check(lib().dcem_scene_get_bvh(h, child.ctypes.data, bounds.ctypes.data, roots.ctypes.data),
           "dcem_scene_get_bvh")
    return child[:nn], bounds[:nn], roots, info


def dcem_scene_get_ray_log(h, n_rays, max_refl):
    W = max_refl + 1
    ids = np.empty((n_rays, W), np.int32)
    t = np.empty((n_rays, W), np.float32)
    ns = np.empty(n_rays, np.int32)
    if n_rays:
        _check(lib().dcem_scene_get_ray_log(h, ids.ctypes.data, t.ctypes.data, ns.ctypes.data),
               "dcem_scene_get_ray_log")
    return ids, t, ns


def dcem_scene_get_candidates(h) -> np.ndarray:
    n = C.c_int64(0)
    rc = lib().dcem_scene_get_candidates(h, None, 0, C.byref(n))
    if rc not in (OK, ERR_CAPACITY):
        _check(rc, "dcem_scene_get_candidates")
    out = np.empty((max(n.value, 1), 3), np.int32)
    if n.value:
        _check(lib().dcem_scene_get_candidates(h, out.ctypes.data, n.value, C.byref(n)),
               "dcem_scene_get_candidates")
    return out[:n.value]


# --------------------------------------------------------------------------
# convenience wrapper
# --------------------------------------------------------------------------
@dataclass
class Frame:
    status: int
    field: np.ndarray        # complex128 (nrx,)
    p_coh_dbm: np.ndarray
    p_inc_dbm: np.ndarray
    paths: np.ndarray        # PATH_DTYPE
    stats: dict


def stats_dict(s: Stats) -> dict:
    d = {k: getattr(s, k) for k, _ in Stats._fields_ if k != "ms_stage"}
    d["ms_stage"] = dict(zip(STAGES, list(s.ms_stage)))
    return d


class Scene:
    """A scene on the current CUDA device (see include/dcem.h)."""

    def __init__(self, tris, tri_mat, materials, tri_obj=None, nobj=0, stream=None):
        self.ntri = int(np.asarray(tris).reshape(-1, 9).shape[0])
        self.nobj = int(nobj)
        self.materials = np.asarray(materials, np.float32).reshape(-1, 3).copy()
        self.h = dcem_scene_create(tris, tri_mat, materials, tri_obj, nobj, stream)
        self.n_rays = 0
        self.max_refl = 3

    @classmethod
    def from_scene(cls, sc, stream=None):
        return cls(sc.tris, sc.tri_mat, sc.materials, sc.tri_obj, sc.nobj, stream)

    def set_rays(self, dirs):
        dcem_scene_set_rays(self.h, dirs)
        self.n_rays = int(np.asarray(dirs).reshape(-1, 3).shape[0])

    def set_ray_sets(self, sets):
        """Ray sets of several transmitters (for trace_links)."""
        dcem_scene_set_ray_sets(self.h, sets)
        self.set_sizes = [int(np.asarray(x).reshape(-1, 3).shape[0]) for x in sets]
        self.n_rays = sum(self.set_sizes)

    def trace_links(self, tx, rx, params: Params | None = None, max_paths: int | None = None,
                    raise_on_error: bool = True) -> Frame:
        """One frame of every transmitter (tx: (ntx, 3)) against the receivers:
        field and powers have shape (ntx, nrx); path records carry tx and rx."""
        params = params or default_params()
        self.max_refl = int(params.max_refl)
        ntx = np.asarray(tx).reshape(-1, 3).shape[0]
        nrx = (rx.numel() if hasattr(rx, "numel") else np.asarray(rx).size) // 3
        nl = ntx * nrx
        if max_paths is None:
            max_paths = max(1024, 256 * nl)
        field = np.empty((max(nl, 1), 2), np.float64)
        pc = np.empty(max(nl, 1), np.float64)
        pi = np.empty(max(nl, 1), np.float64)
        paths = np.empty(max_paths, PATH_DTYPE)
        res = Result()
        res.ptr_kind = PTR_HOST
        res.max_paths = max_paths
        res.field, res.p_coh_dbm, res.p_inc_dbm = field.ctypes.data, pc.ctypes.data, pi.ctypes.data
        res.paths = paths.ctypes.data
        rc = dcem_trace_links(self.h, tx, rx, params, res)
        if rc != OK and raise_on_error:
            raise DcemError(rc, "dcem_trace_links")
        n = min(res.n_paths, max_paths)
        return Frame(rc, (field[:nl, 0] + 1j * field[:nl, 1]).reshape(ntx, nrx), pc[:nl].reshape(ntx, nrx),
                     pi[:nl].reshape(ntx, nrx), paths[:n].copy(), stats_dict(res.stats))

    def update_transforms(self, xf):
        dcem_scene_update_transforms(self.h, xf)

    def trace(self, tx, rx, params: Params | None = None, max_paths: int | None = None,
              raise_on_error: bool = True) -> Frame:
        params = params or default_params()
        self.max_refl = int(params.max_refl)
        nrx = (rx.numel() if hasattr(rx, "numel") else np.asarray(rx).size) // 3
        if max_paths is None:
            max_paths = max(1024, 256 * nrx)
        field = np.empty((max(nrx, 1), 2), np.float64)
        pc = np.empty(max(nrx, 1), np.float64)
        pi = np.empty(max(nrx, 1), np.float64)
        paths = np.empty(max_paths, PATH_DTYPE)
        res = Result()
        res.ptr_kind = PTR_HOST
        res.max_paths = max_paths
        res.field, res.p_coh_dbm, res.p_inc_dbm = field.ctypes.data, pc.ctypes.data, pi.ctypes.data
        res.paths = paths.ctypes.data
        rc = dcem_trace_frame(self.h, tx, rx, params, res)
        if rc != OK and raise_on_error:
            raise DcemError(rc, "dcem_trace_frame")
        n = min(res.n_paths, max_paths)
        return Frame(rc, field[:nrx, 0] + 1j * field[:nrx, 1], pc[:nrx], pi[:nrx], paths[:n].copy(),
                     stats_dict(res.stats))

    def gradients(self, tx, rx, paths: np.ndarray, params: Params | None = None):
        """Field E (nrx,) complex, dE/dtheta (nrx, n_params) complex and
        d P_coh[dBm]/dtheta (nrx, n_params) for host PATH_DTYPE records;
        theta = eps_r, sigma per material, then x, y per object."""
        params = params or default_params()
        nrx = (rx.numel() if hasattr(rx, "numel") else np.asarray(rx).size) // 3
        npar = dcem_scene_gradient_size(self.h)
        field = np.zeros((max(nrx, 1), 2), np.float64)
        dfield = np.zeros((max(nrx, 1), max(npar, 1), 2), np.float64)
        dp = np.zeros((max(nrx, 1), max(npar, 1)), np.float64)
        paths = np.ascontiguousarray(paths, PATH_DTYPE)
        rc = dcem_path_gradients(self.h, tx, rx, paths, params, PTR_HOST, field.ctypes.data,
                                 dfield.ctypes.data, dp.ctypes.data)
        if rc != OK:
            raise DcemError(rc, "dcem_path_gradients")
        e = field[:nrx, 0] + 1j * field[:nrx, 1]
        de = dfield[:nrx, :npar, 0] + 1j * dfield[:nrx, :npar, 1]
        return e, de, dp[:nrx, :npar]

    def adjoint(self, tx, rx, paths: np.ndarray, params: Params | None = None, theta=None, pcoh_bar=None):
        """The adjoint kernel on host PATH_DTYPE records at theta (None: the
        scene's parameters): field E (nrx,) complex, P_coh [dBm] (nrx,),
        dE/dtheta (nrx, n_params) complex, d P_coh/dtheta (nrx, n_params) and,
        with pcoh_bar (nrx,), the vector-Jacobian product (n_params,)."""
        params = params or default_params()
        nrx = (rx.numel() if hasattr(rx, "numel") else np.asarray(rx).size) // 3
        npar = dcem_scene_gradient_size(self.h)
        field = np.zeros((max(nrx, 1), 2), np.float64)
        pc = np.zeros(max(nrx, 1), np.float64)
        dfield = np.zeros((max(nrx, 1), max(npar, 1), 2), np.float64)
        dp = np.zeros((max(nrx, 1), max(npar, 1)), np.float64)
        tb = np.zeros(max(npar, 1), np.float64)
        paths = np.ascontiguousarray(paths, PATH_DTYPE)
        th = None if theta is None else np.ascontiguousarray(theta, np.float64)
        pb = None if pcoh_bar is None else np.ascontiguousarray(pcoh_bar, np.float64)
        rc = dcem_path_adjoint(self.h, tx, rx, paths, params, PTR_HOST,
                               None if th is None else th.ctypes.data, None if pb is None else pb.ctypes.data,
                               field.ctypes.data, pc.ctypes.data, dfield.ctypes.data, dp.ctypes.data,
                               None if pb is None else tb.ctypes.data)
        if rc != OK:
            raise DcemError(rc, "dcem_path_adjoint")
        e = field[:nrx, 0] + 1j * field[:nrx, 1]
        de = dfield[:nrx, :npar, 0] + 1j * dfield[:nrx, :npar, 1]
        return e, pc[:nrx], de, dp[:nrx, :npar], (tb[:npar] if pb is not None else None)

    def theta(self, xf=None) -> np.ndarray:
        """The scene's parameters in the order of the derivatives: eps_r,
        sigma of every material, then the x, y translation of every object
        (from ``xf``, nobj x 12, the transforms last given)."""
        m = self.materials[:, :2].astype(np.float64).ravel()
        if self.nobj == 0:
            return m
        x = np.asarray(xf, np.float32).reshape(self.nobj, 12)
        return np.concatenate([m, np.stack([x[:, 3], x[:, 7]], 1).astype(np.float64).ravel()])

    def reset_cache(self):
        dcem_scene_reset_cache(self.h)

    def set_rebuild_threshold(self, ratio: float):
        dcem_scene_set_rebuild_threshold(self.h, ratio)

    def set_graph_replay(self, on: bool):
        dcem_scene_set_graph_replay(self.h, on)

    def set_transmission(self, loss_db, max_trans: int):
        """Per-material penetration loss [dB] (< 0 opaque) and transmissions per path."""
        dcem_scene_set_transmission(self.h, loss_db, max_trans)
        self.max_trans = int(max_trans)

    def set_diffraction(self, on: bool = True) -> int:
        """First-order edge diffraction paths (UTD); returns the wedge count."""
        return dcem_scene_set_diffraction(self.h, on)

    def set_diffraction_reflections(self, on: int = 1) -> int:
        """With diffraction on: reflections on static reflector planes around
        the diffraction, up to ``on`` (0-2; True is 1) around a first-order
        one, one before or after a chain; 3 adds one between the two wedges
        of an order-2 chain. Returns the reflector-plane count."""
        n = C.c_int32(0)
        _check(lib().dcem_scene_set_diffraction_reflections(self.h, int(on), C.byref(n)),
               "dcem_scene_set_diffraction_reflections")
        return int(n.value)

    def set_diffraction_order(self, max_order: int):
        """With diffraction on: paths over up to max_order (1-3) wedges."""
        _check(lib().dcem_scene_set_diffraction_order(self.h, int(max_order)), "dcem_scene_set_diffraction_order")

    def set_trace_config(self, kernel: int, block: int = 256, stack: int = 24):
        dcem_scene_set_trace_config(self.h, kernel, block, stack)

    def autotune(self, tx, rx, params: Params | None = None, reps: int = 2):
        return dcem_scene_autotune(self.h, tx, rx, params or default_params(), reps)

    def world_tris(self):
        return dcem_scene_get_world_tris(self.h, self.ntri)

    def bvh(self):
        return dcem_scene_get_bvh(self.h)

    def ray_log(self):
        """Primary rays' hit ids, distances (max_refl + max_trans + 1 segments) and segment counts."""
        return dcem_scene_get_ray_log(self.h, self.n_rays, self.max_refl + getattr(self, "max_trans", 0))

    def candidates(self):
        return dcem_scene_get_candidates(self.h)

    def info(self):
        return dcem_scene_info(self.h)

    def close(self):
        if getattr(self, "h", None):
            dcem_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several scenes traced together, one graph launch per frame (see
    dcem_batch_create in include/dcem.h). The scenes stay owned by the caller."""

    def __init__(self, scenes, stream=None):
        self.scenes = list(scenes)
        arr = (C.c_void_p * len(self.scenes))(*[x.h for x in self.scenes])
        h = C.c_void_p()
        _check(lib().dcem_batch_create(arr, len(self.scenes), stream, C.byref(h)), "dcem_batch_create")
        self.h = h

    def update_transforms(self, xfs):
        """xfs: one (nobj, 12) array per scene (None for static scenes), all host or all device."""
        keep, ptrs, kind = [], [], PTR_HOST
        for x in xfs:
            p, k, kp = _ptr(x, np.float32)
            keep.append(kp)
            ptrs.append(p)
            if x is not None:
                kind = k
        arr = (C.c_void_p * len(ptrs))(*ptrs)
        _check(lib().dcem_batch_update_transforms(self.h, arr, kind), "dcem_batch_update_transforms")

    def trace_raw(self, txs, rxs, params: Params, results):
        """txs: per scene an (ntx, 3) array; rxs: per scene receivers (all host or
        all device); results: per scene a Result. Returns (status, failed index)."""
        n = len(self.scenes)
        keep = []
        txa = [np.ascontiguousarray(t, np.float32).reshape(-1, 3) for t in txs]
        ntx = np.array([t.shape[0] for t in txa], np.int32)
        tptr = (C.c_void_p * n)(*[t.ctypes.data for t in txa])
        rptr, kind, nrx = [], PTR_HOST, []
        for r in rxs:
            p, k, kp = _ptr(r, np.float32)
            keep.append(kp)
            rptr.append(p)
            kind = k
            nrx.append((r.numel() if hasattr(r, "numel") else np.asarray(r).size) // 3)
        nrx = np.array(nrx, np.int32)
        rarr = (C.c_void_p * n)(*rptr)
        res = (Result * n)(*results)
        failed = C.c_int32(-1)
        rc = lib().dcem_batch_trace(self.h, tptr, ntx.ctypes.data, rarr, nrx.ctypes.data, kind, C.byref(params),
                                    res, C.byref(failed))
        for i in range(n):
            results[i] = res[i]
        return rc, failed.value

    def trace(self, txs, rxs, params: Params | None = None, max_paths: int | None = None):
        """One frame of every scene with host outputs: a list of Frame."""
        params = params or default_params()
        bufs, results = [], []
        for t, r in zip(txs, rxs):
            ntx = np.asarray(t).reshape(-1, 3).shape[0]
            nrx = (r.numel() if hasattr(r, "numel") else np.asarray(r).size) // 3
            nl = ntx * nrx
            mp = max_paths or max(1024, 256 * nl)
            b = (np.empty((max(nl, 1), 2)), np.empty(max(nl, 1)), np.empty(max(nl, 1)), np.empty(mp, PATH_DTYPE),
                 ntx, nrx)
            res = Result()
            res.ptr_kind = PTR_HOST
            res.max_paths = mp
            res.field, res.p_coh_dbm, res.p_inc_dbm = b[0].ctypes.data, b[1].ctypes.data, b[2].ctypes.data
            res.paths = b[3].ctypes.data
            bufs.append(b)
            results.append(res)
        rc, failed = self.trace_raw(txs, rxs, params, results)
        if rc != OK:
            raise DcemError(rc, f"dcem_batch_trace (scene {failed})")
        out = []
        for (field, pc, pi, paths, ntx, nrx), res in zip(bufs, results):
            nl = ntx * nrx
            n = min(res.n_paths, paths.shape[0])
            out.append(Frame(rc, (field[:nl, 0] + 1j * field[:nl, 1]).reshape(ntx, nrx), pc[:nl].reshape(ntx, nrx),
                             pi[:nl].reshape(ntx, nrx), paths[:n].copy(), stats_dict(res.stats)))
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().dcem_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def path_power(scene: Scene, theta, tx, rx, paths: np.ndarray, params: Params | None = None):
    """Received power P_coh [dBm] per receiver over a fixed path topology, as
    a differentiable function of theta for torch autograd.

    theta (a CUDA torch tensor of dcem_scene_gradient_size values, FP64) holds
    the parameters in the order of the derivatives: eps_r and sigma of every
    material, then the x and y translation of every rigid object (absolute;
    Scene.theta(xf) gives the scene's current values). The forward pass is the
    field of the paths' triangle sequences (Sec. III steps 3, 4 and 6, Eq. 1,
    Eq. 3) evaluated at theta by the library's adjoint kernel: materials
    replaced by theta's values and each object's triangles shifted by theta's
    translation minus its current one; the topology `paths` stays fixed and
    the scene is not modified. The backward pass runs the adjoint kernel again
    with the incoming gradient and returns the vector-Jacobian product it
    computes. Receivers without paths have P = -inf and no gradient. The work
    runs on theta's device, on that device's current stream."""
    import torch

    prm = params or default_params()
    nrx = (rx.numel() if hasattr(rx, "numel") else np.asarray(rx).size) // 3
    recs = np.ascontiguousarray(paths, PATH_DTYPE)

    class _PathPower(torch.autograd.Function):
        @staticmethod
        def forward(ctx, th):
            npar = dcem_scene_gradient_size(scene.h)
            if th.numel() != npar:
                raise DcemError(ERR_ARG, f"path_power: theta has {th.numel()} values, the scene {npar}")
            dev = th.device
            with torch.cuda.device(dev):
                thd = th.detach().to(torch.float64).contiguous()
                pd = torch.from_numpy(recs.view(np.uint8).copy()).to(dev)
                pc = torch.empty(max(nrx, 1), dtype=torch.float64, device=dev)
                # theta comes from torch's stream; the library's call ends with
                # a synchronisation of the scene's stream
                torch.cuda.current_stream(dev).synchronize()
                rc = dcem_path_adjoint(scene.h, tx, rx, pd.data_ptr(), prm, PTR_DEVICE, thd.data_ptr(), None,
                                       None, pc.data_ptr(), n_paths=recs.shape[0])
                if rc != OK:
                    raise DcemError(rc, "dcem_path_adjoint")
            ctx.save_for_backward(thd, pd)
            return pc[:nrx]

        @staticmethod
        def backward(ctx, g):
            thd, pd = ctx.saved_tensors
            dev = thd.device
            with torch.cuda.device(dev):
                gb = torch.zeros(max(nrx, 1), dtype=torch.float64, device=dev)
                gb[:nrx] = g.to(torch.float64)
                tb = torch.empty(thd.numel(), dtype=torch.float64, device=dev)
                torch.cuda.current_stream(dev).synchronize()
                rc = dcem_path_adjoint(scene.h, tx, rx, pd.data_ptr(), prm, PTR_DEVICE, thd.data_ptr(),
                                       gb.data_ptr(), theta_bar_ptr=tb.data_ptr(), n_paths=recs.shape[0])
                if rc != OK:
                    raise DcemError(rc, "dcem_path_adjoint")
            return tb.to(theta.dtype).reshape(theta.shape)

    return _PathPower.apply(theta)
