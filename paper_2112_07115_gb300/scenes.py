"""Seeded synthetic workloads for the dynamic EM ray tracer.

This module only *generates inputs*: triangle meshes, materials, per-frame
rigid transforms (3x4, row major), transmitter and receiver positions, and the
sampled sphere of ray directions. It contains none of the tracer's arithmetic
(no transform application, intersection, reflection, capture, image method or
field computation), so both the CUDA path and the CPU oracle consume exactly
the same FP32 bits from here.

Workloads:
  * ``toy_street``  -- ground, two buildings, four moving PEC vehicles, 8 Rx,
    28 GHz, 10k rays, 3 reflections, 10 frames at 10 Hz.
  * ``highway``     -- 2 km six-lane road with concrete barriers, 200 vehicles
    of three box classes with lane changes, one roadside Tx, one Rx per
    vehicle roof, 1M rays, 4 reflections, 100 frames at 10 Hz.
  * ``urban_grid``  -- Manhattan grid of blocks with extruded-polygon
    buildings (four static material classes), moving vehicles on four-lane
    streets, many roadside Tx with uneven ray budgets, four roof Rx per
    vehicle plus static roadside Rx (the batched multi-transmitter workload).
  * ``scene_batch`` -- independent urban grids of very different sizes (1k-200k
    triangles, 10-2000 vehicles, 1-16 Tx with uneven budgets) traced together.
  * ``office``      -- an indoor floor of rooms with Table II walls (20 dB) and
    glass windows (5 dB), moving metal carts, Tx at 2 m, 30 GHz (transmission).
  * small closed-form scenes (ground plane, parallel plates, random triangles).

The paper (Sec. III) uses an .obj town model and measurement campaigns that
are not available; these seeded scenes stand in for its vehicular workloads.
Material constants: concrete eps_r=5.31, sigma=0.0326 S/m; vehicles are
perfect conductors ("metal").
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

MAT_CONCRETE = 0
MAT_METAL = 1


def default_materials() -> np.ndarray:
    """Material table rows: (eps_r, sigma [S/m], pec flag)."""
    return np.array([[5.31, 0.0326, 0.0],   # concrete: ground, buildings, barriers
                     [1.0, 0.0, 1.0]],      # metal: vehicles (perfect conductor)
                    dtype=np.float32)


@dataclass
class Scene:
    """A dynamic scene plus the radio set-up for a sequence of frames.

    tris     float32 (T,3,3)  vertex coordinates; world space when
                              tri_obj == -1, object space otherwise
    tri_obj  int32 (T,)       -1 for static geometry, else rigid-object id
    tri_mat  int32 (T,)       row of ``materials``
    materials float32 (M,3)   (eps_r, sigma, pec)
    xf       float32 (F,nobj,12) per-frame row-major 3x4 [R | t]
    tx       float32 (3,)     transmitter (static)
    rx       float32 (F,nrx,3) receivers per frame
    """
    name: str
    tris: np.ndarray
    tri_obj: np.ndarray
    tri_mat: np.ndarray
    materials: np.ndarray
    nobj: int
    xf: np.ndarray
    tx: np.ndarray
    rx: np.ndarray
    freq_hz: float = 28e9
    n_rays: int = 10_000
    max_refl: int = 3
    meta: dict = field(default_factory=dict)

    @property
    def ntri(self) -> int:
        return int(self.tris.shape[0])

    @property
    def nframes(self) -> int:
        return int(self.xf.shape[0])

    @property
    def nrx(self) -> int:
        return int(self.rx.shape[1])


# ----------------------------------------------------------------------------
# ray directions
# ----------------------------------------------------------------------------

def fibonacci_sphere(n: int) -> np.ndarray:
    """n unit directions on a Fibonacci lattice, computed in FP64, rounded once to FP32.

    z_i = 1 - (2i+1)/n, phi_i = i*pi*(3 - sqrt 5). This is the "sphere of
    sampled rays" that the tracer casts (Sec. III, backward ray tracing, step 1).
    """
    if n <= 0:
        return np.zeros((0, 3), np.float32)
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * (np.pi * (3.0 - np.sqrt(5.0)))
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    return d.astype(np.float32)


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------

def _quad(a, b, c, d):
    """Two triangles (a,b,c), (a,c,d) of the planar quad a-b-c-d."""
    return [[a, b, c], [a, c, d]]


def box_tris(lx, ly, lz, center=(0.0, 0.0, 0.0), faces=("top", "xm", "xp", "ym", "yp")):
    """Triangles of an axis-aligned box [cx-lx/2,cx+lx/2] x [cy-ly/2,..] x [cz, cz+lz].

    ``faces`` chooses which faces to emit (bottom is omitted by default: it
    rests on the ground and no ray can reach it).
    """
    cx, cy, cz = center
    x0, x1 = cx - lx / 2, cx + lx / 2
    y0, y1 = cy - ly / 2, cy + ly / 2
    z0, z1 = cz, cz + lz
    out = []
    if "top" in faces:
        out += _quad((x0, y0, z1), (x1, y0, z1), (x1, y1, z1), (x0, y1, z1))
    if "bottom" in faces:
        out += _quad((x0, y0, z0), (x0, y1, z0), (x1, y1, z0), (x1, y0, z0))
    if "xm" in faces:
        out += _quad((x0, y0, z0), (x0, y0, z1), (x0, y1, z1), (x0, y1, z0))
    if "xp" in faces:
        out += _quad((x1, y0, z0), (x1, y1, z0), (x1, y1, z1), (x1, y0, z1))
    if "ym" in faces:
        out += _quad((x0, y0, z0), (x1, y0, z0), (x1, y0, z1), (x0, y0, z1))
    if "yp" in faces:
        out += _quad((x0, y1, z0), (x0, y1, z1), (x1, y1, z1), (x1, y1, z0))
    return out


def _xf_row(yaw: float, tx: float, ty: float, tz: float) -> np.ndarray:
    """Row-major 3x4 [R|t] of a rotation about +z by ``yaw`` then a translation."""
    c, s = np.cos(yaw), np.sin(yaw)
    return np.array([c, -s, 0.0, tx,
                     s, c, 0.0, ty,
                     0.0, 0.0, 1.0, tz], dtype=np.float64)


def _assemble(static_tris, static_mat, obj_meshes, obj_mat):
    tris, tobj, tmat = [], [], []
    for t, m in zip(static_tris, static_mat):
        tris.append(t)
        tobj.append(-1)
        tmat.append(m)
    for k, mesh in enumerate(obj_meshes):
        for t in mesh:
            tris.append(t)
            tobj.append(k)
            tmat.append(obj_mat[k])
    return (np.asarray(tris, np.float32).reshape(-1, 3, 3),
            np.asarray(tobj, np.int32), np.asarray(tmat, np.int32))


# ----------------------------------------------------------------------------
# toy street (58 triangles)
# ----------------------------------------------------------------------------

def toy_street(seed: int = 0, n_frames: int = 10, n_rays: int = 10_000,
               max_refl: int = 3, freq_hz: float = 28e9) -> Scene:
    """Toy street: 2 ground tris, two 20x20x15 m buildings (walls only, 8 tris each),
    four 4.5x1.8x1.5 m PEC vehicles (10 tris each) at 15 m/s, Tx at (0,12,6),
    8 Rx at 1.5 m along y = +-12. 58 triangles, 10 frames at 10 Hz.

    The seed jitters the vehicles' start positions by up to +-1 m so that
    different seeds give different geometry; seed 0 is the nominal layout.
    """
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 1])))
    static, smat = [], []
    static += _quad((-100, -100, 0), (100, -100, 0), (100, 100, 0), (-100, 100, 0))
    smat += [MAT_CONCRETE] * 2
    for (bx, by) in [(-30.0, 25.0), (30.0, -25.0)]:
        walls = box_tris(20, 20, 15, (bx, by, 0.0), faces=("xm", "xp", "ym", "yp"))
        static += walls
        smat += [MAT_CONCRETE] * len(walls)
    veh = box_tris(4.5, 1.8, 1.5)
    lanes = [-6.0, -2.0, 2.0, 6.0]
    x0 = np.array([-40.0, -10.0, 10.0, 40.0])
    if seed != 0:
        x0 = x0 + rng.uniform(-1.0, 1.0, size=4)
    vdir = np.array([-1.0, -1.0, 1.0, 1.0])  # y<0 lanes drive -x, y>0 lanes +x
    tris, tobj, tmat = _assemble(static, smat, [veh] * 4, [MAT_METAL] * 4)
    dt, v = 0.1, 15.0
    xf = np.zeros((n_frames, 4, 12), np.float64)
    for f in range(n_frames):
        for k in range(4):
            yaw = 0.0 if vdir[k] > 0 else np.pi
            xf[f, k] = _xf_row(yaw, x0[k] + vdir[k] * v * dt * f, lanes[k], 0.0)
    rx1 = np.array([[x, y, 1.5] for y in (-12.0, 12.0) for x in (-36.0, -12.0, 12.0, 36.0)])
    rx = np.broadcast_to(rx1, (n_frames, 8, 3)).astype(np.float32).copy()
    return Scene("toy_street", tris, tobj, tmat, default_materials(), 4,
                 xf.astype(np.float32), np.array([0.0, 12.0, 6.0], np.float32), rx,
                 freq_hz=freq_hz, n_rays=n_rays, max_refl=max_refl,
                 meta={"seed": seed, "dt": dt})


# ----------------------------------------------------------------------------
# highway V2I (about 4.0k triangles)
# ----------------------------------------------------------------------------

HW_LENGTH = 2000.0
HW_PIECE = 20.0
HW_LANE_W = 3.75
HW_LANES = [4.375 + HW_LANE_W * k for k in range(3)]        # carriageway y>0 (drives +x)
HW_BARRIER_Y = [-14.75, 0.0, 14.75]
VEH_CLASSES = {  # length, width, height
    "car": (4.5, 1.8, 1.5),
    "van": (6.0, 2.2, 2.5),
    "truck": (12.0, 2.5, 4.0),
}


def highway(seed: int = 0, n_frames: int = 100, n_vehicles: int = 200,
            n_rays: int = 1_000_000, max_refl: int = 4, freq_hz: float = 28e9,
            length: float = HW_LENGTH, roadside_rx: int = 0) -> Scene:
    """Highway V2I: straight 6-lane road (30 m wide, 20 m tessellation), three
    2 m x 0.5 m concrete barriers (road edges and median), ``n_vehicles``
    vehicles (70% car, 20% van, 10% truck, 10 tris each) at U[20,35] m/s with
    Poisson(0.05/s) lane changes along a 3 s cosine profile, a 10 m gap rule,
    and wrap-around at the road ends. Tx at (L/2, 20, 8); one Rx 0.1 m above
    each vehicle roof. Frames at 10 Hz. With ``roadside_rx`` > 0 the
    receivers are that many static roadside units instead, 2.5 m high and 2 m
    beyond the outer barriers, evenly spaced along both road edges.
    """
    ss = np.random.SeedSequence([seed, 2])
    r_layout, r_speed, r_lc = [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(3)]
    npieces = int(round(length / HW_PIECE))
    static, smat = [], []
    for p in range(npieces):
        xa, xb = p * HW_PIECE, (p + 1) * HW_PIECE
        static += _quad((xa, -15.0, 0.0), (xb, -15.0, 0.0), (xb, 15.0, 0.0), (xa, 15.0, 0.0))
        smat += [MAT_CONCRETE] * 2
    for by in HW_BARRIER_Y:
        for p in range(npieces):
            xa = p * HW_PIECE
            b = box_tris(HW_PIECE, 0.5, 2.0, (xa + HW_PIECE / 2, by, 0.0), faces=("top", "ym", "yp"))
            static += b
            smat += [MAT_CONCRETE] * len(b)
    # vehicles
    u = r_layout.uniform(size=n_vehicles)
    cls = np.where(u < 0.7, 0, np.where(u < 0.9, 1, 2))
    names = ["car", "van", "truck"]
    dims = np.array([VEH_CLASSES[names[c]] for c in cls])
    lane_y = np.array(HW_LANES + [-y for y in HW_LANES])          # 6 lanes
    lane = r_layout.integers(0, 6, size=n_vehicles)
    # place vehicles per lane with at least (length + 10 m) spacing
    x = np.zeros(n_vehicles)
    for ln in range(6):
        idx = np.nonzero(lane == ln)[0]
        if len(idx) == 0:
            continue
        need = dims[idx, 0] + 10.0
        free = length - need.sum()
        if free < 0:
            raise ValueError("too many vehicles for the road length")
        gaps = r_layout.dirichlet(np.ones(len(idx) + 1)) * free
        pos = r_layout.uniform(0, length)
        order = r_layout.permutation(len(idx))
        cur = pos
        for j, k in enumerate(order):
            cur += gaps[j]
            x[idx[k]] = (cur + need[k] / 2) % length
            cur += need[k]
    speed0 = r_speed.uniform(20.0, 35.0, size=n_vehicles)
    meshes = [box_tris(*dims[k]) for k in range(n_vehicles)]
    tris, tobj, tmat = _assemble(static, smat, meshes, [MAT_METAL] * n_vehicles)

    dt, t_lc = 0.1, 3.0
    y = lane_y[lane].astype(np.float64).copy()
    sgn = np.where(lane < 3, 1.0, -1.0)           # +x on y>0 carriageway
    lc_from = y.copy()
    lc_to = y.copy()
    lc_t = np.full(n_vehicles, -1.0)               # time into current lane change (<0: none)
    xf = np.zeros((n_frames, n_vehicles, 12), np.float64)
    rx = np.zeros((n_frames, n_vehicles, 3), np.float64)
    for f in range(n_frames):
        vy = np.zeros(n_vehicles)
        active = lc_t >= 0
        if np.any(active):
            ph = np.clip(lc_t[active] / t_lc, 0.0, 1.0)
            y[active] = lc_from[active] + (lc_to[active] - lc_from[active]) * 0.5 * (1 - np.cos(np.pi * ph))
            vy[active] = ((lc_to[active] - lc_from[active]) * 0.5 * np.pi / t_lc
                          * np.sin(np.pi * ph))
        vx = sgn * speed0
        yaw = np.arctan2(vy, vx)
        for k in range(n_vehicles):
            xf[f, k] = _xf_row(yaw[k], x[k], y[k], 0.0)
        rx[f, :, 0] = x
        rx[f, :, 1] = y
        rx[f, :, 2] = dims[:, 2] + 0.1
        # --- advance dynamics to the next frame ---
        eff = speed0.copy()
        for ln_sign in (1.0, -1.0):                 # gap rule per carriageway & lane
            sel = np.nonzero(sgn == ln_sign)[0]
            for ly in lane_y[(lane_y > 0) if ln_sign > 0 else (lane_y < 0)]:
                inl = sel[np.abs(y[sel] - ly) < HW_LANE_W / 2]
                if len(inl) < 2:
                    continue
                order = inl[np.argsort(x[inl] * ln_sign)]
                for a, b in zip(order[:-1], order[1:]):
                    gap = (x[b] - x[a]) * ln_sign - (dims[a, 0] + dims[b, 0]) / 2
                    if gap < 10.0:
                        eff[a] = min(eff[a], eff[b])
        x = (x + sgn * eff * dt) % length
        lc_t[active] += dt
        done = active & (lc_t > t_lc)
        y[done] = lc_to[done]
        lc_t[done] = -1.0
        start = (lc_t < 0) & (r_lc.uniform(size=n_vehicles) < 1.0 - np.exp(-0.05 * dt))
        for k in np.nonzero(start)[0]:
            same = lane_y[(lane_y * sgn[k]) > 0]
            cur = same[np.argmin(np.abs(same - y[k]))]
            nb = same[np.abs(np.abs(same - cur) - HW_LANE_W) < 1e-6]
            if len(nb) == 0:
                continue
            lc_from[k] = cur
            lc_to[k] = nb[r_lc.integers(0, len(nb))]
            lc_t[k] = 0.0
    if roadside_rx > 0:
        half = (roadside_rx + 1) // 2
        yo = max(abs(b) for b in HW_BARRIER_Y) + 2.0
        pts = []
        for side, cnt in ((1.0, half), (-1.0, roadside_rx - half)):
            xs = (np.arange(cnt) + 0.5) * (length / cnt)
            pts += [(xx, side * yo, 2.5) for xx in xs]
        rx = np.broadcast_to(np.asarray(pts, np.float64), (n_frames, roadside_rx, 3)).copy()
    return Scene("highway", tris, tobj, tmat, default_materials(), n_vehicles,
                 xf.astype(np.float32), np.array([length / 2, 20.0, 8.0], np.float32),
                 rx.astype(np.float32), freq_hz=freq_hz, n_rays=n_rays, max_refl=max_refl,
                 meta={"seed": seed, "dt": dt, "classes": cls.tolist()})


# ----------------------------------------------------------------------------
# urban grid (batched transmitters)
# ----------------------------------------------------------------------------

# Static material classes of the urban grid, rows of ``urban_materials``:
# concrete (the configs' value), brick, glass, ground; vehicles are metal.
# Brick/glass/ground are ITU-R P.2040-style constants chosen for the build.
URBAN_CONCRETE, URBAN_BRICK, URBAN_GLASS, URBAN_GROUND, URBAN_METAL = range(5)


def urban_materials() -> np.ndarray:
    return np.array([[5.31, 0.0326, 0.0],    # concrete
                     [3.75, 0.038, 0.0],     # brick
                     [6.27, 0.0043, 0.0],    # glass
                     [15.0, 0.035, 0.0],     # ground
                     [1.0, 0.0, 1.0]],       # metal (vehicles)
                    dtype=np.float32)


def urban_grad_materials() -> np.ndarray:
    """Eight (eps_r, sigma) classes for the differentiable urban workload:
    seven building materials and the ground, then metal for the vehicles.
    Concrete is the configs' value; the others are this build's choice of
    ITU-R P.2040-style constants."""
    return np.array([[5.31, 0.0326, 0.0],    # concrete
                     [3.75, 0.038, 0.0],     # brick
                     [6.27, 0.0043, 0.0],    # glass
                     [2.73, 0.0085, 0.0],    # plasterboard
                     [1.99, 0.0047, 0.0],    # wood
                     [7.51, 0.030, 0.0],     # limestone
                     [7.07, 0.0055, 0.0],    # marble
                     [15.0, 0.035, 0.0],     # ground
                     [1.0, 0.0, 1.0]],       # metal (vehicles)
                    dtype=np.float32)


def _extruded_polygon(cx, cy, rmax, n, h, rng):
    """Walls (2 triangles per edge) and a roof fan of a star-shaped polygon of
    n vertices around (cx, cy), radii in [0.55, 1] rmax, extruded to height h."""
    ang = np.sort(rng.uniform(0.0, 2.0 * np.pi, size=n))
    rad = rng.uniform(0.55, 1.0, size=n) * rmax
    px, py = cx + rad * np.cos(ang), cy + rad * np.sin(ang)
    out = []
    for k in range(n):
        a, b = k, (k + 1) % n
        out += _quad((px[a], py[a], 0.0), (px[b], py[b], 0.0), (px[b], py[b], h), (px[a], py[a], h))
        out.append([(cx, cy, h), (px[a], py[a], h), (px[b], py[b], h)])
    return out


def urban_grid(seed: int = 0, blocks: int = 10, pitch: float = 100.0, street: float = 20.0,
               parcels: int = 4, n_vehicles: int = 1000, n_tx: int = 64,
               budgets: tuple = (65_536, 2_097_152), n_static_rx: int = 96, n_frames: int = 200,
               max_refl: int = 5, freq_hz: float = 28e9, building_classes: int = 3) -> Scene:
    """Manhattan grid: ``blocks`` x ``blocks`` blocks at ``pitch`` m with
    ``street`` m streets (street centre lines at x = i * pitch and
    y = j * pitch, i, j = 0..blocks). Each block holds ``parcels`` x
    ``parcels`` buildings: star-shaped polygons of 6-14 vertices extruded to
    U[10, 60] m, each of concrete, brick or glass. Ground of 25 m tiles.
    Vehicles (car/van/truck boxes as on the highway, metal) drive on four
    lanes per street (two each way, 2.5 m and 7.5 m from the centre line) at
    a per-lane speed U[5, 15] m/s with equal spacing and wrap-around, so they
    never overlap. Receivers: the four roof corners of every vehicle (0.2 m
    in, 0.1 m above the roof), then ``n_static_rx`` roadside receivers at
    2 m. Transmitters: ``n_tx`` roadside units at random street corners,
    6-10 m high, with ray budgets log-uniform in ``budgets`` (returned in
    ``meta["tx"]`` and ``meta["budgets"]``; ``tx`` is the first one).
    Frames at 10 Hz. building_classes 7 takes the eight-class table of
    urban_grad_materials (seven building classes, then ground and metal).
    """
    if building_classes == 3:
        mats, m_ground, m_metal = urban_materials(), URBAN_GROUND, URBAN_METAL
    elif building_classes == 7:
        mats, m_ground, m_metal = urban_grad_materials(), 7, 8
    else:
        raise ValueError("building_classes is 3 or 7")
    ss = np.random.SeedSequence([seed, 3])
    r_bld, r_veh, r_tx = [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(3)]
    size = blocks * pitch
    static, smat = [], []
    tile = 25.0
    nt = int(round((size + street) / tile))
    for i in range(nt):
        for j in range(nt):
            x0, y0 = -street / 2 + i * tile, -street / 2 + j * tile
            static += _quad((x0, y0, 0.0), (x0 + tile, y0, 0.0), (x0 + tile, y0 + tile, 0.0), (x0, y0 + tile, 0.0))
            smat += [m_ground] * 2
    lot = pitch - street
    cell = lot / parcels
    for bi in range(blocks):
        for bj in range(blocks):
            for pi in range(parcels):
                for pj in range(parcels):
                    cx = bi * pitch + street / 2 + (pi + 0.5) * cell
                    cy = bj * pitch + street / 2 + (pj + 0.5) * cell
                    n = int(r_bld.integers(6, 15))
                    h = float(r_bld.uniform(10.0, 60.0))
                    m = int(r_bld.integers(0, building_classes))
                    b = _extruded_polygon(cx, cy, 0.45 * cell, n, h, r_bld)
                    static += b
                    smat += [m] * len(b)
    # vehicles: lanes along x (streets y = j * pitch) and along y (x = i * pitch)
    lanes = []
    for axis in (0, 1):
        for k in range(blocks + 1):
            for off, sgn in ((-7.5, -1.0), (-2.5, -1.0), (2.5, 1.0), (7.5, 1.0)):
                lanes.append((axis, k * pitch + off, sgn))
    lane_of = r_veh.integers(0, len(lanes), size=n_vehicles)
    u = r_veh.uniform(size=n_vehicles)
    cls = np.where(u < 0.7, 0, np.where(u < 0.9, 1, 2))
    names = ["car", "van", "truck"]
    dims = np.array([VEH_CLASSES[names[c]] for c in cls])
    s0 = np.zeros(n_vehicles)
    speed = np.zeros(n_vehicles)
    span = size + street
    for ln in range(len(lanes)):
        idx = np.nonzero(lane_of == ln)[0]
        if len(idx) == 0:
            continue
        gap = span / len(idx)
        if gap < 25.0:
            raise ValueError("too many vehicles for the lanes")
        phase = r_veh.uniform(0.0, gap)
        s0[idx] = phase + gap * np.arange(len(idx)) + r_veh.uniform(-0.2, 0.2, size=len(idx)) * (gap - 20.0)
        speed[idx] = r_veh.uniform(5.0, 15.0)
    meshes = [box_tris(*dims[k]) for k in range(n_vehicles)]
    tris, tobj, tmat = _assemble(static, smat, meshes, [m_metal] * n_vehicles)
    dt = 0.1
    xf = np.zeros((n_frames, n_vehicles, 12), np.float64)
    nrx = 4 * n_vehicles + n_static_rx
    rx = np.zeros((n_frames, nrx, 3), np.float64)
    corners = np.array([[1, 1], [1, -1], [-1, 1], [-1, -1]], np.float64)
    for f in range(n_frames):
        for k in range(n_vehicles):
            axis, c, sgn = lanes[lane_of[k]]
            along = (s0[k] + sgn * speed[k] * dt * f) % span - street / 2
            if axis == 0:
                x, y, yaw = along, c, (0.0 if sgn > 0 else np.pi)
            else:
                x, y, yaw = c, along, (np.pi / 2 if sgn > 0 else -np.pi / 2)
            xf[f, k] = _xf_row(yaw, x, y, 0.0)
            cy_, sy_ = np.cos(yaw), np.sin(yaw)
            lx, ly, lz = dims[k, 0] / 2 - 0.2, dims[k, 1] / 2 - 0.2, dims[k, 2] + 0.1
            for q, (a, b) in enumerate(corners):
                px, py = a * lx, b * ly
                rx[f, 4 * k + q] = (x + cy_ * px - sy_ * py, y + sy_ * px + cy_ * py, lz)
    # static roadside receivers and the transmitters, at street corners
    def corner_points(n, rng, hlo, hhi):
        ii = rng.integers(0, blocks + 1, size=n)
        jj = rng.integers(0, blocks + 1, size=n)
        sx = rng.choice([-1.0, 1.0], size=n)
        sy = rng.choice([-1.0, 1.0], size=n)
        return np.stack([ii * pitch + sx * (street / 2 - 1.0), jj * pitch + sy * (street / 2 - 1.0),
                         rng.uniform(hlo, hhi, size=n)], 1)
    rx[:, 4 * n_vehicles:] = corner_points(n_static_rx, r_tx, 2.0, 2.0)[None]
    txs = corner_points(n_tx, r_tx, 6.0, 10.0).astype(np.float32)
    lo, hi = np.log(budgets[0]), np.log(budgets[1])
    bud = np.exp(r_tx.uniform(lo, hi, size=n_tx)).astype(np.int64)
    return Scene("urban_grid", tris, tobj, tmat, mats, n_vehicles,
                 xf.astype(np.float32), txs[0].copy(), rx.astype(np.float32), freq_hz=freq_hz,
                 n_rays=int(bud[0]), max_refl=max_refl,
                 meta={"seed": seed, "dt": dt, "tx": txs, "budgets": bud.tolist(), "classes": cls.tolist()})


def urban_gradient(seed: int = 0, blocks: int = 10, parcels: int = 4, n_vehicles: int = 1000, n_rx: int = 256,
                   n_rays: int = 1_000_000, max_refl: int = 4, n_frames: int = 3, freq_hz: float = 28e9) -> Scene:
    """The differentiable-tracing workload: the urban grid with eight
    (eps_r, sigma) classes (urban_grad_materials), its moving metal vehicles,
    one roadside transmitter with ``n_rays`` rays, and ``n_rx`` static
    roadside receivers at 2 m (the grid's static receivers; the roof
    receivers are dropped)."""
    sc = urban_grid(seed=seed, blocks=blocks, parcels=parcels, n_vehicles=n_vehicles, n_tx=1,
                    budgets=(n_rays, n_rays), n_static_rx=n_rx, n_frames=n_frames, max_refl=max_refl,
                    freq_hz=freq_hz, building_classes=7)
    sc.rx = np.ascontiguousarray(sc.rx[:, 4 * n_vehicles:])
    sc.n_rays = n_rays
    sc.name = "urban_gradient"
    return sc


def city_blocks(n: int = 8, pitch: float = 30.0, seed: int = 0, n_rx: int = 64, n_rays: int = 200_000,
                max_refl: int = 3, freq_hz: float = 28e9) -> Scene:
    """A grid of n x n box buildings (footprints U[10, 20] m per side, heights
    U[8, 40] m, concrete, roofs included, so every building has four vertical
    and four roof wedges) at ``pitch`` spacing on a concrete ground, one
    transmitter at 10 m in a street near the centre and ``n_rx`` receivers at
    1.5 m, uniform over the grid (some fall inside buildings and receive
    nothing). The workload of multi-order diffraction: street corners and
    rooftops. One static frame."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 7])))
    side = n * pitch
    tris = _quad((-50.0, -50.0, 0.0), (side + 50.0, -50.0, 0.0), (side + 50.0, side + 50.0, 0.0),
                 (-50.0, side + 50.0, 0.0))
    mats = [MAT_CONCRETE] * len(tris)
    for i in range(n):
        for j in range(n):
            b = box_tris(rng.uniform(10.0, 20.0), rng.uniform(10.0, 20.0), rng.uniform(8.0, 40.0),
                         center=(i * pitch + pitch / 2, j * pitch + pitch / 2, 0.0))
            tris += b
            mats += [MAT_CONCRETE] * len(b)
    tx = (side / 2 + 2.0, side / 2 + 15.0, 10.0)
    rx = [(rng.uniform(0.0, side), rng.uniform(0.0, side), 1.5) for _ in range(n_rx)]
    return _static_scene("city_blocks", tris, mats, tx, rx, n_rays=n_rays, max_refl=max_refl, freq_hz=freq_hz)


def scene_batch(seed: int = 0, n: int = 32, tris: tuple = (1_000, 200_000), vehicles: tuple = (10, 2000),
                tx_per_scene: tuple = (1, 16), budgets: tuple = (16_384, 524_288), n_frames: int = 10,
                max_refl: int = 4, freq_hz: float = 28e9):
    """``n`` independent urban-grid scenes for a multi-scene batch: triangle
    targets log-uniform in ``tris`` (blocks and buildings per block chosen to
    approach them), vehicles log-uniform in ``vehicles`` (capped at 30% of the
    lanes' room), 1-16 roadside transmitters each with ray budgets
    log-uniform in ``budgets``. Returns a list of Scene (``meta["tx"]``,
    ``meta["budgets"]`` as in ``urban_grid``)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 4])))
    out = []
    for i in range(n):
        target = float(np.exp(rng.uniform(np.log(tris[0]), np.log(tris[1]))))
        best = None
        for b in range(2, 15):
            for p in range(1, 9):
                est = 30.0 * b * b * p * p + 2.0 * ((100.0 * b + 20.0) / 25.0) ** 2
                err = abs(np.log(est / target))
                if best is None or err < best[0]:
                    best = (err, b, p)
        _, b, p = best
        room = int(0.3 * 8 * (b + 1) * (100.0 * b + 20.0) / 25.0)
        nv = int(min(room, np.exp(rng.uniform(np.log(vehicles[0]), np.log(vehicles[1])))))
        ntx = int(rng.integers(tx_per_scene[0], tx_per_scene[1] + 1))
        out.append(urban_grid(seed=1000 * seed + i, blocks=b, parcels=p, n_vehicles=nv, n_tx=ntx, budgets=budgets,
                              n_static_rx=8, n_frames=n_frames, max_refl=max_refl, freq_hz=freq_hz))
    return out


# ----------------------------------------------------------------------------
# indoor office (transmission)
# ----------------------------------------------------------------------------

# Office materials: rows of ``office_materials``; penetration losses (Table
# II: indoor wall 20 dB, glass 5 dB) in ``meta["trans_db"]``.
OFFICE_SLAB, OFFICE_WALL, OFFICE_GLASS, OFFICE_METAL = range(4)


def office_materials() -> np.ndarray:
    return np.array([[5.31, 0.0326, 0.0],    # floor and ceiling slabs (opaque)
                     [5.31, 0.0326, 0.0],    # indoor walls (Table II: 20 dB)
                     [6.27, 0.0043, 0.0],    # glass (Table II: 5 dB)
                     [1.0, 0.0, 1.0]],       # metal carts
                    dtype=np.float32)


def office(seed: int = 0, rooms_x: int = 4, rooms_y: int = 3, room=(6.0, 5.0), height: float = 3.0,
           n_carts: int = 4, rx_per_room: int = 4, n_frames: int = 10, n_rays: int = 1_000_000,
           max_refl: int = 2, max_trans: int = 2, freq_hz: float = 30e9) -> Scene:
    """An office floor of rooms_x x rooms_y rooms (room[0] x room[1] m, 3 m
    high): floor and ceiling slabs, interior walls (Table II indoor wall,
    20 dB), exterior walls with a 2 m glass window per room side (Table II
    glass, 5 dB), and ``n_carts`` metal carts (1.2 x 0.6 x 1 m) moving across
    the floor at 1 m/s. Tx at 2 m in the first room (the paper's indoor
    set-up: 2 m, 30 GHz, 0.5 W), ``rx_per_room`` receivers at 1.5 m in every
    room. ``meta["trans_db"]`` holds the per-material penetration losses
    (-1 = opaque) and ``meta["max_trans"]`` the transmissions per path."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 5])))
    W, H = rooms_x * room[0], rooms_y * room[1]
    static, smat = [], []
    for i in range(rooms_x):
        for j in range(rooms_y):
            x0, y0 = i * room[0], j * room[1]
            x1, y1 = x0 + room[0], y0 + room[1]
            static += _quad((x0, y0, 0.0), (x1, y0, 0.0), (x1, y1, 0.0), (x0, y1, 0.0))
            static += _quad((x0, y0, height), (x0, y1, height), (x1, y1, height), (x1, y0, height))
            smat += [OFFICE_SLAB] * 4

    def wall_x(x, ya, yb, window):
        # a wall in the plane x between y = ya and yb; a window pane in the middle
        out, mats = [], []
        if window:
            ym = 0.5 * (ya + yb)
            for a, b in ((ya, ym - 1.0), (ym + 1.0, yb)):
                out += _quad((x, a, 0.0), (x, b, 0.0), (x, b, height), (x, a, height))
                mats += [OFFICE_WALL] * 2
            out += _quad((x, ym - 1.0, 0.0), (x, ym + 1.0, 0.0), (x, ym + 1.0, 1.0), (x, ym - 1.0, 1.0))
            out += _quad((x, ym - 1.0, 2.5), (x, ym + 1.0, 2.5), (x, ym + 1.0, height), (x, ym - 1.0, height))
            mats += [OFFICE_WALL] * 4
            out += _quad((x, ym - 1.0, 1.0), (x, ym + 1.0, 1.0), (x, ym + 1.0, 2.5), (x, ym - 1.0, 2.5))
            mats += [OFFICE_GLASS] * 2
        else:
            out += _quad((x, ya, 0.0), (x, yb, 0.0), (x, yb, height), (x, ya, height))
            mats += [OFFICE_WALL] * 2
        return out, mats

    def swap_xy(tris):
        return [[(p[1], p[0], p[2]) for p in t] for t in tris]

    for i in range(rooms_x + 1):
        for j in range(rooms_y):
            t, m = wall_x(i * room[0], j * room[1], (j + 1) * room[1], i in (0, rooms_x))
            static += t
            smat += m
    for j in range(rooms_y + 1):
        for i in range(rooms_x):
            t, m = wall_x(j * room[1], i * room[0], (i + 1) * room[0], j in (0, rooms_y))
            static += swap_xy(t)
            smat += m
    meshes = [box_tris(1.2, 0.6, 1.0) for _ in range(n_carts)]
    tris, tobj, tmat = _assemble(static, smat, meshes, [OFFICE_METAL] * n_carts)
    # carts: straight lines across the floor, reflected at the outer walls
    pos = np.stack([rng.uniform(1.0, W - 1.0, n_carts), rng.uniform(1.0, H - 1.0, n_carts)], 1)
    ang = rng.uniform(0.0, 2.0 * np.pi, n_carts)
    vel = np.stack([np.cos(ang), np.sin(ang)], 1)
    dt = 0.1
    xf = np.zeros((n_frames, n_carts, 12), np.float64)
    for f in range(n_frames):
        for k in range(n_carts):
            xf[f, k] = _xf_row(float(np.arctan2(vel[k, 1], vel[k, 0])), pos[k, 0], pos[k, 1], 0.0)
        pos += vel * dt
        for ax, lim in ((0, W), (1, H)):
            out = (pos[:, ax] < 0.8) | (pos[:, ax] > lim - 0.8)
            vel[out, ax] *= -1.0
    rxs = []
    g = int(np.ceil(np.sqrt(rx_per_room)))
    for i in range(rooms_x):
        for j in range(rooms_y):
            for q in range(rx_per_room):
                u, v = (q % g + 0.5) / g, (q // g + 0.5) / g
                rxs.append((i * room[0] + u * room[0], j * room[1] + v * room[1], 1.5))
    rx = np.repeat(np.asarray(rxs, np.float64)[None], n_frames, axis=0)
    tx = np.array([0.5 * room[0] + 0.3, 0.5 * room[1] + 0.2, 2.0], np.float32)
    trans = [-1.0, 20.0, 5.0, -1.0]
    return Scene("office", tris, tobj, tmat, office_materials(), n_carts, xf.astype(np.float32), tx,
                 rx.astype(np.float32), freq_hz=freq_hz, n_rays=n_rays, max_refl=max_refl,
                 meta={"seed": seed, "trans_db": trans, "max_trans": max_trans, "tx_power_w": 0.5})


# ----------------------------------------------------------------------------
# small scenes with closed forms
# ----------------------------------------------------------------------------

def _static_scene(name, tris, mats, tx, rx, **kw) -> Scene:
    tris = np.asarray(tris, np.float32).reshape(-1, 3, 3)
    n = tris.shape[0]
    rx = np.asarray(rx, np.float32).reshape(1, -1, 3)
    return Scene(name, tris, np.full(n, -1, np.int32), np.asarray(mats, np.int32),
                 kw.pop("materials", default_materials()), 0,
                 np.zeros((1, 0, 12), np.float32), np.asarray(tx, np.float32), rx, **kw)


def ground_plane(tx=(0.0, 0.0, 6.0), rx=((50.0, 0.0, 1.5),), half=2000.0,
                 material=MAT_CONCRETE, **kw) -> Scene:
    """One square ground at z = 0 made of two triangles (two-ray model)."""
    t = _quad((-half, -half, 0.0), (half, -half, 0.0), (half, half, 0.0), (-half, half, 0.0))
    return _static_scene("ground", t, [material] * 2, tx, rx, **kw)


def parallel_plates(h: float = 10.0, half: float = 5000.0, tx=(0.0, 0.0, 3.0),
                    rx=((40.0, 0.0, 7.0),), **kw) -> Scene:
    """Two parallel PEC plates z = 0 and z = h (two triangles each)."""
    t = _quad((-half, -half, 0.0), (half, -half, 0.0), (half, half, 0.0), (-half, half, 0.0))
    t += _quad((-half, -half, h), (-half, half, h), (half, half, h), (half, -half, h))
    return _static_scene("plates", t, [MAT_METAL] * 4, tx, rx, **kw)


def free_space(tx=(0.0, 0.0, 0.0), rx=((100.0, 0.0, 0.0),), **kw) -> Scene:
    """No geometry at all (Friis)."""
    return _static_scene("free", np.zeros((0, 3, 3), np.float32), [], tx, rx, **kw)


def random_tiny(seed: int, ntri: int = 8, nobj: int = 2, n_frames: int = 3,
                nrx: int = 3, extent: float = 20.0, **kw) -> Scene:
    """Random triangles in a box plus a large ground; a share of them belong to
    ``nobj`` rigid objects that translate/rotate each frame."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 3])))
    static = _quad((-200, -200, 0), (200, -200, 0), (200, 200, 0), (-200, 200, 0))
    smat = [MAT_CONCRETE] * 2
    meshes = [[] for _ in range(max(nobj, 0))]
    for i in range(ntri):
        c = rng.uniform([-extent, -extent, 1.0], [extent, extent, extent])
        tri = (c + rng.normal(scale=extent / 4, size=(3, 3))).tolist()
        if nobj > 0 and rng.uniform() < 0.5:
            k = int(rng.integers(0, nobj))
            meshes[k].append((np.asarray(tri) - c).tolist())
        else:
            static.append(tri)
            smat.append(MAT_CONCRETE)
    nonempty = [m for m in meshes if m]
    tris, tobj, tmat = _assemble(static, smat, nonempty,
                                 [MAT_METAL if k % 2 else MAT_CONCRETE for k in range(len(nonempty))])
    no = len(nonempty)
    base = rng.uniform([-extent, -extent, 2.0], [extent, extent, extent], size=(no, 3))
    vel = rng.normal(scale=1.0, size=(no, 3)) * np.array([1, 1, 0.2])
    w = rng.normal(scale=0.1, size=no)
    xf = np.zeros((n_frames, no, 12))
    for f in range(n_frames):
        for k in range(no):
            p = base[k] + vel[k] * f
            xf[f, k] = _xf_row(w[k] * f, p[0], p[1], p[2])
    tx = rng.uniform([-extent, -extent, 1.0], [extent, extent, extent])
    rx = rng.uniform([-extent, -extent, 1.0], [extent, extent, extent], size=(nrx, 3))
    rx = np.broadcast_to(rx, (n_frames, nrx, 3)).copy()
    return Scene(f"tiny{seed}", tris, tobj, tmat, default_materials(), no,
                 xf.astype(np.float32), tx.astype(np.float32), rx.astype(np.float32), **kw)
