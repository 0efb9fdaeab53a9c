// paths.cu -- duplicate-path removal, image-method validation, field, and
// the per-link reduction (a link is a transmitter-receiver pair: t * nrx + r;
// with one transmitter, the receiver index).
//
// Sec. III "Backward ray tracing":
//   step 2  a table of visited propagation paths per reflection depth: every
//           capture is keyed by (link, depth, triangle sequence); a
//           device hash table keeps one representative per distinct key
//           (the capture of the lowest ray index), and every other capture
//           is checked against it key by key (a 64-bit collision between
//           distinct keys is reported, never merged);
//   step 3  image receivers: the transmitter is mirrored in the plane of each
//           triangle of the sequence;
//   step 4  path validation: the back-trace from the receiver through the
//           images must cross each plane inside its triangle, and every
//           sub-segment must be unoccluded (FP32 any-hit over the LBVH);
//   step 6  per valid path: total length, delay, and the complex amplitude
//           of the ray field (Eq. 1) with the free-space spreading of Eq. 3
//           (exponent 2) and one Fresnel TE/TM reflection per bounce, with
//           vector polarisation (FP64).
// The per-link sums of amplitudes are formed in a fixed order (paths sorted
// by key), so the received power is reproducible bit for bit.
#include "paths.cuh"

#include <algorithm>

namespace dcem {

// ---------------------------------------------------------------------------
// keys
// ---------------------------------------------------------------------------
// 64-bit hash of (rx, depth, triangle sequence id_at(0..k-1)).
template <class F>
__device__ __forceinline__ unsigned long long seq_key(int rx, int k, F id_at) {
  unsigned long long h = mix64(0x9e3779b97f4a7c15ull + (unsigned long long)(unsigned)rx);
  h = mix64(h + 0x100000001b3ull * (unsigned long long)(k + 1));
  for (int j = 0; j < k; ++j)
    h = mix64(h + ((unsigned long long)(unsigned)id_at(j) | ((unsigned long long)(j + 1) << 40)));
  return h ? h : 1ull;
}

// Hit id of segment j of slot `ray` in the log ((N + T + 1) x R).
__device__ __forceinline__ int log_id_at(const PathArgs& a, int j, int ray) {
  return a.log_id[(size_t)DCEM_IDX(j, a.N + a.max_trans + 1) * a.R + DCEM_IDX(ray, a.R)];
}

// ... of `ray`'s first k logged segments.
__device__ __forceinline__ unsigned long long path_key_of(const PathArgs& a, int ray, int rx, int k) {
  return seq_key(rx, k, [&](int j) { return log_id_at(a, j, ray); });
}

// Hash-table key of a capture: its link (transmitter * nrx + receiver),
// depth and sequence, so that transmitters never share an entry.
__device__ __forceinline__ unsigned long long path_key(const PathArgs& a, Cand c) {
  return path_key_of(a, c.ray, cand_rx(c), cand_seg(c));
}

__device__ __forceinline__ bool same_key(const PathArgs& a, Cand x, Cand y) {
  if (cand_rx(x) != cand_rx(y) || cand_seg(x) != cand_seg(y)) return false;
  for (int j = 0; j < cand_seg(x); ++j)
    if (log_id_at(a, j, x.ray) != log_id_at(a, j, y.ray)) return false;
  return true;
}

__global__ void k_dedupe_insert(PathArgs a) {
  unsigned n = min(a.ctr->n_cand, a.cand_cap);
  unsigned mask = a.hcap - 1u;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    Cand c = a.cand[i];
    unsigned long long h = path_key(a, c);
    unsigned slot = (unsigned)(h & mask);
    bool ok = false;
    for (unsigned p = 0; p < a.hcap; ++p) {
      unsigned long long prev = atomicCAS(&a.hkey[slot], 0ull, h);
      if (prev == 0ull || prev == h) { ok = true; break; }
      slot = (slot + 1u) & mask;
    }
    if (!ok) {
      atomicOr(&a.ctr->err, ERR_HASH_FULL);
      a.cand_slot[i] = -1;
      continue;
    }
    a.cand_slot[i] = (int)slot;
    // representative: the capture of the lowest primary ray (a transmission
    // child counts as its primary; one primary reaches a key at most once)
    int root = c.ray < a.R0 ? c.ray : a.inst_root[DCEM_IDX(c.ray - a.R0, a.R - a.R0)];
    atomicMin(&a.hrep[slot], ((unsigned long long)(unsigned)root << 32) | i);
  }
}

__global__ void k_dedupe_unique(PathArgs a) {
  unsigned n = min(a.ctr->n_cand, a.cand_cap);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int slot = a.cand_slot[i];
    if (slot < 0) continue;
    unsigned rep = (unsigned)(a.hrep[slot] & 0xffffffffull);
    if (rep == i) {
      unsigned u = atomicAdd(&a.ctr->n_unique, 1u);
      if (u < a.ucap) a.uniq[u] = (int)i;
      else atomicOr(&a.ctr->err, ERR_UNIQUE_OVERFLOW);
    } else if (!same_key(a, a.cand[i], a.cand[DCEM_IDX(rep, a.cand_cap)])) {
      atomicOr(&a.ctr->err, ERR_HASH_COLLISION);
    }
  }
}

// Sticky mode (Sec. III "Propagation path caching", paths kept until they are
// removed): each of the previous frame's valid paths is looked up in this
// frame's table; one that no capture has joins the distinct keys as entry ~i.
__global__ void k_sticky_probe(PathArgs a) {
  unsigned n = min(*a.sticky_prev_n, a.sticky_cap);
  unsigned mask = a.hcap - 1u;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const StickyKey& sk = a.sticky_prev[i];
    unsigned long long h = seq_key(sk.link, sk.depth, [&](int j) { return sk.tri[j]; });
    unsigned slot = (unsigned)(h & mask);
    bool found = false;
    for (unsigned p = 0; p < a.hcap; ++p) {
      unsigned long long kk = a.hkey[slot];
      if (kk == 0ull) break;
      if (kk == h) {
        // the same key must be the same path: compare with the representative
        Cand c = a.cand[DCEM_IDX((unsigned)(a.hrep[slot] & 0xffffffffull), a.cand_cap)];
        bool same = cand_rx(c) == sk.link && cand_seg(c) == sk.depth;
        for (int j = 0; same && j < sk.depth; ++j) same = log_id_at(a, j, c.ray) == sk.tri[j];
        if (!same) atomicOr(&a.ctr->err, ERR_HASH_COLLISION);
        found = true;
        break;
      }
      slot = (slot + 1u) & mask;
    }
    if (found) continue;
    unsigned u = atomicAdd(&a.ctr->n_unique, 1u);
    if (u < a.ucap) a.uniq[u] = ~(int)i;
    else atomicOr(&a.ctr->err, ERR_UNIQUE_OVERFLOW);
  }
}

// ---------------------------------------------------------------------------
// FP64 geometry and complex arithmetic
// ---------------------------------------------------------------------------
struct d3 {
  double x, y, z;
};
__device__ __forceinline__ d3 mk3(double x, double y, double z) { return d3{x, y, z}; }
__device__ __forceinline__ d3 operator+(d3 a, d3 b) { return mk3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ d3 operator-(d3 a, d3 b) { return mk3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ d3 operator*(d3 a, double s) { return mk3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ double dd(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ d3 dx(d3 a, d3 b) {
  return mk3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double dn(d3 a) { return sqrt(dd(a, a)); }
__device__ __forceinline__ d3 du(d3 a) { return a * (1.0 / dn(a)); }

// Double-float numbers (hi + lo, two FP32 values, about 44 significant
// bits): the validation geometry in this precision runs on the FP32 pipe.
// Sums and products are formed with the error-free transformations
// (Knuth's two-sum, the FMA two-product); quotients and square roots add
// correction steps from the remainder.
struct df {
  float hi, lo;
};
__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return df{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df operator+(df a, df b) {
  df s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
  df r = quick_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return quick_two_sum(r.hi, __fadd_rn(r.lo, t.lo));
}
__device__ __forceinline__ df operator-(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return quick_two_sum(p, e);
}
__device__ __forceinline__ df operator/(df a, df b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  df r = a - b * df{q1, 0.0f};
  float q2 = __fdiv_rn(r.hi, b.hi);
  r = r - b * df{q2, 0.0f};
  float q3 = __fdiv_rn(r.hi, b.hi);
  return quick_two_sum(q1, q2) + df{q3, 0.0f};
}
__device__ __forceinline__ double root(double a) { return ::sqrt(a); }
__device__ __forceinline__ df root(df a) {
  if (!(a.hi > 0.0f)) return df{0.0f, 0.0f};
  float s = __fsqrt_rn(a.hi);
  float p = __fmul_rn(s, s), pe = __fmaf_rn(s, s, -p);
  float e = __fdiv_rn(__fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo), __fmul_rn(2.0f, s));
  return quick_two_sum(s, e);
}

// Scalars of the validation geometry: FP64 (default) or double-float.
template <class T> __device__ __forceinline__ T sc_of(float v);
template <> __device__ __forceinline__ double sc_of<double>(float v) { return (double)v; }
template <> __device__ __forceinline__ df sc_of<df>(float v) { return df{v, 0.0f}; }
__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(df v) { return (double)v.hi + (double)v.lo; }
__device__ __forceinline__ bool pos(double v) { return v > 0.0; }
__device__ __forceinline__ bool pos(df v) { return v.hi > 0.0f || (v.hi == 0.0f && v.lo > 0.0f); }
__device__ __forceinline__ bool neg(double v) { return v < 0.0; }
__device__ __forceinline__ bool neg(df v) { return v.hi < 0.0f || (v.hi == 0.0f && v.lo < 0.0f); }
__device__ __forceinline__ bool zero(double v) { return v == 0.0; }
__device__ __forceinline__ bool zero(df v) { return v.hi == 0.0f && v.lo == 0.0f; }

template <class T>
struct v3 {
  T x, y, z;
};
template <class T> __device__ __forceinline__ v3<T> operator+(v3<T> a, v3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> __device__ __forceinline__ v3<T> operator-(v3<T> a, v3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> __device__ __forceinline__ v3<T> scale(v3<T> a, T s) { return {a.x * s, a.y * s, a.z * s}; }
template <class T> __device__ __forceinline__ T vdot(v3<T> a, v3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> __device__ __forceinline__ v3<T> vcross(v3<T> a, v3<T> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class T> __device__ __forceinline__ v3<T> vof(float x, float y, float z) {
  return {sc_of<T>(x), sc_of<T>(y), sc_of<T>(z)};
}

// Complex FP64 arithmetic: reflection coefficients, polarisation and the
// diffraction coefficient.
struct zd {
  double re, im;
};
__device__ __forceinline__ zd Z(double r, double i = 0.0) { return zd{r, i}; }
__device__ __forceinline__ zd operator+(zd a, zd b) { return Z(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ zd operator-(zd a, zd b) { return Z(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ zd operator*(zd a, zd b) { return Z(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
__device__ __forceinline__ zd operator*(zd a, double s) { return Z(a.re * s, a.im * s); }
__device__ __forceinline__ zd zdiv(zd a, zd b) {
  double d = b.re * b.re + b.im * b.im;
  return Z((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}
__device__ __forceinline__ zd zexp(zd a) {
  double m = exp(a.re), sn, cs;
  sincos(a.im, &sn, &cs);
  return Z(m * cs, m * sn);
}
__device__ __forceinline__ zd zsqrt(zd a) {  // principal branch
  double r = hypot(a.re, a.im);
  double x = sqrt(0.5 * (r + fabs(a.re)));
  if (x == 0.0) return Z(0.0, 0.0);
  double y = a.im / (2.0 * x);
  return a.re >= 0.0 ? Z(x, y) : Z(fabs(y), a.im >= 0.0 ? x : -x);
}

__device__ __forceinline__ float fdot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

struct z3 {
  zd x, y, z;
};
__device__ __forceinline__ zd zdot(z3 e, d3 v) { return e.x * v.x + e.y * v.y + e.z * v.z; }
__device__ __forceinline__ d3 dir_of(d3 a, d3 b) { return du(b - a); }  // unit vector a -> b
// Polarisation of an isotropic antenna along unit d: u - (u.d) d, normalised
// (a fixed axis instead when u is along d; the path is then flagged).
__device__ __forceinline__ d3 pol_of(d3 u, d3 d, unsigned& flags) {
  d3 p = u - d * dd(u, d);
  double n = dn(p);
  if (n < 1e-9) {
    flags |= DCEM_PATH_POL_DEGENERATE;
    d3 ax = fabs(d.x) < 0.9 ? mk3(1, 0, 0) : mk3(0, 1, 0);
    p = ax - d * dd(ax, d);
    n = dn(p);
  }
  return p * (1.0 / n);
}

// ---------------------------------------------------------------------------
// validation + field in three kernels:
//   k_val_geom   one thread per distinct key: image sources, back-trace,
//                reflection points inside their triangles (FP64)
//   k_val_occ    one thread per (key, sub-segment): FP32 any-hit occlusion
//   k_val_field  one thread per distinct key: length, Fresnel, polarisation,
//                complex amplitude (FP64); valid paths go to their link's
//                bucket
// ---------------------------------------------------------------------------
// Distinct keys are few (thousands): thread t of block b takes keys
// b + gridDim * t, so that every SM gets a share.
__device__ __forceinline__ unsigned spread_index(unsigned i) { return blockIdx.x + gridDim.x * i; }

// Validation reuse (Sec. III "Propagation path caching": the cached paths
// are re-checked each frame; here a check is skipped when its result cannot
// have changed). The previous frame's record of the same link key is copied
// bit for bit when the receiver did not move (a coherent frame has the same
// transmitter and parameters), no triangle of the sequence belongs to an
// object that moved (so the image geometry is the same), and, for a record
// whose geometry was valid, no sub-segment meets a moved object's old or new
// box (so its occlusion test is the same).
__device__ __forceinline__ int vc_find(const PathArgs& a, unsigned long long key) {
  const unsigned mask = a.vc_cap - 1u;
  unsigned slot = (unsigned)(key & mask);
  for (unsigned p = 0; p < a.vc_cap; ++p) {
    unsigned long long k = a.vc_prev_key[slot];
    if (k == 0ull) return -1;
    if (k == key) return (int)a.vc_prev_u[slot];
    slot = (slot + 1u) & mask;
  }
  return -1;
}

__device__ __forceinline__ bool vc_reusable(const PathArgs& a, int pu, int rxi, int k, const int* ids, TStack& st) {
  if (a.rx_moved[rxi % a.nrx]) return false;
  for (int j = 0; j < k; ++j) {
    int o = a.tri_obj[ids[j] & ~(kTransBit | kDiffBit)];
    if (o >= 0 && a.obj_moved[o]) return false;
  }
  if (a.prev_vstate[pu] == 0) return true;  // invalid geometry: depends on nothing else
  const d3* xs = reinterpret_cast<const d3*>(a.prev_vpts) + (size_t)pu * (kMaxRefl + 2);
  for (int j = 0; j <= k; ++j) {
    d3 p0 = xs[j], p1 = xs[j + 1];
    d3 dv = p1 - p0;
    RayPre rp = ray_pre(f3((float)p0.x, (float)p0.y, (float)p0.z), f3((float)dv.x, (float)dv.y, (float)dv.z));
    if (seg_hits_tree(a.mvt, rp, 1.0f, st)) return false;
  }
  return true;
}

// T = double (FP64) or df (double-float) for every step of the geometry;
// path points and length are stored in FP64 either way.
template <class T>
__global__ void __launch_bounds__(64) k_val_geom(PathArgs a) {
  extern __shared__ int sstk[];
  TStack st;
  bind_stack(st, sstk, kStackSmall);
  unsigned nu = min(a.ctr->n_unique, a.ucap);
  const bool reuse = a.reuse && a.ctr->n_moved_boxes <= a.mv_cap;
  for (unsigned t = threadIdx.x;; t += blockDim.x) {
    unsigned u = spread_index(t);
    if (u >= nu) break;
    int ci = a.uniq[u];
    PathRec rec;
    int k, rxi, ray;
    int ids[kMaxRefl];
    unsigned fl0 = 0u;
    unsigned long long lkey = 0ull;  // the link key (0: a sticky record)
    if (ci >= 0) {
      Cand c = a.cand[DCEM_IDX(ci, a.cand_cap)];
      int slot = DCEM_IDX(a.cand_slot[DCEM_IDX(ci, a.cand_cap)], a.hcap);
      rec.key = a.hkey[slot];
      lkey = rec.key;
      // this slot is no longer needed: leave the table empty for the next frame
      a.hkey[slot] = 0ull;
      a.hrep[slot] = ~0ull;
      k = cand_seg(c);
      rxi = cand_rx(c);
      ray = c.ray;
      // the record's key (the output order within a link) leaves the
      // transmitter out: (receiver, depth, sequence), as a single-transmitter
      // frame has it
      if (rxi >= a.nrx) rec.key = path_key_of(a, ray, rxi % a.nrx, k);
      for (int j = 0; j < kMaxRefl; ++j) ids[j] = j < k ? log_id_at(a, j, ray) : -1;
      if (ray >= a.R0) ray = a.inst_root[DCEM_IDX(ray - a.R0, a.R - a.R0)];  // reported as its primary ray
    } else {  // sticky mode: a kept path that no capture of this frame has
      const StickyKey& sk = a.sticky_prev[~ci];
      k = sk.depth;
      rxi = sk.link;
      ray = -1;
      for (int j = 0; j < kMaxRefl; ++j) ids[j] = j < k ? sk.tri[j] : -1;
      rec.key = seq_key(rxi % a.nrx, k, [&](int j) { return ids[j]; });
      fl0 = DCEM_PATH_STICKY;
    }
    if (a.ckey) a.ckey[u] = lkey;
    if (reuse && lkey) {
      int pu = vc_find(a, lkey);
      if (pu >= 0 && vc_reusable(a, pu, rxi, k, ids, st)) {
        PathRec pr = a.prev_prec[pu];
        pr.ray = ray;  // this frame's representative
        const int ps = a.prev_vstate[pu];
        const bool valid = ps == 1 || ps == 3;
        if (ps != 0) {
          const d3* src = reinterpret_cast<const d3*>(a.prev_vpts) + (size_t)pu * (kMaxRefl + 2);
          d3* dst = reinterpret_cast<d3*>(a.vpts) + (size_t)u * (kMaxRefl + 2);
          for (int j = 0; j <= k + 1; ++j) dst[j] = src[j];
        }
        a.prec[u] = pr;
        a.vstate[u] = valid ? 3 : ps;  // 3: valid, reused (occlusion and field skip it)
        if (valid) {
          unsigned pos = atomicAdd(&a.bucket_cnt[rxi], 1u);
          if (pos < (unsigned)a.bucket_cap) a.bucket[(size_t)rxi * a.bucket_cap + pos] = (int)u;
          else atomicOr(&a.ctr->err, ERR_BUCKET_OVERFLOW);
          atomicAdd(&a.ctr->n_valid, 1u);
        }
        atomicAdd(&a.ctr->n_val_reused, 1u);
        continue;
      }
    }
    rec.rx = rxi;
    rec.depth = k;
    rec.ray = ray;
    rec.flags = fl0;
    rec.valid = 0;
    rec.pad = 0;
    rec.len = 0.0;
    rec.amp_re = rec.amp_im = 0.0;
    for (int j = 0; j < kMaxRefl; ++j) {
      rec.tri[j] = ids[j];
      rec.pts[j][0] = rec.pts[j][1] = rec.pts[j][2] = 0.0f;
    }
    // link -> transmitter and receiver
    float4 rxv = a.rx[rxi % a.nrx], txv = a.txs[rxi / a.nrx];
    v3<T> X[kMaxRefl + 2], V0[kMaxRefl], V1[kMaxRefl], V2[kMaxRefl], Nn[kMaxRefl];
    v3<T> tx = vof<T>(txv.x, txv.y, txv.z), rx = vof<T>(rxv.x, rxv.y, rxv.z);
    const T two = sc_of<T>(2.0f), one = sc_of<T>(1.0f);
    bool ok = true;
    // interactions: reflections, and transmissions (kTransBit) straight
    // through a transmitting triangle; rj lists the reflections
    int rj[kMaxRefl], m = 0;
    bool isT[kMaxRefl];
    for (int j = 0; j < k && ok; ++j) {
      isT[j] = (ids[j] & kTransBit) != 0;
      const float4* tp = a.tris + 3 * (size_t)DCEM_IDX(a.slot_of_id[DCEM_IDX(ids[j] & ~kTransBit, a.bvh.ntris)],
                                                        a.bvh.ntris);
      float4 p0 = tp[0], p1 = tp[1], p2 = tp[2];
      if (isT[j] && !(a.mats[__float_as_int(p1.w)].w >= 0.0f)) ok = false;
      V0[j] = vof<T>(p0.x, p0.y, p0.z);
      V1[j] = vof<T>(p1.x, p1.y, p1.z);
      V2[j] = vof<T>(p2.x, p2.y, p2.z);
      v3<T> n = vcross(V1[j] - V0[j], V2[j] - V0[j]);
      if (!pos(vdot(n, n))) ok = false;
      Nn[j] = n;
      if (!isT[j]) rj[m++] = j;
    }
    // step 3: image sources I_1..I_m in the planes of the reflecting triangles
    v3<T> img[kMaxRefl + 1];
    img[0] = tx;
    for (int q = 0; q < m && ok; ++q) {
      int j = rj[q];
      T nn = vdot(Nn[j], Nn[j]);
      img[q + 1] = img[q] - scale(Nn[j], two * vdot(img[q] - V0[j], Nn[j]) / nn);
    }
    // step 4: back-trace from the receiver; XR = reflection points
    v3<T> XR[kMaxRefl + 2];
    XR[0] = tx;
    XR[m + 1] = rx;
    for (int q = m; q >= 1 && ok; --q) {
      int j = rj[q - 1];
      v3<T> dir = img[q] - XR[q + 1];
      T den = vdot(dir, Nn[j]);
      if (zero(den)) { ok = false; break; }
      T sp = vdot(V0[j] - XR[q + 1], Nn[j]) / den;
      if (!(pos(sp) && neg(sp - one))) { ok = false; break; }
      XR[q] = XR[q + 1] + scale(dir, sp);
    }
    // the interaction points in order: a transmission crosses its plane on
    // the straight piece between the surrounding reflection points, after
    // the previous interaction of that piece; every point inside its triangle
    X[0] = tx;
    X[k + 1] = rx;
    {
      int q = 0;
      T s_prev = sc_of<T>(0.0f);
      for (int j = 0; j < k && ok; ++j) {
        if (!isT[j]) {
          X[j + 1] = XR[++q];
          s_prev = sc_of<T>(0.0f);
        } else {
          v3<T> A = XR[q], dir = XR[q + 1] - XR[q];
          T den = vdot(dir, Nn[j]);
          if (zero(den)) { ok = false; break; }
          T sp = vdot(V0[j] - A, Nn[j]) / den;
          if (!(pos(sp - s_prev) && neg(sp - one))) { ok = false; break; }
          X[j + 1] = A + scale(dir, sp);
          s_prev = sp;
        }
        v3<T> v0 = V0[j], v1 = V1[j], v2 = V2[j], n = Nn[j], x = X[j + 1];
        if (neg(vdot(vcross(v1 - v0, x - v0), n)) || neg(vdot(vcross(v2 - v1, x - v1), n)) ||
            neg(vdot(vcross(v0 - v2, x - v2), n)))
          ok = false;
      }
    }
    T L = sc_of<T>(0.0f);
    if (ok) {
      for (int j = 0; j <= k; ++j) {
        v3<T> e = X[j + 1] - X[j];
        L = L + root(vdot(e, e));
      }
      if (!pos(L)) ok = false;
    }
    d3* xs = reinterpret_cast<d3*>(a.vpts) + (size_t)u * (kMaxRefl + 2);
    if (ok) {
      for (int j = 0; j <= k + 1; ++j) xs[j] = mk3(to_d(X[j].x), to_d(X[j].y), to_d(X[j].z));
      rec.len = to_d(L);
    }
    a.vstate[u] = ok ? 1 : 0;   // 1 = geometry valid, occlusion pending
    a.prec[u] = rec;
  }
}

__global__ void __launch_bounds__(64) k_val_occ(PathArgs a) {
  extern __shared__ int sstk[];
  TStack st;
  bind_stack(st, sstk, kStackTrace);
  unsigned nu = min(a.ctr->n_unique, a.ucap);
  unsigned W = (unsigned)(a.N + a.max_trans) + 1u;
  unsigned total = nu * W;
  unsigned ovf = 0;
  for (unsigned t = threadIdx.x;; t += blockDim.x) {
    unsigned q = spread_index(t);
    if (q >= total) break;
    unsigned u = q / W;
    int j = (int)(q - u * W);
    if (a.vstate[u] != 1) continue;
    const PathRec& rec = a.prec[u];
    int k = rec.depth;
    if (j > k) continue;
    const d3* xs = reinterpret_cast<const d3*>(a.vpts) + (size_t)u * (kMaxRefl + 2);
    d3 p0 = xs[j], p1 = xs[j + 1];
    d3 dv = p1 - p0;
    float3 o = f3((float)p0.x, (float)p0.y, (float)p0.z);
    float3 dvf = f3((float)dv.x, (float)dv.y, (float)dv.z);
    RayPre rp = ray_pre(o, dvf);
    int ex0 = j >= 1 ? rec.tri[j - 1] & ~kTransBit : -1;
    int ex1 = j < k ? rec.tri[j] & ~kTransBit : -1;
    if (any_hit(a.bvh, rp, a.eps_occ, 1.0f - a.eps_occ, ex0, ex1, ovf, st)) a.vstate[u] = 2;  // occluded
  }
  if (ovf) {
    atomicAdd(&a.ctr->stack_overflow, 1u);
    atomicOr(&a.ctr->err, ERR_STACK);
  }
}

// Field of a valid path, in FP64 throughout (Sec. III step 6, Eq. 1): the
// directions of the sub-segments, the polarisation basis of each bounce, the
// Fresnel coefficients and the phase k L (reduced modulo 2 pi in FP64 before
// the sincos). FP64 runs at a small fraction of the FP32 rate on this GPU, so
// a key is taken by a group of kFieldLanes lanes: each lane forms the
// coefficients of its own bounces (they depend only on the path points), and
// the group's first lane then carries the field through them in order.
constexpr int kFieldLanes = 8;
constexpr int kFieldThreads = 64;
struct BounceCoef {
  double sv[3], pin[3], pout[3];  // polarisation basis: s, p before and after the bounce
  double te_re, te_im, tm_re, tm_im;  // Gamma_TE, Gamma_TM (a transmission: te_re = field factor)
  int trans;
  int pad;
};
struct FieldEnds {
  double e0[3], prx[3];  // Tx and Rx polarisation along the first and last sub-segment
  double sn, cs;          // sin, cos of the reduced phase
  unsigned fl0, fl1;
};

__global__ void __launch_bounds__(kFieldThreads) k_val_field(PathArgs a) {
  constexpr int kGroups = kFieldThreads / kFieldLanes;
  __shared__ BounceCoef scoef[kGroups][kMaxRefl];
  __shared__ FieldEnds sends[kGroups];
  const unsigned nu = min(a.ctr->n_unique, a.ucap);
  const int grp = threadIdx.x / kFieldLanes, gl = threadIdx.x % kFieldLanes;
  const unsigned gmask = ((1u << kFieldLanes) - 1u) << ((threadIdx.x & 31) & ~(kFieldLanes - 1));
  const d3 upol = mk3(a.pol.x, a.pol.y, a.pol.z);
  const double wfac = -1.0 / (2.0 * M_PI * a.freq * 8.8541878128e-12);
  BounceCoef* C = scoef[grp];
  FieldEnds& ends = sends[grp];
  for (unsigned it = 0;; ++it) {
    unsigned u = blockIdx.x + gridDim.x * (grp + kGroups * it);
    if (u >= nu) break;
    if (a.vstate[u] != 1) continue;
    PathRec& rec = a.prec[u];
    const int k = rec.depth;
    const d3* X = reinterpret_cast<const d3*>(a.vpts) + (size_t)u * (kMaxRefl + 2);
    const double L = rec.len;
    // bounce j (1..k): incoming X[j-1] -> X[j], outgoing X[j] -> X[j+1]
    for (int j = 1 + gl; j <= k; j += kFieldLanes) {
      BounceCoef& c = C[j - 1];
      const int id = rec.tri[j - 1];
      const float4* tp = a.tris + 3 * (size_t)DCEM_IDX(a.slot_of_id[DCEM_IDX(id & ~kTransBit, a.bvh.ntris)],
                                                        a.bvh.ntris);
      float4 p0 = tp[0], p1 = tp[1], p2 = tp[2];
      const float4 mt = a.mats[__float_as_int(p1.w)];
      if (id & kTransBit) {  // penetration loss L dB: field times 10^(-L/20)
        c.trans = 1;
        c.te_re = pow(10.0, -(double)mt.w / 20.0);
        continue;
      }
      c.trans = 0;
      d3 din = dir_of(X[j - 1], X[j]), dout = dir_of(X[j], X[j + 1]);
      d3 q0 = mk3(p0.x, p0.y, p0.z);
      d3 nh = du(dx(mk3(p1.x, p1.y, p1.z) - q0, mk3(p2.x, p2.y, p2.z) - q0));
      double ct = fabs(dd(din, nh));
      d3 sv = dx(din, nh);
      double sn = dn(sv);
      if (sn < 1e-12) {  // normal incidence: any unit vector perpendicular to n
        d3 ax = fabs(nh.x) < 0.9 ? mk3(1, 0, 0) : mk3(0, 1, 0);
        sv = du(dx(nh, ax));
      } else {
        sv = sv * (1.0 / sn);
      }
      d3 pin = dx(sv, din), pout = dx(sv, dout);
      zd gte, gtm;
      if (mt.z != 0.0f) {
        gte = Z(-1.0);
        gtm = Z(1.0);
      } else {
        zd ec = Z((double)mt.x, (double)mt.y * wfac);
        zd root = zsqrt(ec - Z(1.0 - ct * ct));
        gte = zdiv(Z(ct) - root, Z(ct) + root);
        gtm = zdiv(ec * ct - root, ec * ct + root);
      }
      c.sv[0] = sv.x; c.sv[1] = sv.y; c.sv[2] = sv.z;
      c.pin[0] = pin.x; c.pin[1] = pin.y; c.pin[2] = pin.z;
      c.pout[0] = pout.x; c.pout[1] = pout.y; c.pout[2] = pout.z;
      c.te_re = gte.re; c.te_im = gte.im;
      c.tm_re = gtm.re; c.tm_im = gtm.im;
    }
    // the ends, on lanes that hold no bounce of a path of up to 5 bounces
    if (gl == kFieldLanes - 1) {
      unsigned f = 0;
      d3 e0 = pol_of(upol, dir_of(X[0], X[1]), f);
      ends.e0[0] = e0.x; ends.e0[1] = e0.y; ends.e0[2] = e0.z;
      ends.fl0 = f;
    } else if (gl == kFieldLanes - 2) {
      unsigned f = 0;
      d3 prx = pol_of(upol, dir_of(X[k + 1], X[k]), f);
      ends.prx[0] = prx.x; ends.prx[1] = prx.y; ends.prx[2] = prx.z;
      ends.fl1 = f;
    } else if (gl == kFieldLanes - 3) {
      // phase k L reduced modulo 2 pi: subtract the nearest multiple of 2 pi,
      // the product n * 2 pi taken exactly by an FMA against a two-part 2 pi
      double kl = 2.0 * M_PI * a.freq / 299792458.0 * L;
      double nq = rint(kl * (0.5 / M_PI));
      double ph = fma(-nq, 6.283185307179586, kl);
      ph = fma(-nq, 2.4492935982947064e-16, ph);
      sincos(ph, &ends.sn, &ends.cs);
    }
    __syncwarp(gmask);
    if (gl == 0) {
      z3 E = {Z(ends.e0[0]), Z(ends.e0[1]), Z(ends.e0[2])};
      for (int j = 0; j < k; ++j) {
        const BounceCoef& c = C[j];
        if (c.trans) {
          E.x = E.x * c.te_re;
          E.y = E.y * c.te_re;
          E.z = E.z * c.te_re;
          continue;
        }
        const d3 sv = mk3(c.sv[0], c.sv[1], c.sv[2]), pin = mk3(c.pin[0], c.pin[1], c.pin[2]),
                 pout = mk3(c.pout[0], c.pout[1], c.pout[2]);
        zd ts = Z(c.te_re, c.te_im) * zdot(E, sv), tpp = Z(c.tm_re, c.tm_im) * zdot(E, pin);
        E.x = ts * sv.x + tpp * pout.x;
        E.y = ts * sv.y + tpp * pout.y;
        E.z = ts * sv.z + tpp * pout.z;
      }
      const unsigned fl = ends.fl0 | ends.fl1;
      const double sn = ends.sn, cs = ends.cs;
      zd proj = zdot(E, mk3(ends.prx[0], ends.prx[1], ends.prx[2]));
      double lam = 299792458.0 / a.freq;
      double g = lam / (4.0 * M_PI) / L;
      double re = proj.re * cs + proj.im * sn, im = proj.im * cs - proj.re * sn;
      rec.valid = 1;
      rec.flags |= fl;
      rec.amp_re = re * g;
      rec.amp_im = im * g;
      for (int j = 0; j < k; ++j) {
        rec.pts[j][0] = (float)X[j + 1].x;
        rec.pts[j][1] = (float)X[j + 1].y;
        rec.pts[j][2] = (float)X[j + 1].z;
      }
      int rxi = rec.rx;
      unsigned pos = atomicAdd(&a.bucket_cnt[rxi], 1u);
      if (pos < (unsigned)a.bucket_cap) a.bucket[(size_t)rxi * a.bucket_cap + pos] = (int)u;
      else atomicOr(&a.ctr->err, ERR_BUCKET_OVERFLOW);
      atomicAdd(&a.ctr->n_valid, 1u);
      if (a.sticky_next) {  // kept for the next frame
        if (rec.flags & DCEM_PATH_STICKY) atomicAdd(&a.ctr->n_sticky_valid, 1u);
        unsigned q = atomicAdd(&a.ctr->n_sticky_next, 1u);
        if (q < a.sticky_cap) {
          StickyKey sk;
          sk.link = rxi;
          sk.depth = k;
          for (int j = 0; j < kMaxRefl; ++j) sk.tri[j] = rec.tri[j];
          a.sticky_next[q] = sk;
        }
      }
    }
    __syncwarp(gmask);  // the group's shared records are free again
  }
}

// ---------------------------------------------------------------------------
// first-order edge diffraction (Sec. III step 5) with the UTD
// ---------------------------------------------------------------------------
// erfc(z) for Re z > 0: the Maclaurin series of erf (Abramowitz & Stegun
// 7.1.5) for |z| < 3, else the continued fraction of A&S 7.1.14, truncated
// after 40, 30 or 20 terms for |z| from 3, 3.5 or 4.5 on (relative error
// below 3e-15 against a Faddeeva-function reference). Only |z| < 5.5 comes
// here: transition_fn takes its large-argument series from x = 30 on.
__device__ zd erfc_z(zd z) {
  const double rsqpi = 0.56418958354775628695;  // 1/sqrt(pi)
  double az = hypot(z.re, z.im);
  if (az < 3.0) {
    zd z2 = z * z, term = z, sum = z;
    for (int n = 1; n < 200; ++n) {
      term = term * z2 * (-1.0 / n);
      zd t = term * (1.0 / (2 * n + 1));
      sum = sum + t;
      if (fabs(t.re) + fabs(t.im) < 1e-17 * (fabs(sum.re) + fabs(sum.im))) break;
    }
    return Z(1.0) - sum * (2.0 * rsqpi);
  }
  // erfc z = e^{-z^2}/sqrt(pi) * 1/(z + (1/2)/(z + 1/(z + (3/2)/(z + ...)))),
  // the truncated fraction evaluated forward as A_n / B_n (A_k = z A_{k-1} +
  // (k/2) A_{k-2}, B likewise) with one division at the end; for |z| < 5.5
  // and 40 terms |A|, |B| stay below 1e40
  zd A0 = Z(1.0), A1 = z, B0 = Z(0.0), B1 = Z(1.0);
  const int nt = az < 3.5 ? 40 : az < 4.5 ? 30 : 20;
  for (int k = 1; k <= nt; ++k) {
    zd A2 = z * A1 + A0 * (0.5 * k), B2 = z * B1 + B0 * (0.5 * k);
    A0 = A1;
    A1 = A2;
    B0 = B1;
    B1 = B2;
  }
  zd ez = zexp(Z(-(z.re * z.re - z.im * z.im), -2.0 * z.re * z.im));
  return zdiv(ez * rsqpi * B1, A1);
}

// UTD transition function F(x) = 2j sqrt(x) e^{jx} int_{sqrt x}^inf e^{-j t^2} dt,
// the tail integral being (sqrt(pi)/2) e^{-j pi/4} erfc(e^{j pi/4} sqrt x).
// For x >= 30 its large-argument expansion (repeated integration by parts of
// the tail integral, as Kouyoumjian & Pathak give it): F(x) = sum_m t_m with
// t_0 = 1, t_m = t_{m-1} j (2m - 1) / (2x), i.e. 1 + j/(2x) - 3/(4x^2) - ...;
// its terms shrink while 2m - 1 < 2x, and the sum stops there or at 1e-17;
// the error is below 1e-13 for x >= 30. Away from shadow and reflection
// boundaries x = 2kL cos^2(.) is in the thousands, so this is the usual case.
__device__ zd transition_fn(double x) {
  if (!(x > 0.0)) return Z(0.0);
  if (x >= 30.0) {
    const double r = 1.0 / (2.0 * x);
    zd t = Z(1.0), sum = Z(1.0);
    for (int m = 1; m <= 40; ++m) {
      double c = (2.0 * m - 1.0) * r;
      if (c >= 1.0) break;  // the terms grow from here on
      t = Z(-t.im * c, t.re * c);  // times j (2m - 1) / (2x)
      sum = sum + t;
      if (fabs(t.re) + fabs(t.im) < 1e-17 * (fabs(sum.re) + fabs(sum.im))) break;
    }
    return sum;
  }
  double a = sqrt(x);
  const double h = 0.70710678118654752440;
  zd G = Z(h, -h) * erfc_z(Z(h * a, h * a)) * 0.88622692545275801365;  // sqrt(pi)/2
  double sn, cs;
  sincos(x, &sn, &cs);
  return Z(0.0, 2.0 * a) * Z(cs, sn) * G;
}

__device__ zd utd_term(double n, double beta, double s, double kL, unsigned& fl) {
  double N = rint((beta + s * M_PI) / (2.0 * M_PI * n));
  double c = cos((2.0 * n * M_PI * N - beta) / 2.0);
  double arg = (M_PI + s * beta) / (2.0 * n);
  double sn = sin(arg);
  if (fabs(sn) < 1e-9) return Z(0.0);
  return transition_fn(kL * 2.0 * c * c) * (cos(arg) / sn);
}

// Kouyoumjian-Pathak wedge coefficient D = pre (t1 + t2 + r0 t3 + rn t4)
// with face reflection factors r0, rn. The prefactor and the four terms do
// not depend on r0 and rn, so the soft and hard coefficients share them
// (utd_parts once, utd_coeff per polarisation).
struct UtdParts {
  zd pre, t[4];
};
__device__ UtdParts utd_parts(double n, double phi, double phip, double beta0, double L, double k, unsigned& fl) {
  const double h = 0.70710678118654752440;
  UtdParts u;
  u.pre = Z(-h, h) * (1.0 / (2.0 * n * sqrt(2.0 * M_PI * k) * sin(beta0)));  // -e^{-j pi/4} / (...)
  double bm = phi - phip, bp = phi + phip, kL = k * L;
  u.t[0] = utd_term(n, bm, 1.0, kL, fl);
  u.t[1] = utd_term(n, bm, -1.0, kL, fl);
  u.t[2] = utd_term(n, bp, -1.0, kL, fl);
  u.t[3] = utd_term(n, bp, 1.0, kL, fl);
  return u;
}
__device__ zd utd_coeff(const UtdParts& u, zd r0, zd rn) {
  return u.pre * (u.t[0] + u.t[1] + r0 * u.t[2] + rn * u.t[3]);
}

// Fresnel TE / TM coefficients in FP64 (eps_c = eps_r - j sigma/(w eps0)).
__device__ void fresnel_d(float4 mt, double freq, double ct, zd& te, zd& tm) {
  if (mt.z != 0.0f) {
    te = Z(-1.0);
    tm = Z(1.0);
    return;
  }
  zd ec = Z((double)mt.x, -(double)mt.y / (2.0 * M_PI * freq * 8.8541878128e-12));
  zd root = zsqrt(ec - Z(1.0 - ct * ct));
  te = zdiv(Z(ct) - root, Z(ct) + root);
  tm = zdiv(ec * ct - root, ec * ct + root);
}

struct d3w {
  double x, y, z;
};
__device__ __forceinline__ d3w D3(double x, double y, double z) { return d3w{x, y, z}; }
__device__ __forceinline__ d3w operator-(d3w a, d3w b) { return D3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ d3w operator+(d3w a, d3w b) { return D3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ d3w operator*(d3w a, double s) { return D3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ double dotw(d3w a, d3w b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ d3w crossw(d3w a, d3w b) {
  return D3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ d3w unitw(d3w a) { return a * (1.0 / sqrt(dotw(a, a))); }
__device__ __forceinline__ d3w polw(d3w u, d3w d, unsigned& fl) {
  d3w p = u - d * dotw(u, d);
  double n = sqrt(dotw(p, p));
  if (n < 1e-9) {
    fl |= DCEM_PATH_POL_DEGENERATE;
    d3w a = fabs(d.x) < 0.9 ? D3(1, 0, 0) : D3(0, 1, 0);
    p = a - d * dotw(a, d);
    n = sqrt(dotw(p, p));
  }
  return p * (1.0 / n);
}

// Angle of X about the wedge, from face 0 through the exterior.
__device__ __forceinline__ double wedge_angle(const Wedge& W, d3w X) {
  d3w e = D3(W.e[0], W.e[1], W.e[2]);
  d3w d = X - D3(W.p0[0], W.p0[1], W.p0[2]);
  d = d - e * dotw(d, e);
  double a = atan2(dotw(d, D3(W.y0[0], W.y0[1], W.y0[2])), dotw(d, D3(W.t0[0], W.t0[1], W.t0[2])));
  return a < 0.0 ? a + 2.0 * M_PI : a;
}

// FP32 pre-test of a (transmitter, receiver, wedge) triple: false only when
// the FP64 test below rejects the triple too, so that most triples (far from
// the Keller cone of a short vehicle edge, or on the lit side) cost no FP64
// work. Rejections keep margins above the FP32 rounding of the geometry: the
// Keller point off the edge by more than 5 cm (plus 1e-5 of the distances),
// an angle beyond the wedge or the shadow-boundary rule missed by more than
// ten times the angle's rounding bound (at least 1e-3 rad). Angles near the
// 0 / 2 pi cut, or of points near the edge line, reject nothing.
__device__ __forceinline__ float wedge_angle32(float3 d, float3 t0, float3 y0, float r, float dist, bool& sure,
                                               float& tol) {
  float a = atan2f(fdot3(d, y0), fdot3(d, t0));
  if (a < 0.0f) a += 6.2831853f;
  float err = 4e-6f * (dist + 1.0f) / r + 1e-5f;  // rounding of the in-plane direction, radians
  tol = fmaxf(1e-3f, 10.0f * err);
  sure = r > 0.0f && err < 1e-3f && a > tol && a < 6.2831853f - tol;
  return a;
}

__device__ __forceinline__ bool diffract_candidate(const WedgeF& W, float4 txv, float4 rxv) {
  const float3 e = W.e, p0 = W.p0;
  float3 dt = f3(txv.x - p0.x, txv.y - p0.y, txv.z - p0.z), dr = f3(rxv.x - p0.x, rxv.y - p0.y, rxv.z - p0.z);
  float zt = fdot3(dt, e), zr = fdot3(dr, e);
  float3 pt = f3(dt.x - e.x * zt, dt.y - e.y * zt, dt.z - e.z * zt);
  float3 pr = f3(dr.x - e.x * zr, dr.y - e.y * zr, dr.z - e.z * zr);
  float rt = sqrtf(fdot3(pt, pt)), rr = sqrtf(fdot3(pr, pr));
  float lt = sqrtf(fdot3(dt, dt)), lr = sqrtf(fdot3(dr, dr));
  if (!(rt > 1e-3f && rr > 1e-3f)) return true;
  float zq = zt + (zr - zt) * rt / (rt + rr);
  float mz = 0.05f + 1e-5f * (lt + lr);
  if (zq < -mz || zq > W.len + mz) return false;
  bool st, sr;
  float tt, tr;
  float phip = wedge_angle32(pt, W.t0, W.y0, rt, lt, st, tt), phi = wedge_angle32(pr, W.t0, W.y0, rr, lr, sr, tr);
  const float npi = W.npi;
  if ((st && phip > npi + tt) || (sr && phi > npi + tr)) return false;
  if (st && sr && fabsf(phi - phip) < 3.14159265f - (tt + tr)) return false;
  return true;
}

// Triangle slot geometry: vertices and the (unnormalised) normal.
__device__ __forceinline__ void tri64(const PathArgs& a, int id, d3w& v0, d3w& v1, d3w& v2, float4& mat) {
  const float4* tp = a.tris + 3 * (size_t)DCEM_IDX(a.slot_of_id[DCEM_IDX(id, a.bvh.ntris)], a.bvh.ntris);
  float4 p0 = tp[0], p1 = tp[1], p2 = tp[2];
  v0 = D3(p0.x, p0.y, p0.z);
  v1 = D3(p1.x, p1.y, p1.z);
  v2 = D3(p2.x, p2.y, p2.z);
  mat = a.mats[__float_as_int(p1.w)];
}

// The triangles (other than ex0 .. ex3) that the open segment p -> q crosses
// with parameter in (eps_occ, 1 - eps_occ) (FP32 traversal of the scene, as
// any_hit), in order along it: their ids in ids[0 .. n-1]. Returns n, or -1
// when one of them is opaque (a material without penetration loss, loss <
// 0) or there are more than cap (the transmissions a path has left).
__device__ __noinline__ int leg_crossings(const PathArgs& a, d3w p, d3w q, int ex0, int ex1, int ex2, int ex3,
                                          int* ids, int cap, unsigned& ovf, TStack& st) {
  const Bvh& bvh = a.bvh;
  const d3w dv = q - p;
  const RayPre r = ray_pre(f3((float)p.x, (float)p.y, (float)p.z), f3((float)dv.x, (float)dv.y, (float)dv.z));
  const float t0 = a.eps_occ, t1 = 1.0f - a.eps_occ;
  float ts[kMaxRefl];
  int n = 0;
  st.reset();
  if (bvh.root1 != kEmpty) st.push(bvh.root1);
  int cur = bvh.root0;
  for (int visits = 0;; ++visits) {
    if (visits > bvh.max_visits) {
      ovf = 1u;
      break;
    }
    if (cur == kEmpty) {
      if (st.empty()) break;
      cur = st.pop();
      continue;
    }
    if (cur >= 0) {
      const float4* nd = bvh.nodes + 4 * (size_t)DCEM_IDX(cur, bvh.nnodes);
      float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
      float tn0, tn1;
      bool h0 = slab(r, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, t1, tn0);
      bool h1 = slab(r, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, t1, tn1);
      int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
      if (h0 && h1) {
        if (!st.push(c1)) ovf = 1u;
        cur = c0;
      } else if (h0) {
        cur = c0;
      } else if (h1) {
        cur = c1;
      } else {
        cur = kEmpty;
      }
    } else {
      const int slot = DCEM_IDX(~cur, bvh.ntris);
      float3 v0, v1, v2;
      int id;
      load_tri(bvh.tris, slot, v0, v1, v2, id);
      float t;
      cur = kEmpty;
      if (id == ex0 || id == ex1 || id == ex2 || id == ex3 || !tri_hit(r, v0, v1, v2, t) || !(t > t0 && t < t1))
        continue;
      const float loss = a.mats[__float_as_int(__ldg(&bvh.tris[3 * slot + 1]).w)].w;
      if (!(loss >= 0.0f) || n >= cap || n >= kMaxRefl) return -1;
      int k = n++;  // insertion in order along the segment
      while (k > 0 && ts[k - 1] > t) {
        ts[k] = ts[k - 1];
        ids[k] = ids[k - 1];
        --k;
      }
      ts[k] = t;
      ids[k] = id;
    }
  }
  return n;
}

// FP32 any-hit of the open segment a -> b, the wedge faces (and a reflecting
// triangle) excluded.
__device__ __noinline__ bool leg_occluded(const PathArgs& a, d3w p, d3w q, int ex0, int ex1, unsigned& ovf,
                                             TStack& st, int ex2 = -1) {
  d3w dv = q - p;
  RayPre rp = ray_pre(f3((float)p.x, (float)p.y, (float)p.z), f3((float)dv.x, (float)dv.y, (float)dv.z));
  return any_hit(a.bvh, rp, a.eps_occ, 1.0f - a.eps_occ, ex0, ex1, ovf, st, ex2);
}

// Wedge geometry from the current world triangles (moving objects' wedges
// follow their objects): the edge from its lexicographically lower vertex,
// the faces' directions normal to it, and n = exterior angle / pi.
__device__ __forceinline__ bool vless(float4 a, float4 b) {
  if (a.x != b.x) return a.x < b.x;
  if (a.y != b.y) return a.y < b.y;
  return a.z < b.z;
}

__global__ void k_wedge_geom(const float4* __restrict__ tris, const int* __restrict__ slot_of_id,
                             const WedgeTopo* __restrict__ topo, int nw, Wedge* out, WedgeF* outf) {
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
    WedgeTopo t = topo[w];
    const float4* A = tris + 3 * (size_t)slot_of_id[t.ta];
    const float4* B = tris + 3 * (size_t)slot_of_id[t.tb];
    float4 va = A[t.ka0], vb = A[t.ka1], vt = A[t.kat], vu = B[t.kbt];
    if (vless(vb, va)) {
      float4 x = va;
      va = vb;
      vb = x;
    }
    Wedge W;
    d3w p0 = D3(va.x, va.y, va.z), e = D3((double)vb.x - va.x, (double)vb.y - va.y, (double)vb.z - va.z);
    double len = sqrt(dotw(e, e));
    e = e * (1.0 / len);
    d3w da = D3((double)vt.x - va.x, (double)vt.y - va.y, (double)vt.z - va.z);
    d3w db = D3((double)vu.x - va.x, (double)vu.y - va.y, (double)vu.z - va.z);
    da = da - e * dotw(da, e);
    db = db - e * dotw(db, e);
    d3w t0 = da * (1.0 / sqrt(dotw(da, da))), tB = db * (1.0 / sqrt(dotw(db, db)));
    d3w y0 = crossw(e, t0);
    double alpha = atan2(dotw(tB, y0), dotw(tB, t0));
    if (alpha < 0.0) {
      y0 = y0 * -1.0;
      alpha = -alpha;
    }
    y0 = y0 * -1.0;  // the exterior runs away from face n
    W.p0[0] = p0.x; W.p0[1] = p0.y; W.p0[2] = p0.z;
    W.p1[0] = vb.x; W.p1[1] = vb.y; W.p1[2] = vb.z;
    W.e[0] = e.x; W.e[1] = e.y; W.e[2] = e.z;
    W.t0[0] = t0.x; W.t0[1] = t0.y; W.t0[2] = t0.z;
    W.tB[0] = tB.x; W.tB[1] = tB.y; W.tB[2] = tB.z;
    W.y0[0] = y0.x; W.y0[1] = y0.y; W.y0[2] = y0.z;
    W.len = len;
    W.n = 2.0 - alpha / M_PI;
    W.ta = t.ta;
    W.tb = t.tb;
    out[w] = W;
    WedgeF f;
    f.p0 = make_float3((float)W.p0[0], (float)W.p0[1], (float)W.p0[2]);
    f.e = make_float3((float)W.e[0], (float)W.e[1], (float)W.e[2]);
    f.t0 = make_float3((float)W.t0[0], (float)W.t0[1], (float)W.t0[2]);
    f.y0 = make_float3((float)W.y0[0], (float)W.y0[1], (float)W.y0[2]);
    f.len = (float)W.len;
    f.npi = (float)(W.n * M_PI);
    outf[w] = f;
  }
}

// Each cluster's box (one warp per cluster of kWedgeCluster wedges in the
// order perm): the min and max over its edges' two ends in FP32.
__global__ void k_wedge_boxes(const WedgeF* __restrict__ wf, const int* __restrict__ perm, int nw, int nwc,
                              float* __restrict__ box) {
  const int lane = threadIdx.x & 31;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nwc; c += (gridDim.x * blockDim.x) >> 5) {
    const int i = c * kWedgeCluster + lane;
    float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
    if (i < nw) {
      const WedgeF f = wf[perm[i]];
      const float q[3] = {f.p0.x + f.e.x * f.len, f.p0.y + f.e.y * f.len, f.p0.z + f.e.z * f.len};
      const float p[3] = {f.p0.x, f.p0.y, f.p0.z};
      for (int k = 0; k < 3; ++k) {
        lo[k] = fminf(p[k], q[k]);
        hi[k] = fmaxf(p[k], q[k]);
      }
    }
    for (int o = 16; o > 0; o >>= 1)
      for (int k = 0; k < 3; ++k) {
        lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
        hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
      }
    if (lane < 6) box[6 * (size_t)c + lane] = lane < 3 ? lo[lane] : hi[lane - 3];
  }
}

// One thread per (link, wedge): the Keller point on the edge (unfolding the
// path about the edge line), the paper's shadow rule (the receiver beyond the
// incident shadow boundary), both legs unoccluded, then the UTD field; a
// valid path joins its link's bucket like a validated path.
// One (link, wedge) pair that passed the FP32 pre-test: the exact FP64
// test, the legs' occlusion, the UTD field and the path record.
__device__ __forceinline__ void diffract_pair(const PathArgs& a, long idx, double k, double lam, unsigned& ovf,
                                              TStack& st) {
  int link = (int)(idx / a.nw), w = (int)(idx - (long)link * a.nw);
  const Wedge W = a.wedges[w];
  float4 rxv = a.rx[link % a.nrx], txv = a.txs[link / a.nrx];
  d3w T = D3(txv.x, txv.y, txv.z), R = D3(rxv.x, rxv.y, rxv.z);
  d3w e = D3(W.e[0], W.e[1], W.e[2]), p0 = D3(W.p0[0], W.p0[1], W.p0[2]);
  d3w dt = T - p0, dr = R - p0;
  double zt = dotw(dt, e), zr = dotw(dr, e);
  d3w pt = dt - e * zt, pr = dr - e * zr;
  double rt = sqrt(dotw(pt, pt)), rr = sqrt(dotw(pr, pr));
  if (!(rt > 0.0 && rr > 0.0)) return;
  double zq = zt + (zr - zt) * rt / (rt + rr);
  double uq = zq / W.len;
  if (!(uq > 0.0 && uq < 1.0)) return;
  d3w Q = p0 + e * zq;
  double phip = wedge_angle(W, T), phi = wedge_angle(W, R), n = W.n;
  if (phip > n * M_PI || phi > n * M_PI) return;
  if (!(fabs(phi - phip) > M_PI)) return;
  // the legs: unoccluded, or with transmission on, crossing penetrable
  // triangles only, at most max_trans in all (Table II losses)
  int c1[kMaxRefl], c2[kMaxRefl], n1 = 0, n2 = 0;
  if (a.max_trans > 0) {
    const int mt = min(a.max_trans, kMaxRefl - 1);  // the wedge takes one of the record's slots
    n1 = leg_crossings(a, T, Q, W.ta, W.tb, W.tb, W.tb, c1, mt, ovf, st);
    if (n1 < 0) return;
    n2 = leg_crossings(a, Q, R, W.ta, W.tb, W.tb, W.tb, c2, mt - n1, ovf, st);
    if (n2 < 0) return;
  } else if (leg_occluded(a, T, Q, W.ta, W.tb, ovf, st) || leg_occluded(a, Q, R, W.ta, W.tb, ovf, st)) {
    return;
  }
  unsigned fl = 0;
  d3w qt = Q - T, rq = R - Q;
  double sp = sqrt(dotw(qt, qt)), s = sqrt(dotw(rq, rq));
  d3w ip = qt * (1.0 / sp), dd = rq * (1.0 / s);
  double beta0 = acos(fmax(-1.0, fmin(1.0, dotw(ip, e))));
  double sb = sin(beta0);
  double L = s * sp * sb * sb / (s + sp);
  d3w php = unitw(crossw(e, ip)) * -1.0, ph = unitw(crossw(e, dd));
  d3w bp = crossw(ip, php), bd = crossw(dd, ph);
  // Luebbers: the faces' Fresnel factors at the grazing angles phi' and n pi - phi
  const float4 ma =
      a.mats[__float_as_int(a.tris[3 * (size_t)DCEM_IDX(a.slot_of_id[DCEM_IDX(W.ta, a.bvh.ntris)], a.bvh.ntris) + 1].w)];
  const float4 mb =
      a.mats[__float_as_int(a.tris[3 * (size_t)DCEM_IDX(a.slot_of_id[DCEM_IDX(W.tb, a.bvh.ntris)], a.bvh.ntris) + 1].w)];
  zd r0s, r0h, rns, rnh;
  fresnel_d(ma, a.freq, fabs(sin(phip)), r0s, r0h);
  fresnel_d(mb, a.freq, fabs(sin(n * M_PI - phi)), rns, rnh);
  const UtdParts up = utd_parts(n, phi, phip, beta0, L, k, fl);
  zd Ds = utd_coeff(up, r0s, rns);
  zd Dh = utd_coeff(up, r0h, rnh);
  d3w u = D3(a.pol.x, a.pol.y, a.pol.z);
  d3w e0 = polw(u, ip, fl), prx = polw(u, dd * -1.0, fl);
  double sn, cs;
  sincos(-k * sp, &sn, &cs);
  zd Ei = Z(cs / sp, sn / sp);
  zd Eb = Ei * dotw(e0, bp), Ep = Ei * dotw(e0, php);
  sincos(-k * s, &sn, &cs);
  zd A = Z(cs, sn) * sqrt(sp / (s * (s + sp)));
  zd proj = (Ds * Eb) * (-dotw(bd, prx)) + (Dh * Ep) * (-dotw(ph, prx));
  // each crossing's penetration loss (power dB): the field times 10^(-L/20)
  double g = 1.0;
  for (int i = 0; i < n1 + n2; ++i) {
    d3w v0, v1, v2;
    float4 mt;
    tri64(a, i < n1 ? c1[i] : c2[i - n1], v0, v1, v2, mt);
    g *= pow(10.0, -(double)mt.w / 20.0);
  }
  zd amp = proj * A * (lam / (4.0 * M_PI) * g);
  unsigned uu = atomicAdd(&a.ctr->n_unique, 1u);
  if (uu >= a.ucap) {
    atomicOr(&a.ctr->err, ERR_UNIQUE_OVERFLOW);
    return;
  }
  PathRec rec;
  // interactions in path order: the first leg's crossings, the wedge, the second leg's
  const int depth = n1 + 1 + n2;
  auto id_at = [&](int q) {
    return q < n1 ? (c1[q] | kTransBit) : q == n1 ? (w | kDiffBit) : (c2[q - n1 - 1] | kTransBit);
  };
  rec.key = seq_key(link % a.nrx, depth, id_at);
  rec.rx = link;
  rec.depth = depth;
  rec.ray = -1;
  rec.flags = fl;
  rec.valid = 1;
  rec.pad = 0;
  rec.len = sp + s;
  rec.amp_re = amp.re;
  rec.amp_im = amp.im;
  for (int j = 0; j < kMaxRefl; ++j) {
    rec.tri[j] = j < depth ? id_at(j) : -1;
    rec.pts[j][0] = rec.pts[j][1] = rec.pts[j][2] = 0.0f;
  }
  for (int j = 0; j < depth; ++j) {  // the crossings where the legs meet their triangles' planes, and Q
    d3w X = Q;
    if (j != n1) {
      const bool first = j < n1;
      const d3w o = first ? T : Q, dl = first ? qt : rq;
      d3w v0, v1, v2;
      float4 mt;
      tri64(a, first ? c1[j] : c2[j - n1 - 1], v0, v1, v2, mt);
      const d3w nv = crossw(v1 - v0, v2 - v0);
      X = o + dl * (dotw(v0 - o, nv) / dotw(dl, nv));
    }
    rec.pts[j][0] = (float)X.x;
    rec.pts[j][1] = (float)X.y;
    rec.pts[j][2] = (float)X.z;
  }
  a.prec[uu] = rec;
  unsigned pos = atomicAdd(&a.bucket_cnt[link], 1u);
  if (pos < (unsigned)a.bucket_cap) a.bucket[(size_t)link * a.bucket_cap + pos] = (int)uu;
  else atomicOr(&a.ctr->err, ERR_BUCKET_OVERFLOW);
  atomicAdd(&a.ctr->n_valid, 1u);
}

// ---------------------------------------------------------------------------
// one reflection before or after a diffraction (Sec. III steps 3-5)
// ---------------------------------------------------------------------------
// By image theory a reflection on plane (n, c) before the wedge is the
// diffraction of the transmitter's image, a reflection after it the
// diffraction toward the receiver's image; the reflection point is where the
// unfolded leg (image -> Q, or Q -> image) crosses the plane. Candidates are
// (link, wedge, reflector plane, order); survivors of the FP32 pre-test carry
// bit 63 in the survivor list: ((link * nw + wedge) * nrp + plane) * 2 + first.
constexpr unsigned long long kReflTag = 1ull << 63;

__device__ __forceinline__ float3 mirror32(float3 x, float3 n, float c) {
  float h = 2.0f * (fdot3(n, x) - c);
  return f3(x.x - h * n.x, x.y - h * n.y, x.z - h * n.z);
}

// FP32 pre-test: false only when the FP64 test rejects the candidate too
// (Keller point and angles as diffract_candidate with the image; the
// reflection point off the plane's box by more than 5 cm + 1e-4 of the
// distances, or off the unfolded leg).
__device__ __forceinline__ bool diffract_refl_candidate(const WedgeF& W, const RPlane& P, float4 txv, float4 rxv,
                                                        bool first) {
  const float3 n = f3(P.nf[0], P.nf[1], P.nf[2]);
  const float c = P.cf;
  float3 T = f3(txv.x, txv.y, txv.z), R = f3(rxv.x, rxv.y, rxv.z);
  float3 S = first ? mirror32(T, n, c) : T, O = first ? R : mirror32(R, n, c);
  if (!diffract_candidate(W, make_float4(S.x, S.y, S.z, 0.0f), make_float4(O.x, O.y, O.z, 0.0f))) return false;
  const float3 e = W.e, p0 = W.p0;
  float3 dt = f3(S.x - p0.x, S.y - p0.y, S.z - p0.z), dr = f3(O.x - p0.x, O.y - p0.y, O.z - p0.z);
  float zt = fdot3(dt, e), zr = fdot3(dr, e);
  float3 pt = f3(dt.x - e.x * zt, dt.y - e.y * zt, dt.z - e.z * zt);
  float3 pr = f3(dr.x - e.x * zr, dr.y - e.y * zr, dr.z - e.z * zr);
  float rt = sqrtf(fdot3(pt, pt)), rr = sqrtf(fdot3(pr, pr));
  if (!(rt > 1e-3f && rr > 1e-3f)) return true;
  float zq = zt + (zr - zt) * rt / (rt + rr);
  float3 Q = f3(p0.x + e.x * zq, p0.y + e.y * zq, p0.z + e.z * zq);
  float3 a0 = first ? S : Q, a1 = first ? Q : O;
  float3 dv = f3(a1.x - a0.x, a1.y - a0.y, a1.z - a0.z);
  float den = fdot3(n, dv), len = sqrtf(fdot3(dv, dv));
  if (!(fabsf(den) > 1e-6f * len)) return true;
  float t = (c - fdot3(n, a0)) / den;
  float mt = (0.05f + 1e-4f * (len + sqrtf(fdot3(a0, a0)))) / len;
  if (t < -mt || t > 1.0f + mt) return false;
  float3 X = f3(a0.x + t * dv.x, a0.y + t * dv.y, a0.z + t * dv.z);
  float mb = 0.05f + 1e-4f * (len + sqrtf(fdot3(X, X)));
  if (X.x < P.box[0] - mb || X.y < P.box[1] - mb || X.z < P.box[2] - mb || X.x > P.box[3] + mb ||
      X.y > P.box[4] + mb || X.z > P.box[5] + mb)
    return false;
  return true;
}

__global__ void __launch_bounds__(256) k_diffract_refl_pre(PathArgs a, int nlinks) {
  const long total = (long)nlinks * a.nw * a.nrp * 2;
  const int lane = threadIdx.x & 31;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long base = (long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total; base += stride) {
    long idx = base + lane;
    bool keep = false;
    if (idx < total) {
      long r = idx >> 1;
      int p = (int)(r % a.nrp);
      r /= a.nrp;
      int w = (int)(r % a.nw), link = (int)(r / a.nw);
      keep = diffract_refl_candidate(a.wf[w], a.rplanes[p], a.txs[link / a.nrx], a.rx[link % a.nrx],
                                     (idx & 1) != 0);
    }
    unsigned m = __ballot_sync(0xffffffffu, keep);
    if (!m) continue;
    unsigned at = 0;
    if (lane == 0) at = atomicAdd(&a.ctr->n_dsurv, (unsigned)__popc(m));
    at = __shfl_sync(0xffffffffu, at, 0) + __popc(m & ((1u << lane) - 1u));
    if (keep) {
      if (at < a.dsurv_cap) a.dsurv[at] = kReflTag | (unsigned long long)idx;
      else atomicOr(&a.ctr->err, ERR_DIFF_OVERFLOW);
    }
  }
}

// Image, Keller point and reflection point for plane (n, c): false when the
// Keller point leaves the edge, an angle falls inside the wedge, the shadow
// rule fails or the reflection point leaves the unfolded leg.
struct ReflGeom {
  d3w S, O, Q, P;  // source (or image), observer (or image), diffraction and reflection points
  double phip, phi;
};
__device__ __forceinline__ bool refl_geometry(const Wedge& W, d3w n, double c, d3w T, d3w R, bool first,
                                              ReflGeom& g) {
  g.S = first ? T - n * (2.0 * (dotw(n, T) - c)) : T;
  g.O = first ? R : R - n * (2.0 * (dotw(n, R) - c));
  d3w e = D3(W.e[0], W.e[1], W.e[2]), p0 = D3(W.p0[0], W.p0[1], W.p0[2]);
  d3w dt = g.S - p0, dr = g.O - p0;
  double zt = dotw(dt, e), zr = dotw(dr, e);
  d3w pt = dt - e * zt, pr = dr - e * zr;
  double rt = sqrt(dotw(pt, pt)), rr = sqrt(dotw(pr, pr));
  if (!(rt > 0.0 && rr > 0.0)) return false;
  double zq = zt + (zr - zt) * rt / (rt + rr);
  double uq = zq / W.len;
  if (!(uq > 0.0 && uq < 1.0)) return false;
  g.Q = p0 + e * zq;
  g.phip = wedge_angle(W, g.S);
  g.phi = wedge_angle(W, g.O);
  if (g.phip > W.n * M_PI || g.phi > W.n * M_PI) return false;
  if (!(fabs(g.phi - g.phip) > M_PI)) return false;
  d3w a0 = first ? g.S : g.Q, a1 = first ? g.Q : g.O;
  double den = dotw(n, a1 - a0);
  if (den == 0.0) return false;
  double t = (c - dotw(n, a0)) / den;
  if (!(t > 0.0 && t < 1.0)) return false;
  g.P = a0 + (a1 - a0) * t;
  return true;
}


// Can triangle id hold point x (on its plane group's plane, within 1e-4 m of
// the triangle's own)? x must lie in the triangle's FP32 box widened by 1 mm +
// 1e-6 of the coordinates; the FP64 test (inside_tri64) follows for those
// that do.
__device__ __forceinline__ bool tri_box_near(const PathArgs& a, int id, d3w x) {
  const float4* tp = a.tris + 3 * (size_t)DCEM_IDX(a.slot_of_id[DCEM_IDX(id, a.bvh.ntris)], a.bvh.ntris);
  const float4 p0 = tp[0], p1 = tp[1], p2 = tp[2];
  const float X = (float)x.x, Y = (float)x.y, Zc = (float)x.z;
  const float m = 1e-3f + 1e-6f * (fabsf(X) + fabsf(Y) + fabsf(Zc));
  return !(X < fminf(p0.x, fminf(p1.x, p2.x)) - m || X > fmaxf(p0.x, fmaxf(p1.x, p2.x)) + m ||
           Y < fminf(p0.y, fminf(p1.y, p2.y)) - m || Y > fmaxf(p0.y, fmaxf(p1.y, p2.y)) + m ||
           Zc < fminf(p0.z, fminf(p1.z, p2.z)) - m || Zc > fmaxf(p0.z, fmaxf(p1.z, p2.z)) + m);
}

__device__ __forceinline__ bool inside_tri64(d3w v0, d3w v1, d3w v2, d3w x) {
  d3w n = crossw(v1 - v0, v2 - v0);
  return !(dotw(crossw(v1 - v0, x - v0), n) < 0.0 || dotw(crossw(v2 - v1, x - v1), n) < 0.0 ||
           dotw(crossw(v0 - v2, x - v2), n) < 0.0);
}

// The member triangle of plane G holding point x (on G's plane), none of the
// nex ids in ex: the lowest id among the members whose box holds x
// (tri_box_near) and that contain it (inside_tri64) -- the one a scan of the
// members in id order finds first -- with its vertices and material; -1 when
// there is none. The members are sorted by their lowest coordinate along G's
// axis, so only those with that coordinate in [u - 2 m - ext, u + 2 m] can
// pass the box test (u: x's coordinate, m: the test's margin, ext: the
// members' largest extent along the axis): a binary search, then a scan of
// that range.
__device__ int member_at(const PathArgs& a, const RPlane& G, d3w x, const int* ex, int nex, d3w& v0, d3w& v1,
                         d3w& v2, float4& mat) {
  const float X = (float)x.x, Y = (float)x.y, Z = (float)x.z;
  const float m = 1e-3f + 1e-6f * (fabsf(X) + fabsf(Y) + fabsf(Z));
  const float u = G.axis == 0 ? X : (G.axis == 1 ? Y : Z);
  const float hi = u + 2.0f * m, lo = u - 2.0f * m - G.ext * (1.0f + 1e-6f);
  int l = G.first, r = G.first + G.count;  // the first member whose key exceeds hi
  while (l < r) {
    const int mid = (l + r) >> 1;
    if (a.rkeys[mid] <= hi) l = mid + 1;
    else r = mid;
  }
  int best = -1;
  for (int k = l - 1; k >= G.first && a.rkeys[k] >= lo; --k) {
    const int id = a.rmembers[k];
    if (best >= 0 && id > best) continue;
    bool skip = false;
    for (int i = 0; i < nex; ++i) skip = skip || id == ex[i];
    if (skip || !tri_box_near(a, id, x)) continue;
    d3w w0, w1, w2;
    float4 mt;
    tri64(a, id, w0, w1, w2, mt);
    if (inside_tri64(w0, w1, w2, x)) {
      best = id;
      v0 = w0;
      v1 = w1;
      v2 = w2;
      mat = mt;
    }
  }
  return best;
}

struct zv3 {
  zd x, y, z;
};
__device__ __forceinline__ zd zvdot(zv3 E, d3w v) { return E.x * v.x + E.y * v.y + E.z * v.z; }

// One survivor: exact geometry on the plane, the member triangle holding the
// reflection point, the geometry again on that triangle's own plane, the
// three legs, then the UTD field with the Fresnel reflection at P (bounce
// basis as in k_val_field) and the path record (depth 2).
__device__ __forceinline__ void diffract_refl_pair(const PathArgs& a, unsigned long long code, double k,
                                                   double lam, unsigned& ovf, TStack& st) {
  const bool first = (code & 1ull) != 0;
  code >>= 1;
  const int p = (int)(code % (unsigned long long)a.nrp);
  code /= (unsigned long long)a.nrp;
  const int w = (int)(code % (unsigned long long)a.nw), link = (int)(code / (unsigned long long)a.nw);
  const Wedge W = a.wedges[w];
  const RPlane Pl = a.rplanes[p];
  float4 rxv = a.rx[link % a.nrx], txv = a.txs[link / a.nrx];
  d3w T = D3(txv.x, txv.y, txv.z), R = D3(rxv.x, rxv.y, rxv.z);
  ReflGeom g;
  if (!refl_geometry(W, D3(Pl.n[0], Pl.n[1], Pl.n[2]), Pl.c, T, R, first, g)) return;
  d3w v0, v1, v2;
  float4 mj;
  const int exw[2] = {W.ta, W.tb};
  const int j = member_at(a, Pl, g.P, exw, 2, v0, v1, v2, mj);
  if (j < 0) return;
  // the member's own plane
  d3w nj = unitw(crossw(v1 - v0, v2 - v0));
  if (!refl_geometry(W, nj, dotw(nj, v0), T, R, first, g)) return;
  if (!inside_tri64(v0, v1, v2, g.P)) return;
  const d3w Q = g.Q, Pp = g.P;
  if (first) {
    if (leg_occluded(a, T, Pp, j, j, ovf, st) || leg_occluded(a, Pp, Q, j, W.ta, ovf, st, W.tb) ||
        leg_occluded(a, Q, R, W.ta, W.tb, ovf, st))
      return;
  } else {
    if (leg_occluded(a, T, Q, W.ta, W.tb, ovf, st) || leg_occluded(a, Q, Pp, j, W.ta, ovf, st, W.tb) ||
        leg_occluded(a, Pp, R, j, j, ovf, st))
      return;
  }
  unsigned fl = 0;
  const double n = W.n, phip = g.phip, phi = g.phi;
  d3w e = D3(W.e[0], W.e[1], W.e[2]);
  d3w qs = Q - g.S, oq = g.O - Q;
  double sp = sqrt(dotw(qs, qs)), s = sqrt(dotw(oq, oq));
  d3w ip = qs * (1.0 / sp), dd = oq * (1.0 / s);
  double beta0 = acos(fmax(-1.0, fmin(1.0, dotw(ip, e))));
  double sb = sin(beta0);
  double L = s * sp * sb * sb / (s + sp);
  d3w php = unitw(crossw(e, ip)) * -1.0, ph = unitw(crossw(e, dd));
  d3w bp = crossw(ip, php), bd = crossw(dd, ph);
  float4 ma, mb;
  {
    d3w x0, x1, x2;
    tri64(a, W.ta, x0, x1, x2, ma);
    tri64(a, W.tb, x0, x1, x2, mb);
  }
  zd r0s, r0h, rns, rnh;
  fresnel_d(ma, a.freq, fabs(sin(phip)), r0s, r0h);
  fresnel_d(mb, a.freq, fabs(sin(n * M_PI - phi)), rns, rnh);
  const UtdParts up = utd_parts(n, phi, phip, beta0, L, k, fl);
  zd Ds = utd_coeff(up, r0s, rns);
  zd Dh = utd_coeff(up, r0h, rnh);
  // the reflection at P: directions and bounce basis
  d3w din = first ? unitw(Pp - T) : dd;
  d3w dout = first ? ip : unitw(R - Pp);
  double ct = fabs(dotw(din, nj));
  d3w sv = crossw(din, nj);
  double sn_ = sqrt(dotw(sv, sv));
  if (sn_ < 1e-12) {
    d3w ax = fabs(nj.x) < 0.9 ? D3(1, 0, 0) : D3(0, 1, 0);
    sv = unitw(crossw(nj, ax));
  } else {
    sv = sv * (1.0 / sn_);
  }
  d3w pin = crossw(sv, din), pout = crossw(sv, dout);
  zd gte, gtm;
  fresnel_d(mj, a.freq, ct, gte, gtm);
  d3w u = D3(a.pol.x, a.pol.y, a.pol.z);
  double sn, cs;
  sincos(-k * sp, &sn, &cs);
  zd Ei = Z(cs / sp, sn / sp);
  sincos(-k * s, &sn, &cs);
  zd A = Z(cs, sn) * sqrt(sp / (s * (s + sp)));
  zd proj;
  if (first) {
    d3w e0 = polw(u, din, fl);
    zd es = Z(dotw(e0, sv)), ep = Z(dotw(e0, pin));
    zd ts = gte * es, tp = gtm * ep;
    zv3 E1 = {ts * sv.x + tp * pout.x, ts * sv.y + tp * pout.y, ts * sv.z + tp * pout.z};
    zd Eb = Ei * zvdot(E1, bp), Ep = Ei * zvdot(E1, php);
    d3w prx = polw(u, dd * -1.0, fl);
    proj = (Ds * Eb) * (-dotw(bd, prx)) + (Dh * Ep) * (-dotw(ph, prx));
  } else {
    d3w e0 = polw(u, ip, fl);
    zd Eb = Ei * dotw(e0, bp), Ep = Ei * dotw(e0, php);
    zd cb = (Ds * Eb) * -1.0, cp = (Dh * Ep) * -1.0;
    zv3 Ed = {cb * bd.x + cp * ph.x, cb * bd.y + cp * ph.y, cb * bd.z + cp * ph.z};
    zd ts = gte * zvdot(Ed, sv), tp = gtm * zvdot(Ed, pin);
    zv3 E2 = {ts * sv.x + tp * pout.x, ts * sv.y + tp * pout.y, ts * sv.z + tp * pout.z};
    d3w prx = polw(u, dout * -1.0, fl);
    proj = zvdot(E2, prx);
  }
  zd amp = proj * A * (lam / (4.0 * M_PI));
  unsigned uu = atomicAdd(&a.ctr->n_unique, 1u);
  if (uu >= a.ucap) {
    atomicOr(&a.ctr->err, ERR_UNIQUE_OVERFLOW);
    return;
  }
  PathRec rec;
  const int id0 = first ? j : (w | kDiffBit), id1 = first ? (w | kDiffBit) : j;
  rec.key = seq_key(link % a.nrx, 2, [&](int q) { return q == 0 ? id0 : id1; });
  rec.rx = link;
  rec.depth = 2;
  rec.ray = -1;
  rec.flags = fl;
  rec.valid = 1;
  rec.pad = 0;
  rec.len = sp + s;
  rec.amp_re = amp.re;
  rec.amp_im = amp.im;
  for (int q = 0; q < kMaxRefl; ++q) {
    rec.tri[q] = q == 0 ? id0 : q == 1 ? id1 : -1;
    rec.pts[q][0] = rec.pts[q][1] = rec.pts[q][2] = 0.0f;
  }
  const d3w x0 = first ? Pp : Q, x1 = first ? Q : Pp;
  rec.pts[0][0] = (float)x0.x;
  rec.pts[0][1] = (float)x0.y;
  rec.pts[0][2] = (float)x0.z;
  rec.pts[1][0] = (float)x1.x;
  rec.pts[1][1] = (float)x1.y;
  rec.pts[1][2] = (float)x1.z;
  a.prec[uu] = rec;
  unsigned pos = atomicAdd(&a.bucket_cnt[link], 1u);
  if (pos < (unsigned)a.bucket_cap) a.bucket[(size_t)link * a.bucket_cap + pos] = (int)uu;
  else atomicOr(&a.ctr->err, ERR_BUCKET_OVERFLOW);
  atomicAdd(&a.ctr->n_valid, 1u);
}

// ---------------------------------------------------------------------------
// diffraction of order 2 and 3 (Sec. III step 5; the paper's bound is 3)
// ---------------------------------------------------------------------------
// Paths Tx -> Q_1 -> .. -> Q_m -> Rx over m pairwise distinct wedges,
// consecutive ones sharing no vertex, not on one line, neither edge in a
// face plane of the other. Per frame: the
// ordered wedge pairs that can start a path from a transmitter
// (k_diff_pairs), for m = 3 the triples built from them (k_diff_triples),
// then every (sequence, receiver) through an FP32 pre-test
// (k_diff_multi_pre). The pre-tests only reject what the FP64 test rejects
// too (margins above FP32 rounding); the
// survivors go to the diffraction survivor list with their order in the top
// bits: 01 order 2, 11 order 3 (10 is a reflection pair, 00 first order).
constexpr unsigned long long kKindShift = 62;
constexpr unsigned long long kMulti2 = 1ull << kKindShift, kMulti3 = 3ull << kKindShift;

__device__ __forceinline__ WedgeF wedge_f(const Wedge& W) {
  WedgeF f;
  f.p0 = f3((float)W.p0[0], (float)W.p0[1], (float)W.p0[2]);
  f.e = f3((float)W.e[0], (float)W.e[1], (float)W.e[2]);
  f.t0 = f3((float)W.t0[0], (float)W.t0[1], (float)W.t0[2]);
  f.y0 = f3((float)W.y0[0], (float)W.y0[1], (float)W.y0[2]);
  f.len = (float)W.len;
  f.npi = (float)(W.n * M_PI);
  return f;
}
// X in the wedge's normal plane: (along t0, along y0), its distance from the
// edge line and from the wedge's start.
__device__ __forceinline__ float2 wedge_plane(const WedgeF& W, float3 X, float& r, float& dist) {
  float3 d = f3(X.x - W.p0.x, X.y - W.p0.y, X.z - W.p0.z);
  float z = fdot3(d, W.e);
  float3 q = f3(d.x - W.e.x * z, d.y - W.e.y * z, d.z - W.e.z * z);
  r = sqrtf(fdot3(q, q));
  dist = sqrtf(fdot3(d, d));
  return make_float2(fdot3(q, W.t0), fdot3(q, W.y0));
}
// The point at parameter t along the edge.
__device__ __forceinline__ float3 edge_point(const WedgeF& W, float t) {
  return f3(W.p0.x + W.e.x * t, W.p0.y + W.e.y * t, W.p0.z + W.e.z * t);
}
// The edge's end points.
__device__ __forceinline__ void edge_ends(const WedgeF& W, float3& A, float3& B) {
  A = W.p0;
  B = f3(W.p0.x + W.e.x * W.len, W.p0.y + W.e.y * W.len, W.p0.z + W.e.z * W.len);
}
// Could some point of segment A-B lie strictly inside the angular sector
// (lo, hi) about wedge W (angles from face 0 through the exterior, hi - lo
// below pi)? The sector is the intersection of two half-spaces bounded by
// planes through the edge line, so the test clips the segment's parameter
// range against both; each plane is moved outward by `m` (metres) and the
// sector widened by `ta` (radians) first, so the answer is "no" only when
// the exact sector misses the segment by more than the margins.
__device__ __forceinline__ bool sector_meets(const WedgeF& W, float lo, float hi, float ta, float m, float3 A,
                                             float3 B) {
  lo -= ta;
  hi += ta;
  if (hi - lo >= 3.14f) return true;
  float ra, rb, da, db;
  float2 pa = wedge_plane(W, A, ra, da), pb = wedge_plane(W, B, rb, db);
  float u0 = 0.0f, u1 = 1.0f;
  for (int q = 0; q < 2; ++q) {
    float ang = q == 0 ? lo : hi, sg = q == 0 ? 1.0f : -1.0f;
    float c = cosf(ang), s = sinf(ang);
    // signed distance beyond the plane at angle `ang` toward the sector's inside
    float fa = sg * (c * pa.y - s * pa.x) + m, fb = sg * (c * pb.y - s * pb.x) + m;
    if (fa < 0.0f && fb < 0.0f) return false;
    if (fa < 0.0f) u0 = fmaxf(u0, fa / (fa - fb));
    else if (fb < 0.0f) u1 = fminf(u1, fa / (fa - fb));
  }
  return u0 <= u1 + 1e-3f;
}
// Margins of the pre-tests: angles by ten times their rounding bound (at
// least 1e-3 rad), positions by 5 cm plus 1e-5 of the coordinates' size.
__device__ __forceinline__ float pre_margin_m(float3 X) {
  return 0.05f + 1e-5f * (fabsf(X.x) + fabsf(X.y) + fabsf(X.z));
}
// Is X certainly inside wedge W (beyond its exterior [0, n pi])?
__device__ __forceinline__ bool surely_inside(const WedgeF& W, float3 X) {
  float r, dist;
  float2 p = wedge_plane(W, X, r, dist);
  bool sure;
  float tol;
  float a = wedge_angle32(f3(p.x * W.t0.x + p.y * W.y0.x, p.x * W.t0.y + p.y * W.y0.y, p.x * W.t0.z + p.y * W.y0.z),
                          W.t0, W.y0, r, dist, sure, tol);
  return sure && r > pre_margin_m(X) && a > W.npi + tol;
}
// Could some point of edge B's segment be in wedge A's exterior [0, n pi]?
__device__ __forceinline__ bool edge_sees(const WedgeF& A, const WedgeF& B, float m) {
  float3 P, Q;
  edge_ends(B, P, Q);
  // n >= 1: the interior (n pi, 2 pi) is a convex sector, so the segment is
  // inside it only when both ends are; n < 1: the exterior is the convex one
  if (A.npi >= 3.14159265f) return !(surely_inside(A, P) && surely_inside(A, Q));
  return sector_meets(A, 0.0f, A.npi, 1e-3f, m, P, Q);
}
// Could a point of segment P-Q be beyond the incident shadow boundary of a
// source X at wedge W (|phi - phi'| > pi, phi <= n pi)? The rule is
// symmetric in the two points, so this also tests a receiver X against the
// previous edge.
__device__ __forceinline__ bool shadow_meets(const WedgeF& W, float3 X, float3 P, float3 Q) {
  float r, dist;
  float2 p = wedge_plane(W, X, r, dist);
  float m = fmaxf(pre_margin_m(X), fmaxf(pre_margin_m(P), pre_margin_m(Q)));
  if (!(r > m)) return true;
  bool sure;
  float tol;
  float a = wedge_angle32(f3(p.x * W.t0.x + p.y * W.y0.x, p.x * W.t0.y + p.y * W.y0.y, p.x * W.t0.z + p.y * W.y0.z),
                          W.t0, W.y0, r, dist, sure, tol);
  if (!sure) return true;
  if (a > W.npi + tol) return false;  // X inside the wedge
  const float pi = 3.14159265f;
  if (fabsf(a - pi) <= tol) return true;
  float lo = a < pi ? a + pi : 0.0f, hi = a < pi ? W.npi : a - pi;
  if (hi < lo - tol) return false;
  return sector_meets(W, lo, hi, tol, m, P, Q);
}

// Keller points from the convexity of the unfolded length. The length of a
// chain is a sum of distances between affine functions of the edge
// parameters, so it is convex in them jointly and its derivative along one
// edge, e.(Q - A)/|Q - A| + e.(Q - B)/|Q - B| for Q's neighbours A and B,
// does not decrease as Q moves along the edge. When that derivative is
// positive at the edge's start (less a margin) for every position of the
// neighbours on their edges, or negative at its end, the minimum -- the
// Keller points -- has Q, or a neighbour, off its edge, and the exact stage
// rejects the chain. The tests below bound the derivative's two terms.

// Extremes of e.(Q - Y)/|Q - Y| for Y on wedge S's edge with parameter in
// [lo, hi], and a lower bound of |Q - Y| there. The directions from Q to the
// segment's points sweep an arc of a great circle (below pi), along which
// the cosine is |e_p| cos(angle to e_p), e_p the projection of e onto the
// arc's plane: the extremes are at the arc's ends, or +-|e_p| where e_p (or
// -e_p) points into the arc.
__device__ __forceinline__ void cos_over_edge(float3 e, float3 Q, const WedgeF& S, float lo, float hi, float& cmin,
                                              float& cmax, float& dmin) {
  const float3 d0 = f3(Q.x - S.p0.x - S.e.x * lo, Q.y - S.p0.y - S.e.y * lo, Q.z - S.p0.z - S.e.z * lo);
  const float3 d1 = f3(Q.x - S.p0.x - S.e.x * hi, Q.y - S.p0.y - S.e.y * hi, Q.z - S.p0.z - S.e.z * hi);
  const float l0 = sqrtf(fdot3(d0, d0)), l1 = sqrtf(fdot3(d1, d1));
  const float c0 = fdot3(e, d0) / l0, c1 = fdot3(e, d1) / l1;
  cmin = fminf(c0, c1);
  cmax = fmaxf(c0, c1);
  const float3 n = cross3(d0, d1);
  const float nn = sqrtf(fdot3(n, n));
  dmin = fminf(fminf(l0, l1), nn / (hi - lo));  // the distance to the segment's line at most
  if (nn > 1e-3f * l0 * l1) {
    const float3 u = f3(n.x / nn, n.y / nn, n.z / nn);
    const float en = fdot3(e, u), pn = sqrtf(fmaxf(0.0f, 1.0f - en * en));
    const float3 ep = f3(e.x - en * u.x, e.y - en * u.y, e.z - en * u.z);
    // e_p between the arc's ends (with a tolerance that only widens the range)
    const float s0 = fdot3(ep, cross3(u, d0)), s1 = fdot3(ep, cross3(d1, u));
    const float g0 = 1e-3f * l0, g1 = 1e-3f * l1;
    if (s0 >= -g0 && s1 >= -g1) cmax = fmaxf(cmax, pn);
    if (s0 <= g0 && s1 <= g1) cmin = fminf(cmin, -pn);
  } else {  // an arc shorter than 1e-3 rad (or Q on the segment: dmin tells)
    cmin -= 2e-3f;
    cmax += 2e-3f;
  }
}
// Could the Keller point on wedge W's edge lie within m of the edge, its
// neighbours being point F (has_f) or a point of wedge S1's edge, and a
// point of wedge S2's edge, both edges widened by m? False only when the
// derivative's bound keeps its sign at both ends by more than its FP32
// rounding (1e-6 of the coordinates' size over the distance, per term).
__device__ bool keller_on_edge(const WedgeF& W, bool has_f, float3 F, const WedgeF& S1, const WedgeF& S2, float m) {
  for (int q = 0; q < 2; ++q) {
    const float t = q ? W.len + m : -m;
    const float3 Q = edge_point(W, t);
    const float sq = fabsf(Q.x) + fabsf(Q.y) + fabsf(Q.z);
    float lo1, hi1, d1, lo2, hi2, d2, s1;
    if (has_f) {
      const float3 d = f3(Q.x - F.x, Q.y - F.y, Q.z - F.z);
      d1 = sqrtf(fdot3(d, d));
      lo1 = hi1 = fdot3(W.e, d) / d1;
      s1 = fabsf(F.x) + fabsf(F.y) + fabsf(F.z);
    } else {
      cos_over_edge(W.e, Q, S1, -m, S1.len + m, lo1, hi1, d1);
      s1 = fabsf(S1.p0.x) + fabsf(S1.p0.y) + fabsf(S1.p0.z) + S1.len;
    }
    cos_over_edge(W.e, Q, S2, -m, S2.len + m, lo2, hi2, d2);
    const float s2 = fabsf(S2.p0.x) + fabsf(S2.p0.y) + fabsf(S2.p0.z) + S2.len;
    if (!(d1 > 4.0f * m && d2 > 4.0f * m)) return true;
    const float err = 4e-5f + 2e-6f * ((sq + s1) / d1 + (sq + s2) / d2);
    if (q == 0 && lo1 + lo2 > err) return false;
    if (q == 1 && hi1 + hi2 < -err) return false;
  }
  return true;
}
// The margin of these tests: 5 cm plus 1e-5 of the coordinates' size.
__device__ __forceinline__ float keller_margin(const WedgeF& W, float3 F) {
  return 0.05f + 1e-5f * (fabsf(W.p0.x) + fabsf(W.p0.y) + fabsf(W.p0.z) + W.len + fabsf(F.x) + fabsf(F.y) + fabsf(F.z));
}

// Do two edges share an end vertex (identical coordinates)? Consecutive
// wedges of a chain may not (which includes sharing a face): the length's
// minimum then tends to the common corner, or the leg between them runs
// along a face they bound.
__device__ __forceinline__ bool share_vertex(const Wedge& A, const Wedge& B) {
  const double* a[2] = {A.p0, A.p1};
  const double* b[2] = {B.p0, B.p1};
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      if (a[i][0] == b[j][0] && a[i][1] == b[j][1] && a[i][2] == b[j][2]) return true;
  return false;
}

// Do two edges lie on one line (directions parallel to 1e-9, the second's
// start within 1e-9 m, relative to the coordinates' size, of the first's
// line)? Consecutive wedges of a chain may not: the leg between them would
// run along both edges (no Keller points: the length's minimum is where it
// vanishes). Decided in FP64 from the wedges' frames.
__device__ __forceinline__ bool collinear_edges(const Wedge& A, const Wedge& B) {
  d3w ea = D3(A.e[0], A.e[1], A.e[2]), eb = D3(B.e[0], B.e[1], B.e[2]);
  d3w c = crossw(ea, eb);
  if (sqrt(dotw(c, c)) > 1e-9) return false;
  d3w pa = D3(A.p0[0], A.p0[1], A.p0[2]), pb = D3(B.p0[0], B.p0[1], B.p0[2]);
  d3w q = crossw(pb - pa, ea);
  double sa = fmax(fabs(pa.x), fmax(fabs(pa.y), fabs(pa.z))), sb = fmax(fabs(pb.x), fmax(fabs(pb.y), fabs(pb.z)));
  return sqrt(dotw(q, q)) <= 1e-9 * (1.0 + sa + sb);
}

// Does edge B lie in the plane of a face of wedge A (both ends within 1e-9 m,
// relative to the coordinates' size)? Then so does the leg between them,
// along that face (grazing) or its extension beyond A's edge, where no source
// in A's exterior has its shadow boundary crossed: no chain passes.
__device__ __forceinline__ bool in_face_plane(const Wedge& A, const Wedge& B) {
  d3w e = D3(A.e[0], A.e[1], A.e[2]), pa = D3(A.p0[0], A.p0[1], A.p0[2]);
  d3w b0 = D3(B.p0[0], B.p0[1], B.p0[2]) - pa, b1 = D3(B.p1[0], B.p1[1], B.p1[2]) - pa;
  double sa = fmax(fabs(pa.x), fmax(fabs(pa.y), fabs(pa.z)));
  double sb = fmax(fabs(B.p0[0]), fmax(fabs(B.p0[1]), fabs(B.p0[2])));
  double tol = 1e-9 * (1.0 + sa + sb);
  d3w f[2] = {crossw(e, D3(A.t0[0], A.t0[1], A.t0[2])), crossw(e, D3(A.tB[0], A.tB[1], A.tB[2]))};
  for (int q = 0; q < 2; ++q)
    if (fabs(dotw(f[q], b0)) <= tol && fabs(dotw(f[q], b1)) <= tol) return true;
  return false;
}

// Source v of a chain (a transmitter, or its image in a reflector plane) and
// observer rho (a receiver, or its image), in FP32 for the pre-tests.
__device__ __forceinline__ float3 chain_source32(const PathArgs& a, int v) {
  if (v < a.dntx) {
    float4 t = a.txs[v];
    return f3(t.x, t.y, t.z);
  }
  int i = v - a.dntx;
  float4 t = a.txs[i / a.nrpr];
  const RPlane& P = a.rplanes[i % a.nrpr];
  return mirror32(f3(t.x, t.y, t.z), f3(P.nf[0], P.nf[1], P.nf[2]), P.cf);
}
__device__ __forceinline__ float3 chain_observer32(const PathArgs& a, int rho) {
  if (rho < a.nrx) {
    float4 r = a.rx[rho];
    return f3(r.x, r.y, r.z);
  }
  int i = rho - a.nrx;
  float4 r = a.rx[i / a.nrpr];
  const RPlane& P = a.rplanes[i % a.nrpr];
  return mirror32(f3(r.x, r.y, r.z), f3(P.nf[0], P.nf[1], P.nf[2]), P.cf);
}

// Can a leg from S to some point of segment A-B cross reflector plane Pl
// inside its box? The legs fill the triangle S, A, B; its section by the
// plane lies within the box of the crossings of its three sides, so the
// answer is "no" when S, A and B lie on one side of the plane (by more than
// the margin m), or when that box, widened by m, misses the plane's box.
__device__ __forceinline__ bool plane_reachable(const RPlane& Pl, float3 S, float3 A, float3 B, float m) {
  const float3 n = f3(Pl.nf[0], Pl.nf[1], Pl.nf[2]);
  const float c = Pl.cf;
  const float ds = fdot3(n, S) - c, da = fdot3(n, A) - c, db = fdot3(n, B) - c;
  if ((ds > m && da > m && db > m) || (ds < -m && da < -m && db < -m)) return false;
  float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
  bool any = false;
  const float3 P0[3] = {S, S, A}, P1[3] = {A, B, B};
  const float d0[3] = {ds, ds, da}, d1[3] = {da, db, db};
  for (int e = 0; e < 3; ++e) {
    if ((d0[e] > m && d1[e] > m) || (d0[e] < -m && d1[e] < -m)) continue;
    // the part of this side within m of the plane
    float den = d0[e] - d1[e];
    float ta = 0.0f, tb = 1.0f;
    if (fabsf(den) > 1e-30f) {
      float t1 = (d0[e] - m) / den, t2 = (d0[e] + m) / den;
      ta = fmaxf(0.0f, fminf(t1, t2));
      tb = fminf(1.0f, fmaxf(t1, t2));
    }
    if (ta > tb) continue;
    for (int q = 0; q < 2; ++q) {
      float t = q ? tb : ta;
      float x = P0[e].x + t * (P1[e].x - P0[e].x), y = P0[e].y + t * (P1[e].y - P0[e].y),
            z = P0[e].z + t * (P1[e].z - P0[e].z);
      lo[0] = fminf(lo[0], x); lo[1] = fminf(lo[1], y); lo[2] = fminf(lo[2], z);
      hi[0] = fmaxf(hi[0], x); hi[1] = fmaxf(hi[1], y); hi[2] = fmaxf(hi[2], z);
    }
    any = true;
  }
  if (!any) return false;
  for (int k = 0; k < 3; ++k)
    if (hi[k] < Pl.box[k] - m || lo[k] > Pl.box[3 + k] + m) return false;
  return true;
}

// The relation of consecutive wedges in a chain, once per frame (moving
// wedges change it): distinct, no shared vertex, not on one line, neither
// edge in a face plane of the other, each edge partly in the other's
// exterior; one bit per ordered pair (w1, w2) in a.drel.
__global__ void __launch_bounds__(256) k_diff_rel(PathArgs a) {
  const long nw = a.nw, total = nw * nw;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int w1 = (int)(idx / nw), w2 = (int)(idx - (long)w1 * nw);
    bool rel = w1 != w2;
    if (rel) {  // the FP32 exterior tests first: they reject most pairs
      const WedgeF fa = a.wf[w1], fb = a.wf[w2];
      float3 pa, qa;
      edge_ends(fa, pa, qa);
      const float m = fmaxf(pre_margin_m(pa), pre_margin_m(qa));
      rel = edge_sees(fa, fb, m) && edge_sees(fb, fa, m);
    }
    if (rel) {
      const Wedge &A = a.wedges[w1], &B = a.wedges[w2];
      rel = !share_vertex(A, B) && !collinear_edges(A, B) && !in_face_plane(A, B) && !in_face_plane(B, A);
    }
    if (rel) atomicOr(&a.drel[idx >> 5], 1u << (idx & 31));
  }
}

// Ordered pairs (w1, w2) per source (transmitter or transmitter image) that
// can start a path of order >= 2: in the relation (k_diff_rel), the
// transmitter outside w1, some point of edge 2 beyond the incident shadow
// boundary of the transmitter at w1, and a Keller point on w1 possible
// between the transmitter and edge 2 (keller_on_edge).
__global__ void __launch_bounds__(256) k_diff_pairs(PathArgs a, int nsrc) {
  const long nw = a.nw, total = (long)nsrc * nw * nw;
  const int lane = threadIdx.x & 31;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long base = (long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total; base += stride) {
    long idx = base + lane;
    bool keep = false;
    int t = 0, w1 = 0, w2 = 0;
    if (idx < total) {
      t = (int)(idx / (nw * nw));
      long r = idx - (long)t * nw * nw;
      w1 = (int)(r / nw);
      w2 = (int)(r - (long)w1 * nw);
      if ((a.drel[r >> 5] >> (r & 31)) & 1u) {
        const WedgeF fa = a.wf[w1], fb = a.wf[w2];
        float3 T = chain_source32(a, t), P, Q;
        edge_ends(fb, P, Q);
        keep = !surely_inside(fa, T) && shadow_meets(fa, T, P, Q) && keller_on_edge(fa, true, T, fb, fb, keller_margin(fa, T));
        if (keep && t >= a.dntx) {  // the image's leg to edge 1 crosses its plane inside the box
          float3 A1, B1;
          edge_ends(fa, A1, B1);
          float mg = 0.1f + 1e-4f * (fabsf(T.x) + fabsf(T.y) + fabsf(T.z) + fa.len);
          keep = plane_reachable(a.rplanes[(t - a.dntx) % a.nrpr], T, A1, B1, mg);
        }
      }
    }
    unsigned mk = __ballot_sync(0xffffffffu, keep);
    if (!mk) continue;
    unsigned at = 0;
    if (lane == 0) at = atomicAdd(&a.ctr->n_dpair, (unsigned)__popc(mk));
    at = __shfl_sync(0xffffffffu, at, 0) + __popc(mk & ((1u << lane) - 1u));
    if (keep) {
      if (at < a.dseq2_cap) a.dseq2[at] = make_int4(t, w1, w2, -1);
      else atomicOr(&a.ctr->err, ERR_DIFF_OVERFLOW);
    }
  }
}

// A wedge's FP32 frame mirrored in plane (n, c): the point and directions
// mirrored, the length and exterior angle kept (the angle of a mirrored
// point about the mirrored edge is that of the point about the edge).
__device__ __forceinline__ WedgeF wedge_mirror32(const WedgeF& W, float3 n, float c) {
  auto dir = [&](float3 v) {
    const float h = 2.0f * fdot3(n, v);
    return f3(v.x - h * n.x, v.y - h * n.y, v.z - h * n.z);
  };
  WedgeF M = W;
  M.p0 = mirror32(W.p0, n, c);
  M.e = dir(W.e);
  M.t0 = dir(W.t0);
  M.y0 = dir(W.y0);
  return M;
}

// A wedge mirrored in plane (n, c) in FP64 (as wedge_mirror32).
__device__ __forceinline__ Wedge wedge_mirror64(const Wedge& W, d3w n, double c) {
  auto put = [](double* dst, d3w v) {
    dst[0] = v.x;
    dst[1] = v.y;
    dst[2] = v.z;
  };
  auto pt = [&](const double* x) {
    const d3w v = D3(x[0], x[1], x[2]);
    return v - n * (2.0 * (dotw(n, v) - c));
  };
  auto dir = [&](const double* x) {
    const d3w v = D3(x[0], x[1], x[2]);
    return v - n * (2.0 * dotw(n, v));
  };
  Wedge M = W;
  put(M.p0, pt(W.p0));
  put(M.p1, pt(W.p1));
  put(M.e, dir(W.e));
  put(M.t0, dir(W.t0));
  put(M.y0, dir(W.y0));
  put(M.tB, dir(W.tB));
  return M;
}

// Does the edge of W lie in plane (n, c) up to rounding (both ends within
// 1e-12 m, relative to the coordinates' size)? A reflection in that plane
// next to the edge would sit at the diffraction point itself (the oracle
// flags such a reflection point at its leg's end).
__device__ __forceinline__ bool edge_in_plane(const Wedge& W, d3w n, double c) {
  const double tol = 1e-12 * (1.0 + fmax(fabs(W.p0[0]), fmax(fabs(W.p0[1]), fabs(W.p0[2]))));
  return fabs(dotw(n, D3(W.p0[0], W.p0[1], W.p0[2])) - c) <= tol &&
         fabs(dotw(n, D3(W.p1[0], W.p1[1], W.p1[2])) - c) <= tol;
}

// Can a leg from a point of segment A0-A1 to a point of segment B0-B1 cross
// plane Pl inside its box? Such legs fill the tetrahedron of the four ends,
// whose section by the plane lies within the box of the crossings of its six
// edges; "no" when the four ends lie on one side (by more than m) or that
// box, widened by m, misses the plane's box.
__device__ __forceinline__ bool section_reachable(const RPlane& Pl, float3 A0, float3 A1, float3 B0, float3 B1,
                                                  float m) {
  const float3 n = f3(Pl.nf[0], Pl.nf[1], Pl.nf[2]);
  const float3 X[4] = {A0, A1, B0, B1};
  float d[4];
  bool pos = false, neg = false;
  for (int i = 0; i < 4; ++i) {
    d[i] = fdot3(n, X[i]) - Pl.cf;
    pos = pos || d[i] > -m;
    neg = neg || d[i] < m;
  }
  if (!pos || !neg) return false;
  float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
  bool any = false;
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j) {
      if ((d[i] > m && d[j] > m) || (d[i] < -m && d[j] < -m)) continue;
      const float den = d[i] - d[j];
      float ta = 0.0f, tb = 1.0f;
      if (fabsf(den) > 1e-30f) {
        const float t1 = (d[i] - m) / den, t2 = (d[i] + m) / den;
        ta = fmaxf(0.0f, fminf(t1, t2));
        tb = fminf(1.0f, fmaxf(t1, t2));
      }
      if (ta > tb) continue;
      for (int q = 0; q < 2; ++q) {
        const float t = q ? tb : ta;
        const float x = X[i].x + t * (X[j].x - X[i].x), y = X[i].y + t * (X[j].y - X[i].y),
                    z = X[i].z + t * (X[j].z - X[i].z);
        lo[0] = fminf(lo[0], x); lo[1] = fminf(lo[1], y); lo[2] = fminf(lo[2], z);
        hi[0] = fmaxf(hi[0], x); hi[1] = fmaxf(hi[1], y); hi[2] = fmaxf(hi[2], z);
      }
      any = true;
    }
  if (!any) return false;
  for (int k = 0; k < 3; ++k)
    if (hi[k] < Pl.box[k] - m || lo[k] > Pl.box[3 + k] + m) return false;
  return true;
}

// Wedge pairs with a reflection between them (Sec. III steps 3-5): per
// (transmitter, first wedge, reflector plane), one warp, its lanes over the
// second wedge. By image theory the path Tx -> Q1 -> P -> Q2 -> Rx is the
// chain over w1 and w2's image in the plane; the pair is kept when that
// image and w1 satisfy the pair tests of k_diff_pairs (each partly in the
// other's exterior, some point of the image beyond the transmitter's shadow
// boundary at w1, the transmitter outside w1, a Keller point on w1
// possible) and some leg between the two edges can cross the plane inside
// its box. Entries (t, w1, w2, -2 - p) join
// the pair list (k_diff_triples skips them); the FP64 vertex, line and
// face-plane rules are the exact stage's.
__global__ void __launch_bounds__(256) k_diff_mid_pairs(PathArgs a) {
  const long nblk = (long)a.dntx * a.nw * a.nrp;
  const int lane = threadIdx.x & 31;
  const long nwarp = (long)gridDim.x * (blockDim.x >> 5);
  for (long b = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < nblk; b += nwarp) {
    const int p = (int)(b % a.nrp);
    const long r = b / a.nrp;
    const int w1 = (int)(r % a.nw), t = (int)(r / a.nw);
    const WedgeF fa = a.wf[w1];
    const float3 T = chain_source32(a, t);
    if (surely_inside(fa, T)) continue;  // warp-uniform
    const RPlane& Pl = a.rplanes[p];
    const float3 n = f3(Pl.nf[0], Pl.nf[1], Pl.nf[2]);
    float3 A0, A1;
    edge_ends(fa, A0, A1);
    for (int w0 = 0; w0 < a.nw; w0 += 32) {
      const int w2 = w0 + lane;
      bool keep = false;
      if (w2 < a.nw && w2 != w1) {
        const WedgeF fb = wedge_mirror32(a.wf[w2], n, Pl.cf);
        float3 B0, B1;
        edge_ends(fb, B0, B1);
        const float m = fmaxf(pre_margin_m(A0), pre_margin_m(A1));
        keep = edge_sees(fa, fb, m) && edge_sees(fb, fa, m) && shadow_meets(fa, T, B0, B1);
        if (keep) {
          const float mg = 0.1f + 1e-4f * (fabsf(A0.x) + fabsf(A0.y) + fabsf(A0.z) + fa.len + fb.len);
          keep = section_reachable(Pl, A0, A1, B0, B1, mg) && keller_on_edge(fa, true, T, fb, fb, keller_margin(fa, T));
        }
        if (keep) {  // the exact stage's FP64 rules on the group plane's image
          const Wedge &A = a.wedges[w1], &B = a.wedges[w2];
          const d3w n64 = D3(Pl.n[0], Pl.n[1], Pl.n[2]);
          const Wedge Bm = wedge_mirror64(B, n64, Pl.c);
          keep = !edge_in_plane(A, n64, Pl.c) && !edge_in_plane(B, n64, Pl.c) && !share_vertex(A, Bm) &&
                 !collinear_edges(A, Bm) && !in_face_plane(A, Bm) && !in_face_plane(Bm, A);
        }
      }
      const unsigned mk = __ballot_sync(0xffffffffu, keep);
      if (!mk) continue;
      unsigned at = 0;
      if (lane == 0) at = atomicAdd(&a.ctr->n_dpair, (unsigned)__popc(mk));
      at = __shfl_sync(0xffffffffu, at, 0) + __popc(mk & ((1u << lane) - 1u));
      if (keep) {
        if (at < a.dseq2_cap) a.dseq2[at] = make_int4(t, w1, w2, -2 - p);
        else atomicOr(&a.ctr->err, ERR_DIFF_OVERFLOW);
      }
    }
  }
}

// Triples (w1, w2, w3) from the pairs: (w2, w3) in the relation, w3 not w1,
// and a Keller point on w2 possible between edges 1 and 3 (keller_on_edge).
__global__ void __launch_bounds__(256) k_diff_triples(PathArgs a) {
  const long nw = a.nw;
  const long np = (long)min(a.ctr->n_dpair, a.dseq2_cap), total = np * nw;
  const int lane = threadIdx.x & 31;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long base = (long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total; base += stride) {
    long idx = base + lane;
    bool keep = false;
    int4 pr = make_int4(0, 0, 0, -1);
    int w3 = 0;
    if (idx < total) {
      long p = idx / nw;
      w3 = (int)(idx - p * nw);
      pr = a.dseq2[p];
      size_t bit = (size_t)pr.z * nw + w3;
      keep = pr.w == -1 && w3 != pr.y && ((a.drel[bit >> 5] >> (bit & 31)) & 1u);
      if (keep) {  // the Keller point on the middle edge between the other two
        const WedgeF f2 = a.wf[pr.z];
        keep = keller_on_edge(f2, false, f2.p0, a.wf[pr.y], a.wf[w3], keller_margin(f2, f2.p0));
      }
    }
    unsigned mk = __ballot_sync(0xffffffffu, keep);
    if (!mk) continue;
    unsigned at = 0;
    if (lane == 0) at = atomicAdd(&a.ctr->n_dtrip, (unsigned)__popc(mk));
    at = __shfl_sync(0xffffffffu, at, 0) + __popc(mk & ((1u << lane) - 1u));
    if (keep) {
      if (at < a.dseq3_cap) a.dseq3[at] = make_int4(pr.x, pr.y, pr.z, w3);
      else atomicOr(&a.ctr->err, ERR_DIFF_OVERFLOW);
    }
  }
}

// FP32 Keller points of a chain (the pre-test's estimate): Newton's method
// as in keller_chain, in FP32, from the edges' midpoints. Returns true when
// the cosine mismatch fell below 2e-6 at every edge, or a full Newton step
// would move no point by more than step_tol (metres).
__device__ __forceinline__ float chain_len32(const WedgeF* W, int m, float3 T, float3 R, const float* t) {
  float3 prev = T;
  float L = 0.0f;
  for (int i = 0; i < m; ++i) {
    float3 q = edge_point(W[i], t[i]);
    float3 d = f3(q.x - prev.x, q.y - prev.y, q.z - prev.z);
    L += sqrtf(fdot3(d, d));
    prev = q;
  }
  float3 d = f3(R.x - prev.x, R.y - prev.y, R.z - prev.z);
  return L + sqrtf(fdot3(d, d));
}
__device__ bool keller32(const WedgeF* W, int m, float3 T, float3 R, float* t, float step_tol) {
  for (int i = 0; i < m; ++i) t[i] = 0.5f * W[i].len;
  float Lc = chain_len32(W, m, T, R, t);
  for (int it = 0; it < 30; ++it) {
    float3 X[5];
    X[0] = T;
    for (int i = 0; i < m; ++i) X[i + 1] = edge_point(W[i], t[i]);
    X[m + 1] = R;
    float g[3] = {0.0f, 0.0f, 0.0f}, H[3][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
    for (int j = 0; j <= m; ++j) {
      float3 d = f3(X[j + 1].x - X[j].x, X[j + 1].y - X[j].y, X[j + 1].z - X[j].z);
      float l = sqrtf(fdot3(d, d));
      if (!(l > 0.0f)) return false;
      float3 u = f3(d.x / l, d.y / l, d.z / l);
      int ia = j - 1, ib = j;
      float ca = ia >= 0 ? fdot3(W[ia].e, u) : 0.0f, cb = ib < m ? fdot3(W[ib].e, u) : 0.0f;
      if (ib < m) {
        g[ib] += cb;
        H[ib][ib] += (1.0f - cb * cb) / l;
      }
      if (ia >= 0) {
        g[ia] -= ca;
        H[ia][ia] += (1.0f - ca * ca) / l;
      }
      if (ia >= 0 && ib < m) {
        float h = -(fdot3(W[ia].e, W[ib].e) - ca * cb) / l;
        H[ia][ib] += h;
        H[ib][ia] += h;
      }
    }
    float gmax = 0.0f;
    for (int i = 0; i < m; ++i) gmax = fmaxf(gmax, fabsf(g[i]));
    if (gmax < 2e-6f) return true;
    float A[3][4], dx[3];
    for (int i = 0; i < m; ++i) {
      for (int j = 0; j < m; ++j) A[i][j] = H[i][j];
      A[i][m] = -g[i];
    }
    for (int c = 0; c < m; ++c) {
      int piv = c;
      for (int r = c + 1; r < m; ++r)
        if (fabsf(A[r][c]) > fabsf(A[piv][c])) piv = r;
      if (!(fabsf(A[piv][c]) > 1e-30f)) return false;
      if (piv != c)
        for (int j = 0; j <= m; ++j) {
          float x = A[c][j];
          A[c][j] = A[piv][j];
          A[piv][j] = x;
        }
      for (int r = c + 1; r < m; ++r) {
        float f = A[r][c] / A[c][c];
        for (int j = c; j <= m; ++j) A[r][j] -= f * A[c][j];
      }
    }
    for (int i = m - 1; i >= 0; --i) {
      float v = A[i][m];
      for (int j = i + 1; j < m; ++j) v -= A[i][j] * dx[j];
      dx[i] = v / A[i][i];
    }
    float dfull = 0.0f;
    for (int i = 0; i < m; ++i) dfull = fmaxf(dfull, fabsf(dx[i]));
    float step = 1.0f, tn[3] = {t[0], t[1], t[2]};
    bool moved = false;
    for (int q = 0; q < 30; ++q) {
      for (int i = 0; i < m; ++i) tn[i] = t[i] + step * dx[i];
      float Ln = chain_len32(W, m, T, R, tn);
      if (Ln <= Lc * (1.0f + 1e-6f)) {
        Lc = fminf(Lc, Ln);
        moved = true;
        break;
      }
      step *= 0.5f;
    }
    if (!moved) return gmax < 1e-4f;
    for (int i = 0; i < m; ++i) t[i] = tn[i];
    // the full Newton step (the quadratic model's distance to the
    // stationary point) below step_tol: close enough for the margins
    if (dfull < step_tol) return true;
  }
  return false;
}

// Position margin of the FP32 Keller estimate: 5 cm plus 1e-5 of the
// coordinates' size (FP32 rounding of the geometry and of the solve).
__device__ __forceinline__ float chain_margin(float3 T, float3 R) {
  return 0.05f + 1e-5f * (fabsf(T.x) + fabsf(T.y) + fabsf(T.z) + fabsf(R.x) + fabsf(R.y) + fabsf(R.z));
}

// Is the leg o -> o + dv certainly blocked, whatever its true position within
// `delta` of this one? Only a triangle (other than ex0 .. ex3) that the leg
// crosses strictly inside counts: the crossing must lie within the leg's
// occlusion range (eps_occ, 1 - eps_occ) and at least mu from every edge of
// the triangle in its plane, mu = delta (1 + 1/|cos|) + FP32 slack, |cos|
// the leg's angle to the triangle's normal: a leg displaced by delta moves
// its crossing by at most that much. So the exact leg (FP32 any-hit of the
// FP64 points) is blocked too, and the chain is rejected either way. An
// overflow of the stack or of the visit limit answers "not certain".
__device__ __noinline__ bool leg_surely_blocked(const Bvh& bvh, float3 o, float3 dv, float delta, float eps_occ, int ex0,
                                   int ex1, int ex2, int ex3, TStack& st) {
  const float dl = sqrtf(fdot3(dv, dv));
  if (!(dl > 0.0f)) return false;
  const float slack = 2e-3f + 1e-6f * (fabsf(o.x) + fabsf(o.y) + fabsf(o.z) + dl);
  RayPre rp = ray_pre(o, dv);
  st.reset();
  if (bvh.root1 != kEmpty && !st.push(bvh.root1)) return false;
  int cur = bvh.root0;
  for (int visits = 0;; ++visits) {
    if (visits > bvh.max_visits) return false;
    if (cur == kEmpty) {
      if (st.empty()) break;
      cur = st.pop();
      continue;
    }
    if (cur >= 0) {
      const float4* n = bvh.nodes + 4 * (size_t)DCEM_IDX(cur, bvh.nnodes);
      float4 n0 = __ldg(n), n1 = __ldg(n + 1), n2 = __ldg(n + 2), n3 = __ldg(n + 3);
      float tn0, tn1;
      bool h0 = slab(rp, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, 1.0f, tn0);
      bool h1 = slab(rp, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, 1.0f, tn1);
      int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
      if (h0 && h1) {
        if (!st.push(c1)) return false;
        cur = c0;
      } else {
        cur = h0 ? c0 : h1 ? c1 : kEmpty;
      }
      continue;
    }
    float3 v0, v1, v2;
    int id;
    load_tri(bvh.tris, DCEM_IDX(~cur, bvh.ntris), v0, v1, v2, id);
    cur = kEmpty;
    if (id == ex0 || id == ex1 || id == ex2 || id == ex3) continue;
    float3 e01 = f3(v1.x - v0.x, v1.y - v0.y, v1.z - v0.z), e12 = f3(v2.x - v1.x, v2.y - v1.y, v2.z - v1.z);
    float3 e20 = f3(v0.x - v2.x, v0.y - v2.y, v0.z - v2.z);
    float3 nv = cross3(e01, f3(-e20.x, -e20.y, -e20.z));
    float nn = sqrtf(fdot3(nv, nv)), dn = fdot3(dv, nv);
    if (!(fabsf(dn) > 1e-4f * dl * nn)) continue;  // nearly parallel: not certain
    float u = fdot3(f3(v0.x - o.x, v0.y - o.y, v0.z - o.z), nv) / dn;
    float mu = delta * (1.0f + dl * nn / fabsf(dn)) + slack;
    float nu = mu / dl;
    if (!(u > eps_occ + nu && u < 1.0f - eps_occ - nu)) continue;
    float3 H = f3(o.x + dv.x * u, o.y + dv.y * u, o.z + dv.z * u);
    float d0 = fdot3(cross3(e01, f3(H.x - v0.x, H.y - v0.y, H.z - v0.z)), nv) / (sqrtf(fdot3(e01, e01)) * nn);
    float d1 = fdot3(cross3(e12, f3(H.x - v1.x, H.y - v1.y, H.z - v1.z)), nv) / (sqrtf(fdot3(e12, e12)) * nn);
    float d2 = fdot3(cross3(e20, f3(H.x - v2.x, H.y - v2.y, H.z - v2.z)), nv) / (sqrtf(fdot3(e20, e20)) * nn);
    if (fminf(d0, fminf(d1, d2)) > mu) return true;
  }
  return false;
}

// The FP32 estimate of a chain against the FP64 rules, with margins: false
// only when the exact test rejects the chain too -- a Keller point off its
// edge by more than the position margin, or at some wedge a point inside the
// wedge or the shadow rule missed by more than the angle's rounding bound
// plus the angle the position margin subtends at that point's distance from
// the edge.
// *solved: the estimate converged (t then holds it) -- only then can it
// reject anything.
__device__ __noinline__ bool chain_possible(const WedgeF* W, int m, float3 T, float3 R, float* t, bool* solved) {
  float mt = chain_margin(T, R);
  *solved = keller32(W, m, T, R, t, 0.1f * mt);
  if (!*solved) return true;
  float3 X[5];
  X[0] = T;
  for (int i = 0; i < m; ++i) {
    if (t[i] < -mt || t[i] > W[i].len + mt) return false;
    X[i + 1] = edge_point(W[i], t[i]);
  }
  X[m + 1] = R;
  for (int i = 0; i < m; ++i) {
    float a2[2], tl[2];
    bool sure[2];
    for (int q = 0; q < 2; ++q) {
      float r, dist;
      float2 p = wedge_plane(W[i], X[i + 2 * q], r, dist);
      float3 d = f3(p.x * W[i].t0.x + p.y * W[i].y0.x, p.x * W[i].t0.y + p.y * W[i].y0.y,
                    p.x * W[i].t0.z + p.y * W[i].y0.z);
      a2[q] = wedge_angle32(d, W[i].t0, W[i].y0, r, dist, sure[q], tl[q]);
      // points that move with the estimate (the Keller points) carry its margin
      bool moves = q == 0 ? i > 0 : i < m - 1;
      if (moves) {
        if (!(r > 4.0f * mt)) sure[q] = false;
        else tl[q] += 2.0f * mt / r;
      }
    }
    if ((sure[0] && a2[0] > W[i].npi + tl[0]) || (sure[1] && a2[1] > W[i].npi + tl[1])) return false;
    if (sure[0] && sure[1] && fabsf(a2[1] - a2[0]) < 3.14159265f - (tl[0] + tl[1])) return false;
  }
  return true;
}

// Every (sequence, observer): the observer outside the last wedge and some
// point of the previous edge beyond its shadow boundary at the last wedge,
// then the FP32 Keller estimate against the rules, the legs that are real
// (not those to or from an image) against robust occlusion, and, with a
// reflection, its point on the unfolded leg inside the plane's box (5 cm +
// 1e-4 of the distances; as diffract_refl_candidate). Observers: the
// receivers, and with reflector planes their images (rho = nrx + r * nrpr
// + p) for sequences from a real transmitter; a chain has one reflection.
// Stage 1 of k_diff_multi_pre for sequence sq and observer rho: the
// observer outside the last wedge, some point of the previous edge beyond
// its shadow boundary there, and a Keller point on the last edge possible
// between the previous edge and the observer; an image observer's leg from
// the last edge must be able to cross its plane inside the box.
__device__ __forceinline__ bool multi_stage1(const PathArgs& a, int4 sq, bool three, int rho) {
  const bool mid = !three && sq.w <= -2, obs_img = rho >= a.nrx;
  WedgeF fl = a.wf[three ? sq.w : sq.z];
  const WedgeF fp = a.wf[three ? sq.z : sq.y];
  float3 R = chain_observer32(a, rho), P, Q;
  if (mid) {  // a reflection between the wedges: w2 and the receiver mirrored
    const RPlane& Pl = a.rplanes[-2 - sq.w];
    const float3 n = f3(Pl.nf[0], Pl.nf[1], Pl.nf[2]);
    fl = wedge_mirror32(fl, n, Pl.cf);
    R = mirror32(R, n, Pl.cf);
  }
  edge_ends(fp, P, Q);
  bool keep = !surely_inside(fl, R) && shadow_meets(fl, R, P, Q) && keller_on_edge(fl, true, R, fp, fp, keller_margin(fl, R));
  if (keep && !mid && obs_img) {  // the leg from the last edge to the image crosses its plane inside the box
    float3 A1, B1;
    edge_ends(fl, A1, B1);
    float mg = 0.1f + 1e-4f * (fabsf(R.x) + fabsf(R.y) + fabsf(R.z) + fl.len);
    keep = plane_reachable(a.rplanes[(rho - a.nrx) % a.nrpr], R, A1, B1, mg);
  }
  return keep;
}

// Stage 2 for a pair with a reflection between its wedges: the chain over w1
// and w2's image toward the receiver's image (FP32 Keller estimate against
// the rules), the real first and last legs against robust occlusion (the
// last one mirrored back), and the crossing of the unfolded middle leg with
// the plane inside its box.
__device__ __forceinline__ bool mid_stage2(const PathArgs& a, int4 sq, int rho, TStack& st) {
  const RPlane& Pl = a.rplanes[-2 - sq.w];
  const float3 n = f3(Pl.nf[0], Pl.nf[1], Pl.nf[2]);
  WedgeF Wc[2];
  Wc[0] = a.wf[sq.y];
  Wc[1] = wedge_mirror32(a.wf[sq.z], n, Pl.cf);
  const float3 T = chain_source32(a, sq.x), R = chain_observer32(a, rho), Rm = mirror32(R, n, Pl.cf);
  float t[2];
  bool solved;
  bool keep = chain_possible(Wc, 2, T, Rm, t, &solved);
  if (!keep || !solved) return keep;
  const float delta = chain_margin(T, Rm);
  const float3 Q1 = edge_point(Wc[0], t[0]), Q2m = edge_point(Wc[1], t[1]), Q2 = mirror32(Q2m, n, Pl.cf);
  const Wedge &A = a.wedges[sq.y], &B = a.wedges[sq.z];
  float3 dv = f3(Q1.x - T.x, Q1.y - T.y, Q1.z - T.z);
  if (leg_surely_blocked(a.bvh, T, dv, delta, a.eps_occ, -1, -1, A.ta, A.tb, st)) return false;
  dv = f3(R.x - Q2.x, R.y - Q2.y, R.z - Q2.z);
  if (leg_surely_blocked(a.bvh, Q2, dv, delta, a.eps_occ, B.ta, B.tb, -1, -1, st)) return false;
  dv = f3(Q2m.x - Q1.x, Q2m.y - Q1.y, Q2m.z - Q1.z);
  const float den = fdot3(n, dv), len = sqrtf(fdot3(dv, dv));
  if (fabsf(den) > 1e-6f * len) {
    const float tt = (Pl.cf - fdot3(n, Q1)) / den;
    const float mt = (0.05f + delta + 1e-4f * (len + sqrtf(fdot3(Q1, Q1)))) / len;
    if (tt < -mt || tt > 1.0f + mt) return false;
    const float3 Xp = f3(Q1.x + tt * dv.x, Q1.y + tt * dv.y, Q1.z + tt * dv.z);
    const float mb = 0.05f + delta + 1e-4f * (len + sqrtf(fdot3(Xp, Xp)));
    if (Xp.x < Pl.box[0] - mb || Xp.y < Pl.box[1] - mb || Xp.z < Pl.box[2] - mb || Xp.x > Pl.box[3] + mb ||
        Xp.y > Pl.box[4] + mb || Xp.z > Pl.box[5] + mb)
      return false;
    // the two real legs through the reflection point (a crossing near a
    // leg's end, as the reflector's own at P, does not count)
    float3 d1 = f3(Xp.x - Q1.x, Xp.y - Q1.y, Xp.z - Q1.z), d2 = f3(Q2.x - Xp.x, Q2.y - Xp.y, Q2.z - Xp.z);
    if (leg_surely_blocked(a.bvh, Q1, d1, delta, a.eps_occ, A.ta, A.tb, -1, -1, st) ||
        leg_surely_blocked(a.bvh, Xp, d2, delta, a.eps_occ, -1, -1, B.ta, B.tb, st))
      return false;
  }
  return true;
}

// Stage 2 for an index past stage 1: the FP32 Keller estimate against the
// rules, the real legs against robust occlusion, and with a reflection its
// point on the unfolded leg inside the plane's box.
__device__ __forceinline__ bool multi_stage2(const PathArgs& a, long idx, long n2, long nobs, TStack& st) {
  const long e = idx / nobs;
  const int rho = (int)(idx - e * nobs);
  const bool three = e >= n2;
  const long ei = three ? e - n2 : e;
  const int4 sq = three ? a.dseq3[ei] : a.dseq2[ei];
  if (!three && sq.w <= -2) return mid_stage2(a, sq, rho, st);
  const bool src_img = sq.x >= a.dntx, obs_img = rho >= a.nrx;
  const int wl = three ? sq.w : sq.z, wp = three ? sq.z : sq.y;
  WedgeF Wc[3];
  Wc[0] = a.wf[sq.y];
  Wc[1] = a.wf[three ? wp : wl];  // order 2: (w1, last); order 3: (w1, previous, last)
  Wc[2] = a.wf[wl];
  const int m = three ? 3 : 2;
  const float3 T = chain_source32(a, sq.x), R = chain_observer32(a, rho);
  float t[3];
  bool solved;
  bool keep = chain_possible(Wc, m, T, R, t, &solved);
  if (keep && solved) {
    const int w[3] = {sq.y, sq.z, sq.w};
    const float delta = chain_margin(T, R);
    float3 X[5];
    X[0] = T;
    for (int i = 0; i < m; ++i) X[i + 1] = edge_point(Wc[i], t[i]);
    X[m + 1] = R;
    // a leg certainly blocked rejects the chain (legs to or from an
    // image are not real: the reflection breaks them)
    for (int q = 0; keep && q <= m; ++q) {
      if ((q == 0 && src_img) || (q == m && obs_img)) continue;
      const Wedge* A = q >= 1 ? &a.wedges[w[q - 1]] : nullptr;
      const Wedge* B = q < m ? &a.wedges[w[q]] : nullptr;
      float3 dv = f3(X[q + 1].x - X[q].x, X[q + 1].y - X[q].y, X[q + 1].z - X[q].z);
      if (leg_surely_blocked(a.bvh, X[q], dv, delta, a.eps_occ, A ? A->ta : -1, A ? A->tb : -1,
                             B ? B->ta : -1, B ? B->tb : -1, st))
        keep = false;
    }
    if (keep && (src_img || obs_img)) {  // the reflection point within the plane's box
      const RPlane& Pl = a.rplanes[src_img ? (sq.x - a.dntx) % a.nrpr : (rho - a.nrx) % a.nrpr];
      const float3 n = f3(Pl.nf[0], Pl.nf[1], Pl.nf[2]);
      const float3 a0 = src_img ? X[0] : X[m], a1 = src_img ? X[1] : X[m + 1];
      const float3 dv = f3(a1.x - a0.x, a1.y - a0.y, a1.z - a0.z);
      const float den = fdot3(n, dv), len = sqrtf(fdot3(dv, dv));
      if (fabsf(den) > 1e-6f * len) {
        float tt = (Pl.cf - fdot3(n, a0)) / den;
        float mt = (0.05f + delta + 1e-4f * (len + sqrtf(fdot3(a0, a0)))) / len;
        if (tt < -mt || tt > 1.0f + mt) keep = false;
        float3 Xp = f3(a0.x + tt * dv.x, a0.y + tt * dv.y, a0.z + tt * dv.z);
        float mb = 0.05f + delta + 1e-4f * (len + sqrtf(fdot3(Xp, Xp)));
        if (Xp.x < Pl.box[0] - mb || Xp.y < Pl.box[1] - mb || Xp.z < Pl.box[2] - mb ||
            Xp.x > Pl.box[3] + mb || Xp.y > Pl.box[4] + mb || Xp.z > Pl.box[5] + mb)
          keep = false;
        if (keep) {  // the two real legs through the reflection point (its own crossing is at their end)
          const float4 ev = src_img ? a.txs[(sq.x - a.dntx) / a.nrpr] : a.rx[(rho - a.nrx) / a.nrpr];
          const float3 E = f3(ev.x, ev.y, ev.z);        // the real transmitter or receiver
          const float3 Qn = src_img ? X[1] : X[m];     // the diffraction point next to the reflection
          const Wedge& Wn = a.wedges[src_img ? w[0] : w[m - 1]];
          const float3 d1 = f3(Xp.x - E.x, Xp.y - E.y, Xp.z - E.z), d2 = f3(Qn.x - Xp.x, Qn.y - Xp.y, Qn.z - Xp.z);
          if (leg_surely_blocked(a.bvh, E, d1, delta, a.eps_occ, -1, -1, -1, -1, st) ||
              leg_surely_blocked(a.bvh, Xp, d2, delta, a.eps_occ, -1, -1, Wn.ta, Wn.tb, st))
            keep = false;
        }
      }
    }
  }
  return keep;
}

// One warp per sequence, its lanes over the observers: every (sequence,
// observer) through stage 1; the indices (sequence * nobs + observer) that
// pass wait in a per-warp queue and go through stage 2 (the Newton estimate,
// the legs) 32 at a time, so that the costly stage runs on full warps.
// Observers: the receivers, and with reflector planes their images (rho =
// nrx + r * nrpr + p) for sequences from a real transmitter (a chain has one
// reflection: a sequence from an image sees the receivers only).
__global__ void __launch_bounds__(256) k_diff_multi_pre(PathArgs a) {
  extern __shared__ int sstk[];
  __shared__ long wq[8][64];
  TStack st;
  bind_stack(st, sstk, kStackTrace);
  const long n2 = a.diff_order >= 2 ? (long)min(a.ctr->n_dpair, a.dseq2_cap) : 0;
  const long n3 = a.diff_order >= 3 ? (long)min(a.ctr->n_dtrip, a.dseq3_cap) : 0;
  const long nobs = (long)a.nrx * (1 + a.nrpr);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // work items: (sequence, run of kObsRun observers), so that the sequences
  // from a real transmitter, which see every observer, split over warps
  constexpr long kObsRun = 512;
  const long nrun = (nobs + kObsRun - 1) / kObsRun, nitem = (n2 + n3) * nrun;
  const long nwarps = (long)gridDim.x * (blockDim.x >> 5);
  long item = (long)blockIdx.x * (blockDim.x >> 5) + wid - nwarps;
  long e = 0, r0 = 0, r1 = 0;  // the item's sequence and observer range (warp-uniform)
  int4 sq = make_int4(0, 0, 0, 0);
  int qn = 0;                  // queued indices of this warp (warp-uniform)
  for (;;) {
    while (r0 >= r1) {  // the next item with observers
      item += nwarps;
      if (item >= nitem) break;
      e = item / nrun;
      sq = e >= n2 ? a.dseq3[e - n2] : a.dseq2[e];
      const long nob = sq.x >= a.dntx || (e < n2 && sq.w <= -2) ? a.nrx : nobs;
      r0 = (item - e * nrun) * kObsRun;
      r1 = min(r0 + kObsRun, nob);
    }
    const bool more = item < nitem;
    if (more) {
      const long rho = r0 + lane;
      const bool pass = rho < r1 && multi_stage1(a, sq, e >= n2, (int)rho);
      const unsigned mk = __ballot_sync(0xffffffffu, pass);
      if (pass) wq[wid][qn + __popc(mk & ((1u << lane) - 1u))] = e * nobs + rho;
      qn += __popc(mk);
      __syncwarp();
      r0 += 32;
    }
    while (qn >= 32 || (!more && qn > 0)) {
      const int nn = min(qn, 32);
      const long idx = lane < nn ? wq[wid][qn - nn + lane] : -1;
      __syncwarp();
      qn -= nn;
      const bool keep = idx >= 0 && multi_stage2(a, idx, n2, nobs, st);
      const unsigned mk = __ballot_sync(0xffffffffu, keep);
      if (!mk) continue;
      unsigned at = 0;
      if (lane == 0) at = atomicAdd(&a.ctr->n_dsurv, (unsigned)__popc(mk));
      at = __shfl_sync(0xffffffffu, at, 0) + __popc(mk & ((1u << lane) - 1u));
      if (keep) {
        const bool three = idx >= n2 * nobs;
        const unsigned long long code =
            (unsigned long long)(three ? idx - n2 * nobs : idx) | (three ? kMulti3 : kMulti2);
        if (at < a.dsurv_cap) a.dsurv[at] = code;
        else atomicOr(&a.ctr->err, ERR_DIFF_OVERFLOW);
      }
    }
    if (!more) break;
  }
}

// Unfolded length of the chain with edge parameters t.
__device__ __forceinline__ double chain_len(const Wedge* const* E, int m, d3w T, d3w R, const double* t) {
  d3w prev = T;
  double L = 0.0;
  for (int i = 0; i < m; ++i) {
    d3w q = D3(E[i]->p0[0], E[i]->p0[1], E[i]->p0[2]) + D3(E[i]->e[0], E[i]->e[1], E[i]->e[2]) * t[i];
    d3w d = q - prev;
    L += sqrt(dotw(d, d));
    prev = q;
  }
  d3w d = R - prev;
  return L + sqrt(dotw(d, d));
}

// Keller points: the stationary point (the minimum: the length is convex in
// t) of the unfolded length over the edge parameters, by Newton's method
// from the edges' midpoints (at most 50 steps), a step that does not
// shorten the chain halved (at most 40 times) until the cosine mismatch is
// below 1e-8 or the Newton decrement below 1e-15 of the length, full steps
// after that; converged when every edge's mismatch is below 1e-12. A leg shorter than kLegMin stops it: the
// minimum is then at a kink of the length (consecutive edge lines meet),
// where Keller's law has no solution.
constexpr double kLegMin = 1e-6;
__device__ bool keller_chain(const Wedge* const* E, int m, d3w T, d3w R, double* t) {
  for (int i = 0; i < m; ++i) t[i] = 0.5 * E[i]->len;
  double Lc = chain_len(E, m, T, R, t);
  for (int it = 0; it < 50; ++it) {
    d3w X[5];
    X[0] = T;
    for (int i = 0; i < m; ++i)
      X[i + 1] = D3(E[i]->p0[0], E[i]->p0[1], E[i]->p0[2]) + D3(E[i]->e[0], E[i]->e[1], E[i]->e[2]) * t[i];
    X[m + 1] = R;
    double g[3] = {0.0, 0.0, 0.0}, H[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    for (int j = 0; j <= m; ++j) {
      d3w d = X[j + 1] - X[j];
      double l = sqrt(dotw(d, d));
      if (!(l > kLegMin)) return false;
      d3w u = d * (1.0 / l);
      int ia = j - 1, ib = j;
      d3w ea = ia >= 0 ? D3(E[ia]->e[0], E[ia]->e[1], E[ia]->e[2]) : D3(0, 0, 0);
      d3w eb = ib < m ? D3(E[ib]->e[0], E[ib]->e[1], E[ib]->e[2]) : D3(0, 0, 0);
      double ca = dotw(ea, u), cb = dotw(eb, u);
      if (ib < m) {
        g[ib] += cb;
        H[ib][ib] += (1.0 - cb * cb) / l;
      }
      if (ia >= 0) {
        g[ia] -= ca;
        H[ia][ia] += (1.0 - ca * ca) / l;
      }
      if (ia >= 0 && ib < m) {
        double h = -(dotw(ea, eb) - ca * cb) / l;
        H[ia][ib] += h;
        H[ib][ia] += h;
      }
    }
    double gmax = 0.0;
    for (int i = 0; i < m; ++i) gmax = fmax(gmax, fabs(g[i]));
    if (gmax < 1e-12) return true;
    // H dx = -g by elimination with partial pivoting
    double A[3][4], dx[3];
    for (int i = 0; i < m; ++i) {
      for (int j = 0; j < m; ++j) A[i][j] = H[i][j];
      A[i][m] = -g[i];
    }
    for (int c = 0; c < m; ++c) {
      int piv = c;
      for (int r = c + 1; r < m; ++r)
        if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
      if (!(fabs(A[piv][c]) > 1e-300)) return false;
      if (piv != c)
        for (int j = 0; j <= m; ++j) {
          double x = A[c][j];
          A[c][j] = A[piv][j];
          A[piv][j] = x;
        }
      for (int r = c + 1; r < m; ++r) {
        double f = A[r][c] / A[c][c];
        for (int j = c; j <= m; ++j) A[r][j] -= f * A[c][j];
      }
    }
    for (int i = m - 1; i >= 0; --i) {
      double v = A[i][m];
      for (int j = i + 1; j < m; ++j) v -= A[i][j] * dx[j];
      dx[i] = v / A[i][i];
    }
    // near the minimum the full step: the length it saves (the Newton
    // decrement, -g.dx / 2) is below the length's rounding there, so a
    // comparison of lengths cannot judge it -- a mismatch below 1e-8, or a
    // decrement below 1e-15 of the length (long chains reach that floor at
    // larger mismatches)
    double gdx = 0.0;
    for (int i = 0; i < m; ++i) gdx += g[i] * dx[i];
    const bool floor = gmax < 1e-8 || fabs(gdx) <= 2e-15 * Lc;
    double step = 1.0, tn[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < 40; ++q) {
      for (int i = 0; i < m; ++i) tn[i] = t[i] + step * dx[i];
      double Ln = chain_len(E, m, T, R, tn);
      if (Ln <= Lc || floor) {
        Lc = Ln;
        break;
      }
      step *= 0.5;
    }
    double dmax = 0.0;
    for (int i = 0; i < m; ++i) {
      dmax = fmax(dmax, fabs(tn[i] - t[i]));
      t[i] = tn[i];
    }
    if (dmax == 0.0) return gmax < 1e-9;
  }
  return false;
}

// The Keller points of a chain from src to obs and the rules on the
// unfolded chain: every point inside its edge, every leg longer than 1e-9 m,
// at every wedge both neighbours in the exterior and the next point beyond
// the incident shadow boundary of the previous one. X: the chain's points.
__device__ bool chain_geometry(const Wedge* const* E, int m, d3w src, d3w obs, d3w* X, double* ell,
                               double* phip, double* phi) {
  if (wedge_angle(*E[0], src) > E[0]->n * M_PI || wedge_angle(*E[m - 1], obs) > E[m - 1]->n * M_PI) return false;
  double t[3];
  if (!keller_chain(E, m, src, obs, t)) return false;
  X[0] = src;
  for (int i = 0; i < m; ++i) {
    double uq = t[i] / E[i]->len;
    if (!(uq > 0.0 && uq < 1.0)) return false;
    X[i + 1] = D3(E[i]->p0[0], E[i]->p0[1], E[i]->p0[2]) + D3(E[i]->e[0], E[i]->e[1], E[i]->e[2]) * t[i];
  }
  X[m + 1] = obs;
  for (int q = 0; q <= m; ++q) {
    d3w d = X[q + 1] - X[q];
    ell[q] = sqrt(dotw(d, d));
    if (!(ell[q] > 1e-9)) return false;
  }
  for (int i = 0; i < m; ++i) {
    phip[i] = wedge_angle(*E[i], X[i]);
    phi[i] = wedge_angle(*E[i], X[i + 2]);
    const double nn = E[i]->n;
    if (phip[i] > nn * M_PI || phi[i] > nn * M_PI) return false;
    if (!(fabs(phi[i] - phip[i]) > M_PI)) return false;
  }
  return true;
}

// The reflection point of the unfolded leg a0 -> a1 on plane (n, c): false
// when the leg does not cross the plane between its ends.
__device__ __forceinline__ bool leg_plane(d3w a0, d3w a1, d3w n, double c, d3w& P) {
  double den = dotw(n, a1 - a0);
  if (den == 0.0) return false;
  double t = (c - dotw(n, a0)) / den;
  if (!(t > 0.0 && t < 1.0)) return false;
  P = a0 + (a1 - a0) * t;
  return true;
}

// The specular reflection of field E at a triangle with unit normal nj and
// material mj, incoming direction din, outgoing dout: Fresnel TE / TM in the
// bounce basis of k_val_field (s = din x n, p_in = s x din, p_out = s x dout).
__device__ zv3 reflect_field_d(const PathArgs& a, d3w nj, float4 mj, d3w din, d3w dout, zv3 E) {
  double ct = fabs(dotw(din, nj));
  d3w sv = crossw(din, nj);
  double sn = sqrt(dotw(sv, sv));
  if (sn < 1e-12) {
    d3w ax = fabs(nj.x) < 0.9 ? D3(1, 0, 0) : D3(0, 1, 0);
    sv = unitw(crossw(nj, ax));
  } else {
    sv = sv * (1.0 / sn);
  }
  d3w pin = crossw(sv, din), pout = crossw(sv, dout);
  zd gte, gtm;
  fresnel_d(mj, a.freq, ct, gte, gtm);
  zd ts = gte * zvdot(E, sv), tp = gtm * zvdot(E, pin);
  return zv3{ts * sv.x + tp * pout.x, ts * sv.y + tp * pout.y, ts * sv.z + tp * pout.z};
}

// One (sequence, observer) survivor of order m: with an image source or
// observer, the chain is solved on the plane group's image, the member
// triangle j holding the reflection point is found, and everything is
// redone with j's own plane (the oracle takes each static triangle as the
// mirror). Then the Keller points and rules (chain_geometry), the real legs
// (FP32 any-hit; triangle j excluded at the reflection point, the wedges'
// faces at theirs), and the UTD chain: at each wedge the coefficient acts on
// the arriving field in the wedge's edge-fixed bases; the wave behind it has
// a caustic on the edge (radius s along phi^) and one rho_e behind it
// (radius rho_e + s along beta^), rho_e the arriving wavefront's radius of
// curvature along the edge's projection (Euler's formula; the source's
// distance for its spherical wave); spreading sqrt(rho_e / (s (rho_e + s)))
// and distance parameter L = s (rho_e + s) rho_1 rho_2 sin^2 beta_0 /
// (rho_e (rho_1 + s) (rho_2 + s)) (Kouyoumjian & Pathak 1974, straight
// edge), over the unfolded distances (a plane mirror keeps the wavefront's
// radii); the reflection applies Fresnel in the real directions.
// One survivor of a pair with a reflection between its wedges (Sec. III
// steps 3-5): the FP64 chain over w1 and w2's image in the plane toward the
// receiver's image (chain_geometry), the vertex, line and face-plane rules
// on the image, the reflection point where the unfolded middle leg crosses
// the plane, the member triangle holding it and everything again on that
// triangle's own plane; the four real legs (FP32 any-hit; the wedges' faces
// excluded at Q1 and Q2, the triangle at P); then the field: UTD at w1,
// Fresnel at P in the real directions with the wavefront's principal
// directions mirrored, UTD at w2 in the real directions (its angles are
// those about the image). Record: depth 3, {w1 | diffract, triangle,
// w2 | diffract}.
__device__ __noinline__ void diffract_mid(const PathArgs& a, int4 sq, int r, double k, double lam, unsigned& ovf,
                                          TStack& st) {
  const int w1 = sq.y, w2 = sq.z, tx = sq.x;
  const int link = tx * a.nrx + r;
  const Wedge& A = a.wedges[w1];
  const Wedge& B = a.wedges[w2];
  const float4 rxv = a.rx[r], txv = a.txs[tx];
  const d3w T = D3(txv.x, txv.y, txv.z), R = D3(rxv.x, rxv.y, rxv.z);
  const RPlane& G = a.rplanes[-2 - sq.w];
  d3w n = D3(G.n[0], G.n[1], G.n[2]);
  double c = G.c;
  auto mir = [&](d3w x) { return x - n * (2.0 * (dotw(n, x) - c)); };
  int j = -1;
  float4 mj = make_float4(0.f, 0.f, 0.f, 0.f);
  d3w X[4], Pp = D3(0, 0, 0);
  double ell[3], phip[2], phi[2];
  for (int pass = 0; pass < 2; ++pass) {
    const Wedge Bm = wedge_mirror64(B, n, c);  // w2's image in the plane
    if (edge_in_plane(A, n, c) || edge_in_plane(B, n, c)) return;
    if (share_vertex(A, Bm) || collinear_edges(A, Bm) || in_face_plane(A, Bm) || in_face_plane(Bm, A)) return;
    const Wedge* E[2] = {&A, &Bm};
    if (!chain_geometry(E, 2, T, mir(R), X, ell, phip, phi)) return;
    if (!leg_plane(X[1], X[2], n, c, Pp)) return;
    d3w v0, v1, v2;
    if (pass == 0) {  // the member triangle holding P: its own plane next
      const int exw[4] = {A.ta, A.tb, B.ta, B.tb};
      j = member_at(a, G, Pp, exw, 4, v0, v1, v2, mj);
      if (j < 0) return;
      n = unitw(crossw(v1 - v0, v2 - v0));
      c = dotw(n, v0);
    } else {
      tri64(a, j, v0, v1, v2, mj);
      if (!inside_tri64(v0, v1, v2, Pp)) return;
    }
  }
  const d3w Q1 = X[1], Q2 = mir(X[2]);
  // the real legs: two excluded triangles at each point
  const d3w Y[5] = {T, Q1, Pp, Q2, R};
  const int ex[5][2] = {{-1, -1}, {A.ta, A.tb}, {j, j}, {B.ta, B.tb}, {-1, -1}};
  for (int q = 0; q < 4; ++q) {
    const d3w dv = Y[q + 1] - Y[q];
    RayPre rp = ray_pre(f3((float)Y[q].x, (float)Y[q].y, (float)Y[q].z), f3((float)dv.x, (float)dv.y, (float)dv.z));
    if (any_hit(a.bvh, rp, a.eps_occ, 1.0f - a.eps_occ, ex[q][0], ex[q][1], ovf, st, ex[q + 1][0], ex[q + 1][1]))
      return;
  }
  unsigned fl = 0;
  const d3w u = D3(a.pol.x, a.pol.y, a.pol.z);
  d3w ip = (Q1 - T) * (1.0 / ell[0]);
  double sn, cs;
  sincos(-k * ell[0], &sn, &cs);
  const zd Ei = Z(cs / ell[0], sn / ell[0]);
  const d3w e0 = polw(u, ip, fl);
  zv3 Ev = {Ei * e0.x, Ei * e0.y, Ei * e0.z};
  double rho1 = ell[0], rho2 = ell[0];
  d3w dir1 = D3(0, 0, 0), dir2 = D3(0, 0, 0);
  const d3w din = unitw(Pp - Q1), dout = unitw(Q2 - Pp);
  for (int i = 0; i < 2; ++i) {
    const Wedge& W = i == 0 ? A : B;
    const d3w dd = i == 0 ? din : unitw(R - Q2);
    const double s = ell[i + 1], nn = W.n;
    if (i == 1) {  // the reflection at P; the wavefront's principal directions mirrored
      Ev = reflect_field_d(a, n, mj, din, dout, Ev);
      dir1 = dir1 - n * (2.0 * dotw(dir1, n));
      dir2 = dir2 - n * (2.0 * dotw(dir2, n));
      ip = dout;
    }
    const d3w e = D3(W.e[0], W.e[1], W.e[2]);
    const double beta0 = acos(fmax(-1.0, fmin(1.0, dotw(ip, e))));
    const double sb = sin(beta0);
    const d3w php = unitw(crossw(e, ip)) * -1.0, ph = unitw(crossw(e, dd));
    const d3w bp = crossw(ip, php), bd = crossw(dd, ph);
    double rhoe;
    if (i == 0) rhoe = ell[0];
    else {
      const double c1 = dotw(bp, dir1), c2 = dotw(bp, dir2);
      rhoe = 1.0 / (c1 * c1 / rho1 + c2 * c2 / rho2);
    }
    const double L = s * (rhoe + s) * rho1 * rho2 * sb * sb / (rhoe * (rho1 + s) * (rho2 + s));
    const float4 ma =
        a.mats[__float_as_int(a.tris[3 * (size_t)DCEM_IDX(a.slot_of_id[DCEM_IDX(W.ta, a.bvh.ntris)], a.bvh.ntris) + 1].w)];
    const float4 mb =
        a.mats[__float_as_int(a.tris[3 * (size_t)DCEM_IDX(a.slot_of_id[DCEM_IDX(W.tb, a.bvh.ntris)], a.bvh.ntris) + 1].w)];
    zd r0s, r0h, rns, rnh;
    fresnel_d(ma, a.freq, fabs(sin(phip[i])), r0s, r0h);
    fresnel_d(mb, a.freq, fabs(sin(nn * M_PI - phi[i])), rns, rnh);
    const UtdParts up = utd_parts(nn, phi[i], phip[i], beta0, L, k, fl);
    const zd Ds = utd_coeff(up, r0s, rns), Dh = utd_coeff(up, r0h, rnh);
    sincos(-k * s, &sn, &cs);
    const zd Am = Z(cs, sn) * sqrt(rhoe / (s * (rhoe + s)));
    const zd cb = Ds * zvdot(Ev, bp) * Am * -1.0, cp = Dh * zvdot(Ev, php) * Am * -1.0;
    Ev = zv3{cb * bd.x + cp * ph.x, cb * bd.y + cp * ph.y, cb * bd.z + cp * ph.z};
    rho1 = s;
    dir1 = ph;
    rho2 = rhoe + s;
    dir2 = bd;
    ip = dd;
  }
  const d3w prx = polw(u, ip * -1.0, fl);
  const zd amp = zvdot(Ev, prx) * (lam / (4.0 * M_PI));
  unsigned uu = atomicAdd(&a.ctr->n_unique, 1u);
  if (uu >= a.ucap) {
    atomicOr(&a.ctr->err, ERR_UNIQUE_OVERFLOW);
    return;
  }
  const int ids[3] = {w1 | kDiffBit, j, w2 | kDiffBit};
  PathRec rec;
  rec.key = seq_key(r, 3, [&](int q) { return ids[q]; });
  rec.rx = link;
  rec.depth = 3;
  rec.ray = -1;
  rec.flags = fl;
  rec.valid = 1;
  rec.pad = 0;
  rec.len = ell[0] + ell[1] + ell[2];
  rec.amp_re = amp.re;
  rec.amp_im = amp.im;
  for (int q = 0; q < kMaxRefl; ++q) {
    rec.tri[q] = q < 3 ? ids[q] : -1;
    rec.pts[q][0] = rec.pts[q][1] = rec.pts[q][2] = 0.0f;
  }
  for (int q = 0; q < 3; ++q) {
    rec.pts[q][0] = (float)Y[q + 1].x;
    rec.pts[q][1] = (float)Y[q + 1].y;
    rec.pts[q][2] = (float)Y[q + 1].z;
  }
  a.prec[uu] = rec;
  unsigned pos = atomicAdd(&a.bucket_cnt[link], 1u);
  if (pos < (unsigned)a.bucket_cap) a.bucket[(size_t)link * a.bucket_cap + pos] = (int)uu;
  else atomicOr(&a.ctr->err, ERR_BUCKET_OVERFLOW);
  atomicAdd(&a.ctr->n_valid, 1u);
}

__device__ __noinline__ void diffract_multi(const PathArgs& a, unsigned long long code, double k, double lam,
                                            unsigned& ovf, TStack& st) {
  const bool three = (code >> kKindShift) == 3ull;
  const int m = three ? 3 : 2;
  const unsigned long long c = code & ((1ull << kKindShift) - 1ull);
  const unsigned long long nobs = (unsigned long long)a.nrx * (1 + a.nrpr);
  const long ei = (long)(c / nobs);
  const int rho = (int)(c - (unsigned long long)ei * nobs);
  const int4 sq = three ? a.dseq3[ei] : a.dseq2[ei];
  if (!three && sq.w <= -2) {  // a reflection between the two wedges
    if (rho < a.nrx) diffract_mid(a, sq, rho, k, lam, ovf, st);
    return;
  }
  const int w[3] = {sq.y, sq.z, sq.w};
  const bool first = sq.x >= a.dntx, last = rho >= a.nrx;  // a reflection before / after the chain
  if (first && last) return;
  const int tx = first ? (sq.x - a.dntx) / a.nrpr : sq.x, r = last ? (rho - a.nrx) / a.nrpr : rho;
  const int pl = first ? (sq.x - a.dntx) % a.nrpr : last ? (rho - a.nrx) % a.nrpr : -1;
  const int link = tx * a.nrx + r;
  const Wedge* E[3] = {&a.wedges[w[0]], &a.wedges[w[1]], three ? &a.wedges[w[2]] : &a.wedges[w[1]]};
  float4 rxv = a.rx[r], txv = a.txs[tx];
  const d3w T = D3(txv.x, txv.y, txv.z), R = D3(rxv.x, rxv.y, rxv.z);
  d3w X[5], Pp = D3(0, 0, 0), nj = D3(0, 0, 0);
  double ell[4], phip[3], phi[3];
  int j = -1;
  float4 mj = make_float4(0.f, 0.f, 0.f, 0.f);
  if (pl < 0) {
    if (!chain_geometry(E, m, T, R, X, ell, phip, phi)) return;
  } else {
    const RPlane Pg = a.rplanes[pl];
    d3w n = D3(Pg.n[0], Pg.n[1], Pg.n[2]);
    double cg = Pg.c;
    for (int pass = 0; pass < 2; ++pass) {
      d3w src = first ? T - n * (2.0 * (dotw(n, T) - cg)) : T;
      d3w obs = last ? R - n * (2.0 * (dotw(n, R) - cg)) : R;
      if (!chain_geometry(E, m, src, obs, X, ell, phip, phi)) return;
      if (!leg_plane(first ? X[0] : X[m], first ? X[1] : X[m + 1], n, cg, Pp)) return;
      if (pass == 0) {  // the member triangle holding the point: its own plane next
        d3w v0, v1, v2;
        int exw[6];
        for (int i = 0; i < m; ++i) {
          exw[2 * i] = E[i]->ta;
          exw[2 * i + 1] = E[i]->tb;
        }
        j = member_at(a, Pg, Pp, exw, 2 * m, v0, v1, v2, mj);
        if (j < 0) return;
        nj = unitw(crossw(v1 - v0, v2 - v0));
        n = nj;
        cg = dotw(nj, v0);
      } else {
        d3w v0, v1, v2;
        tri64(a, j, v0, v1, v2, mj);
        if (!inside_tri64(v0, v1, v2, Pp)) return;
      }
    }
  }
  // the real legs: Y the path's points, two excluded triangles at each
  d3w Y[6];
  int ex[6][2], ny = 0;
  Y[ny] = T; ex[ny][0] = ex[ny][1] = -1; ++ny;
  if (first) { Y[ny] = Pp; ex[ny][0] = ex[ny][1] = j; ++ny; }
  for (int i = 0; i < m; ++i) { Y[ny] = X[i + 1]; ex[ny][0] = E[i]->ta; ex[ny][1] = E[i]->tb; ++ny; }
  if (last) { Y[ny] = Pp; ex[ny][0] = ex[ny][1] = j; ++ny; }
  Y[ny] = R; ex[ny][0] = ex[ny][1] = -1; ++ny;
  for (int q = 0; q + 1 < ny; ++q) {
    d3w dv = Y[q + 1] - Y[q];
    RayPre rp = ray_pre(f3((float)Y[q].x, (float)Y[q].y, (float)Y[q].z), f3((float)dv.x, (float)dv.y, (float)dv.z));
    if (any_hit(a.bvh, rp, a.eps_occ, 1.0f - a.eps_occ, ex[q][0], ex[q][1], ovf, st, ex[q + 1][0], ex[q + 1][1]))
      return;
  }
  unsigned fl = 0;
  const d3w u = D3(a.pol.x, a.pol.y, a.pol.z);
  d3w ip = (X[1] - X[0]) * (1.0 / ell[0]);  // the real direction into Q_1
  double sn, cs;
  sincos(-k * ell[0], &sn, &cs);
  zd Ei = Z(cs / ell[0], sn / ell[0]);
  zv3 Ev;
  if (first) {
    d3w din = unitw(Pp - T);
    d3w e0 = polw(u, din, fl);
    zv3 E0 = {Z(e0.x), Z(e0.y), Z(e0.z)};
    zv3 Er = reflect_field_d(a, nj, mj, din, ip, E0);
    Ev = zv3{Er.x * Ei, Er.y * Ei, Er.z * Ei};
  } else {
    d3w e0 = polw(u, ip, fl);
    Ev = zv3{Ei * e0.x, Ei * e0.y, Ei * e0.z};
  }
  double rho1 = ell[0], rho2 = ell[0];
  d3w dir1 = D3(0, 0, 0), dir2 = D3(0, 0, 0), dd = ip;
  for (int i = 0; i < m; ++i) {
    const Wedge& W = *E[i];
    const double s = ell[i + 1], nn = W.n;
    const d3w e = D3(W.e[0], W.e[1], W.e[2]);
    dd = (X[i + 2] - X[i + 1]) * (1.0 / s);
    double beta0 = acos(fmax(-1.0, fmin(1.0, dotw(ip, e))));
    double sb = sin(beta0);
    d3w php = unitw(crossw(e, ip)) * -1.0, ph = unitw(crossw(e, dd));
    d3w bp = crossw(ip, php), bd = crossw(dd, ph);
    double rhoe;
    if (i == 0) rhoe = ell[0];
    else {
      double c1 = dotw(bp, dir1), c2 = dotw(bp, dir2);
      rhoe = 1.0 / (c1 * c1 / rho1 + c2 * c2 / rho2);
    }
    double L = s * (rhoe + s) * rho1 * rho2 * sb * sb / (rhoe * (rho1 + s) * (rho2 + s));
    const float4 ma =
        a.mats[__float_as_int(a.tris[3 * (size_t)DCEM_IDX(a.slot_of_id[DCEM_IDX(W.ta, a.bvh.ntris)], a.bvh.ntris) + 1].w)];
    const float4 mb =
        a.mats[__float_as_int(a.tris[3 * (size_t)DCEM_IDX(a.slot_of_id[DCEM_IDX(W.tb, a.bvh.ntris)], a.bvh.ntris) + 1].w)];
    zd r0s, r0h, rns, rnh;
    fresnel_d(ma, a.freq, fabs(sin(phip[i])), r0s, r0h);
    fresnel_d(mb, a.freq, fabs(sin(nn * M_PI - phi[i])), rns, rnh);
    const UtdParts up = utd_parts(nn, phi[i], phip[i], beta0, L, k, fl);
    zd Ds = utd_coeff(up, r0s, rns), Dh = utd_coeff(up, r0h, rnh);
    sincos(-k * s, &sn, &cs);
    zd A = Z(cs, sn) * sqrt(rhoe / (s * (rhoe + s)));
    zd cb = Ds * zvdot(Ev, bp) * A * -1.0, cp = Dh * zvdot(Ev, php) * A * -1.0;
    Ev = zv3{cb * bd.x + cp * ph.x, cb * bd.y + cp * ph.y, cb * bd.z + cp * ph.z};
    rho1 = s;
    dir1 = ph;
    rho2 = rhoe + s;
    dir2 = bd;
    ip = dd;
  }
  d3w dlast = dd;
  if (last) {  // reflected last, toward the real receiver
    d3w dout = unitw(R - Pp);
    Ev = reflect_field_d(a, nj, mj, dd, dout, Ev);
    dlast = dout;
  }
  d3w prx = polw(u, dlast * -1.0, fl);
  zd amp = zvdot(Ev, prx) * (lam / (4.0 * M_PI));
  double Ltot = 0.0;
  for (int q = 0; q <= m; ++q) Ltot += ell[q];
  unsigned uu = atomicAdd(&a.ctr->n_unique, 1u);
  if (uu >= a.ucap) {
    atomicOr(&a.ctr->err, ERR_UNIQUE_OVERFLOW);
    return;
  }
  const int depth = m + (pl >= 0 ? 1 : 0);
  int ids[4];
  for (int q = 0; q < depth; ++q) {
    if (first) ids[q] = q == 0 ? j : (w[q - 1] | kDiffBit);
    else if (last) ids[q] = q == m ? j : (w[q] | kDiffBit);
    else ids[q] = w[q] | kDiffBit;
  }
  PathRec rec;
  rec.key = seq_key(r, depth, [&](int q) { return ids[q]; });
  rec.rx = link;
  rec.depth = depth;
  rec.ray = -1;
  rec.flags = fl;
  rec.valid = 1;
  rec.pad = 0;
  rec.len = Ltot;
  rec.amp_re = amp.re;
  rec.amp_im = amp.im;
  for (int q = 0; q < kMaxRefl; ++q) {
    rec.tri[q] = q < depth ? ids[q] : -1;
    rec.pts[q][0] = rec.pts[q][1] = rec.pts[q][2] = 0.0f;
  }
  for (int q = 1; q + 1 < ny; ++q) {
    rec.pts[q - 1][0] = (float)Y[q].x;
    rec.pts[q - 1][1] = (float)Y[q].y;
    rec.pts[q - 1][2] = (float)Y[q].z;
  }
  a.prec[uu] = rec;
  unsigned pos = atomicAdd(&a.bucket_cnt[link], 1u);
  if (pos < (unsigned)a.bucket_cap) a.bucket[(size_t)link * a.bucket_cap + pos] = (int)uu;
  else atomicOr(&a.ctr->err, ERR_BUCKET_OVERFLOW);
  atomicAdd(&a.ctr->n_valid, 1u);
}

// ---------------------------------------------------------------------------
// two reflections around a first-order diffraction (Sec. III steps 3-5; the
// paper's evaluation allows two reflections and one diffraction per path)
// ---------------------------------------------------------------------------
// Candidates (kind, link, p1, p2, wedge), the reflector planes p1, p2 in path
// order: kind 0 both before the wedge (Tx -> P1 -> P2 -> Q -> Rx), 1 one on
// each side (Tx -> P1 -> Q -> P2 -> Rx), 2 both after it (Tx -> Q -> P1 -> P2
// -> Rx). By image theory the diffraction runs from the transmitter's image
// in the planes before the wedge (taken in path order) toward the receiver's
// image in the planes after it (the last one first); the reflection points
// follow by unfolding back from Q. A block (kind, link, p1, p2) goes to one
// warp, which queues the block's candidate wedges (k_diffract_refl2_pre).
// Survivors carry 10 in bits 63-62 and 1 in bit 61 over (block * nw + wedge).
constexpr unsigned long long kRefl2Tag = kReflTag | (1ull << 61);
constexpr unsigned long long kRefl2Mask = (1ull << 61) - 1ull;

// Can a leg from S to some point of `box` cross plane P1 inside P1's box?
// With every corner of the box across the plane from S, the legs' crossings
// lie within the box of the corner legs' crossings; "no" when every corner
// lies on S's side (no leg crosses the plane) or when the crossings' box,
// widened by m, misses P1's box.
__device__ __forceinline__ bool box_reachable(const RPlane& P1, float3 S, const float* box, float m) {
  const float3 n = f3(P1.nf[0], P1.nf[1], P1.nf[2]);
  const float c = P1.cf;
  const float ds = fdot3(n, S) - c;
  if (fabsf(ds) <= m) return true;
  float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
  int same = 0;
  for (int q = 0; q < 8; ++q) {
    const float3 X = f3((q & 1) ? box[3] + m : box[0] - m, (q & 2) ? box[4] + m : box[1] - m,
                        (q & 4) ? box[5] + m : box[2] - m);
    const float dx = fdot3(n, X) - c;
    if (fabsf(dx) <= m) return true;
    if ((dx > 0.0f) == (ds > 0.0f)) {
      ++same;
      continue;
    }
    const float t = ds / (ds - dx);
    const float x = S.x + t * (X.x - S.x), y = S.y + t * (X.y - S.y), z = S.z + t * (X.z - S.z);
    lo[0] = fminf(lo[0], x); lo[1] = fminf(lo[1], y); lo[2] = fminf(lo[2], z);
    hi[0] = fmaxf(hi[0], x); hi[1] = fmaxf(hi[1], y); hi[2] = fmaxf(hi[2], z);
  }
  if (same == 8) return false;
  if (same > 0) return true;
  for (int k = 0; k < 3; ++k)
    if (hi[k] < P1.box[k] - m || lo[k] > P1.box[3 + k] + m) return false;
  return true;
}

// The crossing X of the unfolded leg a0 -> a1 with plane P, within margins
// (delta + 2e-4 of the distances): 0 when it certainly lies off the leg or
// off P's box, 1 with X set, 2 when the leg runs nearly parallel to the
// plane (no conclusion).
__device__ __forceinline__ int refl_cross32(const RPlane& P, float3 a0, float3 a1, float delta, float3& X) {
  const float3 n = f3(P.nf[0], P.nf[1], P.nf[2]);
  const float3 dv = f3(a1.x - a0.x, a1.y - a0.y, a1.z - a0.z);
  const float den = fdot3(n, dv), len = sqrtf(fdot3(dv, dv));
  if (!(fabsf(den) > 1e-6f * len)) return 2;
  const float t = (P.cf - fdot3(n, a0)) / den;
  const float mt = (delta + 2e-4f * (len + sqrtf(fdot3(a0, a0)))) / len;
  if (t < -mt || t > 1.0f + mt) return 0;
  X = f3(a0.x + t * dv.x, a0.y + t * dv.y, a0.z + t * dv.z);
  const float mb = delta + 2e-4f * (len + sqrtf(fdot3(X, X)));
  if (X.x < P.box[0] - mb || X.y < P.box[1] - mb || X.z < P.box[2] - mb || X.x > P.box[3] + mb ||
      X.y > P.box[4] + mb || X.z > P.box[5] + mb)
    return 0;
  return 1;
}

// FP32 pre-test of one candidate: false only when the FP64 test rejects it
// too. S, O: the source and observer of the diffraction (images); S1: the
// transmitter's image in P1 (kind 0), O1: the receiver's image in P2 (kind 2).
// The Keller point's place on the edge and the crossings with the planes
// there come first, the angle rules (diffract_candidate) last.
__device__ __forceinline__ bool refl2_candidate(const WedgeF& W, const RPlane& P1, const RPlane& P2, int kind,
                                                float3 S, float3 S1, float3 O, float3 O1) {
  const float3 e = W.e, p0 = W.p0;
  const float3 dt = f3(S.x - p0.x, S.y - p0.y, S.z - p0.z), dr = f3(O.x - p0.x, O.y - p0.y, O.z - p0.z);
  const float zt = fdot3(dt, e), zr = fdot3(dr, e);
  const float3 pt = f3(dt.x - e.x * zt, dt.y - e.y * zt, dt.z - e.z * zt);
  const float3 pr = f3(dr.x - e.x * zr, dr.y - e.y * zr, dr.z - e.z * zr);
  const float rt = sqrtf(fdot3(pt, pt)), rr = sqrtf(fdot3(pr, pr));
  if (!(rt > 1e-3f && rr > 1e-3f)) return true;  // as diffract_candidate: no conclusion
  const float zq = zt + (zr - zt) * rt / (rt + rr);
  const float mz = 0.05f + 1e-5f * (sqrtf(fdot3(dt, dt)) + sqrtf(fdot3(dr, dr)));
  if (zq < -mz || zq > W.len + mz) return false;  // the Keller point off the edge (as diffract_candidate)
  const float3 Q = f3(p0.x + e.x * zq, p0.y + e.y * zq, p0.z + e.z * zq);
  const float d = 0.1f;
  float3 X;
  if (kind == 0) {
    const int r = refl_cross32(P2, S, Q, d, X);
    if (r == 0) return false;
    if (r == 1 && refl_cross32(P1, S1, X, d, X) == 0) return false;
  } else if (kind == 1) {
    if (refl_cross32(P1, S, Q, d, X) == 0) return false;
    if (refl_cross32(P2, Q, O, d, X) == 0) return false;
  } else {
    const int r = refl_cross32(P1, Q, O, d, X);
    if (r == 0) return false;
    if (r == 1 && refl_cross32(P2, X, O1, d, X) == 0) return false;
  }
  return diffract_candidate(W, make_float4(S.x, S.y, S.z, 0.0f), make_float4(O.x, O.y, O.z, 0.0f));
}

static_assert(kWedgeCluster == 32, "a wedge cluster is one warp's lanes and one mask word");

// Wedge masks of the two-reflection pre-test, per frame. For every end point
// X (the transmitters, then the receivers) and plane p, bit i of word
// (X, p, c) is set when the i-th wedge of cluster c could take part in a
// path with a reflection on p next to X: X's image in p outside the wedge,
// and some leg from the image to the edge crossing p inside its box
// (plane_reachable). Plane index nrp stands for no reflection: X itself
// outside the wedge. A path with one reflection on each side of the wedge
// needs its wedge in the transmitter's mask for p1 and the receiver's for
// p2; one with both reflections on one side, in the other end point's mask
// for no reflection.
__global__ void __launch_bounds__(256) k_refl2_masks(PathArgs a, int ntx) {
  const int np1 = a.nrp + 1;
  const long nitem = (long)(ntx + a.nrx) * np1 * a.nwc;
  const int lane = threadIdx.x & 31;
  const long nwarp = (long)gridDim.x * (blockDim.x >> 5);
  for (long it = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < nitem; it += nwarp) {
    const int c = (int)(it % a.nwc);
    const long r = it / a.nwc;
    const int p = (int)(r % np1), x = (int)(r / np1);
    const float4 xv = x < ntx ? a.txs[x] : a.rx[x - ntx];
    float3 X = f3(xv.x, xv.y, xv.z);
    const int i = c * kWedgeCluster + lane;
    bool bit = false;
    if (i < a.nw) {
      const WedgeF W = a.wf[a.wperm[i]];
      if (p == a.nrp) {
        bit = !surely_inside(W, X);
      } else {
        const RPlane& Pl = a.rplanes[p];
        X = mirror32(X, f3(Pl.nf[0], Pl.nf[1], Pl.nf[2]), Pl.cf);
        float3 A, B;
        edge_ends(W, A, B);
        const float mg = 0.1f + 1e-4f * (fabsf(X.x) + fabsf(X.y) + fabsf(X.z) + W.len);
        bit = plane_reachable(Pl, X, A, B, mg) && !surely_inside(W, X);
      }
    }
    const unsigned mk = __ballot_sync(0xffffffffu, bit);
    if (lane == 0) a.rmask[it] = mk;
  }
}

// The images of block (kind, link, p1, p2): S, O the diffraction's source
// and observer, S1 the transmitter's image in P1 (kind 0), O1 the
// receiver's image in P2 (kind 2); m the block's margin.
__device__ __forceinline__ void refl2_images(const PathArgs& a, int kind, int link, const RPlane& P1,
                                             const RPlane& P2, float3& S, float3& S1, float3& O, float3& O1,
                                             float& m) {
  const float4 tv = a.txs[link / a.nrx], rv = a.rx[link % a.nrx];
  const float3 T = f3(tv.x, tv.y, tv.z), R = f3(rv.x, rv.y, rv.z);
  const float3 n1 = f3(P1.nf[0], P1.nf[1], P1.nf[2]);
  const float3 n2 = f3(P2.nf[0], P2.nf[1], P2.nf[2]);
  m = 0.1f + 1e-4f * (fabsf(T.x) + fabsf(T.y) + fabsf(T.z) + fabsf(R.x) + fabsf(R.y) + fabsf(R.z));
  S = S1 = T;
  O = O1 = R;
  if (kind == 0) {
    S1 = mirror32(T, n1, P1.cf);
    S = mirror32(S1, n2, P2.cf);
  } else if (kind == 1) {
    S = S1 = mirror32(T, n1, P1.cf);
    O = O1 = mirror32(R, n2, P2.cf);
  } else {
    O1 = mirror32(R, n2, P2.cf);
    O = mirror32(O1, n1, P1.cf);
  }
}

// Block b's parts: kind, link and the two planes (32-bit division when b fits).
__device__ __forceinline__ void refl2_block(const PathArgs& a, int nlinks, long b, int& kind, int& link, int& p1,
                                            int& p2) {
  if (b < 0x7fffffffL) {
    unsigned r = (unsigned)b;
    p2 = (int)(r % (unsigned)a.nrp);
    r /= (unsigned)a.nrp;
    p1 = (int)(r % (unsigned)a.nrp);
    r /= (unsigned)a.nrp;
    link = (int)(r % (unsigned)nlinks);
    kind = (int)(r / (unsigned)nlinks);
  } else {
    long r = b;
    p2 = (int)(r % a.nrp);
    r /= a.nrp;
    p1 = (int)(r % a.nrp);
    r /= a.nrp;
    link = (int)(r % nlinks);
    kind = (int)(r / nlinks);
  }
}

// A block's record in a warp's ring: its images, planes, kind and index.
struct Refl2Blk {
  float3 S, S1, O, O1;
  int p1, p2, kind;
  long b;
};
constexpr int kRefl2Queue = 64;  // queue entries and block records per warp

// One warp per block (kind, link, p1, p2). Its wedges: with one reflection
// on each side, those in both end points' masks (k_refl2_masks); with both
// on one side, the wedges of the clusters that the unfolded legs can reach
// through the planes' boxes (lane c tests cluster c), less those the other,
// real end point lies inside. The candidates wait in a per-warp FIFO queue
// in shared memory and go through refl2_candidate 32 at a time, so that the
// test runs on full warps; each entry names its wedge and its block's record
// in a ring of 64. At most 63 entries wait, each block with an entry adds
// one, so a record is overwritten only after its entries left the queue.
__global__ void __launch_bounds__(256, 3) k_diffract_refl2_pre(PathArgs a, int nlinks) {
  __shared__ Refl2Blk rec[8][kRefl2Queue];
  __shared__ int qw[8][kRefl2Queue];
  __shared__ unsigned char qs[8][kRefl2Queue];
  const long nblk = 3L * nlinks * a.nrp * a.nrp;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long nwarp = (long)gridDim.x * (blockDim.x >> 5);
  const int np1 = a.nrp + 1, ntx = nlinks / a.nrx;
  // warp-uniform: queue head and tail (entries head .. tail - 1), next record
  int head = 0, tail = 0, nrec = 0;
  // the oldest min(tail - head, 32) entries through the test
  auto drain = [&]() {
    const int nn = min(tail - head, 32);
    bool keep = false;
    int w = 0;
    long b = 0;
    if (lane < nn) {
      const int e = (head + lane) & (kRefl2Queue - 1);
      w = qw[wid][e];
      const Refl2Blk& R = rec[wid][qs[wid][e]];
      b = R.b;
      keep = refl2_candidate(a.wf[w], a.rplanes[R.p1], a.rplanes[R.p2], R.kind, R.S, R.S1, R.O, R.O1);
    }
    head += nn;
    const unsigned mk = __ballot_sync(0xffffffffu, keep);
    if (!mk) return;
    unsigned at = 0;
    if (lane == 0) at = atomicAdd(&a.ctr->n_dsurv, (unsigned)__popc(mk));
    at = __shfl_sync(0xffffffffu, at, 0) + __popc(mk & ((1u << lane) - 1u));
    if (keep) {
      if (at < a.dsurv_cap) a.dsurv[at] = kRefl2Tag | ((unsigned long long)b * a.nw + w);
      else atomicOr(&a.ctr->err, ERR_DIFF_OVERFLOW);
    }
  };
  for (long b = (long)blockIdx.x * (blockDim.x >> 5) + wid; b < nblk; b += nwarp) {
    int kind, link, p1, p2;
    refl2_block(a, nlinks, b, kind, link, p1, p2);
    if (kind != 1 && p1 == p2) continue;  // two reflections in a row on one plane
    const RPlane &P1 = a.rplanes[p1], &P2 = a.rplanes[p2];
    float3 S, S1, O, O1;
    float m;
    refl2_images(a, kind, link, P1, P2, S, S1, O, O1, m);
    if (kind == 0 && !box_reachable(P1, S1, P2.box, m)) continue;
    if (kind == 2 && !box_reachable(P2, O1, P1.box, m)) continue;
    const int t = link / a.nrx, rr = link % a.nrx;
    const unsigned* mt = a.rmask + ((long)t * np1 + (kind == 1 ? p1 : a.nrp)) * a.nwc;
    const unsigned* mr = a.rmask + ((long)(ntx + rr) * np1 + (kind == 1 ? p2 : a.nrp)) * a.nwc;
    int slot = -1;  // this block's record (written with its first entry)
    for (int c0 = 0; c0 < a.nwc; c0 += 32) {
      const int c = c0 + lane;
      unsigned word = 0;
      if (c < a.nwc) {
        if (kind == 1) {
          word = mt[c] & mr[c];
        } else {
          word = kind == 0 ? mr[c] : mt[c];
          const float* cb = a.wcbox + 6 * (size_t)c;
          if (word && !(kind == 0 ? box_reachable(P2, S, cb, m) : box_reachable(P1, O, cb, m))) word = 0;
        }
      }
      for (unsigned cm = __ballot_sync(0xffffffffu, word != 0); cm; cm &= cm - 1u) {
        const int src = __ffs(cm) - 1;
        const unsigned wd = __shfl_sync(0xffffffffu, word, src);
        if (slot < 0) {
          slot = nrec++ & (kRefl2Queue - 1);
          if (lane == 0) {
            Refl2Blk& R = rec[wid][slot];
            R.S = S; R.S1 = S1; R.O = O; R.O1 = O1;
            R.p1 = p1; R.p2 = p2; R.kind = kind; R.b = b;
          }
        }
        const bool bit = (wd >> lane) & 1u;
        const unsigned bm = __ballot_sync(0xffffffffu, bit);
        if (bit) {
          const int e = (tail + __popc(bm & ((1u << lane) - 1u))) & (kRefl2Queue - 1);
          qw[wid][e] = a.wperm[(c0 + src) * kWedgeCluster + lane];
          qs[wid][e] = (unsigned char)slot;
        }
        tail += __popc(bm);
        __syncwarp();
        if (tail - head >= 32) drain();
        __syncwarp();
      }
    }
  }
  while (tail > head) drain();
}

__device__ __forceinline__ d3w mirror_d(d3w x, d3w n, double c) { return x - n * (2.0 * (dotw(n, x) - c)); }

// One survivor of k_diffract_refl2_pre: the images, the Keller point and the
// wedge rules (chain_geometry with one wedge) and the reflection points on
// the group planes; the member triangles holding those points; everything
// again on the members' own planes (the oracle's mirrors are the static
// triangles); the four real legs (FP32 any-hit; the triangle excluded at a
// reflection point, the wedge's faces at Q); then the field: the
// transmitter's wave along its first real leg, Fresnel at each reflection
// before the wedge in the real directions, the UTD coefficient over the
// unfolded distances, Fresnel at each reflection after it. Record: depth 3.
__device__ __noinline__ void diffract_refl2(const PathArgs& a, unsigned long long code, double k, double lam,
                                            unsigned& ovf, TStack& st) {
  const int w = (int)(code % (unsigned long long)a.nw);
  unsigned long long b = code / (unsigned long long)a.nw;
  const int p2 = (int)(b % (unsigned long long)a.nrp);
  b /= (unsigned long long)a.nrp;
  const int p1 = (int)(b % (unsigned long long)a.nrp);
  b /= (unsigned long long)a.nrp;
  const unsigned long long nlinks = (unsigned long long)a.dntx * a.nrx;
  const int link = (int)(b % nlinks), kind = (int)(b / nlinks);
  const int nb = kind == 0 ? 2 : kind == 1 ? 1 : 0, na = 2 - nb;
  const Wedge& W = a.wedges[w];
  const Wedge* E[1] = {&W};
  const float4 rxv = a.rx[link % a.nrx], txv = a.txs[link / a.nrx];
  const d3w T = D3(txv.x, txv.y, txv.z), R = D3(rxv.x, rxv.y, rxv.z);
  // the planes of the two reflections in path order: the groups', then the members'
  const int pg[2] = {p1, p2};
  d3w pn[2];
  double pc[2];
  int pj[2] = {-1, -1};
  float4 pm[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
  for (int i = 0; i < 2; ++i) {
    const RPlane& G = a.rplanes[pg[i]];
    pn[i] = D3(G.n[0], G.n[1], G.n[2]);
    pc[i] = G.c;
  }
  d3w X[3], Y[2];
  double ell[2], phip[1], phi[1];
  for (int pass = 0; pass < 2; ++pass) {
    d3w Sim[3], Oim[3];
    Sim[0] = T;
    for (int i = 0; i < nb; ++i) Sim[i + 1] = mirror_d(Sim[i], pn[i], pc[i]);
    Oim[na] = R;
    for (int i = na - 1; i >= 0; --i) Oim[i] = mirror_d(Oim[i + 1], pn[nb + i], pc[nb + i]);
    if (!chain_geometry(E, 1, Sim[nb], Oim[0], X, ell, phip, phi)) return;
    d3w bp = X[1];
    for (int i = nb - 1; i >= 0; --i) {
      if (!leg_plane(Sim[i + 1], bp, pn[i], pc[i], Y[i])) return;
      bp = Y[i];
    }
    d3w ap = X[1];
    for (int i = 0; i < na; ++i) {
      if (!leg_plane(ap, Oim[i], pn[nb + i], pc[nb + i], Y[nb + i])) return;
      ap = Y[nb + i];
    }
    for (int i = 0; i < 2; ++i) {
      d3w v0, v1, v2;
      float4 mj;
      if (pass == 0) {  // the member triangle holding the point: its own plane next
        const RPlane& G = a.rplanes[pg[i]];
        const int exw[2] = {W.ta, W.tb};
        pj[i] = member_at(a, G, Y[i], exw, 2, v0, v1, v2, mj);
        if (pj[i] < 0) return;
        pm[i] = mj;
        pn[i] = unitw(crossw(v1 - v0, v2 - v0));
        pc[i] = dotw(pn[i], v0);
      } else {
        tri64(a, pj[i], v0, v1, v2, mj);
        if (!inside_tri64(v0, v1, v2, Y[i])) return;
      }
    }
  }
  // the real legs: P the path's points, two excluded triangles at each
  d3w P[5];
  int ex[5][2], ny = 0;
  P[ny] = T; ex[ny][0] = ex[ny][1] = -1; ++ny;
  for (int i = 0; i < nb; ++i) { P[ny] = Y[i]; ex[ny][0] = ex[ny][1] = pj[i]; ++ny; }
  P[ny] = X[1]; ex[ny][0] = W.ta; ex[ny][1] = W.tb; ++ny;
  for (int i = 0; i < na; ++i) { P[ny] = Y[nb + i]; ex[ny][0] = ex[ny][1] = pj[nb + i]; ++ny; }
  P[ny] = R; ex[ny][0] = ex[ny][1] = -1; ++ny;
  for (int q = 0; q + 1 < ny; ++q) {
    const d3w dv = P[q + 1] - P[q];
    RayPre rp = ray_pre(f3((float)P[q].x, (float)P[q].y, (float)P[q].z), f3((float)dv.x, (float)dv.y, (float)dv.z));
    if (any_hit(a.bvh, rp, a.eps_occ, 1.0f - a.eps_occ, ex[q][0], ex[q][1], ovf, st, ex[q + 1][0], ex[q + 1][1]))
      return;
  }
  unsigned fl = 0;
  const d3w u = D3(a.pol.x, a.pol.y, a.pol.z);
  const d3w ip = (X[1] - X[0]) * (1.0 / ell[0]);  // the real direction into Q
  double sn, cs;
  sincos(-k * ell[0], &sn, &cs);
  const zd Ei = Z(cs / ell[0], sn / ell[0]);
  d3w din = nb ? unitw(P[1] - T) : ip;
  const d3w e0 = polw(u, din, fl);
  zv3 Er = {Z(e0.x), Z(e0.y), Z(e0.z)};
  for (int i = 0; i < nb; ++i) {
    const d3w dout = i == nb - 1 ? ip : unitw(P[i + 2] - P[i + 1]);
    Er = reflect_field_d(a, pn[i], pm[i], din, dout, Er);
    din = dout;
  }
  zv3 Ev = {Er.x * Ei, Er.y * Ei, Er.z * Ei};
  {  // the wedge: UTD over the unfolded distances, a spherical wave arriving
    const double s = ell[1], nn = W.n, rhoe = ell[0], rho1 = ell[0], rho2 = ell[0];
    const d3w e = D3(W.e[0], W.e[1], W.e[2]);
    const d3w dd = (X[2] - X[1]) * (1.0 / s);
    const double beta0 = acos(fmax(-1.0, fmin(1.0, dotw(ip, e))));
    const double sb = sin(beta0);
    const d3w php = unitw(crossw(e, ip)) * -1.0, ph = unitw(crossw(e, dd));
    const d3w bpv = crossw(ip, php), bd = crossw(dd, ph);
    const double L = s * (rhoe + s) * rho1 * rho2 * sb * sb / (rhoe * (rho1 + s) * (rho2 + s));
    const float4 ma =
        a.mats[__float_as_int(a.tris[3 * (size_t)DCEM_IDX(a.slot_of_id[DCEM_IDX(W.ta, a.bvh.ntris)], a.bvh.ntris) + 1].w)];
    const float4 mb =
        a.mats[__float_as_int(a.tris[3 * (size_t)DCEM_IDX(a.slot_of_id[DCEM_IDX(W.tb, a.bvh.ntris)], a.bvh.ntris) + 1].w)];
    zd r0s, r0h, rns, rnh;
    fresnel_d(ma, a.freq, fabs(sin(phip[0])), r0s, r0h);
    fresnel_d(mb, a.freq, fabs(sin(nn * M_PI - phi[0])), rns, rnh);
    const UtdParts up = utd_parts(nn, phi[0], phip[0], beta0, L, k, fl);
    const zd Ds = utd_coeff(up, r0s, rns), Dh = utd_coeff(up, r0h, rnh);
    sincos(-k * s, &sn, &cs);
    const zd A = Z(cs, sn) * sqrt(rhoe / (s * (rhoe + s)));
    const zd cb = Ds * zvdot(Ev, bpv) * A * -1.0, cp = Dh * zvdot(Ev, php) * A * -1.0;
    Ev = zv3{cb * bd.x + cp * ph.x, cb * bd.y + cp * ph.y, cb * bd.z + cp * ph.z};
    din = dd;
  }
  for (int i = 0; i < na; ++i) {  // reflected after the wedge, toward the real receiver
    const int at = ny - 1 - na + i;
    const d3w dout = unitw(P[at + 1] - P[at]);
    Ev = reflect_field_d(a, pn[nb + i], pm[nb + i], din, dout, Ev);
    din = dout;
  }
  const d3w prx = polw(u, din * -1.0, fl);
  const zd amp = zvdot(Ev, prx) * (lam / (4.0 * M_PI));
  unsigned uu = atomicAdd(&a.ctr->n_unique, 1u);
  if (uu >= a.ucap) {
    atomicOr(&a.ctr->err, ERR_UNIQUE_OVERFLOW);
    return;
  }
  int ids[3];
  for (int i = 0; i < nb; ++i) ids[i] = pj[i];
  ids[nb] = w | kDiffBit;
  for (int i = 0; i < na; ++i) ids[nb + 1 + i] = pj[nb + i];
  PathRec rec;
  rec.key = seq_key(link % a.nrx, 3, [&](int q) { return ids[q]; });
  rec.rx = link;
  rec.depth = 3;
  rec.ray = -1;
  rec.flags = fl;
  rec.valid = 1;
  rec.pad = 0;
  rec.len = ell[0] + ell[1];
  rec.amp_re = amp.re;
  rec.amp_im = amp.im;
  for (int q = 0; q < kMaxRefl; ++q) {
    rec.tri[q] = q < 3 ? ids[q] : -1;
    rec.pts[q][0] = rec.pts[q][1] = rec.pts[q][2] = 0.0f;
  }
  for (int q = 1; q + 1 < ny; ++q) {
    rec.pts[q - 1][0] = (float)P[q].x;
    rec.pts[q - 1][1] = (float)P[q].y;
    rec.pts[q - 1][2] = (float)P[q].z;
  }
  a.prec[uu] = rec;
  unsigned pos = atomicAdd(&a.bucket_cnt[link], 1u);
  if (pos < (unsigned)a.bucket_cap) a.bucket[(size_t)link * a.bucket_cap + pos] = (int)uu;
  else atomicOr(&a.ctr->err, ERR_BUCKET_OVERFLOW);
  atomicAdd(&a.ctr->n_valid, 1u);
}

// Pass 1 over every (link, wedge) pair: the FP32 pre-test rejects most of
// them; the survivors' indices go to a list (one atomic per warp).
__global__ void __launch_bounds__(256) k_diffract_pre(PathArgs a, int nlinks) {
  const long total = (long)nlinks * a.nw;
  const int lane = threadIdx.x & 31;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long base = (long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total; base += stride) {
    long idx = base + lane;
    bool keep = false;
    if (idx < total) {
      int link = (int)(idx / a.nw), w = (int)(idx - (long)link * a.nw);
      keep = diffract_candidate(a.wf[w], a.txs[link / a.nrx], a.rx[link % a.nrx]);
    }
    unsigned m = __ballot_sync(0xffffffffu, keep);
    if (!m) continue;
    unsigned at = 0;
    if (lane == 0) at = atomicAdd(&a.ctr->n_dsurv, (unsigned)__popc(m));
    at = __shfl_sync(0xffffffffu, at, 0) + __popc(m & ((1u << lane) - 1u));
    if (keep) {
      if (at < a.dsurv_cap) a.dsurv[at] = (unsigned long long)idx;
      else atomicOr(&a.ctr->err, ERR_DIFF_OVERFLOW);
    }
  }
}

// Pass 2 over the survivors: the exact FP64 test, the occlusion legs and the
// UTD field. The SM's FP64 pipe is narrow and a warp instruction costs it the
// same whatever the number of active lanes, so survivor i goes to block
// i mod grid, slot i / grid: every SM gets an equal share, packed into its
// first warp while there are few survivors and into more warps as they grow
// (orders 2 and 3 can leave many), instead of a few SMs taking whole batches.
constexpr int kDiffThreads = 256;
__global__ void __launch_bounds__(kDiffThreads) k_diffract(PathArgs a) {
  extern __shared__ int sstk[];
  TStack st;
  bind_stack(st, sstk, kStackTrace);
  const unsigned n = min(a.ctr->n_dsurv, a.dsurv_cap);
  const double k = 2.0 * M_PI * a.freq / 299792458.0, lam = 299792458.0 / a.freq;
  unsigned ovf = 0;
  for (unsigned i = blockIdx.x + gridDim.x * threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned long long c = a.dsurv[i];
    const unsigned kind = (unsigned)(c >> kKindShift);
    if (kind == 2u && ((c >> 61) & 1ull)) diffract_refl2(a, c & kRefl2Mask, k, lam, ovf, st);
    else if (kind == 2u) diffract_refl_pair(a, c & ~kReflTag, k, lam, ovf, st);
    else if (kind != 0u) diffract_multi(a, c, k, lam, ovf, st);
    else diffract_pair(a, (long)c, k, lam, ovf, st);
  }
  if (ovf) {
    atomicAdd(&a.ctr->stack_overflow, 1u);
    atomicOr(&a.ctr->err, ERR_STACK);
  }
}

// ---------------------------------------------------------------------------
// per link: sort paths by key, sum in that order, write them out
// ---------------------------------------------------------------------------
constexpr int kReduceThreads = 256;

// Exclusive scan of the links' valid-path counts (one CTA: each thread sums
// a contiguous run of links, the run totals are scanned in shared memory,
// then each thread writes its run's offsets).
__global__ void __launch_bounds__(1024) k_link_scan(const unsigned* __restrict__ cnt, int n, unsigned cap,
                                                    unsigned* __restrict__ off) {
  __shared__ unsigned part[1024];
  int tid = threadIdx.x;
  int per = (n + 1023) / 1024;
  int lo = min(n, tid * per), hi = min(n, lo + per);
  unsigned sum = 0;
  for (int i = lo; i < hi; ++i) sum += min(cnt[i], cap);
  part[tid] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    unsigned v = tid >= o ? part[tid - o] : 0u;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  unsigned base = tid ? part[tid - 1] : 0u;
  for (int i = lo; i < hi; ++i) {
    off[i] = base;
    base += min(cnt[i], cap);
  }
}

__global__ void __launch_bounds__(kReduceThreads) k_reduce(PathArgs a) {
  extern __shared__ unsigned long long skey[];   // bucket_cap keys, then bucket_cap ints
  int* sidx = reinterpret_cast<int*>(skey + a.bucket_cap);
  __shared__ double red[4][kReduceThreads];
  __shared__ unsigned soff;
  int r = blockIdx.x, tid = threadIdx.x;
  int cnt = (int)min(a.bucket_cnt[r], (unsigned)a.bucket_cap);
  // output offset: valid paths of all lower links (scanned beforehand when
  // there are many links)
  if (tid == 0) soff = a.link_off ? a.link_off[r] : 0u;
  __syncthreads();
  if (!a.link_off) {
    unsigned part = 0;
    for (int q = tid; q < r; q += kReduceThreads) part += min(a.bucket_cnt[q], (unsigned)a.bucket_cap);
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    if ((tid & 31) == 0) atomicAdd(&soff, part);
  }
  int np2 = 1;
  while (np2 < cnt) np2 <<= 1;
  for (int i = tid; i < np2; i += kReduceThreads) {
    if (i < cnt) {
      int u = DCEM_IDX(a.bucket[(size_t)r * a.bucket_cap + i], a.ucap);
      skey[i] = a.prec[u].key;
      sidx[i] = u;
    } else {
      skey[i] = ~0ull;
      sidx[i] = -1;
    }
  }
  __syncthreads();
  for (int k = 2; k <= np2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < np2; i += kReduceThreads) {
        int ixj = i ^ j;
        if (ixj > i) {
          unsigned long long x = skey[i], y = skey[ixj];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            skey[i] = y; skey[ixj] = x;
            int t = sidx[i]; sidx[i] = sidx[ixj]; sidx[ixj] = t;
          }
        }
      }
      __syncthreads();
    }
  }
  // fixed-order sums: thread t takes sorted positions t, t+256, ... in order,
  // then a fixed binary tree over the 256 partial sums
  double sre = 0.0, sim = 0.0, sinc = 0.0;
  unsigned off = soff;
  for (int i = tid; i < cnt; i += kReduceThreads) {
    const PathRec& p = a.prec[sidx[i]];
    sre += p.amp_re;
    sim += p.amp_im;
    sinc += p.amp_re * p.amp_re + p.amp_im * p.amp_im;
    unsigned o = off + (unsigned)i;
    if (o < a.pout_cap) {
      dcem_path q;
      q.rx = p.rx % a.nrx;
      q.tx = p.rx / a.nrx;
      q.reserved = 0;
      q.depth = p.depth;
      for (int j = 0; j < kMaxRefl; ++j) {
        q.tri[j] = p.tri[j];
        q.pts[j][0] = p.pts[j][0];
        q.pts[j][1] = p.pts[j][1];
        q.pts[j][2] = p.pts[j][2];
      }
      q.flags = p.flags;
      q.ray = p.ray >= 0 ? a.ray_perm[p.ray] : -1;
      q.key = p.key;
      q.len_m = p.len;
      q.delay_s = p.len / 299792458.0;
      q.amp_re = p.amp_re;
      q.amp_im = p.amp_im;
      a.pout[o] = q;
    }
  }
  red[0][tid] = sre;
  red[1][tid] = sim;
  red[2][tid] = sinc;
  __syncthreads();
  for (int s = kReduceThreads / 2; s > 0; s >>= 1) {
    if (tid < s)
      for (int q = 0; q < 3; ++q) red[q][tid] += red[q][tid + s];
    __syncthreads();
  }
  if (tid == 0) {
    double fr = red[0][0], fi = red[1][0], pinc = red[2][0];
    if (a.out_field) {
      a.out_field[2 * (size_t)r] = fr;
      a.out_field[2 * (size_t)r + 1] = fi;
    }
    if (a.out_pc) a.out_pc[r] = 10.0 * log10(a.tx_power * (fr * fr + fi * fi)) + 30.0;
    if (a.out_pi) a.out_pi[r] = 10.0 * log10(a.tx_power * pinc) + 30.0;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_dedupe(const PathArgs& a, int grid, cudaStream_t st) {
  k_dedupe_insert<<<grid, 256, 0, st>>>(a);
  k_dedupe_unique<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_diffract(const PathArgs& a, int nlinks, int sms, cudaStream_t st) {
  if (!a.wedges || a.nw <= 0) return cudaSuccess;
  k_wedge_geom<<<(a.nw + 255) / 256, 256, 0, st>>>(a.tris, a.slot_of_id, a.wtopo, a.nw, a.wedges, a.wf);
  if (a.drefl2 && a.rplanes && a.nrp > 0)
    k_wedge_boxes<<<(a.nwc * 32 + 255) / 256, 256, 0, st>>>(a.wf, a.wperm, a.nw, a.nwc, a.wcbox);
  if (nlinks > 0) {
    long total = (long)nlinks * a.nw;
    long g = std::min<long>((total + 255) / 256, 8L * sms);
    k_diffract_pre<<<(int)std::max<long>(g, 1), 256, 0, st>>>(a, nlinks);
    if (a.rplanes && a.nrp > 0) {
      long tr = (long)nlinks * a.nw * a.nrp * 2;
      long gr = std::min<long>((tr + 255) / 256, 8L * sms);
      k_diffract_refl_pre<<<(int)std::max<long>(gr, 1), 256, 0, st>>>(a, nlinks);
      if (a.drefl2) {
        const int ntx = nlinks / a.nrx;
        long nm = (long)(ntx + a.nrx) * (a.nrp + 1) * a.nwc;
        k_refl2_masks<<<(int)std::max<long>(std::min<long>((nm + 7) / 8, 8L * sms), 1), 256, 0, st>>>(a, ntx);
        long nblk = 3L * nlinks * a.nrp * a.nrp;
        long g2 = std::min<long>((nblk + 7) / 8, 8L * sms);
        k_diffract_refl2_pre<<<(int)std::max<long>(g2, 1), 256, 0, st>>>(a, nlinks);
      }
    }
    PathArgs b = a;  // chains: transmitters, and the reflector planes applied to them
    b.dntx = nlinks / a.nrx;
    b.nrpr = a.rplanes && a.diff_order >= 2 ? a.nrp : 0;
    if (a.diff_order >= 2 && a.nw > 1) {
      int nsrc = b.dntx * (1 + b.nrpr);
      long tp = (long)nsrc * a.nw * a.nw;
      cudaMemsetAsync(a.drel, 0, sizeof(unsigned) * (((size_t)a.nw * a.nw + 31) / 32), st);
      k_diff_rel<<<(int)std::max<long>(std::min<long>(((long)a.nw * a.nw + 255) / 256, 8L * sms), 1), 256, 0, st>>>(b);
      k_diff_pairs<<<(int)std::max<long>(std::min<long>((tp + 255) / 256, 8L * sms), 1), 256, 0, st>>>(b, nsrc);
      if (a.dmid && a.rplanes && a.nrp > 0) {
        long nblk = (long)b.dntx * a.nw * a.nrp;
        k_diff_mid_pairs<<<(int)std::max<long>(std::min<long>((nblk + 7) / 8, 8L * sms), 1), 256, 0, st>>>(b);
      }
      if (a.diff_order >= 3) k_diff_triples<<<8 * sms, 256, 0, st>>>(b);
      k_diff_multi_pre<<<8 * sms, 256, 256 * kStackTrace * sizeof(int), st>>>(b);
    }
    k_diffract<<<sms, kDiffThreads, kDiffThreads * kStackTrace * sizeof(int), st>>>(b);
  }
  return cudaGetLastError();
}

cudaError_t launch_sticky_probe(const PathArgs& a, int grid, cudaStream_t st) {
  k_sticky_probe<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_validate(const PathArgs& a, int grid, cudaStream_t st) {
  const size_t gsm = 64 * kStackSmall * sizeof(int);
  if (a.prec_df) k_val_geom<df><<<grid, 64, gsm, st>>>(a);
  else k_val_geom<double><<<grid, 64, gsm, st>>>(a);
  k_val_occ<<<grid, 64, 64 * kStackTrace * sizeof(int), st>>>(a);
  k_val_field<<<grid, kFieldThreads, 0, st>>>(a);
  return cudaGetLastError();
}

// The next frame's table: link key -> record index of each distinct key.
__global__ void k_vcache_build(PathArgs a) {
  unsigned nu = min(a.ctr->n_unique, a.ucap);
  const unsigned mask = a.vc_cap - 1u;
  for (unsigned u = blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += gridDim.x * blockDim.x) {
    unsigned long long key = a.ckey[u];
    if (!key) continue;
    unsigned slot = (unsigned)(key & mask);
    for (unsigned p = 0; p < a.vc_cap; ++p) {
      unsigned long long prev = atomicCAS(&a.vc_next_key[slot], 0ull, key);
      if (prev == 0ull || prev == key) {
        a.vc_next_u[slot] = u;
        break;
      }
      slot = (slot + 1u) & mask;
    }
  }
}

cudaError_t launch_vcache_build(const PathArgs& a, int grid, cudaStream_t st) {
  k_vcache_build<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const PathArgs& a, int nlinks, cudaStream_t st) {
  if (nlinks <= 0) return cudaSuccess;
  if (a.link_off) k_link_scan<<<1, 1024, 0, st>>>(a.bucket_cnt, nlinks, (unsigned)a.bucket_cap, a.link_off);
  size_t smem = (size_t)a.bucket_cap * (sizeof(unsigned long long) + sizeof(int));
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    attr = true;
  }
  k_reduce<<<nlinks, kReduceThreads, smem, st>>>(a);
  return cudaGetLastError();
}

DCEM_CHECKS_TAKER(checks_take_paths)

}  // namespace dcem
