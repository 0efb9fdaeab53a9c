// dcem_internal.cuh -- device data layout and inline device functions of the
// GB300 tracer. Compiled with -fmad=false: every fused multiply-add below is
// written explicitly, so a device function evaluates to the same bits in
// every kernel that inlines it (this is what makes a coherent-reuse frame
// equal to a full retrace bit for bit).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dcem.h"

namespace dcem {

constexpr int kMaxRefl = DCEM_MAX_REFL;
constexpr int kStackTrace = 24;         // shared-memory stack entries per thread (scene traversal)
constexpr int kStackSmall = 16;         // ... (per-frame receiver / moved-box trees)
constexpr int kEmpty = (int)0x80000000; // empty tree / no node
constexpr int kSmallBuild = 16384;      // largest tree built by the one-CTA builder
constexpr int kMaxRaySets = 4096;       // transmitters (ray sets) per scene
constexpr int kMaxLinks = 1 << 24;      // transmitter-receiver pairs per frame
constexpr int kMaxBatch = 1024;         // scenes per batch
constexpr int kTransBit = 0x40000000;   // interaction id flag: transmission (DCEM_TRI_TRANSMIT)
constexpr int kDiffBit = 0x20000000;    // interaction id flag: diffraction at wedge id (DCEM_TRI_DIFFRACT)

// A wedge of the static geometry (edge shared by two non-coplanar
// triangles), for first-order diffraction: edge start p0 and unit direction
// e, length, face 0's direction t0 and the exterior's angular direction y0
// in the plane normal to e, n = exterior angle / pi, the two faces.
struct Wedge {
  double p0[3], e[3], t0[3], y0[3];
  double p1[3];  // the edge's end vertex (p0 its start)
  double tB[3];  // face n's direction normal to the edge (t0: face 0's)
  double len, n;
  int ta, tb;
};

// A reflector plane for diffraction combined with a reflection: a maximal
// group of coplanar static triangles (unit normal n, offset c = n . x), the
// box of its triangles and their ids (members[first .. first + count)).
struct RPlane {
  double n[3], c;
  float nf[3], cf;  // n and c rounded to FP32 (for the pre-tests)
  float box[6];
  int first, count;  // members first .. first + count - 1, sorted by their lowest coordinate along `axis`
  int axis;          // the box's longest side
  float ext;         // the members' largest extent along it
};

// A wedge's frame rounded to FP32 for the pre-tests (written with the FP64
// record every frame): start, unit edge direction, face 0's direction and
// the exterior's, the length and n pi.
struct WedgeF {
  float3 p0, e, t0, y0;
  float len, npi;
};
constexpr int kWedgeCluster = 32;  // wedges per cluster (a warp's lanes)

// Wedge topology (fixed for a rigid object): faces ta < tb, the local
// indices of the edge's vertices in ta and of the faces' third vertices.
struct WedgeTopo {
  int ta, tb;
  int ka0, ka1, kat, kbt;
};
constexpr int kSmemRefit = 2047;        // per-frame trees up to this many nodes refit in shared memory

// Bounds-checked build (compiled with DCEM_CHECKS): an index marked with
// DCEM_IDX(i, n) is checked against [0, n) before use. One out of range adds
// to this translation unit's check word, keeps the first failing source line,
// and is replaced by 0 (an index every checked array holds), so the access
// stays in bounds and nothing traps. The host reads and clears the words of
// every translation unit after each frame (checks_take_*) and reports
// DCEM_ERR_CHECK. Without DCEM_CHECKS the macro is the index itself.
#ifdef DCEM_CHECKS
static __device__ unsigned g_check_word[2];  // failures, first failing line
template <class T>
__device__ __forceinline__ T check_index(T i, long long n, int line) {
  if ((long long)i >= 0 && (long long)i < n) return i;
  atomicAdd(&g_check_word[0], 1u);
  atomicCAS(&g_check_word[1], 0u, (unsigned)line);
  return T(0);
}
#define DCEM_IDX(i, n) ::dcem::check_index((i), (long long)(n), __LINE__)
#define DCEM_CHECKS_TAKER(name)                                                   \
  unsigned name(unsigned* line) {                                                 \
    unsigned w[2] = {0u, 0u}, z[2] = {0u, 0u};                                    \
    if (cudaMemcpyFromSymbol(w, g_check_word, sizeof(w)) != cudaSuccess) return ~0u; \
    if (w[0] && cudaMemcpyToSymbol(g_check_word, z, sizeof(z)) != cudaSuccess) return ~0u; \
    if (line) *line = w[1];                                                       \
    return w[0];                                                                  \
  }
#else
#define DCEM_IDX(i, n) (i)
#define DCEM_CHECKS_TAKER(name)          \
  unsigned name(unsigned* line) {        \
    if (line) *line = 0u;                \
    return 0u;                           \
  }
#endif
// Failures counted by the bounds-checked build in each translation unit since
// the last call (0 in the normal build); *line: the first failing line.
unsigned checks_take_api(unsigned* line);
unsigned checks_take_bvh(unsigned* line);
unsigned checks_take_trace(unsigned* line);
unsigned checks_take_paths(unsigned* line);
unsigned checks_take_grad(unsigned* line);

// device error bits (DevCounters::err)
enum : unsigned {
  ERR_CAND_OVERFLOW = 1u,
  ERR_UNIQUE_OVERFLOW = 2u,
  ERR_BUCKET_OVERFLOW = 4u,
  ERR_HASH_COLLISION = 8u,
  ERR_NONFINITE = 16u,
  ERR_STACK = 32u,
  ERR_HASH_FULL = 64u,
  ERR_QUEUE_OVERFLOW = 128u,
  ERR_SPAWN_OVERFLOW = 256u,       // transmission: more child rays than slots
  ERR_DIFF_OVERFLOW = 512u,        // diffraction: more pre-test survivors than list slots
};

struct DevCounters {
  unsigned long long segments_traced;
  unsigned long long segments_reused;
  unsigned int n_cand;
  unsigned int n_cand_reused;
  unsigned int n_unique;
  unsigned int n_valid;
  unsigned int n_retrace;
  unsigned int stack_overflow;
  unsigned int err;
  unsigned int objects_moved;
  unsigned int rx_moved;
  unsigned int n_moved_boxes;
  unsigned int work_trace;         // dynamic work counters of the persistent kernels
  unsigned int work_capture;
  unsigned int n_capitems;         // segments traced this frame (capture work list)
  float sah_refit;                 // moving-object tree cost after the last refit
  float sah_build;                 // ... right after its last rebuild
  unsigned int max_seg_nodes;      // most nodes visited by one closest-hit traversal
  unsigned long long node_visits;  // internal nodes visited by closest-hit traversals
  unsigned long long tri_tests;    // triangles tested by closest-hit traversals
  unsigned int n_sticky_valid;     // sticky mode: valid paths that only the cache kept
  unsigned int n_sticky_next;      // sticky mode: valid paths kept for the next frame
  unsigned int n_spawn[kMaxRefl + 1];    // transmission: child rays spawned by trace pass p
  unsigned int work_pass[kMaxRefl + 1];  // ... work counters of passes p >= 1
  unsigned int n_dsurv;            // diffraction: (link, wedge) pairs past the FP32 pre-test
  unsigned int n_val_reused;       // coherent frames: distinct keys whose validation was reused
  unsigned int n_dpair;            // diffraction of order >= 2: wedge pairs past the pre-test
  unsigned int n_dtrip;            // ... triples
};

// Sticky mode: a valid path kept for the next frame (link, depth, sequence).
struct StickyKey {
  int link;
  int depth;
  int tri[kMaxRefl];
};

// Candidate = one reception-sphere capture: ray index and (rx << 4 | segment).
struct Cand {
  int ray;
  int rxseg;
};
__host__ __device__ inline int cand_rx(Cand c) { return (int)((unsigned)c.rxseg >> 4); }
__host__ __device__ inline int cand_seg(Cand c) { return c.rxseg & 15; }

// Internal record of one distinct candidate after validation.
struct PathRec {
  unsigned long long key;
  int rx;
  int depth;
  int ray;
  unsigned int flags;
  int valid;
  int pad;
  double len;
  double amp_re, amp_im;
  int tri[kMaxRefl];
  float pts[kMaxRefl][3];
};

// ---------------------------------------------------------------------------
// FP32 vector helpers with a fixed evaluation order
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 sub3(float3 a, float3 b) {
  return f3(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z));
}
__device__ __forceinline__ float dot3(float3 a, float3 b) {
  return __fmaf_rn(a.z, b.z, __fmaf_rn(a.y, b.y, __fmul_rn(a.x, b.x)));
}
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return f3(__fmaf_rn(a.y, b.z, -__fmul_rn(a.z, b.y)), __fmaf_rn(a.z, b.x, -__fmul_rn(a.x, b.z)),
            __fmaf_rn(a.x, b.y, -__fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float comp(float3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

// ---------------------------------------------------------------------------
// Triangles: three float4 per leaf slot: (v0, id bits), (v1, material), (v2, 0)
// Nodes: four float4 per internal node:
//   n0 = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)
//   n1 = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//   n2 = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//   n3 = (child0, child1, parent, -) as int bits; child < 0 is leaf slot ~c
// ---------------------------------------------------------------------------

// Traversal stack: the first `cap` entries of each thread live in shared
// memory (entry k of thread t at s[k * blockDim.x + t]: consecutive threads,
// consecutive banks), deeper entries in a small local-memory spill area that
// only deep traversals touch. Local-memory stacks of 1024 threads per SM do
// not fit the L1 cache and turn every push and pop into an L2 access.
constexpr int kSpill = 48;
struct TStack {
  int* s;
  int stride;
  int cap;
  int sp;
  int spill[kSpill];
  __device__ __forceinline__ void reset() { sp = 0; }
  __device__ __forceinline__ bool empty() const { return sp == 0; }
  __device__ __forceinline__ bool push(int v) {
    if (sp < cap) s[sp * stride] = v;
    else if (sp - cap < kSpill) spill[sp - cap] = v;
    else return false;
    ++sp;
    return true;
  }
  __device__ __forceinline__ int pop() {
    sp = DCEM_IDX(sp - 1, cap + kSpill);
    return sp < cap ? s[sp * stride] : spill[sp - cap];
  }
};

// This thread's stack over `cap` shared entries per thread at `smem`.
__device__ __forceinline__ void bind_stack(TStack& t, int* smem, int cap) {
  t.s = smem + threadIdx.x;
  t.stride = blockDim.x;
  t.cap = cap;
  t.sp = 0;
}

struct RayPre {
  float3 o;
  float3 inv;   // 1/d with zero components replaced by +-1e-30 (box tests only)
  int kx, ky, kz;
  float Sx, Sy, Sz;
};

__device__ __forceinline__ RayPre ray_pre(float3 o, float3 d) {
  RayPre r;
  r.o = o;
  float dx = fabsf(d.x) < 1e-30f ? copysignf(1e-30f, d.x) : d.x;
  float dy = fabsf(d.y) < 1e-30f ? copysignf(1e-30f, d.y) : d.y;
  float dz = fabsf(d.z) < 1e-30f ? copysignf(1e-30f, d.z) : d.z;
  r.inv = f3(__fdiv_rn(1.0f, dx), __fdiv_rn(1.0f, dy), __fdiv_rn(1.0f, dz));
  // watertight shear constants (Woop, Benthin, Wald 2013)
  float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
  int kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
  int kx = kz == 2 ? 0 : kz + 1;
  int ky = kx == 2 ? 0 : kx + 1;
  if (comp(d, kz) < 0.0f) { int t = kx; kx = ky; ky = t; }
  r.kx = kx; r.ky = ky; r.kz = kz;
  float dkz = comp(d, kz);
  r.Sx = __fdiv_rn(comp(d, kx), dkz);
  r.Sy = __fdiv_rn(comp(d, ky), dkz);
  r.Sz = __fdiv_rn(1.0f, dkz);
  return r;
}

// Conservative slab test: entry/exit over [0, tcap]; the (1 + 1e-5) widening
// keeps every triangle whose FP32 watertight test could report a hit.
// Three-operand minimum and maximum (one instruction on sm_100 and later;
// the same result as two fminf / fmaxf).
__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// Box entry test with a relative margin: accept when tn <= tf (1 + 1e-5) + 1e-30.
__device__ __forceinline__ bool slab_accept(float tn, float tf) { return tn <= __fmaf_rn(tf, 1.00001f, 1e-30f); }

__device__ __forceinline__ bool slab(const RayPre& r, float lox, float hix, float loy, float hiy,
                                     float loz, float hiz, float tcap, float& tn_out) {
  float t0x = __fmul_rn(__fsub_rn(lox, r.o.x), r.inv.x), t1x = __fmul_rn(__fsub_rn(hix, r.o.x), r.inv.x);
  float t0y = __fmul_rn(__fsub_rn(loy, r.o.y), r.inv.y), t1y = __fmul_rn(__fsub_rn(hiy, r.o.y), r.inv.y);
  float t0z = __fmul_rn(__fsub_rn(loz, r.o.z), r.inv.z), t1z = __fmul_rn(__fsub_rn(hiz, r.o.z), r.inv.z);
  float tn = fmax3(fminf(t0x, t1x), fminf(t0y, t1y), fmaxf(fminf(t0z, t1z), 0.0f));
  float tf = fmin3(fmaxf(t0x, t1x), fmaxf(t0y, t1y), fminf(fmaxf(t0z, t1z), tcap));
  tn_out = tn;
  return slab_accept(tn, tf);
}

// Watertight ray/triangle test in FP32. Returns true and the ray parameter t
// when the ray passes through the triangle (no back-face culling).
__device__ __forceinline__ bool tri_hit(const RayPre& r, float3 v0, float3 v1, float3 v2, float& t) {
  float3 A = sub3(v0, r.o), B = sub3(v1, r.o), C = sub3(v2, r.o);
  float Akx = comp(A, r.kx), Aky = comp(A, r.ky), Akz = comp(A, r.kz);
  float Bkx = comp(B, r.kx), Bky = comp(B, r.ky), Bkz = comp(B, r.kz);
  float Ckx = comp(C, r.kx), Cky = comp(C, r.ky), Ckz = comp(C, r.kz);
  float Ax = __fmaf_rn(-r.Sx, Akz, Akx), Ay = __fmaf_rn(-r.Sy, Akz, Aky);
  float Bx = __fmaf_rn(-r.Sx, Bkz, Bkx), By = __fmaf_rn(-r.Sy, Bkz, Bky);
  float Cx = __fmaf_rn(-r.Sx, Ckz, Ckx), Cy = __fmaf_rn(-r.Sy, Ckz, Cky);
  float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
  float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
  float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
  if (U == 0.0f || V == 0.0f || W == 0.0f) {  // exact edge: decide in double
    double U2 = (double)Cx * (double)By - (double)Cy * (double)Bx;
    double V2 = (double)Ax * (double)Cy - (double)Ay * (double)Cx;
    double W2 = (double)Bx * (double)Ay - (double)By * (double)Ax;
    U = (float)U2; V = (float)V2; W = (float)W2;
    if (U == 0.0f && U2 != 0.0) U = U2 > 0 ? 2e-38f : -2e-38f;
    if (V == 0.0f && V2 != 0.0) V = V2 > 0 ? 2e-38f : -2e-38f;
    if (W == 0.0f && W2 != 0.0) W = W2 > 0 ? 2e-38f : -2e-38f;
  }
  if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return false;
  float det = __fadd_rn(__fadd_rn(U, V), W);
  if (det == 0.0f) return false;
  float Az = __fmul_rn(r.Sz, Akz), Bz = __fmul_rn(r.Sz, Bkz), Cz = __fmul_rn(r.Sz, Ckz);
  float T = __fmaf_rn(W, Cz, __fmaf_rn(V, Bz, __fmul_rn(U, Az)));
  t = __fdiv_rn(T, det);
  return true;
}

__device__ __forceinline__ void load_tri(const float4* __restrict__ tris, int slot, float3& v0,
                                         float3& v1, float3& v2, int& id) {
  float4 a = __ldg(&tris[3 * slot]), b = __ldg(&tris[3 * slot + 1]), c = __ldg(&tris[3 * slot + 2]);
  v0 = f3(a.x, a.y, a.z);
  v1 = f3(b.x, b.y, b.z);
  v2 = f3(c.x, c.y, c.z);
  id = __float_as_int(a.w);
}

struct Bvh {
  const float4* __restrict__ nodes;
  const float4* __restrict__ tris;
  int root0, root1;
  int max_visits;  // nodes + leaves of both trees: a valid traversal never exceeds it
  int nnodes, ntris;  // internal nodes of both trees, triangle (leaf) slots
};

// Closest hit over both trees, t > tmin, excluding triangle id `excl`; ties in
// t go to the lowest triangle id, so the result does not depend on the tree
// shape or the traversal order. Returns the leaf slot or -1.
__device__ __forceinline__ int closest_hit(const Bvh& bvh, const RayPre& r, float tmin, int excl,
                                           float& t_best, int& id_best, unsigned& overflow,
                                           unsigned& n_nodes, unsigned& n_tris, TStack& st) {
  st.reset();
  t_best = __int_as_float(0x7f800000);
  id_best = 0x7fffffff;
  int slot_best = -1;
  if (bvh.root1 != kEmpty) st.push(bvh.root1);
  int cur = bvh.root0;
  for (int visits = 0;; ++visits) {
    if (visits > bvh.max_visits) {  // malformed tree: stop and report
      overflow = 1u;
      break;
    }
    if (cur == kEmpty) {
      if (st.empty()) break;
      cur = st.pop();
      continue;
    }
    if (cur >= 0) {
      ++n_nodes;
      const float4* n = bvh.nodes + 4 * (size_t)DCEM_IDX(cur, bvh.nnodes);
      float4 n0 = __ldg(n), n1 = __ldg(n + 1), n2 = __ldg(n + 2), n3 = __ldg(n + 3);
      float tn0, tn1;
      bool h0 = slab(r, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, t_best, tn0);
      bool h1 = slab(r, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, t_best, tn1);
      int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
      if (h0 && h1) {
        int nearc = tn0 <= tn1 ? c0 : c1, farc = tn0 <= tn1 ? c1 : c0;
        if (!st.push(farc)) overflow = 1u;
        cur = nearc;
      } else if (h0) {
        cur = c0;
      } else if (h1) {
        cur = c1;
      } else {
        cur = kEmpty;
      }
    } else {
      int slot = ~cur;
      ++n_tris;
      float3 v0, v1, v2;
      int id;
      load_tri(bvh.tris, DCEM_IDX(slot, bvh.ntris), v0, v1, v2, id);
      float t;
      if (id != excl && tri_hit(r, v0, v1, v2, t) && t > tmin) {
        if (t < t_best || (t == t_best && id < id_best)) {
          t_best = t;
          id_best = id;
          slot_best = slot;
        }
      }
      cur = kEmpty;
    }
  }
  return slot_best;
}

// ---------------------------------------------------------------------------
// compact nodes for shared memory: child boxes as 16-bit codes on a per-frame
// grid (origin O, step S_k on axis k) that contains both trees, rounded
// outward by three steps, so a code box always contains the exact box. 32
// bytes per node: words 0-2 = child 0 axes x, y, z, words 3-5 = child 1
// axes, words 6-7 = child ids; each axis word holds the lo code in its low
// half and the hi code in its high half.
//
// The slab test runs in grid units: with F = 2^23 + code (the float whose
// bits are 0x4B00'code', built by one byte permute) the plane parameter is
// t = F * (S_k/d_k) + ((O_k - o_k)/d_k - 2^23 S_k/d_k), one FMA per plane.
// For ray origins within 4e6 steps of O on every axis the rounding of the
// two per-ray terms moves a plane by less than 1.3 steps (half a step from
// the 2^23 offset, 0.75 from (O - o)/d, the rest relative), which the
// 3-step margin covers; farther origins take the full-precision traversal
// instead. The per-axis sign of d picks the near and far code, so no
// per-axis min/max is needed.
// ---------------------------------------------------------------------------
struct QFrame {
  float ox, oy, oz, sx, sy, sz;
  int n4;  // 4-wide nodes in the copy (index checks)
};

struct QRay {
  float ix, iy, iz;        // S_k / d_k per axis
  float kx, ky, kz;        // (O_k - o_k) / d_k - 2^23 S_k / d_k per axis
  unsigned nx, ny, nz;     // byte-permute selector of the near code per axis
};

__device__ __forceinline__ bool qray_make(const QFrame& f, const RayPre& r, QRay& q) {
  float ex = __fsub_rn(f.ox, r.o.x), ey = __fsub_rn(f.oy, r.o.y), ez = __fsub_rn(f.oz, r.o.z);
  if (!(fabsf(ex) <= __fmul_rn(4.0e6f, f.sx) && fabsf(ey) <= __fmul_rn(4.0e6f, f.sy) &&
        fabsf(ez) <= __fmul_rn(4.0e6f, f.sz)))
    return false;
  q.ix = __fmul_rn(f.sx, r.inv.x);
  q.iy = __fmul_rn(f.sy, r.inv.y);
  q.iz = __fmul_rn(f.sz, r.inv.z);
  q.kx = __fmaf_rn(-8388608.0f, q.ix, __fmul_rn(ex, r.inv.x));
  q.ky = __fmaf_rn(-8388608.0f, q.iy, __fmul_rn(ey, r.inv.y));
  q.kz = __fmaf_rn(-8388608.0f, q.iz, __fmul_rn(ez, r.inv.z));
  q.nx = r.inv.x >= 0.0f ? 0x5410u : 0x5432u;
  q.ny = r.inv.y >= 0.0f ? 0x5410u : 0x5432u;
  q.nz = r.inv.z >= 0.0f ? 0x5410u : 0x5432u;
  return true;
}

// 2^23 + the near (sel) or far (sel ^ 0x22) code of an axis word
__device__ __forceinline__ float qcode(unsigned w, unsigned sel) {
  return __uint_as_float(__byte_perm(w, 0x4B00u, sel));
}

__device__ __forceinline__ bool qslab(const QRay& q, unsigned wx, unsigned wy, unsigned wz, float tcap,
                                      float& tn_out) {
  float tnx = __fmaf_rn(qcode(wx, q.nx), q.ix, q.kx), tfx = __fmaf_rn(qcode(wx, q.nx ^ 0x22u), q.ix, q.kx);
  float tny = __fmaf_rn(qcode(wy, q.ny), q.iy, q.ky), tfy = __fmaf_rn(qcode(wy, q.ny ^ 0x22u), q.iy, q.ky);
  float tnz = __fmaf_rn(qcode(wz, q.nz), q.iz, q.kz), tfz = __fmaf_rn(qcode(wz, q.nz ^ 0x22u), q.iz, q.kz);
  float tn = fmax3(tnx, tny, fmaxf(tnz, 0.0f));
  float tf = fmin3(tfx, tfy, fminf(tfz, tcap));
  tn_out = tn;
  return slab_accept(tn, tf);
}

// Ray origins far outside the grid: full-precision nodes, out of line so
// that the common path keeps its registers.
static __device__ __noinline__ int closest_hit_far(const Bvh bvh, const RayPre r, float tmin, int excl, float* t_best,
                                            int* id_best, unsigned* overflow, unsigned* n_nodes, unsigned* n_tris,
                                            int* sbase, int stride, int cap) {
  TStack st;
  st.s = sbase;
  st.stride = stride;
  st.cap = cap;
  st.sp = 0;
  float t;
  int id;
  unsigned ovf = 0, nn = 0, nt = 0;
  int slot = closest_hit(bvh, r, tmin, excl, t, id, ovf, nn, nt, st);
  *t_best = t;
  *id_best = id;
  *overflow |= ovf;
  *n_nodes += nn;
  *n_tris += nt;
  return slot;
}

// Closest hit as closest_hit(), with the nodes read from the compact copy
// (shared memory). Same triangle test and tie rule, so the same result.
__device__ __forceinline__ int closest_hit_q(const uint4* qn, const QFrame& f, const Bvh& bvh, const RayPre& r,
                                             float tmin, int excl, float& t_best, int& id_best, unsigned& overflow,
                                             unsigned& n_nodes, unsigned& n_tris, TStack& st) {
  QRay q;
  if (!qray_make(f, r, q))
    return closest_hit_far(bvh, r, tmin, excl, &t_best, &id_best, &overflow, &n_nodes, &n_tris, st.s, st.stride,
                           st.cap);
  st.reset();
  t_best = __int_as_float(0x7f800000);
  id_best = 0x7fffffff;
  int slot_best = -1;
  if (bvh.root1 != kEmpty) st.push(bvh.root1);
  int cur = bvh.root0;
  if (cur == kEmpty) cur = st.empty() ? kEmpty : st.pop();
  for (int visits = 0; cur != kEmpty; ++visits) {
    if (visits > bvh.max_visits) {
      overflow = 1u;
      break;
    }
    if (cur >= 0) {
      ++n_nodes;
      const int ci = DCEM_IDX(cur, bvh.nnodes);
      uint4 a = qn[2 * ci], b = qn[2 * ci + 1];
      float tn0, tn1;
      bool h0 = qslab(q, a.x, a.y, a.z, t_best, tn0);
      bool h1 = qslab(q, a.w, b.x, b.y, t_best, tn1);
      int c0 = (int)b.z, c1 = (int)b.w;
      if (h0 && h1) {
        int nearc = tn0 <= tn1 ? c0 : c1, farc = tn0 <= tn1 ? c1 : c0;
        if (!st.push(farc)) overflow = 1u;
        cur = nearc;
      } else if (h0) {
        cur = c0;
      } else if (h1) {
        cur = c1;
      } else {
        cur = st.empty() ? kEmpty : st.pop();
      }
    } else {
      int slot = ~cur;
      ++n_tris;
      float3 v0, v1, v2;
      int id;
      load_tri(bvh.tris, DCEM_IDX(slot, bvh.ntris), v0, v1, v2, id);
      float t;
      if (id != excl && tri_hit(r, v0, v1, v2, t) && t > tmin) {
        if (t < t_best || (t == t_best && id < id_best)) {
          t_best = t;
          id_best = id;
          slot_best = slot;
        }
      }
      cur = st.empty() ? kEmpty : st.pop();
    }
  }
  return slot_best;
}

// 4-wide compact nodes (shared memory), 64 bytes each: words 0-11 = the axis
// words of children 0-3 (x, y, z per child, as in the 2-wide copy), words
// 12-15 = the child codes (4-wide node index, leaf ~slot, or kEmpty with an
// inverted box that no ray meets).
__device__ __forceinline__ void cswap(float& da, int& ca, float& db, int& cb) {
  bool sw = db < da;
  float t = sw ? db : da;
  db = sw ? da : db;
  da = t;
  int c = sw ? cb : ca;
  cb = sw ? ca : cb;
  ca = c;
}

// Closest hit as closest_hit(), over the 4-wide compact copy: per step the
// four child boxes are tested, the hit ones ordered by entry distance, the
// nearest visited next and the others pushed. Node visits count box pairs
// (a 4-wide step = 2), the unit of the 2-wide traversals. kG: the copy is
// read from global memory (read-only path) instead of shared memory.
template <bool kG = false>
__device__ __forceinline__ int closest_hit_q4(const uint4* qn, const QFrame& f, const Bvh& bvh, int root0,
                                              int root1, const RayPre& r, float tmin, int excl, float& t_best,
                                              int& id_best, unsigned& overflow, unsigned& n_nodes,
                                              unsigned& n_tris, TStack& st) {
  QRay q;
  if (!qray_make(f, r, q))
    return closest_hit_far(bvh, r, tmin, excl, &t_best, &id_best, &overflow, &n_nodes, &n_tris, st.s, st.stride,
                           st.cap);
  const float inf = __int_as_float(0x7f800000);
  st.reset();
  t_best = inf;
  id_best = 0x7fffffff;
  int slot_best = -1;
  if (root1 != kEmpty) st.push(root1);
  int cur = root0;
  if (cur == kEmpty) cur = st.empty() ? kEmpty : st.pop();
  for (int visits = 0; cur != kEmpty; ++visits) {
    if (visits > bvh.max_visits) {
      overflow = 1u;
      break;
    }
    if (cur >= 0) {
      n_nodes += 2;
      const uint4* nd = qn + 4 * (size_t)DCEM_IDX(cur, f.n4);
      uint4 A, B, C, K;
      if (kG) {
        A = __ldg(nd);
        B = __ldg(nd + 1);
        C = __ldg(nd + 2);
        K = __ldg(nd + 3);
      } else {
        A = nd[0];
        B = nd[1];
        C = nd[2];
        K = nd[3];
      }
      float t0, t1, t2, t3;
      float d0 = qslab(q, A.x, A.y, A.z, t_best, t0) ? t0 : inf;
      float d1 = qslab(q, A.w, B.x, B.y, t_best, t1) ? t1 : inf;
      float d2 = qslab(q, B.z, B.w, C.x, t_best, t2) ? t2 : inf;
      float d3 = qslab(q, C.y, C.z, C.w, t_best, t3) ? t3 : inf;
      int c0 = (int)K.x, c1 = (int)K.y, c2 = (int)K.z, c3 = (int)K.w;
      cswap(d0, c0, d1, c1);
      cswap(d2, c2, d3, c3);
      cswap(d0, c0, d2, c2);
      cswap(d1, c1, d3, c3);
      cswap(d1, c1, d2, c2);
      if (d3 < inf && !st.push(c3)) overflow = 1u;
      if (d2 < inf && !st.push(c2)) overflow = 1u;
      if (d1 < inf && !st.push(c1)) overflow = 1u;
      cur = d0 < inf ? c0 : (st.empty() ? kEmpty : st.pop());
    } else {
      int slot = ~cur;
      ++n_tris;
      float3 v0, v1, v2;
      int id;
      load_tri(bvh.tris, DCEM_IDX(slot, bvh.ntris), v0, v1, v2, id);
      float t;
      if (id != excl && tri_hit(r, v0, v1, v2, t) && t > tmin) {
        if (t < t_best || (t == t_best && id < id_best)) {
          t_best = t;
          id_best = id;
          slot_best = slot;
        }
      }
      cur = st.empty() ? kEmpty : st.pop();
    }
  }
  return slot_best;
}

// Any hit with t in (t0, t1), excluding ids ex0 .. ex3 (occlusion test).
__device__ __forceinline__ bool any_hit(const Bvh& bvh, const RayPre& r, float t0, float t1,
                                        int ex0, int ex1, unsigned& overflow, TStack& st, int ex2 = -1,
                                        int ex3 = -1) {
  st.reset();
  if (bvh.root1 != kEmpty) st.push(bvh.root1);
  int cur = bvh.root0;
  for (int visits = 0;; ++visits) {
    if (visits > bvh.max_visits) {
      overflow = 1u;
      break;
    }
    if (cur == kEmpty) {
      if (st.empty()) break;
      cur = st.pop();
      continue;
    }
    if (cur >= 0) {
      const float4* n = bvh.nodes + 4 * (size_t)DCEM_IDX(cur, bvh.nnodes);
      float4 n0 = __ldg(n), n1 = __ldg(n + 1), n2 = __ldg(n + 2), n3 = __ldg(n + 3);
      float tn0, tn1;
      bool h0 = slab(r, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, t1, tn0);
      bool h1 = slab(r, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, t1, tn1);
      int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
      if (h0 && h1) {
        if (!st.push(c1)) overflow = 1u;
        cur = c0;
      } else if (h0) {
        cur = c0;
      } else if (h1) {
        cur = c1;
      } else {
        cur = kEmpty;
      }
    } else {
      float3 v0, v1, v2;
      int id;
      load_tri(bvh.tris, DCEM_IDX(~cur, bvh.ntris), v0, v1, v2, id);
      float t;
      if (id != ex0 && id != ex1 && id != ex2 && id != ex3 && tri_hit(r, v0, v1, v2, t) && t > t0 && t < t1)
        return true;
      cur = kEmpty;
    }
  }
  return false;
}

// Reception-sphere capture of one segment (o, d unit, unfolded start length D,
// length tend) by receiver R: closest approach s in [0, tend], captured iff
// |R - (o + s d)| <= alpha_eff (D + s).
__device__ __forceinline__ bool captured(float3 o, float3 d, float D, float tend, float alpha_eff,
                                         float3 R) {
  float3 w = sub3(R, o);
  float s = dot3(w, d);
  s = fminf(fmaxf(s, 0.0f), tend);
  float3 q = f3(__fmaf_rn(-s, d.x, w.x), __fmaf_rn(-s, d.y, w.y), __fmaf_rn(-s, d.z, w.z));
  float dist2 = dot3(q, q);
  float rho = __fmul_rn(alpha_eff, __fadd_rn(D, s));
  return dist2 <= __fmul_rn(rho, rho);
}

// ---------------------------------------------------------------------------
// small per-frame trees: receivers (points) and moved-object boxes
// ---------------------------------------------------------------------------
struct SmallBvh {
  const float4* __restrict__ nodes;  // same node layout as the scene trees
  const int* __restrict__ perm;      // leaf j -> receiver / box index
  const int* root;                   // device: root code (kEmpty, leaf ~j, or node)
  const float* root_box;             // device: box of a single-leaf tree
  int max_visits;
  int cap;                           // leaves the tree's arrays hold (nodes: cap - 1)
};

// Slab test returning the clipped parameter interval [tn, tf] within [0, tcap].
__device__ __forceinline__ bool slab_io(const RayPre& r, float lox, float hix, float loy, float hiy,
                                        float loz, float hiz, float tcap, float& tn, float& tf) {
  float t0x = __fmul_rn(__fsub_rn(lox, r.o.x), r.inv.x), t1x = __fmul_rn(__fsub_rn(hix, r.o.x), r.inv.x);
  float t0y = __fmul_rn(__fsub_rn(loy, r.o.y), r.inv.y), t1y = __fmul_rn(__fsub_rn(hiy, r.o.y), r.inv.y);
  float t0z = __fmul_rn(__fsub_rn(loz, r.o.z), r.inv.z), t1z = __fmul_rn(__fsub_rn(hiz, r.o.z), r.inv.z);
  tn = fmax3(fminf(t0x, t1x), fminf(t0y, t1y), fmaxf(fminf(t0z, t1z), 0.0f));
  tf = fmin3(fmaxf(t0x, t1x), fmaxf(t0y, t1y), fminf(fmaxf(t0z, t1z), tcap));
  return slab_accept(tn, tf);
}

// Conservative filter for the capture cone of a segment against a box of
// receivers: false only if no point of the box can pass `captured`. A point
// captured at parameter s lies within rho(s) = alpha (D + s) of the segment,
// so the segment meets the box grown by rho(tend); within that clipped
// interval [tn, tf] the radius is at most rho(tf), so the segment also meets
// the box grown by rho(tf). Margins (0.1% and 1 cm) exceed FP32 rounding.
__device__ __forceinline__ bool cone_box(const RayPre& r, float D, float tend, float alpha, float lox,
                                         float hix, float loy, float hiy, float loz, float hiz) {
  float a = alpha * 1.001f;
  float g = a * (D + tend) + 0.01f;
  float tn, tf;
  if (!slab_io(r, lox - g, hix + g, loy - g, hiy + g, loz - g, hiz + g, tend, tn, tf)) return false;
  g = a * (D + fminf(tf * 1.00001f, tend)) + 0.01f;
  return slab_io(r, lox - g, hix + g, loy - g, hiy + g, loz - g, hiz + g, tend, tn, tf);
}

// Every receiver whose reception sphere captures the segment (r.o, d, D,
// tend) is passed to emit(rx index). Returns false on a malformed tree or a
// stack overflow.
template <class Emit>
__device__ __forceinline__ bool capture_tree(const SmallBvh& t, const float4* __restrict__ rx,
                                             const RayPre& r, float3 d, float D, float tend, float alpha,
                                             TStack& st, Emit&& emit) {
  int root = *t.root;
  if (root == kEmpty) return true;
  // Every receiver lies in the root box, so a capture at s puts the segment
  // within rho(s) <= rho(te) of that box: clip the culling length te to the
  // exit of the box grown by the largest radius, twice (the second time
  // with the radius at the first exit). The exact test keeps tend.
  float te = tend;
  {
    const float* rb = t.root_box;
    for (int it = 0; it < 2; ++it) {
      float g = alpha * 1.001f * (D + te) + 0.01f, tn, tf;
      if (!slab_io(r, rb[0] - g, rb[3] + g, rb[1] - g, rb[4] + g, rb[2] - g, rb[5] + g, te, tn, tf)) return true;
      te = fminf(te, tf * 1.00001f + 1e-6f);
    }
  }
  st.reset();
  int cur = root;
  for (int visits = 0; visits <= t.max_visits; ++visits) {
    if (cur < 0) {
      int ri = t.perm[DCEM_IDX(~cur, t.cap)];
      float4 v = rx[DCEM_IDX(ri, t.cap)];
      if (captured(r.o, d, D, tend, alpha, f3(v.x, v.y, v.z))) emit(ri);
    } else {
      const float4* n = t.nodes + 4 * (size_t)DCEM_IDX(cur, t.cap - 1);
      float4 n0 = n[0], n1 = n[1], n2 = n[2], n3 = n[3];
      int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
      bool m0 = cone_box(r, D, te, alpha, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y);
      bool m1 = cone_box(r, D, te, alpha, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w);
      if (m1 && !st.push(c1)) return false;
      if (m0 && !st.push(c0)) return false;
    }
    if (st.empty()) return true;
    cur = st.pop();
  }
  return false;
}

// Does the segment o + t d, t in [0, tend], meet the box (conservatively)?
__device__ __forceinline__ bool seg_box(const RayPre& r, float tend, const float* b) {
  float tn;
  return slab(r, b[0], b[3], b[1], b[4], b[2], b[5], tend, tn);
}

// Does the segment meet any box of the tree? On a malformed tree or a stack
// overflow the answer is conservatively true.
__device__ __forceinline__ bool seg_hits_tree(const SmallBvh& t, const RayPre& r, float tend, TStack& st) {
  int root = *t.root;
  if (root == kEmpty) return false;
  if (root < 0) return seg_box(r, tend, t.root_box);
  st.reset();
  int cur = root;
  for (int visits = 0; visits <= t.max_visits; ++visits) {
    const float4* n = t.nodes + 4 * (size_t)DCEM_IDX(cur, t.cap - 1);
    float4 n0 = n[0], n1 = n[1], n2 = n[2], n3 = n[3];
    int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
    float tn;
    bool h0 = slab(r, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, tend, tn);
    bool h1 = slab(r, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, tend, tn);
    if ((h0 && c0 < 0) || (h1 && c1 < 0)) return true;
    if (h1 && !st.push(c1)) return true;
    if (h0 && !st.push(c0)) return true;
    if (st.empty()) return false;
    cur = st.pop();
  }
  return true;
}

// Copies a per-frame small tree (nn internal nodes, nperm leaves) to shared
// memory at dst (16-byte aligned) and points t at the copy; returns the end
// of the copy (16-byte aligned). All threads of the block call it; the
// caller synchronises before use.
__device__ __forceinline__ char* stage_tree(const SmallBvh& g, int nn, int nperm, char* dst, SmallBvh& t) {
  float4* sn = reinterpret_cast<float4*>(dst);
  for (int i = threadIdx.x; i < 4 * nn; i += blockDim.x) sn[i] = g.nodes[i];
  int* sp = reinterpret_cast<int*>(sn + 4 * nn);
  for (int i = threadIdx.x; i < nperm; i += blockDim.x) sp[i] = g.perm[i];
  int* sr = sp + ((nperm + 3) & ~3);  // root code, then the root box
  if (threadIdx.x == 0) sr[0] = *g.root;
  if (threadIdx.x < 6) reinterpret_cast<float*>(sr + 1)[threadIdx.x] = g.root_box[threadIdx.x];
  t = g;
  t.cap = nn + 1;
  t.nodes = sn;
  t.perm = sp;
  t.root = sr;
  t.root_box = reinterpret_cast<const float*>(sr + 1);
  return reinterpret_cast<char*>(sr + 8);
}

// Shared-memory bytes stage_tree needs.
__host__ __device__ __forceinline__ size_t stage_bytes(int nn, int nperm) {
  return (size_t)nn * 64 + (size_t)((nperm + 3) & ~3) * 4 + 32;
}

// 64-bit path key: (rx, depth, triangle ids) mixed with the SplitMix64 finaliser.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Total order on float bits usable with atomicMin/atomicMax on unsigned.
__device__ __forceinline__ unsigned f2o(float f) {
  unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float o2f(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
#else
  unsigned v = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
  float f;
  memcpy(&f, &v, 4);
  return f;
#endif
}

}  // namespace dcem
