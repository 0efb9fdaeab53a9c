// trace.cu -- shooting-and-bouncing rays and frame-to-frame coherence.
//
// Sec. III "Backward ray tracing", steps 1-2: every ray of the sampled sphere
// is traced from the transmitter through up to N specular reflections; each
// segment's closest hit comes from a stack traversal of the two LBVH trees
// (static scene, moving objects) with a watertight FP32 triangle test, and
// each segment is tested against every receiver's reception sphere. Every
// segment is logged (origin, direction, unfolded length, hit) so that the
// next frame can reuse it.
//
// Sec. III "Propagation path caching": in a coherent frame a logged segment is
// reused unless it meets the old or the new box of an object that moved; a
// ray is retraced from its first such segment. Reused segments are re-tested
// only against receivers that moved; captures of reused segments by receivers
// that did not move are carried over. The arithmetic of every segment is the
// same device code in both modes, so the result equals a full retrace.
#include "trace.cuh"

#include "bvh.cuh"

namespace dcem {

// ---------------------------------------------------------------------------
// per-segment kernel body shared by full and coherent frames
// ---------------------------------------------------------------------------
__device__ __forceinline__ void emit_cand(const TraceArgs& a, int ray, int seg, int rx) {
  unsigned idx = atomicAdd(&a.ctr->n_cand, 1u);
  if (idx < a.cand_cap) a.cand[idx] = Cand{ray, (rx << 4) | seg};
  else atomicOr(&a.ctr->err, ERR_CAND_OVERFLOW);
}

// Index of segment b of slot `ray` in the log arrays ((N + T + 1) x LS).
__device__ __forceinline__ size_t log_at(const TraceArgs& a, int b, int ray) {
  return (size_t)DCEM_IDX(b, a.N + a.max_trans + 1) * a.LS + DCEM_IDX(ray, a.LS);
}
// Capacity of the capture work list.
__device__ __forceinline__ long long capitems_cap(const TraceArgs& a) {
  return (long long)(a.N + a.max_trans + 1) * a.LS;
}

// Warp-wide dynamic work fetch: lane 0 takes the next `n` items.
__device__ __forceinline__ int fetch_warp(unsigned* counter, unsigned n) {
  int base = 0;
  if ((threadIdx.x & 31) == 0) base = (int)atomicAdd(counter, n);
  return __shfl_sync(0xffffffffu, base, 0);
}

// Persistent traversal with a per-lane ray fetch: every lane traces one
// segment of its own ray per step, and a lane whose ray has ended takes the
// next ray of the queue at once (one atomic per warp for all such lanes), so
// a warp never waits for its longest ray. Rays are sorted by direction, so
// consecutive fetches travel together. A queue smaller than the resident
// lanes is spread over every warp (at most `width` lanes of each take rays)
// so that short retrace queues use all SMs. Per segment b from the ray's
// restart point (0 in a full frame) to N: closest hit, segment log, specular
// reflection. Captures are tested by k_capture.
//
// kT (transmission): a hit on a transmitting material also spawns a child
// that continues straight through (Sec. III "Reflected and transmitted
// rays"); the child's slot gets the parent's interaction prefix, the
// transmission (id | kTransBit) and its start state, and the next pass
// traces it. Pass p > 0 takes the children of pass p - 1 as its work.
template <bool kQ, bool kG = false, bool kT = false>
__device__ __forceinline__ void trace_rays(const TraceArgs& a, const uint4* qn, const QFrame& qf, TStack& st,
                                           int qr0, int qr1) {
  const int R = a.R;
  [[maybe_unused]] const int LS = a.LS;  // bounds of the checked build
  int nq, slot0 = 0, spawn_base = R;
  unsigned* work = &a.ctr->work_trace;
  if (kT) {
    // children of earlier passes occupy the slots from R on, pass by pass
    for (int p = 0; p < a.pass; ++p) {
      int n = (int)a.ctr->n_spawn[p];
      if (p == a.pass - 1) slot0 = spawn_base;
      spawn_base += n;
    }
    if (a.pass > 0) {
      nq = min((int)a.ctr->n_spawn[a.pass - 1], max(0, R + a.child_cap - slot0));
      work = &a.ctr->work_pass[a.pass];
    } else {
      nq = R;
    }
  } else {
    nq = a.queue ? (int)min(*a.nq_dev, (unsigned)R) : R;
  }
  const int lane = threadIdx.x & 31;
  const int warps = (int)((gridDim.x * blockDim.x) >> 5);
  const int width = min(32, max(1, (nq + warps - 1) / warps));
  unsigned segs = 0, nodes = 0, tris = 0, ovf = 0, maxn = 0;
  int ray = lane < width ? -1 : -2;  // -1: takes a ray next, -2: finished
  int b = 0, last = -1;
  int nr = 0, ntr = 0, set = 0;     // transmission: reflections, transmissions, ray set
  float3 o = f3(0.0f, 0.0f, 0.0f), d = o;
  float D = 0.0f;
  for (;;) {
    unsigned need = __ballot_sync(0xffffffffu, ray == -1);
    if (need) {
      int leader = __ffs(need) - 1;
      int base = 0;
      if (lane == leader) base = (int)atomicAdd(work, (unsigned)__popc(need));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (ray == -1) {
        int q = base + __popc(need & ((1u << lane) - 1u));
        if (q < nq) {
          if (kT && a.pass > 0) {
            ray = slot0 + q;
            b = a.restart[DCEM_IDX(ray, LS)];
            int inf = a.inst[DCEM_IDX(ray - R, a.child_cap)];
            nr = inf & 15;
            ntr = (inf >> 4) & 15;
            set = inf >> 8;
          } else {
            ray = a.queue ? a.queue[DCEM_IDX(q, R)] : q;
            b = a.queue ? a.restart[DCEM_IDX(ray, R)] : 0;
            nr = b;
            ntr = 0;
          }
          if (b == 0) {
            float4 rd = __ldg(&a.rays[DCEM_IDX(ray, R)]);
            set = __float_as_int(rd.w);
            float4 t4 = __ldg(&a.txs[DCEM_IDX(set, a.nsets)]);
            o = f3(t4.x, t4.y, t4.z);
            d = f3(rd.x, rd.y, rd.z);
            D = 0.0f;
            last = -1;
          } else {
            float4 lo = a.log_o[log_at(a, b, ray)], ld = a.log_d[log_at(a, b, ray)];
            o = f3(lo.x, lo.y, lo.z);
            D = lo.w;
            d = f3(ld.x, ld.y, ld.z);
            last = a.log_id[log_at(a, b - 1, ray)] & ~kTransBit;
          }
        } else {
          ray = -2;
        }
      }
    }
    if (__all_sync(0xffffffffu, ray == -2)) break;
    unsigned item = 0xffffffffu;  // segment traced in this step, for the capture list
    if (ray >= 0) {
      RayPre rp = ray_pre(o, d);
      float t;
      int id;
      unsigned nn = 0, nt = 0;
      int slot = kQ ? closest_hit_q4<kG>(qn, qf, a.bvh, qr0, qr1, rp, a.tmin, last, t, id, ovf, nn, nt, st)
                    : closest_hit(a.bvh, rp, a.tmin, last, t, id, ovf, nn, nt, st);
      ++segs;
      nodes += nn;
      tris += nt;
      maxn = max(maxn, nn);
      bool hit = slot >= 0;
      a.log_o[log_at(a, b, ray)] = make_float4(o.x, o.y, o.z, D);
      a.log_d[log_at(a, b, ray)] = make_float4(d.x, d.y, d.z, hit ? t : __int_as_float(0x7f800000));
      a.log_id[log_at(a, b, ray)] = hit ? id : -1;
      item = ((unsigned)ray << 4) | (unsigned)b;
      if (kT && hit && ntr < a.max_trans) {
        // transmitting material: a child continues straight through
        int m = __float_as_int(__ldg(&a.bvh.tris[3 * DCEM_IDX(slot, a.bvh.ntris) + 1]).w);
        if (__ldg(&a.mats[m]).w >= 0.0f) {
          unsigned c = atomicAdd(&a.ctr->n_spawn[a.pass], 1u);
          int cs = spawn_base + (int)c;
          if (cs < R + a.child_cap) {
            for (int j = 0; j < b; ++j) a.log_id[log_at(a, j, cs)] = a.log_id[log_at(a, j, ray)];
            a.log_id[log_at(a, b, cs)] = id | kTransBit;
            float3 p = f3(__fmaf_rn(t, d.x, o.x), __fmaf_rn(t, d.y, o.y), __fmaf_rn(t, d.z, o.z));
            a.log_o[log_at(a, b + 1, cs)] = make_float4(p.x, p.y, p.z, __fadd_rn(D, t));
            a.log_d[log_at(a, b + 1, cs)] = make_float4(d.x, d.y, d.z, 0.0f);
            a.restart[cs] = b + 1;
            a.inst[DCEM_IDX(cs - R, a.child_cap)] = nr | ((ntr + 1) << 4) | (set << 8);
            a.inst_root[DCEM_IDX(cs - R, a.child_cap)] = ray < R ? ray : a.inst_root[DCEM_IDX(ray - R, a.child_cap)];
          } else {
            atomicOr(&a.ctr->err, ERR_SPAWN_OVERFLOW);
          }
        }
      }
      if (!hit || (kT ? nr >= a.N : b == a.N)) {
        a.nseg[DCEM_IDX(ray, LS)] = b + 1;
        ray = -1;
      } else {
        // specular reflection: d' = d - 2 (d.n)/(n.n) n, renormalised
        float3 v0, v1, v2;
        int tid;
        load_tri(a.bvh.tris, DCEM_IDX(slot, a.bvh.ntris), v0, v1, v2, tid);
        float3 n = cross3(sub3(v1, v0), sub3(v2, v0));
        float k = __fdiv_rn(__fmul_rn(2.0f, dot3(d, n)), dot3(n, n));
        float3 dr = f3(__fmaf_rn(-k, n.x, d.x), __fmaf_rn(-k, n.y, d.y), __fmaf_rn(-k, n.z, d.z));
        float inv = __fdiv_rn(1.0f, __fsqrt_rn(dot3(dr, dr)));
        o = f3(__fmaf_rn(t, d.x, o.x), __fmaf_rn(t, d.y, o.y), __fmaf_rn(t, d.z, o.z));
        d = f3(__fmul_rn(dr.x, inv), __fmul_rn(dr.y, inv), __fmul_rn(dr.z, inv));
        D = __fadd_rn(D, t);
        last = id;
        ++b;
        if (kT) ++nr;
      }
    }
    unsigned logged = __ballot_sync(0xffffffffu, item != 0xffffffffu);
    if (logged) {
      int leader = __ffs(logged) - 1;
      unsigned base = 0;
      if (lane == leader) base = atomicAdd(&a.ctr->n_capitems, (unsigned)__popc(logged));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (item != 0xffffffffu) a.capitems[DCEM_IDX(base + __popc(logged & ((1u << lane) - 1u)), capitems_cap(a))] = item;
    }
  }
  unsigned long long wsegs = segs, wnodes = nodes, wtris = tris;
  for (int off = 16; off > 0; off >>= 1) {
    wsegs += __shfl_down_sync(0xffffffffu, wsegs, off);
    wnodes += __shfl_down_sync(0xffffffffu, wnodes, off);
    wtris += __shfl_down_sync(0xffffffffu, wtris, off);
    maxn = max(maxn, __shfl_down_sync(0xffffffffu, maxn, off));
  }
  if (lane == 0 && wsegs) {
    atomicAdd(&a.ctr->segments_traced, wsegs);
    atomicAdd(&a.ctr->node_visits, wnodes);
    atomicAdd(&a.ctr->tri_tests, wtris);
    atomicMax(&a.ctr->max_seg_nodes, maxn);
  }
  if (ovf) {
    atomicAdd(&a.ctr->stack_overflow, 1u);
    atomicOr(&a.ctr->err, ERR_STACK);
  }
}

__global__ void __launch_bounds__(256) k_trace(TraceArgs a) {
  extern __shared__ int sstk[];
  TStack st;
  bind_stack(st, sstk, a.stack_cap);
  QFrame f{};
  trace_rays<false>(a, nullptr, f, st, kEmpty, kEmpty);
}

// The same with transmission (child rays, one launch per pass).
__global__ void __launch_bounds__(256) k_trace_t(TraceArgs a) {
  extern __shared__ int sstk[];
  TStack st;
  bind_stack(st, sstk, a.stack_cap);
  QFrame f{};
  trace_rays<false, false, true>(a, nullptr, f, st, kEmpty, kEmpty);
}

// ---------------------------------------------------------------------------
// several scenes in one launch
// ---------------------------------------------------------------------------
// Every scene's rays (its retrace queue in a coherent frame) in one
// persistent launch: the scenes' work is cut into chunks of 32 rays of one
// scene, a warp takes the next chunk from a counter shared by all scenes and
// traces its rays over that scene's binary trees (nodes from L2), with the
// same per-segment steps as trace_rays. A chunk's scene is found by a binary
// search over the chunk counts' prefix, formed by every CTA at its start.
__global__ void __launch_bounds__(256) k_trace_batch(const TraceArgs* __restrict__ tab, int n, unsigned* chunk_ctr) {
  extern __shared__ int sstk[];
  __shared__ unsigned pre[kMaxBatch + 1];  // pre[s]: chunks of the scenes before s
  TStack st;
  bind_stack(st, sstk, kStackTrace);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const TraceArgs& t = tab[i];
    unsigned nq = t.queue ? min(*t.nq_dev, (unsigned)t.R) : (unsigned)t.R;
    pre[i + 1] = (nq + 31u) >> 5;
  }
  if (threadIdx.x == 0) pre[0] = 0u;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 1; i <= n; ++i) pre[i] += pre[i - 1];
  __syncthreads();
  const unsigned total = pre[n];
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned c = 0;
    if (lane == 0) c = atomicAdd(chunk_ctr, 1u);
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c >= total) break;
    int lo = 0, hi = n;  // the scene s with pre[s] <= c < pre[s + 1]
    while (hi - lo > 1) {
      int m = (lo + hi) >> 1;
      if (pre[m] <= c) lo = m; else hi = m;
    }
    const TraceArgs& a = tab[lo];
    const Bvh bvh = a.bvh;
    const int R = a.R, N = a.N;
    [[maybe_unused]] const int LS = a.LS;  // bounds of the checked build
    const unsigned nq = a.queue ? min(*a.nq_dev, (unsigned)R) : (unsigned)R;
    const unsigned q = ((c - pre[lo]) << 5) + (unsigned)lane;
    int ray = -1, b = 0, last = -1;
    float3 o = f3(0.0f, 0.0f, 0.0f), d = o;
    float D = 0.0f;
    if (q < nq) {
      ray = a.queue ? a.queue[DCEM_IDX((int)q, R)] : (int)q;
      b = a.queue ? a.restart[DCEM_IDX(ray, R)] : 0;
      if (b == 0) {
        float4 rd = __ldg(&a.rays[DCEM_IDX(ray, R)]);
        float4 t4 = __ldg(&a.txs[DCEM_IDX(__float_as_int(rd.w), a.nsets)]);
        o = f3(t4.x, t4.y, t4.z);
        d = f3(rd.x, rd.y, rd.z);
      } else {
        float4 lo4 = a.log_o[log_at(a, b, ray)], ld = a.log_d[log_at(a, b, ray)];
        o = f3(lo4.x, lo4.y, lo4.z);
        D = lo4.w;
        d = f3(ld.x, ld.y, ld.z);
        last = a.log_id[log_at(a, b - 1, ray)];
      }
    }
    unsigned segs = 0, nodes = 0, tris = 0, ovf = 0, maxn = 0;
    while (__any_sync(0xffffffffu, ray >= 0)) {
      unsigned item = 0xffffffffu;
      if (ray >= 0) {
        RayPre rp = ray_pre(o, d);
        float t;
        int id;
        unsigned nn = 0, nt = 0;
        const int slot = closest_hit(bvh, rp, a.tmin, last, t, id, ovf, nn, nt, st);
        ++segs;
        nodes += nn;
        tris += nt;
        maxn = max(maxn, nn);
        const bool hit = slot >= 0;
        a.log_o[log_at(a, b, ray)] = make_float4(o.x, o.y, o.z, D);
        a.log_d[log_at(a, b, ray)] = make_float4(d.x, d.y, d.z, hit ? t : __int_as_float(0x7f800000));
        a.log_id[log_at(a, b, ray)] = hit ? id : -1;
        item = ((unsigned)ray << 4) | (unsigned)b;
        if (!hit || b == N) {
          a.nseg[DCEM_IDX(ray, LS)] = b + 1;
          ray = -1;
        } else {
          // specular reflection: d' = d - 2 (d.n)/(n.n) n, renormalised (as trace_rays)
          float3 v0, v1, v2;
          int tid;
          load_tri(bvh.tris, DCEM_IDX(slot, bvh.ntris), v0, v1, v2, tid);
          float3 nrm = cross3(sub3(v1, v0), sub3(v2, v0));
          float k = __fdiv_rn(__fmul_rn(2.0f, dot3(d, nrm)), dot3(nrm, nrm));
          float3 dr = f3(__fmaf_rn(-k, nrm.x, d.x), __fmaf_rn(-k, nrm.y, d.y), __fmaf_rn(-k, nrm.z, d.z));
          float inv = __fdiv_rn(1.0f, __fsqrt_rn(dot3(dr, dr)));
          o = f3(__fmaf_rn(t, d.x, o.x), __fmaf_rn(t, d.y, o.y), __fmaf_rn(t, d.z, o.z));
          d = f3(__fmul_rn(dr.x, inv), __fmul_rn(dr.y, inv), __fmul_rn(dr.z, inv));
          D = __fadd_rn(D, t);
          last = id;
          ++b;
        }
      }
      const unsigned logged = __ballot_sync(0xffffffffu, item != 0xffffffffu);
      if (logged) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(&a.ctr->n_capitems, (unsigned)__popc(logged));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (item != 0xffffffffu) a.capitems[DCEM_IDX(base + __popc(logged & ((1u << lane) - 1u)), capitems_cap(a))] = item;
      }
    }
    unsigned long long wsegs = segs, wnodes = nodes, wtris = tris;
    for (int off = 16; off > 0; off >>= 1) {
      wsegs += __shfl_down_sync(0xffffffffu, wsegs, off);
      wnodes += __shfl_down_sync(0xffffffffu, wnodes, off);
      wtris += __shfl_down_sync(0xffffffffu, wtris, off);
      maxn = max(maxn, __shfl_down_sync(0xffffffffu, maxn, off));
    }
    if (lane == 0 && wsegs) {
      atomicAdd(&a.ctr->segments_traced, wsegs);
      atomicAdd(&a.ctr->node_visits, wnodes);
      atomicAdd(&a.ctr->tri_tests, wtris);
      atomicMax(&a.ctr->max_seg_nodes, maxn);
    }
    if (__any_sync(0xffffffffu, ovf != 0u) && lane == 0) {
      atomicAdd(&a.ctr->stack_overflow, 1u);
      atomicOr(&a.ctr->err, ERR_STACK);
    }
  }
}

// Same traversal over the 4-wide compact node copy staged in shared memory
// (one CTA of kTraceQThreads threads per SM, the copy loaded once per CTA).
template <bool kT>
__device__ __forceinline__ void trace_q_body(const TraceArgs& a) {
  extern __shared__ uint4 sq[];
  TStack st;
  bind_stack(st, reinterpret_cast<int*>(sq + 4 * a.q4_bound), a.stack_cap);
  const int n4 = min(*a.q4_count, a.q4_bound);
  for (int i = threadIdx.x; i < 4 * n4; i += blockDim.x) sq[i] = a.qnodes[i];
  const int qr0 = a.q4_roots[0], qr1 = a.q4_roots[1];
  QFrame f;
  f.ox = a.qframe[0];
  f.oy = a.qframe[1];
  f.oz = a.qframe[2];
  f.sx = a.qframe[3];
  f.sy = a.qframe[4];
  f.sz = a.qframe[5];
  f.n4 = n4;
  __syncthreads();
  trace_rays<true, false, kT>(a, sq, f, st, qr0, qr1);
}

__global__ void __launch_bounds__(kTraceQThreads, 1) k_trace_q(TraceArgs a) { trace_q_body<false>(a); }
__global__ void __launch_bounds__(kTraceQThreads, 1) k_trace_qt(TraceArgs a) { trace_q_body<true>(a); }

// The 4-wide compact copy read from global memory (L2), for scenes whose copy
// does not fit in shared memory; stacks in shared memory.
__global__ void __launch_bounds__(256, 3) k_trace_qg(TraceArgs a) {
  extern __shared__ int sstk[];
  TStack st;
  bind_stack(st, sstk, a.stack_cap);
  const int qr0 = a.q4_roots[0], qr1 = a.q4_roots[1];
  QFrame f;
  f.ox = a.qframe[0];
  f.oy = a.qframe[1];
  f.oz = a.qframe[2];
  f.sx = a.qframe[3];
  f.sy = a.qframe[4];
  f.sz = a.qframe[5];
  f.n4 = min(*a.q4_count, a.q4_bound);
  trace_rays<true, true>(a, a.qnodes, f, st, qr0, qr1);
}

// Reception-sphere captures of the segments in the frame's capture list: the
// segments traced this frame (appended by the closest-hit kernel in tracing
// order, so a warp reads segments of neighbouring rays) and, in a coherent
// frame, the reused segments (appended by k_mark), which only the receivers
// that moved need to test.
// Receivers and their tree copied to shared memory after the stacks (kS).
__device__ __forceinline__ char* stage_receivers(const TraceArgs& a, char* p, const float4*& rx, SmallBvh& rxt) {
  float4* srx = reinterpret_cast<float4*>(p);
  for (int i = threadIdx.x; i < a.nrx; i += blockDim.x) srx[i] = a.rx[i];
  rx = srx;
  return stage_tree(a.rxt, max(a.nrx - 1, 0), a.nrx, reinterpret_cast<char*>(srx + a.nrx), rxt);
}

template <bool kS>
__global__ void __launch_bounds__(256) k_capture(TraceArgs a) {
  extern __shared__ __align__(16) int sstk[];
  TStack st;
  bind_stack(st, sstk, kStackSmall);
  SmallBvh rxt = a.rxt;
  const float4* rx = a.rx;
  if (kS) {
    stage_receivers(a, reinterpret_cast<char*>(sstk + blockDim.x * kStackSmall), rx, rxt);
    __syncthreads();
  }
  const int R = a.R, LS = a.LS;
  const unsigned total = min(a.ctr->n_capitems, (unsigned)LS * (unsigned)(a.N + a.max_trans + 1));
  unsigned ovf = 0;
  for (;;) {
    int base = fetch_warp(&a.ctr->work_capture, 32u);
    if ((unsigned)base >= total) break;
    unsigned q = (unsigned)base + (threadIdx.x & 31);
    if (q < total) {
      unsigned it = a.capitems[q];
      bool reused = (it & 0x80000000u) != 0u;
      int ray = (int)((it & 0x7fffffffu) >> 4), b = (int)(it & 15u);
      float4 lo = a.log_o[log_at(a, b, ray)], ld = a.log_d[log_at(a, b, ray)];
      float3 o = f3(lo.x, lo.y, lo.z), d = f3(ld.x, ld.y, ld.z);
      float D = lo.w, t = ld.w;
      float tend = isinf(t) ? a.escape : t;
      // the ray's set: its capture spacing, and the link of its captures
      // (a transmission child: its parent's)
      int set = ray >= R ? (a.inst[DCEM_IDX(ray - R, a.child_cap)] >> 8)
                         : a.nsets > 1 ? __float_as_int(__ldg(reinterpret_cast<const float*>(a.rays) + 4 * (size_t)ray + 3))
                                       : 0;
      float alpha = __ldg(&a.txs[DCEM_IDX(set, a.nsets)].w);
      int link0 = set * a.nrx;
      RayPre rp;
      rp.o = o;
      float dx = fabsf(d.x) < 1e-30f ? copysignf(1e-30f, d.x) : d.x;
      float dy = fabsf(d.y) < 1e-30f ? copysignf(1e-30f, d.y) : d.y;
      float dz = fabsf(d.z) < 1e-30f ? copysignf(1e-30f, d.z) : d.z;
      rp.inv = f3(__fdiv_rn(1.0f, dx), __fdiv_rn(1.0f, dy), __fdiv_rn(1.0f, dz));
      if (!capture_tree(rxt, rx, rp, d, D, tend, alpha, st, [&](int r) {
            if (!reused || a.rx_moved[r]) emit_cand(a, ray, b, link0 + r);
          }))
        ovf = 1u;
    }
    __syncwarp();
  }
  if (ovf) {
    atomicAdd(&a.ctr->stack_overflow, 1u);
    atomicOr(&a.ctr->err, ERR_STACK);
  }
}

// ---------------------------------------------------------------------------
// coherent frame: marking and carry-over
// ---------------------------------------------------------------------------
// Restart points: for every ray the first logged segment that meets a moved
// box; earlier segments are reused and, when receivers moved, appended to the
// capture list (flagged reused), and rays with a restart point go to the
// retrace queue. One thread per ray; each warp takes a static stride of
// 32-ray batches (a work counter measured slower: its round trip and the
// order in which it hands out batches cost more than the balance gains). The
// kernel is bound by memory round trips, so each batch makes few of them:
// segment 0 (every ray has one) comes with the segment count, and the
// batch's appends to the capture list and to the queue take one atomic each,
// issued together. The appended segments are ordered by segment index within
// the batch, so that consecutive capture threads read neighbouring rays.
template <bool kS>
__global__ void __launch_bounds__(256) k_mark(TraceArgs a, CoherentArgs c) {
  extern __shared__ __align__(16) int sstk[];
  TStack st;
  bind_stack(st, sstk, kStackSmall);
  SmallBvh mvt = c.mvt;
  // more moved boxes than the per-frame tree holds: retrace everything
  const unsigned nmb = c.ctr->n_moved_boxes;
  const bool all = nmb > (unsigned)c.mv_cap;
  if (kS) {
    stage_tree(c.mvt, all ? 0 : max((int)nmb - 1, 0), 0, reinterpret_cast<char*>(sstk + blockDim.x * kStackSmall),
               mvt);
    __syncthreads();
  }
  const bool any_rx = c.ctr->rx_moved > 0;
  const int R = a.R, N = a.N;
  [[maybe_unused]] const int LS = a.LS;  // bounds of the checked build
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  unsigned long long reused = 0;
  constexpr int kPre = 5;  // segments held in registers (later ones are loaded when tested)
  const long nwarps = (long)((gridDim.x * blockDim.x) >> 5);
  for (long b0 = (long)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; b0 < R; b0 += 32 * nwarps) {
    const int base = (int)b0;
    const int ray = base + lane;
    const bool in = ray < R;
    float4 plo[kPre], pld[kPre];
#pragma unroll
    for (int b = 0; b < kPre; ++b) plo[b] = pld[b] = make_float4(0.f, 0.f, 0.f, 0.f);
    int ns = 0;
    if (in) {
      ns = a.nseg[ray];
      plo[0] = a.log_o[log_at(a, 0, ray)];
      pld[0] = a.log_d[log_at(a, 0, ray)];
    }
    const int lim = all ? 0 : ns;
#pragma unroll
    for (int b = 1; b < kPre; ++b) {
      if (b < lim) {
        plo[b] = a.log_o[log_at(a, b, ray)];
        pld[b] = a.log_d[log_at(a, b, ray)];
      }
    }
    // restart point: the first segment that meets a moved box (ns if none)
    int bstar = lim;
    auto test = [&](int b, float4 lo, float4 ld) {
      RayPre rp;
      rp.o = f3(lo.x, lo.y, lo.z);
      float dx = fabsf(ld.x) < 1e-30f ? copysignf(1e-30f, ld.x) : ld.x;
      float dy = fabsf(ld.y) < 1e-30f ? copysignf(1e-30f, ld.y) : ld.y;
      float dz = fabsf(ld.z) < 1e-30f ? copysignf(1e-30f, ld.z) : ld.z;
      rp.inv = f3(__fdiv_rn(1.0f, dx), __fdiv_rn(1.0f, dy), __fdiv_rn(1.0f, dz));
      if (seg_hits_tree(mvt, rp, ld.w, st)) bstar = b;
    };
#pragma unroll
    for (int b = 0; b < kPre; ++b)
      if (b < bstar) test(b, plo[b], pld[b]);
    for (int b = kPre; b < bstar; ++b) test(b, a.log_o[log_at(a, b, ray)], a.log_d[log_at(a, b, ray)]);
    // the batch's reused segments (when receivers moved) and retraced rays
    const int nitem = any_rx ? bstar : 0;
    unsigned tot = (unsigned)nitem;
    for (int off = 16; off > 0; off >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, off);
    const bool rq = in && bstar < ns;
    const unsigned qmask = __ballot_sync(0xffffffffu, rq);
    unsigned at = 0, aq = 0;
    if (lane == 0) {
      if (tot) at = atomicAdd(&c.ctr->n_capitems, tot);
      if (qmask) aq = atomicAdd(&c.ctr->n_retrace, (unsigned)__popc(qmask));
    }
    at = __shfl_sync(0xffffffffu, at, 0);
    aq = __shfl_sync(0xffffffffu, aq, 0);
    if (tot) {
      for (int b = 0; b <= N; ++b) {
        unsigned m = __ballot_sync(0xffffffffu, b < nitem);
        if (!m) break;
        if (b < nitem)
          a.capitems[DCEM_IDX(at + __popc(m & lt), capitems_cap(a))] = 0x80000000u | ((unsigned)ray << 4) | (unsigned)b;
        at += (unsigned)__popc(m);
      }
    }
    if (rq) a.queue_w[DCEM_IDX(aq + __popc(qmask & lt), R)] = ray;
    if (in) {
      c.restart[ray] = bstar;
      reused += (unsigned long long)bstar;
    }
  }
  for (int off = 16; off > 0; off >>= 1) reused += __shfl_down_sync(0xffffffffu, reused, off);
  if (lane == 0 && reused) atomicAdd(&c.ctr->segments_reused, reused);
}

// Previous frame's captures by receivers that did not move, from segments
// that are reused.
__global__ void k_carry(TraceArgs a, CoherentArgs c) {
  unsigned n = min(*c.prev_ncand, c.prev_cap);
  unsigned kept = 0;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    Cand x = c.prev_cand[i];
    int l = cand_rx(x), s = cand_seg(x);
    int r = a.nsets > 1 ? l % a.nrx : l;   // link -> receiver
    if (s < c.restart[DCEM_IDX(x.ray, a.R)] && !c.rx_moved[DCEM_IDX(r, a.nrx)]) {
      emit_cand(a, x.ray, s, l);
      ++kept;
    }
  }
  for (int off = 16; off > 0; off >>= 1) kept += __shfl_down_sync(0xffffffffu, kept, off);
  if ((threadIdx.x & 31) == 0 && kept) atomicAdd(&c.ctr->n_cand_reused, kept);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int grid_for(long n, int bs, int max_blocks) {
  long b = (n + bs - 1) / bs;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

// Persistent launches: as many 256-thread blocks as fit on the GPU at once.
static int resident_blocks(const void* fn, int sms, size_t smem, int block = 256) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, smem) != cudaSuccess || nb < 1) nb = 1;
  return nb * sms;
}

int trace_q_stack_cap(int n_nodes) {
  long avail = kTraceQSmem - (long)bvh4_bound(n_nodes) * 4 * (long)sizeof(uint4);
  int cap = avail > 0 ? (int)std::min<long>(kStackTrace, avail / (kTraceQThreads * (long)sizeof(int))) : 0;
  return (n_nodes > 0 && cap >= 12) ? cap : 0;
}

cudaError_t launch_trace(const TraceArgs& a, int sms, cudaStream_t st) {
  long n = a.R;
  const bool tr = a.max_trans > 0;
  if (a.use_q != 1) {
    // kernels 0 and 2: a.block threads, a.stack_cap shared stack entries per
    // thread; resident CTAs per SM looked up once per configuration.
    // Transmission uses the binary-node kernel with child rays (slot 3).
    static int key[4] = {-1, -1, -1, -1}, resident[4] = {0, 0, 0, 0};
    const int v = tr ? 3 : a.use_q;
    const void* fn = v == 3 ? (const void*)k_trace_t : v == 2 ? (const void*)k_trace_qg : (const void*)k_trace;
    size_t smem = (size_t)a.block * a.stack_cap * sizeof(int);
    int k = a.block * 64 + a.stack_cap;
    if (key[v] != k) {
      resident[v] = resident_blocks(fn, sms, smem, a.block);
      key[v] = k;
    }
    if (v == 3) k_trace_t<<<grid_for(n, a.block, resident[3]), a.block, smem, st>>>(a);
    else if (v == 2) k_trace_qg<<<grid_for(n, a.block, resident[2]), a.block, smem, st>>>(a);
    else k_trace<<<grid_for(n, a.block, resident[0]), a.block, smem, st>>>(a);
  } else {
    size_t smem = (size_t)a.q4_bound * 4 * sizeof(uint4) + (size_t)kTraceQThreads * a.stack_cap * sizeof(int);
    static size_t attr[2] = {0, 0};
    const void* fn = tr ? (const void*)k_trace_qt : (const void*)k_trace_q;
    if (smem > attr[tr]) {
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr[tr] = smem;
    }
    if (tr) k_trace_qt<<<grid_for(n, kTraceQThreads, sms), kTraceQThreads, smem, st>>>(a);
    else k_trace_q<<<grid_for(n, kTraceQThreads, sms), kTraceQThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_trace_batch(const TraceArgs* d_tab, int n, unsigned* chunk_ctr, int sms, cudaStream_t st) {
  static int resident = 0;
  size_t smem = 256 * (size_t)kStackTrace * sizeof(int);
  if (!resident) resident = resident_blocks((const void*)k_trace_batch, sms, smem);
  k_trace_batch<<<resident, 256, smem, st>>>(d_tab, n, chunk_ctr);
  return cudaGetLastError();
}

// Shared memory of the capture and marking kernels: stacks, plus the
// receivers, their tree and (marking) the moved-box tree when these fit.
static size_t rx_stage_bytes(int nrx) { return (size_t)nrx * 16 + stage_bytes(nrx > 1 ? nrx - 1 : 0, nrx); }
constexpr size_t kStageLimit = 96 * 1024;

static cudaError_t allow_smem(const void* fn, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_capture(const TraceArgs& a, int sms, cudaStream_t st) {
  size_t base = 256 * kStackSmall * sizeof(int);
  size_t staged = base + rx_stage_bytes(a.nrx);
  bool kS = a.nrx <= 1024 && staged <= kStageLimit;
  const void* fn = kS ? (const void*)k_capture<true> : (const void*)k_capture<false>;
  size_t smem = kS ? staged : base;
  cudaError_t e = allow_smem(fn, smem);
  if (e != cudaSuccess) return e;
  int blocks = grid_for((long)a.LS * (a.N + a.max_trans + 1), 256, resident_blocks(fn, sms, smem));
  if (kS) k_capture<true><<<blocks, 256, smem, st>>>(a);
  else k_capture<false><<<blocks, 256, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mark(const TraceArgs& a, const CoherentArgs& c, int sms, cudaStream_t st) {
  size_t base = 256 * kStackSmall * sizeof(int);
  size_t staged = base + stage_bytes(c.mv_cap > 1 ? c.mv_cap - 1 : 0, 0);
  bool kS = staged <= kStageLimit;
  size_t smem = kS ? staged : base;
  cudaError_t e = allow_smem(kS ? (const void*)k_mark<true> : (const void*)k_mark<false>, smem);
  if (e != cudaSuccess) return e;
  // one wave of resident blocks (each stages the moved-box tree once)
  static size_t key = 0;
  static int resident = 0;
  const void* fn = kS ? (const void*)k_mark<true> : (const void*)k_mark<false>;
  if (key != smem + kS) {
    resident = resident_blocks(fn, sms, smem);
    key = smem + kS;
  }
  int blocks = grid_for(a.R, 256, resident);
  if (kS) k_mark<true><<<blocks, 256, smem, st>>>(a, c);
  else k_mark<false><<<blocks, 256, smem, st>>>(a, c);
  return cudaGetLastError();
}

cudaError_t launch_carry(const TraceArgs& a, const CoherentArgs& c, cudaStream_t st) {
  k_carry<<<grid_for(c.prev_cap, 256, 1024), 256, 0, st>>>(a, c);
  return cudaGetLastError();
}

DCEM_CHECKS_TAKER(checks_take_trace)

}  // namespace dcem
