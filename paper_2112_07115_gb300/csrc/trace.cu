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

namespace dcem {

// ---------------------------------------------------------------------------
// per-segment kernel body shared by full and coherent frames
// ---------------------------------------------------------------------------
__device__ __forceinline__ void emit_cand(const TraceArgs& a, int ray, int seg, int rx) {
  unsigned idx = atomicAdd(&a.ctr->n_cand, 1u);
  if (idx < a.cand_cap) a.cand[idx] = Cand{ray, (rx << 4) | seg};
  else atomicOr(&a.ctr->err, ERR_CAND_OVERFLOW);
}

__device__ __forceinline__ float3 rx_at(const float4* srx, const float4* __restrict__ grx, int r) {
  float4 v = r < kRxSmem ? srx[r] : __ldg(&grx[r]);
  return f3(v.x, v.y, v.z);
}

__global__ void __launch_bounds__(256) k_trace(TraceArgs a) {
  extern __shared__ float4 srx[];
  int nsm = a.nrx < kRxSmem ? a.nrx : kRxSmem;
  for (int r = threadIdx.x; r < nsm; r += blockDim.x) srx[r] = a.rx[r];
  __syncthreads();
  const int R = a.R;
  int nq = a.queue ? (int)min(*a.nq_dev, (unsigned)R) : R;
  unsigned long long segs = 0;
  unsigned ovf = 0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    int ray = a.queue ? a.queue[q] : q;
    int b0 = a.queue ? a.restart[ray] : 0;
    float3 o, d;
    float D;
    int last;
    if (b0 == 0) {
      float4 rd = __ldg(&a.rays[ray]);
      o = a.tx;
      d = f3(rd.x, rd.y, rd.z);
      D = 0.0f;
      last = -1;
    } else {
      float4 lo = a.log_o[(size_t)b0 * R + ray], ld = a.log_d[(size_t)b0 * R + ray];
      o = f3(lo.x, lo.y, lo.z);
      D = lo.w;
      d = f3(ld.x, ld.y, ld.z);
      last = a.log_id[(size_t)(b0 - 1) * R + ray];
    }
    int b = b0;
    for (; b <= a.N; ++b) {
      RayPre rp = ray_pre(o, d);
      float t;
      int id;
      int slot = closest_hit(a.bvh, rp, a.tmin, last, t, id, ovf);
      ++segs;
      bool hit = slot >= 0;
      float tend = hit ? t : a.escape;
      a.log_o[(size_t)b * R + ray] = make_float4(o.x, o.y, o.z, D);
      a.log_d[(size_t)b * R + ray] = make_float4(d.x, d.y, d.z, hit ? t : __int_as_float(0x7f800000));
      a.log_id[(size_t)b * R + ray] = hit ? id : -1;
      for (int r = 0; r < a.nrx; ++r)
        if (captured(o, d, D, tend, a.alpha_eff, rx_at(srx, a.rx, r))) emit_cand(a, ray, b, r);
      if (!hit) break;
      // specular reflection: d' = d - 2 (d.n)/(n.n) n, renormalised
      float3 v0, v1, v2;
      int tid;
      load_tri(a.bvh.tris, slot, v0, v1, v2, tid);
      float3 n = cross3(sub3(v1, v0), sub3(v2, v0));
      float k = __fdiv_rn(__fmul_rn(2.0f, dot3(d, n)), dot3(n, n));
      float3 dr = f3(__fmaf_rn(-k, n.x, d.x), __fmaf_rn(-k, n.y, d.y), __fmaf_rn(-k, n.z, d.z));
      float inv = __fdiv_rn(1.0f, __fsqrt_rn(dot3(dr, dr)));
      o = f3(__fmaf_rn(t, d.x, o.x), __fmaf_rn(t, d.y, o.y), __fmaf_rn(t, d.z, o.z));
      d = f3(__fmul_rn(dr.x, inv), __fmul_rn(dr.y, inv), __fmul_rn(dr.z, inv));
      D = __fadd_rn(D, t);
      last = id;
    }
    a.nseg[ray] = (b > a.N ? a.N : b) + 1;
  }
  // block totals
  for (int off = 16; off > 0; off >>= 1) segs += __shfl_down_sync(0xffffffffu, segs, off);
  if ((threadIdx.x & 31) == 0 && segs) atomicAdd(&a.ctr->segments_traced, segs);
  if (ovf) {
    atomicAdd(&a.ctr->stack_overflow, 1u);
    atomicOr(&a.ctr->err, ERR_STACK);
  }
}

// ---------------------------------------------------------------------------
// coherent frame: moved objects and receivers
// ---------------------------------------------------------------------------
// One thread per object: compares its transform with the cached frame's,
// and for a moved object appends its old and new world boxes (widened by a
// safety margin) to the moved-box list.
__global__ void k_moved_objects(CoherentArgs c) {
  for (int ob = blockIdx.x * blockDim.x + threadIdx.x; ob < c.nobj; ob += gridDim.x * blockDim.x) {
    bool moved = false;
    for (int k = 0; k < 12; ++k)
      moved = moved || (__float_as_uint(c.xf_cur[12 * ob + k]) != __float_as_uint(c.xf_traced[12 * ob + k]));
    if (!moved) continue;
    atomicAdd(&c.ctr->objects_moved, 1u);
    const unsigned* boxes[2] = {c.obj_box_traced, c.obj_box_cur};
    float bx[2][6];
    bool ok[2];
    for (int q = 0; q < 2; ++q) {
      ok[q] = true;
      for (int k = 0; k < 3; ++k) {
        float lo = o2f(boxes[q][3 * (size_t)ob + k]);
        float hi = o2f(boxes[q][3 * (size_t)(c.nobj + ob) + k]);
        ok[q] = ok[q] && (lo <= hi);   // false for an object without triangles
        float m = 1e-3f + 1e-5f * fmaxf(fabsf(lo), fabsf(hi));
        bx[q][k] = lo - m;
        bx[q][k + 3] = hi + m;
      }
    }
    unsigned nq = (ok[0] ? 1u : 0u) + (ok[1] ? 1u : 0u);
    if (!nq) continue;
    unsigned at = atomicAdd(&c.ctr->n_moved_boxes, nq);
    for (int q = 0; q < 2; ++q) {
      if (!ok[q]) continue;
      float* out = c.moved_boxes + 6 * (size_t)at++;
      for (int k = 0; k < 6; ++k) out[k] = bx[q][k];
    }
  }
}

// Receivers: pack to float4, check finiteness, flag the ones that moved.
__global__ void k_rx_pack(const float* __restrict__ rx3, int nrx, float4* rx_cur, const float4* rx_traced,
                          int have_prev, unsigned char* moved, int* moved_list, DevCounters* ctr) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrx; r += gridDim.x * blockDim.x) {
    float x = rx3[3 * r], y = rx3[3 * r + 1], z = rx3[3 * r + 2];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) atomicOr(&ctr->err, ERR_NONFINITE);
    float4 v = make_float4(x, y, z, 0.0f);
    rx_cur[r] = v;
    bool mv = true;
    if (have_prev) {
      float4 p = rx_traced[r];
      mv = __float_as_uint(p.x) != __float_as_uint(x) || __float_as_uint(p.y) != __float_as_uint(y) ||
           __float_as_uint(p.z) != __float_as_uint(z);
    }
    moved[r] = mv ? 1 : 0;
    if (mv) {
      unsigned at = atomicAdd(&ctr->rx_moved, 1u);
      moved_list[at] = r;
    }
  }
}

// One thread per ray: the first logged segment that meets a moved box is the
// restart point; earlier segments are reused and re-tested against the
// receivers that moved.
__global__ void __launch_bounds__(256) k_mark(TraceArgs a, CoherentArgs c) {
  extern __shared__ float4 smem4[];
  // shared layout: c.smem_rx moved receivers (float4), their indices, then
  // up to c.smem_boxes moved boxes (6 floats each)
  int nb = (int)min(c.ctr->n_moved_boxes, (unsigned)c.smem_boxes);
  int nmr = (int)min(c.ctr->rx_moved, (unsigned)c.smem_rx);
  float4* smr = smem4;
  int* smi = reinterpret_cast<int*>(smr + c.smem_rx);
  float* sbox = reinterpret_cast<float*>(smi + c.smem_rx);
  for (int i = threadIdx.x; i < 6 * nb; i += blockDim.x) sbox[i] = c.moved_boxes[i];
  for (int i = threadIdx.x; i < nmr; i += blockDim.x) {
    int r = c.moved_list[i];
    smi[i] = r;
    smr[i] = a.rx[r];
  }
  __syncthreads();
  int nb_all = (int)c.ctr->n_moved_boxes, nmr_all = (int)c.ctr->rx_moved;
  const int R = a.R;
  unsigned long long reused = 0;
  for (int ray = blockIdx.x * blockDim.x + threadIdx.x; ray < R; ray += gridDim.x * blockDim.x) {
    int ns = a.nseg[ray];
    int bstar = ns;
    for (int b = 0; b < ns; ++b) {
      float4 lo = a.log_o[(size_t)b * R + ray], ld = a.log_d[(size_t)b * R + ray];
      float3 o = f3(lo.x, lo.y, lo.z), d = f3(ld.x, ld.y, ld.z);
      float D = lo.w, t = ld.w;
      RayPre rp;
      rp.o = o;
      float dx = fabsf(d.x) < 1e-30f ? copysignf(1e-30f, d.x) : d.x;
      float dy = fabsf(d.y) < 1e-30f ? copysignf(1e-30f, d.y) : d.y;
      float dz = fabsf(d.z) < 1e-30f ? copysignf(1e-30f, d.z) : d.z;
      rp.inv = f3(__fdiv_rn(1.0f, dx), __fdiv_rn(1.0f, dy), __fdiv_rn(1.0f, dz));
      bool hitbox = false;
      for (int k = 0; k < nb_all && !hitbox; ++k)
        hitbox = seg_box(rp, t, k < nb ? sbox + 6 * k : c.moved_boxes + 6 * (size_t)k);
      if (hitbox) { bstar = b; break; }
      float tend = isinf(t) ? a.escape : t;
      for (int m = 0; m < nmr_all; ++m) {
        int r = m < nmr ? smi[m] : c.moved_list[m];
        float4 rv = m < nmr ? smr[m] : a.rx[r];
        if (captured(o, d, D, tend, a.alpha_eff, f3(rv.x, rv.y, rv.z))) emit_cand(a, ray, b, r);
      }
    }
    c.restart[ray] = bstar;
    reused += (unsigned long long)bstar;
    if (bstar < ns) {
      unsigned at = atomicAdd(&c.ctr->n_retrace, 1u);
      a.queue_w[at] = ray;
    }
  }
  for (int off = 16; off > 0; off >>= 1) reused += __shfl_down_sync(0xffffffffu, reused, off);
  if ((threadIdx.x & 31) == 0 && reused) atomicAdd(&c.ctr->segments_reused, reused);
}

// Previous frame's captures by receivers that did not move, from segments
// that are reused.
__global__ void k_carry(TraceArgs a, CoherentArgs c) {
  unsigned n = min(*c.prev_ncand, c.prev_cap);
  unsigned kept = 0;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    Cand x = c.prev_cand[i];
    int r = cand_rx(x), s = cand_seg(x);
    if (s < c.restart[x.ray] && !c.rx_moved[r]) {
      emit_cand(a, x.ray, s, r);
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

cudaError_t launch_trace(const TraceArgs& a, int grid_cap, cudaStream_t st) {
  int nsm = a.nrx < kRxSmem ? a.nrx : kRxSmem;
  size_t smem = (size_t)nsm * sizeof(float4);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_trace, cudaFuncAttributeMaxDynamicSharedMemorySize, kRxSmem * 16);
    attr = true;
  }
  long n = a.R;
  k_trace<<<grid_for(n, 256, grid_cap), 256, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_coherent_prep(const CoherentArgs& c, cudaStream_t st) {
  if (c.nobj > 0) k_moved_objects<<<grid_for(c.nobj, 128, 1024), 128, 0, st>>>(c);
  return cudaGetLastError();
}

cudaError_t launch_rx_pack(const float* d_rx3, int nrx, float4* rx_cur, const float4* rx_traced,
                           int have_prev, unsigned char* moved, int* moved_list, DevCounters* ctr,
                           cudaStream_t st) {
  if (nrx > 0)
    k_rx_pack<<<grid_for(nrx, 256, 1024), 256, 0, st>>>(d_rx3, nrx, rx_cur, rx_traced, have_prev, moved,
                                                         moved_list, ctr);
  return cudaGetLastError();
}

cudaError_t launch_mark(const TraceArgs& a, const CoherentArgs& c, int grid_cap, cudaStream_t st) {
  size_t smem = (size_t)c.smem_rx * (sizeof(float4) + sizeof(int)) + (size_t)6 * c.smem_boxes * sizeof(float);
  static bool attr = false;
  if (!attr) {
    size_t mx = (size_t)kRxSmem * (sizeof(float4) + sizeof(int)) + (size_t)6 * kMovedSmem * sizeof(float);
    cudaFuncSetAttribute(k_mark, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
    attr = true;
  }
  k_mark<<<grid_for(a.R, 256, grid_cap), 256, smem, st>>>(a, c);
  return cudaGetLastError();
}

cudaError_t launch_carry(const TraceArgs& a, const CoherentArgs& c, cudaStream_t st) {
  k_carry<<<grid_for(c.prev_cap, 256, 1024), 256, 0, st>>>(a, c);
  return cudaGetLastError();
}

}  // namespace dcem
