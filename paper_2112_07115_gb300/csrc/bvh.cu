// bvh.cu -- LBVH construction (once per scene) and per-frame update.
//
// Sec. III "Efficient BVH updating": the hierarchy over the scene is built
// once and updated (refit) every frame instead of rebuilt. Construction is a
// linear BVH: 30-bit Morton codes of primitive centroids, a stable sort, and
// the binary radix tree of Karras (HPG 2012) over the (code, index) keys. One
// primitive per leaf. The refit walks bottom-up; the second child to arrive at
// a node (atomic counter) unions the two child boxes and continues, so every
// box is the exact min/max of its leaves' FP32 vertices.
//
// Per frame, the moving objects' vertices are transformed
// (fmaf(R0,x, fmaf(R1,y, fmaf(R2,z,t))) per row) inside the refit kernel.
#include "bvh.cuh"

namespace dcem {

// ---------------------------------------------------------------------------
// Morton codes
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned expand_bits10(unsigned v) {
  v = (v * 0x00010001u) & 0xFF0000FFu;
  v = (v * 0x00000101u) & 0x0F00F00Fu;
  v = (v * 0x00000011u) & 0xC30C30C3u;
  v = (v * 0x00000005u) & 0x49249249u;
  return v;
}

__device__ __forceinline__ unsigned morton30(float cx, float cy, float cz, const float* lo,
                                             const float* ext_inv) {
  float q[3] = {(cx - lo[0]) * ext_inv[0], (cy - lo[1]) * ext_inv[1], (cz - lo[2]) * ext_inv[2]};
  unsigned b[3];
  for (int k = 0; k < 3; ++k) {
    float f = fminf(fmaxf(q[k] * 1024.0f, 0.0f), 1023.0f);
    b[k] = (unsigned)f;
  }
  return (expand_bits10(b[0]) << 2) | (expand_bits10(b[1]) << 1) | expand_bits10(b[2]);
}

__device__ __forceinline__ int delta64(const unsigned long long* k, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  return __clzll(k[i] ^ k[j]);
}

// Karras' radix-tree node i over n sorted unique keys. Writes child codes
// (internal: node_base + c, leaf: ~(leaf_base + c)) and parents.
__device__ __forceinline__ void karras_node(const unsigned long long* k, int n, int i, int node_base,
                                            int leaf_base, float4* nodes, int* leaf_parent) {
  int d = (delta64(k, n, i, i + 1) - delta64(k, n, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = delta64(k, n, i, i - d);
  int lmax = 2;
  while (delta64(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta64(k, n, i, i + (l + t) * d) > dmin) l += t;
  int j = i + l * d;
  int dnode = delta64(k, n, i, j);
  int s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (delta64(k, n, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  int g = i + s * d + (d < 0 ? d : 0);
  int lo = i < j ? i : j, hi = i < j ? j : i;
  int c0 = (lo == g) ? ~(leaf_base + g) : node_base + g;
  int c1 = (hi == g + 1) ? ~(leaf_base + g + 1) : node_base + g + 1;
  float4* nd = nodes + 4 * (size_t)(node_base + i);
  int4 n3 = make_int4(c0, c1, -1, 0);
  // parent of node i is written by its parent; keep the slot's current parent
  int* n3i = reinterpret_cast<int*>(&nd[3]);
  n3i[0] = n3.x;
  n3i[1] = n3.y;
  if (c0 >= 0) reinterpret_cast<int*>(nodes + 4 * (size_t)c0 + 3)[2] = node_base + i;
  else leaf_parent[~c0] = node_base + i;
  if (c1 >= 0) reinterpret_cast<int*>(nodes + 4 * (size_t)c1 + 3)[2] = node_base + i;
  else leaf_parent[~c1] = node_base + i;
}

// Store box b (lo.xyz, hi.xyz) into the child slot `side` of node p.
__device__ __forceinline__ void put_child_box(float4* nodes, int p, int side, const float* b) {
  float* n = reinterpret_cast<float*>(nodes + 4 * (size_t)p);
  // n0 = c0 x/y, n1 = c1 x/y, n2 = (c0.z lo/hi, c1.z lo/hi)
  float* xy = n + (side ? 4 : 0);
  xy[0] = b[0]; xy[1] = b[3]; xy[2] = b[1]; xy[3] = b[4];
  n[8 + 2 * side] = b[2];
  n[8 + 2 * side + 1] = b[5];
}

__device__ __forceinline__ void get_union_cg(const float4* nodes, int p, float* u) {
  const float4* n = nodes + 4 * (size_t)p;
  float4 n0 = __ldcg(n), n1 = __ldcg(n + 1), n2 = __ldcg(n + 2);
  u[0] = fminf(n0.x, n1.x); u[3] = fmaxf(n0.y, n1.y);
  u[1] = fminf(n0.z, n1.z); u[4] = fmaxf(n0.w, n1.w);
  u[2] = fminf(n2.x, n2.z); u[5] = fmaxf(n2.y, n2.w);
}

__device__ __forceinline__ int node_parent_cg(const float4* nodes, int p) {
  return __float_as_int(__ldcg(reinterpret_cast<const float*>(nodes + 4 * (size_t)p + 3) + 2));
}

__device__ __forceinline__ int node_side(const float4* nodes, int p, int code) {
  int c0 = __float_as_int(__ldcg(reinterpret_cast<const float*>(nodes + 4 * (size_t)p + 3)));
  return c0 == code ? 0 : 1;
}

// Bottom-up propagation from a finished child (code, box) at parent p, with
// atomic arrival counters: the second arrival at a node unions its two child
// boxes and continues. Returns when it is the first arrival or after the root.
__device__ __forceinline__ void refit_up(float4* nodes, int* arrive, int node_base, int p, int code,
                                         const float* box, float* root_box) {
  float b[6] = {box[0], box[1], box[2], box[3], box[4], box[5]};
  if (p < 0) {
    for (int k = 0; k < 6; ++k) root_box[k] = b[k];
    return;
  }
  for (int depth = 0; depth < 128; ++depth) {  // LBVH depth <= 64
    put_child_box(nodes, p, node_side(nodes, p, code), b);
    __threadfence();
    int old = atomicAdd(&arrive[p - node_base], 1);
    if (old == 0) return;
    __threadfence();
    get_union_cg(nodes, p, b);
    int pp = node_parent_cg(nodes, p);
    if (pp < 0) {
      for (int k = 0; k < 6; ++k) root_box[k] = b[k];
      return;
    }
    code = p;
    p = pp;
  }
}

// ---------------------------------------------------------------------------
// one-CTA builder: n <= kSmallBuild primitives given as boxes (lo.xyz, hi.xyz)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float box_area(const float* b) {
  float ex = b[3] - b[0], ey = b[4] - b[1], ez = b[5] - b[2];
  return 2.0f * (ex * ey + ey * ez + ez * ex);
}

// Topology of the tree over n primitive boxes: Morton codes of the centroids,
// bitonic sort of (code, index) in shared memory, Karras nodes. Called by all
// threads of one CTA; `keys` holds the next power of two >= n 64-bit keys.
// Leaves the leaf order in perm, child codes and parents in the global
// nodes, and the root code; for n == 1 also the root box.
__device__ void sort_karras_dev(const float* __restrict__ prim, int n, int node_base, int leaf_base,
                                float4* nodes, int* leaf_parent, int* perm, int* root_out, float* root_box,
                                unsigned long long* keys) {
  __shared__ float red[6][32];
  __shared__ float bnd[6];
  int tid = threadIdx.x, nt = blockDim.x;
  if (n <= 0) {
    if (tid == 0) root_out[0] = kEmpty;
    return;
  }
  float lo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, hi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
  for (int i = tid; i < n; i += nt) {
    const float* b = prim + 6 * (size_t)i;
    for (int k = 0; k < 3; ++k) {
      float c = 0.5f * (b[k] + b[k + 3]);
      lo[k] = fminf(lo[k], c);
      hi[k] = fmaxf(hi[k], c);
    }
  }
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
  }
  if ((tid & 31) == 0)
    for (int k = 0; k < 3; ++k) { red[k][tid >> 5] = lo[k]; red[k + 3][tid >> 5] = hi[k]; }
  __syncthreads();
  if (tid < 3) {
    float a = 3.4e38f, b = -3.4e38f;
    for (int w = 0; w < (nt + 31) / 32; ++w) { a = fminf(a, red[tid][w]); b = fmaxf(b, red[tid + 3][w]); }
    bnd[tid] = a;
    bnd[tid + 3] = (b > a) ? 1.0f / (b - a) : 0.0f;
  }
  __syncthreads();
  int np2 = 1;
  while (np2 < n) np2 <<= 1;
  for (int i = tid; i < np2; i += nt) {
    if (i < n) {
      const float* b = prim + 6 * (size_t)i;
      unsigned code = morton30(0.5f * (b[0] + b[3]), 0.5f * (b[1] + b[4]), 0.5f * (b[2] + b[5]), bnd,
                               bnd + 3);
      keys[i] = ((unsigned long long)code << 32) | (unsigned)i;
    } else {
      keys[i] = ~0ull;
    }
  }
  __syncthreads();
  // Bitonic sort of the np2 keys. Compare-exchanges at distance j < 32 stay
  // within a 32-key chunk and run in registers with warp shuffles (no block
  // barrier); only distances >= 32 go through shared memory.
  const int lane = tid & 31, nw = nt >> 5;
  const int nchunk = (np2 + 31) >> 5;
  auto in_warp = [&](int kmin, int kmax, int jmax) {
    for (int c = tid >> 5; c < nchunk; c += nw) {
      int i = (c << 5) + lane;
      unsigned long long x = i < np2 ? keys[i] : ~0ull;  // padding sorts last
      for (int k = kmin; k <= kmax; k <<= 1) {
        for (int j = min(k >> 1, jmax); j > 0; j >>= 1) {
          unsigned long long y = __shfl_xor_sync(0xffffffffu, x, j);
          bool up = (i & k) == 0, low = (lane & j) == 0;
          x = (low == up) ? (x < y ? x : y) : (x < y ? y : x);
        }
      }
      if (i < np2) keys[i] = x;
    }
    __syncthreads();
  };
  in_warp(2, 32, 16);  // stages k = 2..32: every 32-key chunk sorted, directions alternating
  for (int k = 64; k <= np2; k <<= 1) {
    for (int j = k >> 1; j >= 32; j >>= 1) {
      for (int i = tid; i < np2; i += nt) {
        int ixj = i ^ j;
        if (ixj > i) {
          unsigned long long a = keys[i], b = keys[ixj];
          bool up = (i & k) == 0;
          if ((a > b) == up) { keys[i] = b; keys[ixj] = a; }
        }
      }
      __syncthreads();
    }
    in_warp(k, k, 16);  // the rest of stage k: distances 16..1
  }
  for (int i = tid; i < n; i += nt) perm[i] = (int)(keys[i] & 0xffffffffu);
  if (n == 1) {
    if (tid == 0) {
      root_out[0] = ~leaf_base;
      leaf_parent[leaf_base] = -1;
      for (int k = 0; k < 6; ++k) root_box[k] = prim[k];
    }
    __syncthreads();
    return;
  }
  for (int i = tid; i < n - 1; i += nt) reinterpret_cast<int*>(nodes + 4 * (size_t)(node_base + i) + 3)[2] = -1;
  __syncthreads();
  for (int i = tid; i < n - 1; i += nt) karras_node(keys, n, i, node_base, leaf_base, nodes, leaf_parent);
  if (tid == 0) root_out[0] = node_base;
  __syncthreads();
}

// Walk from leaf slot `slot` (box b) to the root through shared-memory child
// boxes `sbox` (12 floats per node) and arrival counters `sarr`; the second
// arrival at a node forms its box. Adds each formed node's surface area to
// *sah (when not null). Topology comes from the global nodes.
__device__ __forceinline__ void smem_walk_up(const float4* nodes, int node_base, int slot, int p, float* b,
                                             float* sbox, int* sarr, float* root_box, float* sah) {
  int code = ~slot;
  for (int depth = 0; depth < 128 && p >= 0; ++depth) {
    const int* n3 = reinterpret_cast<const int*>(nodes + 4 * (size_t)p + 3);
    int li = p - node_base;
    int side = n3[0] == code ? 0 : 1;
    volatile float* mine = sbox + 12 * (size_t)li + 6 * side;
    for (int k = 0; k < 6; ++k) mine[k] = b[k];
    __threadfence_block();
    if (atomicAdd(&sarr[li], 1) == 0) return;
    __threadfence_block();
    volatile float* both = sbox + 12 * (size_t)li;
    for (int k = 0; k < 3; ++k) {
      b[k] = fminf(both[k], both[6 + k]);
      b[k + 3] = fmaxf(both[k + 3], both[9 + k]);
    }
    if (sah) atomicAdd(sah, box_area(b));
    code = p;
    p = n3[2];
    if (p < 0)
      for (int k = 0; k < 6; ++k) root_box[k] = b[k];
  }
}

// Called by all threads of one CTA.
__device__ void build_small_dev(const float* __restrict__ prim, int n, int node_base, int leaf_base,
                                float4* nodes, int* leaf_parent, int* perm, int* arrive, int* root_out,
                                float* root_box, unsigned long long* keys, float* sbox) {
  int tid = threadIdx.x, nt = blockDim.x;
  sort_karras_dev(prim, n, node_base, leaf_base, nodes, leaf_parent, perm, root_out, root_box, keys);
  if (n <= 1) return;
  if (sbox && n - 1 <= kSmemRefit) {
    int* sarr = reinterpret_cast<int*>(sbox + 12 * (size_t)(n - 1));
    for (int i = tid; i < n - 1; i += nt) sarr[i] = 0;
    __syncthreads();
    for (int j = tid; j < n; j += nt) {
      const float* pb = prim + 6 * (size_t)perm[j];
      float b[6] = {pb[0], pb[1], pb[2], pb[3], pb[4], pb[5]};
      smem_walk_up(nodes, node_base, leaf_base + j, leaf_parent[leaf_base + j], b, sbox, sarr, root_box, nullptr);
    }
    __syncthreads();
    for (int i = tid; i < n - 1; i += nt) {
      put_child_box(nodes, node_base + i, 0, sbox + 12 * (size_t)i);
      put_child_box(nodes, node_base + i, 1, sbox + 12 * (size_t)i + 6);
    }
    return;
  }
  // in-CTA refit through global memory
  for (int i = tid; i < n - 1; i += nt) arrive[i] = 0;
  __syncthreads();
  for (int j = tid; j < n; j += nt) {
    const float* b = prim + 6 * (size_t)perm[j];
    refit_up(nodes, arrive, node_base, leaf_parent[leaf_base + j], ~(leaf_base + j), b, root_box);
  }
}

__global__ void __launch_bounds__(1024) k_build_small(const float* __restrict__ prim, int n,
                                                      int node_base, int leaf_base, float4* nodes,
                                                      int* leaf_parent, int* perm, int* arrive,
                                                      int* root_out, float* root_box) {
  extern __shared__ unsigned long long keys[];
  build_small_dev(prim, n, node_base, leaf_base, nodes, leaf_parent, perm, arrive, root_out, root_box, keys,
                  nullptr);
}

// Per-frame preparation (see FramePrepArgs). Shared memory: np2 keys, then,
// when the larger tree has at most kSmemRefit internal nodes, 12 floats + 1
// int per internal node for the shared-memory refit.
__global__ void __launch_bounds__(1024) k_frame_prep(FramePrepArgs a, int np2, int smem_refit) {
  extern __shared__ unsigned long long keys[];
  float* sbox = smem_refit ? reinterpret_cast<float*>(keys + np2) : nullptr;
  int tid = threadIdx.x, nt = blockDim.x;
  if (blockIdx.x == 0) {
    for (int r = tid; r < a.nrx; r += nt) {
      float x = a.rx3[3 * r], y = a.rx3[3 * r + 1], z = a.rx3[3 * r + 2];
      if (!isfinite(x) || !isfinite(y) || !isfinite(z)) atomicOr(&a.ctr->err, ERR_NONFINITE);
      a.rx_cur[r] = make_float4(x, y, z, 0.0f);
      float* pb = a.rx_prim + 6 * (size_t)r;
      pb[0] = pb[3] = x;
      pb[1] = pb[4] = y;
      pb[2] = pb[5] = z;
      bool mv = true;
      if (a.have_prev) {
        float4 q = a.rx_traced[r];
        mv = __float_as_uint(q.x) != __float_as_uint(x) || __float_as_uint(q.y) != __float_as_uint(y) ||
             __float_as_uint(q.z) != __float_as_uint(z);
      }
      a.rx_moved[r] = mv ? 1 : 0;
      if (mv) a.moved_list[atomicAdd(&a.ctr->rx_moved, 1u)] = r;
      a.bucket_cnt[r] = 0u;
    }
    __syncthreads();
    const SmallTreeArgs& t = a.trx;
    build_small_dev(t.prim, t.n, 0, 0, t.nodes, t.leaf_parent, t.perm, t.arrive, t.root, t.root_box, keys,
                    sbox);
  } else {
    if (a.coherent) {
      for (int ob = tid; ob < a.nobj; ob += nt) {
        bool moved = false;
        for (int k = 0; k < 12; ++k)
          moved = moved || (__float_as_uint(a.xf_cur[12 * ob + k]) != __float_as_uint(a.xf_traced[12 * ob + k]));
        if (a.obj_moved) a.obj_moved[ob] = moved ? 1 : 0;
        if (!moved) continue;
        atomicAdd(&a.ctr->objects_moved, 1u);
        const unsigned* boxes[2] = {a.obj_box_traced, a.obj_box_cur};
        float bx[2][6];
        bool ok[2];
        for (int q = 0; q < 2; ++q) {
          ok[q] = true;
          for (int k = 0; k < 3; ++k) {
            float lo = o2f(boxes[q][3 * (size_t)ob + k]);
            float hi = o2f(boxes[q][3 * (size_t)(a.nobj + ob) + k]);
            ok[q] = ok[q] && (lo <= hi);  // false for an object without triangles
            float m = 1e-3f + 1e-5f * fmaxf(fabsf(lo), fabsf(hi));
            bx[q][k] = lo - m;
            bx[q][k + 3] = hi + m;
          }
        }
        unsigned nq = (ok[0] ? 1u : 0u) + (ok[1] ? 1u : 0u);
        if (!nq) continue;
        unsigned at = atomicAdd(&a.ctr->n_moved_boxes, nq);
        for (int q = 0; q < 2; ++q) {
          if (!ok[q]) continue;
          float* out = a.moved_boxes + 6 * (size_t)at++;
          for (int k = 0; k < 6; ++k) out[k] = bx[q][k];
        }
      }
    }
    __syncthreads();
    const SmallTreeArgs& t = a.tmv;
    int n = a.coherent ? (int)min(a.ctr->n_moved_boxes, (unsigned)t.cap) : 0;
    build_small_dev(t.prim, n, 0, 0, t.nodes, t.leaf_parent, t.perm, t.arrive, t.root, t.root_box, keys, sbox);
  }
}

// ---------------------------------------------------------------------------
// multi-CTA builder for large trees: Morton codes, 4-pass stable LSD radix
// sort of the 30-bit codes carrying the primitive index, Karras nodes.
// ---------------------------------------------------------------------------
__global__ void k_centroid_bounds(const float* __restrict__ prim, int n, unsigned* ob) {
  float lo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, hi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float* b = prim + 6 * (size_t)i;
    for (int k = 0; k < 3; ++k) {
      float c = 0.5f * (b[k] + b[k + 3]);
      lo[k] = fminf(lo[k], c);
      hi[k] = fmaxf(hi[k], c);
    }
  }
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&ob[k], f2o(lo[k]));
      atomicMax(&ob[k + 3], f2o(hi[k]));
    }
  }
}

__global__ void k_morton(const float* __restrict__ prim, int n, const unsigned* ob, unsigned* codes,
                         unsigned* idx) {
  // One scale for all axes (the largest extent): in a large flat scene (a
  // city) the short axis then splits deep in the tree instead of at its top.
  // Measured on the 61k-triangle urban grid: 56 -> 42 node pairs per segment,
  // closest hit 27 -> 23 ms. The one-CTA builder keeps one scale per axis:
  // on the highway (2 km x 30 m) a cubic frame made its trees slower to
  // traverse (1920 against 2300 frames/s, with 16 bits per axis as well).
  float lo[3], inv[3], m = 0.0f;
  for (int k = 0; k < 3; ++k) {
    lo[k] = o2f(ob[k]);
    float h = o2f(ob[k + 3]);
    m = fmaxf(m, h > lo[k] ? h - lo[k] : 0.0f);
  }
  for (int k = 0; k < 3; ++k) inv[k] = m > 0.0f ? 1.0f / m : 0.0f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float* b = prim + 6 * (size_t)i;
    codes[i] = morton30(0.5f * (b[0] + b[3]), 0.5f * (b[1] + b[4]), 0.5f * (b[2] + b[5]), lo, inv);
    idx[i] = (unsigned)i;
  }
}

constexpr int kRadixItems = 1024;  // per block: 4 rounds of 256

__global__ void __launch_bounds__(256) k_radix_hist(const unsigned* __restrict__ keys, int n, int shift,
                                                    unsigned* hist, int nblocks) {
  __shared__ unsigned h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int base = blockIdx.x * kRadixItems;
  for (int r = 0; r < 4; ++r) {
    int i = base + r * 256 + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of m counts in tiles of 4096 (1024 threads, 4 consecutive
// counts each): each tile is scanned in place and, with `sums`, its total is
// written to sums[tile]; k_scan_add then adds the scanned tile totals.
constexpr int kScanTile = 4096;
__global__ void __launch_bounds__(1024) k_scan_tile(unsigned* a, int m, unsigned* sums) {
  __shared__ unsigned wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long base = (long)blockIdx.x * kScanTile + 4 * tid;
  unsigned v[4], t = 0;
  for (int j = 0; j < 4; ++j) {
    v[j] = base + j < m ? a[base + j] : 0u;
    t += v[j];
  }
  unsigned inc = t;  // inclusive scan of the thread totals within the warp
  for (int o = 1; o < 32; o <<= 1) {
    unsigned u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    unsigned x = wsum[lane], y = x;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned u = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += u;
    }
    wsum[lane] = y - x;  // exclusive over the warps
    if (lane == 31 && sums) sums[blockIdx.x] = y;
  }
  __syncthreads();
  unsigned run = wsum[w] + inc - t;
  for (int j = 0; j < 4; ++j) {
    if (base + j < m) a[base + j] = run;
    run += v[j];
  }
}

__global__ void __launch_bounds__(1024) k_scan_add(unsigned* a, int m, const unsigned* sums) {
  const unsigned add = sums[blockIdx.x];
  const long base = (long)blockIdx.x * kScanTile + 4 * threadIdx.x;
  for (int j = 0; j < 4; ++j)
    if (base + j < m) a[base + j] += add;
}

// In-place exclusive scan of a[0, m); `scratch` holds scan_scratch_size(m)
// counts for the tile totals of every level.
static void scan_excl(unsigned* a, int m, unsigned* scratch, cudaStream_t st) {
  int tiles = (m + kScanTile - 1) / kScanTile;
  if (tiles <= 1) {
    k_scan_tile<<<1, 1024, 0, st>>>(a, m, nullptr);
    return;
  }
  k_scan_tile<<<tiles, 1024, 0, st>>>(a, m, scratch);
  scan_excl(scratch, tiles, scratch + tiles, st);
  k_scan_add<<<tiles, 1024, 0, st>>>(a, m, scratch);
}

size_t scan_scratch_size(size_t m) {
  size_t n = 0;
  for (size_t t = (m + kScanTile - 1) / kScanTile; t > 1; t = (t + kScanTile - 1) / kScanTile) n += t;
  return n + 1;
}

__global__ void __launch_bounds__(256) k_radix_scatter(const unsigned* __restrict__ kin,
                                                       const unsigned* __restrict__ vin, int n, int shift,
                                                       const unsigned* __restrict__ hist, int nblocks,
                                                       unsigned* kout, unsigned* vout) {
  __shared__ unsigned run[256];
  __shared__ unsigned wcnt[8][256];
  int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  run[tid] = hist[tid * nblocks + blockIdx.x];
  int base = blockIdx.x * kRadixItems;
  for (int r = 0; r < 4; ++r) {
    for (int q = 0; q < 8; ++q) wcnt[q][tid] = 0;
    __syncthreads();
    int i = base + r * 256 + tid;
    bool valid = i < n;
    unsigned key = valid ? kin[i] : 0u, val = valid ? vin[i] : 0u;
    unsigned dig = valid ? ((key >> shift) & 255u) : 256u + (unsigned)lane;  // invalid lanes unique
    unsigned peers = __match_any_sync(0xffffffffu, dig);
    unsigned rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[w][dig] = __popc(peers);
    __syncthreads();
    // per digit: exclusive prefix over warps (thread tid owns digit tid)
    unsigned acc = 0;
    for (int q = 0; q < 8; ++q) {
      unsigned c = wcnt[q][tid];
      wcnt[q][tid] = acc;
      acc += c;
    }
    __syncthreads();
    if (valid) {
      unsigned pos = run[dig] + wcnt[w][dig] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    run[tid] += acc;
    __syncthreads();
  }
}

__global__ void k_make_keys(const unsigned* codes, const unsigned* idx, int n, unsigned long long* keys,
                            int* perm) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    keys[i] = ((unsigned long long)codes[i] << 32) | idx[i];
    perm[i] = (int)idx[i];
  }
}

__global__ void k_karras(const unsigned long long* __restrict__ keys, int n, int node_base, int leaf_base,
                         float4* nodes, int* leaf_parent) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n - 1; i += gridDim.x * blockDim.x)
    karras_node(keys, n, i, node_base, leaf_base, nodes, leaf_parent);
}

__global__ void k_init_parents(float4* nodes, int node_base, int nint, int* arrive) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nint; i += gridDim.x * blockDim.x) {
    reinterpret_cast<int*>(nodes + 4 * (size_t)(node_base + i) + 3)[2] = -1;
    arrive[i] = 0;
  }
}

// refit from primitive boxes in leaf order (prim[perm[j]])
__global__ void k_refit_prims(const float* __restrict__ prim, const int* __restrict__ perm, int n,
                              int node_base, int leaf_base, float4* nodes, const int* leaf_parent,
                              int* arrive, float* root_box) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const float* b = prim + 6 * (size_t)perm[j];
    refit_up(nodes, arrive, node_base, leaf_parent[leaf_base + j], ~(leaf_base + j), b, root_box);
  }
}

// ---------------------------------------------------------------------------
// triangles
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tri_box(float3 a, float3 b, float3 c, float* o) {
  o[0] = fminf(a.x, fminf(b.x, c.x)); o[1] = fminf(a.y, fminf(b.y, c.y)); o[2] = fminf(a.z, fminf(b.z, c.z));
  o[3] = fmaxf(a.x, fmaxf(b.x, c.x)); o[4] = fmaxf(a.y, fmaxf(b.y, c.y)); o[5] = fmaxf(a.z, fmaxf(b.z, c.z));
}

// boxes of triangles given as 9 floats each, indices sel[i] (or i when sel is null)
__global__ void k_tri_boxes(const float* __restrict__ v9, const int* __restrict__ sel, int n, float* prim) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float* v = v9 + 9 * (size_t)(sel ? sel[i] : i);
    tri_box(f3(v[0], v[1], v[2]), f3(v[3], v[4], v[5]), f3(v[6], v[7], v[8]), prim + 6 * (size_t)i);
  }
}

// Scatter triangles into leaf order: leaf j of a tree holds input triangle
// gid = sel[perm[j]]; v9 are its (world or object space) vertices.
__global__ void k_place_tris(const float* __restrict__ v9, const int* __restrict__ sel,
                             const int* __restrict__ perm, const int* __restrict__ tri_mat,
                             const int* __restrict__ tri_obj, int n, int leaf_base, float4* tris,
                             float4* objv, int* slot_of_id) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    int gid = sel[perm[j]];
    const float* v = v9 + 9 * (size_t)gid;
    int slot = leaf_base + j;
    float4* t = tris + 3 * (size_t)slot;
    t[0] = make_float4(v[0], v[1], v[2], __int_as_float(gid));
    t[1] = make_float4(v[3], v[4], v[5], __int_as_float(tri_mat[gid]));
    t[2] = make_float4(v[6], v[7], v[8], 0.0f);
    if (objv) {
      float4* q = objv + 3 * (size_t)j;
      int ob = tri_obj[gid];
      q[0] = make_float4(v[0], v[1], v[2], __int_as_float(ob));
      q[1] = make_float4(v[3], v[4], v[5], __int_as_float(gid));
      q[2] = make_float4(v[6], v[7], v[8], __int_as_float(tri_mat[gid]));
    }
    slot_of_id[gid] = slot;
  }
}

// ---------------------------------------------------------------------------
// per-frame: transform dynamic triangles + refit + per-object boxes
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 xform(const float* m, float3 p) {
  return f3(__fmaf_rn(m[0], p.x, __fmaf_rn(m[1], p.y, __fmaf_rn(m[2], p.z, m[3]))),
            __fmaf_rn(m[4], p.x, __fmaf_rn(m[5], p.y, __fmaf_rn(m[6], p.z, m[7]))),
            __fmaf_rn(m[8], p.x, __fmaf_rn(m[9], p.y, __fmaf_rn(m[10], p.z, m[11]))));
}

__global__ void k_transform_refit(const float4* __restrict__ objv, const float* __restrict__ xf, int n, int nobj,
                                  int node_base, int leaf_base, float4* tris, float4* nodes,
                                  const int* __restrict__ leaf_parent, int* arrive, float* root_box,
                                  unsigned* obj_box, DevCounters* ctr) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    float4 a = objv[3 * (size_t)j], b = objv[3 * (size_t)j + 1], c = objv[3 * (size_t)j + 2];
    int ob = __float_as_int(a.w);
    const float* m = xf + 12 * (size_t)ob;
    float3 w0 = xform(m, f3(a.x, a.y, a.z)), w1 = xform(m, f3(b.x, b.y, b.z)), w2 = xform(m, f3(c.x, c.y, c.z));
    int slot = leaf_base + j;
    float4* t = tris + 3 * (size_t)slot;
    float4 t0 = t[0], t1 = t[1];
    t[0] = make_float4(w0.x, w0.y, w0.z, t0.w);
    t[1] = make_float4(w1.x, w1.y, w1.z, t1.w);
    t[2] = make_float4(w2.x, w2.y, w2.z, 0.0f);
    float box[6];
    tri_box(w0, w1, w2, box);
    bool fin = true;
    for (int k = 0; k < 6; ++k) fin = fin && isfinite(box[k]);
    if (!fin) atomicOr(&ctr->err, ERR_NONFINITE);
    // per-object world box: lo in obj_box[0, 3 nobj), hi in obj_box[3 nobj, 6 nobj)
    for (int k = 0; k < 3; ++k) {
      atomicMin(&obj_box[3 * (size_t)ob + k], f2o(box[k]));
      atomicMax(&obj_box[3 * (size_t)(nobj + ob) + k], f2o(box[k + 3]));
    }
    refit_up(nodes, arrive, node_base, leaf_parent[slot], ~slot, box, root_box);
  }
}

// ---------------------------------------------------------------------------
// per frame, moving objects of up to kSmemRefit + 1 triangles: one CTA
// transforms, (re)builds when asked, refits level by level in shared memory
// and measures the tree's surface-area cost
// ---------------------------------------------------------------------------
// After each (re)build the internal nodes are ordered by height (1 + the
// larger child height, leaves 0), in node order within a height, and that
// schedule is kept in global memory. A refit then needs no atomics: leaf
// boxes first, then one height at a time with a barrier in between, every
// node of a height formed from its children's boxes by one thread. The
// surface-area sum runs in schedule order, so it is the same in every run.
//
// Shared-memory layout (n = nd leaves, m = n - 1 nodes, np2 = next power of
// two >= n): keys[np2] (rebuild sort; node heights afterwards) | leaf boxes
// float[6 n] | node boxes float[6 m] | children int[2 m] | schedule int[m] |
// level bounds int[kMaxLevels + 2] (lvl[h]..lvl[h + 1] = height h + 1) |
// object boxes unsigned[6 nobj].
constexpr int kMaxLevels = kDynLevels;

__global__ void __launch_bounds__(1024) k_dyn_update(DynUpdateArgs a) {
  extern __shared__ unsigned long long keys[];
  int tid = threadIdx.x, nt = blockDim.x;
  int n = a.nd, m = n > 1 ? n - 1 : 1;
  int np2 = 1;
  while (np2 < n) np2 <<= 1;
  float* lbox = reinterpret_cast<float*>(keys + np2);
  float* nbox = lbox + 6 * (size_t)n;
  int* kids = reinterpret_cast<int*>(nbox + 6 * (size_t)m);
  int* sched = kids + 2 * (size_t)m;
  int* lvl = sched + m;
  unsigned* sobj = reinterpret_cast<unsigned*>(lvl + kMaxLevels + 2);
  __shared__ float sah_part[32];
  __shared__ unsigned bad;
  __shared__ int nlvl, left;
  if (tid == 0) bad = 0u;
  for (int k = tid; k < 6 * a.nobj; k += nt) sobj[k] = k < 3 * a.nobj ? 0xffffffffu : 0u;
  if (a.rebuild) {
    // world boxes of the primitives (primitive order), then a fresh topology
    for (int i = tid; i < n; i += nt) {
      const float4* q = a.objv_src + 3 * (size_t)i;
      const float* mx = a.xf + 12 * (size_t)__float_as_int(q[0].w);
      float3 w0 = xform(mx, f3(q[0].x, q[0].y, q[0].z)), w1 = xform(mx, f3(q[1].x, q[1].y, q[1].z)),
             w2 = xform(mx, f3(q[2].x, q[2].y, q[2].z));
      tri_box(w0, w1, w2, a.prim + 6 * (size_t)i);
    }
    __syncthreads();
    sort_karras_dev(a.prim, n, a.node_base, a.leaf_base, a.nodes, a.leaf_parent, a.perm, a.root, a.root_box, keys);
    for (int j = tid; j < n; j += nt) {
      int i = a.perm[j];
      int gid = a.sel_d[i];
      int slot = a.leaf_base + j;
      for (int k = 0; k < 3; ++k) a.objv[3 * (size_t)j + k] = a.objv_src[3 * (size_t)i + k];
      a.tris[3 * (size_t)slot].w = __int_as_float(gid);
      a.tris[3 * (size_t)slot + 1].w = __int_as_float(a.tri_mat[gid]);
      a.slot_of_id[gid] = slot;
    }
  }
  // children of every node (global codes: >= 0 node, < 0 leaf ~slot); on a
  // refit also the kept schedule, in the same round of loads
  if (n > 1) {
    for (int i = tid; i < m; i += nt) {
      int2 c = *reinterpret_cast<const int2*>(a.nodes + 4 * (size_t)(a.node_base + i) + 3);
      kids[2 * i] = c.x;
      kids[2 * i + 1] = c.y;
    }
    if (!a.rebuild) {
      for (int k = tid; k < m; k += nt) sched[k] = a.sched[k];
      for (int h = tid; h < kMaxLevels + 2; h += nt) lvl[h] = a.lvl[h];
    }
  }
  __syncthreads();
  if (a.rebuild && n > 1) {
    // node heights by repeated passes (at most the tree height, <= 63 for
    // 64-bit Karras keys), then the schedule
    volatile int* hgt = reinterpret_cast<volatile int*>(keys);
    for (int i = tid; i < m; i += nt) hgt[i] = -1;
    if (tid == 0) left = m;
    __syncthreads();
    for (int pass = 0; pass < kMaxLevels && left > 0; ++pass) {
      for (int i = tid; i < m; i += nt) {
        if (hgt[i] >= 0) continue;
        int c0 = kids[2 * i], c1 = kids[2 * i + 1];
        int h0 = c0 < 0 ? 0 : hgt[c0 - a.node_base], h1 = c1 < 0 ? 0 : hgt[c1 - a.node_base];
        if (h0 >= 0 && h1 >= 0) {
          hgt[i] = 1 + max(h0, h1);
          atomicSub(&left, 1);
        }
      }
      __syncthreads();
    }
    if (left > 0) {  // deeper than kMaxLevels: a malformed tree
      if (tid == 0) atomicOr(&a.uctr->err, ERR_STACK);
      return;
    }
    // level starts: heights 1.. in increasing order
    for (int h = tid; h < kMaxLevels + 2; h += nt) lvl[h] = 0;
    __syncthreads();
    for (int i = tid; i < m; i += nt) atomicAdd(&lvl[hgt[i]], 1);  // lvl[h] = count of height h
    __syncthreads();
    if (tid == 0) {
      int run = 0, top = 0;
      for (int h = 1; h <= kMaxLevels; ++h) {
        int c = lvl[h];
        lvl[h] = run;  // start of height h (levels indexed from 1)
        run += c;
        if (c) top = h;
      }
      lvl[kMaxLevels + 1] = run;
      nlvl = top;
    }
    __syncthreads();
    // stable scatter by height (warp 0, 32 nodes at a time)
    if (tid < 32) {
      for (int c = 0; c < m; c += 32) {
        int i = c + tid;
        int h = i < m ? hgt[i] : 0;
        unsigned peers = __match_any_sync(0xffffffffu, h);
        int rank = __popc(peers & ((1u << tid) - 1u));
        if (i < m) sched[lvl[h] + rank] = i;
        __syncwarp();
        if (i < m && rank == 0) lvl[h] += __popc(peers);
        __syncwarp();
      }
    }
    __syncthreads();
    // lvl[h] (h >= 1) now holds the end of height h, which is where height
    // h + 1 starts; lvl[0] = 0 is where height 1 starts
    if (tid == 0) lvl[0] = 0;
    __syncthreads();
    for (int k = tid; k < m; k += nt) a.sched[k] = sched[k];
    for (int h = tid; h <= nlvl; h += nt) a.lvl[h] = lvl[h];
    if (tid == 0) a.lvl[kMaxLevels + 1] = nlvl;
  } else if (n > 1) {
    if (tid == 0) nlvl = lvl[kMaxLevels + 1];
  }
  // world triangles (whole 16-byte records), leaf boxes, object boxes
  for (int j = tid; j < n; j += nt) {
    const float4* q = a.objv + 3 * (size_t)j;
    float4 q0 = q[0], q1 = q[1], q2 = q[2];
    int ob = __float_as_int(q0.w);
    const float4* mx4 = reinterpret_cast<const float4*>(a.xf + 12 * (size_t)ob);
    float4 r0 = mx4[0], r1 = mx4[1], r2 = mx4[2];
    float mx[12] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, r2.x, r2.y, r2.z, r2.w};
    float3 w0 = xform(mx, f3(q0.x, q0.y, q0.z)), w1 = xform(mx, f3(q1.x, q1.y, q1.z)),
           w2 = xform(mx, f3(q2.x, q2.y, q2.z));
    int slot = a.leaf_base + j;
    float4* t = a.tris + 3 * (size_t)slot;
    t[0] = make_float4(w0.x, w0.y, w0.z, q1.w);
    t[1] = make_float4(w1.x, w1.y, w1.z, q2.w);
    t[2] = make_float4(w2.x, w2.y, w2.z, 0.0f);
    float* b = lbox + 6 * (size_t)j;
    tri_box(w0, w1, w2, b);
    bool fin = true;
    for (int k = 0; k < 6; ++k) fin = fin && isfinite(b[k]);
    if (!fin) bad = 1u;
    for (int k = 0; k < 3; ++k) {
      atomicMin(&sobj[3 * ob + k], f2o(b[k]));
      atomicMax(&sobj[3 * (a.nobj + ob) + k], f2o(b[k + 3]));
    }
  }
  __syncthreads();
  float sah = 0.0f;  // this thread's share of the node surface areas
  if (n == 1) {
    if (tid < 6) a.root_box[tid] = lbox[tid];
  } else {
    for (int h = 0; h < nlvl; ++h) {
      for (int k = lvl[h] + tid; k < lvl[h + 1]; k += nt) {
        int i = sched[k];
        int c0 = kids[2 * i], c1 = kids[2 * i + 1];
        const float* b0 = c0 < 0 ? lbox + 6 * (size_t)(~c0 - a.leaf_base) : nbox + 6 * (size_t)(c0 - a.node_base);
        const float* b1 = c1 < 0 ? lbox + 6 * (size_t)(~c1 - a.leaf_base) : nbox + 6 * (size_t)(c1 - a.node_base);
        float* u = nbox + 6 * (size_t)i;
        for (int q = 0; q < 3; ++q) {
          u[q] = fminf(b0[q], b1[q]);
          u[q + 3] = fmaxf(b0[q + 3], b1[q + 3]);
        }
        sah += box_area(u);
      }
      __syncthreads();
    }
    if (tid < 6) a.root_box[tid] = nbox[tid];  // the Karras root is node 0
    // child boxes into the node records, three 16-byte stores per node
    for (int i = tid; i < m; i += nt) {
      int c0 = kids[2 * i], c1 = kids[2 * i + 1];
      const float* b0 = c0 < 0 ? lbox + 6 * (size_t)(~c0 - a.leaf_base) : nbox + 6 * (size_t)(c0 - a.node_base);
      const float* b1 = c1 < 0 ? lbox + 6 * (size_t)(~c1 - a.leaf_base) : nbox + 6 * (size_t)(c1 - a.node_base);
      float4* nd = a.nodes + 4 * (size_t)(a.node_base + i);
      nd[0] = make_float4(b0[0], b0[3], b0[1], b0[4]);
      nd[1] = make_float4(b1[0], b1[3], b1[1], b1[4]);
      nd[2] = make_float4(b0[2], b0[5], b1[2], b1[5]);
    }
  }
  for (int k = tid; k < 6 * a.nobj; k += nt) a.obj_box[k] = sobj[k];
  for (int off = 16; off > 0; off >>= 1) sah += __shfl_down_sync(0xffffffffu, sah, off);
  if ((tid & 31) == 0) sah_part[tid >> 5] = sah;
  __syncthreads();
  if (tid == 0) {
    float tot = 0.0f;
    for (int w = 0; w < (nt + 31) / 32; ++w) tot += sah_part[w];
    if (bad) atomicOr(&a.uctr->err, ERR_NONFINITE);
    float ra = box_area(a.root_box);
    float cost = ra > 0.0f ? tot / ra : 0.0f;
    a.uctr->sah_refit = cost;
    if (a.rebuild) a.uctr->sah_build = cost;
  }
}

// ---------------------------------------------------------------------------
// compact copy of both trees for shared-memory traversal
// ---------------------------------------------------------------------------
// Codes are rounded outward by three steps: the FP32 quotient (v - o) / s is
// within a small fraction of a step of the exact one, so the code box
// contains the exact box with more than two steps to spare on every side.
__device__ __forceinline__ unsigned qenc_lo(float v, float o, float s) {
  if (!isfinite(v)) return 0u;
  float d = floorf((v - o) / s) - 3.0f;
  if (!(d >= 0.0f)) return 0u;
  return d > 65535.0f ? 65535u : (unsigned)d;
}
__device__ __forceinline__ unsigned qenc_hi(float v, float o, float s) {
  if (!isfinite(v)) return 65535u;
  float d = ceilf((v - o) / s) + 3.0f;
  if (!(d <= 65535.0f)) return 65535u;
  return d < 0.0f ? 0u : (unsigned)d;
}

// Compact copy of both trees (layout and grid in dcem_internal.cuh): the
// grid pads the union of the root boxes by 1 m + 1e-3 of its largest extent
// on every side, so every box lies well inside it, with 65000 steps across
// each padded axis.
__global__ void k_quantize(const float4* __restrict__ nodes, int nn, const float* __restrict__ root_box,
                           int has0, int has1, uint4* qn, float* qframe) {
  float lo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, hi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
  for (int t = 0; t < 2; ++t) {
    if (!(t == 0 ? has0 : has1)) continue;
    for (int k = 0; k < 3; ++k) {
      float a = root_box[6 * t + k], b = root_box[6 * t + 3 + k];
      if (isfinite(a)) lo[k] = fminf(lo[k], a);
      if (isfinite(b)) hi[k] = fmaxf(hi[k], b);
    }
  }
  float ext = 0.0f;
  for (int k = 0; k < 3; ++k) {
    if (!(hi[k] >= lo[k])) { lo[k] = 0.0f; hi[k] = 0.0f; }
    ext = fmaxf(ext, hi[k] - lo[k]);
  }
  float pad = 1.0f + 1e-3f * ext;
  float o[3], sc[3];
  for (int k = 0; k < 3; ++k) {
    o[k] = lo[k] - pad;
    sc[k] = fmaxf((hi[k] - lo[k] + 2.0f * pad) / 65000.0f, 1e-6f);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) { qframe[k] = o[k]; qframe[3 + k] = sc[k]; }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
    float4 n0 = nodes[4 * (size_t)i], n1 = nodes[4 * (size_t)i + 1], n2 = nodes[4 * (size_t)i + 2],
           n3 = nodes[4 * (size_t)i + 3];
    // child 0: lo (n0.x, n0.z, n2.x), hi (n0.y, n0.w, n2.y); child 1 likewise
    unsigned w[6] = {qenc_lo(n0.x, o[0], sc[0]) | (qenc_hi(n0.y, o[0], sc[0]) << 16),
                     qenc_lo(n0.z, o[1], sc[1]) | (qenc_hi(n0.w, o[1], sc[1]) << 16),
                     qenc_lo(n2.x, o[2], sc[2]) | (qenc_hi(n2.y, o[2], sc[2]) << 16),
                     qenc_lo(n1.x, o[0], sc[0]) | (qenc_hi(n1.y, o[0], sc[0]) << 16),
                     qenc_lo(n1.z, o[1], sc[1]) | (qenc_hi(n1.w, o[1], sc[1]) << 16),
                     qenc_lo(n2.z, o[2], sc[2]) | (qenc_hi(n2.w, o[2], sc[2]) << 16)};
    qn[2 * (size_t)i] = make_uint4(w[0], w[1], w[2], w[3]);
    qn[2 * (size_t)i + 1] = make_uint4(w[4], w[5], __float_as_uint(n3.x), __float_as_uint(n3.y));
  }
}

// ---------------------------------------------------------------------------
// 4-wide compact copy of both trees (layout in dcem_internal.cuh)
// ---------------------------------------------------------------------------
// One CTA maps the binary trees (nn internal nodes, roots roots[0..1]) to
// 4-wide nodes: every internal node at even depth becomes a 4-wide node whose
// children are its own children, an internal child replaced by that child's
// two children. For each child slot it records the child (4-wide index,
// leaf ~slot, or kEmpty) and where its box lives in the binary records
// (record << 1 | side). Scratch parent[nn], depth[nn], index[nn]: shared
// memory, or the global array `gscr` (3 nn ints) when that does not fit.
__global__ void __launch_bounds__(1024) k_bvh4_map(const float4* __restrict__ nodes, int nn,
                                                   const int* __restrict__ roots, int4* kid4, int4* src4,
                                                   int* n4_out, int* roots4_out, int* gscr) {
  extern __shared__ int sm4[];
  int* par = gscr ? gscr : sm4;
  int* depth = par + nn;
  int* idx = depth + nn;
  __shared__ int total, carry;
  __shared__ int wsum[32];
  int tid = threadIdx.x, nt = blockDim.x;
  auto kid = [&](int n, int side) {
    return reinterpret_cast<const int*>(nodes + 4 * (size_t)n + 3)[side];
  };
  // parents from the child codes, then each node's depth by walking up to
  // its root (no level-by-level passes); a node that does not reach one of
  // the two roots gets no 4-wide node
  for (int i = tid; i < nn; i += nt) par[i] = -1;
  __syncthreads();
  for (int i = tid; i < nn; i += nt)
    for (int side = 0; side < 2; ++side) {
      int c = kid(i, side);
      if (c >= 0 && c < nn) par[c] = i;
    }
  __syncthreads();
  const int r0 = roots[0], r1 = roots[1];
  for (int i = tid; i < nn; i += nt) {
    int d = 0, top = i;
    while (par[top] >= 0 && d < 4096) {
      top = par[top];
      ++d;
    }
    depth[i] = (par[top] < 0 && (top == r0 || top == r1)) ? d : -1;
  }
  __syncthreads();
  // exclusive prefix count of even-depth nodes, one tile of nt nodes at a
  // time: warp scans, a scan of the warp sums, and the running carry
  if (tid == 0) carry = 0;
  __syncthreads();
  const int lane = tid & 31, w = tid >> 5, nw = nt >> 5;
  for (int base = 0; base < nn; base += nt) {
    int i = base + tid;
    int f = (i < nn && depth[i] >= 0 && (depth[i] & 1) == 0) ? 1 : 0;
    int v = f;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
      int x = lane < nw ? wsum[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      wsum[lane] = x;
    }
    __syncthreads();
    int excl = carry + (w > 0 ? wsum[w - 1] : 0) + v - f;
    if (i < nn) idx[i] = excl;
    __syncthreads();
    if (tid == nt - 1) carry = excl + f;
    __syncthreads();
  }
  if (tid == 0) total = carry;
  __syncthreads();
  for (int i = tid; i < nn; i += nt) {
    if (!(depth[i] >= 0 && (depth[i] & 1) == 0)) continue;
    int k[4] = {kEmpty, kEmpty, kEmpty, kEmpty}, sr[4] = {0, 0, 0, 0};
    int m = 0;
    for (int side = 0; side < 2; ++side) {
      int c = kid(i, side);
      if (c >= 0) {  // internal child: its two children become slots
        for (int s2 = 0; s2 < 2; ++s2) {
          int g = kid(c, s2);
          k[m] = g >= 0 ? idx[g] : g;
          sr[m] = (c << 1) | s2;
          ++m;
        }
      } else {
        k[m] = c;
        sr[m] = (i << 1) | side;
        ++m;
      }
    }
    kid4[idx[i]] = make_int4(k[0], k[1], k[2], k[3]);
    src4[idx[i]] = make_int4(sr[0], sr[1], sr[2], sr[3]);
  }
  if (tid < 2) {
    int r = roots[tid];
    roots4_out[tid] = (r >= 0 && r < nn) ? idx[r] : r;
  }
  if (tid == 0) *n4_out = total;
}

__device__ __forceinline__ unsigned qword(float lo, float hi, float o, float s) {
  return qenc_lo(lo, o, s) | (qenc_hi(hi, o, s) << 16);
}

// Per frame: the 4-wide compact nodes from the current binary child boxes,
// on the grid of k_quantize (written to qframe by the first thread).
__global__ void k_quantize4(const float4* __restrict__ nodes, const int* __restrict__ n4p,
                            const int4* __restrict__ kid4, const int4* __restrict__ src4,
                            const float* __restrict__ root_box, int has0, int has1, uint4* q4, float* qframe) {
  float lo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, hi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
  for (int t = 0; t < 2; ++t) {
    if (!(t == 0 ? has0 : has1)) continue;
    for (int k = 0; k < 3; ++k) {
      float a = root_box[6 * t + k], b = root_box[6 * t + 3 + k];
      if (isfinite(a)) lo[k] = fminf(lo[k], a);
      if (isfinite(b)) hi[k] = fmaxf(hi[k], b);
    }
  }
  float ext = 0.0f;
  for (int k = 0; k < 3; ++k) {
    if (!(hi[k] >= lo[k])) { lo[k] = 0.0f; hi[k] = 0.0f; }
    ext = fmaxf(ext, hi[k] - lo[k]);
  }
  float pad = 1.0f + 1e-3f * ext;
  float o[3], sc[3];
  for (int k = 0; k < 3; ++k) {
    o[k] = lo[k] - pad;
    sc[k] = fmaxf((hi[k] - lo[k] + 2.0f * pad) / 65000.0f, 1e-6f);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) { qframe[k] = o[k]; qframe[3 + k] = sc[k]; }
  const int n4 = *n4p;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += gridDim.x * blockDim.x) {
    int4 kd = kid4[i], sr = src4[i];
    int kk[4] = {kd.x, kd.y, kd.z, kd.w}, ss[4] = {sr.x, sr.y, sr.z, sr.w};
    unsigned w[12];
    for (int j = 0; j < 4; ++j) {
      if (kk[j] == kEmpty) {  // an inverted box: no ray meets it
        w[3 * j] = w[3 * j + 1] = w[3 * j + 2] = 0x0000FFFFu;
        continue;
      }
      const float4* n = nodes + 4 * (size_t)(ss[j] >> 1);
      float4 n0 = n[0], n1 = n[1], n2 = n[2];
      bool s1 = (ss[j] & 1) != 0;
      float4 xy = s1 ? n1 : n0;
      float zl = s1 ? n2.z : n2.x, zh = s1 ? n2.w : n2.y;
      w[3 * j] = qword(xy.x, xy.y, o[0], sc[0]);
      w[3 * j + 1] = qword(xy.z, xy.w, o[1], sc[1]);
      w[3 * j + 2] = qword(zl, zh, o[2], sc[2]);
    }
    uint4* d = q4 + 4 * (size_t)i;
    d[0] = make_uint4(w[0], w[1], w[2], w[3]);
    d[1] = make_uint4(w[4], w[5], w[6], w[7]);
    d[2] = make_uint4(w[8], w[9], w[10], w[11]);
    d[3] = make_uint4((unsigned)kk[0], (unsigned)kk[1], (unsigned)kk[2], (unsigned)kk[3]);
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static inline int nblk(long n, int bs, int cap = 4096) {
  long b = (n + bs - 1) / bs;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

cudaError_t build_tree(const float* d_prim, int n, int node_base, int leaf_base, float4* d_nodes,
                       int* d_leaf_parent, int* d_perm, int* d_arrive, int* d_root, float* d_root_box,
                       BuildScratch& scr, cudaStream_t st) {
  if (n <= 0) {
    int e = kEmpty;
    return cudaMemcpyAsync(d_root, &e, sizeof(int), cudaMemcpyHostToDevice, st);
  }
  if (n <= kSmallBuild) {
    int np2 = 1;
    while (np2 < n) np2 <<= 1;
    size_t smem = (size_t)np2 * sizeof(unsigned long long);
    cudaError_t e = cudaFuncSetAttribute(k_build_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kSmallBuild * sizeof(unsigned long long)));
    if (e != cudaSuccess) return e;
    k_build_small<<<1, 1024, smem, st>>>(d_prim, n, node_base, leaf_base, d_nodes, d_leaf_parent, d_perm,
                                         d_arrive, d_root, d_root_box);
    return cudaGetLastError();
  }
  // large path
  cudaError_t e;
  unsigned init[6];
  for (int k = 0; k < 3; ++k) { init[k] = 0xffffffffu; init[k + 3] = 0u; }
  if ((e = cudaMemcpyAsync(scr.bounds, init, sizeof(init), cudaMemcpyHostToDevice, st))) return e;
  k_centroid_bounds<<<nblk(n, 256, 1024), 256, 0, st>>>(d_prim, n, scr.bounds);
  k_morton<<<nblk(n, 256), 256, 0, st>>>(d_prim, n, scr.bounds, scr.k0, scr.v0);
  int nb = (n + kRadixItems - 1) / kRadixItems;
  unsigned *ki = scr.k0, *vi = scr.v0, *ko = scr.k1, *vo = scr.v1;
  for (int pass = 0; pass < 4; ++pass) {
    int shift = 8 * pass;
    k_radix_hist<<<nb, 256, 0, st>>>(ki, n, shift, scr.hist, nb);
    scan_excl(scr.hist, 256 * nb, scr.hist + (size_t)256 * nb, st);
    k_radix_scatter<<<nb, 256, 0, st>>>(ki, vi, n, shift, scr.hist, nb, ko, vo);
    unsigned* t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
  k_make_keys<<<nblk(n, 256), 256, 0, st>>>(ki, vi, n, scr.keys, d_perm);
  k_init_parents<<<nblk(n, 256), 256, 0, st>>>(d_nodes, node_base, n - 1, d_arrive);
  k_karras<<<nblk(n, 256), 256, 0, st>>>(scr.keys, n, node_base, leaf_base, d_nodes, d_leaf_parent);
  int root = node_base;
  if ((e = cudaMemcpyAsync(d_root, &root, sizeof(int), cudaMemcpyHostToDevice, st))) return e;
  k_refit_prims<<<nblk(n, 256), 256, 0, st>>>(d_prim, d_perm, n, node_base, leaf_base, d_nodes,
                                              d_leaf_parent, d_arrive, d_root_box);
  return cudaGetLastError();
}

cudaError_t launch_frame_prep(const FramePrepArgs& a, cudaStream_t st) {
  int nmax = a.nrx > a.tmv.cap ? a.nrx : a.tmv.cap;
  int np2 = 1;
  while (np2 < nmax) np2 <<= 1;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_frame_prep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(kSmallBuild * sizeof(unsigned long long)));
    attr = true;
  }
  size_t smem = (size_t)np2 * sizeof(unsigned long long);
  int smem_refit = nmax - 1 <= kSmemRefit ? 1 : 0;
  if (smem_refit) smem += (size_t)(nmax > 1 ? nmax - 1 : 1) * (12 * sizeof(float) + sizeof(int));
  k_frame_prep<<<2, 1024, smem, st>>>(a, np2, smem_refit);
  return cudaGetLastError();
}

// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the
// keys; the result is left in k0/v0 (k1/v1, hist are scratch).
cudaError_t sort_pairs_u32(unsigned* k0, unsigned* v0, unsigned* k1, unsigned* v1, unsigned* hist, int n,
                           int bits, cudaStream_t st) {
  int nb = (n + kRadixItems - 1) / kRadixItems;
  unsigned *ki = k0, *vi = v0, *ko = k1, *vo = v1;
  int passes = (bits + 7) / 8;
  for (int pass = 0; pass < passes; ++pass) {
    int shift = 8 * pass;
    k_radix_hist<<<nb, 256, 0, st>>>(ki, n, shift, hist, nb);
    scan_excl(hist, 256 * nb, hist + (size_t)256 * nb, st);
    k_radix_scatter<<<nb, 256, 0, st>>>(ki, vi, n, shift, hist, nb, ko, vo);
    unsigned* t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
  if (ki != k0) {
    cudaError_t e = cudaMemcpyAsync(k0, ki, sizeof(unsigned) * n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(v0, vi, sizeof(unsigned) * n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

void launch_tri_boxes(const float* d_v9, const int* d_sel, int n, float* d_prim, cudaStream_t st) {
  if (n > 0) k_tri_boxes<<<nblk(n, 256), 256, 0, st>>>(d_v9, d_sel, n, d_prim);
}

void launch_place_tris(const float* d_v9, const int* d_sel, const int* d_perm, const int* d_tri_mat,
                       const int* d_tri_obj, int n, int leaf_base, float4* d_tris, float4* d_objv,
                       int* d_slot_of_id, cudaStream_t st) {
  if (n > 0)
    k_place_tris<<<nblk(n, 256), 256, 0, st>>>(d_v9, d_sel, d_perm, d_tri_mat, d_tri_obj, n, leaf_base,
                                               d_tris, d_objv, d_slot_of_id);
}

void launch_quantize(const float4* d_nodes, int nn, const float* d_root_box, int has0, int has1, uint4* d_qn,
                     float* d_qframe, cudaStream_t st) {
  int g = (nn + 255) / 256;
  if (g < 1) g = 1;
  if (g > 1024) g = 1024;
  k_quantize<<<g, 256, 0, st>>>(d_nodes, nn, d_root_box, has0, has1, d_qn, d_qframe);
}


cudaError_t launch_bvh4_map(const float4* d_nodes, int nn, const int* d_roots, int4* d_kid4, int4* d_src4,
                            int* d_n4, int* d_roots4, int* d_scratch, cudaStream_t st) {
  size_t smem = bvh4_map_smem(nn);
  if (smem == 0 && !d_scratch) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_bvh4_map, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_bvh4_map<<<1, 1024, smem, st>>>(d_nodes, nn, d_roots, d_kid4, d_src4, d_n4, d_roots4,
                                    smem ? nullptr : d_scratch);
  return cudaGetLastError();
}

void launch_quantize4(const float4* d_nodes, int n4_bound, const int* d_n4, const int4* d_kid4, const int4* d_src4,
                      const float* d_root_box, int has0, int has1, uint4* d_q4, float* d_qframe, cudaStream_t st) {
  int g = (n4_bound + 255) / 256;
  if (g < 1) g = 1;
  if (g > 1024) g = 1024;
  k_quantize4<<<g, 256, 0, st>>>(d_nodes, d_n4, d_kid4, d_src4, d_root_box, has0, has1, d_q4, d_qframe);
}

size_t dyn_update_smem(int nd, int nobj) {
  int np2 = 1;
  while (np2 < nd) np2 <<= 1;
  size_t n = (size_t)(nd > 0 ? nd : 1), m = (size_t)(nd > 1 ? nd - 1 : 1);
  return (size_t)np2 * sizeof(unsigned long long) + n * 6 * sizeof(float) + m * 6 * sizeof(float) +
         m * 3 * sizeof(int) + (size_t)(kMaxLevels + 2) * sizeof(int) + (size_t)6 * nobj * sizeof(unsigned);
}

cudaError_t launch_dyn_update(const DynUpdateArgs& a, cudaStream_t st) {
  if (a.nd <= 0) return cudaSuccess;
  size_t smem = dyn_update_smem(a.nd, a.nobj);
  static size_t attr = 0;
  if (smem > attr) {
    cudaError_t e = cudaFuncSetAttribute(k_dyn_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = smem;
  }
  k_dyn_update<<<1, 1024, smem, st>>>(a);
  return cudaGetLastError();
}

void launch_transform_refit(const float4* d_objv, const float* d_xf, int n, int nobj, int node_base, int leaf_base,
                            float4* d_tris, float4* d_nodes, const int* d_leaf_parent, int* d_arrive,
                            float* d_root_box, unsigned* d_obj_box, DevCounters* d_ctr, cudaStream_t st) {
  if (n > 0)
    k_transform_refit<<<nblk(n, 256), 256, 0, st>>>(d_objv, d_xf, n, nobj, node_base, leaf_base, d_tris, d_nodes,
                                                    d_leaf_parent, d_arrive, d_root_box, d_obj_box, d_ctr);
}

DCEM_CHECKS_TAKER(checks_take_bvh)

}  // namespace dcem
