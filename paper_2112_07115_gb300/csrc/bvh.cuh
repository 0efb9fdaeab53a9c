// bvh.cuh -- host launchers of the LBVH build and per-frame refit.
#pragma once

#include "dcem_internal.cuh"

namespace dcem {

// Device scratch of the multi-CTA build path (trees above kSmallBuild leaves).
struct BuildScratch {
  unsigned* bounds = nullptr;           // 6
  unsigned *k0 = nullptr, *v0 = nullptr, *k1 = nullptr, *v1 = nullptr;  // n each
  unsigned* hist = nullptr;             // radix_hist_size(n)
  unsigned long long* keys = nullptr;   // n
};

// Builds one tree over n primitive boxes d_prim (n x 6: lo.xyz, hi.xyz) with
// internal nodes [node_base, node_base + n - 1) and leaf slots
// [leaf_base, leaf_base + n). Writes the leaf order (d_perm[j] = primitive of
// leaf j), parents, child boxes, the root code and the root box.
cudaError_t build_tree(const float* d_prim, int n, int node_base, int leaf_base, float4* d_nodes,
                       int* d_leaf_parent, int* d_perm, int* d_arrive, int* d_root, float* d_root_box,
                       BuildScratch& scr, cudaStream_t st);

// A small per-frame tree (receivers, moved-object boxes) built by one CTA:
// n primitives (or min(*n_dev, cap) when n_dev is set), nodes [0, n-1),
// leaves [0, n) with leaf j holding primitive perm[j].
struct SmallTreeArgs {
  const float* prim = nullptr;
  int n = 0;
  const unsigned* n_dev = nullptr;
  int cap = 0;
  float4* nodes = nullptr;
  int* leaf_parent = nullptr;
  int* perm = nullptr;
  int* arrive = nullptr;
  int* root = nullptr;
  float* root_box = nullptr;
};

// Per-frame preparation in one launch of two CTAs.
//   CTA 0: receivers -> float4 + point boxes, finiteness check, moved flags
//          and list (bitwise against the cached frame when have_prev), zero
//          the per-receiver path counters, then build the receiver tree.
//   CTA 1: (coherent frames) objects whose transform changed -> their old and
//          new world boxes (widened by 1 mm + 1e-5 relative), then build the
//          tree over those boxes.
struct FramePrepArgs {
  const float* rx3 = nullptr;
  int nrx = 0;
  float4* rx_cur = nullptr;
  const float4* rx_traced = nullptr;
  int have_prev = 0;
  unsigned char* rx_moved = nullptr;
  int* moved_list = nullptr;
  float* rx_prim = nullptr;
  unsigned* bucket_cnt = nullptr;
  int coherent = 0;
  int nobj = 0;
  const float* xf_cur = nullptr;
  const float* xf_traced = nullptr;
  const unsigned* obj_box_cur = nullptr;
  const unsigned* obj_box_traced = nullptr;
  float* moved_boxes = nullptr;
  unsigned char* obj_moved = nullptr;  // nobj flags: transform changed (coherent frames)
  DevCounters* ctr = nullptr;
  SmallTreeArgs trx, tmv;
};

cudaError_t launch_frame_prep(const FramePrepArgs& a, cudaStream_t st);

// Counts of scratch the scan of m histogram entries needs beyond them.
size_t scan_scratch_size(size_t m);
// Counts in the radix sort's histogram buffer for n pairs: the histogram and
// its scan scratch.
inline size_t radix_hist_size(int n) {
  size_t m = (size_t)256 * ((n + 1023) / 1024);
  return m + scan_scratch_size(m);
}

// Stable radix sort of n (key, value) pairs by the low `bits` key bits; the
// sorted pairs end in k0/v0 (k1, v1: n scratch each; hist: radix_hist_size(n)).
cudaError_t sort_pairs_u32(unsigned* k0, unsigned* v0, unsigned* k1, unsigned* v1, unsigned* hist, int n,
                           int bits, cudaStream_t st);

// Boxes of triangles v9[sel[i]] (9 floats each).
void launch_tri_boxes(const float* d_v9, const int* d_sel, int n, float* d_prim, cudaStream_t st);

// Places triangles in leaf order; objv (optional) receives object-space
// vertices with the object id in v0.w.
void launch_place_tris(const float* d_v9, const int* d_sel, const int* d_perm, const int* d_tri_mat,
                       const int* d_tri_obj, int n, int leaf_base, float4* d_tris, float4* d_objv,
                       int* d_slot_of_id, cudaStream_t st);

// Per frame, for at most kSmemRefit + 1 moving triangles, in one CTA: world
// vertices (fmaf transform), per-object world boxes, an optional rebuild of
// the tree over the current positions (rebuild != 0), the bottom-up refit in
// shared memory, and the tree's surface-area cost (sum of node areas over
// the root area) in uctr->sah_refit (and sah_build after a rebuild).
struct DynUpdateArgs {
  const float4* objv_src = nullptr;  // primitive order, object space, object id in v0.w
  float4* objv = nullptr;            // leaf order
  const int* sel_d = nullptr;        // primitive -> triangle id
  const int* tri_mat = nullptr;      // triangle id -> material
  const float* xf = nullptr;         // nobj x 12
  float* prim = nullptr;             // scratch: nd x 6 boxes (rebuild)
  int nd = 0, nobj = 0, node_base = 0, leaf_base = 0, rebuild = 0;
  float4* tris = nullptr;
  float4* nodes = nullptr;
  int* leaf_parent = nullptr;
  int* perm = nullptr;
  int* slot_of_id = nullptr;
  unsigned* obj_box = nullptr;       // lo [0, 3 nobj), hi [3 nobj, 6 nobj) as ordered ints
  float* root_box = nullptr;
  int* root = nullptr;
  int* sched = nullptr;              // nd - 1 node indices by height (kept between rebuilds)
  int* lvl = nullptr;                // kDynLevels + 2: starts of each height, then their count
  DevCounters* uctr = nullptr;
};
constexpr int kDynLevels = 128;      // heights the scheduled refit handles (Karras trees over
                                     // 64-bit keys have at most 63)
cudaError_t launch_dyn_update(const DynUpdateArgs& a, cudaStream_t st);
// Shared memory the one-CTA update needs (must stay within 227 KB).
size_t dyn_update_smem(int nd, int nobj);

// Compact copy of the nn nodes of both trees (2 uint4 per node) and its
// frame (origin.xyz, step.xyz), from the current node boxes and root boxes.
void launch_quantize(const float4* d_nodes, int nn, const float* d_root_box, int has0, int has1, uint4* d_qn,
                     float* d_qframe, cudaStream_t st);

// 4-wide compact copy: map the binary trees (nn internal nodes, 2 root codes)
// to 4-wide nodes once per topology (one CTA, nn <= 8192), then encode the
// child boxes every frame. n4 and the 4-wide roots stay on the device.
// Shared memory of the 4-wide mapping of nn binary internal nodes, or 0 when
// it needs the global scratch (3 nn ints) instead.
inline size_t bvh4_map_smem(int nn) {
  size_t b = 3 * (size_t)(nn > 0 ? nn : 1) * sizeof(int);
  return b <= 200 * 1024 ? b : 0;
}
cudaError_t launch_bvh4_map(const float4* d_nodes, int nn, const int* d_roots, int4* d_kid4, int4* d_src4,
                            int* d_n4, int* d_roots4, int* d_scratch, cudaStream_t st);
void launch_quantize4(const float4* d_nodes, int n4_bound, const int* d_n4, const int4* d_kid4, const int4* d_src4,
                      const float* d_root_box, int has0, int has1, uint4* d_q4, float* d_qframe, cudaStream_t st);
// At most (2 + 2 nn) / 3 internal nodes of two trees lie at even depth.
inline int bvh4_bound(int nn) { return (2 + 2 * nn) / 3; }

// Per frame: world vertices of the moving triangles, per-object boxes and the
// bottom-up refit of their tree (d_arrive zeroed by the caller).
void launch_transform_refit(const float4* d_objv, const float* d_xf, int n, int nobj, int node_base,
                            int leaf_base, float4* d_tris, float4* d_nodes, const int* d_leaf_parent,
                            int* d_arrive, float* d_root_box, unsigned* d_obj_box, DevCounters* d_ctr,
                            cudaStream_t st);

}  // namespace dcem
