// bvh.cuh -- host launchers of the LBVH build and per-frame refit.
#pragma once

#include "dcem_internal.cuh"

namespace dcem {

// Device scratch of the multi-CTA build path (trees above kSmallBuild leaves).
struct BuildScratch {
  unsigned* bounds = nullptr;           // 6
  unsigned *k0 = nullptr, *v0 = nullptr, *k1 = nullptr, *v1 = nullptr;  // n each
  unsigned* hist = nullptr;             // 256 * ceil(n / 1024)
  unsigned long long* keys = nullptr;   // n
};

// Builds one tree over n primitive boxes d_prim (n x 6: lo.xyz, hi.xyz) with
// internal nodes [node_base, node_base + n - 1) and leaf slots
// [leaf_base, leaf_base + n). Writes the leaf order (d_perm[j] = primitive of
// leaf j), parents, child boxes, the root code and the root box.
cudaError_t build_tree(const float* d_prim, int n, int node_base, int leaf_base, float4* d_nodes,
                       int* d_leaf_parent, int* d_perm, int* d_arrive, int* d_root, float* d_root_box,
                       BuildScratch& scr, cudaStream_t st);

// Boxes of triangles v9[sel[i]] (9 floats each).
void launch_tri_boxes(const float* d_v9, const int* d_sel, int n, float* d_prim, cudaStream_t st);

// Places triangles in leaf order; objv (optional) receives object-space
// vertices with the object id in v0.w.
void launch_place_tris(const float* d_v9, const int* d_sel, const int* d_perm, const int* d_tri_mat,
                       const int* d_tri_obj, int n, int leaf_base, float4* d_tris, float4* d_objv,
                       int* d_slot_of_id, cudaStream_t st);

// Per frame: world vertices of the moving triangles, per-object boxes and the
// bottom-up refit of their tree (d_arrive zeroed by the caller).
void launch_transform_refit(const float4* d_objv, const float* d_xf, int n, int nobj, int node_base,
                            int leaf_base, float4* d_tris, float4* d_nodes, const int* d_leaf_parent,
                            int* d_arrive, float* d_root_box, unsigned* d_obj_box, DevCounters* d_ctr,
                            cudaStream_t st);

}  // namespace dcem
