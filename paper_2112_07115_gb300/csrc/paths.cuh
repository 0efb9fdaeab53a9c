// paths.cuh -- arguments and launchers of dedupe, validation and reduction.
#pragma once

#include "dcem_internal.cuh"

namespace dcem {

struct PathArgs {
  int R;                          // segment-log stride (rays, plus child slots with transmission)
  const int* log_id;              // (N+1) x R hit ids
  const Cand* cand;
  unsigned cand_cap;
  unsigned long long* hkey;       // hash slots: 64-bit key, 0 = empty
  unsigned long long* hrep;       // (ray << 32 | candidate) of the representative, ~0 = none
  unsigned hcap;                  // power of two
  int* cand_slot;                 // per candidate
  int* uniq;                      // representative candidate per distinct key
  unsigned ucap;
  PathRec* prec;                  // per distinct key
  const int* ray_perm;            // ray slot -> caller's ray index
  double* vpts;                   // per distinct key: (kMaxRefl + 2) FP64 path points
  int* vstate;                    // per distinct key: 0 invalid, 1 valid so far, 2 occluded
  int N;                          // reflections (sub-segments per path <= N + max_trans + 1)
  int max_trans;                  // transmissions per path (ids with kTransBit)
  int R0;                         // primary rays; slots from R0 on are transmission children
  const int* inst_root;           // per child slot: its primary ray's slot
  int* bucket;                    // links x bucket_cap distinct-key indices of valid paths
  unsigned* bucket_cnt;           // links (link = transmitter * nrx + receiver)
  int bucket_cap;                 // power of two
  unsigned* link_off;             // links: output offset of each link's paths (many links), or null
  dcem_path* pout;                // ordered output (link, key): caller's device buffer or staging
  unsigned pout_cap;
  double* out_field;              // links x 2 (re, im), or null
  double* out_pc;                 // links P_coh dBm, or null
  double* out_pi;                 // links P_inc dBm, or null
  const float4* tris;             // leaf-ordered triangles
  const int* slot_of_id;
  const float4* mats;             // eps_r, sigma, pec
  Bvh bvh;
  const float4* rx;               // nrx receivers
  int nrx;
  const float4* txs;              // per transmitter: position (xyz)
  float3 pol;
  float eps_occ;
  int prec_df;                    // 1: validation geometry in double-float, 0: FP64
  double freq, tx_power;
  DevCounters* ctr;
  // sticky mode (null otherwise): the previous frame's valid paths, to be
  // re-validated when no capture of this frame has their key, and the
  // buffer that keeps this frame's valid paths for the next one
  // first-order edge diffraction (null: off)
  Wedge* wedges;                  // geometry, rebuilt every frame from the world triangles
  WedgeF* wf;                     // the same in FP32 (pre-tests)
  const WedgeTopo* wtopo;
  int nw;
  // wedge clusters: the wedges in a fixed spatial order (wperm), 32 per
  // cluster, and each cluster's box of its edges (6 floats, every frame)
  const int* wperm;
  float* wcbox;
  int nwc;
  unsigned long long* dsurv;      // (link, wedge) pair indices past the FP32 pre-test
  unsigned dsurv_cap;
  // one reflection before or after a diffraction (null: off): reflector
  // planes and their member triangle ids
  const RPlane* rplanes;
  const int* rmembers;             // per plane its members, sorted by their lowest coordinate
  const float* rkeys;              // along the plane's axis, and that coordinate
  int nrp;
  int drefl2;                     // 1: also two reflections around a first-order diffraction
  unsigned* rmask;                // with drefl2: the wedge masks of k_refl2_masks, one word per
                                  // (end point: transmitters then receivers, plane or none, cluster)
  int dmid;                       // 1: also a reflection between the two wedges of an order-2 chain
  // diffraction of order 2 and 3 (diff_order <= 1: off): the wedge pairs
  // (v, w1, w2, -1), the pairs with a reflection on plane p between them
  // (t, w1, w2, -2 - p) and triples (v, w1, w2, w3) of the frame, v a source
  // (a transmitter, or with reflector planes the image of transmitter t in
  // plane p: v = dntx + t * nrpr + p), and the pair relation as a bit matrix
  // (nw x nw bits)
  int diff_order;
  int dntx;                       // transmitters (set by launch_diffract)
  int nrpr;                       // reflector planes applied to chains (0: none; set by launch_diffract)
  int4* dseq2;
  unsigned dseq2_cap;
  int4* dseq3;
  unsigned dseq3_cap;
  unsigned* drel;
  // validation reuse (coherent frames; Sec. III "Propagation path caching"):
  // the previous frame's records of its distinct keys, found through a hash
  // table of their link keys, are copied when nothing they depend on moved
  int reuse;                      // 1: look the keys up in the previous frame's table
  const unsigned long long* vc_prev_key;  // previous table: link key (0 = empty) and record index
  const unsigned* vc_prev_u;
  const PathRec* prev_prec;       // the previous frame's records, points and states
  const double* prev_vpts;
  const int* prev_vstate;
  unsigned vc_cap;                // slots of each table (power of two)
  unsigned long long* vc_next_key;  // this frame's table (built after validation), or null
  unsigned* vc_next_u;
  unsigned long long* ckey;       // per distinct key of this frame: its link key
  const unsigned char* rx_moved;  // receivers whose position changed
  const unsigned char* obj_moved; // rigid objects whose transform changed
  const int* tri_obj;             // triangle id -> rigid object (-1 static)
  SmallBvh mvt;                   // the moved objects' old and new boxes
  unsigned mv_cap;                // boxes the tree holds (more moved boxes: no reuse)
  const StickyKey* sticky_prev;
  const unsigned* sticky_prev_n;
  unsigned sticky_cap;
  StickyKey* sticky_next;
};

cudaError_t launch_dedupe(const PathArgs& a, int grid, cudaStream_t st);
// Sticky mode: the previous frame's valid paths whose key no capture of this
// frame has join the distinct keys (validated like them).
cudaError_t launch_sticky_probe(const PathArgs& a, int grid, cudaStream_t st);
cudaError_t launch_validate(const PathArgs& a, int grid, cudaStream_t st);
// The table of this frame's distinct keys for the next frame's validation
// reuse (after validation, before diffraction adds its records).
cudaError_t launch_vcache_build(const PathArgs& a, int grid, cudaStream_t st);
// First-order edge diffraction paths of every (link, wedge) (after validation).
cudaError_t launch_diffract(const PathArgs& a, int nlinks, int sms, cudaStream_t st);
// Per-link sums and ordered output; links above kScanLinks take their output
// offsets from a scan (a.link_off) instead of summing the lower links' counts.
constexpr int kScanLinks = 4096;
cudaError_t launch_reduce(const PathArgs& a, int nlinks, cudaStream_t st);

}  // namespace dcem
