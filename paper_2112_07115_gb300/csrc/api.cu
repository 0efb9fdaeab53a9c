// api.cu -- the C ABI (include/dcem.h): scene state, device buffers and the
// per-frame orchestration of the kernels on the scene's stream.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <array>
#include <vector>

#include "bvh.cuh"
#include "paths.cuh"
#include "grad.cuh"
#include "trace.cuh"

using namespace dcem;

namespace {

template <class T>
cudaError_t dalloc(T** p, size_t n) {
  *p = nullptr;
  return cudaMalloc((void**)p, (n > 0 ? n : 1) * sizeof(T));
}
template <class T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return DCEM_OK;
  if (e == cudaErrorMemoryAllocation) return DCEM_ERR_NOMEM;
  return DCEM_ERR_CUDA;
}

#define CK(x)                              \
  do {                                     \
    cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) {               \
      cudaGetLastError();                  \
      return status_of(e_);                \
    }                                      \
  } while (0)

unsigned pow2_at_least(unsigned long long v) {
  unsigned long long p = 1;
  while (p < v) p <<= 1;
  return (unsigned)p;
}

// End of a frame in one launch: the state the next frame compares against
// (receiver positions, transforms, object boxes, capture count) and both
// counter blocks written straight to mapped host memory; the update
// counters are cleared for the next update.
__global__ void k_frame_end(const float4* __restrict__ rx_cur, float4* rx_traced, int nrx,
                            const float* __restrict__ xf_cur, float* xf_traced,
                            const unsigned* __restrict__ box_cur, unsigned* box_traced, int nobj,
                            const DevCounters* __restrict__ ctr, DevCounters* uctr, unsigned* prev_ncand,
                            DevCounters* host) {
  int i0 = blockIdx.x * blockDim.x + threadIdx.x, step = gridDim.x * blockDim.x;
  for (int i = i0; i < nrx; i += step) rx_traced[i] = rx_cur[i];
  for (int i = i0; i < 12 * nobj; i += step) xf_traced[i] = xf_cur[i];
  for (int i = i0; i < 6 * nobj; i += step) box_traced[i] = box_cur[i];
  if (blockIdx.x == 0) {
    constexpr int W = sizeof(DevCounters) / sizeof(unsigned);
    const unsigned* a = reinterpret_cast<const unsigned*>(ctr);
    unsigned* b = reinterpret_cast<unsigned*>(uctr);
    unsigned* ha = reinterpret_cast<unsigned*>(host);
    unsigned* hb = reinterpret_cast<unsigned*>(host + 1);
    for (int k = threadIdx.x; k < W; k += blockDim.x) {
      ha[k] = a[k];
      hb[k] = b[k];
    }
    if (threadIdx.x == 0) *prev_ncand = ctr->n_cand;
    __syncthreads();
    for (int k = threadIdx.x; k < W; k += blockDim.x) b[k] = 0u;
  }
}

// Object-space vertices of the moving triangles: (v0, object), (v1, triangle
// id), (v2, material); the last two are the .w of the world triangle record.
__global__ void k_objv_src(const float* __restrict__ v9, const int* __restrict__ sel,
                           const int* __restrict__ tri_obj, const int* __restrict__ tri_mat, int n,
                           float4* objv_src) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int gid = sel[i];
    const float* v = v9 + 9 * (size_t)gid;
    objv_src[3 * (size_t)i] = make_float4(v[0], v[1], v[2], __int_as_float(tri_obj[gid]));
    objv_src[3 * (size_t)i + 1] = make_float4(v[3], v[4], v[5], __int_as_float(gid));
    objv_src[3 * (size_t)i + 2] = make_float4(v[6], v[7], v[8], __int_as_float(tri_mat[gid]));
  }
}

// world vertices of the moving triangles in primitive order (for a rebuild)
__global__ void k_xform_prims(const float4* __restrict__ objv_src, const float* __restrict__ xf, int n,
                              float* v9) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float* m = xf + 12 * (size_t)__float_as_int(objv_src[3 * (size_t)i].w);
    for (int k = 0; k < 3; ++k) {
      float4 p = objv_src[3 * (size_t)i + k];
      for (int r = 0; r < 3; ++r)
        v9[9 * (size_t)i + 3 * k + r] =
            __fmaf_rn(m[4 * r], p.x, __fmaf_rn(m[4 * r + 1], p.y, __fmaf_rn(m[4 * r + 2], p.z, m[4 * r + 3])));
    }
  }
}

__global__ void k_place_dyn(const float* __restrict__ v9, const float4* __restrict__ objv_src,
                            const int* __restrict__ perm, const int* __restrict__ sel,
                            const int* __restrict__ tri_mat, int n, int leaf_base, float4* tris, float4* objv,
                            int* slot_of_id) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    int i = perm[j];
    int gid = sel[i];
    const float* v = v9 + 9 * (size_t)i;
    int slot = leaf_base + j;
    tris[3 * (size_t)slot] = make_float4(v[0], v[1], v[2], __int_as_float(gid));
    tris[3 * (size_t)slot + 1] = make_float4(v[3], v[4], v[5], __int_as_float(tri_mat[gid]));
    tris[3 * (size_t)slot + 2] = make_float4(v[6], v[7], v[8], 0.0f);
    for (int k = 0; k < 3; ++k) objv[3 * (size_t)j + k] = objv_src[3 * (size_t)i + k];
    slot_of_id[gid] = slot;
  }
}

__device__ __forceinline__ unsigned spread16(unsigned v) {
  v &= 0xffffu;
  v = (v | (v << 8)) & 0x00ff00ffu;
  v = (v | (v << 4)) & 0x0f0f0f0fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

// Direction-coherence key of each ray: 2D Morton code of its octahedral map.
__global__ void k_ray_keys(const float4* __restrict__ d, int n, unsigned* keys, unsigned* idx) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float4 v = d[i];
    float l1 = fabsf(v.x) + fabsf(v.y) + fabsf(v.z);
    float x = v.x / l1, y = v.y / l1;
    if (v.z < 0.0f) {
      float fx = (1.0f - fabsf(y)) * (x >= 0.0f ? 1.0f : -1.0f);
      float fy = (1.0f - fabsf(x)) * (y >= 0.0f ? 1.0f : -1.0f);
      x = fx;
      y = fy;
    }
    unsigned qu = (unsigned)fminf(fmaxf((x + 1.0f) * 32767.5f, 0.0f), 65535.0f);
    unsigned qv = (unsigned)fminf(fmaxf((y + 1.0f) * 32767.5f, 0.0f), 65535.0f);
    keys[i] = (spread16(qu) << 1) | spread16(qv);
    idx[i] = (unsigned)i;
  }
}

// Sort key of the second pass: the set of the ray at each sorted position.
__global__ void k_set_keys(const float4* __restrict__ src, const unsigned* __restrict__ idx, int n,
                           unsigned* keys) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    keys[i] = __float_as_uint(src[idx[i]].w);
}

__global__ void k_gather_rays(const float4* __restrict__ src, const unsigned* __restrict__ idx, int n,
                              float4* dst, int* perm) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    unsigned j = idx[i];
    dst[i] = src[j];
    perm[i] = (int)j;
  }
}

}  // namespace

// Everything one frame enqueues is fixed by this plan: the kernels' argument
// blocks, the launch shapes they imply and the switches below. Two frames with
// byte-equal plans enqueue the same work, so a plan seen before replays the
// CUDA graph captured from it (one launch) instead of ~16 stream operations.
// The struct is zero-filled before it is set, so its padding compares equal.
struct FramePlan {
  int32_t coherent, tm, tk, use_q, nrx, R, has0, has1, q4_bound, nobj, ptr_dev, nsets, nlinks, sticky;
  TraceArgs a;
  FramePrepArgs fp;
  CoherentArgs c;
  PathArgs q;
  // quantisation and end-of-frame arguments (scene buffers)
  const float4* nodes;
  int* q4_count;
  int4* q4_kid;
  int4* q4_src;
  float* root_box;
  uint4* qnodes;
  float* qframe;
  float4 *rx_cur, *rx_traced;
  float *xf_cur, *xf_traced;
  unsigned *obj_box_cur, *obj_box_traced, *prev_ncand;
  DevCounters *ctr, *uctr, *ctr_hd;
  float4* txs;           // transmitters (device), copied from the pinned txs_h
  const float4* txs_h;
  unsigned* bucket_cnt;  // cleared by a memset when there are more links than receivers
  unsigned* sticky_n_next;  // sticky mode: this frame's kept-path count (persistent)
  cudaEvent_t ev[10];
  cudaStream_t side;     // second branch of the frame (compact copy, end-of-frame state)
  cudaEvent_t br[4];     // its fork and join events
};

struct FrameGraph {
  FramePlan key;
  bool have_key = false;
  cudaGraph_t graph = nullptr;     // the captured frame (also a child of batch graphs)
  cudaGraphExec_t exec = nullptr;  // its instantiation for single-scene replay
  unsigned long long gen = 0;      // capture number (identifies the graph in batch graphs)
  void drop() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  }
};

struct dcem_scene {
  int device = 0;
  int sms = 1;
  cudaStream_t st = nullptr;
  int ntri = 0, nobj = 0, nmat = 0, ns = 0, nd = 0, nint_s = 0, nint_d = 0;
  // geometry and hierarchy
  float4* tris = nullptr;
  int* slot_of_id = nullptr;
  float4* objv = nullptr;       // moving triangles, leaf order, object space
  float4* objv_src = nullptr;   // moving triangles, primitive order, object space
  int* sel_d = nullptr;         // primitive -> triangle id (moving tree)
  int* tri_mat_d = nullptr;
  float* v9d = nullptr;         // world vertices of moving primitives (rebuilds)
  float4* nodes = nullptr;
  uint4* qnodes = nullptr;       // 4-wide compact node copy for shared-memory traversal
  float* qframe = nullptr;
  int4* q4_kid = nullptr;        // 4-wide mapping of the binary trees: children, box sources,
  int4* q4_src = nullptr;        // node count and roots (rebuilt with the topology)
  int* q4_count = nullptr;
  int* q4_roots = nullptr;
  int* q4_scr = nullptr;         // scratch of the 4-wide mapping of large trees
  int* leaf_parent = nullptr;
  int* tri_obj_d = nullptr;  // triangle id -> rigid object (-1 static)
  std::vector<float> tris_h;   // input vertices (static ones are world space) and objects,
  std::vector<int> tri_obj_h;  // kept for the wedge search of edge diffraction
  Wedge* wedges = nullptr;     // first-order diffraction: wedge geometry (per frame)
  WedgeF* wedgesf = nullptr;   // ... the same in FP32
  WedgeTopo* wtopo = nullptr;  // ... and topology
  int nw = 0;
  int* wperm = nullptr;        // wedge clusters: the wedges in spatial order, 32 per cluster,
  float* wcbox = nullptr;      // and the clusters' boxes (per frame)
  int nwc = 0;
  bool diffraction = false;
  unsigned long long* dsurv = nullptr;  // diffraction: pre-test survivor list
  RPlane* rplanes = nullptr;   // diffraction combined with a reflection: reflector planes
  int* rmembers = nullptr;     // ... their triangle ids and sort keys
  float* rkeys = nullptr;
  int nrp = 0;
  int diff_refl = 0;               // reflections with diffraction (0..3, see the header)
  unsigned* rmask = nullptr;   // two reflections: the pre-test's wedge masks, and their words
  size_t rmask_cap = 0;
  unsigned dsurv_cap = 0;
  int diff_order = 1;          // diffraction: most wedges on one path (1-3)
  int4* dseq2 = nullptr;       // ... the frame's wedge pairs and triples, the pair relation
  int4* dseq3 = nullptr;
  unsigned dseq2_cap = 0, dseq3_cap = 0;
  unsigned* drel = nullptr;
  double2* g_items = nullptr;  // field derivatives: per-item results, their parameter,
  int* g_param = nullptr;      // staged outputs and the error flag (dcem_path_gradients)
  double* g_out = nullptr;
  unsigned* g_err = nullptr;
  size_t g_items_cap = 0, g_out_cap = 0;
  dcem_path* g_paths = nullptr;
  double* g_theta = nullptr;   // adjoint: theta staged from the host
  size_t g_theta_cap = 0;
  float4* g_rx = nullptr;
  size_t g_paths_cap = 0, g_rx_cap = 0;
  int* dsched = nullptr;  // moving-object tree: nodes by height, and the height bounds
  int* dlvl = nullptr;
  int* arrive = nullptr;
  int* roots = nullptr;
  float* root_box = nullptr;
  int* perm = nullptr;
  float* prim = nullptr;
  float4* mats = nullptr;
  float* xf_cur = nullptr;
  float* xf_traced = nullptr;
  unsigned* obj_box_cur = nullptr;
  unsigned* obj_box_traced = nullptr;
  float* moved_boxes = nullptr;
  BuildScratch scr;
  int root_h[2] = {kEmpty, kEmpty};
  bool dyn_on_world = false;
  float rebuild_ratio = 1.25f;   // rebuild the moving-object tree above this cost ratio
  float sah_build = 0.0f, sah_now = 0.0f;
  bool rebuilt_since_frame = false;
  DevCounters* ctr = nullptr;
  DevCounters* uctr = nullptr;  // errors raised by per-frame updates
  DevCounters* ctr_h = nullptr; // pinned, mapped: [0] frame counters, [1] update counters
  DevCounters* ctr_hd = nullptr; // device address of ctr_h
  // rays and segment log
  bool rays_set = false;
  int R = 0;
  float4* rays = nullptr;        // sorted by direction: slot order
  int* ray_perm = nullptr;       // slot -> caller's ray index
  std::vector<int> ray_perm_h;
  int nsets = 0;                 // ray sets (transmitters); rays[].w holds the set
  std::vector<int> set_rays_h;   // rays per set
  float4* txs = nullptr;         // per set: transmitter xyz and capture spacing (device)
  float4* txs_h = nullptr;       // the same, pinned host staging copied in every frame
  int logW = 0;                  // segments per slot in the log
  int LS = 0;                    // log stride: R + child_cap
  int max_trans = 0;             // transmission: per path (0 = off)
  int child_cap = 0;             // child-ray slots after the R primaries
  int* inst = nullptr;           // per child slot: reflections | transmissions << 4 | set << 8
  int* inst_root = nullptr;      // per child slot: its primary ray's slot
  std::vector<float4> mats_h;    // host copy of the material table
  float4* log_o = nullptr;
  float4* log_d = nullptr;
  int* log_id = nullptr;
  unsigned* capitems = nullptr;  // segments traced this frame: ray << 4 | segment
  int* nseg = nullptr;
  int* restart = nullptr;
  int* queue = nullptr;
  // captures and distinct paths
  Cand* cand[2] = {nullptr, nullptr};
  unsigned cand_cap = 0;
  int cur = 0;
  unsigned* prev_ncand = nullptr;
  unsigned long long* hkey = nullptr;
  unsigned long long* hrep = nullptr;
  unsigned hcap = 0;
  int* cand_slot = nullptr;
  int* uniq = nullptr;
  unsigned ucap = 0;
  PathRec* prec = nullptr;      // per distinct key (two buffers by frame parity: this
  double* vpts = nullptr;       // frame's and the previous frame's, for validation reuse)
  int* vstate = nullptr;
  PathRec* prec_b = nullptr;
  double* vpts_b = nullptr;
  int* vstate_b = nullptr;
  unsigned long long* ckey = nullptr;      // per distinct key: its link key
  unsigned long long* vc_key[2] = {nullptr, nullptr};  // link key -> record index tables,
  unsigned* vc_u[2] = {nullptr, nullptr};              // one per parity
  unsigned vc_cap = 0;
  bool vc_valid = false;        // the previous frame built its table (parity s->cur)
  unsigned char* obj_moved = nullptr;  // per rigid object: transform changed this frame
  dcem_path* pout = nullptr;
  StickyKey* sticky[2] = {nullptr, nullptr};  // sticky mode: kept paths (by parity)
  unsigned* sticky_n = nullptr;               // their counts (device, by parity)
  // receivers
  int nrx_cap = 0;
  float* rx3 = nullptr;
  float4* rx_cur = nullptr;
  float4* rx_traced = nullptr;
  unsigned char* rx_moved = nullptr;
  int* moved_list = nullptr;
  int* bucket = nullptr;
  unsigned* bucket_cnt = nullptr;
  int bucket_cap = 1024;
  int nlink_cap = 0;             // links (transmitter-receiver pairs) the arrays below hold
  unsigned* link_off = nullptr;  // per link output offset (many links)
  double* rxout = nullptr;
  // per-frame trees over the receivers and over the moved-object boxes
  float* rx_prim = nullptr;
  float4* rxt_nodes = nullptr;
  int *rxt_parent = nullptr, *rxt_perm = nullptr, *rxt_arrive = nullptr, *rxt_root = nullptr;
  float* rxt_root_box = nullptr;
  float4* mvt_nodes = nullptr;
  int *mvt_parent = nullptr, *mvt_perm = nullptr, *mvt_arrive = nullptr, *mvt_root = nullptr;
  float* mvt_root_box = nullptr;
  int mv_cap = 0;
  // coherence cache
  bool cache_valid = false;
  dcem_params cparams;
  std::vector<float> ctx;        // transmitters of the cached frame
  int cnrx = -1;
  unsigned last_ncand = 0;
  cudaEvent_t ev[10] = {};
  cudaStream_t side = nullptr;   // the frame's second branch (see enqueue_frame)
  cudaEvent_t br[4] = {};
  int launches = 0;  // kernels launched since the last completed frame
  int last_use_q = 0;  // closest-hit kernel of the last frame (TraceArgs::use_q)
  // closest-hit configuration (dcem_scene_set_trace_config / dcem_scene_autotune)
  int tc_kernel = -1, tc_block = 256, tc_stack = kStackTrace;
  // graph replay of the frame's device work (see FramePlan)
  FramePlan plan;
  FrameGraph fgraph[2];
  cudaStream_t cap_st = nullptr;
  bool use_graphs = true;
  int graph_replayed = 0;
};

namespace {

void scene_free(dcem_scene* s) {
  if (!s) return;
  cudaStreamSynchronize(s->st);
  dfree(s->tris); dfree(s->slot_of_id); dfree(s->objv); dfree(s->objv_src); dfree(s->sel_d);
  dfree(s->tri_mat_d); dfree(s->v9d); dfree(s->nodes); dfree(s->qnodes); dfree(s->qframe);
  dfree(s->q4_kid); dfree(s->q4_src); dfree(s->q4_count); dfree(s->q4_roots); dfree(s->q4_scr); dfree(s->leaf_parent); dfree(s->arrive);
  dfree(s->dsched); dfree(s->dlvl); dfree(s->tri_obj_d); dfree(s->wedges); dfree(s->wedgesf); dfree(s->wtopo);
  dfree(s->wperm); dfree(s->wcbox); dfree(s->dsurv);
  dfree(s->rplanes); dfree(s->rmembers); dfree(s->rkeys); dfree(s->rmask);
  dfree(s->dseq2); dfree(s->dseq3); dfree(s->drel);
  dfree(s->g_items); dfree(s->g_param); dfree(s->g_out); dfree(s->g_err); dfree(s->g_paths);
  dfree(s->g_rx); dfree(s->g_theta);
  dfree(s->roots); dfree(s->root_box); dfree(s->perm); dfree(s->prim); dfree(s->mats);
  dfree(s->xf_cur); dfree(s->xf_traced); dfree(s->obj_box_cur); dfree(s->obj_box_traced);
  dfree(s->moved_boxes); dfree(s->scr.bounds); dfree(s->scr.k0); dfree(s->scr.v0); dfree(s->scr.k1);
  dfree(s->scr.v1); dfree(s->scr.hist); dfree(s->scr.keys); dfree(s->ctr); dfree(s->uctr);
  if (s->ctr_h) cudaFreeHost(s->ctr_h);
  dfree(s->inst); dfree(s->inst_root);
  dfree(s->rays); dfree(s->ray_perm); dfree(s->log_o); dfree(s->log_d); dfree(s->log_id); dfree(s->capitems); dfree(s->nseg); dfree(s->restart);
  dfree(s->queue); dfree(s->cand[0]); dfree(s->cand[1]); dfree(s->prev_ncand); dfree(s->hkey);
  dfree(s->hrep); dfree(s->cand_slot); dfree(s->uniq); dfree(s->prec); dfree(s->pout); dfree(s->rx3);
  dfree(s->vpts); dfree(s->vstate); dfree(s->sticky[0]); dfree(s->sticky[1]); dfree(s->sticky_n);
  dfree(s->prec_b); dfree(s->vpts_b); dfree(s->vstate_b); dfree(s->ckey); dfree(s->vc_key[0]);
  dfree(s->vc_key[1]); dfree(s->vc_u[0]); dfree(s->vc_u[1]); dfree(s->obj_moved);
  dfree(s->rx_cur); dfree(s->rx_traced); dfree(s->rx_moved); dfree(s->moved_list); dfree(s->bucket);
  dfree(s->bucket_cnt); dfree(s->rxout); dfree(s->link_off); dfree(s->txs);
  if (s->txs_h) cudaFreeHost(s->txs_h);
  dfree(s->rx_prim); dfree(s->rxt_nodes); dfree(s->rxt_parent); dfree(s->rxt_perm); dfree(s->rxt_arrive);
  dfree(s->rxt_root); dfree(s->rxt_root_box); dfree(s->mvt_nodes); dfree(s->mvt_parent); dfree(s->mvt_perm);
  dfree(s->mvt_arrive); dfree(s->mvt_root); dfree(s->mvt_root_box);
  for (auto& e : s->ev)
    if (e) cudaEventDestroy(e);
  for (auto& g : s->fgraph) g.drop();
  if (s->cap_st) cudaStreamDestroy(s->cap_st);
  if (s->side) cudaStreamDestroy(s->side);
  for (auto& e : s->br)
    if (e) cudaEventDestroy(e);
  delete s;
}

// Bounds-checked build: failures of every translation unit since the last
// call (0 in the normal build).
unsigned checks_take_all() {
  unsigned n = 0, line = 0;
  n += checks_take_api(&line);
  n += checks_take_bvh(&line);
  n += checks_take_trace(&line);
  n += checks_take_paths(&line);
  n += checks_take_grad(&line);
  return n;
}

bool finite_arr(const float* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

int root_code(int n, int node_base, int leaf_base) {
  return n >= 2 ? node_base : (n == 1 ? ~leaf_base : kEmpty);
}

bool dyn_fused(const dcem_scene* s) {
  return s->nd <= kSmemRefit + 1 && dyn_update_smem(s->nd, s->nobj) <= 200 * 1024;
}

// The 4-wide mapping of both trees, after any change of topology.
int remap4(dcem_scene* s) {
  if (!s->qnodes) return DCEM_OK;
  CK(launch_bvh4_map(s->nodes, s->nint_s + s->nint_d, s->roots, s->q4_kid, s->q4_src, s->q4_count, s->q4_roots,
                     s->q4_scr, s->st));
  s->launches += 1;
  return DCEM_OK;
}

// One-CTA update of the moving-object tree (see DynUpdateArgs).
int dyn_update(dcem_scene* s, bool rebuild) {
  if (s->nd == 0) return DCEM_OK;
  DynUpdateArgs d;
  d.objv_src = s->objv_src;
  d.objv = s->objv;
  d.sel_d = s->sel_d;
  d.tri_mat = s->tri_mat_d;
  d.xf = s->xf_cur;
  d.prim = s->prim;
  d.nd = s->nd;
  d.nobj = s->nobj;
  d.node_base = s->nint_s;
  d.leaf_base = s->ns;
  d.rebuild = rebuild ? 1 : 0;
  d.tris = s->tris;
  d.nodes = s->nodes;
  d.leaf_parent = s->leaf_parent;
  d.perm = s->perm;
  d.slot_of_id = s->slot_of_id;
  d.obj_box = s->obj_box_cur;
  d.root_box = s->root_box + 6;
  d.root = s->roots + 1;
  d.sched = s->dsched;
  d.lvl = s->dlvl;
  d.uctr = s->uctr;
  CK(launch_dyn_update(d, s->st));
  s->launches += 1;
  if (rebuild) {
    s->rebuilt_since_frame = true;
    return remap4(s);
  }
  return DCEM_OK;
}

// (Re)builds the moving-object tree over the objects' current world positions.
int rebuild_dynamic(dcem_scene* s) {
  if (s->nd == 0) return DCEM_OK;
  if (dyn_fused(s)) return dyn_update(s, true);
  int bs = 256, g = (s->nd + bs - 1) / bs;
  s->launches += 3 + (s->nd <= kSmallBuild ? 1 : 22);
  k_xform_prims<<<g, bs, 0, s->st>>>(s->objv_src, s->xf_cur, s->nd, s->v9d);
  launch_tri_boxes(s->v9d, nullptr, s->nd, s->prim, s->st);
  CK(build_tree(s->prim, s->nd, s->nint_s, s->ns, s->nodes, s->leaf_parent, s->perm, s->arrive, s->roots + 1,
                s->root_box + 6, s->scr, s->st));
  k_place_dyn<<<g, bs, 0, s->st>>>(s->v9d, s->objv_src, s->perm, s->sel_d, s->tri_mat_d, s->nd, s->ns, s->tris,
                                   s->objv, s->slot_of_id);
  CK(cudaGetLastError());
  return remap4(s);
}

int alloc_build_scratch(dcem_scene* s, int n) {
  if (n <= kSmallBuild) return DCEM_OK;
  CK(dalloc(&s->scr.bounds, 6));
  CK(dalloc(&s->scr.k0, n)); CK(dalloc(&s->scr.v0, n)); CK(dalloc(&s->scr.k1, n)); CK(dalloc(&s->scr.v1, n));
  CK(dalloc(&s->scr.hist, radix_hist_size(n)));
  CK(dalloc(&s->scr.keys, n));
  return DCEM_OK;
}

// The segment log for W segments per slot over the R primary rays and
// child_cap transmission children (their restart points, segment counts and
// instance words too).
int ensure_log(dcem_scene* s, int W, int child_cap) {
  if (s->logW >= W && s->log_o && s->child_cap == child_cap) return DCEM_OK;
  const int LS = s->R + child_cap;
  dfree(s->log_o); dfree(s->log_d); dfree(s->log_id); dfree(s->capitems);
  size_t n = (size_t)W * (size_t)(LS > 0 ? LS : 1);
  CK(dalloc(&s->log_o, n));
  CK(dalloc(&s->log_d, n));
  CK(dalloc(&s->log_id, n));
  CK(dalloc(&s->capitems, n));
  if (child_cap != s->child_cap) {
    dfree(s->nseg); dfree(s->restart); dfree(s->inst); dfree(s->inst_root);
    CK(dalloc(&s->nseg, LS > 0 ? LS : 1));
    CK(dalloc(&s->restart, LS > 0 ? LS : 1));
    if (child_cap) CK(dalloc(&s->inst, child_cap));
    if (child_cap) CK(dalloc(&s->inst_root, child_cap));
  }
  s->logW = W;
  s->child_cap = child_cap;
  s->LS = LS;
  s->cache_valid = false;
  return DCEM_OK;
}

int ensure_paths(dcem_scene* s, unsigned cand_cap, unsigned ucap) {
  if (cand_cap > s->cand_cap) {
    dfree(s->cand[0]); dfree(s->cand[1]); dfree(s->cand_slot); dfree(s->hkey); dfree(s->hrep);
    CK(dalloc(&s->cand[0], cand_cap));
    CK(dalloc(&s->cand[1], cand_cap));
    CK(dalloc(&s->cand_slot, cand_cap));
    unsigned hcap = pow2_at_least(2ull * cand_cap);
    CK(dalloc(&s->hkey, hcap));
    CK(dalloc(&s->hrep, hcap));
    CK(cudaMemsetAsync(s->hkey, 0, sizeof(unsigned long long) * hcap, s->st));
    CK(cudaMemsetAsync(s->hrep, 0xff, sizeof(unsigned long long) * hcap, s->st));
    s->hcap = hcap;
    s->cand_cap = cand_cap;
    s->cache_valid = false;  // previous captures are gone
  }
  if (ucap > s->ucap) {
    dfree(s->uniq); dfree(s->prec); dfree(s->pout); dfree(s->vpts); dfree(s->vstate);
    dfree(s->prec_b); dfree(s->vpts_b); dfree(s->vstate_b); dfree(s->ckey);
    dfree(s->vc_key[0]); dfree(s->vc_key[1]); dfree(s->vc_u[0]); dfree(s->vc_u[1]);
    CK(dalloc(&s->uniq, ucap));
    CK(dalloc(&s->prec, ucap));
    CK(dalloc(&s->pout, ucap));
    CK(dalloc(&s->vpts, (size_t)ucap * 3 * (kMaxRefl + 2)));
    CK(dalloc(&s->vstate, ucap));
    CK(dalloc(&s->prec_b, ucap));
    CK(dalloc(&s->vpts_b, (size_t)ucap * 3 * (kMaxRefl + 2)));
    CK(dalloc(&s->vstate_b, ucap));
    CK(dalloc(&s->ckey, ucap));
    s->vc_cap = pow2_at_least(2ull * ucap);
    for (int b = 0; b < 2; ++b) {
      CK(dalloc(&s->vc_key[b], s->vc_cap));
      CK(dalloc(&s->vc_u[b], s->vc_cap));
    }
    s->vc_valid = false;  // the previous frame's records are gone
    // sticky mode: kept paths of the previous frame and of this one
    dfree(s->sticky[0]); dfree(s->sticky[1]);
    CK(dalloc(&s->sticky[0], ucap));
    CK(dalloc(&s->sticky[1], ucap));
    if (!s->sticky_n) CK(dalloc(&s->sticky_n, 2));
    CK(cudaMemsetAsync(s->sticky_n, 0, 2 * sizeof(unsigned), s->st));
    s->ucap = ucap;
  }
  return DCEM_OK;
}

// Receiver arrays for nrx receivers, and link arrays (buckets of valid
// paths, staged outputs, output offsets) for nlinks transmitter-receiver
// pairs with bucket_cap paths each.
int ensure_rx(dcem_scene* s, int nrx, int nlinks, int bucket_cap) {
  if (nrx > s->nrx_cap || !s->rx3) {
    int cap = std::max(1, std::max(nrx, s->nrx_cap));
    dfree(s->rx3); dfree(s->rx_cur); dfree(s->rx_traced); dfree(s->rx_moved); dfree(s->moved_list);
    CK(dalloc(&s->rx3, 3 * (size_t)cap));
    CK(dalloc(&s->rx_cur, cap));
    CK(dalloc(&s->rx_traced, cap));
    CK(dalloc(&s->rx_moved, cap));
    CK(dalloc(&s->moved_list, cap));
    dfree(s->rx_prim); dfree(s->rxt_nodes); dfree(s->rxt_parent); dfree(s->rxt_perm); dfree(s->rxt_arrive);
    CK(dalloc(&s->rx_prim, 6 * (size_t)cap));
    CK(dalloc(&s->rxt_nodes, 4 * (size_t)cap));
    CK(dalloc(&s->rxt_parent, cap));
    CK(dalloc(&s->rxt_perm, cap));
    CK(dalloc(&s->rxt_arrive, cap));
    s->nrx_cap = cap;
    s->cache_valid = false;
  }
  if (nlinks > s->nlink_cap || bucket_cap > s->bucket_cap || !s->bucket) {
    int cap = std::max(1, std::max(nlinks, s->nlink_cap));
    bool first = !s->bucket;
    // many links start with smaller buckets (grown on overflow)
    if (first)
      while (bucket_cap > 64 && (size_t)cap * bucket_cap > ((size_t)1 << 26)) bucket_cap >>= 1;
    dfree(s->bucket); dfree(s->bucket_cnt); dfree(s->rxout); dfree(s->link_off);
    s->bucket_cap = first ? bucket_cap : std::max(bucket_cap, s->bucket_cap);
    CK(dalloc(&s->bucket, (size_t)cap * s->bucket_cap));
    CK(dalloc(&s->bucket_cnt, cap));
    CK(dalloc(&s->rxout, 4 * (size_t)cap));  // staging: field (2 cap), P_coh (cap), P_inc (cap)
    CK(dalloc(&s->link_off, cap));
    s->nlink_cap = cap;
    s->cache_valid = false;
  }
  return DCEM_OK;
}

// The wedge masks of the two-reflection pre-test (k_refl2_masks): one word
// per (end point: ntx transmitters and nrx receivers, reflector plane or
// none, wedge cluster).
static int ensure_rmask(dcem_scene* s, int ntx, int nrx) {
  if (!(s->diffraction && s->nw > 0 && s->diff_refl >= 2 && s->nrp > 0)) return DCEM_OK;
  const size_t need = (size_t)(ntx + nrx) * (size_t)(s->nrp + 1) * (size_t)s->nwc;
  if (s->rmask && need <= s->rmask_cap) return DCEM_OK;
  if (need > ((size_t)1 << 31)) return DCEM_ERR_CAPACITY;
  dfree(s->rmask);
  CK(dalloc(&s->rmask, std::max<size_t>(need, 1)));
  s->rmask_cap = std::max<size_t>(need, 1);
  return DCEM_OK;
}

// Wedges for first-order diffraction: edges whose two end vertices
// (bit-identical input coordinates: world space for static triangles, object
// space for moving ones, which a rigid transform maps alike) belong to
// exactly two triangles of the same rigid object (or both static) whose
// planes differ. Face 0 is the lower triangle id; the list is ordered by
// (face 0, face n). The geometry follows the objects every frame
// (k_wedge_geom); here only the topology is kept.
std::vector<WedgeTopo> find_wedges(const std::vector<float>& tris, const std::vector<int>& tri_obj) {
  struct Rec {
    int obj;
    std::array<float, 3> a, b;
    int tri, k0, k1;
  };
  const int ntri = (int)tri_obj.size();
  std::vector<Rec> r;
  r.reserve(3 * (size_t)ntri);
  for (int i = 0; i < ntri; ++i)
    for (int k = 0; k < 3; ++k) {
      const float* p = &tris[9 * (size_t)i + 3 * k];
      const float* q = &tris[9 * (size_t)i + 3 * ((k + 1) % 3)];
      std::array<float, 3> va = {p[0], p[1], p[2]}, vb = {q[0], q[1], q[2]};
      int k0 = k, k1 = (k + 1) % 3;
      if (vb < va) {
        std::swap(va, vb);
        std::swap(k0, k1);
      }
      r.push_back(Rec{tri_obj[i], va, vb, i, k0, k1});
    }
  std::sort(r.begin(), r.end(), [](const Rec& x, const Rec& y) {
    if (x.obj != y.obj) return x.obj < y.obj;
    if (x.a != y.a) return x.a < y.a;
    if (x.b != y.b) return x.b < y.b;
    return x.tri < y.tri;
  });
  std::vector<WedgeTopo> out;
  for (size_t i = 0; i < r.size();) {
    size_t j = i + 1;
    while (j < r.size() && r[j].obj == r[i].obj && r[j].a == r[i].a && r[j].b == r[i].b) ++j;
    if (j - i == 2) {
      const Rec& A = r[i].tri < r[i + 1].tri ? r[i] : r[i + 1];
      const Rec& B = r[i].tri < r[i + 1].tri ? r[i + 1] : r[i];
      // the third vertex of each face: the one off the edge
      int kat = 3 - A.k0 - A.k1, kbt = 3 - B.k0 - B.k1;
      double p0[3] = {A.a[0], A.a[1], A.a[2]};
      double e[3] = {A.b[0] - p0[0], A.b[1] - p0[1], A.b[2] - p0[2]};
      double len = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
      double t[2][3];
      bool ok = len > 0.0;
      const int tt[2] = {A.tri, B.tri}, kk[2] = {kat, kbt};
      for (int q = 0; q < 2 && ok; ++q) {
        const float* x = &tris[9 * (size_t)tt[q] + 3 * kk[q]];
        double d[3] = {x[0] - p0[0], x[1] - p0[1], x[2] - p0[2]};
        double de = (d[0] * e[0] + d[1] * e[1] + d[2] * e[2]) / (len * len);
        for (int c = 0; c < 3; ++c) d[c] -= de * e[c];
        double l = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (!(l > 0.0)) ok = false;
        for (int c = 0; c < 3; ++c) t[q][c] = ok ? d[c] / l : 0.0;
      }
      if (ok) {
        double cosa = t[0][0] * t[1][0] + t[0][1] * t[1][1] + t[0][2] * t[1][2];
        double alpha = std::acos(std::max(-1.0, std::min(1.0, cosa)));
        if (std::fabs(alpha - M_PI) > 1e-6 && alpha > 1e-9) out.push_back(WedgeTopo{A.tri, B.tri, A.k0, A.k1, kat, kbt});
      }
    }
    i = j;
  }
  std::sort(out.begin(), out.end(), [](const WedgeTopo& x, const WedgeTopo& y) {
    return x.ta != y.ta ? x.ta < y.ta : x.tb < y.tb;
  });
  return out;
}

// The wedges in a spatial order for the clusters of the two-reflection
// pre-test: static wedges by the Morton code (10 bits per axis over their
// box) of their edges' midpoints, then each moving object's wedges together
// (their input coordinates are object space), each group by index.
std::vector<int> wedge_order(const std::vector<float>& tris, const std::vector<int>& tri_obj,
                             const std::vector<WedgeTopo>& w) {
  const size_t nw = w.size();
  std::vector<std::array<double, 3>> mid(nw);
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (size_t i = 0; i < nw; ++i) {
    const float* a = &tris[9 * (size_t)w[i].ta + 3 * w[i].ka0];
    const float* b = &tris[9 * (size_t)w[i].ta + 3 * w[i].ka1];
    for (int k = 0; k < 3; ++k) {
      mid[i][k] = 0.5 * ((double)a[k] + b[k]);
      if (tri_obj[w[i].ta] < 0) {
        lo[k] = std::min(lo[k], mid[i][k]);
        hi[k] = std::max(hi[k], mid[i][k]);
      }
    }
  }
  auto spread = [](uint64_t x) {  // 10 bits to every third bit
    uint64_t r = 0;
    for (int b = 0; b < 10; ++b) r |= ((x >> b) & 1ull) << (3 * b);
    return r;
  };
  std::vector<std::array<uint64_t, 3>> key(nw);
  for (size_t i = 0; i < nw; ++i) {
    const int obj = tri_obj[w[i].ta];
    uint64_t m = 0;
    if (obj < 0)
      for (int k = 0; k < 3; ++k) {
        double ext = hi[k] - lo[k];
        double u = ext > 0.0 ? (mid[i][k] - lo[k]) / ext : 0.0;
        uint64_t q = (uint64_t)std::min(1023.0, std::max(0.0, std::floor(u * 1024.0)));
        m |= spread(q) << k;
      }
    key[i] = {obj < 0 ? 0ull : 1ull + (uint64_t)obj, m, (uint64_t)i};
  }
  std::vector<int> perm(nw);
  for (size_t i = 0; i < nw; ++i) perm[i] = (int)i;
  std::sort(perm.begin(), perm.end(), [&](int x, int y) { return key[x] < key[y]; });
  return perm;
}

// Reflector planes: the static triangles grouped by plane (unit normal
// oriented with its first nonzero component positive, offset c = n . v0),
// planes equal when the normals agree to 1e-7 and the offsets to 1e-4 m.
// Each plane's members are sorted by their lowest coordinate along the
// longest side of the plane's box (keys: that coordinate), ties by id, so
// that the member holding a point is found by a binary search.
void group_planes(const std::vector<float>& tris, const std::vector<int>& tri_obj, std::vector<RPlane>& planes,
                  std::vector<int>& members, std::vector<float>& keys) {
  struct Item {
    double n[3], c;
    int id;
  };
  std::vector<Item> it;
  const int ntri = (int)tri_obj.size();
  for (int i = 0; i < ntri; ++i) {
    if (tri_obj[i] >= 0) continue;
    const float* v = &tris[9 * (size_t)i];
    double e1[3] = {(double)v[3] - v[0], (double)v[4] - v[1], (double)v[5] - v[2]};
    double e2[3] = {(double)v[6] - v[0], (double)v[7] - v[1], (double)v[8] - v[2]};
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (!(len > 0.0)) continue;
    for (double& x : n) x /= len;
    double sg = n[0] != 0.0 ? n[0] : (n[1] != 0.0 ? n[1] : n[2]);
    if (sg < 0.0)
      for (double& x : n) x = -x;
    Item q;
    for (int k = 0; k < 3; ++k) q.n[k] = n[k];
    q.c = n[0] * v[0] + n[1] * v[1] + n[2] * v[2];
    q.id = i;
    it.push_back(q);
  }
  auto key = [](const Item& q, int k) {
    return k < 3 ? std::llround(q.n[k] * 1e7) : std::llround(q.c * 1e4);
  };
  std::sort(it.begin(), it.end(), [&](const Item& a, const Item& b) {
    for (int k = 0; k < 4; ++k) {
      long long x = key(a, k), y = key(b, k);
      if (x != y) return x < y;
    }
    return a.id < b.id;
  });
  for (size_t i = 0; i < it.size();) {
    size_t j = i + 1;
    while (j < it.size() && key(it[j], 0) == key(it[i], 0) && key(it[j], 1) == key(it[i], 1) &&
           key(it[j], 2) == key(it[i], 2) && key(it[j], 3) == key(it[i], 3))
      ++j;
    RPlane p;
    for (int k = 0; k < 3; ++k) {
      p.n[k] = it[i].n[k];
      p.nf[k] = (float)it[i].n[k];
    }
    p.c = it[i].c;
    p.cf = (float)it[i].c;
    p.first = (int)members.size();
    p.count = (int)(j - i);
    for (int k = 0; k < 3; ++k) {
      p.box[k] = 3.4e38f;
      p.box[k + 3] = -3.4e38f;
    }
    for (size_t q = i; q < j; ++q) {
      const float* v = &tris[9 * (size_t)it[q].id];
      for (int c = 0; c < 3; ++c)
        for (int k = 0; k < 3; ++k) {
          p.box[k] = std::min(p.box[k], v[3 * c + k]);
          p.box[k + 3] = std::max(p.box[k + 3], v[3 * c + k]);
        }
    }
    p.axis = 0;
    for (int k = 1; k < 3; ++k)
      if (p.box[k + 3] - p.box[k] > p.box[p.axis + 3] - p.box[p.axis]) p.axis = k;
    std::vector<std::pair<float, int>> sm;  // (lowest coordinate along the axis, id)
    p.ext = 0.0f;
    for (size_t q = i; q < j; ++q) {
      const float* v = &tris[9 * (size_t)it[q].id];
      const float lo = std::min(v[p.axis], std::min(v[3 + p.axis], v[6 + p.axis]));
      const float hi = std::max(v[p.axis], std::max(v[3 + p.axis], v[6 + p.axis]));
      p.ext = std::max(p.ext, hi - lo);
      sm.push_back({lo, it[q].id});
    }
    std::sort(sm.begin(), sm.end());
    for (const auto& e : sm) {
      members.push_back(e.second);
      keys.push_back(e.first);
    }
    planes.push_back(p);
    i = j;
  }
}

bool same_traversal(const dcem_params& a, const dcem_params& b) {
  return a.max_refl == b.max_refl && a.rx_radius_scale == b.rx_radius_scale && a.t_min == b.t_min &&
         a.escape_len == b.escape_len;
}

// Reception-sphere spacing of a set of n rays (Sec. III step 1: angular
// spacing alpha = sqrt(4 pi / n)), times the radius scale, over sqrt(3).
float alpha_eff_of(int n, const dcem_params* p) {
  double alpha = std::sqrt(4.0 * M_PI / (double)(n > 0 ? n : 1));
  return (float)((double)p->rx_radius_scale * alpha / std::sqrt(3.0));
}

}  // namespace

extern "C" {

void dcem_params_default(dcem_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->freq_hz = 28e9;
  p->tx_power_w = 5.0;
  p->max_refl = 3;
  p->mode = DCEM_MODE_FULL;
  p->rx_radius_scale = 1.35f;
  p->t_min = 1e-4f;
  p->escape_len = 1e4f;
  p->eps_occ = 1e-4f;
  p->pol[0] = 0.0f;
  p->pol[1] = 0.0f;
  p->pol[2] = 1.0f;
  p->timing = 0;
  p->prec = DCEM_PREC_F64;
}

const char* dcem_status_string(int st) {
  switch (st) {
    case DCEM_OK: return "ok";
    case DCEM_ERR_ARG: return "invalid argument";
    case DCEM_ERR_CUDA: return "CUDA error";
    case DCEM_ERR_CAPACITY: return "capacity exceeded";
    case DCEM_ERR_NONFINITE: return "non-finite input";
    case DCEM_ERR_STACK: return "traversal stack overflow";
    case DCEM_ERR_HASH: return "path-key hash collision";
    case DCEM_ERR_STATE: return "call out of order";
    case DCEM_ERR_NOMEM: return "device allocation failed";
    case DCEM_ERR_CHECK: return "bounds check failed (bounds-checked build)";
    default: return "unknown status";
  }
}

int dcem_scene_create(const float* tris, int32_t ntri, const int32_t* tri_mat, const dcem_material* mats,
                      int32_t nmat, const int32_t* tri_obj, int32_t nobj, void* stream, dcem_scene** out) {
  if (!out) return DCEM_ERR_ARG;
  *out = nullptr;
  if (ntri < 0 || nmat < 0 || nobj < 0) return DCEM_ERR_ARG;
  if (ntri > 0 && (!tris || !tri_mat)) return DCEM_ERR_ARG;
  if (nmat > 0 && !mats) return DCEM_ERR_ARG;
  if (ntri > 0 && nmat == 0) return DCEM_ERR_ARG;
  if (ntri > (1 << 26)) return DCEM_ERR_ARG;
  for (int i = 0; i < ntri; ++i) {
    if (tri_mat[i] < 0 || tri_mat[i] >= nmat) return DCEM_ERR_ARG;
    if (tri_obj && (tri_obj[i] < -1 || tri_obj[i] >= nobj)) return DCEM_ERR_ARG;
  }
  for (int m = 0; m < nmat; ++m)
    if (!std::isfinite(mats[m].eps_r) || !std::isfinite(mats[m].sigma) || mats[m].sigma < 0.0f)
      return DCEM_ERR_ARG;
  if (ntri > 0 && !finite_arr(tris, 9 * (size_t)ntri)) return DCEM_ERR_NONFINITE;

  dcem_scene* s = new (std::nothrow) dcem_scene();
  if (!s) return DCEM_ERR_NOMEM;
  dcem_params_default(&s->cparams);
  int rc = DCEM_OK;
  auto fail = [&](int code) {
    scene_free(s);
    return code;
  };
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) { cudaGetLastError(); return fail(status_of(e)); }
  cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
  if (s->sms < 1) s->sms = 1;
  s->st = (cudaStream_t)stream;
  s->ntri = ntri;
  s->nobj = nobj;
  s->nmat = nmat;
  std::vector<int> sel_s, sel_d;
  for (int i = 0; i < ntri; ++i) ((tri_obj && tri_obj[i] >= 0) ? sel_d : sel_s).push_back(i);
  s->ns = (int)sel_s.size();
  s->nd = (int)sel_d.size();
  s->nint_s = s->ns > 1 ? s->ns - 1 : 0;
  s->nint_d = s->nd > 1 ? s->nd - 1 : 0;
  int nmax = s->ns > s->nd ? s->ns : s->nd;

  float* v9 = nullptr;
  int* sel_s_d = nullptr;
  auto fail2 = [&](int code) {
    dfree(v9); dfree(sel_s_d);
    return fail(code);
  };
#define CKF(x)                                  \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) {                    \
      cudaGetLastError();                       \
      return fail2(status_of(e_));              \
    }                                           \
  } while (0)
  CKF(dalloc(&s->tris, 3 * (size_t)ntri));
  CKF(dalloc(&s->slot_of_id, ntri));
  CKF(dalloc(&s->objv, 3 * (size_t)s->nd));
  CKF(dalloc(&s->objv_src, 3 * (size_t)s->nd));
  CKF(dalloc(&s->sel_d, s->nd));
  CKF(dalloc(&s->tri_mat_d, ntri));
  CKF(dalloc(&s->v9d, 9 * (size_t)s->nd));
  CKF(dalloc(&s->nodes, 4 * (size_t)(s->nint_s + s->nint_d)));
  {
    // the 4-wide compact copy: traversed from shared memory when it fits
    // there, else from global memory
    int nn = s->nint_s + s->nint_d;
    if (nn > 0) {
      CKF(dalloc(&s->qnodes, 4 * (size_t)bvh4_bound(nn)));
      CKF(dalloc(&s->q4_kid, nn));
      CKF(dalloc(&s->q4_src, nn));
      CKF(dalloc(&s->q4_count, 1));
      CKF(dalloc(&s->q4_roots, 2));
      if (bvh4_map_smem(nn) == 0) CKF(dalloc(&s->q4_scr, 3 * (size_t)nn));
    }
  }
  CKF(dalloc(&s->qframe, 6));
  CKF(dalloc(&s->leaf_parent, ntri));
  CKF(dalloc(&s->dsched, ntri > 1 ? ntri : 1));
  CKF(dalloc(&s->dlvl, kDynLevels + 2));
  CKF(dalloc(&s->arrive, nmax));
  CKF(dalloc(&s->roots, 2));
  {
    // both trees empty until built: a scene without moving triangles never
    // builds the second, and the 4-wide mapping reads both roots
    const int empty[2] = {kEmpty, kEmpty};
    CKF(cudaMemcpy(s->roots, empty, sizeof(empty), cudaMemcpyHostToDevice));
  }
  CKF(dalloc(&s->root_box, 12));
  CKF(dalloc(&s->perm, nmax));
  CKF(dalloc(&s->prim, 6 * (size_t)nmax));
  CKF(dalloc(&s->mats, nmat));
  CKF(dalloc(&s->xf_cur, 12 * (size_t)nobj));
  CKF(dalloc(&s->xf_traced, 12 * (size_t)nobj));
  CKF(dalloc(&s->obj_box_cur, 6 * (size_t)nobj));
  CKF(dalloc(&s->obj_box_traced, 6 * (size_t)nobj));
  CKF(dalloc(&s->moved_boxes, 12 * (size_t)nobj));
  CKF(dalloc(&s->obj_moved, (size_t)std::max(nobj, 1)));
  s->mv_cap = std::min(2 * nobj, kSmallBuild);
  CKF(dalloc(&s->mvt_nodes, 4 * (size_t)s->mv_cap));
  CKF(dalloc(&s->mvt_parent, s->mv_cap));
  CKF(dalloc(&s->mvt_perm, s->mv_cap));
  CKF(dalloc(&s->mvt_arrive, s->mv_cap));
  CKF(dalloc(&s->mvt_root, 1));
  CKF(dalloc(&s->mvt_root_box, 6));
  CKF(dalloc(&s->rxt_root, 1));
  CKF(dalloc(&s->rxt_root_box, 6));
  CKF(dalloc(&s->ctr, 1));
  CKF(dalloc(&s->uctr, 1));
  CKF(dalloc(&s->prev_ncand, 1));
  CKF(cudaHostAlloc((void**)&s->ctr_h, 2 * sizeof(DevCounters), cudaHostAllocMapped));
  CKF(cudaHostGetDevicePointer((void**)&s->ctr_hd, s->ctr_h, 0));
  if ((rc = alloc_build_scratch(s, nmax)) != DCEM_OK) return fail2(rc);
  CKF(dalloc(&v9, 9 * (size_t)ntri));
  CKF(dalloc(&s->tri_obj_d, ntri));
  int* tri_obj_d = s->tri_obj_d;
  s->tris_h.assign(tris, tris + 9 * (size_t)ntri);
  s->tri_obj_h.assign(ntri, -1);
  if (tri_obj) std::memcpy(s->tri_obj_h.data(), tri_obj, sizeof(int) * ntri);
  CKF(dalloc(&sel_s_d, s->ns));
  cudaStream_t st = s->st;
  if (ntri > 0) {
    CKF(cudaMemcpyAsync(v9, tris, sizeof(float) * 9 * (size_t)ntri, cudaMemcpyHostToDevice, st));
    CKF(cudaMemcpyAsync(s->tri_mat_d, tri_mat, sizeof(int) * ntri, cudaMemcpyHostToDevice, st));
    std::vector<int> to(ntri, -1);
    if (tri_obj) std::memcpy(to.data(), tri_obj, sizeof(int) * ntri);
    CKF(cudaMemcpyAsync(tri_obj_d, to.data(), sizeof(int) * ntri, cudaMemcpyHostToDevice, st));
    CKF(cudaStreamSynchronize(st));  // `to` goes out of scope
  }
  if (s->ns) CKF(cudaMemcpyAsync(sel_s_d, sel_s.data(), sizeof(int) * s->ns, cudaMemcpyHostToDevice, st));
  if (s->nd) CKF(cudaMemcpyAsync(s->sel_d, sel_d.data(), sizeof(int) * s->nd, cudaMemcpyHostToDevice, st));
  std::vector<float4> mh(nmat > 0 ? nmat : 1);
  // .w: penetration loss [dB] of a transmitting material, < 0 opaque (default)
  for (int m = 0; m < nmat; ++m) mh[m] = make_float4(mats[m].eps_r, mats[m].sigma, mats[m].pec ? 1.0f : 0.0f, -1.0f);
  s->mats_h = mh;
  if (nmat) CKF(cudaMemcpyAsync(s->mats, mh.data(), sizeof(float4) * nmat, cudaMemcpyHostToDevice, st));
  // static tree (built once)
  launch_tri_boxes(v9, sel_s_d, s->ns, s->prim, st);
  CKF(build_tree(s->prim, s->ns, 0, 0, s->nodes, s->leaf_parent, s->perm, s->arrive, s->roots, s->root_box,
                 s->scr, st));
  launch_place_tris(v9, sel_s_d, s->perm, s->tri_mat_d, tri_obj_d, s->ns, 0, s->tris, nullptr, s->slot_of_id, st);
  CKF(cudaGetLastError());
  // moving objects: identity transforms until the first update
  if (s->nd) {
    int g = (s->nd + 255) / 256;
    k_objv_src<<<g, 256, 0, st>>>(v9, s->sel_d, tri_obj_d, s->tri_mat_d, s->nd, s->objv_src);
    CKF(cudaGetLastError());
  }
  if (nobj) {
    std::vector<float> id(12 * (size_t)nobj, 0.0f);
    for (int o = 0; o < nobj; ++o) id[12 * o] = id[12 * o + 5] = id[12 * o + 10] = 1.0f;
    CKF(cudaMemcpyAsync(s->xf_cur, id.data(), sizeof(float) * id.size(), cudaMemcpyHostToDevice, st));
    CKF(cudaMemcpyAsync(s->xf_traced, id.data(), sizeof(float) * id.size(), cudaMemcpyHostToDevice, st));
    CKF(cudaStreamSynchronize(st));
  }
  if ((rc = rebuild_dynamic(s)) != DCEM_OK) return fail2(rc);
  CKF(cudaMemsetAsync(s->ctr, 0, sizeof(DevCounters), st));
  CKF(cudaMemsetAsync(s->uctr, 0, sizeof(DevCounters), st));
  CKF(cudaMemsetAsync(s->prev_ncand, 0, sizeof(unsigned), st));
  if (nobj) {
    if (!(s->nd && dyn_fused(s))) {  // the fused update already wrote the object boxes
      CKF(cudaMemsetAsync(s->obj_box_cur, 0xff, sizeof(unsigned) * 3 * nobj, st));
      CKF(cudaMemsetAsync(s->obj_box_cur + 3 * nobj, 0, sizeof(unsigned) * 3 * nobj, st));
    }
    if (s->nd && !dyn_fused(s)) {
      CKF(cudaMemsetAsync(s->arrive, 0, sizeof(int) * (s->nint_d > 0 ? s->nint_d : 1), st));
      launch_transform_refit(s->objv, s->xf_cur, s->nd, nobj, s->nint_s, s->ns, s->tris, s->nodes, s->leaf_parent,
                             s->arrive, s->root_box + 6, s->obj_box_cur, s->uctr, st);
      CKF(cudaGetLastError());
    }
    CKF(cudaMemcpyAsync(s->obj_box_traced, s->obj_box_cur, sizeof(unsigned) * 6 * nobj, cudaMemcpyDeviceToDevice, st));
  }
  s->root_h[0] = root_code(s->ns, 0, 0);
  s->root_h[1] = root_code(s->nd, s->nint_s, s->ns);
  CKF(cudaStreamSynchronize(st));
  if ((rc = remap4(s)) != DCEM_OK) return fail2(rc);
  CKF(cudaStreamSynchronize(st));
  for (auto& ev : s->ev) CKF(cudaEventCreate(&ev));
  CKF(cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking));
  for (auto& e : s->br) CKF(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  dfree(v9); dfree(sel_s_d);
#undef CKF
  *out = s;
  return DCEM_OK;
}

int dcem_scene_set_rays(dcem_scene* s, const float* dirs, int32_t n_rays) {
  if (!s || n_rays < 0) return DCEM_ERR_ARG;
  return dcem_scene_set_ray_sets(s, dirs, &n_rays, 1);
}

int dcem_scene_set_ray_sets(dcem_scene* s, const float* dirs, const int32_t* n_rays, int32_t ntx) {
  if (!s || !n_rays || ntx < 1 || ntx > kMaxRaySets) return DCEM_ERR_ARG;
  long long total = 0;
  for (int t = 0; t < ntx; ++t) {
    // one set may be empty only when it is the only one (dcem_scene_set_rays(s, _, 0))
    if (n_rays[t] < (ntx > 1 ? 1 : 0)) return DCEM_ERR_ARG;
    total += n_rays[t];
  }
  if (total > (1 << 27) || (total > 0 && !dirs)) return DCEM_ERR_ARG;
  const int n = (int)total;
  if (n > 0 && !finite_arr(dirs, 3 * (size_t)n)) return DCEM_ERR_NONFINITE;
  for (int i = 0; i < n; ++i) {
    float x = dirs[3 * i], y = dirs[3 * i + 1], z = dirs[3 * i + 2];
    if (!(x * x + y * y + z * z > 0.0f)) return DCEM_ERR_ARG;
  }
  CK(cudaStreamSynchronize(s->st));
  dfree(s->rays); dfree(s->ray_perm); dfree(s->nseg); dfree(s->restart); dfree(s->queue);
  dfree(s->log_o); dfree(s->log_d); dfree(s->log_id); dfree(s->capitems);
  dfree(s->txs);
  if (s->txs_h) cudaFreeHost(s->txs_h);
  s->txs_h = nullptr;
  s->logW = 0;
  s->R = n;
  s->LS = n;
  s->child_cap = 0;
  dfree(s->inst);
  dfree(s->inst_root);
  s->rays_set = false;
  s->nsets = ntx;
  s->set_rays_h.assign(n_rays, n_rays + ntx);
  CK(dalloc(&s->txs, ntx));
  CK(cudaHostAlloc((void**)&s->txs_h, sizeof(float4) * ntx, cudaHostAllocDefault));
  CK(dalloc(&s->rays, n));
  CK(dalloc(&s->ray_perm, n));
  CK(dalloc(&s->nseg, n));
  CK(dalloc(&s->restart, n));
  CK(dalloc(&s->queue, n));
  s->ray_perm_h.assign(n, 0);
  if (n) {
    // upload (.w = the ray's set), then order the rays by set and, within a
    // set, by direction, so that a warp's rays share a transmitter and are
    // close in angle (the caller's order is kept in ray_perm)
    std::vector<float4> h(n);
    for (int t = 0, i = 0; t < ntx; ++t)
      for (int k = 0; k < n_rays[t]; ++k, ++i) {
        float sid;
        std::memcpy(&sid, &t, sizeof(int));
        h[i] = make_float4(dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], sid);
      }
    float4* src = nullptr;
    unsigned *k0 = nullptr, *v0 = nullptr, *k1 = nullptr, *v1 = nullptr, *hist = nullptr;
    cudaError_t e = dalloc(&src, n);
    if (!e) e = dalloc(&k0, n);
    if (!e) e = dalloc(&v0, n);
    if (!e) e = dalloc(&k1, n);
    if (!e) e = dalloc(&v1, n);
    if (!e) e = dalloc(&hist, radix_hist_size(n));
    if (!e) e = cudaMemcpyAsync(src, h.data(), sizeof(float4) * n, cudaMemcpyHostToDevice, s->st);
    if (!e) {
      int g = std::min((n + 255) / 256, 4096);
      k_ray_keys<<<g, 256, 0, s->st>>>(src, n, k0, v0);
      e = sort_pairs_u32(k0, v0, k1, v1, hist, n, 32, s->st);
      if (!e && ntx > 1) {
        // stable second pass by set
        k_set_keys<<<g, 256, 0, s->st>>>(src, v0, n, k0);
        e = sort_pairs_u32(k0, v0, k1, v1, hist, n, ntx > 256 ? 16 : 8, s->st);
      }
      if (!e) {
        k_gather_rays<<<g, 256, 0, s->st>>>(src, v0, n, s->rays, s->ray_perm);
        e = cudaGetLastError();
      }
    }
    if (!e) e = cudaMemcpyAsync(s->ray_perm_h.data(), s->ray_perm, sizeof(int) * n, cudaMemcpyDeviceToHost, s->st);
    if (!e) e = cudaStreamSynchronize(s->st);
    dfree(src); dfree(k0); dfree(v0); dfree(k1); dfree(v1); dfree(hist);
    CK(e);
  }
  s->rays_set = true;
  s->cache_valid = false;
  return DCEM_OK;
}

int dcem_scene_update_transforms(dcem_scene* s, const float* xf, int32_t ptr_kind) {
  if (!s) return DCEM_ERR_ARG;
  if (ptr_kind != DCEM_PTR_HOST && ptr_kind != DCEM_PTR_DEVICE) return DCEM_ERR_ARG;
  if (s->nobj == 0) return DCEM_OK;
  if (!xf) return DCEM_ERR_ARG;
  if (ptr_kind == DCEM_PTR_HOST && !finite_arr(xf, 12 * (size_t)s->nobj)) return DCEM_ERR_NONFINITE;
  cudaStream_t st = s->st;
  CK(cudaMemcpyAsync(s->xf_cur, xf, sizeof(float) * 12 * s->nobj,
                     ptr_kind == DCEM_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
  if (dyn_fused(s)) {
    // Sec. III: refit every frame; rebuild when the measured quality of the
    // refit tree has degraded (surface-area cost ratio above the threshold)
    bool rebuild = !s->dyn_on_world ||
                   (s->rebuild_ratio > 0.0f && s->sah_build > 0.0f && s->sah_now > s->rebuild_ratio * s->sah_build);
    int rc = dyn_update(s, rebuild);
    if (rc != DCEM_OK) return rc;
    s->dyn_on_world = true;
    if (rebuild) s->sah_now = 0.0f;  // until the next measurement
    return DCEM_OK;
  }
  if (!s->dyn_on_world) {
    int rc = rebuild_dynamic(s);
    if (rc != DCEM_OK) return rc;
    s->dyn_on_world = true;
  }
  CK(cudaMemsetAsync(s->obj_box_cur, 0xff, sizeof(unsigned) * 3 * s->nobj, st));
  CK(cudaMemsetAsync(s->obj_box_cur + 3 * s->nobj, 0, sizeof(unsigned) * 3 * s->nobj, st));
  if (s->nd) {
    CK(cudaMemsetAsync(s->arrive, 0, sizeof(int) * (s->nint_d > 0 ? s->nint_d : 1), st));
    launch_transform_refit(s->objv, s->xf_cur, s->nd, s->nobj, s->nint_s, s->ns, s->tris, s->nodes,
                           s->leaf_parent, s->arrive, s->root_box + 6, s->obj_box_cur, s->uctr, st);
    CK(cudaGetLastError());
  }
  return DCEM_OK;
}

int dcem_scene_set_rebuild_threshold(dcem_scene* s, float ratio) {
  if (!s || !std::isfinite(ratio)) return DCEM_ERR_ARG;
  s->rebuild_ratio = ratio;
  return DCEM_OK;
}

int dcem_scene_set_trace_config(dcem_scene* s, int32_t kernel, int32_t block, int32_t stack) {
  if (!s || kernel < -1 || kernel > 2) return DCEM_ERR_ARG;
  bool okb = false;
  for (int b : kTraceBlocks) okb = okb || b == block;
  if (!okb || stack < kTraceStackMin || stack > kTraceStackMax) return DCEM_ERR_ARG;
  if (kernel == 1 && (!s->qnodes || trace_q_stack_cap(s->nint_s + s->nint_d) == 0)) return DCEM_ERR_ARG;
  if (kernel == 2 && !s->qnodes) return DCEM_ERR_ARG;
  s->tc_kernel = kernel;
  s->tc_block = block;
  s->tc_stack = stack;
  return DCEM_OK;
}

int dcem_scene_autotune(dcem_scene* s, const float* tx, int32_t ntx, const float* rx, int32_t nrx,
                        int32_t rx_ptr_kind, const dcem_params* params, int32_t reps, int32_t* kernel,
                        int32_t* block, int32_t* stack) {
  if (!s || !params || reps < 1 || reps > 16) return DCEM_ERR_ARG;
  dcem_params p = *params;
  p.mode = DCEM_MODE_FULL;
  p.timing = 2;
  dcem_result r;
  std::memset(&r, 0, sizeof(r));
  r.ptr_kind = DCEM_PTR_HOST;
  struct Cfg {
    int k, b, st;
  };
  std::vector<Cfg> cands;
  if (s->qnodes && trace_q_stack_cap(s->nint_s + s->nint_d) > 0) cands.push_back({1, s->tc_block, s->tc_stack});
  for (int k : {2, 0}) {
    if (k == 2 && !s->qnodes) continue;
    for (int b : {128, 256})
      for (int sd : {16, 24, 32}) cands.push_back({k, b, sd});
  }
  const int ok = s->tc_kernel, ob = s->tc_block, os = s->tc_stack;
  float best = INFINITY;
  Cfg pick{ok, ob, os};
  for (const Cfg& c : cands) {
    s->tc_kernel = c.k;
    s->tc_block = c.b;
    s->tc_stack = c.st;
    float t = INFINITY;
    for (int i = 0; i < reps; ++i) {
      int rc = dcem_trace_links(s, tx, ntx, rx, nrx, rx_ptr_kind, &p, &r);
      if (rc != DCEM_OK) {
        s->tc_kernel = ok;
        s->tc_block = ob;
        s->tc_stack = os;
        return rc;
      }
      t = std::min(t, r.stats.ms_stage[2]);
    }
    if (t < best) {
      best = t;
      pick = c;
    }
  }
  s->tc_kernel = pick.k;
  s->tc_block = pick.b;
  s->tc_stack = pick.st;
  s->cache_valid = false;
  if (kernel) *kernel = pick.k;
  if (block) *block = pick.k == 1 ? kTraceQThreads : pick.b;
  if (stack) *stack = pick.k == 1 ? trace_q_stack_cap(s->nint_s + s->nint_d) : pick.st;
  return DCEM_OK;
}

int dcem_scene_set_transmission(dcem_scene* s, const float* loss_db, int32_t nmat, int32_t max_trans) {
  if (!s || max_trans < 0 || max_trans > DCEM_MAX_REFL) return DCEM_ERR_ARG;
  if (nmat != s->nmat || (nmat > 0 && !loss_db)) return DCEM_ERR_ARG;
  for (int m = 0; m < nmat; ++m)
    if (!std::isfinite(loss_db[m])) return DCEM_ERR_NONFINITE;
  CK(cudaStreamSynchronize(s->st));
  for (int m = 0; m < nmat; ++m) s->mats_h[m].w = loss_db[m] >= 0.0f ? loss_db[m] : -1.0f;
  if (nmat) CK(cudaMemcpy(s->mats, s->mats_h.data(), sizeof(float4) * nmat, cudaMemcpyHostToDevice));
  s->max_trans = max_trans;
  s->cache_valid = false;
  return DCEM_OK;
}

int dcem_scene_set_diffraction(dcem_scene* s, int32_t on, int32_t* n_wedges) {
  if (!s || (on != 0 && on != 1)) return DCEM_ERR_ARG;
  if (on && !s->wtopo) {
    std::vector<WedgeTopo> w = find_wedges(s->tris_h, s->tri_obj_h);
    s->nw = (int)w.size();
    if (s->nw) {
      std::vector<int> perm = wedge_order(s->tris_h, s->tri_obj_h, w);
      s->nwc = (s->nw + kWedgeCluster - 1) / kWedgeCluster;
      CK(dalloc(&s->wtopo, s->nw));
      CK(dalloc(&s->wedges, s->nw));
      CK(dalloc(&s->wedgesf, s->nw));
      CK(dalloc(&s->wperm, s->nw));
      CK(dalloc(&s->wcbox, 6 * (size_t)s->nwc));
      CK(cudaMemcpy(s->wtopo, w.data(), sizeof(WedgeTopo) * w.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(s->wperm, perm.data(), sizeof(int) * perm.size(), cudaMemcpyHostToDevice));
    }
  }
  if (on && s->nw && !s->dsurv) {  // grown (and the frame traced again) when a frame needs more
    CK(dalloc(&s->dsurv, (size_t)1024));
    s->dsurv_cap = 1024;
  }
  s->diffraction = on != 0;
  if (n_wedges) *n_wedges = s->nw;
  return DCEM_OK;
}

int dcem_scene_set_diffraction_reflections(dcem_scene* s, int32_t on, int32_t* n_planes) {
  if (!s || on < 0 || on > 3) return DCEM_ERR_ARG;
  if (on && !s->diffraction) return DCEM_ERR_STATE;
  if (on && !s->rplanes) {
    std::vector<RPlane> planes;
    std::vector<int> members;
    std::vector<float> keys;
    group_planes(s->tris_h, s->tri_obj_h, planes, members, keys);
    s->nrp = (int)planes.size();
    if (s->nrp) {
      CK(dalloc(&s->rplanes, planes.size()));
      CK(dalloc(&s->rmembers, members.size()));
      CK(dalloc(&s->rkeys, keys.size()));
      CK(cudaMemcpy(s->rplanes, planes.data(), sizeof(RPlane) * planes.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(s->rmembers, members.data(), sizeof(int) * members.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(s->rkeys, keys.data(), sizeof(float) * keys.size(), cudaMemcpyHostToDevice));
    }
  }
  s->diff_refl = on;
  if (n_planes) *n_planes = s->nrp;
  return DCEM_OK;
}

int dcem_scene_set_diffraction_order(dcem_scene* s, int32_t max_order) {
  if (!s || max_order < 1 || max_order > 3) return DCEM_ERR_ARG;
  if (max_order > 1 && !s->diffraction) return DCEM_ERR_STATE;
  if (max_order >= 2 && !s->dseq2 && s->nw > 1) {  // lists grown (and the frame traced again) on demand
    CK(dalloc(&s->dseq2, (size_t)4096));
    s->dseq2_cap = 4096;
    CK(dalloc(&s->drel, ((size_t)s->nw * s->nw + 31) / 32));
  }
  if (max_order >= 3 && !s->dseq3 && s->nw > 2) {
    CK(dalloc(&s->dseq3, (size_t)4096));
    s->dseq3_cap = 4096;
  }
  CK(cudaStreamSynchronize(s->st));
  s->diff_order = max_order;
  return DCEM_OK;
}

int dcem_scene_set_graph_replay(dcem_scene* s, int32_t on) {
  if (!s || (on != 0 && on != 1)) return DCEM_ERR_ARG;
  s->use_graphs = on != 0;
  return DCEM_OK;
}

int dcem_scene_reset_cache(dcem_scene* s) {
  if (!s) return DCEM_ERR_ARG;
  s->cache_valid = false;
  return DCEM_OK;
}

int dcem_scene_set_stream(dcem_scene* s, void* stream) {
  if (!s) return DCEM_ERR_ARG;
  CK(cudaStreamSynchronize(s->st));
  s->st = (cudaStream_t)stream;
  return DCEM_OK;
}

void dcem_scene_destroy(dcem_scene* s) { scene_free(s); }

static void make_plan(dcem_scene* s, int nrx, const dcem_params* p, bool coherent, const dcem_result* out,
                      FramePlan& P) {
  std::memset(&P, 0, sizeof(P));
  int N = p->max_refl;
  int nxt = s->cur ^ 1;
  P.coherent = coherent ? 1 : 0;
  P.tm = p->timing == 1;                       // every stage
  P.tk = p->timing == 1 || p->timing == 2;     // the closest-hit kernel
  P.nrx = nrx;
  P.R = s->R;
  P.nobj = s->nobj;
  P.has0 = s->root_h[0] != kEmpty;
  P.has1 = s->root_h[1] != kEmpty;
  P.ptr_dev = out->ptr_kind == DCEM_PTR_DEVICE;
  P.nsets = s->nsets;
  P.nlinks = s->nsets * nrx;

  TraceArgs& a = P.a;
  a.bvh.nodes = s->nodes;
  a.bvh.tris = s->tris;
  a.bvh.root0 = s->root_h[0];
  a.bvh.root1 = s->root_h[1];
  a.bvh.max_visits = 2 * (s->nint_s + s->nint_d + s->ntri) + 8;
  a.bvh.nnodes = s->nint_s + s->nint_d;
  a.bvh.ntris = s->ntri;
  a.rays = s->rays;
  a.txs = s->txs;
  a.nsets = s->nsets;
  a.R = s->R;
  a.LS = s->LS;
  a.mats = s->mats;
  a.max_trans = s->max_trans;
  a.pass = 0;
  a.child_cap = s->child_cap;
  a.inst = s->inst;
  a.inst_root = s->inst_root;
  a.N = N;
  a.tmin = p->t_min;
  a.escape = p->escape_len;
  a.rx = s->rx_cur;
  a.nrx = nrx;
  a.log_o = s->log_o;
  a.log_d = s->log_d;
  a.log_id = s->log_id;
  a.capitems = s->capitems;
  a.nseg = s->nseg;
  a.queue = nullptr;
  a.rx_moved = nullptr;
  a.queue_w = s->queue;
  a.restart = s->restart;
  a.nq_dev = &s->ctr->n_retrace;
  a.cand = s->cand[nxt];
  a.cand_cap = s->cand_cap;
  a.ctr = s->ctr;
  a.rxt.nodes = s->rxt_nodes;
  a.rxt.perm = s->rxt_perm;
  a.rxt.root = s->rxt_root;
  a.rxt.root_box = s->rxt_root_box;
  a.rxt.max_visits = 2 * nrx + 8;
  a.rxt.cap = s->nrx_cap;
  a.qnodes = s->qnodes;
  a.qframe = s->qframe;
  a.n_nodes = s->nint_s + s->nint_d;
  a.q4_count = s->q4_count;
  a.q4_roots = s->q4_roots;
  a.q4_bound = bvh4_bound(a.n_nodes);
  // closest-hit kernel: the configured one, or automatically the compact
  // copy from shared memory when it and the CTA's stacks fit there (1), else
  // from global memory (2); binary nodes (0) when there is no compact copy
  {
    int qcap = trace_q_stack_cap(a.n_nodes);
    int k = s->tc_kernel;
    if (k < 0 || (k == 1 && qcap == 0) || (k > 0 && !s->qnodes)) k = !s->qnodes ? 0 : (qcap > 0 ? 1 : 2);
    a.use_q = k;
    a.stack_cap = k == 1 ? qcap : s->tc_stack;
    a.block = k == 1 ? kTraceQThreads : s->tc_block;
  }
  P.use_q = a.use_q;
  P.q4_bound = a.q4_bound;

  FramePrepArgs& fp = P.fp;
  fp.rx3 = s->rx3;
  fp.nrx = nrx;
  fp.rx_cur = s->rx_cur;
  fp.rx_traced = s->rx_traced;
  fp.have_prev = coherent ? 1 : 0;
  fp.rx_moved = s->rx_moved;
  fp.moved_list = s->moved_list;
  fp.rx_prim = s->rx_prim;
  fp.bucket_cnt = s->bucket_cnt;
  fp.coherent = coherent ? 1 : 0;
  fp.nobj = s->nobj;
  fp.xf_cur = s->xf_cur;
  fp.xf_traced = s->xf_traced;
  fp.obj_box_cur = s->obj_box_cur;
  fp.obj_box_traced = s->obj_box_traced;
  fp.moved_boxes = s->moved_boxes;
  fp.obj_moved = s->obj_moved;
  fp.ctr = s->ctr;
  fp.trx.prim = s->rx_prim;
  fp.trx.n = nrx;
  fp.trx.nodes = s->rxt_nodes;
  fp.trx.leaf_parent = s->rxt_parent;
  fp.trx.perm = s->rxt_perm;
  fp.trx.arrive = s->rxt_arrive;
  fp.trx.root = s->rxt_root;
  fp.trx.root_box = s->rxt_root_box;
  fp.tmv.prim = s->moved_boxes;
  fp.tmv.cap = s->mv_cap;
  fp.tmv.nodes = s->mvt_nodes;
  fp.tmv.leaf_parent = s->mvt_parent;
  fp.tmv.perm = s->mvt_perm;
  fp.tmv.arrive = s->mvt_arrive;
  fp.tmv.root = s->mvt_root;
  fp.tmv.root_box = s->mvt_root_box;

  if (coherent) {
    CoherentArgs& c = P.c;
    c.moved_list = s->moved_list;
    c.rx_moved = s->rx_moved;
    c.restart = s->restart;
    c.ctr = s->ctr;
    c.prev_cand = s->cand[s->cur];
    c.prev_ncand = s->prev_ncand;
    c.prev_cap = s->cand_cap;
    c.mvt.nodes = s->mvt_nodes;
    c.mvt.perm = s->mvt_perm;
    c.mvt.root = s->mvt_root;
    c.mvt.root_box = s->mvt_root_box;
    c.mvt.max_visits = 2 * s->mv_cap + 8;
    c.mvt.cap = s->mv_cap;
    c.mv_cap = s->mv_cap;
  }

  PathArgs& q = P.q;
  q.R = s->LS;
  q.max_trans = s->max_trans;
  q.R0 = s->R;
  q.inst_root = s->inst_root;
  q.log_id = s->log_id;
  q.cand = s->cand[nxt];
  q.cand_cap = s->cand_cap;
  q.hkey = s->hkey;
  q.hrep = s->hrep;
  q.hcap = s->hcap;
  q.cand_slot = s->cand_slot;
  q.uniq = s->uniq;
  q.ucap = s->ucap;
  // this frame's records: buffer nxt (a = the frame's parity); the previous
  // frame's: buffer cur
  PathRec* precs[2] = {s->prec, s->prec_b};
  double* vptss[2] = {s->vpts, s->vpts_b};
  int* vstates[2] = {s->vstate, s->vstate_b};
  q.prec = precs[nxt];
  q.ray_perm = s->ray_perm;
  q.vpts = vptss[nxt];
  q.vstate = vstates[nxt];
  // validation reuse: exact coherent mode (not sticky), same validation
  // parameters as the previous frame, whose table and records are intact
  const bool vc_on = p->mode == DCEM_MODE_COHERENT && s->max_trans == 0;
  q.reuse = (coherent && vc_on && s->vc_valid && p->freq_hz == s->cparams.freq_hz &&
             std::memcmp(p->pol, s->cparams.pol, sizeof(p->pol)) == 0 && p->eps_occ == s->cparams.eps_occ &&
             p->prec == s->cparams.prec) ? 1 : 0;
  q.vc_prev_key = s->vc_key[s->cur];
  q.vc_prev_u = s->vc_u[s->cur];
  q.prev_prec = precs[s->cur];
  q.prev_vpts = vptss[s->cur];
  q.prev_vstate = vstates[s->cur];
  q.vc_cap = s->vc_cap;
  q.vc_next_key = vc_on ? s->vc_key[nxt] : nullptr;
  q.vc_next_u = s->vc_u[nxt];
  q.ckey = vc_on ? s->ckey : nullptr;
  q.rx_moved = s->rx_moved;
  q.obj_moved = s->obj_moved;
  q.tri_obj = s->tri_obj_d;
  q.mvt.nodes = s->mvt_nodes;
  q.mvt.perm = s->mvt_perm;
  q.mvt.root = s->mvt_root;
  q.mvt.root_box = s->mvt_root_box;
  q.mvt.max_visits = 2 * s->mv_cap + 8;
  q.mvt.cap = s->mv_cap;
  q.mv_cap = (unsigned)s->mv_cap;
  q.N = N;
  q.bucket = s->bucket;
  q.bucket_cnt = s->bucket_cnt;
  q.bucket_cap = s->bucket_cap;
  q.link_off = P.nlinks > kScanLinks ? s->link_off : nullptr;
  if (out->ptr_kind == DCEM_PTR_DEVICE) {  // results go straight to the caller's buffers
    q.pout = out->paths;
    q.pout_cap = out->paths ? (unsigned)out->max_paths : 0u;
    q.out_field = out->field;
    q.out_pc = out->p_coh_dbm;
    q.out_pi = out->p_inc_dbm;
  } else {
    q.pout = s->pout;
    q.pout_cap = s->ucap;
    q.out_field = s->rxout;
    q.out_pc = s->rxout + 2 * (size_t)s->nlink_cap;
    q.out_pi = s->rxout + 3 * (size_t)s->nlink_cap;
  }
  q.tris = s->tris;
  q.slot_of_id = s->slot_of_id;
  q.mats = s->mats;
  q.bvh = a.bvh;
  q.rx = s->rx_cur;
  q.nrx = nrx;
  q.txs = s->txs;
  q.pol = make_float3(p->pol[0], p->pol[1], p->pol[2]);
  q.eps_occ = p->eps_occ;
  q.prec_df = p->prec == DCEM_PREC_DF32 ? 1 : 0;
  q.freq = p->freq_hz;
  q.tx_power = p->tx_power_w;
  q.ctr = s->ctr;
  q.wedges = s->diffraction && s->nw > 0 ? s->wedges : nullptr;
  q.wf = s->wedgesf;
  q.wtopo = s->wtopo;
  q.nw = s->nw;
  q.wperm = s->wperm;
  q.wcbox = s->wcbox;
  q.nwc = s->nwc;
  q.dsurv = s->dsurv;
  q.dsurv_cap = s->dsurv_cap;
  const bool dr = q.wedges && s->diff_refl && s->nrp > 0;
  q.rplanes = dr ? s->rplanes : nullptr;
  const int dord = q.wedges && s->nw > 1 ? std::min(s->diff_order, s->nw > 2 ? 3 : 2) : 1;
  q.diff_order = dord;
  q.dseq2 = dord >= 2 ? s->dseq2 : nullptr;
  q.dseq2_cap = dord >= 2 ? s->dseq2_cap : 0;
  q.dseq3 = dord >= 3 ? s->dseq3 : nullptr;
  q.dseq3_cap = dord >= 3 ? s->dseq3_cap : 0;
  q.drel = dord >= 2 ? s->drel : nullptr;
  q.rmembers = dr ? s->rmembers : nullptr;
  q.rkeys = dr ? s->rkeys : nullptr;
  q.nrp = dr ? s->nrp : 0;
  q.drefl2 = dr && s->diff_refl >= 2 ? 1 : 0;
  q.rmask = q.drefl2 ? s->rmask : nullptr;
  q.dmid = dr && s->diff_refl >= 3 && dord >= 2 ? 1 : 0;
  // sticky mode: the previous frame's kept paths (when the cache is valid),
  // and this frame's
  P.sticky = p->mode == DCEM_MODE_STICKY;
  q.sticky_prev = P.sticky && coherent && s->cparams.mode == DCEM_MODE_STICKY ? s->sticky[s->cur] : nullptr;
  q.sticky_prev_n = s->sticky_n ? s->sticky_n + s->cur : nullptr;
  q.sticky_cap = s->ucap;
  q.sticky_next = P.sticky ? s->sticky[nxt] : nullptr;
  P.sticky_n_next = s->sticky_n ? s->sticky_n + nxt : nullptr;

  P.nodes = s->nodes;
  P.q4_count = s->q4_count;
  P.q4_kid = s->q4_kid;
  P.q4_src = s->q4_src;
  P.root_box = s->root_box;
  P.qnodes = s->qnodes;
  P.qframe = s->qframe;
  P.rx_cur = s->rx_cur;
  P.rx_traced = s->rx_traced;
  P.xf_cur = s->xf_cur;
  P.xf_traced = s->xf_traced;
  P.obj_box_cur = s->obj_box_cur;
  P.obj_box_traced = s->obj_box_traced;
  P.prev_ncand = s->prev_ncand;
  P.ctr = s->ctr;
  P.uctr = s->uctr;
  P.ctr_hd = s->ctr_hd;
  P.txs = s->txs;
  P.txs_h = s->txs_h;
  P.bucket_cnt = s->bucket_cnt;
  for (int i = 0; i < 10; ++i) P.ev[i] = s->ev[i];
  P.side = s->side;
  for (int i = 0; i < 4; ++i) P.br[i] = s->br[i];
}

// Event record on a stream, or an event-record node when the stream is being
// captured (so that the replayed graph records the event too).
static cudaError_t rec(cudaEvent_t e, cudaStream_t st, bool cap) {
  return cap ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal) : cudaEventRecord(e, st);
}

// The frame's trace arguments: in a coherent frame the retrace queue the
// marking pass writes and the moved-receiver flags.
static TraceArgs frame_trace_args(const FramePlan& P) {
  TraceArgs a = P.a;
  if (P.coherent) {
    a.queue = P.a.queue_w;
    a.rx_moved = P.c.rx_moved;
  }
  return a;
}

// The frame's device work before the closest hit, in stream order (timing
// events only with `timed`).
static int enqueue_pre(const FramePlan& P, int sms, cudaStream_t st, bool cap, bool timed) {
  bool tm = P.tm && timed;
  if (tm) CK(rec(P.ev[0], st, cap));
  CK(cudaMemsetAsync(P.ctr, 0, sizeof(DevCounters), st));
  // transmitters and their capture spacing, from the pinned staging the
  // host filled for this frame
  CK(cudaMemcpyAsync(P.txs, P.txs_h, sizeof(float4) * P.nsets, cudaMemcpyHostToDevice, st));
  if (P.nlinks > P.nrx) CK(cudaMemsetAsync(P.bucket_cnt, 0, sizeof(unsigned) * P.nlinks, st));
  // second branch: the compact node copy, concurrent with the frame
  // preparation and the marking pass (joined before the closest hit)
  if (P.use_q) {
    CK(cudaEventRecord(P.br[0], st));
    CK(cudaStreamWaitEvent(P.side, P.br[0], 0));
    launch_quantize4(P.nodes, P.q4_bound, P.q4_count, P.q4_kid, P.q4_src, P.root_box, P.has0, P.has1, P.qnodes,
                     P.qframe, P.side);
    CK(cudaGetLastError());
    CK(cudaEventRecord(P.br[1], P.side));
  }
  if (P.q.vc_next_key)  // the key table this frame builds for the next one
    CK(cudaMemsetAsync(P.q.vc_next_key, 0, sizeof(unsigned long long) * P.q.vc_cap, st));
  CK(launch_frame_prep(P.fp, st));
  if (tm) CK(rec(P.ev[1], st, cap));
  if (P.coherent) {
    CK(launch_mark(P.a, P.c, sms, st));
    CK(launch_carry(P.a, P.c, st));
  }
  if (P.use_q) CK(cudaStreamWaitEvent(st, P.br[1], 0));
  return DCEM_OK;
}

// The closest-hit pass (and, with transmission, its passes over the children).
static int enqueue_trace(const FramePlan& P, int sms, cudaStream_t st, bool cap, bool timed) {
  bool tk = P.tk && timed;
  TraceArgs a = frame_trace_args(P);
  if (tk) CK(rec(P.ev[2], st, cap));
  if (P.R > 0) CK(launch_trace(a, sms, st));
  // transmission: pass p traces the children pass p - 1 spawned
  for (int p = 1; P.R > 0 && p <= a.max_trans; ++p) {
    TraceArgs ap = a;
    ap.pass = p;
    CK(launch_trace(ap, sms, st));
  }
  if (tk) CK(rec(P.ev[3], st, cap));
  return DCEM_OK;
}

// The frame's device work after the closest hit: capture, dedupe,
// validation, reduction and the state the next frame compares against.
static int enqueue_post(const FramePlan& P, int sms, cudaStream_t st, bool cap, bool timed) {
  bool tm = P.tm && timed;
  TraceArgs a = frame_trace_args(P);
  if (P.R > 0) CK(launch_capture(a, sms, st));
  if (tm) CK(rec(P.ev[4], st, cap));
  CK(launch_dedupe(P.q, sms * 4, st));
  if (P.q.sticky_prev) CK(launch_sticky_probe(P.q, sms * 4, st));
  if (tm) CK(rec(P.ev[5], st, cap));
  CK(launch_validate(P.q, sms * 4, st));
  if (P.q.vc_next_key) CK(launch_vcache_build(P.q, sms * 4, st));
  if (P.q.wedges) CK(launch_diffract(P.q, P.nlinks, sms, st));
  if (tm) CK(rec(P.ev[6], st, cap));
  // every counter is final here: the state the next frame compares against
  // and the counters to the host go on the second branch, concurrent with
  // the reduction
  CK(cudaEventRecord(P.br[2], st));
  CK(cudaStreamWaitEvent(P.side, P.br[2], 0));
  {
    int n = std::max(P.nrx, 12 * P.nobj);
    int g = std::max(1, std::min(64, (n + 255) / 256));
    k_frame_end<<<g, 256, 0, P.side>>>(P.rx_cur, P.rx_traced, P.nrx, P.xf_cur, P.xf_traced, P.obj_box_cur,
                                       P.obj_box_traced, P.nobj, P.ctr, P.uctr, P.prev_ncand, P.ctr_hd);
    CK(cudaGetLastError());
  }
  if (P.sticky)  // the kept-path count, for the next frame
    CK(cudaMemcpyAsync(P.sticky_n_next, &P.ctr->n_sticky_next, sizeof(unsigned), cudaMemcpyDeviceToDevice,
                       P.side));
  CK(cudaEventRecord(P.br[3], P.side));
  CK(launch_reduce(P.q, P.nlinks, st));
  if (tm) CK(rec(P.ev[7], st, cap));
  CK(cudaStreamWaitEvent(st, P.br[3], 0));
  // with device outputs nothing follows on the stream: the frame ends here
  if (tm && P.ptr_dev) CK(rec(P.ev[8], st, cap));
  return DCEM_OK;
}

// The frame's device work, in stream order; no host synchronisation.
static int enqueue_frame(const FramePlan& P, int sms, cudaStream_t st, bool cap) {
  int rc = enqueue_pre(P, sms, st, cap, true);
  if (rc == DCEM_OK) rc = enqueue_trace(P, sms, st, cap, true);
  if (rc == DCEM_OK) rc = enqueue_post(P, sms, st, cap, true);
  return rc;
}
// Captures the frame's work from its plan into a graph on the scene's
// capture stream (nothing runs while capturing) and instantiates it.
static int capture_frame(dcem_scene* s, const FramePlan& P, FrameGraph& G) {
  if (!s->cap_st) CK(cudaStreamCreateWithFlags(&s->cap_st, cudaStreamNonBlocking));
  CK(cudaStreamBeginCapture(s->cap_st, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_frame(P, s->sms, s->cap_st, true);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s->cap_st, &g);
  if (rc == DCEM_OK && e != cudaSuccess) rc = status_of(e);
  if (rc == DCEM_OK) {
    e = cudaGraphInstantiate(&G.exec, g, 0);
    if (e != cudaSuccess) {
      G.exec = nullptr;
      rc = status_of(e);
    }
  }
  if (rc == DCEM_OK) {
    static unsigned long long captures = 0;
    G.graph = g;
    G.gen = ++captures;
  } else if (g) {
    cudaGraphDestroy(g);
  }
  cudaGetLastError();
  return rc;
}

// The frame's plan, and its captured graph when the plan repeats. Plans
// alternate with the candidate buffers' parity: one cached graph per parity.
// A plan is captured the second time it is seen in a row (the first run also
// sets every kernel's launch attributes), then replayed. Returns whether the
// graph is ready (G.exec and G.graph).
// The kernels launch_diffract runs in a frame of plan P.
static int diffraction_launches(const FramePlan& P) {
  const PathArgs& q = P.q;
  if (!q.wedges) return 0;
  int n = 1 + (q.drefl2 && q.rplanes ? 1 : 0);  // wedge geometry, cluster boxes
  if (P.nlinks > 0) {
    n += 2;  // first-order pre-test, exact stage
    if (q.rplanes) n += 1 + (q.drefl2 ? 2 : 0);  // one reflection; wedge masks, two reflections
    if (q.diff_order >= 2 && q.nw > 1)  // relation, pairs, [pairs around a plane], [triples], chains
      n += q.diff_order + 1 + (q.dmid ? 1 : 0);
  }
  return n;
}
static int plan_frame(dcem_scene* s, int nrx, const dcem_params* p, bool coherent, const dcem_result* out,
                      bool* ready) {
  FramePlan& P = s->plan;
  make_plan(s, nrx, p, coherent, out, P);
  s->last_use_q = P.use_q;
  // kernels of this frame: prep, [mark, carry], trace, capture, dedupe x2, validate x3, reduce, end
  s->launches += 2 + (coherent ? 2 : 0) + (s->R > 0 ? 2 + P.a.max_trans : 0) + 5 + (nrx > 0 ? 1 : 0) +
                 (P.q.vc_next_key ? 1 : 0) +
                 (P.use_q ? 1 : 0) + (P.q.link_off ? 1 : 0) + (P.q.sticky_prev ? 1 : 0) +
                 diffraction_launches(P);
  s->graph_replayed = 0;
  FrameGraph& G = s->fgraph[s->cur];
  bool same = G.have_key && std::memcmp(&G.key, &P, sizeof(P)) == 0;
  if (!same) {
    G.drop();
    G.key = P;
    G.have_key = true;
  }
  if (s->use_graphs && same && !G.exec) {
    int rc = capture_frame(s, P, G);
    if (rc != DCEM_OK) {
      G.have_key = false;
      return rc;
    }
  }
  *ready = s->use_graphs && same && G.exec != nullptr;
  return DCEM_OK;
}

static int trace_once(dcem_scene* s, int nrx, const dcem_params* p, bool coherent, const dcem_result* out) {
  cudaStream_t st = s->st;
  bool ready = false;
  int rc = plan_frame(s, nrx, p, coherent, out, &ready);
  if (rc != DCEM_OK) return rc;
  if (ready) {
    CK(cudaGraphLaunch(s->fgraph[s->cur].exec, st));
    s->graph_replayed = 1;
  } else {
    rc = enqueue_frame(s->plan, s->sms, st, false);
    if (rc != DCEM_OK) return rc;
  }
  CK(cudaStreamSynchronize(st));
  s->cur ^= 1;
  return DCEM_OK;
}

int dcem_trace_frame(dcem_scene* s, const float* tx, const float* rx, int32_t nrx, int32_t rx_ptr_kind,
                     const dcem_params* p, dcem_result* out) {
  if (s && s->rays_set && s->nsets != 1) return DCEM_ERR_STATE;
  return dcem_trace_links(s, tx, 1, rx, nrx, rx_ptr_kind, p, out);
}

// Checks a frame's arguments, sizes the buffers and stages its inputs (the
// receivers' copy on the scene stream, the transmitters in pinned memory);
// decides whether the frame may reuse the cache.
static int frame_begin(dcem_scene* s, const float* tx, int32_t ntx, const float* rx, int32_t nrx,
                       int32_t rx_ptr_kind, const dcem_params* p, dcem_result* out, bool* coherent) {
  if (!s || !tx || !p || !out || ntx < 1) return DCEM_ERR_ARG;
  if (nrx < 0 || (nrx > 0 && !rx)) return DCEM_ERR_ARG;
  if (nrx > kSmallBuild || (long long)ntx * nrx > kMaxLinks) return DCEM_ERR_ARG;
  if (rx_ptr_kind != DCEM_PTR_HOST && rx_ptr_kind != DCEM_PTR_DEVICE) return DCEM_ERR_ARG;
  if (out->ptr_kind != DCEM_PTR_HOST && out->ptr_kind != DCEM_PTR_DEVICE) return DCEM_ERR_ARG;
  if (out->max_paths < 0 || (out->max_paths > 0 && !out->paths)) return DCEM_ERR_ARG;
  if (p->max_refl < 0 || p->max_refl + s->max_trans > DCEM_MAX_REFL) return DCEM_ERR_ARG;
  if (p->mode != DCEM_MODE_FULL && p->mode != DCEM_MODE_COHERENT && p->mode != DCEM_MODE_STICKY)
    return DCEM_ERR_ARG;
  if (p->timing < 0 || p->timing > 2) return DCEM_ERR_ARG;
  if (p->prec != DCEM_PREC_F64 && p->prec != DCEM_PREC_DF32) return DCEM_ERR_ARG;
  if (!(p->freq_hz > 0) || !std::isfinite(p->freq_hz) || !(p->tx_power_w > 0) || !std::isfinite(p->tx_power_w))
    return DCEM_ERR_ARG;
  if (!(p->rx_radius_scale > 0) || !std::isfinite(p->rx_radius_scale) || !(p->t_min >= 0) ||
      !std::isfinite(p->t_min) || !(p->escape_len > 0) || !std::isfinite(p->escape_len) ||
      !(p->eps_occ >= 0) || !(p->eps_occ < 0.5f))
    return DCEM_ERR_ARG;
  if (!finite_arr(p->pol, 3) || !(p->pol[0] * p->pol[0] + p->pol[1] * p->pol[1] + p->pol[2] * p->pol[2] > 0))
    return DCEM_ERR_ARG;
  if (!finite_arr(tx, 3 * (size_t)ntx)) return DCEM_ERR_NONFINITE;
  if (rx_ptr_kind == DCEM_PTR_HOST && nrx > 0 && !finite_arr(rx, 3 * (size_t)nrx)) return DCEM_ERR_NONFINITE;
  if (!s->rays_set || ntx != s->nsets) return DCEM_ERR_STATE;
  std::memset(&out->stats, 0, sizeof(out->stats));
  out->n_paths = 0;

  int rc;
  // transmission: W segments per slot and child slots after the primaries
  const int W = p->max_refl + s->max_trans + 1;
  const int cc = s->max_trans > 0 ? std::max(s->child_cap, std::max(s->R, 1024)) : 0;
  if ((long long)s->R + cc > (1ll << 27)) return DCEM_ERR_CAPACITY;
  if ((rc = ensure_log(s, W, cc)) != DCEM_OK) return rc;
  unsigned want_c = s->cand_cap ? s->cand_cap : (unsigned)std::max(65536, s->R / 8);
  unsigned want_u = s->ucap ? s->ucap : std::min(want_c, 1u << 18);
  if ((rc = ensure_paths(s, want_c, want_u)) != DCEM_OK) return rc;
  const int nlinks = ntx * nrx;
  if ((rc = ensure_rx(s, nrx, nlinks, s->bucket_cap)) != DCEM_OK) return rc;
  if ((rc = ensure_rmask(s, ntx, nrx)) != DCEM_OK) return rc;
  cudaStream_t st = s->st;
  for (int t = 0; t < ntx; ++t)
    s->txs_h[t] = make_float4(tx[3 * t], tx[3 * t + 1], tx[3 * t + 2], alpha_eff_of(s->set_rays_h[t], p));
  if (nrx)
    CK(cudaMemcpyAsync(s->rx3, rx, sizeof(float) * 3 * nrx,
                       rx_ptr_kind == DCEM_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));

  *coherent = p->mode != DCEM_MODE_FULL && s->cache_valid && same_traversal(*p, s->cparams) &&
                  nrx == s->cnrx && s->ctx.size() == 3 * (size_t)ntx &&
                  std::memcmp(tx, s->ctx.data(), sizeof(float) * 3 * ntx) == 0 &&
                  s->logW == p->max_refl + 1 && s->max_trans == 0;
  return DCEM_OK;
}

// After the frame's first trace: regrowth and retrace on an internal
// capacity overflow, the statistics, the copy-out and the cache state.
static int frame_finish(dcem_scene* s, const float* tx, int32_t ntx, const float* rx, int32_t nrx,
                        int32_t rx_ptr_kind, const dcem_params* p, dcem_result* out, bool coherent, bool traced) {
  int rc = DCEM_OK;
  cudaStream_t st = s->st;
  const int nlinks = ntx * nrx;
  DevCounters* c = nullptr;
  for (int attempt = 0; attempt < 4; ++attempt) {
    if (!(traced && attempt == 0)) {
      rc = trace_once(s, nrx, p, coherent, out);
      if (rc != DCEM_OK) {
        s->cache_valid = false;
        return rc;
      }
    }
    c = s->ctr_h;
    unsigned err = c[0].err | c[1].err;
    unsigned grow = err & (ERR_CAND_OVERFLOW | ERR_UNIQUE_OVERFLOW | ERR_HASH_FULL | ERR_BUCKET_OVERFLOW |
                           ERR_SPAWN_OVERFLOW | ERR_DIFF_OVERFLOW);
    if (!grow) break;
    // internal capacity exceeded: grow and retrace the frame from scratch
    CK(cudaStreamSynchronize(st));
    unsigned nc = std::max(s->cand_cap, (unsigned)std::min<unsigned long long>(
                                            0x3fffffffull, (unsigned long long)c[0].n_cand * 3 / 2 + 1024));
    unsigned nu = std::max(s->ucap, std::min(nc, c[0].n_unique * 3 / 2 + 1024));
    if (err & (ERR_CAND_OVERFLOW | ERR_HASH_FULL)) nc = std::max(nc, 2 * s->cand_cap);
    if ((rc = ensure_paths(s, nc, nu)) != DCEM_OK) return rc;
    CK(cudaMemsetAsync(s->hkey, 0, sizeof(unsigned long long) * s->hcap, st));
    CK(cudaMemsetAsync(s->hrep, 0xff, sizeof(unsigned long long) * s->hcap, st));
    if (err & ERR_SPAWN_OVERFLOW) {  // more transmission children than slots
      unsigned long long sp = 0;
      for (int k = 0; k <= kMaxRefl; ++k) sp += c[0].n_spawn[k];
      long long cc = std::max<long long>(2ll * s->child_cap, (long long)(sp * 5 / 4) + 1024);
      if ((long long)s->R + cc > (1ll << 27)) return DCEM_ERR_CAPACITY;
      if ((rc = ensure_log(s, s->logW, (int)cc)) != DCEM_OK) return rc;
    }
    if (err & ERR_DIFF_OVERFLOW) {  // more diffraction pre-test survivors (or wedge pairs, triples) than slots
      auto grow = [&](unsigned n, unsigned& cap, auto*& buf) -> int {
        if (n <= cap) return DCEM_OK;
        unsigned long long want = std::max<unsigned long long>(2ull * cap, (unsigned long long)n * 5 / 4 + 1024);
        if (want > 0x7fffffffull) return DCEM_ERR_CAPACITY;
        dfree(buf);
        CK(dalloc(&buf, (size_t)want));
        cap = (unsigned)want;
        return DCEM_OK;
      };
      if ((rc = grow(c[0].n_dsurv, s->dsurv_cap, s->dsurv)) != DCEM_OK) return rc;
      if (s->dseq2 && (rc = grow(c[0].n_dpair, s->dseq2_cap, s->dseq2)) != DCEM_OK) return rc;
      if (s->dseq3 && (rc = grow(c[0].n_dtrip, s->dseq3_cap, s->dseq3)) != DCEM_OK) return rc;
    }
    if (err & ERR_BUCKET_OVERFLOW) {
      int nb = s->bucket_cap * 2;
      if (nb > 8192) {
        s->cache_valid = false;
        return DCEM_ERR_CAPACITY;
      }
      if ((rc = ensure_rx(s, nrx, nlinks, nb)) != DCEM_OK) return rc;
      CK(cudaMemcpyAsync(s->rx3, rx, sizeof(float) * 3 * nrx,
                         rx_ptr_kind == DCEM_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    }
    coherent = false;
    s->cache_valid = false;
    if (attempt == 3) return DCEM_ERR_CAPACITY;
  }
  unsigned err = c[0].err | c[1].err;
  dcem_stats& S = out->stats;
  S.n_rays = s->R;
  S.segments_traced = (int64_t)c[0].segments_traced;
  S.segments_reused = (int64_t)c[0].segments_reused;
  S.rays_retraced = coherent ? (int64_t)c[0].n_retrace : (int64_t)s->R;
  S.candidates = c[0].n_cand;
  S.candidates_reused = c[0].n_cand_reused;
  S.unique_candidates = c[0].n_unique;
  S.paths_valid = c[0].n_valid;
  S.objects_moved = coherent ? (int64_t)c[0].objects_moved : (int64_t)s->nobj;
  S.rx_moved = c[0].rx_moved;
  S.node_visits = (int64_t)c[0].node_visits;
  S.max_segment_nodes = (int32_t)c[0].max_seg_nodes;
  S.trace_kernel = s->last_use_q;
  S.graph_replayed = s->graph_replayed;
  S.paths_sticky = (int32_t)c[0].n_sticky_valid;
  {
    unsigned long long sp = 0;
    for (int k = 0; k <= kMaxRefl; ++k) sp += c[0].n_spawn[k];
    S.child_rays = (int32_t)std::min<unsigned long long>(sp, 0x7fffffffull);
  }
  S.keys_reused = (int32_t)c[0].n_val_reused;
  S.diff_candidates = (int32_t)std::min(c[0].n_dsurv, 0x7fffffffu);
  S.diff_pairs = (int32_t)std::min(c[0].n_dpair, 0x7fffffffu);
  S.diff_triples = (int32_t)std::min(c[0].n_dtrip, 0x7fffffffu);
  S.tri_tests = (int64_t)c[0].tri_tests;
  S.stack_overflow = (int32_t)c[0].stack_overflow;
  S.coherent = coherent ? 1 : 0;
  S.kernel_launches = s->launches;
  s->launches = 0;
  if (c[1].sah_build > 0.0f) s->sah_build = c[1].sah_build;
  if (c[1].sah_refit > 0.0f) s->sah_now = c[1].sah_refit;
  S.bvh_rebuilt = s->rebuilt_since_frame ? 1 : 0;
  s->rebuilt_since_frame = false;
  S.bvh_cost_ratio = s->sah_build > 0.0f ? s->sah_now / s->sah_build : 0.0f;
  s->last_ncand = std::min(c[0].n_cand, s->cand_cap);
  if (err & ERR_HASH_COLLISION) {
    s->cache_valid = false;
    CK(cudaMemsetAsync(s->hkey, 0, sizeof(unsigned long long) * s->hcap, st));
    CK(cudaMemsetAsync(s->hrep, 0xff, sizeof(unsigned long long) * s->hcap, st));
    return DCEM_ERR_HASH;
  }
  if (err & ERR_NONFINITE) {
    s->cache_valid = false;
    return DCEM_ERR_NONFINITE;
  }
  // copy out
  bool tm = p->timing == 1;
  int nvalid = (int)c[0].n_valid;
  if (out->ptr_kind == DCEM_PTR_HOST) {
    cudaMemcpyKind k = cudaMemcpyDeviceToHost;
    size_t cap = (size_t)s->nlink_cap;
    if (nlinks) {
      if (out->field) CK(cudaMemcpyAsync(out->field, s->rxout, sizeof(double) * 2 * nlinks, k, st));
      if (out->p_coh_dbm)
        CK(cudaMemcpyAsync(out->p_coh_dbm, s->rxout + 2 * cap, sizeof(double) * nlinks, k, st));
      if (out->p_inc_dbm)
        CK(cudaMemcpyAsync(out->p_inc_dbm, s->rxout + 3 * cap, sizeof(double) * nlinks, k, st));
    }
    int ncopy = std::min(nvalid, out->max_paths);
    if (ncopy > 0 && out->paths) CK(cudaMemcpyAsync(out->paths, s->pout, sizeof(dcem_path) * ncopy, k, st));
  }
  if (out->ptr_kind == DCEM_PTR_HOST) {
    if (tm) CK(cudaEventRecord(s->ev[8], st));
    CK(cudaStreamSynchronize(st));
  }
  if (tm) {
    for (int i = 0; i < 8; ++i) cudaEventElapsedTime(&S.ms_stage[i], s->ev[i], s->ev[i + 1]);
    cudaEventElapsedTime(&S.ms_stage[8], s->ev[0], s->ev[8]);
  } else if (p->timing == 2 && s->R > 0) {
    for (int i = 0; i < 10; ++i) S.ms_stage[i] = 0.0f;
    cudaEventElapsedTime(&S.ms_stage[2], s->ev[2], s->ev[3]);
  }
  if (checks_take_all()) {  // bounds-checked build: an index was out of range
    s->cache_valid = false;
    return DCEM_ERR_CHECK;
  }
  out->n_paths = nvalid;
  s->cache_valid = true;
  s->vc_valid = p->mode == DCEM_MODE_COHERENT && s->max_trans == 0;  // this frame built its key table
  s->cparams = *p;
  s->ctx.assign(tx, tx + 3 * ntx);
  s->cnrx = nrx;
  if (err & ERR_STACK) return DCEM_ERR_STACK;
  if (nvalid > out->max_paths && out->paths) return DCEM_ERR_CAPACITY;
  return DCEM_OK;
}

int dcem_trace_links(dcem_scene* s, const float* tx, int32_t ntx, const float* rx, int32_t nrx,
                     int32_t rx_ptr_kind, const dcem_params* p, dcem_result* out) {
  bool coherent = false;
  int rc = frame_begin(s, tx, ntx, rx, nrx, rx_ptr_kind, p, out, &coherent);
  if (rc != DCEM_OK) return rc;
  return frame_finish(s, tx, ntx, rx, nrx, rx_ptr_kind, p, out, coherent, false);
}

// ---------------------------------------------------------------------------
// several scenes per frame
// ---------------------------------------------------------------------------
}  // extern "C"

struct dcem_batch {
  std::vector<dcem_scene*> sc;
  cudaStream_t st = nullptr;
  std::vector<cudaStream_t> fork;  // streams of the concurrent per-scene updates
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork_ev = nullptr;
  // batch graphs: one child per scene (its captured frame), keyed by the
  // children's capture numbers; two kept (the candidate parities alternate)
  struct Parent {
    std::vector<unsigned long long> kids;
    cudaGraphExec_t exec = nullptr;
  } parent[2];
  int victim = 0;
  // one closest-hit launch for every scene (frames without timing or
  // transmission): the scenes' trace arguments staged in pinned memory and
  // copied in by the frame, the launch's chunk counter, and the captured
  // frames keyed by the scenes' plans (captured the second time a key is seen)
  TraceArgs* h_tab = nullptr;
  TraceArgs* d_tab = nullptr;
  unsigned* d_chunk = nullptr;
  cudaStream_t cap_st = nullptr;
  struct One {
    std::vector<FramePlan> keys;
    cudaGraphExec_t exec = nullptr;
  } one[2];
  std::vector<FramePlan> pending[2];  // by the frames' parity (the candidate buffers alternate)
  int one_victim = 0;
};

namespace {

void batch_free(dcem_batch* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  for (auto& p : b->parent)
    if (p.exec) cudaGraphExecDestroy(p.exec);
  for (auto& o : b->one)
    if (o.exec) cudaGraphExecDestroy(o.exec);
  if (b->h_tab) cudaFreeHost(b->h_tab);
  dfree(b->d_tab);
  dfree(b->d_chunk);
  if (b->cap_st) cudaStreamDestroy(b->cap_st);
  for (auto f : b->fork) cudaStreamDestroy(f);
  for (auto e : b->join) cudaEventDestroy(e);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  delete b;
}

// The batch graph over the scenes' current frame graphs: reused when the
// same captures are its children, else built (and the older one replaced).
int batch_graph(dcem_batch* b, cudaGraphExec_t* exec) {
  std::vector<unsigned long long> kids;
  for (dcem_scene* s : b->sc) kids.push_back(s->fgraph[s->cur].gen);
  for (auto& p : b->parent)
    if (p.exec && p.kids == kids) {
      *exec = p.exec;
      return DCEM_OK;
    }
  auto& p = b->parent[b->victim];
  b->victim ^= 1;
  if (p.exec) cudaGraphExecDestroy(p.exec);
  p.exec = nullptr;
  p.kids.clear();
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaError_t e = cudaSuccess;
  for (dcem_scene* s : b->sc) {
    cudaGraphNode_t node;
    e = cudaGraphAddChildGraphNode(&node, g, nullptr, 0, s->fgraph[s->cur].graph);
    if (e != cudaSuccess) break;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p.exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    p.exec = nullptr;
    return status_of(e);
  }
  p.kids = kids;
  *exec = p.exec;
  return DCEM_OK;
}

// Every scene's frame with one closest-hit launch between the scenes'
// preparation and their capture, dedupe, validation and reduction; the
// scenes' own stages run on the fork streams in turn. Stream order only.
int batch_enqueue(dcem_batch* b, cudaStream_t st, bool cap) {
  const int n = (int)b->sc.size(), nf = (int)b->fork.size();
  CK(cudaEventRecord(b->fork_ev, st));
  for (int k = 0; k < nf; ++k) CK(cudaStreamWaitEvent(b->fork[k], b->fork_ev, 0));
  for (int i = 0; i < n; ++i) {
    int rc = enqueue_pre(b->sc[i]->plan, b->sc[i]->sms, b->fork[i % nf], cap, false);
    if (rc != DCEM_OK) return rc;
  }
  for (int k = 0; k < nf; ++k) {
    CK(cudaEventRecord(b->join[k], b->fork[k]));
    CK(cudaStreamWaitEvent(st, b->join[k], 0));
  }
  CK(cudaMemcpyAsync(b->d_tab, b->h_tab, sizeof(TraceArgs) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(b->d_chunk, 0, sizeof(unsigned), st));
  CK(launch_trace_batch(b->d_tab, n, b->d_chunk, b->sc[0]->sms, st));
  CK(cudaEventRecord(b->fork_ev, st));
  for (int k = 0; k < nf; ++k) CK(cudaStreamWaitEvent(b->fork[k], b->fork_ev, 0));
  for (int i = 0; i < n; ++i) {
    int rc = enqueue_post(b->sc[i]->plan, b->sc[i]->sms, b->fork[i % nf], cap, false);
    if (rc != DCEM_OK) return rc;
  }
  for (int k = 0; k < nf; ++k) {
    CK(cudaEventRecord(b->join[k], b->fork[k]));
    CK(cudaStreamWaitEvent(st, b->join[k], 0));
  }
  return DCEM_OK;
}

bool same_plans(const std::vector<FramePlan>& a, const std::vector<FramePlan>& b) {
  if (a.size() != b.size()) return false;
  for (size_t i = 0; i < a.size(); ++i)
    if (std::memcmp(&a[i], &b[i], sizeof(FramePlan)) != 0) return false;
  return true;
}

// The one-launch frame of the batch: replays its captured graph when the
// scenes' plans were captured before, captures it the second time the plans
// are seen in a row, else runs it directly (which also sets every kernel's
// launch attributes).
int batch_one_launch(dcem_batch* b, bool* replayed) {
  *replayed = false;
  std::vector<FramePlan> keys;
  for (dcem_scene* s : b->sc) keys.push_back(s->plan);
  for (auto& o : b->one)
    if (o.exec && same_plans(o.keys, keys)) {
      CK(cudaGraphLaunch(o.exec, b->st));
      *replayed = true;
      return DCEM_OK;
    }
  std::vector<FramePlan>& pend = b->pending[b->sc[0]->cur];
  if (!same_plans(pend, keys)) {
    pend = keys;
    return batch_enqueue(b, b->st, false);
  }
  if (!b->cap_st) CK(cudaStreamCreateWithFlags(&b->cap_st, cudaStreamNonBlocking));
  auto& o = b->one[b->one_victim];
  b->one_victim ^= 1;
  if (o.exec) cudaGraphExecDestroy(o.exec);
  o.exec = nullptr;
  o.keys.clear();
  CK(cudaStreamBeginCapture(b->cap_st, cudaStreamCaptureModeThreadLocal));
  int rc = batch_enqueue(b, b->cap_st, true);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->cap_st, &g);
  if (rc == DCEM_OK && e != cudaSuccess) rc = status_of(e);
  if (rc == DCEM_OK) {
    e = cudaGraphInstantiate(&o.exec, g, 0);
    if (e != cudaSuccess) {
      o.exec = nullptr;
      rc = status_of(e);
    }
  }
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  if (rc != DCEM_OK) return rc;
  o.keys = keys;
  CK(cudaGraphLaunch(o.exec, b->st));
  *replayed = true;
  return DCEM_OK;
}

}  // namespace

extern "C" {

int dcem_batch_create(dcem_scene* const* scenes, int32_t n, void* stream, dcem_batch** out) {
  if (!scenes || !out || n < 1 || n > kMaxBatch) return DCEM_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!scenes[i]) return DCEM_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (scenes[j] == scenes[i]) return DCEM_ERR_ARG;
  }
  dcem_batch* b = new dcem_batch;
  b->st = (cudaStream_t)stream;
  b->sc.assign(scenes, scenes + n);
  int nf = std::min(n, 8);
  cudaError_t e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
  for (int k = 0; k < nf && e == cudaSuccess; ++k) {
    cudaStream_t f;
    cudaEvent_t j;
    e = cudaStreamCreateWithFlags(&f, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->fork.push_back(f);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
    if (e == cudaSuccess) b->join.push_back(j);
  }
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    int rc = dcem_scene_set_stream(scenes[i], stream);
    if (rc != DCEM_OK) e = cudaErrorUnknown;
  }
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_tab, sizeof(TraceArgs) * n);
  if (e == cudaSuccess) e = dalloc(&b->d_tab, (size_t)n);
  if (e == cudaSuccess) e = dalloc(&b->d_chunk, (size_t)1);
  if (e != cudaSuccess) {
    batch_free(b);
    return status_of(e);
  }
  *out = b;
  return DCEM_OK;
}

int dcem_batch_update_transforms(dcem_batch* b, const float* const* xf, int32_t ptr_kind) {
  if (!b || !xf) return DCEM_ERR_ARG;
  if (ptr_kind != DCEM_PTR_HOST && ptr_kind != DCEM_PTR_DEVICE) return DCEM_ERR_ARG;
  // host transforms are checked before any work is enqueued
  for (size_t i = 0; i < b->sc.size(); ++i) {
    dcem_scene* s = b->sc[i];
    if (s->nobj > 0 && !xf[i]) return DCEM_ERR_ARG;
    if (s->nobj > 0 && ptr_kind == DCEM_PTR_HOST && !finite_arr(xf[i], 12 * (size_t)s->nobj))
      return DCEM_ERR_NONFINITE;
  }
  const int nf = (int)b->fork.size();
  CK(cudaEventRecord(b->fork_ev, b->st));
  for (int k = 0; k < nf; ++k) CK(cudaStreamWaitEvent(b->fork[k], b->fork_ev, 0));
  int rc = DCEM_OK;
  for (size_t i = 0; i < b->sc.size() && rc == DCEM_OK; ++i) {
    dcem_scene* s = b->sc[i];
    if (s->nobj == 0) continue;
    s->st = b->fork[i % nf];
    rc = dcem_scene_update_transforms(s, xf[i], ptr_kind);
    s->st = b->st;
  }
  for (int k = 0; k < nf; ++k) {
    CK(cudaEventRecord(b->join[k], b->fork[k]));
    CK(cudaStreamWaitEvent(b->st, b->join[k], 0));
  }
  return rc;
}

int dcem_batch_trace(dcem_batch* b, const float* const* tx, const int32_t* ntx, const float* const* rx,
                     const int32_t* nrx, int32_t rx_ptr_kind, const dcem_params* p, dcem_result* out,
                     int32_t* failed) {
  if (failed) *failed = -1;
  if (!b || !tx || !ntx || !rx || !nrx || !p || !out) return DCEM_ERR_ARG;
  const int n = (int)b->sc.size();
  std::vector<char> coh(n, 0);
  auto fail = [&](int i, int rc) {
    if (failed) *failed = i;
    return rc;
  };
  for (int i = 0; i < n; ++i) {
    bool c = false;
    int rc = frame_begin(b->sc[i], tx[i], ntx[i], rx[i], nrx[i], rx_ptr_kind, p, &out[i], &c);
    if (rc != DCEM_OK) return fail(i, rc);
    coh[i] = c;
  }
  // frames without timing and transmission: one closest-hit launch for
  // every scene's rays
  bool one = p->timing == 0;
  for (int i = 0; i < n; ++i) one = one && b->sc[i]->max_trans == 0;
  if (one) {
    for (int i = 0; i < n; ++i) {
      dcem_scene* s = b->sc[i];
      make_plan(s, nrx[i], p, coh[i] != 0, &out[i], s->plan);
      FramePlan& P = s->plan;
      P.use_q = 0;  // the batch launch reads the binary nodes from L2: no compact copy
      P.a.use_q = 0;
      s->last_use_q = 3;  // every scene's rays in one launch
      s->launches += 2 + (coh[i] ? 2 : 0) + (s->R > 0 ? 1 : 0) + 5 + (nrx[i] > 0 ? 1 : 0) +
                     (P.q.vc_next_key ? 1 : 0) + (P.use_q ? 1 : 0) + (P.q.link_off ? 1 : 0) +
                     (P.q.sticky_prev ? 1 : 0) + diffraction_launches(P) + (i == 0 ? 1 : 0);
      s->graph_replayed = 0;
      b->h_tab[i] = frame_trace_args(P);
    }
    bool replayed = false;
    int rc = batch_one_launch(b, &replayed);
    if (rc != DCEM_OK) return fail(0, rc);
    CK(cudaStreamSynchronize(b->st));
    for (dcem_scene* s : b->sc) {
      s->cur ^= 1;
      s->graph_replayed = replayed ? 1 : 0;
    }
    int first = DCEM_OK;
    for (int i = 0; i < n; ++i) {
      int rc2 = frame_finish(b->sc[i], tx[i], ntx[i], rx[i], nrx[i], rx_ptr_kind, p, &out[i], coh[i] != 0, true);
      if (rc2 != DCEM_OK && first == DCEM_OK) {
        first = rc2;
        if (failed) *failed = i;
      }
    }
    return first;
  }
  // every scene's frame graph ready (and no event timing): one launch
  bool all = p->timing == 0;
  for (int i = 0; i < n; ++i) {
    bool ready = false;
    int rc = plan_frame(b->sc[i], nrx[i], p, coh[i] != 0, &out[i], &ready);
    if (rc != DCEM_OK) return fail(i, rc);
    all = all && ready;
  }
  if (all) {
    cudaGraphExec_t exec = nullptr;
    int rc = batch_graph(b, &exec);
    if (rc != DCEM_OK) return fail(0, rc);
    CK(cudaGraphLaunch(exec, b->st));
    for (dcem_scene* s : b->sc) s->graph_replayed = 1;
  } else {
    for (int i = 0; i < n; ++i) {
      int rc = enqueue_frame(b->sc[i]->plan, b->sc[i]->sms, b->st, false);
      if (rc != DCEM_OK) return fail(i, rc);
    }
  }
  CK(cudaStreamSynchronize(b->st));
  for (dcem_scene* s : b->sc) s->cur ^= 1;
  int first = DCEM_OK;
  for (int i = 0; i < n; ++i) {
    int rc = frame_finish(b->sc[i], tx[i], ntx[i], rx[i], nrx[i], rx_ptr_kind, p, &out[i], coh[i] != 0, true);
    if (rc != DCEM_OK && first == DCEM_OK) {
      first = rc;
      if (failed) *failed = i;
    }
  }
  return first;
}

void dcem_batch_destroy(dcem_batch* b) { batch_free(b); }

int dcem_scene_gradient_size(const dcem_scene* s, int32_t* n_params) {
  if (!s || !n_params) return DCEM_ERR_ARG;
  *n_params = grad_nparam(s->nmat, s->nobj);
  return DCEM_OK;
}

}  // extern "C"

// Field derivatives over a fixed path topology: forward mode (one thread per
// (path, parameter)) at the scene's parameters, or the adjoint kernel (one
// thread per path) at theta (null: the scene's parameters).
static int path_derivs(dcem_scene* s, const float* tx, const float* rx, int32_t nrx, int32_t rx_ptr_kind,
                       const dcem_path* paths, int32_t n_paths, const dcem_params* p, const double* theta,
                       const double* pcoh_bar, int32_t ptr_kind, double* field, double* pcoh_dbm, double* dfield,
                       double* dpcoh_dbm, double* theta_bar, bool adjoint) {
  if (!s || !tx || !p) return DCEM_ERR_ARG;
  if (nrx < 0 || nrx > kSmallBuild || (nrx > 0 && !rx) || n_paths < 0 || (n_paths > 0 && !paths))
    return DCEM_ERR_ARG;
  if (!adjoint && nrx > 0 && !dfield) return DCEM_ERR_ARG;
  if (theta_bar && !pcoh_bar) return DCEM_ERR_ARG;
  if (rx_ptr_kind != DCEM_PTR_HOST && rx_ptr_kind != DCEM_PTR_DEVICE) return DCEM_ERR_ARG;
  if (ptr_kind != DCEM_PTR_HOST && ptr_kind != DCEM_PTR_DEVICE) return DCEM_ERR_ARG;
  if (p->max_refl < 0 || p->max_refl > DCEM_MAX_REFL) return DCEM_ERR_ARG;
  if (!(p->freq_hz > 0) || !std::isfinite(p->freq_hz) || !(p->tx_power_w > 0) || !std::isfinite(p->tx_power_w))
    return DCEM_ERR_ARG;
  if (!finite_arr(p->pol, 3) || !(p->pol[0] * p->pol[0] + p->pol[1] * p->pol[1] + p->pol[2] * p->pol[2] > 0))
    return DCEM_ERR_ARG;
  if (!finite_arr(tx, 3)) return DCEM_ERR_NONFINITE;
  if (rx_ptr_kind == DCEM_PTR_HOST && nrx > 0 && !finite_arr(rx, 3 * (size_t)nrx)) return DCEM_ERR_NONFINITE;
  const int np = grad_nparam(s->nmat, s->nobj);
  if (theta && ptr_kind == DCEM_PTR_HOST) {
    for (int i = 0; i < np; ++i)
      if (!std::isfinite(theta[i])) return DCEM_ERR_NONFINITE;
  }
  cudaStream_t st = s->st;
  if (nrx == 0) {  // no receiver: nothing depends on theta
    if (theta_bar && np > 0) {
      if (ptr_kind == DCEM_PTR_HOST) std::fill(theta_bar, theta_bar + np, 0.0);
      else CK(cudaMemsetAsync(theta_bar, 0, sizeof(double) * np, st));
      CK(cudaStreamSynchronize(st));
    }
    return DCEM_OK;
  }
  const int W = 1 + 4 * p->max_refl;
  // device copies of the inputs given on the host, scratch, staged outputs
  if ((size_t)nrx > s->g_rx_cap) {
    dfree(s->g_rx);
    CK(dalloc(&s->g_rx, (size_t)nrx));
    s->g_rx_cap = (size_t)nrx;
  }
  if (rx_ptr_kind == DCEM_PTR_HOST) {
    std::vector<float4> h((size_t)nrx);
    for (int i = 0; i < nrx; ++i) h[i] = make_float4(rx[3 * i], rx[3 * i + 1], rx[3 * i + 2], 0.0f);
    CK(cudaMemcpyAsync(s->g_rx, h.data(), sizeof(float4) * nrx, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));  // h goes out of scope
  } else {
    CK(launch_pack_rx(rx, nrx, s->g_rx, st));
  }
  const dcem_path* pd = paths;
  if (ptr_kind == DCEM_PTR_HOST && n_paths > 0) {
    if ((size_t)n_paths > s->g_paths_cap) {
      dfree(s->g_paths);
      CK(dalloc(&s->g_paths, (size_t)n_paths));
      s->g_paths_cap = (size_t)n_paths;
    }
    CK(cudaMemcpyAsync(s->g_paths, paths, sizeof(dcem_path) * n_paths, cudaMemcpyHostToDevice, st));
    pd = s->g_paths;
  }
  size_t nitems = (size_t)n_paths * W;
  if (nitems > s->g_items_cap) {
    dfree(s->g_items);
    dfree(s->g_param);
    CK(dalloc(&s->g_items, nitems));
    CK(dalloc(&s->g_param, nitems));
    s->g_items_cap = nitems;
  }
  // staging: field 2 nrx, P_coh nrx, dfield 2 nrx np, dpcoh nrx np, theta_bar np,
  // pcoh_bar nrx, theta np
  const size_t o_pc = 2 * (size_t)nrx, o_df = o_pc + nrx, o_dp = o_df + 2 * (size_t)nrx * np,
               o_tb = o_dp + (size_t)nrx * np, o_pb = o_tb + np, o_th = o_pb + nrx, nout = o_th + np;
  if (nout > s->g_out_cap) {
    dfree(s->g_out);
    CK(dalloc(&s->g_out, nout));
    s->g_out_cap = nout;
  }
  double* G = s->g_out;
  if (!s->g_err) CK(dalloc(&s->g_err, 1));
  CK(cudaMemsetAsync(s->g_err, 0, sizeof(unsigned), st));
  const bool dev = ptr_kind == DCEM_PTR_DEVICE;
  const double* theta_d = theta;
  const double* pbar_d = pcoh_bar;
  if (!dev && theta) {
    CK(cudaMemcpyAsync(G + o_th, theta, sizeof(double) * np, cudaMemcpyHostToDevice, st));
    theta_d = G + o_th;
  }
  if (!dev && pcoh_bar) {
    CK(cudaMemcpyAsync(G + o_pb, pcoh_bar, sizeof(double) * nrx, cudaMemcpyHostToDevice, st));
    pbar_d = G + o_pb;
  }
  GradArgs g;
  g.theta = theta_d;
  g.xf = s->xf_cur;
  g.pcoh_bar = pbar_d;
  g.paths = pd;
  g.n_paths = n_paths;
  g.W = W;
  g.max_refl = p->max_refl;
  g.tris = s->tris;
  g.slot_of_id = s->slot_of_id;
  g.tri_mat = s->tri_mat_d;
  g.tri_obj = s->tri_obj_d;
  g.ntri = s->ntri;
  g.mats = s->mats;
  g.nmat = s->nmat;
  g.nobj = s->nobj;
  g.rx = s->g_rx;
  g.nrx = nrx;
  for (int k = 0; k < 3; ++k) {
    g.tx[k] = tx[k];
    g.pol[k] = p->pol[k];
  }
  g.freq = p->freq_hz;
  g.tx_power = p->tx_power_w;
  g.items = s->g_items;
  g.param = s->g_param;
  g.err = s->g_err;
  g.field = dev && field ? field : G;
  g.pcoh = dev && pcoh_dbm ? pcoh_dbm : G + o_pc;
  g.dfield = dev && dfield ? dfield : G + o_df;
  g.dpcoh = dev && dpcoh_dbm ? dpcoh_dbm : G + o_dp;
  g.theta_bar = theta_bar ? (dev ? theta_bar : G + o_tb) : nullptr;
  CK(adjoint ? launch_adjoint(g, st) : launch_gradients(g, st));
  s->launches += (n_paths > 0 ? 1 : 0) + 1 + (rx_ptr_kind == DCEM_PTR_DEVICE ? 1 : 0) + (g.theta_bar ? 1 : 0);
  unsigned err = 0;
  CK(cudaMemcpyAsync(&err, s->g_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  if (!dev) {
    cudaMemcpyKind k = cudaMemcpyDeviceToHost;
    if (field) CK(cudaMemcpyAsync(field, g.field, sizeof(double) * 2 * nrx, k, st));
    if (pcoh_dbm) CK(cudaMemcpyAsync(pcoh_dbm, g.pcoh, sizeof(double) * nrx, k, st));
    if (dfield) CK(cudaMemcpyAsync(dfield, g.dfield, sizeof(double) * 2 * (size_t)nrx * np, k, st));
    if (dpcoh_dbm) CK(cudaMemcpyAsync(dpcoh_dbm, g.dpcoh, sizeof(double) * (size_t)nrx * np, k, st));
    if (theta_bar) CK(cudaMemcpyAsync(theta_bar, g.theta_bar, sizeof(double) * np, k, st));
  }
  CK(cudaStreamSynchronize(st));
  if (checks_take_all()) return DCEM_ERR_CHECK;
  return err ? DCEM_ERR_ARG : DCEM_OK;
}

extern "C" {

int dcem_path_gradients(dcem_scene* s, const float* tx, const float* rx, int32_t nrx, int32_t rx_ptr_kind,
                        const dcem_path* paths, int32_t n_paths, const dcem_params* p, int32_t ptr_kind,
                        double* field, double* dfield, double* dpcoh_dbm) {
  return path_derivs(s, tx, rx, nrx, rx_ptr_kind, paths, n_paths, p, nullptr, nullptr, ptr_kind, field, nullptr,
                     dfield, dpcoh_dbm, nullptr, false);
}

int dcem_path_adjoint(dcem_scene* s, const float* tx, const float* rx, int32_t nrx, int32_t rx_ptr_kind,
                      const dcem_path* paths, int32_t n_paths, const dcem_params* p, const double* theta,
                      const double* pcoh_bar, int32_t ptr_kind, double* field, double* pcoh_dbm, double* dfield,
                      double* dpcoh_dbm, double* theta_bar) {
  return path_derivs(s, tx, rx, nrx, rx_ptr_kind, paths, n_paths, p, theta, pcoh_bar, ptr_kind, field, pcoh_dbm,
                     dfield, dpcoh_dbm, theta_bar, true);
}

int dcem_scene_info(const dcem_scene* s, int32_t* ntri, int32_t* nobj, int32_t* n_rays, int32_t* static_nodes,
                    int32_t* dynamic_nodes) {
  if (!s) return DCEM_ERR_ARG;
  if (ntri) *ntri = s->ntri;
  if (nobj) *nobj = s->nobj;
  if (n_rays) *n_rays = s->R;
  if (static_nodes) *static_nodes = s->nint_s;
  if (dynamic_nodes) *dynamic_nodes = s->nint_d;
  return DCEM_OK;
}

int dcem_scene_get_world_tris(dcem_scene* s, float* out) {
  if (!s || (!out && s->ntri > 0)) return DCEM_ERR_ARG;
  if (s->ntri == 0) return DCEM_OK;
  std::vector<float4> t(3 * (size_t)s->ntri);
  CK(cudaStreamSynchronize(s->st));
  CK(cudaMemcpy(t.data(), s->tris, sizeof(float4) * t.size(), cudaMemcpyDeviceToHost));
  for (int slot = 0; slot < s->ntri; ++slot) {
    int id;
    std::memcpy(&id, &t[3 * (size_t)slot].w, 4);
    if (id < 0 || id >= s->ntri) return DCEM_ERR_STATE;
    for (int k = 0; k < 3; ++k) {
      out[9 * (size_t)id + 3 * k] = t[3 * (size_t)slot + k].x;
      out[9 * (size_t)id + 3 * k + 1] = t[3 * (size_t)slot + k].y;
      out[9 * (size_t)id + 3 * k + 2] = t[3 * (size_t)slot + k].z;
    }
  }
  return DCEM_OK;
}

int dcem_scene_get_bvh(dcem_scene* s, int32_t* child, float* bounds, int32_t* roots) {
  if (!s) return DCEM_ERR_ARG;
  int nn = s->nint_s + s->nint_d;
  std::vector<float4> nodes(4 * (size_t)(nn > 0 ? nn : 1));
  std::vector<float4> t(3 * (size_t)(s->ntri > 0 ? s->ntri : 1));
  CK(cudaStreamSynchronize(s->st));
  if (nn) CK(cudaMemcpy(nodes.data(), s->nodes, sizeof(float4) * 4 * nn, cudaMemcpyDeviceToHost));
  if (s->ntri) CK(cudaMemcpy(t.data(), s->tris, sizeof(float4) * 3 * s->ntri, cudaMemcpyDeviceToHost));
  auto conv = [&](int code) -> int {
    if (code == kEmpty || code >= 0) return code;
    int id;
    std::memcpy(&id, &t[3 * (size_t)(~code)].w, 4);
    return -id - 1;
  };
  for (int i = 0; i < nn; ++i) {
    const float4* n = &nodes[4 * (size_t)i];
    int c0, c1;
    std::memcpy(&c0, &n[3].x, 4);
    std::memcpy(&c1, &n[3].y, 4);
    if (child) {
      child[2 * i] = conv(c0);
      child[2 * i + 1] = conv(c1);
    }
    if (bounds) {
      float* b = bounds + 12 * (size_t)i;
      b[0] = n[0].x; b[1] = n[0].z; b[2] = n[2].x; b[3] = n[0].y; b[4] = n[0].w; b[5] = n[2].y;
      b[6] = n[1].x; b[7] = n[1].z; b[8] = n[2].z; b[9] = n[1].y; b[10] = n[1].w; b[11] = n[2].w;
    }
  }
  if (roots) {
    roots[0] = conv(s->root_h[0]);
    roots[1] = conv(s->root_h[1]);
  }
  return DCEM_OK;
}

int dcem_scene_get_ray_log(dcem_scene* s, int32_t* hit_id, float* hit_t, int32_t* nseg) {
  if (!s) return DCEM_ERR_ARG;
  if (!s->rays_set || s->logW == 0) return DCEM_ERR_STATE;
  // the last frame's segments per ray (the log may hold more rows)
  int R = s->R, W = std::min(s->logW, s->cparams.max_refl + s->max_trans + 1), LS = s->LS;
  CK(cudaStreamSynchronize(s->st));
  std::vector<int> ns(R > 0 ? R : 1), ids((size_t)W * (LS > 0 ? LS : 1));
  std::vector<float4> ld((size_t)W * (LS > 0 ? LS : 1));
  if (R) {
    CK(cudaMemcpy(ns.data(), s->nseg, sizeof(int) * R, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(ids.data(), s->log_id, sizeof(int) * (size_t)W * LS, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(ld.data(), s->log_d, sizeof(float4) * (size_t)W * LS, cudaMemcpyDeviceToHost));
  }
  for (int i = 0; i < R; ++i) {  // slot i holds the caller's ray ray_perm[i]
    size_t o = (size_t)s->ray_perm_h[i];
    if (nseg) nseg[o] = ns[i];
    for (int b = 0; b < W; ++b) {
      bool live = b < ns[i];
      if (hit_id) hit_id[o * W + b] = live ? ids[(size_t)b * LS + i] : -2;
      if (hit_t) hit_t[o * W + b] = live ? ld[(size_t)b * LS + i].w : NAN;
    }
  }
  return DCEM_OK;
}

int dcem_scene_get_candidates(dcem_scene* s, int32_t* out, int64_t cap, int64_t* n) {
  if (!s || !n || cap < 0 || (cap > 0 && !out)) return DCEM_ERR_ARG;
  *n = s->last_ncand;
  if (s->last_ncand == 0) return DCEM_OK;
  std::vector<Cand> c(s->last_ncand);
  CK(cudaStreamSynchronize(s->st));
  CK(cudaMemcpy(c.data(), s->cand[s->cur], sizeof(Cand) * c.size(), cudaMemcpyDeviceToHost));
  // a transmission child's capture is reported with its primary ray
  std::vector<int> root;
  if (s->child_cap > 0 && s->inst_root) {
    root.resize(s->child_cap);
    CK(cudaMemcpy(root.data(), s->inst_root, sizeof(int) * root.size(), cudaMemcpyDeviceToHost));
  }
  int64_t m = std::min<int64_t>(cap, (int64_t)c.size());
  for (int64_t i = 0; i < m; ++i) {
    int r = c[i].ray;
    if (r >= s->R) r = r - s->R < (int)root.size() ? root[r - s->R] : -1;
    out[3 * i] = r >= 0 && r < s->R ? s->ray_perm_h[r] : -1;
    out[3 * i + 1] = cand_seg(c[i]);
    out[3 * i + 2] = cand_rx(c[i]);
  }
  return cap < (int64_t)c.size() ? DCEM_ERR_CAPACITY : DCEM_OK;
}

}  // extern "C"

namespace dcem {
DCEM_CHECKS_TAKER(checks_take_api)
}  // namespace dcem
