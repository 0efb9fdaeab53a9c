// trace.cuh -- arguments and launchers of the shooting and coherence kernels.
#pragma once

#include "dcem_internal.cuh"

namespace dcem {

struct TraceArgs {
  Bvh bvh;
  const float4* rays;      // R unit directions (xyz)
  float3 tx;
  int R, N;                // rays, reflections
  float tmin, escape, alpha_eff;
  const float4* rx;        // nrx receivers (xyz)
  int nrx;
  float4* log_o;           // (N+1) x R: origin, unfolded length D
  float4* log_d;           // (N+1) x R: direction, hit t (+inf escaped)
  int* log_id;             // (N+1) x R: hit triangle id or -1
  int* nseg;               // R
  const int* queue;        // retrace queue (null: all rays from segment 0)
  int* queue_w;            // retrace queue written by the marking kernel
  const int* restart;      // R: first segment to retrace
  const unsigned* nq_dev;  // queue length (device)
  Cand* cand;
  unsigned cand_cap;
  DevCounters* ctr;
};

struct CoherentArgs {
  int nobj;
  const float* xf_cur;
  const float* xf_traced;
  const unsigned* obj_box_cur;     // ordered-int boxes: lo [0,3nobj), hi [3nobj,6nobj)
  const unsigned* obj_box_traced;
  float* moved_boxes;              // 2 nobj x 6
  const int* moved_list;           // moved receivers
  const unsigned char* rx_moved;   // nrx flags
  int* restart;                    // R
  DevCounters* ctr;
  const Cand* prev_cand;
  const unsigned* prev_ncand;
  unsigned prev_cap;
  int smem_boxes, smem_rx;         // shared-memory staging sizes
};

cudaError_t launch_trace(const TraceArgs& a, int grid_cap, cudaStream_t st);
cudaError_t launch_coherent_prep(const CoherentArgs& c, cudaStream_t st);
cudaError_t launch_rx_pack(const float* d_rx3, int nrx, float4* rx_cur, const float4* rx_traced,
                           int have_prev, unsigned char* moved, int* moved_list, DevCounters* ctr,
                           cudaStream_t st);
cudaError_t launch_mark(const TraceArgs& a, const CoherentArgs& c, int grid_cap, cudaStream_t st);
cudaError_t launch_carry(const TraceArgs& a, const CoherentArgs& c, cudaStream_t st);

}  // namespace dcem
