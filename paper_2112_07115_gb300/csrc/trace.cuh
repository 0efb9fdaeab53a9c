// trace.cuh -- arguments and launchers of the shooting and coherence kernels.
#pragma once

#include "dcem_internal.cuh"

namespace dcem {

struct TraceArgs {
  Bvh bvh;
  const float4* rays;      // R unit directions (xyz), .w = the ray's set (int bits)
  const float4* txs;       // per ray set: transmitter position (xyz) and the
                           // effective capture spacing alpha_t / sqrt(3) (w)
  int nsets;
  int R, N;                // rays, reflections
  int LS;                  // segment-log stride: R, plus the child slots with transmission
  // transmission (Sec. III "Reflected and transmitted rays"): a hit on a
  // material with mats[m].w >= 0 also spawns a child ray straight through
  // it, up to max_trans per path; child slots R .. R + child_cap - 1 carry
  // inst = reflections | transmissions << 4 | ray set << 8. Pass p traces
  // the children pass p - 1 spawned.
  const float4* mats;
  int max_trans, pass, child_cap;
  int* inst;
  int* inst_root;          // per child slot: its primary ray's slot
  float tmin, escape;
  const float4* rx;        // nrx receivers (xyz); a capture's link is set * nrx + r
  int nrx;
  SmallBvh rxt;            // per-frame tree over the receivers
  const uint4* qnodes;     // 4-wide compact node copy (4 uint4 per node) and its frame
  const float* qframe;
  int n_nodes;             // internal nodes of both trees (2-wide)
  const int* q4_count;     // 4-wide nodes (device), at most q4_bound
  const int* q4_roots;     // roots of both trees in the 4-wide copy (device)
  int q4_bound;
  int use_q;               // closest-hit kernel: 0 binary nodes (k_trace), 1 the 4-wide compact
                           // copy from shared memory (k_trace_q), 2 from global memory (k_trace_qg)
  int stack_cap;           // shared-memory stack entries per thread
  int block;               // threads per CTA of kernels 0 and 2 (kernel 1: kTraceQThreads)
  float4* log_o;           // (N+1) x R: origin, unfolded length D
  float4* log_d;           // (N+1) x R: direction, hit t (+inf escaped)
  int* log_id;             // (N+1) x R: hit triangle id or -1
  unsigned* capitems;      // (N+1) x R capacity: segments to capture-test, ray << 4 | segment,
                           // bit 31 set: reused segment, test only the moved receivers
  const unsigned char* rx_moved;  // coherent frame: nrx flags (null in a full frame)
  int* nseg;               // R
  const int* queue;        // retrace queue (null: all rays from segment 0)
  int* queue_w;            // retrace queue written by the marking kernel
  int* restart;            // R + child slots: first segment to (re)trace
  const unsigned* nq_dev;  // queue length (device)
  Cand* cand;
  unsigned cand_cap;
  DevCounters* ctr;
};

struct CoherentArgs {
  const int* moved_list;           // moved receivers
  const unsigned char* rx_moved;   // nrx flags
  int* restart;                    // R
  DevCounters* ctr;
  const Cand* prev_cand;
  const unsigned* prev_ncand;
  unsigned prev_cap;
  SmallBvh mvt;                    // per-frame tree over the moved boxes
  int mv_cap;                      // boxes the tree can hold
};

// Persistent traversal of every ray (or of the retrace queue) followed by
// the capture pass over the traced segments. `sms`: multiprocessor count.
// Closest-hit kernel with the compact node copy in shared memory: threads
// per CTA (one CTA per SM) and the shared memory it may use.
constexpr int kTraceQThreads = 768;
constexpr long kTraceQSmem = 220L * 1024;
// Shared-memory stack entries per thread for a compact copy of n_nodes
// nodes, or 0 if copy and stacks do not fit (then nodes come from global).
int trace_q_stack_cap(int n_nodes);
// Closest-hit configurations of kernels 0 and 2: threads per CTA and shared
// stack entries per thread.
constexpr int kTraceBlocks[] = {64, 128, 256};
constexpr int kTraceStackMin = 8, kTraceStackMax = 32;
cudaError_t launch_trace(const TraceArgs& a, int sms, cudaStream_t st);
cudaError_t launch_capture(const TraceArgs& a, int sms, cudaStream_t st);
// The closest-hit pass of n scenes in one launch (d_tab: their arguments on the
// device; chunk_ctr zeroed before). No transmission.
cudaError_t launch_trace_batch(const TraceArgs* d_tab, int n, unsigned* chunk_ctr, int sms, cudaStream_t st);
cudaError_t launch_mark(const TraceArgs& a, const CoherentArgs& c, int sms, cudaStream_t st);
cudaError_t launch_carry(const TraceArgs& a, const CoherentArgs& c, cudaStream_t st);

}  // namespace dcem
