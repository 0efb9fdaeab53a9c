// paths.cuh -- arguments and launchers of dedupe, validation and reduction.
#pragma once

#include "dcem_internal.cuh"

namespace dcem {

struct PathArgs {
  int R;                          // rays (log stride)
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
  int* bucket;                    // nrx x bucket_cap distinct-key indices of valid paths
  unsigned* bucket_cnt;           // nrx
  int bucket_cap;                 // power of two
  dcem_path* pout;                // ordered output (rx, key)
  unsigned pout_cap;
  double* rxout;                  // nrx x 4: field re, im, P_coh dBm, P_inc dBm
  const float4* tris;             // leaf-ordered triangles
  const int* slot_of_id;
  const float4* mats;             // eps_r, sigma, pec
  Bvh bvh;
  const float4* rx;
  float3 tx;
  float3 pol;
  float eps_occ;
  double freq, tx_power;
  DevCounters* ctr;
};

cudaError_t launch_dedupe(const PathArgs& a, int grid, cudaStream_t st);
cudaError_t launch_validate(const PathArgs& a, int grid, cudaStream_t st);
cudaError_t launch_reduce(const PathArgs& a, int nrx, cudaStream_t st);

}  // namespace dcem
