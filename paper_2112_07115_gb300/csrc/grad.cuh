// grad.cuh -- derivatives of the received field over a fixed path topology.
#pragma once

#include "dcem_internal.cuh"

namespace dcem {

struct GradArgs {
  const dcem_path* paths;   // n_paths, grouped by receiver in non-decreasing rx order
  int n_paths;
  int W;                    // items per path: 1 (value) + 4 * max_refl
  int max_refl;
  const float4* tris;       // leaf-ordered world triangles (v, .w = id / material)
  const int* slot_of_id;
  const int* tri_mat;       // triangle id -> material
  const int* tri_obj;       // triangle id -> rigid object, -1 static
  int ntri;
  const float4* mats;       // eps_r, sigma, pec
  int nmat, nobj;
  const float4* rx;         // nrx receivers
  int nrx;
  double tx[3];
  double pol[3];
  double freq, tx_power;
  double2* items;           // n_paths * W: value or d a / d theta of one item
  int* param;               // n_paths * W: theta index, -2 value item, -1 no item
  unsigned* err;            // 1: paths not grouped by receiver, 2: bad depth or triangle id
  double* field;            // nrx x 2
  double* dfield;           // nrx x nparam x 2
  double* dpcoh;            // nrx x nparam, d P_coh[dBm] / d theta
  // adjoint kernel only: the parameters to evaluate at (null: the scene's),
  // eps_r, sigma per material, then x, y translation per object, and the
  // objects' current transforms (the translations theta is measured against)
  const double* theta;
  const float* xf;          // nobj x 12, row-major [R | t]
  double* pcoh;             // nrx P_coh [dBm] at theta, or null
  const double* pcoh_bar;   // nrx upstream d loss / d P_coh[dBm], or null
  double* theta_bar;        // nparam: sum over receivers of pcoh_bar * d P_coh / d theta
};

inline int grad_nparam(int nmat, int nobj) { return 2 * nmat + 2 * nobj; }

cudaError_t launch_gradients(const GradArgs& a, cudaStream_t st);
// The same outputs from the reverse-mode (adjoint) kernel, one thread per path.
cudaError_t launch_adjoint(const GradArgs& a, cudaStream_t st);
// nrx receivers as 3 floats each (device) -> float4
cudaError_t launch_pack_rx(const float* rx3, int n, float4* out, cudaStream_t st);

}  // namespace dcem
