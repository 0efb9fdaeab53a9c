// noalloc.cu -- per-receiver reduction of caller-provided path records that
// allocates no device memory.
//
// Some callers cannot allocate device memory at the time they need the
// received power: a host framework that owns the whole device memory pool
// and forbids allocations outside it, or a real-time loop that must not call
// cudaMalloc after start-up (cudaMalloc can synchronise the device and stall
// the loop). dcem_reduce_paths_noalloc serves them: the caller passes device
// buffers for the inputs and outputs, and the only scratch the kernels need
// lives in one file-scope device array of fixed size. The CUDA runtime may
// load this file's kernels and reserve that array lazily, at the first use
// on a device; a set-up call (n_paths = 0, nrx = 0) made once per device at
// start-up does that work, so that later calls allocate nothing.
#include <mutex>

#include "dcem_internal.cuh"

namespace {

constexpr int kNaMaxRx = 4096;          // receivers per call
constexpr int kNaMaxPaths = 1 << 16;    // path records per call
constexpr int kNaMaxPerRx = 4096;       // paths of one receiver (sorted in shared memory)
constexpr int kNaThreads = 256;
constexpr int kNaMaxDevices = 64;

enum : unsigned { NA_ERR_RX_RANGE = 1u, NA_ERR_PER_RX = 2u };

struct NaScratch {
  unsigned count[kNaMaxRx];    // paths per receiver
  unsigned cursor[kNaMaxRx];   // scatter cursors
  unsigned offset[kNaMaxRx];   // exclusive prefix sum of count
  unsigned err;                // error bits of the current call
  unsigned pad[63];
  int order[kNaMaxPaths];      // path indices grouped by receiver
};

// The scratch of every call on a device (about 310 KB per device, held from
// the first use on that device until the process exits). Host code reaches it
// only through the address returned by cudaGetSymbolAddress.
static __device__ __align__(256) NaScratch g_na_scratch;

__global__ void k_na_clear(NaScratch* s, int nrx) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrx; r += gridDim.x * blockDim.x) {
    s->count[r] = 0u;
    s->cursor[r] = 0u;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) s->err = 0u;
}

__global__ void k_na_count(NaScratch* s, const dcem_path* __restrict__ p, int n, int nrx) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int r = p[i].rx;
    if (r < 0 || r >= nrx) {
      atomicOr(&s->err, NA_ERR_RX_RANGE);
      continue;
    }
    atomicAdd(&s->count[r], 1u);
  }
}

// exclusive prefix sum of count over nrx <= kNaMaxRx receivers, one CTA
__global__ void __launch_bounds__(1024) k_na_scan(NaScratch* s, int nrx) {
  __shared__ unsigned part[1024];
  int per = (nrx + 1023) / 1024;
  int b = threadIdx.x * per, e = min(b + per, nrx);
  unsigned acc = 0;
  for (int i = b; i < e; ++i) {
    if (s->count[i] > (unsigned)kNaMaxPerRx) atomicOr(&s->err, NA_ERR_PER_RX);
    acc += s->count[i];
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    unsigned v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
  for (int i = b; i < e; ++i) {
    s->offset[i] = run;
    run += s->count[i];
  }
}

__global__ void k_na_scatter(NaScratch* s, const dcem_path* __restrict__ p, int n, int nrx) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int r = p[i].rx;
    if (r < 0 || r >= nrx) continue;
    s->order[s->offset[r] + atomicAdd(&s->cursor[r], 1u)] = i;
  }
}

// One CTA per receiver: its paths sorted by key, records with equal keys (the
// same sequence from two transmitters) by record index, then the same
// fixed-order sums as the frame reduction (thread t takes sorted positions t,
// t+256, ..., then a fixed binary tree). The order, and so every bit of the
// sums, depends only on the records, not on the order in which the scatter's
// atomics placed them; for one transmitter's records (distinct keys) it is
// the frame's order, so the results match dcem_trace_frame's.
__global__ void __launch_bounds__(kNaThreads) k_na_reduce(NaScratch* s, const dcem_path* __restrict__ p, int nrx,
                                                          double tx_power, double* field, double* pc,
                                                          double* pi) {
  extern __shared__ unsigned long long skey[];  // kNaMaxPerRx keys, then as many ints
  int* sidx = reinterpret_cast<int*>(skey + kNaMaxPerRx);
  __shared__ double red[3][kNaThreads];
  int r = blockIdx.x, tid = threadIdx.x;
  if (r >= nrx) return;
  int cnt = (int)min(s->count[r], (unsigned)kNaMaxPerRx);
  unsigned off = s->offset[r];
  int np2 = 1;
  while (np2 < cnt) np2 <<= 1;
  for (int i = tid; i < np2; i += kNaThreads) {
    if (i < cnt) {
      int u = s->order[off + i];
      skey[i] = p[u].key;
      sidx[i] = u;
    } else {
      skey[i] = ~0ull;
      sidx[i] = -1;
    }
  }
  __syncthreads();
  for (int k = 2; k <= np2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < np2; i += kNaThreads) {
        int ixj = i ^ j;
        if (ixj > i) {
          unsigned long long x = skey[i], y = skey[ixj];
          int xi = sidx[i], yi = sidx[ixj];
          // (key, record index); padding (~0, -1) sorts last
          bool gt = x != y ? x > y : (unsigned)xi > (unsigned)yi;
          bool up = (i & k) == 0;
          if (gt == up) {
            skey[i] = y;
            skey[ixj] = x;
            int t = sidx[i];
            sidx[i] = sidx[ixj];
            sidx[ixj] = t;
          }
        }
      }
      __syncthreads();
    }
  }
  double sre = 0.0, sim = 0.0, sinc = 0.0;
  for (int i = tid; i < cnt; i += kNaThreads) {
    const dcem_path& q = p[sidx[i]];
    sre += q.amp_re;
    sim += q.amp_im;
    sinc += q.amp_re * q.amp_re + q.amp_im * q.amp_im;
  }
  red[0][tid] = sre;
  red[1][tid] = sim;
  red[2][tid] = sinc;
  __syncthreads();
  for (int h = kNaThreads / 2; h > 0; h >>= 1) {
    if (tid < h)
      for (int k = 0; k < 3; ++k) red[k][tid] += red[k][tid + h];
    __syncthreads();
  }
  if (tid == 0) {
    double fr = red[0][0], fi = red[1][0], pinc = red[2][0];
    if (field) {
      field[2 * (size_t)r] = fr;
      field[2 * (size_t)r + 1] = fi;
    }
    if (pc) pc[r] = 10.0 * log10(tx_power * (fr * fr + fi * fi)) + 30.0;
    if (pi) pi[r] = 10.0 * log10(tx_power * pinc) + 30.0;
  }
}

// Per-device address of g_na_scratch, looked up once per device.
std::mutex g_na_mutex;
NaScratch* g_na_addr[kNaMaxDevices] = {};
bool g_na_attr[kNaMaxDevices] = {};

int na_status(cudaError_t e) {
  if (e == cudaSuccess) return DCEM_OK;
  cudaGetLastError();
  return DCEM_ERR_CUDA;
}

}  // namespace

extern "C" int dcem_reduce_paths_noalloc(const dcem_path* paths, int32_t n_paths, int32_t nrx,
                                         double tx_power_w, double* field, double* p_coh_dbm,
                                         double* p_inc_dbm, void* stream) {
  if (n_paths < 0 || nrx < 0 || (n_paths > 0 && !paths)) return DCEM_ERR_ARG;
  if (!(tx_power_w > 0.0)) return DCEM_ERR_ARG;
  if (n_paths > kNaMaxPaths || nrx > kNaMaxRx) return DCEM_ERR_CAPACITY;
  if (nrx == 0 && n_paths > 0) return DCEM_ERR_ARG;  // no receiver can hold them
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_status(e);
  if (dev < 0 || dev >= kNaMaxDevices) return DCEM_ERR_CUDA;
  NaScratch* s = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
      // set-up on the first call on this device, with the device current
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_na_scratch);
      if (e != cudaSuccess) return na_status(e);
      g_na_addr[dev] = static_cast<NaScratch*>(ptr);
    }
    if (!g_na_attr[dev]) {
      size_t smem = (size_t)kNaMaxPerRx * (sizeof(unsigned long long) + sizeof(int));
      e = cudaFuncSetAttribute(k_na_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return na_status(e);
      // the other kernels too, so that a lazily loading runtime loads them
      // all now rather than at a later call
      cudaFuncAttributes fa;
      const void* fns[] = {(const void*)k_na_clear, (const void*)k_na_count, (const void*)k_na_scan,
                           (const void*)k_na_scatter};
      for (const void* fn : fns) {
        e = cudaFuncGetAttributes(&fa, fn);
        if (e != cudaSuccess) return na_status(e);
      }
      g_na_attr[dev] = true;
    }
    s = g_na_addr[dev];
  }
  if (nrx == 0) return DCEM_OK;  // the set-up call
  cudaStream_t st = (cudaStream_t)stream;
  int g = (nrx + 255) / 256;
  k_na_clear<<<g, 256, 0, st>>>(s, nrx);
  if (n_paths > 0) {
    int gp = (n_paths + 255) / 256;
    k_na_count<<<gp, 256, 0, st>>>(s, paths, n_paths, nrx);
    k_na_scan<<<1, 1024, 0, st>>>(s, nrx);
    k_na_scatter<<<gp, 256, 0, st>>>(s, paths, n_paths, nrx);
  }
  size_t smem = (size_t)kNaMaxPerRx * (sizeof(unsigned long long) + sizeof(int));
  k_na_reduce<<<nrx, kNaThreads, smem, st>>>(s, paths, nrx, tx_power_w, field, p_coh_dbm, p_inc_dbm);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_status(e);
  unsigned err = 0;
  e = cudaMemcpyAsync(&err, &s->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return na_status(e);
  if (err & NA_ERR_RX_RANGE) return DCEM_ERR_ARG;
  if (err & NA_ERR_PER_RX) return DCEM_ERR_CAPACITY;
  return DCEM_OK;
}
