// paths.cu -- duplicate-path removal, image-method validation, field, and
// the per-receiver reduction.
//
// Sec. III "Backward ray tracing":
//   step 2  a table of visited propagation paths per reflection depth: every
//           capture is keyed by (receiver, depth, triangle sequence); a
//           device hash table keeps one representative per distinct key
//           (the capture of the lowest ray index), and every other capture
//           is checked against it key by key (a 64-bit collision between
//           distinct keys is reported, never merged);
//   step 3  image receivers: the transmitter is mirrored in the plane of each
//           triangle of the sequence;
//   step 4  path validation: the back-trace from the receiver through the
//           images must cross each plane inside its triangle, and every
//           sub-segment must be unoccluded (FP32 any-hit over the LBVH);
//   step 6  per valid path: total length, delay, and the complex amplitude
//           of the ray field (Eq. 1) with the free-space spreading of Eq. 3
//           (exponent 2) and one Fresnel TE/TM reflection per bounce, with
//           vector polarisation (FP64).
// The per-receiver sums of amplitudes are formed in a fixed order (paths
// sorted by key), so the received power is reproducible bit for bit.
#include "paths.cuh"

namespace dcem {

// ---------------------------------------------------------------------------
// keys
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long path_key(const PathArgs& a, Cand c) {
  int rx = cand_rx(c), k = cand_seg(c);
  unsigned long long h = mix64(0x9e3779b97f4a7c15ull + (unsigned long long)(unsigned)rx);
  h = mix64(h + 0x100000001b3ull * (unsigned long long)(k + 1));
  for (int j = 0; j < k; ++j)
    h = mix64(h + ((unsigned long long)(unsigned)a.log_id[(size_t)j * a.R + c.ray] |
                   ((unsigned long long)(j + 1) << 40)));
  return h ? h : 1ull;
}

__device__ __forceinline__ bool same_key(const PathArgs& a, Cand x, Cand y) {
  if (cand_rx(x) != cand_rx(y) || cand_seg(x) != cand_seg(y)) return false;
  for (int j = 0; j < cand_seg(x); ++j)
    if (a.log_id[(size_t)j * a.R + x.ray] != a.log_id[(size_t)j * a.R + y.ray]) return false;
  return true;
}

__global__ void k_dedupe_insert(PathArgs a) {
  unsigned n = min(a.ctr->n_cand, a.cand_cap);
  unsigned mask = a.hcap - 1u;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    Cand c = a.cand[i];
    unsigned long long h = path_key(a, c);
    unsigned slot = (unsigned)(h & mask);
    bool ok = false;
    for (unsigned p = 0; p < a.hcap; ++p) {
      unsigned long long prev = atomicCAS(&a.hkey[slot], 0ull, h);
      if (prev == 0ull || prev == h) { ok = true; break; }
      slot = (slot + 1u) & mask;
    }
    if (!ok) {
      atomicOr(&a.ctr->err, ERR_HASH_FULL);
      a.cand_slot[i] = -1;
      continue;
    }
    a.cand_slot[i] = (int)slot;
    atomicMin(&a.hrep[slot], ((unsigned long long)(unsigned)c.ray << 32) | i);
  }
}

__global__ void k_dedupe_unique(PathArgs a) {
  unsigned n = min(a.ctr->n_cand, a.cand_cap);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int slot = a.cand_slot[i];
    if (slot < 0) continue;
    unsigned rep = (unsigned)(a.hrep[slot] & 0xffffffffull);
    if (rep == i) {
      unsigned u = atomicAdd(&a.ctr->n_unique, 1u);
      if (u < a.ucap) a.uniq[u] = (int)i;
      else atomicOr(&a.ctr->err, ERR_UNIQUE_OVERFLOW);
    } else if (!same_key(a, a.cand[i], a.cand[rep])) {
      atomicOr(&a.ctr->err, ERR_HASH_COLLISION);
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 geometry and complex arithmetic
// ---------------------------------------------------------------------------
struct d3 {
  double x, y, z;
};
__device__ __forceinline__ d3 mk3(double x, double y, double z) { return d3{x, y, z}; }
__device__ __forceinline__ d3 operator+(d3 a, d3 b) { return mk3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ d3 operator-(d3 a, d3 b) { return mk3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ d3 operator*(d3 a, double s) { return mk3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ double dd(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ d3 dx(d3 a, d3 b) {
  return mk3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double dn(d3 a) { return sqrt(dd(a, a)); }
__device__ __forceinline__ d3 du(d3 a) { return a * (1.0 / dn(a)); }

struct cx {
  double re, im;
};
__device__ __forceinline__ cx C(double r, double i = 0.0) { return cx{r, i}; }
__device__ __forceinline__ cx operator+(cx a, cx b) { return C(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ cx operator-(cx a, cx b) { return C(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ cx operator*(cx a, cx b) {
  return C(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
__device__ __forceinline__ cx operator*(cx a, double s) { return C(a.re * s, a.im * s); }
__device__ __forceinline__ cx cdiv(cx a, cx b) {
  // Smith's algorithm
  if (fabs(b.re) >= fabs(b.im)) {
    double r = b.im / b.re, den = b.re + b.im * r;
    return C((a.re + a.im * r) / den, (a.im - a.re * r) / den);
  }
  double r = b.re / b.im, den = b.re * r + b.im;
  return C((a.re * r + a.im) / den, (a.im * r - a.re) / den);
}
// principal square root
__device__ __forceinline__ cx csqrt_p(cx z) {
  double m = hypot(z.re, z.im);
  if (m == 0.0) return C(0.0, 0.0);
  double a = sqrt(0.5 * (m + fabs(z.re)));
  if (z.re >= 0.0) return C(a, z.im / (2.0 * a));
  return C(fabs(z.im) / (2.0 * a), copysign(a, z.im));
}

struct cv3 {
  cx x, y, z;
};
__device__ __forceinline__ cx cdot(cv3 e, d3 v) { return e.x * v.x + e.y * v.y + e.z * v.z; }

__device__ __forceinline__ void load_tri_d(const PathArgs& a, int id, d3& v0, d3& v1, d3& v2, int& mat) {
  int slot = a.slot_of_id[id];
  const float4* t = a.tris + 3 * (size_t)slot;
  float4 p = t[0], q = t[1], r = t[2];
  v0 = mk3(p.x, p.y, p.z);
  v1 = mk3(q.x, q.y, q.z);
  v2 = mk3(r.x, r.y, r.z);
  mat = __float_as_int(q.w);
}

// Polarisation of an isotropic antenna along d: u - (u.d) d, normalised.
__device__ __forceinline__ d3 pol_of(d3 u, d3 d, unsigned& flags) {
  d3 p = u - d * dd(u, d);
  double n = dn(p);
  if (n < 1e-9) {
    flags |= DCEM_PATH_POL_DEGENERATE;
    d3 ax = fabs(d.x) < 0.9 ? mk3(1, 0, 0) : mk3(0, 1, 0);
    p = ax - d * dd(ax, d);
    n = dn(p);
  }
  return p * (1.0 / n);
}

// ---------------------------------------------------------------------------
// validation + field, one thread per distinct candidate
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_validate(PathArgs a) {
  unsigned nu = min(a.ctr->n_unique, a.ucap);
  unsigned ovf = 0;
  for (unsigned u = blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += gridDim.x * blockDim.x) {
    int ci = a.uniq[u];
    Cand c = a.cand[ci];
    int slot = a.cand_slot[ci];
    PathRec rec;
    rec.key = a.hkey[slot];
    // this slot is no longer needed: leave the table empty for the next frame
    a.hkey[slot] = 0ull;
    a.hrep[slot] = ~0ull;
    int k = cand_seg(c), rxi = cand_rx(c);
    rec.rx = rxi;
    rec.depth = k;
    rec.ray = c.ray;
    rec.flags = 0;
    rec.valid = 0;
    rec.len = 0.0;
    rec.amp_re = rec.amp_im = 0.0;
    int ids[kMaxRefl];
    for (int j = 0; j < kMaxRefl; ++j) {
      ids[j] = j < k ? a.log_id[(size_t)j * a.R + c.ray] : -1;
      rec.tri[j] = ids[j];
      rec.pts[j][0] = rec.pts[j][1] = rec.pts[j][2] = 0.0f;
    }
    float4 rxv = a.rx[rxi];
    d3 X[kMaxRefl + 2], V0[kMaxRefl], Nn[kMaxRefl];
    int mats[kMaxRefl];
    d3 tx = mk3(a.tx.x, a.tx.y, a.tx.z), rx = mk3(rxv.x, rxv.y, rxv.z);
    // step 3: image sources I_1..I_k
    d3 img[kMaxRefl + 1];
    img[0] = tx;
    bool ok = true;
    for (int j = 0; j < k && ok; ++j) {
      d3 v0, v1, v2;
      load_tri_d(a, ids[j], v0, v1, v2, mats[j]);
      d3 n = dx(v1 - v0, v2 - v0);
      double nn = dd(n, n);
      if (!(nn > 0.0)) { ok = false; break; }
      V0[j] = v0;
      Nn[j] = n;
      img[j + 1] = img[j] - n * (2.0 * dd(img[j] - v0, n) / nn);
    }
    // step 4: back-trace from the receiver, reflection points in their triangles
    X[0] = tx;
    X[k + 1] = rx;
    for (int j = k; j >= 1 && ok; --j) {
      d3 dir = img[j] - X[j + 1];
      double den = dd(dir, Nn[j - 1]);
      if (den == 0.0) { ok = false; break; }
      double s = dd(V0[j - 1] - X[j + 1], Nn[j - 1]) / den;
      if (!(s > 0.0 && s < 1.0)) { ok = false; break; }
      X[j] = X[j + 1] + dir * s;
      d3 v0, v1, v2;
      int m;
      load_tri_d(a, ids[j - 1], v0, v1, v2, m);
      d3 n = Nn[j - 1];
      if (dd(dx(v1 - v0, X[j] - v0), n) < 0.0 || dd(dx(v2 - v1, X[j] - v1), n) < 0.0 ||
          dd(dx(v0 - v2, X[j] - v2), n) < 0.0)
        ok = false;
    }
    double L = 0.0;
    if (ok) {
      for (int j = 0; j <= k; ++j) L += dn(X[j + 1] - X[j]);
      if (!(L > 0.0)) ok = false;
    }
    // sub-segment occlusion in FP32 over (eps, 1 - eps)
    for (int j = 0; j <= k && ok; ++j) {
      d3 dv = X[j + 1] - X[j];
      float3 o = f3((float)X[j].x, (float)X[j].y, (float)X[j].z);
      float3 dvf = f3((float)dv.x, (float)dv.y, (float)dv.z);
      RayPre rp = ray_pre(o, dvf);
      int ex0 = j >= 1 ? ids[j - 1] : -1, ex1 = j < k ? ids[j] : -1;
      if (any_hit(a.bvh, rp, a.eps_occ, 1.0f - a.eps_occ, ex0, ex1, ovf)) ok = false;
    }
    if (ok) {
      // step 6: field with vector polarisation
      unsigned fl = 0;
      d3 upol = mk3(a.pol.x, a.pol.y, a.pol.z);
      d3 e0 = pol_of(upol, du(X[1] - X[0]), fl);
      cv3 E = {C(e0.x), C(e0.y), C(e0.z)};
      for (int j = 1; j <= k; ++j) {
        d3 din = du(X[j] - X[j - 1]), dout = du(X[j + 1] - X[j]);
        d3 nh = du(Nn[j - 1]);
        double ct = fabs(dd(din, nh));
        d3 sv = dx(din, nh);
        double sn = dn(sv);
        if (sn < 1e-12) {
          d3 ax = fabs(nh.x) < 0.9 ? mk3(1, 0, 0) : mk3(0, 1, 0);
          sv = du(dx(nh, ax));
        } else {
          sv = sv * (1.0 / sn);
        }
        d3 pin = dx(sv, din), pout = dx(sv, dout);
        const float4 mt = a.mats[mats[j - 1]];
        cx gte, gtm;
        if (mt.z != 0.0f) {
          gte = C(-1.0);
          gtm = C(1.0);
        } else {
          cx ec = C((double)mt.x, -(double)mt.y / (2.0 * M_PI * a.freq * 8.8541878128e-12));
          cx root = csqrt_p(ec - C(1.0 - ct * ct));
          gte = cdiv(C(ct) - root, C(ct) + root);
          gtm = cdiv(ec * ct - root, ec * ct + root);
        }
        cx es = cdot(E, sv), ep = cdot(E, pin);
        cx ts = gte * es, tp = gtm * ep;
        E.x = ts * sv.x + tp * pout.x;
        E.y = ts * sv.y + tp * pout.y;
        E.z = ts * sv.z + tp * pout.z;
      }
      d3 drx = du(X[k + 1] - X[k]);
      d3 prx = pol_of(upol, drx * -1.0, fl);
      double lam = 299792458.0 / a.freq;
      double kw = 2.0 * M_PI * a.freq / 299792458.0;
      double sn, cs;
      sincos(kw * L, &sn, &cs);
      cx amp = cdot(E, prx) * C(cs, -sn) * (lam / (4.0 * M_PI) / L);
      rec.valid = 1;
      rec.flags = fl;
      rec.len = L;
      rec.amp_re = amp.re;
      rec.amp_im = amp.im;
      for (int j = 0; j < k; ++j) {
        rec.pts[j][0] = (float)X[j + 1].x;
        rec.pts[j][1] = (float)X[j + 1].y;
        rec.pts[j][2] = (float)X[j + 1].z;
      }
      unsigned pos = atomicAdd(&a.bucket_cnt[rxi], 1u);
      if (pos < (unsigned)a.bucket_cap) a.bucket[(size_t)rxi * a.bucket_cap + pos] = (int)u;
      else atomicOr(&a.ctr->err, ERR_BUCKET_OVERFLOW);
      atomicAdd(&a.ctr->n_valid, 1u);
    }
    a.prec[u] = rec;
  }
  if (ovf) {
    atomicAdd(&a.ctr->stack_overflow, 1u);
    atomicOr(&a.ctr->err, ERR_STACK);
  }
}

// ---------------------------------------------------------------------------
// per receiver: sort paths by key, sum in that order, write them out
// ---------------------------------------------------------------------------
constexpr int kReduceThreads = 256;

__global__ void __launch_bounds__(kReduceThreads) k_reduce(PathArgs a) {
  extern __shared__ unsigned long long skey[];   // bucket_cap keys, then bucket_cap ints
  int* sidx = reinterpret_cast<int*>(skey + a.bucket_cap);
  __shared__ double red[4][kReduceThreads];
  __shared__ unsigned soff;
  int r = blockIdx.x, tid = threadIdx.x;
  int cnt = (int)min(a.bucket_cnt[r], (unsigned)a.bucket_cap);
  // output offset: valid paths of all lower receivers
  unsigned part = 0;
  for (int q = tid; q < r; q += kReduceThreads) part += min(a.bucket_cnt[q], (unsigned)a.bucket_cap);
  for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
  if (tid == 0) soff = 0;
  __syncthreads();
  if ((tid & 31) == 0) atomicAdd(&soff, part);
  int np2 = 1;
  while (np2 < cnt) np2 <<= 1;
  for (int i = tid; i < np2; i += kReduceThreads) {
    if (i < cnt) {
      int u = a.bucket[(size_t)r * a.bucket_cap + i];
      skey[i] = a.prec[u].key;
      sidx[i] = u;
    } else {
      skey[i] = ~0ull;
      sidx[i] = -1;
    }
  }
  __syncthreads();
  for (int k = 2; k <= np2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < np2; i += kReduceThreads) {
        int ixj = i ^ j;
        if (ixj > i) {
          unsigned long long x = skey[i], y = skey[ixj];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            skey[i] = y; skey[ixj] = x;
            int t = sidx[i]; sidx[i] = sidx[ixj]; sidx[ixj] = t;
          }
        }
      }
      __syncthreads();
    }
  }
  // fixed-order sums: thread t takes sorted positions t, t+256, ... in order,
  // then a fixed binary tree over the 256 partial sums
  double sre = 0.0, sim = 0.0, sinc = 0.0;
  unsigned off = soff;
  for (int i = tid; i < cnt; i += kReduceThreads) {
    const PathRec& p = a.prec[sidx[i]];
    sre += p.amp_re;
    sim += p.amp_im;
    sinc += p.amp_re * p.amp_re + p.amp_im * p.amp_im;
    unsigned o = off + (unsigned)i;
    if (o < a.pout_cap) {
      dcem_path q;
      q.rx = p.rx;
      q.depth = p.depth;
      for (int j = 0; j < kMaxRefl; ++j) {
        q.tri[j] = p.tri[j];
        q.pts[j][0] = p.pts[j][0];
        q.pts[j][1] = p.pts[j][1];
        q.pts[j][2] = p.pts[j][2];
      }
      q.flags = p.flags;
      q.ray = p.ray;
      q.key = p.key;
      q.len_m = p.len;
      q.delay_s = p.len / 299792458.0;
      q.amp_re = p.amp_re;
      q.amp_im = p.amp_im;
      a.pout[o] = q;
    }
  }
  red[0][tid] = sre;
  red[1][tid] = sim;
  red[2][tid] = sinc;
  __syncthreads();
  for (int s = kReduceThreads / 2; s > 0; s >>= 1) {
    if (tid < s)
      for (int q = 0; q < 3; ++q) red[q][tid] += red[q][tid + s];
    __syncthreads();
  }
  if (tid == 0) {
    double fr = red[0][0], fi = red[1][0], pinc = red[2][0];
    double* o = a.rxout + 4 * (size_t)r;
    o[0] = fr;
    o[1] = fi;
    o[2] = 10.0 * log10(a.tx_power * (fr * fr + fi * fi)) + 30.0;
    o[3] = 10.0 * log10(a.tx_power * pinc) + 30.0;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_dedupe(const PathArgs& a, int grid, cudaStream_t st) {
  k_dedupe_insert<<<grid, 256, 0, st>>>(a);
  k_dedupe_unique<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_validate(const PathArgs& a, int grid, cudaStream_t st) {
  k_validate<<<grid, 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const PathArgs& a, int nrx, cudaStream_t st) {
  if (nrx <= 0) return cudaSuccess;
  size_t smem = (size_t)a.bucket_cap * (sizeof(unsigned long long) + sizeof(int));
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    attr = true;
  }
  k_reduce<<<nrx, kReduceThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace dcem
