// grad.cu -- derivatives of the per-receiver field over a fixed path
// topology, with respect to each material's (eps_r, sigma) and each rigid
// object's (x, y) translation.
//
// The amplitude of a path is Sec. III steps 3, 4 and 6 again: image sources
// of the transmitter in the planes of the path's triangles, back-trace from
// the receiver to the reflection points, Fresnel reflection (TE/TM) with
// vector polarisation, and the amplitude of Eq. 1 with the Friis spreading of
// Eq. 3. Here it is evaluated in FP64 forward-mode dual numbers (value and
// derivative along one parameter): translating an object moves the vertices
// of its triangles, a material parameter enters through the complex
// permittivity. One work item is one (path, parameter) pair, where the
// parameter is that of one bounce's material or object; the first bounce that
// uses a material (object) seeds every bounce that shares it, later ones
// contribute no item. The per-receiver sums run in path order, one warp per
// receiver, so results are the same in every run.
#include "grad.cuh"

namespace dcem {
namespace {

constexpr double kC0 = 299792458.0;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kPi = 3.141592653589793;

struct Dd {
  double v, d;
};
__device__ __forceinline__ Dd cst(double v) { return Dd{v, 0.0}; }
__device__ __forceinline__ Dd operator+(Dd a, Dd b) { return Dd{a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dd operator-(Dd a, Dd b) { return Dd{a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dd operator-(Dd a) { return Dd{-a.v, -a.d}; }
__device__ __forceinline__ Dd operator*(Dd a, Dd b) { return Dd{a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dd operator*(double s, Dd a) { return Dd{s * a.v, s * a.d}; }
__device__ __forceinline__ Dd operator/(Dd a, Dd b) {
  double q = a.v / b.v;
  return Dd{q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ Dd dsqrt(Dd a) {
  double r = sqrt(a.v);
  return Dd{r, r > 0.0 ? a.d / (2.0 * r) : 0.0};
}
__device__ __forceinline__ Dd dabs(Dd a) { return a.v < 0.0 ? -a : a; }

struct V3 {
  Dd x, y, z;
};
__device__ __forceinline__ V3 vc(double x, double y, double z) { return V3{cst(x), cst(y), cst(z)}; }
__device__ __forceinline__ V3 operator+(const V3& a, const V3& b) { return V3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(const V3& a, const V3& b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator-(const V3& a) { return V3{-a.x, -a.y, -a.z}; }
__device__ __forceinline__ V3 scl(Dd s, const V3& a) { return V3{s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ Dd vdot(const V3& a, const V3& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 vcross(const V3& a, const V3& b) {
  return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ Dd vnorm(const V3& a) { return dsqrt(vdot(a, a)); }
__device__ __forceinline__ V3 vunit(const V3& a) {
  Dd n = vnorm(a);
  return V3{a.x / n, a.y / n, a.z / n};
}

struct Cd {
  Dd re, im;
};
__device__ __forceinline__ Cd cre(Dd r) { return Cd{r, cst(0.0)}; }
__device__ __forceinline__ Cd operator+(const Cd& a, const Cd& b) { return Cd{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ Cd operator-(const Cd& a, const Cd& b) { return Cd{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ Cd operator*(const Cd& a, const Cd& b) {
  return Cd{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ Cd operator*(Dd s, const Cd& a) { return Cd{s * a.re, s * a.im}; }
__device__ __forceinline__ Cd operator/(const Cd& a, const Cd& b) {
  Dd den = b.re * b.re + b.im * b.im;
  return Cd{(a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den};
}
// principal square root; derivative dz / (2 w)
__device__ __forceinline__ Cd csqrt_d(const Cd& z) {
  double x = z.re.v, y = z.im.v;
  double r = hypot(x, y), wr, wi;
  if (x >= 0.0) {
    double t = sqrt(0.5 * (r + x));
    wr = t;
    wi = t > 0.0 ? y / (2.0 * t) : 0.0;
  } else {
    double t = sqrt(0.5 * (r - x));
    wr = fabs(y) / (2.0 * t);
    wi = copysign(t, y);
  }
  double m = 2.0 * (wr * wr + wi * wi);
  double dr = m > 0.0 ? (z.re.d * wr + z.im.d * wi) / m : 0.0;
  double di = m > 0.0 ? (z.im.d * wr - z.re.d * wi) / m : 0.0;
  return Cd{Dd{wr, dr}, Dd{wi, di}};
}

struct C3 {
  Cd x, y, z;
};
__device__ __forceinline__ Cd cdotv(const C3& e, const V3& v) {
  return v.x * e.x + v.y * e.y + v.z * e.z;
}

// unit vector of u - (u.d) d; u parallel to d falls back to a fixed axis
__device__ __forceinline__ V3 pol_dir(const V3& u, const V3& d) {
  V3 p = u - scl(vdot(u, d), d);
  if (vnorm(p).v < 1e-9) {
    V3 a = fabs(d.x.v) < 0.9 ? vc(1, 0, 0) : vc(0, 1, 0);
    p = a - scl(vdot(a, d), d);
  }
  return vunit(p);
}

// Gamma_TE, Gamma_TM of a half-space with eps_c = eps_r - j sigma / (w eps0)
__device__ __forceinline__ void fresnel_d(Dd eps_r, Dd sigma, bool pec, double freq, Dd ct, Cd& te, Cd& tm) {
  if (pec) {
    te = cre(cst(-1.0));
    tm = cre(cst(1.0));
    return;
  }
  Cd ec{eps_r, (-1.0 / (2.0 * kPi * freq * kEps0)) * sigma};
  Dd sin2 = cst(1.0) - ct * ct;
  Cd root = csqrt_d(ec - cre(sin2));
  Cd c = cre(ct);
  te = (c - root) / (c + root);
  Cd ecc = ec * c;
  tm = (ecc - root) / (ecc + root);
}

__device__ __forceinline__ V3 vertex(const float4& f, int seed_axis) {
  V3 v = vc(f.x, f.y, f.z);
  if (seed_axis == 0) v.x.d = 1.0;
  if (seed_axis == 1) v.y.d = 1.0;
  return v;
}

// Amplitude of path P and its derivative along one parameter: kind 0/1 =
// eps_r / sigma of material `sid`, 2/3 = x / y translation of object `sid`,
// -1 = value only. False if the triangle sequence has no reflection geometry.
__device__ bool path_amp(const GradArgs& g, const dcem_path& P, int kind, int sid, Cd& amp) {
  const int k = P.depth;
  V3 tx = vc(g.tx[0], g.tx[1], g.tx[2]);
  float4 rv = g.rx[P.rx];
  V3 rx = vc(rv.x, rv.y, rv.z);
  V3 img[kMaxRefl + 1], X[kMaxRefl + 2], V0[kMaxRefl], Nn[kMaxRefl];
  Dd er[kMaxRefl], sg[kMaxRefl];
  bool pec[kMaxRefl];
  img[0] = tx;
  for (int j = 0; j < k; ++j) {
    int id = P.tri[j];
    const float4* t = g.tris + 3 * (size_t)g.slot_of_id[id];
    int ax = (kind >= 2 && g.tri_obj[id] == sid) ? kind - 2 : -1;
    V3 v0 = vertex(t[0], ax), v1 = vertex(t[1], ax), v2 = vertex(t[2], ax);
    V3 n = vcross(v1 - v0, v2 - v0);
    Dd nn = vdot(n, n);
    if (!(nn.v > 0.0)) return false;
    Dd h = vdot(img[j] - v0, n) / nn;
    img[j + 1] = img[j] - scl(2.0 * h, n);
    V0[j] = v0;
    Nn[j] = n;
    int m = g.tri_mat[id];
    float4 mt = g.mats[m];
    er[j] = cst(mt.x);
    sg[j] = cst(mt.y);
    pec[j] = mt.z != 0.0f;
    if (kind == 0 && m == sid) er[j].d = 1.0;
    if (kind == 1 && m == sid) sg[j].d = 1.0;
  }
  X[0] = tx;
  X[k + 1] = rx;
  for (int j = k; j >= 1; --j) {
    V3 dir = img[j] - X[j + 1];
    Dd den = vdot(dir, Nn[j - 1]);
    if (den.v == 0.0) return false;
    Dd s = vdot(V0[j - 1] - X[j + 1], Nn[j - 1]) / den;
    X[j] = X[j + 1] + scl(s, dir);
  }
  Dd L = cst(0.0);
  for (int j = 0; j <= k; ++j) L = L + vnorm(X[j + 1] - X[j]);
  if (!(L.v > 0.0)) return false;
  // field with vector polarisation
  V3 u = vc(g.pol[0], g.pol[1], g.pol[2]);
  V3 e0 = pol_dir(u, vunit(X[1] - X[0]));
  C3 E{cre(e0.x), cre(e0.y), cre(e0.z)};
  for (int j = 1; j <= k; ++j) {
    V3 din = vunit(X[j] - X[j - 1]), dout = vunit(X[j + 1] - X[j]);
    V3 nh = vunit(Nn[j - 1]);
    Dd ct = dabs(vdot(din, nh));
    V3 sv = vcross(din, nh);
    Dd sn = vnorm(sv);
    if (sn.v < 1e-12) {  // normal incidence: a fixed unit vector perpendicular to n
      V3 a = fabs(nh.x.v) < 0.9 ? vc(1, 0, 0) : vc(0, 1, 0);
      sv = vunit(vcross(nh, a));
    } else {
      sv = V3{sv.x / sn, sv.y / sn, sv.z / sn};
    }
    V3 pin = vcross(sv, din), pout = vcross(sv, dout);
    Cd gte, gtm;
    fresnel_d(er[j - 1], sg[j - 1], pec[j - 1], g.freq, ct, gte, gtm);
    Cd es = gte * cdotv(E, sv), ep = gtm * cdotv(E, pin);
    E = C3{sv.x * es + pout.x * ep, sv.y * es + pout.y * ep, sv.z * es + pout.z * ep};
  }
  V3 prx = pol_dir(u, -vunit(X[k + 1] - X[k]));
  double lam = kC0 / g.freq, kw = 2.0 * kPi * g.freq / kC0;
  double sp, cp;
  sincos(kw * L.v, &sp, &cp);
  Cd ph{Dd{cp, -kw * L.d * sp}, Dd{-sp, -kw * L.d * cp}};  // e^{-j k L}
  Cd a = cdotv(E, prx) * ph;
  amp = cst(lam / (4.0 * kPi)) * (a / cre(L));
  return true;
}

__global__ void k_grad_items(GradArgs g) {
  long total = (long)g.n_paths * g.W;
  for (long it = blockIdx.x * (long)blockDim.x + threadIdx.x; it < total; it += (long)gridDim.x * blockDim.x) {
    int p = (int)(it / g.W), slot = (int)(it - (long)p * g.W);
    const dcem_path& P = g.paths[p];
    g.param[it] = -1;
    bool good = P.depth >= 0 && P.depth <= g.max_refl && P.rx >= 0 && P.rx < g.nrx;
    for (int j = 0; good && j < P.depth; ++j) good = P.tri[j] >= 0 && P.tri[j] < g.ntri;
    if (!good) {
      if (slot == 0) atomicOr(g.err, 2u);
      continue;
    }
    Cd amp;
    if (slot == 0) {
      if (p > 0 && g.paths[p - 1].rx > P.rx) atomicOr(g.err, 1u);
      if (!path_amp(g, P, -1, -1, amp)) {
        atomicOr(g.err, 4u);
        continue;
      }
      g.items[it] = make_double2(amp.re.v, amp.im.v);
      g.param[it] = -2;
      continue;
    }
    int j = (slot - 1) >> 2, w = (slot - 1) & 3;
    if (j >= P.depth) continue;
    int id = P.tri[j], sid, theta;
    if (w < 2) {
      sid = g.tri_mat[id];
      if (g.mats[sid].z != 0.0f) continue;  // perfect conductor: no material dependence
      bool first = true;
      for (int q = 0; q < j; ++q) first = first && g.tri_mat[P.tri[q]] != sid;
      if (!first) continue;
      theta = 2 * sid + w;
    } else {
      sid = g.tri_obj[id];
      if (sid < 0) continue;
      bool first = true;
      for (int q = 0; q < j; ++q) first = first && g.tri_obj[P.tri[q]] != sid;
      if (!first) continue;
      theta = 2 * g.nmat + 2 * sid + (w - 2);
    }
    if (!path_amp(g, P, w, sid, amp)) continue;  // reported by the value item
    g.items[it] = make_double2(amp.re.d, amp.im.d);
    g.param[it] = theta;
  }
}

// One warp per receiver: its paths are contiguous (grouped by rx).
__global__ void k_grad_reduce(GradArgs g, int nparam) {
  int r = (int)((blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (r >= g.nrx) return;
  int lo = 0, hi = 0;
  if (lane == 0) {
    int a = 0, b = g.n_paths;  // first path with rx >= r
    while (a < b) {
      int m = (a + b) >> 1;
      if (g.paths[m].rx < r) a = m + 1; else b = m;
    }
    lo = a;
    b = g.n_paths;  // first path with rx > r
    while (a < b) {
      int m = (a + b) >> 1;
      if (g.paths[m].rx <= r) a = m + 1; else b = m;
    }
    hi = a;
  }
  lo = __shfl_sync(0xffffffffu, lo, 0);
  hi = __shfl_sync(0xffffffffu, hi, 0);
  double* df = g.dfield + 2 * (size_t)r * nparam;
  for (int t = lane; t < 2 * nparam; t += 32) df[t] = 0.0;
  __syncwarp();
  double er = 0.0, ei = 0.0;
  if (lane == 0) {
    for (long it = (long)lo * g.W; it < (long)hi * g.W; ++it) {
      int pm = g.param[it];
      double2 v = g.items[it];
      if (pm == -2) {
        er += v.x;
        ei += v.y;
      } else if (pm >= 0) {
        df[2 * pm] += v.x;
        df[2 * pm + 1] += v.y;
      }
    }
    if (g.field) {
      g.field[2 * (size_t)r] = er;
      g.field[2 * (size_t)r + 1] = ei;
    }
  }
  __syncwarp();
  er = __shfl_sync(0xffffffffu, er, 0);
  ei = __shfl_sync(0xffffffffu, ei, 0);
  if (g.dpcoh) {
    // P = P_t |E|^2: dP = 2 P_t Re(conj(E) dE), d(dBm) = 10 / ln 10 * dP / P
    double p = er * er + ei * ei;
    for (int t = lane; t < nparam; t += 32) {
      double dp = 2.0 * (er * df[2 * t] + ei * df[2 * t + 1]);
      g.dpcoh[(size_t)r * nparam + t] = p > 0.0 ? 4.342944819032518 * dp / p : 0.0;
    }
  }
}

__global__ void k_pack_rx(const float* __restrict__ rx3, int n, float4* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = make_float4(rx3[3 * i], rx3[3 * i + 1], rx3[3 * i + 2], 0.0f);
}

}  // namespace

cudaError_t launch_pack_rx(const float* rx3, int n, float4* out, cudaStream_t st) {
  if (n > 0) k_pack_rx<<<(n + 255) / 256, 256, 0, st>>>(rx3, n, out);
  return cudaGetLastError();
}

cudaError_t launch_gradients(const GradArgs& a, cudaStream_t st) {
  long total = (long)a.n_paths * a.W;
  if (total > 0) {
    long b = (total + 127) / 128;
    k_grad_items<<<(int)(b < 65535 ? b : 65535), 128, 0, st>>>(a);
  }
  if (a.nrx > 0) {
    int nparam = grad_nparam(a.nmat, a.nobj);
    k_grad_reduce<<<(a.nrx + 3) / 4, 128, 0, st>>>(a, nparam);
  }
  return cudaGetLastError();
}

}  // namespace dcem
