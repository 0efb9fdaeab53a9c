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
  if (g.pcoh && lane == 0) {
    double p = er * er + ei * ei;
    g.pcoh[r] = p > 0.0 ? 10.0 * log10(g.tx_power * p) + 30.0 : -INFINITY;
  }
  if (g.dpcoh) {
    // P = P_t |E|^2: dP = 2 P_t Re(conj(E) dE), d(dBm) = 10 / ln 10 * dP / P
    double p = er * er + ei * ei;
    for (int t = lane; t < nparam; t += 32) {
      double dp = 2.0 * (er * df[2 * t] + ei * df[2 * t + 1]);
      g.dpcoh[(size_t)r * nparam + t] = p > 0.0 ? 4.342944819032518 * dp / p : 0.0;
    }
  }
}

// ---------------------------------------------------------------------------
// reverse mode: one thread per path
// ---------------------------------------------------------------------------
// The forward sweep evaluates the path's geometry in FP64 (image sources,
// back-trace) and keeps only its vertices X_0 .. X_{k+1} (the checkpoint);
// the field state of a bounce (directions, polarisation basis, Fresnel
// coefficients, the field before it) is recomputed from the vertices when the
// backward sweep needs it. The backward sweep carries d a / d v for every
// intermediate v (complex: the field is holomorphic in its complex
// intermediates) from a back to the vertices and to each bounce's complex
// permittivity. A material's eps_r and sigma take d a / d eps_c directly; an
// object's translation moves the planes of its triangles, whose effect on the
// vertices is a tangent of the (cheap, real) image geometry, contracted with
// d a / d X.
struct R3 {
  double x, y, z;
};
__device__ __forceinline__ R3 r3(double x, double y, double z) { return R3{x, y, z}; }
__device__ __forceinline__ R3 operator+(R3 a, R3 b) { return r3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ R3 operator-(R3 a, R3 b) { return r3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ R3 operator*(R3 a, double s) { return r3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ double rdot(R3 a, R3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ R3 rcross(R3 a, R3 b) {
  return r3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double rnorm(R3 a) { return sqrt(rdot(a, a)); }
__device__ __forceinline__ R3 runit(R3 a) { return a * (1.0 / rnorm(a)); }

struct Zc {
  double re, im;
};
__device__ __forceinline__ Zc zc(double r, double i = 0.0) { return Zc{r, i}; }
__device__ __forceinline__ Zc operator+(Zc a, Zc b) { return zc(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ Zc operator-(Zc a, Zc b) { return zc(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ Zc operator*(Zc a, Zc b) { return zc(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
__device__ __forceinline__ Zc operator*(Zc a, double s) { return zc(a.re * s, a.im * s); }
__device__ __forceinline__ Zc operator/(Zc a, Zc b) {
  double d = b.re * b.re + b.im * b.im;
  return zc((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}
__device__ __forceinline__ Zc zsqrt_p(Zc z) {  // principal branch
  double r = hypot(z.re, z.im);
  if (z.re >= 0.0) {
    double t = sqrt(0.5 * (r + z.re));
    return zc(t, t > 0.0 ? z.im / (2.0 * t) : 0.0);
  }
  double t = sqrt(0.5 * (r - z.re));
  return zc(fabs(z.im) / (2.0 * t), copysign(t, z.im));
}

struct Z3 {
  Zc x, y, z;
};
__device__ __forceinline__ Z3 z3of(R3 v, Zc s) { return Z3{s * v.x, s * v.y, s * v.z}; }  // s v
__device__ __forceinline__ Z3 operator+(const Z3& a, const Z3& b) { return Z3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ Z3 operator-(const Z3& a, const Z3& b) { return Z3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ Z3 operator*(const Z3& a, Zc s) { return Z3{a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ Z3 operator*(const Z3& a, double s) { return Z3{a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ Zc zdot(const Z3& a, R3 v) { return a.x * v.x + a.y * v.y + a.z * v.z; }
__device__ __forceinline__ Z3 zcross(R3 a, const Z3& b) {  // real x complex
  return Z3{b.z * a.y - b.y * a.z, b.x * a.z - b.z * a.x, b.y * a.x - b.x * a.y};
}
__device__ __forceinline__ Z3 zcross(const Z3& a, R3 b) {  // complex x real
  return Z3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Polarisation of an isotropic antenna along unit d: normalize(u - (u.d) d),
// a fixed axis in place of u when u is along d.
struct Pol {
  R3 n, ueff;
  double qn;
};
__device__ __forceinline__ Pol pol_fwd(R3 u, R3 d) {
  Pol p;
  p.ueff = u;
  R3 q = u - d * rdot(u, d);
  p.qn = rnorm(q);
  if (p.qn < 1e-9) {
    p.ueff = fabs(d.x) < 0.9 ? r3(1, 0, 0) : r3(0, 1, 0);
    q = p.ueff - d * rdot(p.ueff, d);
    p.qn = rnorm(q);
  }
  p.n = q * (1.0 / p.qn);
  return p;
}
// d a / d d from d a / d n
__device__ __forceinline__ Z3 pol_bwd(const Pol& p, R3 d, const Z3& nbar) {
  Z3 g = (nbar - z3of(p.n, zdot(nbar, p.n))) * (1.0 / p.qn);
  Zc gd = zdot(g, d);
  return z3of(p.ueff, gd * -1.0) - g * rdot(p.ueff, d);
}

// One bounce's field quantities, from its incoming and outgoing directions.
struct Bounce {
  R3 nh, sv, pin, pout;
  double c, sgn, vn;  // |d_in . n|, its sign, |d_in x n| (fixed s below 1e-12)
  bool fixed_s, pec;
  Zc te, tm, ec, root;
};
__device__ __forceinline__ Bounce bounce_of(R3 din, R3 dout, R3 nrm, double er, double sg, bool pec, double wfac) {
  Bounce b;
  b.nh = runit(nrm);
  double dn = rdot(din, b.nh);
  b.c = fabs(dn);
  b.sgn = dn < 0.0 ? -1.0 : 1.0;
  R3 v = rcross(din, b.nh);
  b.vn = rnorm(v);
  b.fixed_s = b.vn < 1e-12;
  if (b.fixed_s) {  // normal incidence: a fixed unit vector perpendicular to n
    R3 a = fabs(b.nh.x) < 0.9 ? r3(1, 0, 0) : r3(0, 1, 0);
    b.sv = runit(rcross(b.nh, a));
  } else {
    b.sv = v * (1.0 / b.vn);
  }
  b.pin = rcross(b.sv, din);
  b.pout = rcross(b.sv, dout);
  b.pec = pec;
  if (pec) {
    b.te = zc(-1.0);
    b.tm = zc(1.0);
  } else {
    b.ec = zc(er, sg * wfac);
    b.root = zsqrt_p(b.ec - zc(1.0 - b.c * b.c));
    Zc cc = zc(b.c);
    b.te = (cc - b.root) / (cc + b.root);
    Zc ecc = b.ec * b.c;
    b.tm = (ecc - b.root) / (ecc + b.root);
  }
  return b;
}
__device__ __forceinline__ Z3 bounce_apply(const Bounce& b, const Z3& E) {
  return z3of(b.sv, b.te * zdot(E, b.sv)) + z3of(b.pout, b.tm * zdot(E, b.pin));
}

__global__ void k_grad_adjoint(GradArgs g) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < g.n_paths; p += gridDim.x * blockDim.x) {
    const dcem_path& P = g.paths[p];
    const long base = (long)p * g.W;
    for (int q = 0; q < g.W; ++q) g.param[base + q] = -1;
    const int k = P.depth;
    bool good = k >= 0 && k <= g.max_refl && P.rx >= 0 && P.rx < g.nrx;
    for (int j = 0; good && j < k; ++j) good = P.tri[j] >= 0 && P.tri[j] < g.ntri;
    if (!good) {
      atomicOr(g.err, 2u);
      continue;
    }
    if (p > 0 && g.paths[p - 1].rx > P.rx) atomicOr(g.err, 1u);
    // ---- forward sweep: geometry in FP64 at theta
    const double wfac = -1.0 / (2.0 * kPi * g.freq * kEps0);
    R3 V0[kMaxRefl], Nn[kMaxRefl], img[kMaxRefl + 1], X[kMaxRefl + 2];
    double er[kMaxRefl], sg[kMaxRefl];
    int mat[kMaxRefl], obj[kMaxRefl];
    bool pec[kMaxRefl];
    const R3 tx = r3(g.tx[0], g.tx[1], g.tx[2]);
    const float4 rv = g.rx[P.rx];
    bool ok = true;
    img[0] = tx;
    for (int j = 0; j < k && ok; ++j) {
      const int id = P.tri[j];
      const float4* t = g.tris + 3 * (size_t)g.slot_of_id[id];
      obj[j] = g.tri_obj[id];
      R3 off = r3(0.0, 0.0, 0.0);
      if (g.theta && obj[j] >= 0) {
        const double* th = g.theta + 2 * g.nmat + 2 * obj[j];
        const float* xf = g.xf + 12 * (size_t)obj[j];
        off = r3(th[0] - (double)xf[3], th[1] - (double)xf[7], 0.0);
      }
      R3 v0 = r3(t[0].x, t[0].y, t[0].z) + off, v1 = r3(t[1].x, t[1].y, t[1].z) + off,
         v2 = r3(t[2].x, t[2].y, t[2].z) + off;
      R3 n = rcross(v1 - v0, v2 - v0);
      double nn = rdot(n, n);
      if (!(nn > 0.0)) ok = false;
      img[j + 1] = img[j] - n * (2.0 * rdot(img[j] - v0, n) / nn);
      V0[j] = v0;
      Nn[j] = n;
      mat[j] = g.tri_mat[id];
      const float4 mt = g.mats[mat[j]];
      pec[j] = mt.z != 0.0f;
      er[j] = g.theta ? g.theta[2 * mat[j]] : (double)mt.x;
      sg[j] = g.theta ? g.theta[2 * mat[j] + 1] : (double)mt.y;
    }
    X[0] = tx;
    X[k + 1] = r3(rv.x, rv.y, rv.z);
    for (int j = k; j >= 1 && ok; --j) {
      R3 dir = img[j] - X[j + 1];
      double den = rdot(dir, Nn[j - 1]);
      if (den == 0.0) {
        ok = false;
        break;
      }
      double s = rdot(V0[j - 1] - X[j + 1], Nn[j - 1]) / den;
      X[j] = X[j + 1] + dir * s;
    }
    R3 dv[kMaxRefl + 1];
    double ell[kMaxRefl + 1], L = 0.0;
    for (int i = 0; i <= k && ok; ++i) {
      R3 e = X[i + 1] - X[i];
      ell[i] = rnorm(e);
      if (!(ell[i] > 0.0)) ok = false;
      else dv[i] = e * (1.0 / ell[i]);
      L += ell[i];
    }
    if (!ok) {
      atomicOr(g.err, 4u);
      continue;
    }
    // ---- the field (the bounces are recomputed from the vertices below)
    const R3 u = r3(g.pol[0], g.pol[1], g.pol[2]);
    const Pol pol0 = pol_fwd(u, dv[0]);
    const Z3 E0 = Z3{zc(pol0.n.x), zc(pol0.n.y), zc(pol0.n.z)};
    Z3 E = E0;
    for (int j = 1; j <= k; ++j)
      E = bounce_apply(bounce_of(dv[j - 1], dv[j], Nn[j - 1], er[j - 1], sg[j - 1], pec[j - 1], wfac), E);
    const R3 mdk = dv[k] * -1.0;
    const Pol polr = pol_fwd(u, mdk);
    const double lam = kC0 / g.freq, kw = 2.0 * kPi * g.freq / kC0, K = lam / (4.0 * kPi);
    double sp, cp;
    sincos(kw * L, &sp, &cp);
    const Zc ph = zc(cp, -sp);  // e^{-j k L}
    const Zc Pp = zdot(E, polr.n);
    const Zc a = Pp * ph * (K / L);
    // ---- backward sweep from a-bar = 1
    Z3 Xb[kMaxRefl + 2], db[kMaxRefl + 1];
    const Z3 z0 = Z3{zc(0.0), zc(0.0), zc(0.0)};
    for (int i = 0; i <= k + 1; ++i) Xb[i] = z0;
    for (int i = 0; i <= k; ++i) db[i] = z0;
    Zc ebar[kMaxRefl];
    const Zc Pbar = ph * (K / L);
    const Zc Lbar = a * zc(-1.0 / L, -kw);
    Z3 Eb = z3of(polr.n, Pbar);
    db[k] = db[k] - pol_bwd(polr, mdk, E * Pbar);  // the Rx polarisation is taken along -d_k
    for (int j = k; j >= 1; --j) {
      // the field before bounce j, recomputed from the vertices
      Z3 Em = E0;
      for (int q = 1; q < j; ++q)
        Em = bounce_apply(bounce_of(dv[q - 1], dv[q], Nn[q - 1], er[q - 1], sg[q - 1], pec[q - 1], wfac), Em);
      const Bounce b = bounce_of(dv[j - 1], dv[j], Nn[j - 1], er[j - 1], sg[j - 1], pec[j - 1], wfac);
      const Zc es = zdot(Em, b.sv), ep = zdot(Em, b.pin);
      const Zc A = b.te * es, B = b.tm * ep;
      const Zc Ab = zdot(Eb, b.sv), Bb = zdot(Eb, b.pout);
      Z3 svb = Eb * A + Em * (Ab * b.te);
      const Z3 poutb = Eb * B;
      const Z3 pinb = Em * (Bb * b.tm);
      const Zc teb = Ab * es, tmb = Bb * ep;
      Eb = z3of(b.sv, Ab * b.te) + z3of(b.pin, Bb * b.tm);
      ebar[j - 1] = zc(0.0);
      if (!b.pec) {
        const Zc r = b.root, cc = zc(b.c), c2 = zc(b.c * b.c);
        const Zc Dte = cc + r, Dtm = b.ec * b.c + r;
        const Zc w = r - c2 / r;                      // r - c^2 / r
        const Zc dte_dc = w * 2.0 / (Dte * Dte);
        const Zc dte_de = (cc / r) * -1.0 / (Dte * Dte);
        const Zc dtm_dc = b.ec * w * 2.0 / (Dtm * Dtm);
        const Zc dtm_de = cc * (r * 2.0 - b.ec / r) / (Dtm * Dtm);
        const Zc cb = teb * dte_dc + tmb * dtm_dc;
        ebar[j - 1] = teb * dte_de + tmb * dtm_de;
        db[j - 1] = db[j - 1] + z3of(b.nh, cb * b.sgn);
      }
      svb = svb + zcross(dv[j - 1], pinb) + zcross(dv[j], poutb);
      db[j - 1] = db[j - 1] + zcross(pinb, b.sv);
      db[j] = db[j] + zcross(poutb, b.sv);
      if (!b.fixed_s) {
        Z3 vb = (svb - z3of(b.sv, zdot(svb, b.sv))) * (1.0 / b.vn);
        db[j - 1] = db[j - 1] + zcross(b.nh, vb);
      }
    }
    db[0] = db[0] + pol_bwd(pol0, dv[0], Eb);
    // directions and lengths -> vertices
    for (int i = 0; i <= k; ++i) {
      Z3 t = (db[i] - z3of(dv[i], zdot(db[i], dv[i]))) * (1.0 / ell[i]);
      t = t + z3of(dv[i], Lbar);
      Xb[i + 1] = Xb[i + 1] + t;
      Xb[i] = Xb[i] - t;
    }
    // ---- outputs: the value, then each parameter at its first bounce
    g.items[base] = make_double2(a.re, a.im);
    g.param[base] = -2;
    for (int j = 0; j < k; ++j) {
      if (!pec[j]) {
        bool first = true;
        for (int q = 0; q < j; ++q) first = first && mat[q] != mat[j];
        if (first) {
          Zc de = zc(0.0);
          for (int q = j; q < k; ++q)
            if (mat[q] == mat[j]) de = de + ebar[q];
          g.items[base + 1 + 4 * j] = make_double2(de.re, de.im);                 // d / d eps_r
          g.param[base + 1 + 4 * j] = 2 * mat[j];
          g.items[base + 2 + 4 * j] = make_double2(-de.im * wfac, de.re * wfac);  // d / d sigma
          g.param[base + 2 + 4 * j] = 2 * mat[j] + 1;
        }
      }
      if (obj[j] >= 0) {
        bool first = true;
        for (int q = 0; q < j; ++q) first = first && obj[q] != obj[j];
        if (!first) continue;
        for (int ax = 0; ax < 2; ++ax) {
          // tangent of the image geometry when every plane of object obj[j] moves along axis ax
          R3 ti[kMaxRefl + 1], tX[kMaxRefl + 2];
          ti[0] = r3(0, 0, 0);
          for (int q = 0; q < k; ++q) {
            R3 dv0 = obj[q] == obj[j] ? r3(ax == 0 ? 1.0 : 0.0, ax == 1 ? 1.0 : 0.0, 0.0) : r3(0, 0, 0);
            ti[q + 1] = ti[q] - Nn[q] * (2.0 * rdot(ti[q] - dv0, Nn[q]) / rdot(Nn[q], Nn[q]));
          }
          tX[k + 1] = r3(0, 0, 0);
          for (int q = k; q >= 1; --q) {
            R3 dv0 = obj[q - 1] == obj[j] ? r3(ax == 0 ? 1.0 : 0.0, ax == 1 ? 1.0 : 0.0, 0.0) : r3(0, 0, 0);
            R3 dir = img[q] - X[q + 1], tdir = ti[q] - tX[q + 1];
            double den = rdot(dir, Nn[q - 1]), tden = rdot(tdir, Nn[q - 1]);
            double s = rdot(V0[q - 1] - X[q + 1], Nn[q - 1]) / den;
            double ts = (rdot(dv0 - tX[q + 1], Nn[q - 1]) - s * tden) / den;
            tX[q] = tX[q + 1] + dir * ts + tdir * s;
          }
          Zc da = zc(0.0);
          for (int i = 1; i <= k; ++i) da = da + zdot(Xb[i], tX[i]);
          g.items[base + 3 + ax + 4 * j] = make_double2(da.re, da.im);
          g.param[base + 3 + ax + 4 * j] = 2 * g.nmat + 2 * obj[j] + ax;
        }
      }
    }
  }
}

// Vector-Jacobian product of the received powers: one thread per parameter,
// receivers summed in order.
__global__ void k_theta_bar(GradArgs g, int nparam) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nparam; t += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int r = 0; r < g.nrx; ++r) acc += g.pcoh_bar[r] * g.dpcoh[(size_t)r * nparam + t];
    g.theta_bar[t] = acc;
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

cudaError_t launch_adjoint(const GradArgs& a, cudaStream_t st) {
  if (a.n_paths > 0) k_grad_adjoint<<<(a.n_paths + 63) / 64, 64, 0, st>>>(a);
  int nparam = grad_nparam(a.nmat, a.nobj);
  if (a.nrx > 0) k_grad_reduce<<<(a.nrx + 3) / 4, 128, 0, st>>>(a, nparam);
  if (a.theta_bar && nparam > 0) k_theta_bar<<<(nparam + 127) / 128, 128, 0, st>>>(a, nparam);
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

DCEM_CHECKS_TAKER(checks_take_grad)

}  // namespace dcem
