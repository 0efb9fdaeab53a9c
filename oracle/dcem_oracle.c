/*
 * dcem_oracle.c -- plain, slow, brute-force FP64 CPU oracle of the dynamic
 * coherence-based EM ray tracer (DCEM, arXiv 2112.07115).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes, in the paper's order (Sec. III "Backward ray tracing",
 * steps 1-4 and 6; Eq. 1-3 for the field):
 *   or_transform   rigid transform of moving objects' vertices (per-frame
 *                  update of the scene, Sec. III "Efficient BVH updating"),
 *                  evaluated as fmaf(R0,x, fmaf(R1,y, fmaf(R2,z,t))) in FP32.
 *   or_trace       step 1-2: shoot every ray of the sampled sphere, find the
 *                  closest hit against ALL triangles (no acceleration
 *                  structure), reflect specularly up to N times, and record
 *                  every reception-sphere capture (ray, segment, receiver).
 *   or_validate    steps 3-4 and 6: image-receiver chain through the planes
 *                  of a triangle sequence, back-trace, point-in-triangle and
 *                  occlusion tests, then length, delay, Fresnel TE/TM
 *                  reflection with vector polarisation and complex amplitude
 *                  (ray field of Eq. 1 with the free-space loss of Eq. 3).
 *   or_exhaustive  every triangle sequence of length <= N validated by the
 *                  image method (no sampling): the complete valid path set.
 *   or_trace_tree  steps 1-2 with transmission (Sec. III "Reflected and
 *                  transmitted rays"; Table II penetration losses): at a hit
 *                  on a transmitting material the ray both reflects and
 *                  continues straight through (a child ray), up to N
 *                  reflections and T transmissions per path; or_validate
 *                  takes such sequences (transmission marked by OR_TRANS in
 *                  the triangle id) and scales the field by the material's
 *                  penetration loss at each transmission.
 *   or_fresnel     Fresnel reflection coefficients.
 *   or_diffract    step 5, first order: edge diffraction paths Tx -> Q -> Rx
 *                  over the wedges of the scene (edges shared by two
 *                  non-coplanar triangles of one rigid object or both
 *                  static), Q on the edge by Keller's law,
 *                  kept when the receiver lies in the source's shadow region
 *                  behind the wedge and both legs are unoccluded; field by the
 *                  uniform theory of diffraction (UTD): R. G. Kouyoumjian and
 *                  P. H. Pathak, "A uniform geometrical theory of diffraction
 *                  for an edge in a perfectly conducting surface", Proc. IEEE
 *                  62(11), 1974, with R. J. Luebbers' finite-conductivity
 *                  reflection factors (IEEE Trans. Antennas Propag. 32(1),
 *                  1984). The transition function is evaluated from its
 *                  integral definition by quadrature along a rotated contour.
 *   or_diffract_refl, or_diffract_multi, or_diffract_multi_refl,
 *   or_diffract_refl2, or_diffract_mid
 *                  step 5 with steps 3-4: one reflection before or after a
 *                  first-order diffraction, chains of 2-3 wedges (Keller
 *                  points by minimising the unfolded length), such chains
 *                  with one reflection before or after them, two reflections
 *                  around one diffraction, and one reflection between two
 *                  diffractions; reflections by image theory on static
 *                  triangles.
 *   or_diffract_trans
 *                  first-order diffraction whose legs pass straight through
 *                  penetrable triangles (Table II losses), up to T in all.
 *   or_diffract_multi_trans
 *                  chains of 2-3 wedges whose legs cross penetrable
 *                  triangles likewise.
 *   or_keller_points
 *                  the Keller points of a chain of 1-3 edges between two
 *                  points (the solver the functions above use), for pins.
 *
 * Everything after the FP32 inputs is FP64. Decisions that FP32 arithmetic
 * could take differently (a ray passing within a margin of a triangle edge,
 * two hits at almost equal distance, a receiver on the capture-sphere
 * boundary, an occluder near a sub-segment end) are FLAGGED here so that
 * callers can exclude them from bit-exact comparisons.
 *
 * Build: gcc -O2 -ffp-contract=off -shared -fPIC -pthread dcem_oracle.c -lm
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define OR_MAX_REFL 10
#define OR_TRANS 0x40000000  /* interaction id flag: transmission through the triangle */
#define OR_DIFF 0x20000000   /* interaction id flag: diffraction at edge `id` */

/* ray / path flag bits */
#define ORF_NEAR_EDGE 1u     /* a triangle's in/out decision is within the margin */
#define ORF_TIE 2u           /* two hit candidates at nearly equal distance       */
#define ORF_NEAR_TMIN 4u     /* a hit candidate near the self-hit offset t_min    */
#define ORF_NEAR_SPHERE 8u   /* a receiver near its capture-sphere boundary       */
#define ORF_VAL_EDGE 16u     /* a reflection point near its triangle's boundary   */
#define ORF_VAL_PARAM 32u    /* back-trace parameter near 0 or 1                  */
#define ORF_OCC_NEAR 64u     /* an occlusion decision within the margin           */
#define ORF_POL_DEGEN 128u   /* polarisation reference parallel to a path end     */

typedef struct { double x, y, z; } v3;

static inline v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static inline v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static inline v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static inline v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static inline double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static inline v3 cross(v3 a, v3 b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static inline double norm(v3 a) { return sqrt(dot(a, a)); }
static inline v3 unit(v3 a) { return scl(a, 1.0 / norm(a)); }
static inline double maxabs(v3 a) { return fmax(fabs(a.x), fmax(fabs(a.y), fabs(a.z))); }

/* ------------------------------------------------------------------------ */
/* parameters (the oracle's own copy; the CUDA path has its own struct)      */
/* ------------------------------------------------------------------------ */
typedef struct {
  double freq_hz;          /* carrier frequency                                */
  double tx_power_w;       /* transmit power (Sec. III: 5 W outdoor)           */
  double alpha;            /* angular ray spacing sqrt(4 pi / n_rays)          */
  double rx_radius_scale;  /* capture radius = scale * alpha * (D + s) / sqrt 3 */
  double t_min;            /* self-hit offset after a reflection [m]           */
  double escape_len;       /* length of an escaping segment for capture [m]    */
  double eps_occ;          /* occlusion tests ignore (0,eps) and (1-eps,1)     */
  double edge_eps;         /* relative flag margin for FP32 decisions          */
  double val_eps;          /* relative flag margin for FP64 validation         */
  double pol[3];           /* antenna polarisation reference vector u          */
  int32_t max_refl;        /* N reflections                                    */
  int32_t nthreads;        /* 0 = all cores                                     */
  const double* trans_db;  /* per material penetration loss [dB]; < 0 opaque;
                              NULL: every material opaque                       */
  int32_t max_trans;       /* T transmissions per path (N + T <= OR_MAX_REFL)   */
  int32_t pad_;
} or_params;



/* ------------------------------------------------------------------------ */
/* scene: FP32 world triangles widened to FP64                               */
/* ------------------------------------------------------------------------ */
typedef struct {
  v3 v[3];
  v3 n;       /* (v1-v0) x (v2-v0) */
  v3 nh;      /* unit normal */
  v3 e[3];    /* edges v0->v1, v1->v2, v2->v0 */
  double elen[3];
  int mat;
} otri;

typedef struct {
  int ntri;
  otri* t;
  double* mats;  /* nmat x 3: eps_r, sigma, pec (owned copy) */
  int nmat;
} oscene;

static int transmits(const oscene* S, const or_params* P, int mat) {
  return P->trans_db && P->max_trans > 0 && mat >= 0 && mat < S->nmat && P->trans_db[mat] >= 0.0;
}

static void tri_setup(otri* T) {
    T->e[0] = sub(T->v[1], T->v[0]);
    T->e[1] = sub(T->v[2], T->v[1]);
    T->e[2] = sub(T->v[0], T->v[2]);
    for (int k = 0; k < 3; ++k) T->elen[k] = norm(T->e[k]);
    T->n = cross(sub(T->v[1], T->v[0]), sub(T->v[2], T->v[0]));
    double nn = norm(T->n);
    T->nh = nn > 0 ? scl(T->n, 1.0 / nn) : mk(0, 0, 0);
}

/* Exactly one of tris / tris_d (vertices) and of mats / mats_d is given. */
static int scene_load_any(oscene* s, const float* tris, const double* tris_d, const int32_t* tri_mat,
                          int ntri, const float* mats, const double* mats_d, int nmat) {
  s->ntri = ntri;
  s->nmat = nmat;
  s->t = (otri*)calloc((size_t)(ntri > 0 ? ntri : 1), sizeof(otri));
  s->mats = (double*)calloc((size_t)(nmat > 0 ? 3 * nmat : 3), sizeof(double));
  if (!s->t || !s->mats) return -1;
  for (int i = 0; i < 3 * nmat; ++i) s->mats[i] = mats_d ? mats_d[i] : (double)mats[i];
  for (int i = 0; i < ntri; ++i) {
    otri* T = &s->t[i];
    for (int k = 0; k < 3; ++k)
      T->v[k] = tris_d ? mk(tris_d[9 * i + 3 * k], tris_d[9 * i + 3 * k + 1], tris_d[9 * i + 3 * k + 2])
                       : mk(tris[9 * i + 3 * k], tris[9 * i + 3 * k + 1], tris[9 * i + 3 * k + 2]);
    tri_setup(T);
    T->mat = tri_mat ? tri_mat[i] : 0;
  }
  return 0;
}

/* FP32 world triangles and materials widened to FP64 */
static int scene_load(oscene* s, const float* tris, const int32_t* tri_mat, int ntri,
                      const float* mats, int nmat) {
  return scene_load_any(s, tris, NULL, tri_mat, ntri, mats, NULL, nmat);
}

static void scene_free(oscene* s) { free(s->t); free(s->mats); }

static int default_threads(int req) {
  if (req > 0) return req;
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)n : 1;
}

/* ------------------------------------------------------------------------ */
/* A1: rigid transform of the moving objects' vertices                      */
/* ------------------------------------------------------------------------ */
/* x' = R0.x*x + R0.y*y + R0.z*z + t0, evaluated innermost-first with
 * correctly rounded fused multiply-adds (C99 fmaf) in FP32. */
void or_transform(int32_t ntri, const float* tris_in, const int32_t* tri_obj,
                  const float* xf, int32_t nobj, float* tris_out) {
  for (int i = 0; i < ntri; ++i) {
    int o = tri_obj ? tri_obj[i] : -1;
    for (int k = 0; k < 3; ++k) {
      const float* p = &tris_in[9 * i + 3 * k];
      float* q = &tris_out[9 * i + 3 * k];
      if (o < 0 || o >= nobj) {
        q[0] = p[0]; q[1] = p[1]; q[2] = p[2];
        continue;
      }
      const float* m = &xf[12 * o];
      for (int r = 0; r < 3; ++r)
        q[r] = fmaf(m[4 * r + 0], p[0], fmaf(m[4 * r + 1], p[1], fmaf(m[4 * r + 2], p[2], m[4 * r + 3])));
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Fresnel reflection (eps_c = eps_r - j sigma / (omega eps0), exp(+j w t))   */
/* ------------------------------------------------------------------------ */
static const double EPS0 = 8.8541878128e-12;
static const double C0 = 299792458.0;

/* Gamma_TE, Gamma_TM at incidence cos(theta) = cos_t for a half-space of
 * relative permittivity eps_r and conductivity sigma; pec selects the perfect
 * conductor limits (-1, +1). */
static void fresnel64(double eps_r, double sigma, int pec, double freq, double cos_t,
                      double complex* g_te, double complex* g_tm) {
  if (pec) {
    *g_te = -1.0;
    *g_tm = 1.0;
    return;
  }
  double complex ec = eps_r - I * (sigma / (2.0 * M_PI * freq * EPS0));
  double sin2 = 1.0 - cos_t * cos_t;
  double complex root = csqrt(ec - sin2);
  *g_te = (cos_t - root) / (cos_t + root);
  *g_tm = (ec * cos_t - root) / (ec * cos_t + root);
}

/* material row (eps_r, sigma, pec) */
static void fresnel(const double* mat, double freq, double cos_t, double complex* g_te,
                    double complex* g_tm) {
  fresnel64(mat[0], mat[1], mat[2] != 0.0, freq, cos_t, g_te, g_tm);
}

void or_fresnel(double eps_r, double sigma, int32_t pec, double freq, double cos_t,
                double* out4) {
  double m[3] = {(double)(float)eps_r, (double)(float)sigma, (double)pec};
  double complex te, tm;
  fresnel(m, freq, cos_t, &te, &tm);
  out4[0] = creal(te); out4[1] = cimag(te);
  out4[2] = creal(tm); out4[3] = cimag(tm);
}

/* Same with eps_r, sigma taken at full double precision (closed-form pins). */
void or_fresnel64(double eps_r, double sigma, int32_t pec, double freq, double cos_t,
                  double* out4) {
  double complex te, tm;
  fresnel64(eps_r, sigma, pec != 0, freq, cos_t, &te, &tm);
  out4[0] = creal(te); out4[1] = cimag(te);
  out4[2] = creal(tm); out4[3] = cimag(tm);
}

/* ------------------------------------------------------------------------ */
/* ray vs triangle, exact definition: the ray line passes through the        */
/* triangle iff the three signed volumes d.((P-o)x(Q-o)) of its edges share  */
/* a sign; the hit distance is the plane crossing. No back-face culling.    */
/* ------------------------------------------------------------------------ */
typedef struct {
  double t;       /* plane crossing parameter (NAN if parallel) */
  int inside;     /* ray line passes through the closed triangle */
  int flippable;  /* a perturbation of the ray by `delta` could change `inside` */
  double cos_t;   /* |d . n^| */
} xinfo;

/* delta: ray-line displacement budget at the crossing. */
static void ray_tri(const otri* T, v3 o, v3 d, double delta_base, double delta_slope, xinfo* x) {
  double dn = dot(d, T->n);
  x->cos_t = T->elen[0] > 0 ? fabs(dot(d, T->nh)) : 0.0;
  if (dn == 0.0 || !(norm(T->n) > 0)) {
    x->t = NAN; x->inside = 0; x->flippable = 0;
    return;
  }
  x->t = dot(sub(T->v[0], o), T->n) / dn;
  double delta = delta_base + delta_slope * fabs(x->t);
  v3 a = sub(T->v[0], o), b = sub(T->v[1], o), c = sub(T->v[2], o);
  double E[3];
  E[0] = dot(d, cross(a, b));
  E[1] = dot(d, cross(b, c));
  E[2] = dot(d, cross(c, a));
  int pos = (E[0] >= 0) && (E[1] >= 0) && (E[2] >= 0);
  int neg = (E[0] <= 0) && (E[1] <= 0) && (E[2] <= 0);
  x->inside = (pos || neg) && !(E[0] == 0 && E[1] == 0 && E[2] == 0);
  /* line distance between the ray and edge k: |E_k| / |d x e_k| (d unit, so
   * |d x e_k| <= |e_k|: when |E_k| >= delta |e_k| the edge is surely farther
   * than delta and the exact distance is not needed). */
  double dist[3];
  for (int k = 0; k < 3; ++k) {
    if (fabs(E[k]) >= delta * T->elen[k]) { dist[k] = INFINITY; continue; }
    double den = norm(cross(d, T->e[k]));
    dist[k] = den > 0 ? fabs(E[k]) / den : INFINITY;
  }
  if (x->inside) {
    x->flippable = (dist[0] < delta) || (dist[1] < delta) || (dist[2] < delta);
  } else {
    int to_pos = 1, to_neg = 1;
    for (int k = 0; k < 3; ++k) {
      if (E[k] < 0 && !(dist[k] < delta)) to_pos = 0;
      if (E[k] > 0 && !(dist[k] < delta)) to_neg = 0;
    }
    x->flippable = to_pos || to_neg;
  }
}

/* Closest hit of the ray (o, d unit) over all triangles except `excl`, with
 * t > t_min; ties in t go to the lowest triangle id. Sets flag bits. */
static int closest_hit(const oscene* S, v3 o, v3 d, double D, int excl, const or_params* P,
                       xinfo* xs, double* t_out, double* cos_out, uint32_t* flags) {
  double base = P->edge_eps * (maxabs(o) + D);
  double slope = P->edge_eps;
  int best = -1;
  double bt = INFINITY;
  for (int j = 0; j < S->ntri; ++j) {
    if (j == excl) { xs[j].t = NAN; xs[j].inside = 0; xs[j].flippable = 0; continue; }
    ray_tri(&S->t[j], o, d, base, slope, &xs[j]);
    if (xs[j].inside && xs[j].t > P->t_min) {
      if (xs[j].t < bt) { bt = xs[j].t; best = j; }
    }
  }
  /* flags */
  double dtb = 0;
  if (best >= 0) dtb = (base + slope * bt) / fmax(xs[best].cos_t, 1e-6);
  for (int j = 0; j < S->ntri; ++j) {
    if (j == excl || isnan(xs[j].t)) continue;
    if (!(xs[j].inside || xs[j].flippable)) continue;
    double dt = (base + slope * fabs(xs[j].t)) / fmax(xs[j].cos_t, 1e-6);
    if (xs[j].t < P->t_min - dt) continue;
    if (best >= 0 && xs[j].t > bt + dt + dtb) continue;
    if (xs[j].flippable) *flags |= ORF_NEAR_EDGE;
    if (fabs(xs[j].t - P->t_min) <= dt) *flags |= ORF_NEAR_TMIN;
    if (best >= 0 && j != best && fabs(xs[j].t - bt) <= dt + dtb) *flags |= ORF_TIE;
  }
  *t_out = bt;
  *cos_out = best >= 0 ? xs[best].cos_t : 0;
  return best;
}

/* ------------------------------------------------------------------------ */
/* or_trace: SBR shooting of all rays (steps 1-2)                            */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t ray, seg, rx;
} ocand;

typedef struct {
  ocand* c;
  long n, cap;
} cvec;

static int cpush(cvec* v, int ray, int seg, int rx) {
  if (v->n == v->cap) {
    long nc = v->cap ? 2 * v->cap : 1024;
    ocand* p = (ocand*)realloc(v->c, (size_t)nc * sizeof(ocand));
    if (!p) return -1;
    v->c = p; v->cap = nc;
  }
  v->c[v->n].ray = ray; v->c[v->n].seg = seg; v->c[v->n].rx = rx;
  v->n++;
  return 0;
}

typedef struct {
  const oscene* S;
  const or_params* P;
  v3 tx;
  const float* rays;
  int nrays;
  const float* rx;
  int nrx;
  int32_t* hit_id;    /* nrays x (N+1) */
  double* hit_t;      /* nrays x (N+1) */
  int32_t* nseg;      /* nrays */
  uint32_t* flags;    /* nrays */
  double* seg_od;     /* optional nrays x (N+1) x 7: o, d, D */
  atomic_long next;
  cvec* cv;           /* per thread */
  int err;
} trace_job;

typedef struct { trace_job* J; int tid; } targ;

static void trace_one(trace_job* J, int i, xinfo* xs, cvec* cv) {
  const or_params* P = J->P;
  int N = P->max_refl, W = N + 1;
  v3 o = J->tx;
  v3 d = unit(mk(J->rays[3 * i], J->rays[3 * i + 1], J->rays[3 * i + 2]));
  double D = 0;
  int last = -1;
  uint32_t fl = 0;
  double ae = P->rx_radius_scale * P->alpha / sqrt(3.0);
  for (int b = 0; b <= N; ++b) {
    double t, ct;
    int id = closest_hit(J->S, o, d, D, last, P, xs, &t, &ct, &fl);
    double tend = id >= 0 ? t : P->escape_len;
    double base = P->edge_eps * (maxabs(o) + D);
    double dtb = id >= 0 ? (base + P->edge_eps * t) / fmax(ct, 1e-6) : 0.0;
    if (J->seg_od) {
      double* q = &J->seg_od[((size_t)i * W + b) * 7];
      q[0] = o.x; q[1] = o.y; q[2] = o.z; q[3] = d.x; q[4] = d.y; q[5] = d.z; q[6] = D;
    }
    /* reception-sphere capture of this segment */
    for (int r = 0; r < J->nrx; ++r) {
      v3 R = mk(J->rx[3 * r], J->rx[3 * r + 1], J->rx[3 * r + 2]);
      v3 w = sub(R, o);
      double s = dot(w, d);
      int clamped = 0;
      if (s < 0) s = 0;
      if (s > tend) { s = tend; clamped = 1; }
      double dist = norm(sub(w, scl(d, s)));
      double rho = ae * (D + s);
      double m = (base + P->edge_eps * s) * (1.0 + ae) + (clamped ? dtb * (1.0 + ae) : 0.0);
      if (fabs(dist - rho) <= m) fl |= ORF_NEAR_SPHERE;
      if (dist <= rho) {
        if (cpush(cv, i, b, r)) J->err = 1;
      }
    }
    J->hit_id[(size_t)i * W + b] = id;
    J->hit_t[(size_t)i * W + b] = id >= 0 ? t : INFINITY;
    if (id < 0) { J->nseg[i] = b + 1; break; }
    J->nseg[i] = b + 1;
    /* specular reflection: d' = d - 2 (d.n^) n^ */
    const otri* T = &J->S->t[id];
    v3 p = add(o, scl(d, t));
    d = unit(sub(d, scl(T->nh, 2.0 * dot(d, T->nh))));
    o = p;
    D += t;
    last = id;
  }
  for (int b = J->nseg[i]; b <= N; ++b) {
    J->hit_id[(size_t)i * W + b] = -2;
    J->hit_t[(size_t)i * W + b] = NAN;
  }
  J->flags[i] = fl;
}

static void* trace_worker(void* p) {
  targ* a = (targ*)p;
  trace_job* J = a->J;
  xinfo* xs = (xinfo*)malloc(sizeof(xinfo) * (size_t)(J->S->ntri > 0 ? J->S->ntri : 1));
  if (!xs) { J->err = 1; return NULL; }
  for (;;) {
    long s = atomic_fetch_add(&J->next, 64);
    if (s >= J->nrays) break;
    long e = s + 64 < J->nrays ? s + 64 : J->nrays;
    for (long i = s; i < e; ++i) trace_one(J, (int)i, xs, &J->cv[a->tid]);
  }
  free(xs);
  return NULL;
}

static int cand_cmp(const void* a, const void* b) {
  const ocand* x = (const ocand*)a;
  const ocand* y = (const ocand*)b;
  if (x->ray != y->ray) return x->ray < y->ray ? -1 : 1;
  if (x->seg != y->seg) return x->seg < y->seg ? -1 : 1;
  if (x->rx != y->rx) return x->rx < y->rx ? -1 : 1;
  return 0;
}

/* Returns 0 on success. *cand_out is malloc'd (3 ints per capture, sorted by
 * ray, segment, receiver); free it with or_free. */
int or_trace(const float* tris, const int32_t* tri_mat, int32_t ntri, const float* mats,
             int32_t nmat, const float* tx, const float* rays, int32_t nrays, const float* rx,
             int32_t nrx, const or_params* P, int32_t* hit_id, double* hit_t, int32_t* nseg,
             uint32_t* flags, double* seg_od, int32_t** cand_out, int64_t* ncand_out) {
  if (P->max_refl < 0 || P->max_refl > OR_MAX_REFL) return -1;
  oscene S;
  if (scene_load(&S, tris, tri_mat, ntri, mats, nmat)) return -2;
  trace_job J;
  memset(&J, 0, sizeof(J));
  J.S = &S; J.P = P; J.tx = mk(tx[0], tx[1], tx[2]);
  J.rays = rays; J.nrays = nrays; J.rx = rx; J.nrx = nrx;
  J.hit_id = hit_id; J.hit_t = hit_t; J.nseg = nseg; J.flags = flags; J.seg_od = seg_od;
  atomic_init(&J.next, 0);
  int nt = default_threads(P->nthreads);
  J.cv = (cvec*)calloc((size_t)nt, sizeof(cvec));
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
  targ* args = (targ*)malloc(sizeof(targ) * (size_t)nt);
  for (int k = 0; k < nt; ++k) {
    args[k].J = &J; args[k].tid = k;
    pthread_create(&th[k], NULL, trace_worker, &args[k]);
  }
  for (int k = 0; k < nt; ++k) pthread_join(th[k], NULL);
  long tot = 0;
  for (int k = 0; k < nt; ++k) tot += J.cv[k].n;
  ocand* all = (ocand*)malloc(sizeof(ocand) * (size_t)(tot > 0 ? tot : 1));
  long pos = 0;
  for (int k = 0; k < nt; ++k) {
    if (J.cv[k].n) memcpy(all + pos, J.cv[k].c, sizeof(ocand) * (size_t)J.cv[k].n);
    pos += J.cv[k].n;
    free(J.cv[k].c);
  }
  qsort(all, (size_t)tot, sizeof(ocand), cand_cmp);
  *cand_out = (int32_t*)all;
  *ncand_out = tot;
  free(J.cv); free(th); free(args);
  scene_free(&S);
  return J.err ? -3 : 0;
}

/* ------------------------------------------------------------------------ */
/* or_trace_tree: steps 1-2 with transmission                                */
/* ------------------------------------------------------------------------ */
/* A ray instance: the primary ray of a sampled direction, or a child that
 * continues straight through a transmitting triangle its parent hit. Its
 * interaction ids (hit[0..nseg-1]; OR_TRANS marks a transmission) include
 * the parent's prefix, so any capture's key is hit[0..seg-1]. */
#define OR_MAX_SEG (OR_MAX_REFL + 1)
typedef struct {
  int32_t root;         /* sampled direction (primary ray index)          */
  int32_t start;        /* first segment this instance traces              */
  int32_t nseg;
  uint32_t flags;       /* own and inherited flag bits                     */
  int32_t hit[OR_MAX_SEG];
  double t[OR_MAX_SEG];
} oinst;

typedef struct {
  oinst* v;
  long n, cap;
} ivec;

static int ipush(ivec* v, const oinst* x) {
  if (v->n == v->cap) {
    long nc = v->cap ? 2 * v->cap : 256;
    oinst* p = (oinst*)realloc(v->v, (size_t)nc * sizeof(oinst));
    if (!p) return -1;
    v->v = p; v->cap = nc;
  }
  v->v[v->n++] = *x;
  return 0;
}

/* one pending instance: state at the start of segment b */
typedef struct {
  oinst in;
  v3 o, d;
  double D;
  int b, nr, nt, last;
} opend;

typedef struct {
  const oscene* S;
  const or_params* P;
  v3 tx;
  const float* rays;
  int nrays;
  const float* rx;
  int nrx;
  oinst* prim;        /* nrays primary instances */
  ivec* kids;         /* per thread: children, in (root, spawn) order */
  cvec* cv;           /* per thread: captures; ray = instance code (see below) */
  atomic_long next;
  int err;
} tree_job;

typedef struct { tree_job* J; int tid; } tree_arg;

/* capture code of an instance: primary i -> i; the c-th child of this thread
 * -> -(1 + c) (mapped to global ids after the merge) */
static void trace_tree_one(tree_job* J, int tid, int i, xinfo* xs) {
  const oscene* S = J->S;
  const or_params* P = J->P;
  const int N = P->max_refl, T = P->max_trans;
  const double ae = P->rx_radius_scale * P->alpha / sqrt(3.0);
  /* pending instances (depth first): at most N+T+1 spawns per instance on
   * each of at most T+1 levels */
  opend stack[128];
  int sp = 0;
  opend* q = &stack[sp++];
  memset(q, 0, sizeof(*q));
  q->in.root = i;
  q->o = J->tx;
  q->d = unit(mk(J->rays[3 * i], J->rays[3 * i + 1], J->rays[3 * i + 2]));
  q->last = -1;
  int first = 1;
  while (sp > 0) {
    opend cur = stack[--sp];
    int code;
    if (first) {
      code = i;
    } else {
      code = -(int)(1 + J->kids[tid].n);
    }
    oinst in = cur.in;
    in.start = cur.b;
    v3 o = cur.o, d = cur.d;
    double D = cur.D;
    int b = cur.b, nr = cur.nr, nt = cur.nt, last = cur.last;
    uint32_t fl = in.flags;
    for (;;) {
      double t, ct;
      int id = closest_hit(S, o, d, D, last, P, xs, &t, &ct, &fl);
      double tend = id >= 0 ? t : P->escape_len;
      double base = P->edge_eps * (maxabs(o) + D);
      double dtb = id >= 0 ? (base + P->edge_eps * t) / fmax(ct, 1e-6) : 0.0;
      for (int r = 0; r < J->nrx; ++r) {
        v3 R = mk(J->rx[3 * r], J->rx[3 * r + 1], J->rx[3 * r + 2]);
        v3 w = sub(R, o);
        double s = dot(w, d);
        int clamped = 0;
        if (s < 0) s = 0;
        if (s > tend) { s = tend; clamped = 1; }
        double dist = norm(sub(w, scl(d, s)));
        double rho = ae * (D + s);
        double m = (base + P->edge_eps * s) * (1.0 + ae) + (clamped ? dtb * (1.0 + ae) : 0.0);
        if (fabs(dist - rho) <= m) fl |= ORF_NEAR_SPHERE;
        if (dist <= rho && cpush(&J->cv[tid], code, b, r)) J->err = 1;
      }
      in.hit[b] = id;
      in.t[b] = id >= 0 ? t : INFINITY;
      in.nseg = b + 1;
      if (id < 0) break;
      const otri* Tr = &S->t[id];
      v3 p = add(o, scl(d, t));
      /* transmission: a child continues straight through */
      if (nt < T && b + 1 <= N + T && transmits(S, P, Tr->mat)) {
        if (sp >= 128) { J->err = 1; break; }
        opend* c = &stack[sp++];
        c->in = in;
        c->in.hit[b] = id | OR_TRANS;
        c->in.flags = fl;
        c->o = p;
        c->d = d;
        c->D = D + t;
        c->b = b + 1;
        c->nr = nr;
        c->nt = nt + 1;
        c->last = id;
      }
      if (nr >= N) break;
      /* specular reflection: d' = d - 2 (d.n^) n^ */
      d = unit(sub(d, scl(Tr->nh, 2.0 * dot(d, Tr->nh))));
      o = p;
      D += t;
      last = id;
      ++nr;
      ++b;
    }
    for (int k = in.nseg; k < OR_MAX_SEG; ++k) { in.hit[k] = -2; in.t[k] = NAN; }
    in.flags = fl;
    if (first) {
      J->prim[i] = in;
      first = 0;
    } else if (ipush(&J->kids[tid], &in)) {
      J->err = 1;
    }
    /* children of this instance inherit its flags at spawn (set above) */
  }
}

static void* trace_tree_worker(void* p) {
  tree_arg* a = (tree_arg*)p;
  tree_job* J = a->J;
  xinfo* xs = (xinfo*)malloc(sizeof(xinfo) * (size_t)(J->S->ntri > 0 ? J->S->ntri : 1));
  if (!xs) { J->err = 1; return NULL; }
  for (;;) {
    long s = atomic_fetch_add(&J->next, 16);
    if (s >= J->nrays) break;
    long e = s + 16 < J->nrays ? s + 16 : J->nrays;
    for (long i = s; i < e; ++i) trace_tree_one(J, a->tid, (int)i, xs);
  }
  free(xs);
  return NULL;
}

static int inst_cmp(const void* a, const void* b) {
  const long* x = (const long*)a;
  const long* y = (const long*)b;
  return x[0] < y[0] ? -1 : (x[0] > y[0] ? 1 : (x[1] < y[1] ? -1 : (x[1] > y[1] ? 1 : 0)));
}

/* Steps 1-2 with transmission. Instances: the nrays primaries (index = ray)
 * then the children ordered by (root ray, spawn order). Outputs (malloc'd,
 * free with or_free): inst (n_inst records), cands (3 ints per capture:
 * instance, segment, receiver; sorted). */
int or_trace_tree(const float* tris, const int32_t* tri_mat, int32_t ntri, const float* mats,
                  int32_t nmat, const float* tx, const float* rays, int32_t nrays, const float* rx,
                  int32_t nrx, const or_params* P, oinst** inst_out, int64_t* ninst_out,
                  int32_t** cand_out, int64_t* ncand_out) {
  if (P->max_refl < 0 || P->max_trans < 0 || P->max_refl + P->max_trans > OR_MAX_REFL) return -1;
  oscene S;
  if (scene_load(&S, tris, tri_mat, ntri, mats, nmat)) return -2;
  tree_job J;
  memset(&J, 0, sizeof(J));
  J.S = &S; J.P = P; J.tx = mk(tx[0], tx[1], tx[2]);
  J.rays = rays; J.nrays = nrays; J.rx = rx; J.nrx = nrx;
  J.prim = (oinst*)calloc((size_t)(nrays > 0 ? nrays : 1), sizeof(oinst));
  atomic_init(&J.next, 0);
  int nt = default_threads(P->nthreads);
  J.kids = (ivec*)calloc((size_t)nt, sizeof(ivec));
  J.cv = (cvec*)calloc((size_t)nt, sizeof(cvec));
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
  tree_arg* args = (tree_arg*)malloc(sizeof(tree_arg) * (size_t)nt);
  for (int k = 0; k < nt; ++k) {
    args[k].J = &J; args[k].tid = k;
    pthread_create(&th[k], NULL, trace_tree_worker, &args[k]);
  }
  for (int k = 0; k < nt; ++k) pthread_join(th[k], NULL);
  /* order the children by (root, spawn order): sort (root, thread, index) */
  long nk = 0;
  for (int k = 0; k < nt; ++k) nk += J.kids[k].n;
  long* ord = (long*)malloc(sizeof(long) * 3 * (size_t)(nk > 0 ? nk : 1));
  long pos = 0;
  for (int k = 0; k < nt; ++k)
    for (long c = 0; c < J.kids[k].n; ++c) {
      ord[3 * pos] = J.kids[k].v[c].root;
      ord[3 * pos + 1] = c;  /* spawn order within the thread (rays of a thread are processed in order) */
      ord[3 * pos + 2] = k;
      ++pos;
    }
  qsort(ord, (size_t)nk, 3 * sizeof(long), inst_cmp);
  /* global id of each thread's child c */
  long** gid = (long**)calloc((size_t)nt, sizeof(long*));
  for (int k = 0; k < nt; ++k) gid[k] = (long*)malloc(sizeof(long) * (size_t)(J.kids[k].n > 0 ? J.kids[k].n : 1));
  oinst* inst = (oinst*)malloc(sizeof(oinst) * (size_t)(nrays + nk > 0 ? nrays + nk : 1));
  if (nrays) memcpy(inst, J.prim, sizeof(oinst) * (size_t)nrays);
  for (long r = 0; r < nk; ++r) {
    int k = (int)ord[3 * r + 2];
    long c = ord[3 * r + 1];
    gid[k][c] = nrays + r;
    inst[nrays + r] = J.kids[k].v[c];
  }
  long tot = 0;
  for (int k = 0; k < nt; ++k) tot += J.cv[k].n;
  ocand* all = (ocand*)malloc(sizeof(ocand) * (size_t)(tot > 0 ? tot : 1));
  pos = 0;
  for (int k = 0; k < nt; ++k) {
    for (long c = 0; c < J.cv[k].n; ++c) {
      ocand x = J.cv[k].c[c];
      if (x.ray < 0) x.ray = (int32_t)gid[k][-x.ray - 1];
      all[pos++] = x;
    }
    free(J.cv[k].c);
    free(J.kids[k].v);
    free(gid[k]);
  }
  qsort(all, (size_t)tot, sizeof(ocand), cand_cmp);
  *inst_out = inst;
  *ninst_out = nrays + nk;
  *cand_out = (int32_t*)all;
  *ncand_out = tot;
  free(ord); free(gid); free(J.kids); free(J.cv); free(th); free(args); free(J.prim);
  scene_free(&S);
  return J.err ? -3 : 0;
}

int32_t or_inst_size(void) { return (int32_t)sizeof(oinst); }

void or_free(void* p) { free(p); }

/* ------------------------------------------------------------------------ */
/* or_validate: image method + field (steps 3, 4, 6)                         */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t valid;
  uint32_t flags;
  double len_m;
  double delay_s;
  double amp_re, amp_im;
  double pts[OR_MAX_REFL][3];
} opath;

/* distance from point p (in the triangle's plane) to the triangle boundary */
static double edge_margin(const otri* T, v3 p) {
  double m = INFINITY;
  for (int k = 0; k < 3; ++k) {
    v3 a = T->v[k], e = T->e[k];
    double L2 = dot(e, e);
    double u = L2 > 0 ? dot(sub(p, a), e) / L2 : 0;
    if (u < 0) u = 0;
    if (u > 1) u = 1;
    double dd = norm(sub(p, add(a, scl(e, u))));
    if (dd < m) m = dd;
  }
  return m;
}

/* p inside triangle T (p lies in its plane): same-side test of p against each
 * edge, measured along the triangle normal. */
static int point_in_tri(const otri* T, v3 p) {
  double s0 = dot(cross(T->e[0], sub(p, T->v[0])), T->n);
  double s1 = dot(cross(T->e[1], sub(p, T->v[1])), T->n);
  double s2 = dot(cross(T->e[2], sub(p, T->v[2])), T->n);
  return s0 >= 0 && s1 >= 0 && s2 >= 0;
}

/* Occlusion of the open sub-segment a->b by any triangle except ex0/ex1.
 * Parameter range (eps_occ, 1-eps_occ). Returns 1 if occluded. */
static int occluded4(const oscene* S, v3 a, v3 b, int ex0, int ex1, int ex2, int ex3, const or_params* P,
                     double scale, uint32_t* fl);

static int occluded3(const oscene* S, v3 a, v3 b, int ex0, int ex1, int ex2, const or_params* P,
                     double scale, uint32_t* fl) {
  return occluded4(S, a, b, ex0, ex1, ex2, ex2, P, scale, fl);
}

static int occluded(const oscene* S, v3 a, v3 b, int ex0, int ex1, const or_params* P,
                    double scale, uint32_t* fl) {
  return occluded3(S, a, b, ex0, ex1, ex1, P, scale, fl);
}

/* Is the open segment a-b (its first and last eps_occ trimmed) blocked by a
 * triangle other than ex0 .. ex3? Flags decisions within the FP32 margin. */
static int occluded4(const oscene* S, v3 a, v3 b, int ex0, int ex1, int ex2, int ex3, const or_params* P,
                     double scale, uint32_t* fl) {
  v3 dv = sub(b, a);
  double len = norm(dv);
  if (!(len > 0)) return 0;
  v3 d = scl(dv, 1.0 / len);  /* unit; parameter u = t / len */
  double base = P->edge_eps * scale;
  int occ = 0;
  for (int j = 0; j < S->ntri; ++j) {
    if (j == ex0 || j == ex1 || j == ex2 || j == ex3) continue;
    xinfo x;
    ray_tri(&S->t[j], a, d, base, P->edge_eps, &x);
    if (isnan(x.t)) continue;
    double u = x.t / len;
    double du = (base + P->edge_eps * fabs(x.t)) / fmax(x.cos_t, 1e-6) / len;
    double lo = P->eps_occ, hi = 1.0 - P->eps_occ;
    if (x.inside && u > lo && u < hi) occ = 1;
    if (x.inside || x.flippable) {
      if (u > lo - du && u < hi + du) {
        if (x.flippable) *fl |= ORF_OCC_NEAR;
        if (fabs(u - lo) <= du || fabs(u - hi) <= du) *fl |= ORF_OCC_NEAR;
      }
    }
  }
  return occ;
}

typedef struct { double complex x, y, z; } c3;

static inline double complex cdot(c3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

/* antenna polarisation for a path leaving/arriving along d: u - (u.d) d, unit */
static v3 pol_dir(v3 u, v3 d, uint32_t* fl) {
  v3 p = sub(u, scl(d, dot(u, d)));
  double n = norm(p);
  if (n < 1e-9) {  /* u parallel to d: fall back to a fixed perpendicular */
    *fl |= ORF_POL_DEGEN;
    v3 a = fabs(d.x) < 0.9 ? mk(1, 0, 0) : mk(0, 1, 0);
    p = sub(a, scl(d, dot(a, d)));
    n = norm(p);
  }
  return scl(p, 1.0 / n);
}

/* Sec. III steps 3, 4 and 6 for one candidate: image sources, back-trace,
 * reflection points inside their triangles, (if check_occ) unoccluded
 * sub-segments, then the path length and complex amplitude. */
static void validate_one(const oscene* S, const or_params* P, v3 tx, v3 rx, int k,
                         const int32_t* ids, opath* out, int check_occ) {
  memset(out, 0, sizeof(*out));
  uint32_t fl = 0;
  /* interactions: reflections, and transmissions (OR_TRANS) straight through
   * a transmitting triangle */
  int tid[OR_MAX_REFL], isT[OR_MAX_REFL], rj[OR_MAX_REFL], m = 0;
  for (int j = 0; j < k; ++j) {
    if (ids[j] < 0) { out->valid = 0; return; }
    isT[j] = (ids[j] & OR_TRANS) != 0;
    tid[j] = ids[j] & ~OR_TRANS;
    if (tid[j] >= S->ntri) { out->valid = 0; return; }
    if (isT[j] && !transmits(S, P, S->t[tid[j]].mat)) { out->valid = 0; return; }
    if (!isT[j]) rj[m++] = j;
  }
  /* image sources I_1..I_m of the transmitter in the planes of the
   * reflecting triangles (transmissions do not turn the path) */
  v3 img[OR_MAX_REFL + 1];
  img[0] = tx;
  for (int q = 1; q <= m; ++q) {
    const otri* T = &S->t[tid[rj[q - 1]]];
    double nn = dot(T->n, T->n);
    if (!(nn > 0)) { out->valid = 0; return; }
    double h = dot(sub(img[q - 1], T->v[0]), T->n) / nn;
    img[q] = sub(img[q - 1], scl(T->n, 2.0 * h));
  }
  /* back-trace from the receiver: XR_{m+1} = Rx, reflection point q on its
   * plane toward I_q */
  v3 XR[OR_MAX_REFL + 2];
  XR[m + 1] = rx;
  XR[0] = tx;
  double scale = fmax(maxabs(tx), maxabs(rx));
  double ve = P->val_eps;
  for (int q = m; q >= 1; --q) {
    const otri* T = &S->t[tid[rj[q - 1]]];
    v3 dir = sub(img[q], XR[q + 1]);
    double den = dot(dir, T->n);
    if (den == 0) { out->valid = 0; out->flags = fl; return; }
    double sv = dot(sub(T->v[0], XR[q + 1]), T->n) / den;
    if (fabs(sv) <= ve || fabs(sv - 1.0) <= ve) fl |= ORF_VAL_PARAM;
    if (!(sv > 0 && sv < 1)) { out->valid = 0; out->flags = fl; return; }
    XR[q] = add(XR[q + 1], scl(dir, sv));
    scale = fmax(scale, maxabs(XR[q]));
  }
  /* the interaction points in order: a transmission crosses its triangle's
   * plane on the straight piece between the surrounding reflection points,
   * after the previous interaction of that piece */
  v3 X[OR_MAX_REFL + 2];
  X[0] = tx;
  X[k + 1] = rx;
  {
    int q = 0;
    double s_prev = 0.0;
    for (int j = 0; j < k; ++j) {
      if (!isT[j]) {
        X[j + 1] = XR[++q];
        s_prev = 0.0;
        continue;
      }
      const otri* T = &S->t[tid[j]];
      v3 A = XR[q], B = XR[q + 1], dir = sub(B, A);
      double den = dot(dir, T->n);
      if (den == 0) { out->valid = 0; out->flags = fl; return; }
      double sv = dot(sub(T->v[0], A), T->n) / den;
      if (fabs(sv - s_prev) <= ve || fabs(sv - 1.0) <= ve) fl |= ORF_VAL_PARAM;
      if (!(sv > s_prev && sv < 1)) { out->valid = 0; out->flags = fl; return; }
      X[j + 1] = add(A, scl(dir, sv));
      s_prev = sv;
    }
  }
  int ok = 1;
  for (int j = 1; j <= k; ++j) {
    const otri* T = &S->t[tid[j - 1]];
    double mg = edge_margin(T, X[j]);
    if (mg <= P->val_eps * (scale + 1.0)) fl |= ORF_VAL_EDGE;
    if (!point_in_tri(T, X[j])) ok = 0;
  }
  if (!ok) { out->valid = 0; out->flags = fl; return; }
  /* every sub-segment X_j -> X_{j+1} must be unoccluded */
  double L = 0;
  for (int j = 0; j <= k; ++j) L += norm(sub(X[j + 1], X[j]));
  if (!(L > 0)) { out->valid = 0; out->flags = fl; return; }
  for (int j = 0; check_occ && j <= k; ++j) {
    int ex0 = j >= 1 ? tid[j - 1] : -1;
    int ex1 = j + 1 <= k ? tid[j] : -1;
    if (occluded(S, X[j], X[j + 1], ex0, ex1, P, scale + L, &fl)) ok = 0;
  }
  out->flags = fl;
  if (!ok) { out->valid = 0; return; }
  /* geometry of the valid path */
  out->valid = 1;
  out->len_m = L;
  out->delay_s = L / C0;
  for (int j = 1; j <= k; ++j) {
    out->pts[j - 1][0] = X[j].x; out->pts[j - 1][1] = X[j].y; out->pts[j - 1][2] = X[j].z;
  }
  /* field with vector polarisation */
  v3 u = mk(P->pol[0], P->pol[1], P->pol[2]);
  v3 d0 = unit(sub(X[1], X[0]));
  v3 e0 = pol_dir(u, d0, &fl);
  c3 E = {e0.x, e0.y, e0.z};
  for (int j = 1; j <= k; ++j) {
    const otri* T = &S->t[tid[j - 1]];
    if (isT[j - 1]) {  /* penetration loss (power dB): field times 10^(-L/20) */
      double g = pow(10.0, -P->trans_db[T->mat] / 20.0);
      E.x *= g; E.y *= g; E.z *= g;
      continue;
    }
    v3 din = unit(sub(X[j], X[j - 1]));
    v3 dout = unit(sub(X[j + 1], X[j]));
    v3 nh = T->nh;
    double ct = fabs(dot(din, nh));
    v3 sv = cross(din, nh);
    double sn = norm(sv);
    if (sn < 1e-12) {  /* normal incidence: any unit vector perpendicular to n */
      v3 a = fabs(nh.x) < 0.9 ? mk(1, 0, 0) : mk(0, 1, 0);
      sv = unit(cross(nh, a));
    } else {
      sv = scl(sv, 1.0 / sn);
    }
    v3 pin = cross(sv, din), pout = cross(sv, dout);
    double complex gte, gtm;
    int mi = T->mat;
    if (mi < 0 || mi >= S->nmat) mi = 0;
    fresnel(&S->mats[3 * mi], P->freq_hz, ct, &gte, &gtm);
    double complex es = cdot(E, sv), ep = cdot(E, pin);
    c3 En;
    En.x = gte * es * sv.x + gtm * ep * pout.x;
    En.y = gte * es * sv.y + gtm * ep * pout.y;
    En.z = gte * es * sv.z + gtm * ep * pout.z;
    E = En;
  }
  v3 drx = unit(sub(X[k + 1], X[k]));
  v3 prx = pol_dir(u, scl(drx, -1.0), &fl);
  double lam = C0 / P->freq_hz;
  double kw = 2.0 * M_PI * P->freq_hz / C0;
  double complex a = (lam / (4.0 * M_PI)) * cdot(E, prx) * cexp(-I * kw * L) / L;
  out->amp_re = creal(a);
  out->amp_im = cimag(a);
  out->flags = fl;
}

typedef struct {
  const oscene* S;
  const or_params* P;
  v3 tx;
  const float* rx;
  const int32_t* keys;  /* ncand x (2 + N): rx, depth, ids[N] */
  int stride;
  long ncand;
  opath* out;
  atomic_long next;
} val_job;

static void* val_worker(void* p) {
  val_job* J = (val_job*)p;
  for (;;) {
    long s = atomic_fetch_add(&J->next, 16);
    if (s >= J->ncand) break;
    long e = s + 16 < J->ncand ? s + 16 : J->ncand;
    for (long i = s; i < e; ++i) {
      const int32_t* kk = &J->keys[(size_t)i * J->stride];
      int r = kk[0], depth = kk[1];
      v3 R = mk(J->rx[3 * r], J->rx[3 * r + 1], J->rx[3 * r + 2]);
      validate_one(J->S, J->P, J->tx, R, depth, kk + 2, &J->out[i], 1);
    }
  }
  return NULL;
}

/* keys: ncand rows of (2 + max_refl + max_trans) int32: rx index, depth k
 * (interactions), tri ids (k used; OR_TRANS marks a transmission). */
int or_validate(const float* tris, const int32_t* tri_mat, int32_t ntri, const float* mats,
                int32_t nmat, const float* tx, const float* rx, int32_t nrx,
                const int32_t* keys, int64_t ncand, const or_params* P, opath* out) {
  (void)nrx;
  if (P->max_refl < 0 || P->max_trans < 0 || P->max_refl + P->max_trans > OR_MAX_REFL) return -1;
  oscene S;
  if (scene_load(&S, tris, tri_mat, ntri, mats, nmat)) return -2;
  val_job J;
  J.S = &S; J.P = P; J.tx = mk(tx[0], tx[1], tx[2]); J.rx = rx; J.keys = keys;
  J.stride = 2 + P->max_refl + P->max_trans; J.ncand = ncand; J.out = out;
  atomic_init(&J.next, 0);
  int nt = default_threads(P->nthreads);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
  for (int k = 0; k < nt; ++k) pthread_create(&th[k], NULL, val_worker, &J);
  for (int k = 0; k < nt; ++k) pthread_join(th[k], NULL);
  free(th);
  scene_free(&S);
  return 0;
}

/* Path amplitude of fixed triangle sequences (keys as in or_validate) with
 * FP64 vertices (ntri x 9), materials (nmat x 3), Tx and receivers: the same
 * steps without the occlusion test, for derivatives of the field by central
 * differences over a fixed path topology. */
int or_path_amp_d(const double* tris, const int32_t* tri_mat, int32_t ntri, const double* mats,
                  int32_t nmat, const double* tx, const double* rx, int32_t nrx, const int32_t* keys,
                  int64_t nkeys, const or_params* P, opath* out) {
  if (P->max_refl < 0 || P->max_refl > OR_MAX_REFL) return -1;
  oscene S;
  if (scene_load_any(&S, NULL, tris, tri_mat, ntri, NULL, mats, nmat)) return -2;
  int stride = 2 + P->max_refl;
  for (int64_t i = 0; i < nkeys; ++i) {
    const int32_t* kk = &keys[(size_t)i * stride];
    int r = kk[0];
    if (r < 0 || r >= nrx) { memset(&out[i], 0, sizeof(opath)); continue; }
    v3 R = mk(rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]);
    validate_one(&S, P, mk(tx[0], tx[1], tx[2]), R, kk[1], kk + 2, &out[i], 0);
  }
  scene_free(&S);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* or_diffract: first-order edge diffraction (step 5) with the UTD            */
/* ------------------------------------------------------------------------ */
/* UTD transition function F(x) = 2j sqrt(x) e^{jx} int_{sqrt x}^inf e^{-j t^2} dt
 * (x >= 0). The integral, with t = a + e^{-j pi/4} v, becomes
 * e^{-j pi/4} e^{-j a^2} int_0^inf exp(-2 a e^{j pi/4} v - v^2) dv: a smooth,
 * decaying integrand, integrated by the composite Simpson rule. */
static double complex transition_fn(double x) {
  if (!(x > 0)) return 0.0;
  double a = sqrt(x);
  double complex c = 2.0 * a * cexp(I * M_PI / 4.0);
  double vmax = fmin(9.0, 60.0 / (creal(c) + 1e-300));
  double h = fmin(2e-4, 0.005 / (1.0 + cabs(c)));
  long n = (long)ceil(vmax / h);
  if (n % 2) ++n;
  h = vmax / (double)n;
  double complex sum = 0.0;
  for (long i = 0; i <= n; ++i) {
    double v = i * h;
    double complex f = cexp(-c * v - v * v);
    double w = (i == 0 || i == n) ? 1.0 : ((i % 2) ? 4.0 : 2.0);
    sum += w * f;
  }
  double complex G = cexp(-I * M_PI / 4.0) * cexp(-I * x) * (sum * h / 3.0);
  return 2.0 * I * a * cexp(I * x) * G;
}

void or_transition(double x, double* out2) {
  double complex f = transition_fn(x);
  out2[0] = creal(f);
  out2[1] = cimag(f);
}

/* one cot((pi + s beta)/(2n)) F(k L a^s(beta)) term; a^s(beta) = 2 cos^2((2 n pi N - beta)/2)
 * with N the integer closest to a solution of 2 pi n N - beta = s pi */
static double complex utd_term(double n, double beta, double s, double kL, uint32_t* fl) {
  double N = round((beta + s * M_PI) / (2.0 * M_PI * n));
  double c = cos((2.0 * n * M_PI * N - beta) / 2.0);
  double arg = (M_PI + s * beta) / (2.0 * n);
  double sn = sin(arg);
  if (fabs(sn) < 1e-9) { if (fl) *fl |= ORF_VAL_PARAM; return 0.0; }  /* on a shadow boundary */
  return cos(arg) / sn * transition_fn(kL * 2.0 * c * c);
}

/* Wedge diffraction coefficient: n = exterior angle / pi; phi, phip the
 * receiver and source angles from face 0 through the exterior; beta0 the
 * angle between the incident ray and the edge; L the distance parameter;
 * R0, Rn the reflection factors of faces 0 and n (-1 soft / +1 hard for a
 * perfect conductor, the faces' Fresnel coefficients after Luebbers). */
static double complex utd_coeff(double n, double phi, double phip, double beta0, double L, double k,
                                double complex R0, double complex Rn, uint32_t* fl) {
  double complex pre = -cexp(-I * M_PI / 4.0) / (2.0 * n * sqrt(2.0 * M_PI * k) * sin(beta0));
  double bm = phi - phip, bp = phi + phip, kL = k * L;
  return pre * (utd_term(n, bm, +1.0, kL, fl) + utd_term(n, bm, -1.0, kL, fl) +
                R0 * utd_term(n, bp, -1.0, kL, fl) + Rn * utd_term(n, bp, +1.0, kL, fl));
}

void or_utd(double n, double phi, double phip, double beta0, double L, double k, const double* r0,
            const double* rn, double* out2) {
  double complex d = utd_coeff(n, phi, phip, beta0, L, k, r0[0] + I * r0[1], rn[0] + I * rn[1], NULL);
  out2[0] = creal(d);
  out2[1] = cimag(d);
}

/* Wedges: edges shared by exactly two triangles of the same rigid object
 * (or both static) with identical world vertex coordinates, whose planes
 * differ. Edge list in (lower triangle id, higher triangle id) order; face 0
 * is the lower id. */
typedef struct {
  int ta, tb;       /* faces 0 and n                                   */
  v3 p0, e;         /* edge start and unit direction                   */
  v3 p1;            /* edge end (the input vertex)                     */
  double len;
  v3 t0, y0;        /* in the plane normal to e: face 0's direction and
                       the exterior's positive angular direction        */
  v3 tB;            /* ... and face n's direction                      */
  double n;         /* exterior angle / pi                             */
} owedge;

static int vkey_cmp(const float* a, const float* b) {
  for (int k = 0; k < 3; ++k) if (a[k] != b[k]) return a[k] < b[k] ? -1 : 1;
  return 0;
}

typedef struct { float a[3], b[3]; int tri, obj; } oedge_rec;

static int oedge_cmp(const void* x, const void* y) {
  const oedge_rec* p = (const oedge_rec*)x;
  const oedge_rec* q = (const oedge_rec*)y;
  if (p->obj != q->obj) return p->obj < q->obj ? -1 : 1;
  int c = vkey_cmp(p->a, q->a);
  if (c) return c;
  c = vkey_cmp(p->b, q->b);
  if (c) return c;
  return p->tri < q->tri ? -1 : (p->tri > q->tri);
}

static int wedge_cmp(const void* x, const void* y) {
  const owedge* p = (const owedge*)x;
  const owedge* q = (const owedge*)y;
  if (p->ta != q->ta) return p->ta < q->ta ? -1 : 1;
  return p->tb < q->tb ? -1 : (p->tb > q->tb);
}

static long find_wedges(const float* tris, const int32_t* tri_obj, int ntri, owedge** out) {
  oedge_rec* r = (oedge_rec*)malloc(sizeof(oedge_rec) * (size_t)(3 * ntri + 1));
  long m = 0;
  for (int i = 0; i < ntri; ++i) {
    for (int k = 0; k < 3; ++k) {
      const float* a = &tris[9 * i + 3 * k];
      const float* b = &tris[9 * i + 3 * ((k + 1) % 3)];
      oedge_rec* e = &r[m++];
      if (vkey_cmp(a, b) <= 0) { memcpy(e->a, a, 12); memcpy(e->b, b, 12); }
      else { memcpy(e->a, b, 12); memcpy(e->b, a, 12); }
      e->tri = i;
      e->obj = tri_obj ? tri_obj[i] : -1;
    }
  }
  qsort(r, (size_t)m, sizeof(oedge_rec), oedge_cmp);
  owedge* w = (owedge*)malloc(sizeof(owedge) * (size_t)(m + 1));
  long nw = 0;
  for (long i = 0; i < m;) {
    long j = i + 1;
    while (j < m && r[j].obj == r[i].obj && !vkey_cmp(r[j].a, r[i].a) && !vkey_cmp(r[j].b, r[i].b)) ++j;
    if (j - i == 2) {
      int ta = r[i].tri < r[i + 1].tri ? r[i].tri : r[i + 1].tri;
      int tb = r[i].tri < r[i + 1].tri ? r[i + 1].tri : r[i].tri;
      v3 p0 = mk(r[i].a[0], r[i].a[1], r[i].a[2]), p1 = mk(r[i].b[0], r[i].b[1], r[i].b[2]);
      v3 e = sub(p1, p0);
      double len = norm(e);
      if (len > 0) {
        e = scl(e, 1.0 / len);
        /* third vertices of the two faces, projected normal to the edge */
        v3 third[2];
        int tt[2] = {ta, tb};
        for (int q = 0; q < 2; ++q) {
          third[q] = p0;
          for (int k = 0; k < 3; ++k) {
            const float* v = &tris[9 * tt[q] + 3 * k];
            v3 vv = mk(v[0], v[1], v[2]);
            if (vkey_cmp(v, r[i].a) && vkey_cmp(v, r[i].b)) third[q] = vv;
          }
        }
        v3 da = sub(third[0], p0), db = sub(third[1], p0);
        da = sub(da, scl(e, dot(da, e)));
        db = sub(db, scl(e, dot(db, e)));
        double la = norm(da), lb = norm(db);
        if (la > 0 && lb > 0) {
          v3 t0 = scl(da, 1.0 / la), tB = scl(db, 1.0 / lb);
          v3 y0 = cross(e, t0);
          /* the interior (face n side) is at a positive angle alpha from face 0
           * about +y0; the exterior angles run the other way */
          double alpha = atan2(dot(tB, y0), dot(tB, t0));
          if (alpha < 0) { y0 = scl(y0, -1.0); alpha = -alpha; }
          y0 = scl(y0, -1.0);  /* exterior direction */
          if (fabs(alpha - M_PI) > 1e-6 && alpha > 1e-9) {
            owedge* W = &w[nw++];
            W->ta = ta; W->tb = tb; W->p0 = p0; W->p1 = p1; W->e = e; W->len = len;
            W->t0 = t0; W->y0 = y0; W->tB = tB; W->n = 2.0 - alpha / M_PI;
          }
        }
      }
    }
    i = j;
  }
  free(r);
  qsort(w, (size_t)nw, sizeof(owedge), wedge_cmp);
  *out = w;
  return nw;
}

/* angle of point X about the wedge (from face 0 through the exterior) */
static double wedge_angle(const owedge* W, v3 X) {
  v3 d = sub(X, W->p0);
  d = sub(d, scl(W->e, dot(d, W->e)));
  double a = atan2(dot(d, W->y0), dot(d, W->t0));
  if (a < 0) a += 2.0 * M_PI;
  return a;
}

int32_t or_count_wedges(const float* tris, const int32_t* tri_obj, int32_t ntri) {
  owedge* w = NULL;
  long n = find_wedges(tris, tri_obj, ntri, &w);
  free(w);
  return (int32_t)n;
}

/* First-order diffraction paths for every (receiver, wedge); writes the
 * valid ones (keys: rx, 1, wedge | OR_DIFF; -1 padded to 2 + width) and
 * returns their count (may exceed cap). */
int64_t or_diffract(const float* tris, const int32_t* tri_mat, const int32_t* tri_obj, int32_t ntri,
                    const float* mats, int32_t nmat, const float* tx, const float* rx, int32_t nrx,
                    const or_params* P, int32_t width, int32_t* keys_out, opath* paths_out, int64_t cap) {
  oscene S;
  if (scene_load(&S, tris, tri_mat, ntri, mats, nmat)) return -2;
  owedge* W = NULL;
  long nw = find_wedges(tris, tri_obj, ntri, &W);
  const double k = 2.0 * M_PI * P->freq_hz / C0, lam = C0 / P->freq_hz;
  v3 T = mk(tx[0], tx[1], tx[2]);
  v3 u = mk(P->pol[0], P->pol[1], P->pol[2]);
  int64_t nvalid = 0;
  for (int r = 0; r < nrx; ++r) {
    v3 R = mk(rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]);
    for (long w = 0; w < nw; ++w) {
      const owedge* E = &W[w];
      uint32_t fl = 0;
      /* Keller's law: Q where the unfolded path crosses the edge line */
      v3 dt = sub(T, E->p0), dr = sub(R, E->p0);
      double zt = dot(dt, E->e), zr = dot(dr, E->e);
      double rt = norm(sub(dt, scl(E->e, zt))), rr = norm(sub(dr, scl(E->e, zr)));
      if (!(rt > 0 && rr > 0)) continue;
      double zq = zt + (zr - zt) * rt / (rt + rr);
      double uq = zq / E->len;
      if (fabs(uq) <= P->val_eps || fabs(uq - 1.0) <= P->val_eps) fl |= ORF_VAL_PARAM;
      if (!(uq > 0 && uq < 1)) continue;
      v3 Q = add(E->p0, scl(E->e, zq));
      double phip = wedge_angle(E, T), phi = wedge_angle(E, R), nn = E->n;
      double ang_eps = 1e-9;
      if (phip > nn * M_PI || phi > nn * M_PI) continue;        /* inside the wedge */
      /* the paper's step 5: the source lies in the shadow region seen from
       * the receiver, i.e. the receiver is beyond the incident shadow boundary */
      if (fabs(fabs(phi - phip) - M_PI) <= ang_eps) fl |= ORF_VAL_PARAM;
      if (!(fabs(phi - phip) > M_PI)) continue;
      double scale = fmax(maxabs(T), maxabs(R));
      if (occluded(&S, T, Q, E->ta, E->tb, P, scale, &fl)) continue;
      if (occluded(&S, Q, R, E->ta, E->tb, P, scale, &fl)) continue;
      /* UTD field */
      double sp = norm(sub(Q, T)), s = norm(sub(R, Q));
      v3 ip = scl(sub(Q, T), 1.0 / sp), dd = scl(sub(R, Q), 1.0 / s);
      double cb = dot(ip, E->e);
      double beta0 = acos(fmax(-1.0, fmin(1.0, cb)));
      double L = s * sp * sin(beta0) * sin(beta0) / (s + sp);
      v3 php = cross(E->e, ip), ph = cross(E->e, dd);
      php = scl(php, -1.0 / norm(php));
      ph = scl(ph, 1.0 / norm(ph));
      v3 bp = cross(ip, php), bd = cross(dd, ph);
      /* Luebbers: faces' reflection coefficients at the grazing angles
       * phi' (face 0) and n pi - phi (face n) */
      int ma = S.t[E->ta].mat, mb = S.t[E->tb].mat;
      if (ma < 0 || ma >= S.nmat) ma = 0;
      if (mb < 0 || mb >= S.nmat) mb = 0;
      double complex r0s, r0h, rns, rnh;
      fresnel(&S.mats[3 * ma], P->freq_hz, fabs(sin(phip)), &r0s, &r0h);
      fresnel(&S.mats[3 * mb], P->freq_hz, fabs(sin(nn * M_PI - phi)), &rns, &rnh);
      double complex Ds = utd_coeff(nn, phi, phip, beta0, L, k, r0s, rns, &fl);
      double complex Dh = utd_coeff(nn, phi, phip, beta0, L, k, r0h, rnh, &fl);
      v3 e0 = pol_dir(u, ip, &fl);
      double complex Ei = cexp(-I * k * sp) / sp;
      double complex Eb = Ei * dot(e0, bp), Ep = Ei * dot(e0, php);
      double complex A = csqrt(sp / (s * (s + sp))) * cexp(-I * k * s);
      /* E_d = (-Ds E_beta' beta0^ - Dh E_phi' phi^) A e^{-jks} */
      v3 prx = pol_dir(u, scl(dd, -1.0), &fl);
      double complex proj = (-Ds * Eb) * dot(bd, prx) + (-Dh * Ep) * dot(ph, prx);
      double complex a = (lam / (4.0 * M_PI)) * proj * A;
      if (nvalid < cap) {
        int32_t* kk = &keys_out[(size_t)nvalid * (2 + width)];
        kk[0] = r; kk[1] = 1; kk[2] = (int32_t)w | OR_DIFF;
        for (int j = 1; j < width; ++j) kk[2 + j] = -1;
        opath* o = &paths_out[nvalid];
        memset(o, 0, sizeof(*o));
        o->valid = 1;
        o->flags = fl;
        o->len_m = sp + s;
        o->delay_s = (sp + s) / C0;
        o->amp_re = creal(a);
        o->amp_im = cimag(a);
        o->pts[0][0] = Q.x; o->pts[0][1] = Q.y; o->pts[0][2] = Q.z;
      }
      nvalid++;
    }
  }
  free(W);
  scene_free(&S);
  return nvalid;
}

/* The triangles (other than ex0 .. ex3) that cross the open segment a->b (its
 * first and last eps_occ trimmed), in order along it: their ids in ids[],
 * at most cap. Returns their count, or -1 when one of them is opaque (no
 * penetration loss: trans_db NULL or < 0) or there are more than cap.
 * Decisions within the FP32 margin are flagged as in occluded4. */
static int leg_crossings(const oscene* S, v3 a, v3 b, int ex0, int ex1, int ex2, int ex3, const or_params* P,
                         double scale, uint32_t* fl, int* ids, int cap) {
  v3 dv = sub(b, a);
  double len = norm(dv);
  if (!(len > 0)) return 0;
  v3 d = scl(dv, 1.0 / len);
  double base = P->edge_eps * scale;
  double us[OR_MAX_REFL + 1];
  int n = 0, bad = 0;
  for (int j = 0; j < S->ntri; ++j) {
    if (j == ex0 || j == ex1 || j == ex2 || j == ex3) continue;
    xinfo x;
    ray_tri(&S->t[j], a, d, base, P->edge_eps, &x);
    if (isnan(x.t)) continue;
    double u = x.t / len;
    double du = (base + P->edge_eps * fabs(x.t)) / fmax(x.cos_t, 1e-6) / len;
    double lo = P->eps_occ, hi = 1.0 - P->eps_occ;
    if (x.inside || x.flippable) {
      if (u > lo - du && u < hi + du) {
        if (x.flippable) *fl |= ORF_OCC_NEAR;
        if (fabs(u - lo) <= du || fabs(u - hi) <= du) *fl |= ORF_OCC_NEAR;
      }
    }
    if (!(x.inside && u > lo && u < hi)) continue;
    int m = S->t[j].mat;
    if (!P->trans_db || m < 0 || m >= S->nmat || P->trans_db[m] < 0) { bad = 1; continue; }
    if (n >= cap) { bad = 1; continue; }
    /* insertion in order of the parameter along the leg */
    int q = n++;
    while (q > 0 && us[q - 1] > u) { us[q] = us[q - 1]; ids[q] = ids[q - 1]; --q; }
    us[q] = u;
    ids[q] = j;
  }
  return bad ? -1 : n;
}

/* Sec. III steps 1-5 combined (the runtime comparisons of Sec. IV allow two
 * transmissions and one diffraction per path): first-order diffraction
 * paths Tx -> Q -> Rx whose legs pass straight through penetrable triangles
 * (Table II losses), at least one and at most max_trans in all. Q, the
 * rules and the UTD field are or_diffract's; each crossing multiplies the
 * field by 10^(-L/20), L its material's penetration loss in dB. Keys (rx,
 * depth, ids): the crossings of the first leg in order from the
 * transmitter (| OR_TRANS), the wedge (| OR_DIFF), then those of the second
 * leg in order from Q; -1 padded to 2 + width. Points in path order. Paths
 * with no crossing are or_diffract's and are not written here. Returns the
 * count (may exceed cap). */
int64_t or_diffract_trans(const float* tris, const int32_t* tri_mat, const int32_t* tri_obj, int32_t ntri,
                          const float* mats, int32_t nmat, const float* tx, const float* rx, int32_t nrx,
                          const or_params* P, int32_t width, int32_t* keys_out, opath* paths_out, int64_t cap) {
  if (!P->trans_db || P->max_trans < 1) return 0;
  oscene S;
  if (scene_load(&S, tris, tri_mat, ntri, mats, nmat)) return -2;
  owedge* W = NULL;
  long nw = find_wedges(tris, tri_obj, ntri, &W);
  const double k = 2.0 * M_PI * P->freq_hz / C0, lam = C0 / P->freq_hz;
  v3 T = mk(tx[0], tx[1], tx[2]);
  v3 u = mk(P->pol[0], P->pol[1], P->pol[2]);
  const int mt = P->max_trans < OR_MAX_REFL - 1 ? P->max_trans : OR_MAX_REFL - 1;
  int64_t nvalid = 0;
  for (int r = 0; r < nrx; ++r) {
    v3 R = mk(rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]);
    for (long w = 0; w < nw; ++w) {
      const owedge* E = &W[w];
      uint32_t fl = 0;
      v3 dt = sub(T, E->p0), dr = sub(R, E->p0);
      double zt = dot(dt, E->e), zr = dot(dr, E->e);
      double rt = norm(sub(dt, scl(E->e, zt))), rr = norm(sub(dr, scl(E->e, zr)));
      if (!(rt > 0 && rr > 0)) continue;
      double zq = zt + (zr - zt) * rt / (rt + rr);
      double uq = zq / E->len;
      if (fabs(uq) <= P->val_eps || fabs(uq - 1.0) <= P->val_eps) fl |= ORF_VAL_PARAM;
      if (!(uq > 0 && uq < 1)) continue;
      v3 Q = add(E->p0, scl(E->e, zq));
      double phip = wedge_angle(E, T), phi = wedge_angle(E, R), nn = E->n;
      if (phip > nn * M_PI || phi > nn * M_PI) continue;
      if (fabs(fabs(phi - phip) - M_PI) <= 1e-9) fl |= ORF_VAL_PARAM;
      if (!(fabs(phi - phip) > M_PI)) continue;
      double scale = fmax(maxabs(T), maxabs(R));
      int c1[OR_MAX_REFL], c2[OR_MAX_REFL];
      int n1 = leg_crossings(&S, T, Q, E->ta, E->tb, E->tb, E->tb, P, scale, &fl, c1, mt);
      if (n1 < 0) continue;
      int n2 = leg_crossings(&S, Q, R, E->ta, E->tb, E->tb, E->tb, P, scale, &fl, c2, mt);
      if (n2 < 0 || n1 + n2 < 1 || n1 + n2 > mt) continue;
      /* UTD field as or_diffract */
      double sp = norm(sub(Q, T)), s = norm(sub(R, Q));
      v3 ip = scl(sub(Q, T), 1.0 / sp), dd = scl(sub(R, Q), 1.0 / s);
      double cb = dot(ip, E->e);
      double beta0 = acos(fmax(-1.0, fmin(1.0, cb)));
      double L = s * sp * sin(beta0) * sin(beta0) / (s + sp);
      v3 php = cross(E->e, ip), ph = cross(E->e, dd);
      php = scl(php, -1.0 / norm(php));
      ph = scl(ph, 1.0 / norm(ph));
      v3 bp = cross(ip, php), bd = cross(dd, ph);
      int ma = S.t[E->ta].mat, mb = S.t[E->tb].mat;
      if (ma < 0 || ma >= S.nmat) ma = 0;
      if (mb < 0 || mb >= S.nmat) mb = 0;
      double complex r0s, r0h, rns, rnh;
      fresnel(&S.mats[3 * ma], P->freq_hz, fabs(sin(phip)), &r0s, &r0h);
      fresnel(&S.mats[3 * mb], P->freq_hz, fabs(sin(nn * M_PI - phi)), &rns, &rnh);
      double complex Ds = utd_coeff(nn, phi, phip, beta0, L, k, r0s, rns, &fl);
      double complex Dh = utd_coeff(nn, phi, phip, beta0, L, k, r0h, rnh, &fl);
      v3 e0 = pol_dir(u, ip, &fl);
      double complex Ei = cexp(-I * k * sp) / sp;
      double complex Eb = Ei * dot(e0, bp), Ep = Ei * dot(e0, php);
      double complex A = csqrt(sp / (s * (s + sp))) * cexp(-I * k * s);
      v3 prx = pol_dir(u, scl(dd, -1.0), &fl);
      double complex proj = (-Ds * Eb) * dot(bd, prx) + (-Dh * Ep) * dot(ph, prx);
      /* the penetration losses of the crossings (power dB: field 10^(-L/20)) */
      double g = 1.0;
      for (int i = 0; i < n1; ++i) g *= pow(10.0, -P->trans_db[S.t[c1[i]].mat] / 20.0);
      for (int i = 0; i < n2; ++i) g *= pow(10.0, -P->trans_db[S.t[c2[i]].mat] / 20.0);
      double complex a = (lam / (4.0 * M_PI)) * proj * A * g;
      const int depth = n1 + 1 + n2;
      if (nvalid < cap && depth <= width) {
        int32_t* kk = &keys_out[(size_t)nvalid * (2 + width)];
        kk[0] = r;
        kk[1] = depth;
        int q = 0;
        for (int i = 0; i < n1; ++i) kk[2 + q++] = c1[i] | OR_TRANS;
        kk[2 + q++] = (int32_t)w | OR_DIFF;
        for (int i = 0; i < n2; ++i) kk[2 + q++] = c2[i] | OR_TRANS;
        for (; q < width; ++q) kk[2 + q] = -1;
        opath* o = &paths_out[nvalid];
        memset(o, 0, sizeof(*o));
        o->valid = 1;
        o->flags = fl;
        o->len_m = sp + s;
        o->delay_s = (sp + s) / C0;
        o->amp_re = creal(a);
        o->amp_im = cimag(a);
        /* points in path order: the crossings, Q, the crossings after it */
        int pq = 0;
        v3 d1 = sub(Q, T), d2 = sub(R, Q);
        for (int i = 0; i < n1; ++i, ++pq) {
          const otri* Tc = &S.t[c1[i]];
          double tt = dot(sub(Tc->v[0], T), Tc->n) / dot(d1, Tc->n);
          v3 X = add(T, scl(d1, tt));
          o->pts[pq][0] = X.x; o->pts[pq][1] = X.y; o->pts[pq][2] = X.z;
        }
        o->pts[pq][0] = Q.x; o->pts[pq][1] = Q.y; o->pts[pq][2] = Q.z;
        ++pq;
        for (int i = 0; i < n2; ++i, ++pq) {
          const otri* Tc = &S.t[c2[i]];
          double tt = dot(sub(Tc->v[0], Q), Tc->n) / dot(d2, Tc->n);
          v3 X = add(Q, scl(d2, tt));
          o->pts[pq][0] = X.x; o->pts[pq][1] = X.y; o->pts[pq][2] = X.z;
        }
      }
      nvalid++;
    }
  }
  free(W);
  scene_free(&S);
  return nvalid;
}

/* Sec. III steps 3-5 combined: one reflection on a static triangle j before
 * or after a first-order diffraction at wedge w. By image theory the path
 * Tx -> P -> Q -> Rx (reflection first) is the diffraction of the
 * transmitter's image T' in j's plane, and Tx -> Q -> P -> Rx (reflection
 * last) the diffraction toward the receiver's image R'; Q follows Keller's
 * law for that pair, P is where the unfolded leg crosses the plane. The path
 * is kept when Q lies inside the edge, P inside j, the receiver (or its
 * image) beyond the incident shadow boundary of the source (or its image),
 * and the three legs unoccluded. Field: the UTD coefficient (as or_diffract)
 * with the image's distances (spreading and phase over the unfolded length)
 * and the Fresnel reflection at P in the bounce basis of validate_one.
 * Keys: rx, 2, then j, w | OR_DIFF (reflection first) or w | OR_DIFF, j;
 * -1 padded to 2 + width. Returns the number of valid paths (may exceed
 * cap). */
int64_t or_diffract_refl(const float* tris, const int32_t* tri_mat, const int32_t* tri_obj, int32_t ntri,
                         const float* mats, int32_t nmat, const float* tx, const float* rx, int32_t nrx,
                         const or_params* P, int32_t width, int32_t* keys_out, opath* paths_out, int64_t cap) {
  if (width < 2) return -1;
  oscene S;
  if (scene_load(&S, tris, tri_mat, ntri, mats, nmat)) return -2;
  owedge* W = NULL;
  long nw = find_wedges(tris, tri_obj, ntri, &W);
  const double k = 2.0 * M_PI * P->freq_hz / C0, lam = C0 / P->freq_hz;
  v3 T = mk(tx[0], tx[1], tx[2]);
  v3 u = mk(P->pol[0], P->pol[1], P->pol[2]);
  int64_t nvalid = 0;
  for (int r = 0; r < nrx; ++r) {
    v3 R = mk(rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]);
    for (long w = 0; w < nw; ++w) {
      const owedge* E = &W[w];
      for (int j = 0; j < ntri; ++j) {
        if ((tri_obj && tri_obj[j] >= 0) || j == E->ta || j == E->tb) continue;
        const otri* Tj = &S.t[j];
        double cpl = dot(Tj->nh, Tj->v[0]);
        for (int first = 1; first >= 0; --first) {  /* 1: reflection before the wedge */
          uint32_t fl = 0;
          v3 src = T, obs = R;
          if (first) src = sub(T, scl(Tj->nh, 2.0 * (dot(Tj->nh, T) - cpl)));
          else obs = sub(R, scl(Tj->nh, 2.0 * (dot(Tj->nh, R) - cpl)));
          /* Keller's law for (src, obs) */
          v3 dt = sub(src, E->p0), dr = sub(obs, E->p0);
          double zt = dot(dt, E->e), zr = dot(dr, E->e);
          double rt = norm(sub(dt, scl(E->e, zt))), rr = norm(sub(dr, scl(E->e, zr)));
          if (!(rt > 0 && rr > 0)) continue;
          double zq = zt + (zr - zt) * rt / (rt + rr);
          double uq = zq / E->len;
          if (fabs(uq) <= P->val_eps || fabs(uq - 1.0) <= P->val_eps) fl |= ORF_VAL_PARAM;
          if (!(uq > 0 && uq < 1)) continue;
          v3 Q = add(E->p0, scl(E->e, zq));
          double phip = wedge_angle(E, src), phi = wedge_angle(E, obs), nn = E->n;
          if (phip > nn * M_PI || phi > nn * M_PI) continue;
          if (fabs(fabs(phi - phip) - M_PI) <= 1e-9) fl |= ORF_VAL_PARAM;
          if (!(fabs(phi - phip) > M_PI)) continue;
          /* the reflection point on the unfolded leg src -> Q or Q -> obs */
          v3 a0 = first ? src : Q, a1 = first ? Q : obs;
          double den = dot(Tj->nh, sub(a1, a0));
          if (den == 0.0) continue;
          double sp_ = (cpl - dot(Tj->nh, a0)) / den;
          if (fabs(sp_) <= P->val_eps || fabs(sp_ - 1.0) <= P->val_eps) fl |= ORF_VAL_PARAM;
          if (!(sp_ > 0 && sp_ < 1)) continue;
          v3 Pp = add(a0, scl(sub(a1, a0), sp_));
          double scale = fmax(maxabs(T), maxabs(R));
          if (edge_margin(Tj, Pp) <= P->val_eps * (scale + 1.0)) fl |= ORF_VAL_EDGE;
          if (!point_in_tri(Tj, Pp)) continue;
          /* the three legs */
          if (first) {
            if (occluded3(&S, T, Pp, j, j, j, P, scale, &fl)) continue;
            if (occluded3(&S, Pp, Q, j, E->ta, E->tb, P, scale, &fl)) continue;
            if (occluded3(&S, Q, R, E->ta, E->tb, E->tb, P, scale, &fl)) continue;
          } else {
            if (occluded3(&S, T, Q, E->ta, E->tb, E->tb, P, scale, &fl)) continue;
            if (occluded3(&S, Q, Pp, j, E->ta, E->tb, P, scale, &fl)) continue;
            if (occluded3(&S, Pp, R, j, j, j, P, scale, &fl)) continue;
          }
          /* UTD with the image's geometry */
          double sp = norm(sub(Q, src)), sd = norm(sub(obs, Q));
          v3 ip = scl(sub(Q, src), 1.0 / sp), dd = scl(sub(obs, Q), 1.0 / sd);
          double beta0 = acos(fmax(-1.0, fmin(1.0, dot(ip, E->e))));
          double Ld = sd * sp * sin(beta0) * sin(beta0) / (sd + sp);
          v3 php = cross(E->e, ip), ph = cross(E->e, dd);
          php = scl(php, -1.0 / norm(php));
          ph = scl(ph, 1.0 / norm(ph));
          v3 bp = cross(ip, php), bd = cross(dd, ph);
          int ma = S.t[E->ta].mat, mb = S.t[E->tb].mat;
          if (ma < 0 || ma >= S.nmat) ma = 0;
          if (mb < 0 || mb >= S.nmat) mb = 0;
          double complex r0s, r0h, rns, rnh;
          fresnel(&S.mats[3 * ma], P->freq_hz, fabs(sin(phip)), &r0s, &r0h);
          fresnel(&S.mats[3 * mb], P->freq_hz, fabs(sin(nn * M_PI - phi)), &rns, &rnh);
          double complex Ds = utd_coeff(nn, phi, phip, beta0, Ld, k, r0s, rns, &fl);
          double complex Dh = utd_coeff(nn, phi, phip, beta0, Ld, k, r0h, rnh, &fl);
          /* the reflection at P: incoming and outgoing directions, bounce basis */
          v3 din = first ? unit(sub(Pp, T)) : dd;
          v3 dout = first ? ip : unit(sub(R, Pp));
          v3 nh = Tj->nh;
          double ct = fabs(dot(din, nh));
          v3 sv = cross(din, nh);
          double sn = norm(sv);
          if (sn < 1e-12) {
            v3 ax = fabs(nh.x) < 0.9 ? mk(1, 0, 0) : mk(0, 1, 0);
            sv = unit(cross(nh, ax));
          } else {
            sv = scl(sv, 1.0 / sn);
          }
          v3 pin = cross(sv, din), pout = cross(sv, dout);
          int mj = Tj->mat;
          if (mj < 0 || mj >= S.nmat) mj = 0;
          double complex gte, gtm;
          fresnel(&S.mats[3 * mj], P->freq_hz, ct, &gte, &gtm);
          double complex A = csqrt(sp / (sd * (sd + sp))) * cexp(-I * k * sd);
          double complex a;
          if (first) {
            /* Tx field along T -> P, reflected at P, arrives at Q from T' */
            v3 e0 = pol_dir(u, din, &fl);
            double complex es = dot(e0, sv), ep = dot(e0, pin);
            c3 E1;
            E1.x = gte * es * sv.x + gtm * ep * pout.x;
            E1.y = gte * es * sv.y + gtm * ep * pout.y;
            E1.z = gte * es * sv.z + gtm * ep * pout.z;
            double complex Ei = cexp(-I * k * sp) / sp;
            double complex Eb = Ei * cdot(E1, bp), Ep = Ei * cdot(E1, php);
            v3 prx = pol_dir(u, scl(dd, -1.0), &fl);
            double complex proj = (-Ds * Eb) * dot(bd, prx) + (-Dh * Ep) * dot(ph, prx);
            a = (lam / (4.0 * M_PI)) * proj * A;
          } else {
            /* diffracted field toward R', reflected at P */
            v3 e0 = pol_dir(u, ip, &fl);
            double complex Ei = cexp(-I * k * sp) / sp;
            double complex Eb = Ei * dot(e0, bp), Ep = Ei * dot(e0, php);
            c3 Ed;
            Ed.x = (-Ds * Eb) * bd.x + (-Dh * Ep) * ph.x;
            Ed.y = (-Ds * Eb) * bd.y + (-Dh * Ep) * ph.y;
            Ed.z = (-Ds * Eb) * bd.z + (-Dh * Ep) * ph.z;
            double complex es = cdot(Ed, sv), ep = cdot(Ed, pin);
            c3 E2;
            E2.x = gte * es * sv.x + gtm * ep * pout.x;
            E2.y = gte * es * sv.y + gtm * ep * pout.y;
            E2.z = gte * es * sv.z + gtm * ep * pout.z;
            v3 prx = pol_dir(u, scl(dout, -1.0), &fl);
            a = (lam / (4.0 * M_PI)) * cdot(E2, prx) * A;
          }
          if (nvalid < cap) {
            int32_t* kk = &keys_out[(size_t)nvalid * (2 + width)];
            kk[0] = r;
            kk[1] = 2;
            kk[2] = first ? j : ((int32_t)w | OR_DIFF);
            kk[3] = first ? ((int32_t)w | OR_DIFF) : j;
            for (int q = 2; q < width; ++q) kk[2 + q] = -1;
            opath* o = &paths_out[nvalid];
            memset(o, 0, sizeof(*o));
            o->valid = 1;
            o->flags = fl;
            o->len_m = sp + sd;
            o->delay_s = (sp + sd) / C0;
            o->amp_re = creal(a);
            o->amp_im = cimag(a);
            v3 p1 = first ? Pp : Q, p2 = first ? Q : Pp;
            o->pts[0][0] = p1.x; o->pts[0][1] = p1.y; o->pts[0][2] = p1.z;
            o->pts[1][0] = p2.x; o->pts[1][1] = p2.y; o->pts[1][2] = p2.z;
          }
          nvalid++;
        }
      }
    }
  }
  free(W);
  scene_free(&S);
  return nvalid;
}

/* ------------------------------------------------------------------------ */
/* Diffraction of order 2 and 3 (Sec. III step 5; the paper's bound is 3)    */
/* ------------------------------------------------------------------------ */
#define OR_LEG_MIN 1e-6  /* shortest leg of a diffraction chain while its Keller points are sought [m] */

/* Do two edges share an end vertex (identical input coordinates)? Consecutive
 * wedges of a chain may not (which includes sharing a face): the length's
 * minimum then tends to the common corner (a vertex, not an edge, would
 * diffract), or the leg between them runs along a face they bound. */
static int share_vertex(const owedge* A, const owedge* B) {
  const v3* a[2] = {&A->p0, &A->p1};
  const v3* b[2] = {&B->p0, &B->p1};
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      if (a[i]->x == b[j]->x && a[i]->y == b[j]->y && a[i]->z == b[j]->z) return 1;
  return 0;
}

/* Do two edges lie on one line (directions parallel to 1e-9, the second's
 * start within 1e-9 m (relative to the coordinates' size) of the first's
 * line)? Consecutive wedges of a chain may not: the leg between them would
 * run along both edges, and the unfolded length has its minimum where that
 * leg vanishes (no Keller points). */
static int collinear_edges(const owedge* A, const owedge* B) {
  if (norm(cross(A->e, B->e)) > 1e-9) return 0;
  v3 d = sub(B->p0, A->p0);
  return norm(cross(d, A->e)) <= 1e-9 * (1.0 + maxabs(A->p0) + maxabs(B->p0));
}

/* Does edge B lie in the plane of a face of wedge A (both its ends within
 * 1e-9 m, relative to the coordinates' size, of the plane)? Then so does the
 * leg between them, and at A its direction is that face's (grazing), or the
 * face's extension beyond the edge, where no source in A's exterior has its
 * shadow boundary crossed: no chain passes. */
static int in_face_plane(const owedge* A, const owedge* B) {
  double tol = 1e-9 * (1.0 + maxabs(A->p0) + maxabs(B->p0));
  v3 f[2] = {cross(A->e, A->t0), cross(A->e, A->tB)};
  for (int q = 0; q < 2; ++q)
    if (fabs(dot(f[q], sub(B->p0, A->p0))) <= tol && fabs(dot(f[q], sub(B->p1, A->p0))) <= tol) return 1;
  return 0;
}

/* Unfolded length of T -> Q_1 .. Q_m -> R with Q_i = p0_i + t_i e_i. */
static double chain_length(const owedge* const* E, int m, v3 T, v3 R, const double* t) {
  v3 prev = T;
  double L = 0.0;
  for (int i = 0; i < m; ++i) {
    v3 q = add(E[i]->p0, scl(E[i]->e, t[i]));
    L += norm(sub(q, prev));
    prev = q;
  }
  return L + norm(sub(R, prev));
}

/* Solves the m x m system H x = b (m <= 3) by Gaussian elimination with
 * partial pivoting; 0 when H is singular. */
static int solve_small(int m, double H[3][3], double* b, double* x) {
  double A[3][4];
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) A[i][j] = H[i][j];
    A[i][m] = b[i];
  }
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r) if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    if (!(fabs(A[piv][c]) > 1e-300)) return 0;
    if (piv != c) for (int j = 0; j <= m; ++j) { double tmp = A[c][j]; A[c][j] = A[piv][j]; A[piv][j] = tmp; }
    for (int r = c + 1; r < m; ++r) {
      double f = A[r][c] / A[c][c];
      for (int j = c; j <= m; ++j) A[r][j] -= f * A[c][j];
    }
  }
  for (int i = m - 1; i >= 0; --i) {
    double v = A[i][m];
    for (int j = i + 1; j < m; ++j) v -= A[i][j] * x[j];
    x[i] = v / A[i][i];
  }
  return 1;
}

/* Keller points of a chain of m wedges: the edge parameters t that make the
 * unfolded length stationary, i.e. at every edge the incident and the
 * diffracted leg make the same angle with the edge (Keller's law). The
 * length is a convex function of t (a sum of distances between points
 * moving linearly with t), so its stationary point is its minimum; it is
 * found by Newton's method from the edges' midpoints (at most 50 steps),
 * halving a step that does not shorten the chain (at most 40 times) until
 * the cosine mismatch is below 1e-8 or the Newton decrement below 1e-15 of
 * the length, full steps after that.
 * Returns 1 when converged (every edge's cosine mismatch below 1e-12); 0
 * when not, or when a leg shrinks below OR_LEG_MIN: the minimum is then at
 * a kink of the length (two consecutive edge lines meet), where Keller's
 * law has no solution. */
static int keller_points(const owedge* const* E, int m, v3 T, v3 R, double* t) {
  for (int i = 0; i < m; ++i) t[i] = 0.5 * E[i]->len;
  double Lc = chain_length(E, m, T, R, t);
  for (int it = 0; it < 50; ++it) {
    v3 X[OR_MAX_REFL + 2];
    X[0] = T;
    for (int i = 0; i < m; ++i) X[i + 1] = add(E[i]->p0, scl(E[i]->e, t[i]));
    X[m + 1] = R;
    double g[3] = {0, 0, 0}, H[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int j = 0; j <= m; ++j) {  /* leg j: X[j] -> X[j+1]; moves with t[j-1] and t[j] */
      v3 d = sub(X[j + 1], X[j]);
      double l = norm(d);
      if (!(l > OR_LEG_MIN)) return 0;
      v3 u = scl(d, 1.0 / l);
      int a = j - 1, b = j;
      double ca = a >= 0 ? dot(E[a]->e, u) : 0.0, cb = b < m ? dot(E[b]->e, u) : 0.0;
      if (b < m) { g[b] += cb; H[b][b] += (1.0 - cb * cb) / l; }
      if (a >= 0) { g[a] -= ca; H[a][a] += (1.0 - ca * ca) / l; }
      if (a >= 0 && b < m) {
        double h = -(dot(E[a]->e, E[b]->e) - ca * cb) / l;
        H[a][b] += h;
        H[b][a] += h;
      }
    }
    double gmax = 0.0;
    for (int i = 0; i < m; ++i) gmax = fmax(gmax, fabs(g[i]));
    if (gmax < 1e-12) return 1;
    double mg[3] = {-g[0], -g[1], -g[2]}, dx[3];
    if (!solve_small(m, H, mg, dx)) return 0;
    /* near the minimum the full Newton step is taken: the length it saves
     * (the Newton decrement, -g.dx / 2) is below the length's own rounding
     * there, so comparing lengths cannot judge it -- a mismatch below 1e-8,
     * or a decrement below 1e-15 of the length (long chains reach that floor
     * at larger mismatches) */
    double gdx = 0.0;
    for (int i = 0; i < m; ++i) gdx += g[i] * dx[i];
    int at_floor = gmax < 1e-8 || fabs(gdx) <= 2e-15 * Lc;
    double step = 1.0, tn[3];
    for (int k = 0; k < 40; ++k) {
      for (int i = 0; i < m; ++i) tn[i] = t[i] + step * dx[i];
      double Ln = chain_length(E, m, T, R, tn);
      if (Ln <= Lc || at_floor) { Lc = Ln; break; }
      step *= 0.5;
    }
    double dmax = 0.0;
    for (int i = 0; i < m; ++i) { dmax = fmax(dmax, fabs(tn[i] - t[i])); t[i] = tn[i]; }
    if (dmax == 0.0) return gmax < 1e-9;
  }
  return 0;
}

/* Keller points of a chain of m (1..3) edges from T to R, each edge a row
 * of 7 doubles (start, unit direction, length): keller_points on them.
 * Returns 1 when it converged, with the edge parameters in t[0 .. m-1]
 * (test infrastructure: lets pins check the solver alone). */
int or_keller_points(int32_t m, const double* edges, const double* T, const double* R, double* t) {
  if (m < 1 || m > 3) return 0;
  owedge W[3];
  const owedge* E[3];
  for (int i = 0; i < m; ++i) {
    const double* r = edges + 7 * i;
    memset(&W[i], 0, sizeof W[i]);
    W[i].p0 = mk(r[0], r[1], r[2]);
    W[i].e = mk(r[3], r[4], r[5]);
    W[i].len = r[6];
    W[i].p1 = add(W[i].p0, scl(W[i].e, W[i].len));
    E[i] = &W[i];
  }
  return keller_points(E, m, mk(T[0], T[1], T[2]), mk(R[0], R[1], R[2]), t);
}

/* The specular reflection of field E at triangle Tj for incoming direction
 * din and outgoing dout: Fresnel TE / TM of Tj's material in the bounce
 * basis of validate_one (s = din x n, p_in = s x din, p_out = s x dout). */
static c3 reflect_field(const oscene* S, const or_params* P, const otri* Tj, v3 din, v3 dout, c3 E) {
  v3 nh = Tj->nh;
  double ct = fabs(dot(din, nh));
  v3 sv = cross(din, nh);
  double sn = norm(sv);
  if (sn < 1e-12) {
    v3 ax = fabs(nh.x) < 0.9 ? mk(1, 0, 0) : mk(0, 1, 0);
    sv = unit(cross(nh, ax));
  } else {
    sv = scl(sv, 1.0 / sn);
  }
  v3 pin = cross(sv, din), pout = cross(sv, dout);
  int mj = Tj->mat;
  if (mj < 0 || mj >= S->nmat) mj = 0;
  double complex gte, gtm;
  fresnel(&S->mats[3 * mj], P->freq_hz, ct, &gte, &gtm);
  double complex es = cdot(E, sv), ep = cdot(E, pin);
  c3 out;
  out.x = gte * es * sv.x + gtm * ep * pout.x;
  out.y = gte * es * sv.y + gtm * ep * pout.y;
  out.z = gte * es * sv.z + gtm * ep * pout.z;
  return out;
}

static inline c3 mk3c(v3 v) {
  c3 c = {v.x, v.y, v.z};
  return c;
}

/* The chain rules of a wedge sequence w[0..m-1]: pairwise distinct, and
 * consecutive wedges share no vertex (share_vertex), do not lie on one line
 * (collinear_edges), and neither edge lies in a face plane of the other
 * (in_face_plane). */
static int chain_allowed(const owedge* W, const long* w, int m) {
  int ok = w[0] != w[1] && (m < 3 || (w[2] != w[0] && w[2] != w[1]));
  for (int i = 0; ok && i + 1 < m; ++i) {
    const owedge *A = &W[w[i]], *B = &W[w[i + 1]];
    if (share_vertex(A, B) || collinear_edges(A, B) || in_face_plane(A, B) || in_face_plane(B, A)) ok = 0;
  }
  return ok;
}

/* The point where the segment a -> b crosses the plane of triangle Tj
 * (parameter strictly inside (0, 1), flagged within val_eps of an end), inside
 * the triangle (flagged within val_eps of its border). Returns 0 when the
 * segment misses the triangle. */
static int mirror_point(const otri* Tj, v3 a, v3 b, const or_params* P, double scale, uint32_t* fl, v3* X) {
  double cpl = dot(Tj->nh, Tj->v[0]);
  double den = dot(Tj->nh, sub(b, a));
  if (den == 0.0) return 0;
  double sp_ = (cpl - dot(Tj->nh, a)) / den;
  if (fabs(sp_) <= P->val_eps || fabs(sp_ - 1.0) <= P->val_eps) *fl |= ORF_VAL_PARAM;
  if (!(sp_ > 0 && sp_ < 1)) return 0;
  *X = add(a, scl(sub(b, a), sp_));
  if (edge_margin(Tj, *X) <= P->val_eps * (scale + 1.0)) *fl |= ORF_VAL_EDGE;
  return point_in_tri(Tj, *X);
}

static v3 mirror_in(const otri* Tj, v3 x) {
  double cpl = dot(Tj->nh, Tj->v[0]);
  return sub(x, scl(Tj->nh, 2.0 * (dot(Tj->nh, x) - cpl)));
}

/* One diffraction chain over the wedges E[0..m-1] (m = 1..3) from T to R,
 * with specular reflections on the static triangles jb[0..nb-1] before the
 * first wedge and ja[0..na-1] after the last (both in path order, nb + na <=
 * 2). By image theory the chain is solved between the source, the
 * transmitter's image in the planes of jb[0], jb[1], .. in turn, and the
 * observer, the receiver's image in the planes of ja[na-1], .., ja[0]. The
 * reflection points follow by unfolding back: the last one before the chain
 * is where the leg from the source to Q_1 crosses its plane, the one before
 * it where the leg from the previous image to that point crosses its plane,
 * and the same after the chain from Q_m outward; each must lie strictly
 * inside its leg and inside its triangle. Every rule of or_diffract_multi
 * applies to the unfolded chain (the angles about an edge are those of the
 * real points: the real and the unfolded leg lie on one line through Q); the
 * real legs are unoccluded (the triangle excluded at a reflection point, the
 * wedge's faces at a diffraction point). Field: the transmitter's wave along
 * its real first leg, the Fresnel coefficients of each reflection's material
 * in the bounce basis of the real directions (validate_one's), the UTD chain
 * of or_diffract_multi over the unfolded distances (a plane mirror keeps the
 * wavefront's radii of curvature). Returns 1 when the path is valid, with o
 * filled (points in path order). */
/* Crossings of a path's real legs by transmitting triangles (chain_path_r
 * with a record: instead of unoccluded legs, legs that cross transmitting
 * triangles only, at most cap in all): per leg their count, and their ids
 * in path order. */
typedef struct {
  int cap;
  int total;
  int n[OR_MAX_REFL + 2];
  int id[OR_MAX_REFL];
} ocross;

static int chain_path_r(const oscene* S, const owedge* const* E, int m, v3 T, v3 R, const int* jb, int nb,
                        const int* ja, int na, const or_params* P, opath* o, ocross* cr) {
  const double k = 2.0 * M_PI * P->freq_hz / C0, lam = C0 / P->freq_hz;
  const double ang_eps = 1e-9;
  const v3 u = mk(P->pol[0], P->pol[1], P->pol[2]);
  uint32_t fl = 0;
  v3 Simg[3], Oimg[3];
  Simg[0] = T;
  for (int i = 0; i < nb; ++i) Simg[i + 1] = mirror_in(&S->t[jb[i]], Simg[i]);
  Oimg[na] = R;
  for (int i = na - 1; i >= 0; --i) Oimg[i] = mirror_in(&S->t[ja[i]], Oimg[i + 1]);
  const v3 src = Simg[nb], obs = Oimg[0];
  /* the source outside the first wedge, the observer outside the last (the
   * angles about an edge do not depend on the Keller points; the same tests
   * are repeated below with the others) */
  if (wedge_angle(E[0], src) > E[0]->n * M_PI || wedge_angle(E[m - 1], obs) > E[m - 1]->n * M_PI) return 0;
  double t[3];
  if (!keller_points(E, m, src, obs, t)) return 0;
  v3 X[5];
  X[0] = src;
  for (int i = 0; i < m; ++i) X[i + 1] = add(E[i]->p0, scl(E[i]->e, t[i]));
  X[m + 1] = obs;
  for (int i = 0; i < m; ++i) {
    double uq = t[i] / E[i]->len;
    if (fabs(uq) <= P->val_eps || fabs(uq - 1.0) <= P->val_eps) fl |= ORF_VAL_PARAM;
    if (!(uq > 0 && uq < 1)) return 0;
  }
  double ell[4];
  for (int q = 0; q <= m; ++q) {
    ell[q] = norm(sub(X[q + 1], X[q]));
    if (!(ell[q] > 1e-9)) return 0;
  }
  /* exterior and shadow rule at every wedge */
  double phip[3], phi[3];
  for (int i = 0; i < m; ++i) {
    phip[i] = wedge_angle(E[i], X[i]);
    phi[i] = wedge_angle(E[i], X[i + 2]);
    double nn = E[i]->n;
    if (phip[i] > nn * M_PI || phi[i] > nn * M_PI) return 0;
    if (fabs(fabs(phi[i] - phip[i]) - M_PI) <= ang_eps) fl |= ORF_VAL_PARAM;
    if (!(fabs(phi[i] - phip[i]) > M_PI)) return 0;
  }
  double scale = fmax(maxabs(T), maxabs(R));
  /* the reflection points, unfolded back from the chain's ends */
  v3 Yb[2], Ya[2];
  v3 b = X[1];
  for (int i = nb - 1; i >= 0; --i) {
    if (!mirror_point(&S->t[jb[i]], Simg[i + 1], b, P, scale, &fl, &Yb[i])) return 0;
    b = Yb[i];
  }
  v3 a0 = X[m];
  for (int i = 0; i < na; ++i) {
    if (!mirror_point(&S->t[ja[i]], a0, Oimg[i], P, scale, &fl, &Ya[i])) return 0;
    a0 = Ya[i];
  }
  /* the real legs: Y[] the path's points, ex[] two excluded triangles each */
  v3 Y[8];
  int ex[8][2], ny = 0;
  Y[ny] = T; ex[ny][0] = ex[ny][1] = -1; ++ny;
  for (int i = 0; i < nb; ++i) { Y[ny] = Yb[i]; ex[ny][0] = ex[ny][1] = jb[i]; ++ny; }
  for (int i = 0; i < m; ++i) { Y[ny] = X[i + 1]; ex[ny][0] = E[i]->ta; ex[ny][1] = E[i]->tb; ++ny; }
  for (int i = 0; i < na; ++i) { Y[ny] = Ya[i]; ex[ny][0] = ex[ny][1] = ja[i]; ++ny; }
  Y[ny] = R; ex[ny][0] = ex[ny][1] = -1; ++ny;
  if (cr) cr->total = 0;
  for (int q = 0; q + 1 < ny; ++q) {
    if (!cr) {
      if (occluded4(S, Y[q], Y[q + 1], ex[q][0], ex[q][1], ex[q + 1][0], ex[q + 1][1], P, scale, &fl)) return 0;
      continue;
    }
    int nq = leg_crossings(S, Y[q], Y[q + 1], ex[q][0], ex[q][1], ex[q + 1][0], ex[q + 1][1], P, scale, &fl,
                           cr->id + cr->total, cr->cap - cr->total);
    if (nq < 0) return 0;
    cr->n[q] = nq;
    cr->total += nq;
  }
  /* field: the transmitter's wave along its real first leg, reflected at
   * each point before the chain */
  v3 ip = scl(sub(X[1], X[0]), 1.0 / ell[0]);   /* the real direction into Q_1 */
  double complex Ei = cexp(-I * k * ell[0]) / ell[0];
  v3 din = nb ? unit(sub(Y[1], T)) : ip;
  c3 Er = mk3c(pol_dir(u, din, &fl));
  for (int i = 0; i < nb; ++i) {
    v3 dout = i == nb - 1 ? ip : unit(sub(Y[i + 2], Y[i + 1]));
    Er = reflect_field(S, P, &S->t[jb[i]], din, dout, Er);
    din = dout;
  }
  c3 Ev;
  Ev.x = Ei * Er.x; Ev.y = Ei * Er.y; Ev.z = Ei * Er.z;
  double rho1 = ell[0], rho2 = ell[0];
  v3 dir1 = mk(0, 0, 0), dir2 = mk(0, 0, 0);
  v3 dd = ip;
  for (int i = 0; i < m; ++i) {
    const owedge* Ew = E[i];
    double s = ell[i + 1];
    dd = scl(sub(X[i + 2], X[i + 1]), 1.0 / s);
    double cb = dot(ip, Ew->e);
    double beta0 = acos(fmax(-1.0, fmin(1.0, cb)));
    double sb = sin(beta0);
    v3 php = cross(Ew->e, ip), ph = cross(Ew->e, dd);
    php = scl(php, -1.0 / norm(php));
    ph = scl(ph, 1.0 / norm(ph));
    v3 bp = cross(ip, php), bd = cross(dd, ph);
    /* incident radius of curvature in the plane of the edge */
    double rhoe;
    if (i == 0) rhoe = ell[0];
    else {
      double c1 = dot(bp, dir1), c2 = dot(bp, dir2);
      rhoe = 1.0 / (c1 * c1 / rho1 + c2 * c2 / rho2);
    }
    double L = s * (rhoe + s) * rho1 * rho2 * sb * sb / (rhoe * (rho1 + s) * (rho2 + s));
    int ma = S->t[Ew->ta].mat, mb = S->t[Ew->tb].mat;
    if (ma < 0 || ma >= S->nmat) ma = 0;
    if (mb < 0 || mb >= S->nmat) mb = 0;
    double nn = Ew->n;
    double complex r0s, r0h, rns, rnh;
    fresnel(&S->mats[3 * ma], P->freq_hz, fabs(sin(phip[i])), &r0s, &r0h);
    fresnel(&S->mats[3 * mb], P->freq_hz, fabs(sin(nn * M_PI - phi[i])), &rns, &rnh);
    double complex Ds = utd_coeff(nn, phi[i], phip[i], beta0, L, k, r0s, rns, &fl);
    double complex Dh = utd_coeff(nn, phi[i], phip[i], beta0, L, k, r0h, rnh, &fl);
    double complex Eb = cdot(Ev, bp), Ep = cdot(Ev, php);
    double complex A = csqrt(rhoe / (s * (rhoe + s))) * cexp(-I * k * s);
    double complex cb_ = -Ds * Eb * A, cp_ = -Dh * Ep * A;
    Ev.x = cb_ * bd.x + cp_ * ph.x;
    Ev.y = cb_ * bd.y + cp_ * ph.y;
    Ev.z = cb_ * bd.z + cp_ * ph.z;
    /* the wave behind the edge: caustic on the edge (along phi^), the other
     * at rho_e behind it (along beta^) */
    rho1 = s;
    dir1 = ph;
    rho2 = rhoe + s;
    dir2 = bd;
    ip = dd;
  }
  /* reflected at each point after the chain, toward the real receiver */
  v3 dlast = dd;
  for (int i = 0; i < na; ++i) {
    const int at = ny - 1 - na + i;   /* Y[at] is the reflection point on ja[i] */
    v3 dout = unit(sub(Y[at + 1], Y[at]));
    Ev = reflect_field(S, P, &S->t[ja[i]], dlast, dout, Ev);
    dlast = dout;
  }
  v3 prx = pol_dir(u, scl(dlast, -1.0), &fl);
  double complex a = (lam / (4.0 * M_PI)) * cdot(Ev, prx);
  /* the penetration losses of the crossings (power dB: field 10^(-L/20)) */
  if (cr)
    for (int i = 0; i < cr->total; ++i) a *= pow(10.0, -P->trans_db[S->t[cr->id[i]].mat] / 20.0);
  double Ltot = 0.0;
  for (int q = 0; q <= m; ++q) Ltot += ell[q];
  memset(o, 0, sizeof(*o));
  o->valid = 1;
  o->flags = fl;
  o->len_m = Ltot;
  o->delay_s = Ltot / C0;
  o->amp_re = creal(a);
  o->amp_im = cimag(a);
  for (int q = 1; q + 1 < ny; ++q) {
    o->pts[q - 1][0] = Y[q].x;
    o->pts[q - 1][1] = Y[q].y;
    o->pts[q - 1][2] = Y[q].z;
  }
  return 1;
}

/* chain_path_r with at most one reflection, on static triangle j (j < 0:
 * none) before the first wedge (first = 1) or after the last (first = 0). */
static int chain_path(const oscene* S, const owedge* const* E, int m, v3 T, v3 R, int j, int first,
                      const or_params* P, opath* o) {
  const int nb = j >= 0 && first ? 1 : 0, na = j >= 0 && !first ? 1 : 0;
  return chain_path_r(S, E, m, T, R, &j, nb, &j, na, P, o, NULL);
}

/* Paths Tx -> Q_1 -> ... -> Q_m -> Rx over m pairwise distinct wedges
 * (m = 2 or 3) allowed by chain_allowed (consecutive wedges sharing no
 * vertex, not on one line, neither edge in a face plane of the other). Each
 * Q_i is a Keller point (keller_points) strictly inside its edge; at every
 * wedge the previous point (Tx or Q_{i-1}) and the next point (Q_{i+1} or
 * Rx) lie in the exterior and the next point lies beyond the incident
 * shadow boundary of the previous one (or_diffract's rule, edge by edge);
 * every leg is unoccluded (the faces of the wedges at its ends excluded).
 * Field: at each wedge the UTD coefficient of or_diffract (Luebbers' face
 * factors) acts on the field the previous leg brings, in the edge-fixed
 * bases of that wedge. The spreading follows Kouyoumjian & Pathak (1974)
 * for a straight edge: the wave leaving wedge i has one caustic on the edge
 * (radius of curvature s along phi^) and the other at rho_e behind it
 * (radius rho_e + s along beta^), rho_e being the incident wavefront's
 * radius of curvature in the plane of the edge (Euler's formula on the
 * principal radii rho_1, rho_2 along the edge's projection; rho_e = s' for
 * the spherical wave of the transmitter); the spreading factor is
 * sqrt(rho_e / (s (rho_e + s))) and the distance parameter L = s (rho_e +
 * s) rho_1 rho_2 sin^2 beta_0 / (rho_e (rho_1 + s) (rho_2 + s)), which is
 * s s' sin^2 beta_0 / (s + s') for the spherical wave (chain_path). Keys:
 * rx, m, w_1 | OR_DIFF, .., w_m | OR_DIFF, -1 padded to 2 + width (width >=
 * m). Returns the number of valid paths (may exceed cap). */
int64_t or_diffract_multi(const float* tris, const int32_t* tri_mat, const int32_t* tri_obj, int32_t ntri,
                          const float* mats, int32_t nmat, const float* tx, const float* rx, int32_t nrx,
                          const or_params* P, int32_t order, int32_t width, int32_t* keys_out,
                          opath* paths_out, int64_t cap) {
  if (order < 2 || order > 3 || width < order) return -1;
  oscene S;
  if (scene_load(&S, tris, tri_mat, ntri, mats, nmat)) return -2;
  owedge* W = NULL;
  long nw = find_wedges(tris, tri_obj, ntri, &W);
  const int m = order;
  v3 T = mk(tx[0], tx[1], tx[2]);
  int64_t nvalid = 0;
  long w[3] = {0, 0, 0};
  opath tmp;
  for (int r = 0; r < nrx; ++r) {
    v3 R = mk(rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]);
    for (w[0] = 0; w[0] < nw; ++w[0])
      for (w[1] = 0; w[1] < nw; ++w[1])
        for (w[2] = 0; w[2] < (m == 3 ? nw : 1); ++w[2]) {
          if (!chain_allowed(W, w, m)) continue;
          const owedge* E[3] = {&W[w[0]], &W[w[1]], m == 3 ? &W[w[2]] : NULL};
          if (!chain_path(&S, E, m, T, R, -1, 0, P, &tmp)) continue;
          if (nvalid < cap) {
            int32_t* kk = &keys_out[(size_t)nvalid * (2 + width)];
            kk[0] = r;
            kk[1] = m;
            for (int q = 0; q < width; ++q) kk[2 + q] = q < m ? ((int32_t)w[q] | OR_DIFF) : -1;
            paths_out[nvalid] = tmp;
          }
          nvalid++;
        }
  }
  free(W);
  scene_free(&S);
  return nvalid;
}

/* Chains of m = 2 or 3 wedges (as or_diffract_multi) whose legs pass
 * straight through transmitting triangles (Table II losses), at least one
 * and at most max_trans crossings in all (and at most OR_MAX_REFL - m): the
 * Keller points, rules and field of the chain, each crossing scaling the
 * field by 10^(-L/20). Keys: rx, m + crossings, then in path order the
 * crossings of each leg (| OR_TRANS) and the wedges (| OR_DIFF); -1 padded
 * to 2 + width. Points in the same order. Chains with no crossing are
 * or_diffract_multi's and are not written here. Returns the number of
 * valid paths (may exceed cap). */
int64_t or_diffract_multi_trans(const float* tris, const int32_t* tri_mat, const int32_t* tri_obj, int32_t ntri,
                                const float* mats, int32_t nmat, const float* tx, const float* rx, int32_t nrx,
                                const or_params* P, int32_t order, int32_t width, int32_t* keys_out,
                                opath* paths_out, int64_t cap) {
  if (order < 2 || order > 3 || width < order) return -1;
  if (!P->trans_db || P->max_trans < 1) return 0;
  oscene S;
  if (scene_load(&S, tris, tri_mat, ntri, mats, nmat)) return -2;
  owedge* W = NULL;
  long nw = find_wedges(tris, tri_obj, ntri, &W);
  const int m = order, none = -1;
  v3 T = mk(tx[0], tx[1], tx[2]);
  int64_t nvalid = 0;
  long w[3] = {0, 0, 0};
  opath tmp;
  ocross cr;
  for (int r = 0; r < nrx; ++r) {
    v3 R = mk(rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]);
    for (w[0] = 0; w[0] < nw; ++w[0])
      for (w[1] = 0; w[1] < nw; ++w[1])
        for (w[2] = 0; w[2] < (m == 3 ? nw : 1); ++w[2]) {
          if (!chain_allowed(W, w, m)) continue;
          const owedge* E[3] = {&W[w[0]], &W[w[1]], m == 3 ? &W[w[2]] : NULL};
          cr.cap = P->max_trans < OR_MAX_REFL - m ? P->max_trans : OR_MAX_REFL - m;
          if (!chain_path_r(&S, E, m, T, R, &none, 0, &none, 0, P, &tmp, &cr) || cr.total < 1) continue;
          const int depth = m + cr.total;
          if (nvalid < cap && depth <= width) {
            int32_t* kk = &keys_out[(size_t)nvalid * (2 + width)];
            kk[0] = r;
            kk[1] = depth;
            /* path order: leg 0's crossings, w_1, leg 1's, .., w_m, leg m's */
            v3 Pt[OR_MAX_REFL];
            v3 ends[5];
            ends[0] = T;
            for (int i = 0; i < m; ++i) ends[i + 1] = mk(tmp.pts[i][0], tmp.pts[i][1], tmp.pts[i][2]);
            ends[m + 1] = R;
            int q = 0, c = 0;
            for (int leg = 0; leg <= m; ++leg) {
              v3 a0 = ends[leg], dl = sub(ends[leg + 1], ends[leg]);
              for (int i = 0; i < cr.n[leg]; ++i, ++c, ++q) {
                const otri* Tc = &S.t[cr.id[c]];
                kk[2 + q] = cr.id[c] | OR_TRANS;
                Pt[q] = add(a0, scl(dl, dot(sub(Tc->v[0], a0), Tc->n) / dot(dl, Tc->n)));
              }
              if (leg < m) {
                kk[2 + q] = (int32_t)w[leg] | OR_DIFF;
                Pt[q] = ends[leg + 1];
                ++q;
              }
            }
            for (int j = q; j < width; ++j) kk[2 + j] = -1;
            opath* o = &paths_out[nvalid];
            *o = tmp;
            memset(o->pts, 0, sizeof(o->pts));
            for (int j = 0; j < depth; ++j) {
              o->pts[j][0] = Pt[j].x;
              o->pts[j][1] = Pt[j].y;
              o->pts[j][2] = Pt[j].z;
            }
          }
          nvalid++;
        }
  }
  free(W);
  scene_free(&S);
  return nvalid;
}

/* Sec. III steps 3-5 combined: one reflection on a static triangle j before
 * a chain of m = 2 or 3 wedges or after it (chain_path), the chain allowed
 * by chain_allowed and j none of its wedges' faces. Keys: rx, m + 1, then
 * j, w_1 | OR_DIFF, .. (reflection first) or w_1 | OR_DIFF, .., j
 * (reflection last); -1 padded to 2 + width (width >= m + 1). Returns the
 * number of valid paths (may exceed cap). */
int64_t or_diffract_multi_refl(const float* tris, const int32_t* tri_mat, const int32_t* tri_obj, int32_t ntri,
                               const float* mats, int32_t nmat, const float* tx, const float* rx, int32_t nrx,
                               const or_params* P, int32_t order, int32_t width, int32_t* keys_out,
                               opath* paths_out, int64_t cap) {
  if (order < 2 || order > 3 || width < order + 1) return -1;
  oscene S;
  if (scene_load(&S, tris, tri_mat, ntri, mats, nmat)) return -2;
  owedge* W = NULL;
  long nw = find_wedges(tris, tri_obj, ntri, &W);
  const int m = order;
  v3 T = mk(tx[0], tx[1], tx[2]);
  int64_t nvalid = 0;
  long w[3] = {0, 0, 0};
  opath tmp;
  for (int r = 0; r < nrx; ++r) {
    v3 R = mk(rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]);
    for (w[0] = 0; w[0] < nw; ++w[0])
      for (w[1] = 0; w[1] < nw; ++w[1])
        for (w[2] = 0; w[2] < (m == 3 ? nw : 1); ++w[2]) {
          if (!chain_allowed(W, w, m)) continue;
          const owedge* E[3] = {&W[w[0]], &W[w[1]], m == 3 ? &W[w[2]] : NULL};
          for (int j = 0; j < ntri; ++j) {
            if (tri_obj && tri_obj[j] >= 0) continue;
            int face = 0;
            for (int i = 0; i < m; ++i) face |= j == E[i]->ta || j == E[i]->tb;
            if (face) continue;
            for (int first = 1; first >= 0; --first) {
              if (!chain_path(&S, E, m, T, R, j, first, P, &tmp)) continue;
              if (nvalid < cap) {
                int32_t* kk = &keys_out[(size_t)nvalid * (2 + width)];
                kk[0] = r;
                kk[1] = m + 1;
                for (int q = 0; q < width; ++q) {
                  int v = -1;
                  if (q <= m) {
                    if (first) v = q == 0 ? j : ((int32_t)w[q - 1] | OR_DIFF);
                    else v = q == m ? j : ((int32_t)w[q] | OR_DIFF);
                  }
                  kk[2 + q] = v;
                }
                paths_out[nvalid] = tmp;
              }
              nvalid++;
            }
          }
        }
  }
  free(W);
  scene_free(&S);
  return nvalid;
}

/* Sec. III steps 3-5 with the evaluation's mechanism limits (two reflections,
 * one diffraction): a first-order diffraction at wedge w with two
 * reflections on static triangles, both before it (j1, j2, w), one on each
 * side (j1, w, j2) or both after it (w, j1, j2) (chain_path_r with m = 1).
 * Neither triangle is a face of the wedge; two reflections in a row are on
 * different triangles (one on each side of the wedge may be on the same
 * triangle). Keys: rx, 3, then the three ids in path order (the wedge's with
 * OR_DIFF); -1 padded to 2 + width (width >= 3). Returns the number of
 * valid paths (may exceed cap). */
int64_t or_diffract_refl2(const float* tris, const int32_t* tri_mat, const int32_t* tri_obj, int32_t ntri,
                          const float* mats, int32_t nmat, const float* tx, const float* rx, int32_t nrx,
                          const or_params* P, int32_t width, int32_t* keys_out, opath* paths_out, int64_t cap) {
  if (width < 3) return -1;
  oscene S;
  if (scene_load(&S, tris, tri_mat, ntri, mats, nmat)) return -2;
  owedge* W = NULL;
  long nw = find_wedges(tris, tri_obj, ntri, &W);
  v3 T = mk(tx[0], tx[1], tx[2]);
  int64_t nvalid = 0;
  opath tmp;
  for (int r = 0; r < nrx; ++r) {
    v3 R = mk(rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]);
    for (long w = 0; w < nw; ++w) {
      const owedge* E[1] = {&W[w]};
      for (int j1 = 0; j1 < ntri; ++j1) {
        if ((tri_obj && tri_obj[j1] >= 0) || j1 == W[w].ta || j1 == W[w].tb) continue;
        for (int j2 = 0; j2 < ntri; ++j2) {
          if ((tri_obj && tri_obj[j2] >= 0) || j2 == W[w].ta || j2 == W[w].tb) continue;
          for (int nb = 2; nb >= 0; --nb) {   /* reflections before the wedge */
            const int na = 2 - nb;
            if (nb != 1 && j1 == j2) continue;
            const int j[2] = {j1, j2};
            if (!chain_path_r(&S, E, 1, T, R, j, nb, j + nb, na, P, &tmp, NULL)) continue;
            if (nvalid < cap) {
              int32_t* kk = &keys_out[(size_t)nvalid * (2 + width)];
              kk[0] = r;
              kk[1] = 3;
              kk[2 + nb] = (int32_t)w | OR_DIFF;
              kk[2 + (nb == 0 ? 1 : 0)] = j1;
              kk[2 + (nb == 2 ? 1 : 2)] = j2;
              for (int q = 3; q < width; ++q) kk[2 + q] = -1;
              paths_out[nvalid] = tmp;
            }
            nvalid++;
          }
        }
      }
    }
  }
  free(W);
  scene_free(&S);
  return nvalid;
}

/* A wedge mirrored in the plane of triangle Tj: its points and directions
 * mirrored (the angle of a mirrored point about the mirrored edge is that of
 * the point about the edge), its faces and exterior angle kept. */
static owedge mirror_wedge(const otri* Tj, const owedge* W) {
  owedge M = *W;
  M.p0 = mirror_in(Tj, W->p0);
  M.p1 = mirror_in(Tj, W->p1);
  v3 n = Tj->nh;
  M.e = sub(W->e, scl(n, 2.0 * dot(W->e, n)));
  M.t0 = sub(W->t0, scl(n, 2.0 * dot(W->t0, n)));
  M.y0 = sub(W->y0, scl(n, 2.0 * dot(W->y0, n)));
  M.tB = sub(W->tB, scl(n, 2.0 * dot(W->tB, n)));
  return M;
}

/* Tx -> Q1 -> P -> Q2 -> Rx: a specular reflection on static triangle j
 * between two diffractions (wedges A then B). By image theory, mirroring
 * the part after P in j's plane, it is the chain over A and B's image B'
 * toward the receiver's image R': the Keller points of that chain
 * (keller_points), its rules (chain_allowed's, and the exterior and shadow
 * rule at both wedges), and P where the unfolded leg Q1 -> Q2' crosses the
 * plane, strictly inside the leg and inside triangle j; Q2 is the mirror of
 * Q2'. The four real legs are unoccluded (the wedge's faces excluded at Q1
 * and Q2, j at P). Field: the UTD chain of chain_path_r, with at P the
 * Fresnel reflection of j's material in the real directions (the bounce
 * basis of validate_one) and the principal directions of the wavefront
 * mirrored (a plane mirror keeps its radii of curvature); at B the real
 * geometry (the direction from P, the angles of P and Rx about B's edge).
 * Returns 1 when the path is valid, with o filled (points Q1, P, Q2). */
static int mid_path(const oscene* S, const owedge* A, const owedge* B, int j, v3 T, v3 R, const or_params* P,
                    opath* o) {
  const double k = 2.0 * M_PI * P->freq_hz / C0, lam = C0 / P->freq_hz;
  const double ang_eps = 1e-9;
  const v3 u = mk(P->pol[0], P->pol[1], P->pol[2]);
  const otri* Tj = &S->t[j];
  uint32_t fl = 0;
  const owedge Bm = mirror_wedge(Tj, B);
  if (share_vertex(A, &Bm) || collinear_edges(A, &Bm) || in_face_plane(A, &Bm) || in_face_plane(&Bm, A)) return 0;
  const v3 Rm = mirror_in(Tj, R);
  const owedge* E[2] = {A, &Bm};
  if (wedge_angle(A, T) > A->n * M_PI || wedge_angle(&Bm, Rm) > Bm.n * M_PI) return 0;
  double t[2];
  if (!keller_points(E, 2, T, Rm, t)) return 0;
  v3 X[4];
  X[0] = T;
  for (int i = 0; i < 2; ++i) {
    double uq = t[i] / E[i]->len;
    if (fabs(uq) <= P->val_eps || fabs(uq - 1.0) <= P->val_eps) fl |= ORF_VAL_PARAM;
    if (!(uq > 0 && uq < 1)) return 0;
    X[i + 1] = add(E[i]->p0, scl(E[i]->e, t[i]));
  }
  X[3] = Rm;
  double ell[3];
  for (int q = 0; q < 3; ++q) {
    ell[q] = norm(sub(X[q + 1], X[q]));
    if (!(ell[q] > 1e-9)) return 0;
  }
  double phip[2], phi[2];
  for (int i = 0; i < 2; ++i) {
    phip[i] = wedge_angle(E[i], X[i]);
    phi[i] = wedge_angle(E[i], X[i + 2]);
    double nn = E[i]->n;
    if (phip[i] > nn * M_PI || phi[i] > nn * M_PI) return 0;
    if (fabs(fabs(phi[i] - phip[i]) - M_PI) <= ang_eps) fl |= ORF_VAL_PARAM;
    if (!(fabs(phi[i] - phip[i]) > M_PI)) return 0;
  }
  double scale = fmax(maxabs(T), maxabs(R));
  v3 Pp;
  if (!mirror_point(Tj, X[1], X[2], P, scale, &fl, &Pp)) return 0;
  const v3 Q1 = X[1], Q2 = mirror_in(Tj, X[2]);
  /* the real legs */
  const v3 Y[5] = {T, Q1, Pp, Q2, R};
  const int ex[5][2] = {{-1, -1}, {A->ta, A->tb}, {j, j}, {B->ta, B->tb}, {-1, -1}};
  for (int q = 0; q < 4; ++q)
    if (occluded4(S, Y[q], Y[q + 1], ex[q][0], ex[q][1], ex[q + 1][0], ex[q + 1][1], P, scale, &fl)) return 0;
  /* field: the transmitter's wave, UTD at A (spherical incidence) */
  v3 ip = scl(sub(Q1, T), 1.0 / ell[0]);
  double complex Ei = cexp(-I * k * ell[0]) / ell[0];
  c3 Ev;
  {
    v3 e0 = pol_dir(u, ip, &fl);
    Ev.x = Ei * e0.x; Ev.y = Ei * e0.y; Ev.z = Ei * e0.z;
  }
  double rho1 = ell[0], rho2 = ell[0];
  v3 dir1 = mk(0, 0, 0), dir2 = mk(0, 0, 0);
  const double s1 = ell[1];  /* Q1 to Q2 along the real path (P between) */
  const v3 din = unit(sub(Pp, Q1)), dout = unit(sub(Q2, Pp));
  for (int i = 0; i < 2; ++i) {
    const owedge* Ew = i == 0 ? A : B;
    const v3 dd = i == 0 ? din : unit(sub(R, Q2));
    const double s = i == 0 ? s1 : ell[2];
    if (i == 1) {
      /* the reflection at P: Fresnel in the real directions, the wavefront's
       * principal directions mirrored */
      Ev = reflect_field(S, P, Tj, din, dout, Ev);
      dir1 = sub(dir1, scl(Tj->nh, 2.0 * dot(dir1, Tj->nh)));
      dir2 = sub(dir2, scl(Tj->nh, 2.0 * dot(dir2, Tj->nh)));
      ip = dout;
    }
    double cb = dot(ip, Ew->e);
    double beta0 = acos(fmax(-1.0, fmin(1.0, cb)));
    double sb = sin(beta0);
    v3 php = cross(Ew->e, ip), ph = cross(Ew->e, dd);
    php = scl(php, -1.0 / norm(php));
    ph = scl(ph, 1.0 / norm(ph));
    v3 bp = cross(ip, php), bd = cross(dd, ph);
    double rhoe;
    if (i == 0) rhoe = ell[0];
    else {
      double c1 = dot(bp, dir1), c2 = dot(bp, dir2);
      rhoe = 1.0 / (c1 * c1 / rho1 + c2 * c2 / rho2);
    }
    double L = s * (rhoe + s) * rho1 * rho2 * sb * sb / (rhoe * (rho1 + s) * (rho2 + s));
    int ma = S->t[Ew->ta].mat, mb = S->t[Ew->tb].mat;
    if (ma < 0 || ma >= S->nmat) ma = 0;
    if (mb < 0 || mb >= S->nmat) mb = 0;
    double nn = Ew->n;
    /* the angles about the real edge: those about the unfolded one */
    double pp = phip[i], pf = phi[i];
    double complex r0s, r0h, rns, rnh;
    fresnel(&S->mats[3 * ma], P->freq_hz, fabs(sin(pp)), &r0s, &r0h);
    fresnel(&S->mats[3 * mb], P->freq_hz, fabs(sin(nn * M_PI - pf)), &rns, &rnh);
    double complex Ds = utd_coeff(nn, pf, pp, beta0, L, k, r0s, rns, &fl);
    double complex Dh = utd_coeff(nn, pf, pp, beta0, L, k, r0h, rnh, &fl);
    double complex Eb = cdot(Ev, bp), Ep = cdot(Ev, php);
    double complex Amp = csqrt(rhoe / (s * (rhoe + s))) * cexp(-I * k * s);
    double complex cb_ = -Ds * Eb * Amp, cp_ = -Dh * Ep * Amp;
    Ev.x = cb_ * bd.x + cp_ * ph.x;
    Ev.y = cb_ * bd.y + cp_ * ph.y;
    Ev.z = cb_ * bd.z + cp_ * ph.z;
    rho1 = s;
    dir1 = ph;
    rho2 = rhoe + s;
    dir2 = bd;
    ip = dd;
  }
  v3 prx = pol_dir(u, scl(ip, -1.0), &fl);
  double complex a = (lam / (4.0 * M_PI)) * cdot(Ev, prx);
  double Ltot = ell[0] + ell[1] + ell[2];
  memset(o, 0, sizeof(*o));
  o->valid = 1;
  o->flags = fl;
  o->len_m = Ltot;
  o->delay_s = Ltot / C0;
  o->amp_re = creal(a);
  o->amp_im = cimag(a);
  const v3 pts[3] = {Q1, Pp, Q2};
  for (int q = 0; q < 3; ++q) {
    o->pts[q][0] = pts[q].x;
    o->pts[q][1] = pts[q].y;
    o->pts[q][2] = pts[q].z;
  }
  return 1;
}

/* Sec. III steps 3-5: a specular reflection on a static triangle j between
 * two diffractions (mid_path) over distinct wedges A, B, j a face of
 * neither. Keys: rx, 3, A | OR_DIFF, j, B | OR_DIFF; -1 padded to 2 + width
 * (width >= 3). Returns the number of valid paths (may exceed cap). */
int64_t or_diffract_mid(const float* tris, const int32_t* tri_mat, const int32_t* tri_obj, int32_t ntri,
                        const float* mats, int32_t nmat, const float* tx, const float* rx, int32_t nrx,
                        const or_params* P, int32_t width, int32_t* keys_out, opath* paths_out, int64_t cap) {
  if (width < 3) return -1;
  oscene S;
  if (scene_load(&S, tris, tri_mat, ntri, mats, nmat)) return -2;
  owedge* W = NULL;
  long nw = find_wedges(tris, tri_obj, ntri, &W);
  v3 T = mk(tx[0], tx[1], tx[2]);
  int64_t nvalid = 0;
  opath tmp;
  for (int r = 0; r < nrx; ++r) {
    v3 R = mk(rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]);
    for (long a = 0; a < nw; ++a)
      for (long b = 0; b < nw; ++b) {
        if (a == b) continue;
        for (int j = 0; j < ntri; ++j) {
          if ((tri_obj && tri_obj[j] >= 0) || j == W[a].ta || j == W[a].tb || j == W[b].ta || j == W[b].tb) continue;
          if (!mid_path(&S, &W[a], &W[b], j, T, R, P, &tmp)) continue;
          if (nvalid < cap) {
            int32_t* kk = &keys_out[(size_t)nvalid * (2 + width)];
            kk[0] = r;
            kk[1] = 3;
            kk[2] = (int32_t)a | OR_DIFF;
            kk[3] = j;
            kk[4] = (int32_t)b | OR_DIFF;
            for (int q = 3; q < width; ++q) kk[2 + q] = -1;
            paths_out[nvalid] = tmp;
          }
          nvalid++;
        }
      }
  }
  free(W);
  scene_free(&S);
  return nvalid;
}

/* One given path of the combined mechanisms, for checking paths found
 * elsewhere: ids[0..depth-1] in path order, static triangles (reflections)
 * before and after a run of 1-3 wedge ids marked OR_DIFF, at most two
 * reflections (chain_path_r), or a wedge, a triangle and a wedge (mid_path);
 * for transmitter tx and receiver rx. Returns 1 (valid, o filled), 0 (not a
 * valid path) or -1 (ids not of that form). */
int32_t or_diffract_path(const float* tris, const int32_t* tri_mat, const int32_t* tri_obj, int32_t ntri,
                         const float* mats, int32_t nmat, const float* tx, const float* rx, const int32_t* ids,
                         int32_t depth, const or_params* P, opath* o) {
  int jb[2], ja[2], nb = 0, na = 0, m = 0;
  long wi[3];
  const int mid = depth == 3 && (ids[0] & OR_DIFF) && !(ids[1] & OR_DIFF) && (ids[2] & OR_DIFF);
  for (int q = 0; q < depth && !mid; ++q) {
    if (ids[q] & OR_DIFF) {
      if (na || m == 3) return -1;
      wi[m++] = ids[q] & ~OR_DIFF;
    } else if (m == 0) {
      if (nb == 2) return -1;
      jb[nb++] = ids[q];
    } else {
      if (na == 2) return -1;
      ja[na++] = ids[q];
    }
  }
  if (mid) {
    m = 2;
    wi[0] = ids[0] & ~OR_DIFF;
    wi[1] = ids[2] & ~OR_DIFF;
    ja[0] = ids[1];
  }
  if (m == 0 || nb + na > 2) return -1;
  oscene S;
  if (scene_load(&S, tris, tri_mat, ntri, mats, nmat)) return -2;
  owedge* W = NULL;
  long nw = find_wedges(tris, tri_obj, ntri, &W);
  int ok = 1;
  if (mid) {
    ok = wi[0] >= 0 && wi[0] < nw && wi[1] >= 0 && wi[1] < nw && ja[0] >= 0 && ja[0] < ntri;
    int r = -1;
    if (ok) r = mid_path(&S, &W[wi[0]], &W[wi[1]], ja[0], mk(tx[0], tx[1], tx[2]), mk(rx[0], rx[1], rx[2]), P, o);
    free(W);
    scene_free(&S);
    return r;
  }
  for (int i = 0; i < m; ++i) ok &= wi[i] >= 0 && wi[i] < nw;
  for (int i = 0; i < nb; ++i) ok &= jb[i] >= 0 && jb[i] < ntri;
  for (int i = 0; i < na; ++i) ok &= ja[i] >= 0 && ja[i] < ntri;
  int r = -1;
  if (ok) {
    const owedge* E[3] = {&W[wi[0]], m > 1 ? &W[wi[1]] : NULL, m > 2 ? &W[wi[2]] : NULL};
    v3 T = mk(tx[0], tx[1], tx[2]), R = mk(rx[0], rx[1], rx[2]);
    r = chain_path_r(&S, E, m, T, R, jb, nb, ja, na, P, o, NULL);
  }
  free(W);
  scene_free(&S);
  return r;
}

int32_t or_path_size(void) { return (int32_t)sizeof(opath); }

/* ------------------------------------------------------------------------ */
/* or_exhaustive: image-method validation of EVERY sequence of length <= N   */
/* ------------------------------------------------------------------------ */
/* Writes up to `cap` valid keys (rows of 2 + max_refl ints) and their path
 * records; returns the number of valid paths (may exceed cap). */
int64_t or_exhaustive(const float* tris, const int32_t* tri_mat, int32_t ntri, const float* mats,
                      int32_t nmat, const float* tx, const float* rx, int32_t nrx,
                      const or_params* P, int32_t* keys_out, opath* paths_out, int64_t cap) {
  if (P->max_refl < 0 || P->max_trans < 0 || P->max_refl + P->max_trans > OR_MAX_REFL) return -1;
  oscene S;
  if (scene_load(&S, tris, tri_mat, ntri, mats, nmat)) return -2;
  const int N = P->max_refl, T = P->trans_db ? P->max_trans : 0, W = N + T, stride = 2 + W;
  /* each interaction: a triangle and (with transmission) reflect or transmit */
  const int ch = T > 0 ? 2 * ntri : ntri;
  int64_t nvalid = 0;
  int32_t ids[OR_MAX_REFL], c[OR_MAX_REFL];
  opath tmp;
  for (int r = 0; r < nrx; ++r) {
    v3 R = mk(rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]);
    for (int k = 0; k <= W; ++k) {
      if (k > 0 && ntri == 0) break;
      for (int j = 0; j < k; ++j) c[j] = 0;
      for (;;) {
        int okseq = 1, nr = 0, ntr = 0;
        for (int j = 0; j < k; ++j) {
          int tri = T > 0 ? c[j] >> 1 : c[j], tr = T > 0 ? (c[j] & 1) : 0;
          ids[j] = tr ? (tri | OR_TRANS) : tri;
          if (tr) ++ntr; else ++nr;
          if (tr && !transmits(&S, P, S.t[tri].mat)) okseq = 0;
          if (j > 0 && (ids[j] & ~OR_TRANS) == (ids[j - 1] & ~OR_TRANS)) okseq = 0;
        }
        if (nr > N || ntr > T) okseq = 0;
        if (okseq) {
          validate_one(&S, P, mk(tx[0], tx[1], tx[2]), R, k, ids, &tmp, 1);
          if (tmp.valid) {
            if (nvalid < cap) {
              int32_t* kk = &keys_out[(size_t)nvalid * stride];
              kk[0] = r; kk[1] = k;
              for (int j = 0; j < W; ++j) kk[2 + j] = j < k ? ids[j] : -1;
              paths_out[nvalid] = tmp;
            }
            nvalid++;
          }
        }
        /* next sequence (odometer) */
        int j = k - 1;
        while (j >= 0) {
          if (++c[j] < ch) break;
          c[j] = 0;
          --j;
        }
        if (j < 0) break;
      }
    }
  }
  scene_free(&S);
  return nvalid;
}
