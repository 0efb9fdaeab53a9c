/*
 * dcem.h -- C ABI of the GB300 dynamic coherence-based EM ray tracer.
 *
 * The library computes, per frame, the propagation paths between one
 * transmitter (Tx) and a set of receivers (Rx) in a scene of static triangles
 * plus rigid moving objects, and the power each Rx receives, following
 * arXiv 2112.07115 (DCEM), Sec. III:
 *   - per-frame update of the scene and of its bounding volume hierarchy
 *     ("Efficient BVH updating": the hierarchy is refit every frame);
 *   - shooting a sphere of sampled rays with up to N specular reflections
 *     ("Backward ray tracing", steps 1-2; shot from the Tx, which gives the
 *     same valid path set by reciprocity);
 *   - a table of visited triangle sequences per reflection depth, image
 *     receivers and path validation (steps 2-4);
 *   - total distance, direction, attenuation and phase of every valid path
 *     (step 6; ray field of Eq. 1, free-space loss of Eq. 3, reflection per
 *     Fresnel TE/TM);
 *   - reuse of the previous frame's work where objects did not move
 *     ("Propagation path caching", frame-to-frame coherence).
 *
 * Conventions for every entry point:
 *   - Return DCEM_OK (0) or a negative dcem_status; nothing aborts, traps or
 *     throws across the ABI. dcem_status_string() names a status.
 *   - Arguments are validated before any device work; an invalid argument
 *     returns DCEM_ERR_ARG and leaves the scene unchanged.
 *   - A scene is NOT thread-safe. All its device work is ordered on the CUDA
 *     stream given at creation (or by dcem_scene_set_stream). Calls that
 *     return results to the caller synchronise that stream before returning.
 *   - Triangle ids are the caller's input indices (0..ntri-1) and stay fixed.
 *   - Coordinates are metres, FP32, right-handed; a 3x4 transform is row
 *     major [R | t]: x' = R x + t.
 *   - Pointers marked "host" must be host memory; pointers whose kind is
 *     selected by a DCEM_PTR_* argument may be host (pageable or pinned) or
 *     device memory of the scene's GPU. The library never keeps caller
 *     pointers beyond the call.
 *   - The scene owns all the device memory it allocates and frees it in
 *     dcem_scene_destroy.
 */
#ifndef DCEM_H
#define DCEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Largest reflection order (Sec. III: the maximum number of reflections is
 * limited to 10). */
#define DCEM_MAX_REFL 10

typedef enum {
  DCEM_OK = 0,
  DCEM_ERR_ARG = -1,       /* invalid argument (null, size, index out of range) */
  DCEM_ERR_CUDA = -2,      /* a CUDA call failed (no device, launch error, ...)  */
  DCEM_ERR_CAPACITY = -3,  /* an output or internal buffer is too small          */
  DCEM_ERR_NONFINITE = -4, /* NaN or Inf in geometry, transforms, Tx or Rx       */
  DCEM_ERR_STACK = -5,     /* BVH traversal stack overflow (counted, not trapped) */
  DCEM_ERR_HASH = -6,      /* 64-bit path-key collision between distinct keys    */
  DCEM_ERR_STATE = -7,     /* call out of order (e.g. trace before set_rays)     */
  DCEM_ERR_NOMEM = -8,     /* device allocation failed                           */
  DCEM_ERR_CHECK = -9      /* bounds-checked build only: an index was out of range
                              (replaced, not used; see the library's build) */
} dcem_status;

/* FULL: every ray traced every frame. COHERENT: segments reused across
 * frames (the result equals FULL bit for bit). STICKY: COHERENT plus the
 * paper's path-cache retention (Sec. III "Propagation path caching": cached
 * paths are kept and updated until removed): every valid path of the
 * previous frame is re-validated against the current geometry and kept if
 * still valid, even when no ray of this frame captured it (flag
 * DCEM_PATH_STICKY, count stats.paths_sticky); a superset of FULL. */
typedef enum { DCEM_MODE_FULL = 0, DCEM_MODE_COHERENT = 1, DCEM_MODE_STICKY = 2 } dcem_mode;
/* Arithmetic of the validation geometry (image sources, back-trace,
 * reflection points, path length) and of the phase: FP64, or double-float
 * (pairs of FP32 values, about 44 significant bits) on the FP32 pipe. */
typedef enum { DCEM_PREC_F64 = 0, DCEM_PREC_DF32 = 1 } dcem_prec;
typedef enum { DCEM_PTR_HOST = 0, DCEM_PTR_DEVICE = 1 } dcem_ptr_kind;

/* Path flag bits (dcem_path.flags). */
#define DCEM_PATH_POL_DEGENERATE 1u /* polarisation reference parallel to a path end */
#define DCEM_PATH_STICKY 2u         /* DCEM_MODE_STICKY: kept from the previous frame
                                       (re-validated), no ray captured it this frame */
/* dcem_path.tri[j] flag: interaction j is a transmission through the
 * triangle (straight through, penetration loss), not a reflection. */
#define DCEM_TRI_TRANSMIT 0x40000000
/* dcem_path.tri[0] flag of a diffraction path: the rest is the wedge index
 * (see dcem_scene_set_diffraction). */
#define DCEM_TRI_DIFFRACT 0x20000000

typedef struct dcem_scene dcem_scene;

/* Half-space material for Fresnel reflection: complex permittivity
 * eps_c = eps_r - j sigma / (2 pi f eps0); pec != 0 selects a perfect
 * conductor (Gamma_TE = -1, Gamma_TM = +1). */
typedef struct {
  float eps_r;
  float sigma;   /* S/m */
  int32_t pec;
} dcem_material;

typedef struct {
  double freq_hz;         /* carrier frequency; default 28e9                     */
  double tx_power_w;      /* transmit power; default 5 W (Sec. III, outdoor)     */
  int32_t max_refl;       /* N: reflections per ray, 0..DCEM_MAX_REFL; default 3 */
  int32_t mode;           /* DCEM_MODE_FULL, _COHERENT or _STICKY                */
  float rx_radius_scale;  /* capture radius = scale * alpha * (D+s) / sqrt(3),
                             alpha = sqrt(4 pi / n_rays); default 1.35           */
  float t_min;            /* self-hit offset after a reflection [m]; 1e-4        */
  float escape_len;       /* capture length of a ray that leaves the scene; 1e4 */
  float eps_occ;          /* occlusion ignores the first/last eps of a sub-
                             segment (relative); default 1e-4                    */
  float pol[3];           /* antenna polarisation reference u; default (0,0,1)  */
  int32_t timing;         /* 1: record per-stage device times in the stats;
                             2: only the closest-hit kernel's (ms_stage[2]),
                             with two event records instead of nine         */
  int32_t prec;           /* DCEM_PREC_F64 (default) or DCEM_PREC_DF32       */
} dcem_params;

/* One valid propagation path (Sec. III step 6). */
typedef struct {
  int32_t rx;                       /* receiver index                           */
  int32_t depth;                    /* number of reflections k                  */
  int32_t tri[DCEM_MAX_REFL];       /* reflecting triangle ids, Tx side first   */
  uint32_t flags;                   /* DCEM_PATH_* bits                         */
  int32_t ray;                      /* a ray that discovered the path (index
                                       into the caller's directions; with
                                       several ray sets, into their
                                       concatenation)                           */
  int32_t tx;                       /* transmitter (ray set); 0 from
                                       dcem_trace_frame                         */
  int32_t reserved;                 /* 0                                        */
  uint64_t key;                     /* 64-bit hash of (rx, depth, tri[0..k))    */
  double len_m;                     /* unfolded path length L                   */
  double delay_s;                   /* L / c                                    */
  double amp_re, amp_im;            /* complex amplitude a (received field per
                                       unit transmit amplitude, isotropic)      */
  float pts[DCEM_MAX_REFL][3];      /* reflection points, Tx side first         */
} dcem_path;

typedef struct {
  int64_t n_rays;              /* rays in the sampled sphere                     */
  int64_t segments_traced;     /* closest-hit traversals this frame              */
  int64_t segments_reused;     /* logged segments reused without traversal       */
  int64_t rays_retraced;       /* rays (partially) retraced in COHERENT mode     */
  int64_t candidates;          /* reception-sphere captures (with duplicates)    */
  int64_t candidates_reused;   /* captures carried over from the previous frame  */
  int64_t unique_candidates;   /* distinct (rx, depth, sequence) keys            */
  int64_t paths_valid;         /* validated paths                                */
  int64_t objects_moved;       /* rigid objects whose transform changed          */
  int64_t rx_moved;            /* receivers whose position changed               */
  int64_t node_visits;         /* BVH internal nodes visited by closest-hit
                                  traversals (64 B each)                         */
  int64_t tri_tests;           /* triangles tested by closest-hit traversals
                                  (48 B each)                                    */
  int32_t stack_overflow;      /* traversals that overflowed the stack           */
  int32_t coherent;            /* 1 if the frame reused the cache                */
  int32_t kernel_launches;     /* kernels launched by this call and by the
                                  transform updates since the previous frame    */
  int32_t bvh_rebuilt;         /* 1 if the moving-object tree was rebuilt since
                                  the previous frame                             */
  float ms_stage[10];          /* if params.timing == 1: prep, mark, trace, capture,
                                  dedupe, validate, reduce, copy-out, total,
                                  (unused)                                       */
  float bvh_cost_ratio;        /* surface-area cost of the moving-object tree
                                  over its cost right after the last rebuild     */
  int32_t max_segment_nodes;   /* most BVH nodes visited by one traversal        */
  int32_t trace_kernel;        /* closest-hit kernel of this frame: 0 = binary
                                  nodes read from global memory, 1 = 4-wide
                                  compact copy in shared memory, 2 = 4-wide
                                  compact copy read from global memory, 3 =
                                  one launch for every scene of a batch
                                  (binary nodes from global memory)           */
  int32_t graph_replayed;      /* 1 if the frame's device work was launched as
                                  one replayed CUDA graph                        */
  int32_t paths_sticky;        /* DCEM_MODE_STICKY: valid paths that only the
                                  path cache kept (no ray captured them)         */
  int32_t child_rays;          /* transmission: child rays spawned this frame   */
  int32_t keys_reused;         /* coherent: distinct keys whose validation was
                                  copied from the previous frame               */
  int32_t diff_candidates;     /* diffraction: candidates past the FP32 pre-tests
                                  (all orders), given the exact FP64 test      */
  int32_t diff_pairs;          /* diffraction of order >= 2: wedge pairs that can
                                  start a path (all transmitters)              */
  int32_t diff_triples;        /* diffraction of order 3: wedge triples          */
} dcem_stats;

typedef struct {
  int32_t ptr_kind;     /* DCEM_PTR_HOST / DCEM_PTR_DEVICE for the arrays below */
  int32_t max_paths;    /* capacity of `paths`                                  */
  double* field;        /* links x 2 (re, im) of sum a, or NULL; links = nrx
                           (dcem_trace_frame) or ntx * nrx (dcem_trace_links,
                           link t * nrx + r)                                    */
  double* p_coh_dbm;    /* links: P_t |sum a|^2 in dBm (-inf without paths)    */
  double* p_inc_dbm;    /* links: P_t sum |a|^2 in dBm                         */
  dcem_path* paths;     /* max_paths records ordered by (link, key), or NULL   */
  int32_t n_paths;      /* out: number of valid paths (may exceed max_paths:
                           then DCEM_ERR_CAPACITY and the first max_paths are
                           written)                                             */
  dcem_stats stats;     /* out                                                  */
} dcem_result;

/* Fills `p` with the defaults listed in dcem_params. */
void dcem_params_default(dcem_params* p);

/* Creates a scene on the current CUDA device (Sec. III: BVH built once).
 *   tris     host, ntri*9 floats: v0,v1,v2 of each triangle; world space if
 *            tri_obj[i] < 0, else object space of rigid object tri_obj[i]
 *   tri_mat  host, ntri material indices into mats (0..nmat-1)
 *   mats     host, nmat materials
 *   tri_obj  host, ntri object ids (-1 static, else 0..nobj-1); NULL = all static
 *   nobj     number of rigid objects (>= 0)
 *   stream   cudaStream_t (NULL = legacy default stream)
 *   out      receives the scene handle
 * Objects start at the identity transform until dcem_scene_update_transforms.
 * Errors: DCEM_ERR_ARG, DCEM_ERR_NONFINITE, DCEM_ERR_CUDA, DCEM_ERR_NOMEM. */
int dcem_scene_create(const float* tris, int32_t ntri, const int32_t* tri_mat,
                      const dcem_material* mats, int32_t nmat, const int32_t* tri_obj,
                      int32_t nobj, void* stream, dcem_scene** out);

/* Sets the sampled sphere of ray directions (Sec. III step 1): host, n*3
 * floats of unit vectors, uploaded once and reused every frame. n may be 0
 * and at most 2^27 (DCEM_ERR_ARG above). Invalidates the coherence cache. */
int dcem_scene_set_rays(dcem_scene* s, const float* dirs, int32_t n_rays);

/* Ray sets of several transmitters (Sec. III step 1 for each of them), for
 * dcem_trace_links: host; dirs holds the sets' unit directions one after the
 * other (n_rays[0] + ... + n_rays[ntx-1] rows of 3 floats), and set t is the
 * sampled sphere of transmitter t. Each set keeps its own angular spacing
 * alpha_t = sqrt(4 pi / n_rays[t]) for its reception spheres, so budgets may
 * differ. 1 <= ntx <= 4096, every n_rays[t] >= 1, total <= 2^27
 * (DCEM_ERR_ARG otherwise). dcem_scene_set_rays(s, d, n) is one set of n.
 * Invalidates the coherence cache. */
int dcem_scene_set_ray_sets(dcem_scene* s, const float* dirs, const int32_t* n_rays, int32_t ntx);

/* Per-frame update (Sec. III "Efficient BVH updating"): xf holds nobj
 * row-major 3x4 transforms (host or device per ptr_kind). World vertices are
 * recomputed as fmaf(R0,x, fmaf(R1,y, fmaf(R2,z,t))) per row and the moving
 * objects' hierarchy is refit bottom-up. Asynchronous on the scene stream.
 * Errors: DCEM_ERR_ARG; DCEM_ERR_NONFINITE if a host transform holds NaN/Inf
 * (device transforms are checked on the device and reported by the next
 * dcem_trace_frame). */
int dcem_scene_update_transforms(dcem_scene* s, const float* xf, int32_t ptr_kind);

/* Traces one frame (Sec. III steps 1-4 and 6; coherence reuse when
 * params->mode == DCEM_MODE_COHERENT and the cache is valid):
 *   tx       host, 3 floats
 *   rx       nrx*3 floats (host or device per rx_ptr_kind)
 *   params   host
 *   out      host struct; its arrays are caller-owned (see dcem_result)
 * COHERENT mode falls back to a full retrace (stats.coherent = 0) when the
 * ray set, tx, nrx or the parameters changed since the cached frame. Results
 * equal a full retrace bit for bit. Synchronises the scene stream.
 * Errors: DCEM_ERR_ARG, DCEM_ERR_STATE (no rays set, or more than one ray
 * set), DCEM_ERR_NONFINITE,
 * DCEM_ERR_CAPACITY (out->n_paths holds the required count),
 * DCEM_ERR_STACK, DCEM_ERR_HASH, DCEM_ERR_CUDA. */
int dcem_trace_frame(dcem_scene* s, const float* tx, const float* rx, int32_t nrx,
                     int32_t rx_ptr_kind, const dcem_params* params, dcem_result* out);

/* One frame of ntx transmitters against the same receivers, every
 * transmitter's ray set traced, captured, deduplicated, validated and summed
 * in the same kernel launches (as dcem_trace_frame per transmitter, at once):
 *   tx       host, ntx x 3 floats; ntx equals the scene's number of ray sets
 *   rx       nrx*3 floats (host or device per rx_ptr_kind), shared by all
 *   params   host (tx_power_w applies to every transmitter)
 *   out      per link l = t * nrx + r: field[l], p_coh_dbm[l], p_inc_dbm[l];
 *            path records carry tx and rx and are ordered by (link, key)
 * Transmitter t's paths and power equal those of dcem_trace_frame with tx[t]
 * and set t alone as the scene's rays. ntx * nrx <= 2^24. COHERENT mode
 * reuses the cache when no transmitter, parameter or nrx changed.
 * dcem_trace_frame is this call with ntx = 1 (and requires one ray set).
 * Errors: as dcem_trace_frame; DCEM_ERR_STATE if ntx differs from the
 * scene's ray-set count. */
int dcem_trace_links(dcem_scene* s, const float* tx, int32_t ntx, const float* rx, int32_t nrx,
                     int32_t rx_ptr_kind, const dcem_params* params, dcem_result* out);

/* Quality-driven rebuild of the moving-object hierarchy (Sec. III "Efficient
 * BVH updating": update every frame, rebuild only when the measured
 * degradation warrants it). After every refit the library measures the
 * tree's surface-area cost (sum of node surface areas over the root's); when
 * it exceeds `ratio` times the cost right after the last rebuild, the next
 * dcem_scene_update_transforms rebuilds the tree (LBVH over the current
 * positions) instead of refitting it. ratio <= 0: refit only. Default 1.25.
 * Results never depend on the tree shape. Errors: DCEM_ERR_ARG. */
int dcem_scene_set_rebuild_threshold(dcem_scene* s, float ratio);

/* Transmission (Sec. III "Reflected and transmitted rays"; Table II
 * penetration losses). loss_db[m] >= 0 makes material m transmitting: a ray
 * hitting it both reflects and continues straight through (thin slab, no
 * refraction), and a path's field is scaled by 10^(-loss/20) at each such
 * transmission; loss_db[m] < 0: opaque (the default). max_trans: most
 * transmissions per path (0 = off); max_refl + max_trans <= DCEM_MAX_REFL
 * at trace time. A transmission appears in dcem_path.tri as the id with
 * DCEM_TRI_TRANSMIT set; depth counts reflections and transmissions. With
 * first-order diffraction on, its legs may cross transmitting triangles too
 * (see dcem_scene_set_diffraction). While
 * max_trans > 0 every frame is a full trace (COHERENT and STICKY frames are
 * traced in full). host loss_db, nmat entries (the scene's material count).
 * Errors: DCEM_ERR_ARG, DCEM_ERR_NONFINITE. */
int dcem_scene_set_transmission(dcem_scene* s, const float* loss_db, int32_t nmat, int32_t max_trans);

/* First-order edge diffraction (Sec. III step 5; uniform theory of
 * diffraction after Kouyoumjian & Pathak, Proc. IEEE 1974, with Luebbers'
 * finite-conductivity face factors, IEEE Trans. AP 1984). on = 1 finds the
 * wedges once: edges whose two vertices (identical input coordinates) belong
 * to exactly two triangles of the same rigid object (or both static) with
 * different planes, numbered in the order of their faces' (lower, higher)
 * triangle ids; moving objects' wedges follow their objects. Every
 * frame then adds, for each (link, wedge), the path Tx -> Q -> Rx with Q on
 * the edge by Keller's law, kept when the receiver lies beyond the incident
 * shadow boundary (the paper keeps sources in the receiver's shadow region)
 * and both legs are unoccluded, with its UTD field. Record: depth 1,
 * tri[0] = wedge | DCEM_TRI_DIFFRACT, pts[0] = Q, ray = -1. With transmission
 * on (dcem_scene_set_transmission, max_trans > 0) a leg may instead cross
 * transmitting triangles, at most max_trans (and 9) on the two legs
 * together, the field scaled by 10^(-loss/20) at each; the record then lists
 * the first leg's crossings in order from the transmitter (id |
 * DCEM_TRI_TRANSMIT), the wedge, then the second leg's from Q, depth their
 * count + 1, pts the crossing points and Q in the same order. on = 0 turns it
 * off. *n_wedges (may be NULL): the
 * wedge count. Cost: one thread per (link, wedge) per frame. Errors:
 * DCEM_ERR_ARG, DCEM_ERR_CUDA. */
int dcem_scene_set_diffraction(dcem_scene* s, int32_t on, int32_t* n_wedges);

/* With diffraction on: one reflection before or after the diffraction (Sec.
 * III steps 3-5 combined). on = 1 groups the static triangles into
 * reflector planes once (triangles whose unit normals and offsets agree to
 * 1e-7 and 1e-4 m; normals oriented so that their first nonzero component is
 * positive). Every frame then adds, for each (link, wedge, reflector plane),
 * the path Tx -> P -> Q -> Rx, the diffraction of the transmitter's image in
 * the plane, and the path Tx -> Q -> P -> Rx, the diffraction toward the
 * receiver's image (image theory), with Q on the edge by Keller's law for
 * that image, the receiver (or its image) beyond the incident shadow boundary
 * of the transmitter (or its image), P inside a triangle of the plane (the
 * image is then taken in that triangle's own plane) and the three legs
 * unoccluded; field: the UTD coefficient with the image's distances and the
 * Fresnel reflection at P. Record: depth 2, tri = {P's triangle id,
 * wedge | DCEM_TRI_DIFFRACT} or {wedge | DCEM_TRI_DIFFRACT, triangle id},
 * pts = the two points in path order, ray = -1. on = 0 turns it off.
 * *n_planes (may be NULL): the reflector-plane count. Cost: one pre-test
 * thread per (link, wedge, plane, order) per frame. With diffraction chains
 * on (dcem_scene_set_diffraction_order, max_order m >= 2) the reflection also
 * comes before or after every chain of 2..m wedges: the chain from the
 * transmitter's image or toward the receiver's image in the plane (Keller
 * points, wedge rules and spreading over the unfolded chain), the
 * reflection point inside a triangle of the plane, every real leg
 * unoccluded, Fresnel at the reflection point; record: depth k + 1 with
 * tri = {triangle, wedges...} or {wedges..., triangle}. on = 2 adds, to
 * on = 1, two reflections around a first-order diffraction (the paper's
 * evaluation allows two reflections and one diffraction per path): for each
 * (link, wedge, ordered pair of reflector planes) the paths Tx -> P1 -> P2 ->
 * Q -> Rx, Tx -> P1 -> Q -> P2 -> Rx and Tx -> Q -> P1 -> P2 -> Rx (two
 * reflections in a row on different planes), Q by Keller's law between the
 * transmitter's image in the planes before the wedge (in path order) and the
 * receiver's image in those after it (the last first), the reflection points
 * by unfolding back from Q, each inside a triangle of its plane (the images
 * are then taken in those triangles' own planes), the rules of first-order
 * diffraction on the unfolded path, the four legs unoccluded; field: Fresnel
 * at each reflection in the real directions and the UTD coefficient over the
 * unfolded distances. Record: depth 3, tri = the two triangle ids and
 * wedge | DCEM_TRI_DIFFRACT in path order, pts = the three points. Cost: one
 * warp per (kind, link, plane pair) per frame, its lanes over the wedges.
 * on = 3 adds, to on = 2 and with diffraction chains on (max_order >= 2), a
 * reflection between the two wedges of an order-2 chain: Tx -> Q1 -> P ->
 * Q2 -> Rx, by image theory the chain over the first wedge and the second
 * one's image in the plane toward the receiver's image (Keller points, the
 * chain rules, exterior and shadow rules on that chain), P where its middle
 * leg crosses the plane, inside a triangle of the plane (the images then
 * taken in that triangle's own plane), the four legs unoccluded; field: the
 * UTD coefficients and Fresnel at P, the wavefront's principal directions
 * mirrored there. Record: depth 3, tri = {wedge_1 | DCEM_TRI_DIFFRACT,
 * triangle id, wedge_2 | DCEM_TRI_DIFFRACT}, pts = Q1, P, Q2. Cost: one warp
 * per (transmitter, wedge, plane) forming the pairs, then the chains' pre-test
 * per (pair, receiver). Errors: DCEM_ERR_ARG (on outside 0..3),
 * DCEM_ERR_STATE (diffraction is off), DCEM_ERR_CUDA. */
int dcem_scene_set_diffraction_reflections(dcem_scene* s, int32_t on, int32_t* n_planes);

/* With diffraction on: paths over up to max_order wedges (1, 2 or 3; Sec.
 * III step 5, whose bound is 3 diffractions). For m = 2, 3 every frame adds,
 * for each link and each sequence of m pairwise distinct wedges whose
 * consecutive members share no vertex and do not lie on one line, the path
 * Tx -> Q_1 -> .. -> Q_m -> Rx whose points make the unfolded length
 * stationary (Keller's law at every edge: the minimum of that convex
 * length), kept when every Q_i lies inside
 * its edge, at every wedge the previous and the next point lie in the
 * exterior and the next point beyond the incident shadow boundary of the
 * previous one, neither edge of consecutive wedges lies in a face plane of
 * the other, and every leg is unoccluded (the faces of the wedges at its ends
 * excluded). Field: the UTD coefficient of each wedge applied to the field
 * the previous leg brings, with the astigmatic spreading of an
 * edge-diffracted wave (Kouyoumjian & Pathak 1974, straight edge: a caustic
 * on the edge and one at the arriving wavefront's radius of curvature along
 * the edge). Record: depth m, tri[i] = wedge_i | DCEM_TRI_DIFFRACT, pts[i]
 * = Q_i, ray = -1. Cost per frame: the wedge-pair relation once (one thread
 * per ordered pair, nw * nw bits of device memory), one pre-test thread per
 * (transmitter, wedge pair), for m = 3 per (pair, wedge), then per
 * (sequence, receiver).
 * With reflector planes on (dcem_scene_set_diffraction_reflections) every
 * chain may also have one reflection before or after it. max_order = 1
 * turns the higher orders off. Errors: DCEM_ERR_ARG, DCEM_ERR_STATE
 * (diffraction is off), DCEM_ERR_CUDA. */
int dcem_scene_set_diffraction_order(dcem_scene* s, int32_t max_order);

/* Closest-hit kernel configuration. Results never depend on it (closest hit
 * and lowest-id ties are decided by the triangle test alone):
 *   kernel  -1 automatic (default: 1 when the compact copy and the stacks fit
 *           in shared memory, else 2), 0 binary nodes read from global
 *           memory, 1 the 4-wide compact copy staged in shared memory (768
 *           threads per CTA, one CTA per SM), 2 the 4-wide compact copy read
 *           from global memory
 *   block   threads per CTA of kernels 0 and 2: 64, 128 or 256 (default 256)
 *   stack   shared-memory stack entries per thread of kernels 0 and 2, 8..32
 *           (default 24; deeper traversals continue in a 48-entry local
 *           extension)
 * Errors: DCEM_ERR_ARG (out of range, or kernel 1 or 2 where the scene has no
 * compact copy that fits). */
int dcem_scene_set_trace_config(dcem_scene* s, int32_t kernel, int32_t block, int32_t stack);

/* Autotuner of the closest-hit kernel: traces the given frame (as
 * dcem_trace_links, FULL mode, params otherwise as given) `reps` times
 * (1..16) under each candidate configuration: kernel 1 if it fits, then
 * kernels 2 and 0 with 128 or 256 threads and 16, 24 or 32 stack entries.
 * It times the closest-hit kernel with CUDA events, keeps the fastest
 * (minimum over reps) as the scene's configuration, and returns it in
 * kernel, block and stack (any may be NULL). The scene's transforms should
 * be those of a representative frame. Drops the coherence cache.
 * Errors: as dcem_trace_links (the configuration is then left unchanged). */
int dcem_scene_autotune(dcem_scene* s, const float* tx, int32_t ntx, const float* rx, int32_t nrx,
                        int32_t rx_ptr_kind, const dcem_params* params, int32_t reps, int32_t* kernel,
                        int32_t* block, int32_t* stack);

/* Graph replay of dcem_trace_frame's and dcem_trace_links' device work
 * (default on = 1). The work a frame enqueues (about 16 kernels, memsets,
 * copies and events) is fixed by the scene's buffers, nrx, the traversal and
 * field parameters, the output pointers and whether the frame is coherent;
 * transmitter positions and capture radii are copied in as data. When these
 * equal those of the call two frames earlier (the candidate buffers
 * alternate), the work captured from that call is launched as one CUDA graph
 * instead of operation by operation.
 * Results are identical either way; stats.graph_replayed tells which ran.
 * on = 0 launches every frame operation by operation. Errors: DCEM_ERR_ARG
 * (on not 0 or 1). */
int dcem_scene_set_graph_replay(dcem_scene* s, int32_t on);

/* Drops the coherence cache: the next COHERENT frame is a full retrace. */
int dcem_scene_reset_cache(dcem_scene* s);

/* Changes the stream used by the scene (after synchronising the old one). */
int dcem_scene_set_stream(dcem_scene* s, void* stream);

/* Frees every device and host resource of the scene. NULL is a no-op. */
void dcem_scene_destroy(dcem_scene* s);

/* Static string for a status code. */
const char* dcem_status_string(int status);

/* ---- several scenes per frame ---- */

/* A batch of n distinct scenes traced together. In a frame, every scene's
 * rays (its retrace queue in a coherent frame) are traced by one persistent
 * closest-hit launch that takes chunks of 32 rays of any scene from a shared
 * counter; each scene's preparation before it and its capture, dedupe,
 * validation and reduction after it run concurrently on forked streams, and
 * the whole frame is one CUDA graph once the scenes' plans repeat. The scenes
 * stay owned by the caller, must outlive the batch, and are moved to
 * `stream` (dcem_scene_set_stream).
 * Errors: DCEM_ERR_ARG (null, n < 1, n > 1024, a scene listed twice),
 * DCEM_ERR_CUDA. */
typedef struct dcem_batch dcem_batch;
int dcem_batch_create(dcem_scene* const* scenes, int32_t n, void* stream, dcem_batch** out);

/* Per-frame update of every scene, as dcem_scene_update_transforms(scene i,
 * xf[i], ptr_kind) (xf[i] may be NULL for a scene without moving objects).
 * The scenes' updates run concurrently on streams forked from the batch
 * stream and joined back to it. Host transforms are checked before any work
 * is enqueued. Errors: as dcem_scene_update_transforms. */
int dcem_batch_update_transforms(dcem_batch* b, const float* const* xf, int32_t ptr_kind);

/* One frame of every scene: scene i as dcem_trace_links(scene i, tx[i],
 * ntx[i], rx[i], nrx[i], rx_ptr_kind, params, &out[i]), with bit-identical
 * results. With params->timing == 0 and no scene with transmission, the
 * scenes' rays share one closest-hit launch (stats.trace_kernel = 3), and
 * from the second time the scenes' plans repeat the frame is one graph
 * launch (stats.graph_replayed = 1 in every result); with timing or
 * transmission the scenes' frames are launched one after another. Synchronises
 * the batch stream. Errors: the first failing scene's status, its index in
 * *failed (if not NULL; -1 when all succeed). */
int dcem_batch_trace(dcem_batch* b, const float* const* tx, const int32_t* ntx, const float* const* rx,
                     const int32_t* nrx, int32_t rx_ptr_kind, const dcem_params* params, dcem_result* out,
                     int32_t* failed);

/* Frees the batch (not its scenes). NULL is a no-op. */
void dcem_batch_destroy(dcem_batch* b);

/* ---- introspection (tests and tools; synchronise the scene stream) ---- */

/* Counts of the scene: ntri, nobj, n_rays, internal nodes of the static and
 * dynamic trees. Any pointer may be NULL. */
int dcem_scene_info(const dcem_scene* s, int32_t* ntri, int32_t* nobj, int32_t* n_rays,
                    int32_t* static_nodes, int32_t* dynamic_nodes);

/* Current world-space vertices in input triangle order: host, ntri*9 floats. */
int dcem_scene_get_world_tris(dcem_scene* s, float* out);

/* The hierarchy as flat host arrays, static tree first then dynamic tree:
 *   child   (static_nodes+dynamic_nodes)*2 int32: >= 0 internal node index,
 *           < 0 leaf holding triangle id (-c-1)
 *   bounds  (static_nodes+dynamic_nodes)*12 floats: lo.xyz, hi.xyz of child 0
 *           then child 1 (bit-exact min/max of the children's vertices)
 *   roots   2 int32: root code of the static and dynamic tree (node index,
 *           leaf code as in `child`, or INT32_MIN when the tree is empty) */
int dcem_scene_get_bvh(dcem_scene* s, int32_t* child, float* bounds, int32_t* roots);

/* Per-ray log of the last traced frame: hit_id n_rays*(max_refl+max_trans+1)
 * int32 (triangle id, -1 escaped, -2 not reached; with transmission, the
 * primary rays, which reflect at every hit), hit_t same shape (FP32 ray
 * parameter; +inf when escaped), nseg n_rays. Any pointer may be NULL. */
int dcem_scene_get_ray_log(dcem_scene* s, int32_t* hit_id, float* hit_t, int32_t* nseg);

/* Reception-sphere captures of the last traced frame as (ray, segment, rx)
 * int32 triples in unspecified order (rx: the link t * nrx + r with several
 * transmitters; ray: a transmission child's primary ray). *n receives the
 * count; at most cap triples are written (DCEM_ERR_CAPACITY if cap < count). */
int dcem_scene_get_candidates(dcem_scene* s, int32_t* out, int64_t cap, int64_t* n);

/* ---- received power without device allocation ---- */

/* Number of parameters dcem_path_gradients differentiates by:
 * 2 * (materials) + 2 * (rigid objects). */
int dcem_scene_gradient_size(const dcem_scene* s, int32_t* n_params);

/* Derivatives of the received field over a fixed set of paths (a frame's
 * path topology) with respect to every material's relative permittivity
 * eps_r and conductivity sigma and every rigid object's translation in x and
 * y. The amplitude of each path is recomputed from the scene's current world
 * triangles as in Sec. III steps 3, 4 and 6 -- image sources, back-trace,
 * Fresnel reflection with vector polarisation, the amplitude of Eq. 1 with
 * the spreading of Eq. 3 -- in FP64 with forward-mode derivatives, without
 * the occlusion test (the paths are given). Translating an object moves all
 * its triangles; a material enters through eps_c = eps_r - j sigma/(w eps0).
 *   tx          host, 3 floats
 *   rx          nrx x 3 floats (host or device per rx_ptr_kind)
 *   paths       n_paths records (host or device per ptr_kind) grouped by
 *               receiver in non-decreasing rx order, as dcem_trace_frame
 *               writes them; rx, depth and tri[0..depth) are read (the
 *               paths of the one transmitter tx: their tx field is not read)
 *   params      freq_hz, tx_power_w, pol, max_refl (>= every path's depth)
 *   field       nrx x 2 (re, im) of sum a over the paths, or NULL
 *   dfield      nrx x n_params x 2 (re, im) of d(sum a)/d theta, theta in
 *               the order eps_r(0), sigma(0), eps_r(1), sigma(1), ...,
 *               x(0), y(0), x(1), y(1), ... (materials, then objects)
 *   dpcoh_dbm   nrx x n_params of d P_coh[dBm] / d theta, or NULL
 *               (0 for a receiver without paths)
 * The outputs are host or device per ptr_kind, caller-owned. Perfect
 * conductors have no material derivative. Sums run in path order, so
 * repeated calls give identical results. The call synchronises the scene
 * stream. Errors: DCEM_ERR_ARG (null or out-of-range arguments, paths not
 * grouped by receiver, a depth above max_refl, a triangle id out of range, a
 * triangle sequence without reflection geometry; transmission and
 * diffraction records are not differentiated and are argument errors),
 * DCEM_ERR_NONFINITE, DCEM_ERR_CUDA. */
int dcem_path_gradients(dcem_scene* s, const float* tx, const float* rx, int32_t nrx, int32_t rx_ptr_kind,
                        const dcem_path* paths, int32_t n_paths, const dcem_params* params, int32_t ptr_kind,
                        double* field, double* dfield, double* dpcoh_dbm);

/* The field derivatives of dcem_path_gradients from a hand-written
 * reverse-mode (adjoint) kernel, evaluated at the parameters theta, and the
 * gradient of a loss of the received powers: the field of Sec. III step 6
 * (Eq. 1 with the spreading of Eq. 3) over the fixed paths, differentiated by
 * one backward sweep per path. The kernel keeps only the path's vertices from
 * its forward sweep (FP64 image sources and back-trace) and recomputes each
 * bounce's directions, polarisation basis, Fresnel coefficients and incident
 * field from them during the backward sweep; an object's translation reaches
 * the vertices through the tangent of the image geometry. The cost per path
 * does not grow with the number of parameters.
 *   theta       n_params values, or NULL for the scene's current values:
 *               eps_r, sigma of every material, then the x, y translation of
 *               every rigid object (absolute: an object's triangles are
 *               shifted by theta's translation minus the translation of its
 *               current transform)
 *   pcoh_bar    nrx values d loss / d P_coh[dBm] (a receiver without paths
 *               contributes nothing), or NULL; needed for theta_bar
 *   field       nrx x 2 (re, im) of sum a at theta, or NULL
 *   pcoh_dbm    nrx values P_t |sum a|^2 in dBm at theta (-inf without
 *               paths), or NULL
 *   dfield      nrx x n_params x 2 of d(sum a)/d theta, or NULL
 *   dpcoh_dbm   nrx x n_params of d P_coh[dBm] / d theta, or NULL
 *   theta_bar   n_params values sum_r pcoh_bar[r] d P_coh[r] / d theta
 *               (receivers in order), or NULL
 * theta, pcoh_bar and every output are host or device per ptr_kind and
 * caller-owned; tx, rx, paths, params as in dcem_path_gradients. With theta
 * NULL both calls give the same derivatives up to rounding. Errors: those of
 * dcem_path_gradients, DCEM_ERR_ARG for theta_bar without pcoh_bar,
 * DCEM_ERR_NONFINITE for a non-finite host theta. */
int dcem_path_adjoint(dcem_scene* s, const float* tx, const float* rx, int32_t nrx, int32_t rx_ptr_kind,
                      const dcem_path* paths, int32_t n_paths, const dcem_params* params,
                      const double* theta, const double* pcoh_bar, int32_t ptr_kind, double* field,
                      double* pcoh_dbm, double* dfield, double* dpcoh_dbm, double* theta_bar);

/* Per-receiver sum of given path records, with no device allocation. The
 * paper has no counterpart of this call. It is for callers that cannot
 * allocate device memory when they need the result: a host framework that
 * owns the whole device memory pool, or a real-time loop that must not call
 * cudaMalloc after start-up (an allocation can synchronise the device and
 * stall the loop). The caller passes the inputs and outputs; the scratch
 * lives in one fixed device array of the library (about 310 KB per device,
 * held from the first call on that device until the process exits).
 *   paths      device, n_paths records (e.g. the paths dcem_trace_frame
 *              wrote to a device result); order does not matter
 *   nrx        receivers; every paths[i].rx must lie in [0, nrx) (the
 *              records of one transmitter: paths[i].tx is not read)
 *   tx_power_w transmit power (> 0)
 *   field      device, nrx x 2 (re, im) of sum a, or NULL
 *   p_coh_dbm  device, nrx values of P_t |sum a|^2 in dBm, or NULL
 *   p_inc_dbm  device, nrx values of P_t sum |a|^2 in dBm, or NULL
 *   stream     cudaStream_t of the work (NULL = legacy default stream)
 * The sums use the same order as dcem_trace_frame (paths of a receiver
 * sorted by key; records with equal keys, e.g. one sequence from two
 * transmitters, by their index in `paths`), so the results equal those of
 * the frame for the same records bit for bit and never depend on the
 * scheduling of the device work.
 * Limits: n_paths <= 65536, nrx <= 4096, at most 4096 paths per receiver;
 * beyond them the call returns DCEM_ERR_CAPACITY without touching the GPU
 * (the per-receiver limit is checked on the device).
 * Set-up: the first call on a device looks up the scratch array's device
 * address (cudaGetSymbolAddress) and the kernels' attributes with that device
 * current. A CUDA runtime that loads modules lazily (the default) loads this
 * call's kernels and reserves the scratch array at that moment, which may
 * allocate device memory; so make one set-up call per device at start-up:
 * n_paths = 0 and nrx = 0 (paths may be NULL) does the set-up and nothing
 * else. Calls after it allocate nothing.
 * Every call on a device shares the one scratch array and clears what it
 * needs at its start: calls whose work overlaps on the GPU (for instance on
 * two streams) race, so order them. The call synchronises `stream` before
 * returning, to report device-side errors, so it cannot be recorded into a
 * CUDA graph (no call of it may run while `stream` is capturing).
 * Errors: DCEM_ERR_ARG (null or negative arguments, records but no
 * receivers, a receiver index out of range), DCEM_ERR_CAPACITY,
 * DCEM_ERR_CUDA. */
int dcem_reduce_paths_noalloc(const dcem_path* paths, int32_t n_paths, int32_t nrx, double tx_power_w,
                              double* field, double* p_coh_dbm, double* p_inc_dbm, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DCEM_H */
