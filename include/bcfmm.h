/*
 * bcfmm — boundary-concentrated fast multipole evaluation of the Laplace
 * volume potential on one GB300 (sm_103a).
 *
 * Method: Mohyaddin & Tausch, "A fast method for evaluating volume
 * potentials in the Galerkin boundary element method" (arXiv 2112.00864).
 *
 *   VtV  u_t = int_t  int_Omega G(x,y) f(y) dy dx   for every tet t     (Sec. 1, task 1; Algorithm 1)
 *   VtB  u_g = int_g  int_Omega G(x,y) f(y) dy ds   for every triangle g (task 2; Algorithm 2)
 *   BtV  u_t = int_t  int_Gamma G(x,y) g(y) ds dx   for every tet t      (task 3; Algorithm 3,
 *                                                                         single-layer part)
 * with G(x,y) = 1/(4 pi |x-y|) (Sec. 1.1) and piecewise-constant (P0)
 * densities and test functions (Sec. 1.2, Eq. galerkin:vol with p = 0).
 *
 * Discrete operator (identical to the FP64 CPU oracle's definition):
 *   far element pairs : 4-point tet / 3-point triangle product rule
 *   near element pairs: eta(t,s) = (rho_t + rho_s)/|x_t - x_s| > eta_ns
 *                       (Eq. def:diam, Eq. def:sepRatio with centroids) use
 *                       the near rule: closed-form potential of the uniform
 *                       source element, composite collapsed Gauss-Legendre
 *                       over the target element (near_n nodes per direction,
 *                       near_k uniform refinements).
 * The far field goes through truncated Cartesian Taylor expansions of order
 * p (Sec. 3.3) on an adaptive octree of quadrature points (<= leaf_size
 * points per leaf); same-level boxes are neighbours when their separation
 * ratio exceeds eta0 (Eq. def:neighbors), interaction lists are the children
 * of the parent's neighbours that are not neighbours (Sec. 2), and the near
 * field of a leaf is its extended neighbour list N* (Sec. 3, Lemma 3.1).
 *
 * Conventions for every entry point:
 *  - Return value is a bcfmm_status; nothing throws across this boundary.
 *    On failure, bcfmm_last_error() returns a message (thread-local).
 *  - The caller owns every pointer it passes.  The library copies the mesh
 *    at build time and never keeps a caller pointer after a call returns.
 *  - A context is bound to the CUDA device current at build time and to the
 *    stream given there; all its device work is ordered on that stream.  It
 *    is not thread-safe: one host thread at a time per context.
 *  - Element order in inputs and outputs is the caller's.  Outputs are FP64
 *    in every precision mode.
 */
#ifndef BCFMM_H
#define BCFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bcfmm_ctx bcfmm_ctx;

typedef enum {
  BCFMM_OK = 0,
  BCFMM_ERR_ARG = -1,      /* bad argument (null pointer, size, parameter)      */
  BCFMM_ERR_MESH = -2,     /* degenerate or non-finite element (index in msg)   */
  BCFMM_ERR_CUDA = -3,     /* a CUDA call failed (message holds the CUDA error) */
  BCFMM_ERR_OOM = -4,      /* device or host allocation failed                  */
  BCFMM_ERR_TIMEOUT = -5,  /* a bounded device wait expired                     */
  BCFMM_ERR_STATE = -6     /* call out of order (e.g. eval before set_density)  */
} bcfmm_status;

/* Arithmetic of the evaluation.  Setup (geometry, tree, near rule, tables)
 * is FP64 in every mode. */
typedef enum {
  BCFMM_FP64 = 0,          /* plain: every pass in FP64 on CUDA cores              */
  BCFMM_FP32 = 1,          /* P2P, P2M/M2M/L2L/L2P and M2L in FP32 (CUDA cores); M2L
                              in the Taylor-coefficient form (FP32 products,
                              compensated sums over list chunks)                  */
  BCFMM_FP32_BF16X2 = 2,   /* FP32, M2L on tcgen05 tensor cores, BF16 hi+lo split
                              (hi*hi + hi*lo + lo*hi), FP32 accumulation in TMEM   */
  BCFMM_FP32_BF16X3 = 3    /* as above with a 3-term split (6 products)            */
} bcfmm_precision;

/* Densities: f of VtV/VtB (per tet), the single-layer density q = gamma_1 u
 * of BtV (per triangle) and the double-layer density g = gamma_0 u of BtV
 * (per triangle; contexts built with double_layer = 1).  BtV evaluates
 * <phi_t, V~ q - K~ g> (Algorithm 3, Eq. green:ie:vol). */
typedef enum { BCFMM_VOLUME = 0, BCFMM_BOUNDARY = 1, BCFMM_DIPOLE = 2 } bcfmm_density_kind;

#define BCFMM_MAX_LEVELS 20   /* entries of bcfmm_params.p_level */

typedef struct {
  int32_t p;            /* expansion order (total degree), 0..12; default 6            */
  int32_t leaf_size;    /* max points per octree leaf (tet + triangle points); 64       */
  double eta_ns;        /* near-pair threshold; default 1 - 2^-20 (all touching pairs)  */
  int32_t near_n;       /* near rule: Gauss-Legendre nodes per direction; default 3     */
  int32_t near_k;       /* near rule: uniform refinements of the target; default 1      */
  int32_t precision;    /* bcfmm_precision; default BCFMM_FP64                          */
  int32_t timing;       /* nonzero: record per-stage CUDA-event times of each eval      */
  double eta0;          /* box neighbours: eta = sqrt(3)/|o| > eta0, o the integer offset
                           of two same-level box centres (Eq. def:neighbors applied to
                           boxes); default 0.5 as in Sec. 5; values in (0.866, 1] give the
                           27 boxes whose closures touch; range 0.3..1                  */
  int32_t tc_unit;      /* tensor-core M2L: interaction entries per work unit (one CTA);
                           0 = automatic (about 4 units per SM); 1..4096               */
  int32_t near_mode;    /* near-singular pairs (near pairs whose closures are apart):
                           0 = near rule in FP64 like every near pair (default);
                           1 = learned correction (bcfmm_mlp_* below) wherever the
                               network's calibrated error is <= mlp_tol, the FP64 near
                               rule elsewhere;
                           2 = no correction: product rule only (the reference point
                               the learned correction is measured against)             */
  double mlp_tol;       /* near_mode 1: largest accepted calibrated error of one pair's
                           correction, relative to the pair's product-rule value; 5e-3 */
  const void* mlp_blob; /* near_mode 1: trained network and calibration, format of
                           bcfmm_mlp_blob_size(); read during the build only           */
  int64_t mlp_blob_bytes;
  int32_t p_level[BCFMM_MAX_LEVELS];
                        /* expansion order of each octree level (Sec. 3.3 uses q_l in
                           the interaction phase; Sec. 4.3, Eq. def:q0, sets
                           q_l = q0 + L - l, Sec. 5 uses q0 = 4): the interaction
                           phase of level l keeps |alpha| + |beta| <= q_l and a
                           level-l local expansion has total degree <= q_l (a
                           parent's expansion is cut to the child's order);
                           moments are kept to order p on every level, so p must be
                           >= every q_l.  0 = p (default: uniform order p); 0..p  */
  int32_t q0;           /* > 0: the schedule of Sec. 4.3 (Eq. def:q0) instead of
                           p_level: q_l = min(p, q0 + L - l), L the deepest level of
                           the octree (over every mesh of a batch); 0 = use p_level;
                           0..12                                                    */
  int32_t double_layer; /* 1: BtV also takes the double-layer density (BCFMM_DIPOLE):
                           the build computes the FP64 near-rule corrections of the
                           kernel dG/dn_y (closed-form solid angle of the source
                           triangle, the composite rule of near_n / near_k over the
                           target tet) for BtV's near pairs, whatever near_mode says
                           for the single layer (near_mode 2: none).  Triangle
                           normals follow the right-hand rule of tris (outward).
                           0 = single layer only (default)                          */
} bcfmm_params;

/* Fills *prm with the defaults above.  Never fails. */
void bcfmm_default_params(bcfmm_params* prm);

/*
 * Build the context for one mesh: quadrature points (Sec. 1.2), the octree,
 * interaction and extended neighbour lists (Sec. 2, Sec. 3), the near-pair
 * list and its FP64 corrections N_ts - Q_ts (near rule minus product rule),
 * and the translation tables (Sec. 3.3).
 *   verts  [nvert][3] FP64, host memory
 *   tets   [ntet][4]  int32 vertex ids, host memory (ntet >= 1)
 *   tris   [ntri][3]  int32 vertex ids, host memory (ntri >= 0)
 *   stream cudaStream_t (NULL = legacy default stream) used for all work
 * Errors: BCFMM_ERR_ARG (null pointers, ids out of range, bad params),
 * BCFMM_ERR_MESH (zero-volume tet / zero-area triangle / non-finite
 * coordinate; the element index is in the message), BCFMM_ERR_OOM,
 * BCFMM_ERR_CUDA.  On error *out is NULL.
 */
int bcfmm_build_bc_tree(const double* verts, int64_t nvert,
                        const int32_t* tets, int64_t ntet,
                        const int32_t* tris, int64_t ntri,
                        const bcfmm_params* prm, void* stream, bcfmm_ctx** out);

/*
 * Build one context for a batch of nmesh independent meshes (the paper
 * treats one mesh at a time; a batch is that computation for every mesh,
 * with no interaction between meshes).  Each mesh gets its own octree,
 * lists and near pairs exactly as bcfmm_build_bc_tree would build them;
 * the library then concatenates them into one forest so that every stage
 * of an evaluation is one launch over all meshes.
 *   verts     [vert_off[nmesh]][3] FP64, mesh m's vertices at rows
 *             vert_off[m] .. vert_off[m+1]-1
 *   tets      [tet_off[nmesh]][4] int32 vertex ids LOCAL to the mesh
 *   tris      [tri_off[nmesh]][3] int32 local vertex ids (may be NULL when
 *             tri_off[nmesh] == 0)
 *   vert_off, tet_off, tri_off  [nmesh+1] prefix sums starting at 0; every
 *             mesh has >= 1 vertex and >= 1 tet, triangles may be absent
 * All arrays are host memory.  Densities and outputs of the context are
 * the concatenation over meshes: [ndens][tet_off[nmesh]] for volume
 * quantities, [ndens][tri_off[nmesh]] for boundary ones, mesh m's
 * elements at columns tet_off[m] .. tet_off[m+1]-1 (tri_off likewise).
 * Errors as bcfmm_build_bc_tree; the message names the failing mesh.
 */
int bcfmm_build_batch(const double* verts, const int64_t* vert_off,
                      const int32_t* tets, const int64_t* tet_off,
                      const int32_t* tris, const int64_t* tri_off, int32_t nmesh,
                      const bcfmm_params* prm, void* stream, bcfmm_ctx** out);

/*
 * Build a context on the same meshes as `base` with other tree, expansion
 * or precision parameters (p, leaf_size, eta0, precision, tc_unit, timing).
 * The near pairs and their corrections do not depend on those parameters
 * and are copied from `base` on the device instead of being recomputed, so
 * an autotuner can try many configurations for the price of the tree and
 * list builds.  eta_ns, near_n, near_k and near_mode must equal base's.
 * The new context uses base's stream; base stays valid and independent.
 * Errors: BCFMM_ERR_ARG (mismatching near-pair parameters), BCFMM_ERR_STATE
 * (base's device is not current), as bcfmm_build_bc_tree otherwise.
 */
int bcfmm_build_like(const bcfmm_ctx* base, const bcfmm_params* prm, bcfmm_ctx** out);

/*
 * Set the P0 density coefficients (one value per element, Sec. 1.2).
 *   kind   BCFMM_VOLUME: vals [ndens][ntet] (f of VtV/VtB);
 *          BCFMM_BOUNDARY: vals [ndens][ntri] (single layer q of BtV);
 *          BCFMM_DIPOLE: vals [ndens][ntri] (double layer g of BtV; the
 *          context must be built with double_layer = 1; its ndens must
 *          equal the single layer's when BtV runs; vals = NULL with
 *          ndens = 0 removes it)
 *   vals   FP64; device memory if is_device != 0 (read on the context's
 *          stream before this call returns control of the buffer to the
 *          stream order), else host memory (copied synchronously)
 *   ndens  number of densities evaluated together, 1..16
 * Errors: BCFMM_ERR_ARG, BCFMM_ERR_MESH (non-finite value), BCFMM_ERR_CUDA.
 */
int bcfmm_set_density(bcfmm_ctx* ctx, int32_t kind, const double* vals,
                      int32_t ndens, int32_t is_device);

/*
 * Evaluate one task (Algorithms 1, 2, 3).  The work is enqueued on the
 * context's stream.
 *   out    FP64 [ndens][ntet] (VtV, BtV) or [ndens][ntri] (VtB); device memory
 *          if out_is_device != 0 (written asynchronously on the stream),
 *          else host memory (the call synchronises the stream before return)
 * Errors: BCFMM_ERR_STATE (density of the needed kind not set),
 * BCFMM_ERR_ARG, BCFMM_ERR_CUDA.
 */
int bcfmm_eval_vtv(bcfmm_ctx* ctx, double* out, int32_t out_is_device);
int bcfmm_eval_vtb(bcfmm_ctx* ctx, double* out, int32_t out_is_device);
int bcfmm_eval_btv(bcfmm_ctx* ctx, double* out, int32_t out_is_device);
/* BtV output: <phi_t, V~ q> for the boundary density q, minus <phi_t, K~ g>
 * when a double-layer density g is set (BCFMM_DIPOLE): the moments take
 * <gamma_1 (y - c)^beta, g> (Algorithm 3), the near field dG/dn_y
 * (FP32 or FP64 as the precision says) and the element sums the FP64
 * double-layer corrections.  BCFMM_ERR_STATE: g set with a different
 * ndens than q. */

/*
 * Evaluate the tasks in task_mask (bit 0 VtV, bit 1 VtB, bit 2 BtV) as one
 * CUDA graph launch on the context's stream (the paper evaluates tasks one
 * by one; the graph removes the per-kernel launch overhead of the many
 * small per-level stages).  Outputs as in bcfmm_eval_*, device memory only;
 * a pointer whose bit is clear is ignored.  When VtV and VtB are both in
 * the mask, VtB reuses VtV's weights, upward pass and local expansions (same
 * density and source points: the same interaction lists; VtV's far field
 * covers every box with tet or triangle points), so VtB adds only its near
 * field, L2P and element sums.
 * The first call for a given (mask, output pointers, density counts, work
 * buffers) combination captures and instantiates the graph on a stream the
 * library owns (this allocates); later calls with the same combination
 * only launch it.  Densities may change between calls through
 * bcfmm_set_density (the graph reads the context's density buffer).
 * Expired bounded device waits are reported through bcfmm_stats
 * ("device_error"), not by this call.
 * Errors: BCFMM_ERR_ARG (mask, null output), BCFMM_ERR_STATE (density not
 * set), BCFMM_ERR_CUDA (capture or instantiation failed).
 */
int bcfmm_eval_graph(bcfmm_ctx* ctx, int32_t task_mask, double* out_vtv, double* out_vtb, double* out_btv);

/*
 * Evaluate one task (0 = VtV, 1 = VtB, 2 = BtV) for ONE density without
 * allocating any memory.  For callers that must not call the CUDA allocator
 * during evaluation: a host framework that owns and budgets all device
 * memory itself, or a latency-critical loop where cudaMalloc/cudaFree could
 * synchronise the device.  The paper has no counterpart; this is a
 * deployment variant of the FP32 evaluation (precision BCFMM_FP32 or a
 * BF16 split).
 *   dens_dev  FP64 device array, one P0 value per source element (tets for
 *             VtV/VtB, triangles for BtV: the single layer only, a
 *             double-layer density set on the context is not used);
 *             read on the context's stream
 *   out_dev   FP64 device array, one value per target element; written
 *             asynchronously on the context's stream
 * The M2L keeps its partial sums (tensor cores: per work unit; Taylor
 * form: per list chunk) in a fixed static device array of 64 MiB (every GPU that loads the library holds it until
 * the process exits) instead of the context's scratch; all other buffers
 * are the context's, sized by an earlier bcfmm_set_density (required once).
 * The first call on a device looks up that array's device address (a
 * one-time set-up, per device); make that first call before any stream
 * capture.  The address is kept for the life of the process, so a device
 * reset (cudaDeviceReset, or a reset of the primary context) after the
 * first call on that device is not supported.  Every call on a device
 * shares the array and overwrites it completely, so nothing carries over
 * between calls, and calls that overlap on the GPU (different streams or
 * contexts on one device) race on it.
 * The call does not synchronise: an expired bounded device wait of the
 * tensor-core M2L shows only in bcfmm_stats ("device_error") and is
 * returned, and cleared, by the next evaluation with host output.  The
 * call records no stage timings.
 * Errors: BCFMM_ERR_ARG (null pointer, bad task, context built with
 * precision BCFMM_FP64, or a mesh whose M2L needs more scratch than the
 * array holds: the message gives both sizes), BCFMM_ERR_STATE (no earlier
 * bcfmm_set_density, or the current device is not the context's),
 * BCFMM_ERR_CUDA.
 */
int bcfmm_eval_noalloc(bcfmm_ctx* ctx, int32_t task, const double* dens_dev, double* out_dev);

/*
 * The discrete operator itself, summed pair by pair in FP64 on the GPU for
 * the target elements targets[0..n): every source quadrature point with
 * the product rule (r = 0 skipped) plus the element's near corrections,
 * no expansions.  It is the reference the fast evaluation approximates,
 * at O(n * #source points) cost; the autotuner measures errors against it.
 *   targets  host int64 [n] element indices of the task's target kind, n <= 2^20
 *   out      host FP64 [ndens][n]; the call synchronises the stream
 * Errors: BCFMM_ERR_ARG (index out of range), BCFMM_ERR_STATE (density
 * not set), BCFMM_ERR_CUDA.
 */
int bcfmm_direct_sample(bcfmm_ctx* ctx, int32_t task, const int64_t* targets, int64_t n, double* out);

/*
 * Learned correction of near-singular pairs (bcfmm_params.near_mode 1).
 * The paper computes every near pair with an accurate rule; this optional
 * path replaces the rule, for pairs whose closures are apart, by a small
 * network trained on the GPU with the kernels below.
 *
 * Pair features (12): the source vertices in the affine frame of the target
 * (target vertices t0..t3, frame columns t1-t0, t2-t0, t3-t0; a triangle
 * target uses its unit normal times sqrt(2 area) on the source's side as
 * the third column), centred at the target centroid; both vertex orders
 * ascending in distance to the other element's centroid; a triangle
 * source fills 9 slots, the rest 0.
 * qhat (16): product-rule terms q_ij = W_i W_j / (4 pi r_ij) in those
 * orders (i target point, j source point, [4][4], unused slots 0) over their
 * sum Q.  Network 12 -> 64 -> 64 -> 16 (exact GELU), output dw; the pair's
 * correction is Q * sum_k dw_k qhat_k.  Parameters, FP32 [6032]:
 * W1[64][12] b1[64] W2[64][64] b2[64] W3[16][64] b3[16]; the kernels compute
 * with their BF16 roundings and FP32 accumulation.
 * Blob (bcfmm_mlp_blob_size() bytes): uint32 header {0x4C4D4342, 1, 6032,
 * 32, has_vtv, has_vtb, has_btv, 0}, then per task params[6032] and the
 * calibrated error of each of 32 geometric bins, float32.
 * All pointers below are device memory unless stated; stream is a
 * cudaStream_t (NULL = legacy default stream).
 */
int64_t bcfmm_mlp_blob_size(void);

/* Training data from a context built with near_mode 1 or 2: up to max_pairs
 * of its near-singular pairs of `task`, evenly spaced in CSR order.
 *   feat [max][12], qhat [max][16], chat [max] FP32: label (N - Q) / Q with
 *   N the FP64 near rule; bin [max] int32 calibration bin; pairs [max][2]
 *   int32 (target, source) element indices; *n_out (host) pairs written.
 * Synchronises the context's stream.
 * Errors: BCFMM_ERR_STATE (context built with near_mode 0), BCFMM_ERR_ARG. */
int bcfmm_mlp_dataset(bcfmm_ctx* ctx, int32_t task, int64_t max_pairs, float* feat, float* qhat, float* chat,
                      int32_t* bin, int32_t* pairs, int64_t* n_out);

/* grad[6032] and loss[1] (both zeroed first) of the mean over n pairs of
 * (sum_k dw_k qhat_k - chat)^2, gradient with respect to the BF16-rounded
 * parameters (applied to the FP32 masters by bcfmm_mlp_adam). */
int bcfmm_mlp_grad(const float* params, const float* feat, const float* qhat, const float* chat, int64_t n,
                   float* grad, float* loss, void* stream);

/* One Adam step (step >= 1, bias-corrected) on the FP32 masters. */
int bcfmm_mlp_adam(float* params, const float* grad, float* m1, float* m2, int32_t step, float lr, float beta1,
                   float beta2, float eps, void* stream);

/* out[n] = sum_k dw_k qhat_k for each pair (inference on BF16 weights). */
int bcfmm_mlp_predict(const float* params, const float* feat, const float* qhat, int64_t n, float* out,
                      void* stream);

/*
 * Context statistics as one JSON object (points, boxes, levels, list sizes,
 * near pairs, setup seconds, last eval's stage times in ms when timing is
 * on).  Writes at most cap bytes including the terminating NUL.
 * Errors: BCFMM_ERR_ARG (null, or cap too small: the message gives the size).
 */
int bcfmm_stats(const bcfmm_ctx* ctx, char* json, size_t cap);

/* Message of the last failed call on this host thread ("" if none). */
const char* bcfmm_last_error(void);

/* Release every resource of the context (synchronises its stream). NULL is a no-op. */
void bcfmm_destroy(bcfmm_ctx* ctx);

/*
 * Test hook: the box-scaled M2L matrix of Sec. 3.3 that the library uses,
 * for offset o = (x_t - x_s)/s between same-level box centres (o integer in
 * use; any nonzero o accepted here):
 *   T[a][b] = D^{a+b}G(o) (-1)^{|b|} / (a! b!),   G = 1/(4 pi |.|),
 * for |a| + |b| <= p (zero otherwise), multi-indices ordered by total
 * degree, then lexicographically descending.  T: host [np][np], np =
 * (p+1)(p+2)(p+3)/6.  Errors: BCFMM_ERR_ARG.
 */
int bcfmm_debug_m2l_matrix(int32_t p, const double* o, double* T);

/*
 * Test hook: the per-offset coefficients of the Taylor-form M2L (precision
 * BCFMM_FP32), g[gamma] = D^gamma G(o) for |gamma| <= q (same multi-index
 * order), from which the kernel rebuilds the matrix above as
 *   T[a][b] = g[a + b] (-1)^{|b|} / (a! b!),   |a| + |b| <= q.
 * The kernel stores them in FP32.  g: host [(q+1)(q+2)(q+3)/6].
 * Errors: BCFMM_ERR_ARG.
 */
int bcfmm_debug_m2l_taylor_coeffs(int32_t q, const double* o, double* g);

/*
 * Test hook: the box-scaled shift of Sec. 3.3 between a parent box and its
 * child in octant `octant` (bit 0 x, bit 1 y, bit 2 z set: the child lies on
 * the + side; child centre = parent centre +- s/4, child side s/2).
 *   kind 0 (M2M): mhat_parent[b] += sum_g out[b][g] mhat_child[g]
 *   kind 1 (L2L): lhat_child[a]  += sum_b out[a][b] lhat_parent[b]
 * with moments scaled by s^-|beta| and locals by s^|alpha| (s the box's
 * own side), multi-indices ordered as for bcfmm_debug_m2l_matrix.
 * out: host [np][np].  Errors: BCFMM_ERR_ARG.
 */
int bcfmm_debug_shift_matrix(int32_t kind, int32_t p, int32_t octant, double* out);

/*
 * Test hook for the failure path of the bounded device waits (the paper has
 * no counterpart): enqueues on the context's stream one thread that waits,
 * through the same bounded mbarrier wait the tensor-core M2L uses, on a
 * barrier whose expected arrival never comes, giving up after `spins`
 * polls (1..2^20).  It then sets the context's device error word, exactly
 * as an expired wait inside an evaluation would: the next evaluation with
 * host output returns BCFMM_ERR_TIMEOUT and clears the word, and the
 * context stays usable.  Nothing faults, traps or hangs.
 */
int bcfmm_debug_expire_wait(bcfmm_ctx* ctx, int32_t spins);

/*
 * Measured FP32 FMA throughput of CUDA device `device` (flop/s, an FMA
 * counted as 2): a probe kernel of independent FMA chains on every SM,
 * timed with CUDA events (best of three after a warm-up, ~ms).  The paper
 * has no counterpart; it is the denominator check for the roofline of
 * the CUDA-core passes.  flops: host double.  Synchronises the device.
 * Errors: BCFMM_ERR_ARG, BCFMM_ERR_CUDA.
 */
int bcfmm_measure_ffma(int32_t device, double* flops);

/*
 * Test hook, host only (no GPU, no context): boxes and leaves per level of
 * the octree the build makes for one mesh with the given leaf size (root =
 * bounding cube of the vertices; a box holding more than leaf_size points
 * of both classes is split; a point goes to the upper child where its
 * coordinate is >= the box centre).  boxes, leaves: host int64 [nlev_cap].
 * Errors: BCFMM_ERR_ARG (also when the tree is deeper than nlev_cap).
 */
int bcfmm_debug_tree_counts(const double* verts, int64_t nvert, const int32_t* tets, int64_t ntet,
                            const int32_t* tris, int64_t ntri, int32_t leaf_size, int64_t* boxes, int64_t* leaves,
                            int32_t nlev_cap);

/*
 * Test hook, host only (no GPU, no context): the near element pairs the
 * build finds for one mesh and task (eta(t,s) > eta_ns, Eq. def:sepRatio
 * with centroids and largest vertex distances), as a CSR over target
 * elements with ascending source indices.
 *   row_off  host int64 [ntarget + 1] (ntet for VtV/BtV, ntri for VtB)
 *   cols     host int32 [cap]; *nnz receives the pair count
 * Errors: BCFMM_ERR_ARG (also when cap < pair count: *nnz and row_off are
 * filled, cols is not), BCFMM_ERR_MESH.
 */
int bcfmm_debug_near_pairs(const double* verts, int64_t nvert, const int32_t* tets, int64_t ntet,
                           const int32_t* tris, int64_t ntri, double eta_ns, int32_t task, int64_t cap,
                           int64_t* row_off, int32_t* cols, int64_t* nnz);

/*
 * Test hook, host only (no GPU, no context): builds the octree and lists of
 * the meshes exactly as bcfmm_build_batch does (one mesh: nmesh = 1; same
 * array conventions) and checks the FMM's covering of the interactions
 * (Sec. 2 and Sec. 3: near field N* plus the interaction lists of a leaf
 * and its ancestors).  out (host): out[0..2], per task (VtV, VtB, BtV),
 * the number of (target leaf, source point) pairs not covered exactly once,
 * counting a source point of another mesh of a batch as one that must not
 * be covered (0: every pair is evaluated once, by P2P or by one M2L);
 * out[3..5], per task, the interaction-list entries that the tensor-core
 * tiles (128 target rows of one expansion order, one source box per row and
 * offset) miss, duplicate or invent, plus rows whose order differs from the
 * tile's (0: the tiles reproduce every list exactly); out[6..8], per task,
 * the faults of the tensor-core schedule built for 1, 7 and 152 SMs (an
 * entry not in exactly one unit, a unit not exactly once in one CTA's
 * sequence, wrong first / last flags, partial slots of cut tiles not
 * consecutive); out[9..11], per task, the faults of the Taylor-form M2L
 * schedule built for 1, 7 and 152 SMs (a list entry of a target of order
 * 1..7 missing, duplicated, invented or in a lane whose chunk is another
 * target's; a chunk not in exactly one lane; a target of another order not
 * exactly once in the generic kernel's list); out[12..14], per task, the
 * faults of the packed FP32 near field's blocks built with chunks of 96
 * points and of the library's 8192 (a source point of a leaf's list in no
 * chunk or in two, a chunk over its size, the leaf's own run not whole at
 * the front of chunk 0, scratch rows not one per chunk, work increasing
 * along the block order).  out: host int64 [15].
 * Errors: BCFMM_ERR_ARG, BCFMM_ERR_MESH.
 */
int bcfmm_debug_list_coverage(const double* verts, const int64_t* vert_off, const int32_t* tets,
                              const int64_t* tet_off, const int32_t* tris, const int64_t* tri_off, int32_t nmesh,
                              const bcfmm_params* prm, int64_t* out);

#ifdef __cplusplus
}
#endif
#endif /* BCFMM_H */
