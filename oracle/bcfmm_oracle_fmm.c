/*
 * CPU ORACLE (test infrastructure only), part 2: reference FMM "O2".
 *
 * Same discrete operator as orc_direct (see bcfmm_oracle.c), with the far
 * field through the truncated Cartesian Taylor expansion of Sec. 3.3:
 *   lambda^alpha = sum_{|beta| <= p-|alpha|} D^{alpha+beta}G(x_t - x_s)
 *                  / (alpha! beta!) (-1)^{|beta|} m^beta,
 *   m^beta = int (y - x_s)^beta f(y) dy  (by the element point rules).
 * Algorithms 1-3 give the order of the passes: moments in leaves, upward
 * pass (M), interaction phase (T), downward pass (L), evaluation (U), and
 * the near field over the extended neighbour list N* (Sec. 3, Lemma 3.1).
 *
 * The hierarchy is an adaptive octree over the quadrature points (Sec. 2's
 * tet hierarchy replaced by boxes).  Box definitions:
 *   root: centre = midpoint of the bounding box of all element vertices,
 *         half width R0 = largest half extent; level-l box (i,j,k) has side
 *         s = 2 R0 / 2^l and centre lo + (i + 1/2) s per axis, lo = c0 - R0.
 *   a box holding more than Ls points (volume + boundary points together)
 *   is split; a point goes to the child on the upper side of every axis
 *   where its coordinate is >= the box centre; empty children are dropped.
 *   neighbours: same-level boxes B, C with separation ratio
 *         eta(B,C) = (rho_B + rho_C)/|x_B - x_C| > eta0 (Eq. def:sepRatio,
 *         Eq. def:neighbors), rho = sqrt(3)/2 s the box circumradius; with
 *         o = (x_B - x_C)/s this is |o|^2 eta0^2 < 3.  eta0 in (sqrt3/2, 1]
 *         gives the 27 boxes whose closures touch.
 *   interaction list I(B): same-level boxes C, C not a neighbour of B,
 *         parent(C) a neighbour of parent(B).
 *   extended neighbour list N*(b) of a leaf b: all points in the subtrees
 *         of b's neighbours, plus every coarser leaf that is a neighbour of
 *         an ancestor of b.
 * Multi-indices are stored by total degree, then lexicographically.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FOUR_PI 12.566370614359172953850573533118

/* from bcfmm_oracle.c */
void orc_tet_quad(const double *tets, int64_t ntet, double *pts, double *wts);
void orc_tri_quad(const double *tris, int64_t ntri, double *pts, double *wts);
double orc_near_pair(int task, const double *tgt, const double *src,
                     const double *glx, const double *glw, int n, int k);
int orc_is_near(const double *tv, int ntv, const double *sv, int nsv, double eta_ns);
void orc_tri_normal(const double *v, double *n);

/* ------------------------------------------------------------------ */
/* multi-indices                                                        */
/* ------------------------------------------------------------------ */
typedef struct { int P; int n; int (*mi)[3]; int *lut; } MIdx;

static int nterms(int P) { return (P+1)*(P+2)*(P+3)/6; }

static void midx_init(MIdx *M, int P) {
  M->P = P; M->n = nterms(P);
  M->mi = malloc(sizeof(int[3]) * M->n);
  M->lut = malloc(sizeof(int) * (P+1)*(P+1)*(P+1));
  for (int i = 0; i < (P+1)*(P+1)*(P+1); ++i) M->lut[i] = -1;
  int q = 0;
  for (int d = 0; d <= P; ++d)
    for (int a = d; a >= 0; --a)
      for (int b = d - a; b >= 0; --b) {
        int c = d - a - b;
        M->mi[q][0] = a; M->mi[q][1] = b; M->mi[q][2] = c;
        M->lut[(a*(P+1) + b)*(P+1) + c] = q;
        ++q;
      }
}
static void midx_free(MIdx *M) { free(M->mi); free(M->lut); }
static inline int midx(const MIdx *M, int a, int b, int c) {
  if (a < 0 || b < 0 || c < 0 || a+b+c > M->P) return -1;
  return M->lut[(a*(M->P+1) + b)*(M->P+1) + c];
}

static double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

/* b_k(r) = (-1)^{|k|} D^k (1/|r|) / k!  for |k| <= P, by the recurrence
 *   |k| |r|^2 b_k = (2|k|-1) sum_i r_i b_{k-e_i} - (|k|-1) sum_i b_{k-2e_i}
 * (the Taylor-coefficient recurrence of Cartesian treecodes; it follows
 * from |r|^2 grad(1/|r|) = -r/|r| by Leibniz' rule). */
void orc_taylor_b(const double *r, int P, double *out) {
  MIdx M; midx_init(&M, P);
  double r2 = r[0]*r[0] + r[1]*r[1] + r[2]*r[2];
  out[0] = 1.0 / sqrt(r2);
  for (int q = 1; q < M.n; ++q) {
    int k[3] = { M.mi[q][0], M.mi[q][1], M.mi[q][2] };
    int n = k[0] + k[1] + k[2];
    double s1 = 0, s2 = 0;
    for (int i = 0; i < 3; ++i) {
      int k1[3] = { k[0], k[1], k[2] }; k1[i] -= 1;
      int j1 = midx(&M, k1[0], k1[1], k1[2]);
      if (j1 >= 0) s1 += r[i] * out[j1];
      int k2[3] = { k[0], k[1], k[2] }; k2[i] -= 2;
      int j2 = midx(&M, k2[0], k2[1], k2[2]);
      if (j2 >= 0) s2 += out[j2];
    }
    out[q] = ((2.0*n - 1.0) * s1 - (n - 1.0) * s2) / (n * r2);
  }
  midx_free(&M);
}

/* T[alpha][beta] = D^{alpha+beta}G(r) (-1)^{|beta|} / (alpha! beta!)
 *               = (-1)^{|alpha|} C(alpha+beta, alpha) b_{alpha+beta}(r) / (4 pi),
 * zero unless |alpha| + |beta| <= p.  Row-major [np][np]. */
void orc_m2l_matrix(const double *r, int p, double *T) {
  MIdx M2; midx_init(&M2, 2*p);
  MIdx M; midx_init(&M, p);
  double *b = malloc(sizeof(double) * M2.n);
  orc_taylor_b(r, 2*p, b);
  for (int a = 0; a < M.n; ++a) for (int c = 0; c < M.n; ++c) {
    const int *al = M.mi[a], *be = M.mi[c];
    double v = 0.0;
    if (al[0]+al[1]+al[2] + be[0]+be[1]+be[2] <= p) {
      int j = midx(&M2, al[0]+be[0], al[1]+be[1], al[2]+be[2]);
      double sgn = ((al[0]+al[1]+al[2]) & 1) ? -1.0 : 1.0;
      v = sgn * binom(al[0]+be[0], al[0]) * binom(al[1]+be[1], al[1]) * binom(al[2]+be[2], al[2])
          * b[j] / FOUR_PI;
    }
    T[a*M.n + c] = v;
  }
  free(b); midx_free(&M); midx_free(&M2);
}

static double ipow(double x, int n) { double r = 1.0; for (int i = 0; i < n; ++i) r *= x; return r; }

/* moments m^beta = sum_j w_j (y_j - c)^beta */
void orc_p2m(const double *pts, const double *w, int64_t n, const double *c, int p, double *m) {
  MIdx M; midx_init(&M, p);
  for (int q = 0; q < M.n; ++q) m[q] = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double d[3] = { pts[3*j]-c[0], pts[3*j+1]-c[1], pts[3*j+2]-c[2] };
    for (int q = 0; q < M.n; ++q)
      m[q] += w[j] * ipow(d[0], M.mi[q][0]) * ipow(d[1], M.mi[q][1]) * ipow(d[2], M.mi[q][2]);
  }
  midx_free(&M);
}

/* M2M: (y - c_p)^beta = sum_{gamma<=beta} C(beta,gamma) (y-c_c)^gamma (c_c-c_p)^{beta-gamma} */
void orc_m2m(const double *mc, const double *cc, const double *cp, int p, double *mp_acc) {
  MIdx M; midx_init(&M, p);
  double d[3] = { cc[0]-cp[0], cc[1]-cp[1], cc[2]-cp[2] };
  for (int q = 0; q < M.n; ++q) {
    const int *be = M.mi[q];
    double s = 0.0;
    for (int g = 0; g < M.n; ++g) {
      const int *ga = M.mi[g];
      if (ga[0] > be[0] || ga[1] > be[1] || ga[2] > be[2]) continue;
      s += binom(be[0], ga[0]) * binom(be[1], ga[1]) * binom(be[2], ga[2])
           * ipow(d[0], be[0]-ga[0]) * ipow(d[1], be[1]-ga[1]) * ipow(d[2], be[2]-ga[2]) * mc[g];
    }
    mp_acc[q] += s;
  }
  midx_free(&M);
}

/* L2L: (x - c_p)^beta = sum_{alpha<=beta} C(beta,alpha) (x-c_c)^alpha (c_c-c_p)^{beta-alpha} */
void orc_l2l(const double *lp, const double *cp, const double *cc, int p, double *lc_acc) {
  MIdx M; midx_init(&M, p);
  double d[3] = { cc[0]-cp[0], cc[1]-cp[1], cc[2]-cp[2] };
  for (int a = 0; a < M.n; ++a) {
    const int *al = M.mi[a];
    double s = 0.0;
    for (int q = 0; q < M.n; ++q) {
      const int *be = M.mi[q];
      if (al[0] > be[0] || al[1] > be[1] || al[2] > be[2]) continue;
      s += binom(be[0], al[0]) * binom(be[1], al[1]) * binom(be[2], al[2])
           * ipow(d[0], be[0]-al[0]) * ipow(d[1], be[1]-al[1]) * ipow(d[2], be[2]-al[2]) * lp[q];
    }
    lc_acc[a] += s;
  }
  midx_free(&M);
}

double orc_l2p(const double *l, const double *c, int p, const double *x) {
  MIdx M; midx_init(&M, p);
  double d[3] = { x[0]-c[0], x[1]-c[1], x[2]-c[2] }, s = 0.0;
  for (int a = 0; a < M.n; ++a)
    s += l[a] * ipow(d[0], M.mi[a][0]) * ipow(d[1], M.mi[a][1]) * ipow(d[2], M.mi[a][2]);
  midx_free(&M);
  return s;
}

/* ------------------------------------------------------------------ */
/* octree                                                               */
/* ------------------------------------------------------------------ */
typedef struct {
  int level, parent, nkids, kids[8];
  int64_t ijk[3];
  int64_t v0, v1, b0, b1;  /* ranges in the sorted volume / boundary points */
  double c[3], s;
} OBox;

typedef struct {
  OBox *box; int n, cap;
  uint64_t *hkey; int *hval; int64_t hcap;
  double lo[3], R0;
  int64_t *pv, *pb;        /* sorted order -> original point index */
} OTree;

static uint64_t okey(int level, int64_t i, int64_t j, int64_t k) {
  return ((uint64_t)(level + 1) << 57) | ((uint64_t)i << 38) | ((uint64_t)j << 19) | (uint64_t)k;
}
static void hput(OTree *T, uint64_t key, int val) {
  uint64_t h = (key * 0x9E3779B97F4A7C15ull) & (uint64_t)(T->hcap - 1);
  while (T->hkey[h]) h = (h + 1) & (uint64_t)(T->hcap - 1);
  T->hkey[h] = key; T->hval[h] = val;
}
static int hget(const OTree *T, int level, int64_t i, int64_t j, int64_t k) {
  int64_t lim = (int64_t)1 << level;
  if (i < 0 || j < 0 || k < 0 || i >= lim || j >= lim || k >= lim) return -1;
  uint64_t key = okey(level, i, j, k);
  uint64_t h = (key * 0x9E3779B97F4A7C15ull) & (uint64_t)(T->hcap - 1);
  while (T->hkey[h]) { if (T->hkey[h] == key) return T->hval[h]; h = (h + 1) & (uint64_t)(T->hcap - 1); }
  return -1;
}

static int new_box(OTree *T, int level, int parent, const int64_t *ijk) {
  if (T->n == T->cap) { T->cap = T->cap ? 2*T->cap : 1024; T->box = realloc(T->box, sizeof(OBox) * T->cap); }
  OBox *B = &T->box[T->n];
  memset(B, 0, sizeof(*B));
  B->level = level; B->parent = parent;
  B->ijk[0] = ijk[0]; B->ijk[1] = ijk[1]; B->ijk[2] = ijk[2];
  B->s = ldexp(2.0 * T->R0, -level);
  for (int a = 0; a < 3; ++a) B->c[a] = T->lo[a] + ((double)ijk[a] + 0.5) * B->s;
  return T->n++;
}

static void split(OTree *T, int bi, const double *VP, const double *BP, int Ls, int maxlev,
                  int64_t *tmp) {
  OBox B = T->box[bi];
  int64_t cnt = (B.v1 - B.v0) + (B.b1 - B.b0);
  if (cnt <= Ls || B.level >= maxlev) return;
  int64_t vs[9] = {0}, bs[9] = {0};
  /* stable partition of both point classes into octants */
  for (int cls = 0; cls < 2; ++cls) {
    int64_t *perm = cls ? T->pb : T->pv;
    const double *P = cls ? BP : VP;
    int64_t a = cls ? B.b0 : B.v0, e = cls ? B.b1 : B.v1;
    int64_t *st = cls ? bs : vs;
    int64_t c8[8] = {0};
    for (int64_t q = a; q < e; ++q) {
      const double *x = P + 3*perm[q];
      int o = (x[0] >= B.c[0]) | ((x[1] >= B.c[1]) << 1) | ((x[2] >= B.c[2]) << 2);
      c8[o]++;
    }
    st[0] = a;
    for (int o = 0; o < 8; ++o) st[o+1] = st[o] + c8[o];
    int64_t pos[8]; for (int o = 0; o < 8; ++o) pos[o] = st[o];
    for (int64_t q = a; q < e; ++q) {
      const double *x = P + 3*perm[q];
      int o = (x[0] >= B.c[0]) | ((x[1] >= B.c[1]) << 1) | ((x[2] >= B.c[2]) << 2);
      tmp[pos[o]++] = perm[q];
    }
    memcpy(perm + a, tmp + a, sizeof(int64_t) * (e - a));
  }
  for (int o = 0; o < 8; ++o) {
    if (vs[o+1] - vs[o] + bs[o+1] - bs[o] == 0) continue;
    int64_t ijk[3] = { 2*B.ijk[0] + (o & 1), 2*B.ijk[1] + ((o >> 1) & 1), 2*B.ijk[2] + ((o >> 2) & 1) };
    int ci = new_box(T, B.level + 1, bi, ijk);
    T->box[ci].v0 = vs[o]; T->box[ci].v1 = vs[o+1];
    T->box[ci].b0 = bs[o]; T->box[ci].b1 = bs[o+1];
    T->box[bi].kids[T->box[bi].nkids++] = ci;
    split(T, ci, VP, BP, Ls, maxlev, tmp);
  }
}

static void build_tree(OTree *T, const double *VP, int64_t nv, const double *BP, int64_t nb,
                       const double *lo, const double *hi, int Ls) {
  memset(T, 0, sizeof(*T));
  double R0 = 0;
  for (int a = 0; a < 3; ++a) { double h = 0.5 * (hi[a] - lo[a]); if (h > R0) R0 = h; }
  T->R0 = R0;
  for (int a = 0; a < 3; ++a) T->lo[a] = 0.5 * (lo[a] + hi[a]) - R0;
  T->pv = malloc(sizeof(int64_t) * (nv ? nv : 1));
  T->pb = malloc(sizeof(int64_t) * (nb ? nb : 1));
  for (int64_t i = 0; i < nv; ++i) T->pv[i] = i;
  for (int64_t i = 0; i < nb; ++i) T->pb[i] = i;
  int64_t z[3] = {0,0,0};
  int r = new_box(T, 0, -1, z);
  T->box[r].v0 = 0; T->box[r].v1 = nv; T->box[r].b0 = 0; T->box[r].b1 = nb;
  int64_t *tmp = malloc(sizeof(int64_t) * ((nv > nb ? nv : nb) + 1));
  split(T, r, VP, BP, Ls, 18, tmp);
  free(tmp);
  T->hcap = 1; while (T->hcap < 2 * (int64_t)T->n + 16) T->hcap <<= 1;
  T->hkey = calloc(T->hcap, sizeof(uint64_t));
  T->hval = malloc(sizeof(int) * T->hcap);
  for (int i = 0; i < T->n; ++i) hput(T, okey(T->box[i].level, T->box[i].ijk[0], T->box[i].ijk[1], T->box[i].ijk[2]), i);
}

static void free_tree(OTree *T) { free(T->box); free(T->hkey); free(T->hval); free(T->pv); free(T->pb); }

static int is_neighbour(const OBox *A, const OBox *B, double eta0) {
  int64_t o2 = 0;
  for (int a = 0; a < 3; ++a) { int64_t d = A->ijk[a] - B->ijk[a]; o2 += d * d; }
  return (double)o2 * eta0 * eta0 < 3.0;
}

/* all integer offsets o with |o|^2 eta0^2 < 3 */
static int neighbour_offsets(double eta0, int (*off)[3], int cap) {
  int R = (int)floor(sqrt(3.0) / eta0) + 1, n = 0;
  for (int z = -R; z <= R; ++z) for (int y = -R; y <= R; ++y) for (int x = -R; x <= R; ++x) {
    double o2 = (double)(x*x + y*y + z*z);
    if (o2 * eta0 * eta0 < 3.0 && n < cap) { off[n][0] = x; off[n][1] = y; off[n][2] = z; ++n; }
  }
  return n;
}

/* ------------------------------------------------------------------ */
/* O2 driver                                                            */
/* ------------------------------------------------------------------ */
/* task 0 VtV (sources/targets: tet points), 1 VtB (sources tet, targets tri),
 * 2 BtV (sources tri, targets tet), 3 BtV double layer K~ (sources tri with
 * their unit normals n, targets tet; Algorithm 3: the moment of a source
 * point is <gamma_1 (y - c)^beta, g> = w g n . grad_y (y - c)^beta, the near
 * field uses dG/dn_y).  dens: [ndens][nsrc elements].
 * targets: requested target elements; out[ndens][ntargets].
 * stats (optional, int64[8]): nbox, nleaf, maxlevel, n_m2l, n_p2p, 0,0,0.
 * qlev (optional, int[20]): expansion order q_l of level l (Sec. 3.3 uses
 * q_l in the interaction phase; Sec. 4.3, Eq. def:q0, sets
 * q_l = q0 + L - l).  Entries <= 0, or qlev NULL, mean p.  Moments are kept
 * to order p (= the largest q_l) on every level, because a parent's
 * moments of order q_{l-1} need its children's moments of that order; the
 * interaction phase at level l keeps |alpha| + |beta| <= q_l, and the local
 * expansion of a level-l box is truncated to |alpha| <= q_l (a parent's
 * expansion is translated to the child and cut to the child's order). */
static int level_order(const int *qlev, int level, int p) {
  if (!qlev || level >= 20 || qlev[level] <= 0 || qlev[level] > p) return p;
  return qlev[level];
}

int orc_fmm(int task, const double *tets, int64_t ntet, const double *tris, int64_t ntri,
            const double *dens, int ndens, int p, int Ls, double eta0, double eta_ns,
            const double *glx, const double *glw, int n, int k,
            const int64_t *targets, int64_t ntargets, double *out, double *out_fmm_only,
            int nthreads, int64_t *stats, const int *qlev) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  int64_t nvp = 4*ntet, nbp = 3*ntri;
  double *VP = malloc(sizeof(double)*3*(nvp+1)), *VW = malloc(sizeof(double)*(nvp+1));
  double *BP = malloc(sizeof(double)*3*(nbp+1)), *BW = malloc(sizeof(double)*(nbp+1));
  orc_tet_quad(tets, ntet, VP, VW);
  orc_tri_quad(tris, ntri, BP, BW);
  double lo[3] = { INFINITY, INFINITY, INFINITY }, hi[3] = { -INFINITY, -INFINITY, -INFINITY };
  for (int64_t i = 0; i < 4*ntet; ++i) for (int a = 0; a < 3; ++a) {
    double x = tets[3*i+a]; if (x < lo[a]) lo[a] = x; if (x > hi[a]) hi[a] = x; }
  for (int64_t i = 0; i < 3*ntri; ++i) for (int a = 0; a < 3; ++a) {
    double x = tris[3*i+a]; if (x < lo[a]) lo[a] = x; if (x > hi[a]) hi[a] = x; }
  OTree T; build_tree(&T, VP, nvp, BP, nbp, lo, hi, Ls);
  static int noff_cap = 4096;
  int (*NB)[3] = malloc(sizeof(int[3]) * noff_cap);
  int nnb = neighbour_offsets(eta0, NB, noff_cap);

  int src_is_v = (task != 2 && task != 3), tgt_is_v = (task != 1), dl = (task == 3);
  const double *SP = src_is_v ? VP : BP, *SW = src_is_v ? VW : BW;
  const double *TP = tgt_is_v ? VP : BP, *TW = tgt_is_v ? VW : BW;
  const int64_t *sperm = src_is_v ? T.pv : T.pb, *tperm = tgt_is_v ? T.pv : T.pb;
  int nqs = src_is_v ? 4 : 3, nqt = tgt_is_v ? 4 : 3;
  int64_t nsrc_el = src_is_v ? ntet : ntri, ntgt_el = tgt_is_v ? ntet : ntri;
  int64_t nsp = src_is_v ? nvp : nbp, ntp = tgt_is_v ? nvp : nbp;
#define SRANGE(B, a, e) do { a = src_is_v ? (B)->v0 : (B)->b0; e = src_is_v ? (B)->v1 : (B)->b1; } while (0)
#define TRANGE(B, a, e) do { a = tgt_is_v ? (B)->v0 : (B)->b0; e = tgt_is_v ? (B)->v1 : (B)->b1; } while (0)

  MIdx M; midx_init(&M, p);
  int np = M.n;
  /* source point weights per density: W_j = w_j f_{e(j)} */
  double *SWd = malloc(sizeof(double) * ndens * (nsp + 1));
  for (int d = 0; d < ndens; ++d)
    for (int64_t j = 0; j < nsp; ++j) SWd[(int64_t)d*nsp + j] = SW[j] * dens[(int64_t)d*nsrc_el + j/nqs];
  /* double layer: unit normal of each source triangle */
  double *SN = calloc(3 * (size_t)(nsrc_el + 1), sizeof(double));
  if (dl) for (int64_t e = 0; e < nsrc_el; ++e) orc_tri_normal(tris + 9*e, SN + 3*e);
  double *mom = calloc((size_t)T.n * ndens * np, sizeof(double));
  double *loc = calloc((size_t)T.n * ndens * np, sizeof(double));
  double *phi = calloc((size_t)ndens * (ntp + 1), sizeof(double));

  /* moments in leaves, then the upward pass (children are created after
   * their parent, so reverse creation order visits children first) */
#pragma omp parallel for schedule(dynamic, 16)
  for (int bi = 0; bi < T.n; ++bi) {
    OBox *B = &T.box[bi];
    if (B->nkids) continue;
    int64_t a, e; SRANGE(B, a, e);
    for (int64_t q = a; q < e; ++q) {
      int64_t j = sperm[q];
      double dx[3] = { SP[3*j]-B->c[0], SP[3*j+1]-B->c[1], SP[3*j+2]-B->c[2] };
      for (int c = 0; c < np; ++c) {
        const int *be = M.mi[c];
        double mono;
        if (!dl) {
          mono = ipow(dx[0], be[0]) * ipow(dx[1], be[1]) * ipow(dx[2], be[2]);
        } else {
          /* n . grad (y - c)^beta = sum_i n_i beta_i (y - c)^(beta - e_i) */
          const double *nn = SN + 3*(j/nqs);
          mono = 0.0;
          if (be[0]) mono += nn[0] * be[0] * ipow(dx[0], be[0]-1) * ipow(dx[1], be[1]) * ipow(dx[2], be[2]);
          if (be[1]) mono += nn[1] * be[1] * ipow(dx[0], be[0]) * ipow(dx[1], be[1]-1) * ipow(dx[2], be[2]);
          if (be[2]) mono += nn[2] * be[2] * ipow(dx[0], be[0]) * ipow(dx[1], be[1]) * ipow(dx[2], be[2]-1);
        }
        for (int d = 0; d < ndens; ++d) mom[((size_t)bi*ndens + d)*np + c] += SWd[(int64_t)d*nsp + j] * mono;
      }
    }
  }
  for (int bi = T.n - 1; bi > 0; --bi) {
    OBox *B = &T.box[bi];
    OBox *P = &T.box[B->parent];
    for (int d = 0; d < ndens; ++d)
      orc_m2m(mom + ((size_t)bi*ndens + d)*np, B->c, P->c, p, mom + ((size_t)B->parent*ndens + d)*np);
  }
  /* interaction phase */
  int64_t n_m2l = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+:n_m2l)
  for (int bi = 1; bi < T.n; ++bi) {
    OBox *B = &T.box[bi];
    int64_t ta, te; TRANGE(B, ta, te);
    if (ta == te) continue;
    OBox *P = &T.box[B->parent];
    double *Tm = malloc(sizeof(double) * np * np);
    for (int q = 0; q < nnb; ++q) {
      int qi = hget(&T, P->level, P->ijk[0]+NB[q][0], P->ijk[1]+NB[q][1], P->ijk[2]+NB[q][2]);
      if (qi < 0) continue;
      OBox *Q = &T.box[qi];
      for (int c = 0; c < Q->nkids; ++c) {
        OBox *C = &T.box[Q->kids[c]];
        if (is_neighbour(B, C, eta0)) continue;
        int64_t sa, se; SRANGE(C, sa, se);
        if (sa == se) continue;
        double r[3] = { B->c[0]-C->c[0], B->c[1]-C->c[1], B->c[2]-C->c[2] };
        /* order q_l of this level: T of order q (zero unless |a|+|b| <= q),
         * applied to the first nterms(q) moments */
        const int q = level_order(qlev, B->level, p), nq = nterms(q);
        orc_m2l_matrix(r, q, Tm);
        for (int d = 0; d < ndens; ++d) {
          const double *mc = mom + ((size_t)Q->kids[c]*ndens + d)*np;
          double *lb = loc + ((size_t)bi*ndens + d)*np;
          for (int a = 0; a < nq; ++a) {
            double s = 0.0;
            for (int b = 0; b < nq; ++b) s += Tm[a*nq + b] * mc[b];
            lb[a] += s;
          }
        }
        ++n_m2l;
      }
    }
    free(Tm);
  }
  /* downward pass (parents first) */
  for (int bi = 1; bi < T.n; ++bi) {
    OBox *B = &T.box[bi]; OBox *P = &T.box[B->parent];
    const int nq = nterms(level_order(qlev, B->level, p));
    for (int d = 0; d < ndens; ++d) {
      double *lc = loc + ((size_t)bi*ndens + d)*np;
      orc_l2l(loc + ((size_t)B->parent*ndens + d)*np, P->c, B->c, p, lc);
      for (int a = nq; a < np; ++a) lc[a] = 0.0;      /* the child's order */
    }
  }
  /* evaluation and near field in leaves */
  int64_t n_p2p = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+:n_p2p)
  for (int bi = 0; bi < T.n; ++bi) {
    OBox *B = &T.box[bi];
    if (B->nkids) continue;
    int64_t ta, te; TRANGE(B, ta, te);
    if (ta == te) continue;
    /* source ranges of N*(B) */
    int64_t *rng = malloc(sizeof(int64_t) * 2 * nnb * 20); int nr = 0;
    for (int q = 0; q < nnb; ++q) {
      int ci = hget(&T, B->level, B->ijk[0]+NB[q][0], B->ijk[1]+NB[q][1], B->ijk[2]+NB[q][2]);
      if (ci < 0) continue;
      int64_t sa, se; SRANGE(&T.box[ci], sa, se);
      if (sa < se) { rng[2*nr] = sa; rng[2*nr+1] = se; ++nr; }
    }
    int ai = B->parent;
    while (ai >= 0) {
      OBox *A = &T.box[ai];
      for (int q = 0; q < nnb; ++q) {
        int ci = hget(&T, A->level, A->ijk[0]+NB[q][0], A->ijk[1]+NB[q][1], A->ijk[2]+NB[q][2]);
        if (ci < 0 || T.box[ci].nkids) continue;
        int64_t sa, se; SRANGE(&T.box[ci], sa, se);
        if (sa < se) { rng[2*nr] = sa; rng[2*nr+1] = se; ++nr; }
      }
      ai = A->parent;
    }
    for (int64_t q = ta; q < te; ++q) {
      int64_t i = tperm[q];
      const double *x = TP + 3*i;
      for (int d = 0; d < ndens; ++d) {
        double s = 0.0;
        for (int r = 0; r < nr; ++r)
          for (int64_t sq = rng[2*r]; sq < rng[2*r+1]; ++sq) {
            int64_t j = sperm[sq];
            double dd[3] = { x[0]-SP[3*j], x[1]-SP[3*j+1], x[2]-SP[3*j+2] };
            double rr = sqrt(dd[0]*dd[0] + dd[1]*dd[1] + dd[2]*dd[2]);
            if (rr == 0.0) continue;
            if (dl) {
              const double *nn = SN + 3*(j/nqs);
              s += SWd[(int64_t)d*nsp + j] * (nn[0]*dd[0] + nn[1]*dd[1] + nn[2]*dd[2]) / (FOUR_PI * rr * rr * rr);
            } else {
              s += SWd[(int64_t)d*nsp + j] / (FOUR_PI * rr);
            }
          }
        s += orc_l2p(loc + ((size_t)bi*ndens + d)*np, B->c, p, x);
        phi[(int64_t)d*ntp + i] = s;
      }
      for (int r = 0; r < nr; ++r) n_p2p += rng[2*r+1] - rng[2*r];
    }
    free(rng);
  }
  /* Galerkin test sums and near-rule corrections for the requested targets */
  const double *tel = tgt_is_v ? tets : tris, *sel = src_is_v ? tets : tris;
  int nvt = tgt_is_v ? 4 : 3, nvs = src_is_v ? 4 : 3;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t ti = 0; ti < ntargets; ++ti) {
    int64_t t = targets[ti];
    for (int d = 0; d < ndens; ++d) {
      double s = 0.0;
      for (int i = 0; i < nqt; ++i) s += TW[nqt*t + i] * phi[(int64_t)d*ntp + nqt*t + i];
      out[(int64_t)d*ntargets + ti] = s;
      if (out_fmm_only) out_fmm_only[(int64_t)d*ntargets + ti] = s;
    }
    const double *tv = tel + 3*nvt*t;
    for (int64_t s = 0; s < nsrc_el; ++s) {
      const double *sv = sel + 3*nvs*s;
      if (!orc_is_near(tv, nvt, sv, nvs, eta_ns)) continue;
      double a = orc_near_pair(task, tv, sv, glx, glw, n, k);
      double q = 0.0;
      for (int i = 0; i < nqt; ++i) for (int j = 0; j < nqs; ++j) {
        const double *x = TP + 3*(nqt*t + i), *y = SP + 3*(nqs*s + j);
        double dd[3] = { x[0]-y[0], x[1]-y[1], x[2]-y[2] };
        double rr = sqrt(dd[0]*dd[0] + dd[1]*dd[1] + dd[2]*dd[2]);
        if (rr == 0.0) continue;
        if (dl) {
          const double *nn = SN + 3*s;
          q += TW[nqt*t + i] * SW[nqs*s + j] * (nn[0]*dd[0] + nn[1]*dd[1] + nn[2]*dd[2]) / (FOUR_PI * rr * rr * rr);
        } else {
          q += TW[nqt*t + i] * SW[nqs*s + j] / (FOUR_PI * rr);
        }
      }
      for (int d = 0; d < ndens; ++d) out[(int64_t)d*ntargets + ti] += (a - q) * dens[(int64_t)d*nsrc_el + s];
    }
  }
  (void)ntgt_el;
  if (stats) {
    int64_t nleaf = 0, maxl = 0;
    for (int i = 0; i < T.n; ++i) { if (!T.box[i].nkids) ++nleaf; if (T.box[i].level > maxl) maxl = T.box[i].level; }
    stats[0] = T.n; stats[1] = nleaf; stats[2] = maxl; stats[3] = n_m2l; stats[4] = n_p2p;
    stats[5] = stats[6] = stats[7] = 0;
  }
  free(VP); free(VW); free(BP); free(BW); free(SWd); free(SN); free(mom); free(loc); free(phi);
  midx_free(&M); free_tree(&T); free(NB);
  return 0;
}

/* Leaf statistics of the oracle tree (for cross-checking another tree
 * builder): per level the number of boxes and of leaves. */
int orc_tree_stats(const double *tets, int64_t ntet, const double *tris, int64_t ntri, int Ls,
                   int64_t *boxes_per_level /*[20]*/, int64_t *leaves_per_level /*[20]*/) {
  int64_t nvp = 4*ntet, nbp = 3*ntri;
  double *VP = malloc(sizeof(double)*3*(nvp+1)), *VW = malloc(sizeof(double)*(nvp+1));
  double *BP = malloc(sizeof(double)*3*(nbp+1)), *BW = malloc(sizeof(double)*(nbp+1));
  orc_tet_quad(tets, ntet, VP, VW);
  orc_tri_quad(tris, ntri, BP, BW);
  double lo[3] = { INFINITY, INFINITY, INFINITY }, hi[3] = { -INFINITY, -INFINITY, -INFINITY };
  for (int64_t i = 0; i < 4*ntet; ++i) for (int a = 0; a < 3; ++a) {
    double x = tets[3*i+a]; if (x < lo[a]) lo[a] = x; if (x > hi[a]) hi[a] = x; }
  for (int64_t i = 0; i < 3*ntri; ++i) for (int a = 0; a < 3; ++a) {
    double x = tris[3*i+a]; if (x < lo[a]) lo[a] = x; if (x > hi[a]) hi[a] = x; }
  OTree T; build_tree(&T, VP, nvp, BP, nbp, lo, hi, Ls);
  for (int l = 0; l < 20; ++l) boxes_per_level[l] = leaves_per_level[l] = 0;
  for (int i = 0; i < T.n; ++i) {
    boxes_per_level[T.box[i].level]++;
    if (!T.box[i].nkids) leaves_per_level[T.box[i].level]++;
  }
  int n = T.n;
  free(VP); free(VW); free(BP); free(BW); free_tree(&T);
  return n;
}
