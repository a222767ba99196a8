/*
 * CPU ORACLE (test infrastructure only) for the boundary-concentrated FMM of
 * Mohyaddin & Tausch, "A fast method for evaluating volume potentials in the
 * Galerkin boundary element method" (arXiv 2112.00864).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code with the CUDA path.  Everything is
 * plain FP64, written for readability, not speed (OpenMP over targets only).
 *
 * Kernel G(x,y) = 1/(4 pi |x-y|) (Sec. 1.1).  P0 (piecewise-constant)
 * Galerkin discretisation (Sec. 1.2): u_t = sum_s A_ts f_s with
 * A_ts = int_t int_s G.  Task 3 is the double-layer part of BtV
 * (Algorithm 3, the term K~[gamma_0 u] of Eq. green:ie:vol): kernel
 * dG/dn_y(x,y) = n_s.(x-y) / (4 pi |x-y|^3), n_s the unit normal of the
 * source triangle by the right-hand rule (outward for the meshes used).
 * The discrete operator the method approximates:
 *   far pairs  : product rule Q_ts = sum_i sum_j W_i W_j G(x_i, y_j)
 *                (4-point tet rule, 3-point triangle rule; the self point
 *                 x_i == y_j of a coincident pair is skipped)
 *   near pairs : the near rule N_ts (closed-form inner potential of the
 *                uniform source element, fixed composite Gauss outer rule)
 *   near       : eta(t,s) = (rho_t + rho_s)/|x_t - x_s| > eta_ns, with
 *                centre = centroid and rho = max vertex distance (Eq. def:diam,
 *                Eq. def:sepRatio).
 *
 * O1 (orc_direct): the definition above, pair by pair.
 * O2 (orc_fmm): the same operator with the far field through Cartesian Taylor
 *   expansions, following Algorithm 1 (VtV), Algorithm 2 (VtB) and
 *   Algorithm 3 (BtV, single layer) on an adaptive octree of quadrature
 *   points: moments (Sec. 3.3), upward pass M, interaction phase T, downward
 *   pass L, evaluation U, and the near field over the extended neighbour
 *   lists N* (Sec. 3, Lemma 3.1), plus the near-rule corrections.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FOUR_PI 12.566370614359172953850573533118

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */
static inline void sub3(const double *a, const double *b, double *o) { o[0]=a[0]-b[0]; o[1]=a[1]-b[1]; o[2]=a[2]-b[2]; }
static inline double dot3(const double *a, const double *b) { return a[0]*b[0]+a[1]*b[1]+a[2]*b[2]; }
static inline void cross3(const double *a, const double *b, double *o) {
  o[0]=a[1]*b[2]-a[2]*b[1]; o[1]=a[2]*b[0]-a[0]*b[2]; o[2]=a[0]*b[1]-a[1]*b[0];
}
static inline double norm3(const double *a) { return sqrt(dot3(a,a)); }

double orc_tet_volume(const double *v /*[4][3]*/) {
  double a[3], b[3], c[3], n[3];
  sub3(v+3, v, a); sub3(v+6, v, b); sub3(v+9, v, c);
  cross3(a, b, n);
  return fabs(dot3(n, c)) / 6.0;
}
double orc_tri_area(const double *v /*[3][3]*/) {
  double a[3], b[3], n[3];
  sub3(v+3, v, a); sub3(v+6, v, b); cross3(a, b, n);
  return 0.5 * norm3(n);
}

/* ------------------------------------------------------------------ */
/* Closed-form potential of a flat triangle: I(x) = int_T ds_y / |x-y|.  */
/* Derivation (in-plane divergence theorem): with w the height of x     */
/* over the plane, rho its projection and s = |y - rho|, the field       */
/* F = (y-rho)(R-|w|)/s^2 has in-plane divergence 1/R, R = |x-y|.  On an */
/* edge with outward in-plane normal m the flux is                        */
/*   d [ln(t+R)] + |w| [atan(t|w|/(dR)) - atan(t/d)],  d = (y-rho).m,    */
/* and the atan terms summed over the edges give minus |w| times the     */
/* solid angle of T seen from x.                                          */
/* ------------------------------------------------------------------ */
double orc_tri_potential(const double *x, const double *v /*[3][3]*/) {
  const double *P[3] = { v, v+3, v+6 };
  double e1[3], e2[3], n[3];
  sub3(P[1], P[0], e1); sub3(P[2], P[0], e2); cross3(e1, e2, n);
  double nn = norm3(n);
  n[0]/=nn; n[1]/=nn; n[2]/=nn;
  double xv[3]; sub3(x, P[0], xv);
  double w = dot3(xv, n);
  double rho[3] = { x[0]-w*n[0], x[1]-w*n[1], x[2]-w*n[2] };
  double acc = 0.0;
  double scale = sqrt(nn);  /* a length scale of the triangle */
  for (int e = 0; e < 3; ++e) {
    const double *A = P[e], *B = P[(e+1)%3];
    double t[3]; sub3(B, A, t);
    double L = norm3(t);
    t[0]/=L; t[1]/=L; t[2]/=L;
    double m[3]; cross3(t, n, m);          /* outward in-plane normal (ccw w.r.t. n) */
    double ar[3]; sub3(A, rho, ar);
    double d = dot3(ar, m);
    if (fabs(d) <= 1e-14 * scale) continue;   /* projection on the edge line: zero flux */
    double ax[3], bx[3]; sub3(A, x, ax); sub3(B, x, bx);
    double t1 = dot3(ax, t), t2 = dot3(bx, t);   /* = (A-rho).t, (B-rho).t */
    double R1 = norm3(ax), R2 = norm3(bx);
    double lg;
    if (t1 + t2 >= 0.0) lg = log((R2 + t2) / (R1 + t1));
    else                lg = log((R1 - t1) / (R2 - t2));
    acc += d * lg;
  }
  /* solid angle (Van Oosterom & Strackee) */
  double r1[3], r2[3], r3[3], c23[3];
  sub3(P[0], x, r1); sub3(P[1], x, r2); sub3(P[2], x, r3);
  double l1 = norm3(r1), l2 = norm3(r2), l3 = norm3(r3);
  cross3(r2, r3, c23);
  double num = dot3(r1, c23);
  double den = l1*l2*l3 + dot3(r1,r2)*l3 + dot3(r1,r3)*l2 + dot3(r2,r3)*l1;
  double omega = 2.0 * atan2(num, den);
  acc -= fabs(w) * fabs(omega);
  return acc;
}

/* Double-layer potential of the flat triangle with unit density:
 *   int_T n.(x-y)/|x-y|^3 ds_y = Omega(x),
 * the solid angle T subtends at x, signed: positive when x lies on the side
 * the normal n = (v1-v0) x (v2-v0) points to (for y in the plane,
 * n.(x-y) is the height w of x).  Van Oosterom & Strackee give
 * tan(Omega_u/2) = r1.(r2 x r3) / (l1 l2 l3 + (r1.r2) l3 + (r1.r3) l2 +
 * (r2.r3) l1), r_i = v_i - x, l_i = |r_i|; for x at height w > 0 the
 * triple product r1.(r2 x r3) = -w |(v1-v0) x (v2-v0)| is negative, so the
 * signed angle is minus twice the atan2 of that quotient.  Over a closed
 * outward-oriented surface the angles add up to -4 pi inside, 0 outside. */
double orc_tri_solid_angle(const double *x, const double *v /*[3][3]*/) {
  double r1[3], r2[3], r3[3], c23[3];
  sub3(v, x, r1); sub3(v+3, x, r2); sub3(v+6, x, r3);
  double l1 = norm3(r1), l2 = norm3(r2), l3 = norm3(r3);
  cross3(r2, r3, c23);
  double num = dot3(r1, c23);
  double den = l1*l2*l3 + dot3(r1,r2)*l3 + dot3(r1,r3)*l2 + dot3(r2,r3)*l1;
  return -2.0 * atan2(num, den);
}

/* unit normal of a triangle by the right-hand rule */
void orc_tri_normal(const double *v, double *n) {
  double a[3], b[3];
  sub3(v+3, v, a); sub3(v+6, v, b); cross3(a, b, n);
  double nn = norm3(n);
  n[0] /= nn; n[1] /= nn; n[2] /= nn;
}

/* Potential of the uniform tetrahedron: psi(x) = int_tau dy/|x-y|.
 * div_y((y-x)/|y-x|) = 2/|y-x| and the divergence theorem give
 * psi(x) = 1/2 sum_F h_F(x) I_F(x), h_F = n_F.(y_F - x), n_F outward. */
double orc_tet_potential(const double *x, const double *v /*[4][3]*/) {
  static const int F[4][3] = { {1,2,3}, {0,3,2}, {0,1,3}, {0,2,1} };
  double cen[3] = {0,0,0};
  for (int i = 0; i < 4; ++i) for (int k = 0; k < 3; ++k) cen[k] += 0.25*v[3*i+k];
  double acc = 0.0;
  for (int f = 0; f < 4; ++f) {
    double tri[9];
    for (int i = 0; i < 3; ++i) for (int k = 0; k < 3; ++k) tri[3*i+k] = v[3*F[f][i]+k];
    double a[3], b[3], n[3];
    sub3(tri+3, tri, a); sub3(tri+6, tri, b); cross3(a, b, n);
    double nn = norm3(n); n[0]/=nn; n[1]/=nn; n[2]/=nn;
    double cf[3]; sub3(tri, cen, cf);
    if (dot3(cf, n) < 0) { n[0]=-n[0]; n[1]=-n[1]; n[2]=-n[2]; }
    double yx[3]; sub3(tri, x, yx);
    double h = dot3(n, yx);
    if (h == 0.0) continue;
    acc += 0.5 * h * orc_tri_potential(x, tri);
  }
  return acc;
}

/* ------------------------------------------------------------------ */
/* Element quadrature rules                                            */
/* tet: degree-2, barycentric (a,b,b,b), a=(5+3sqrt5)/20, b=(5-sqrt5)/20 */
/* tri: degree-2 interior rule (2/3,1/6,1/6), weights 1/3               */
/* ------------------------------------------------------------------ */
void orc_tet_quad(const double *tets, int64_t ntet, double *pts, double *wts) {
  const double a = (5.0 + 3.0*sqrt(5.0)) / 20.0, b = (5.0 - sqrt(5.0)) / 20.0;
  for (int64_t t = 0; t < ntet; ++t) {
    const double *v = tets + 12*t;
    double vol = orc_tet_volume(v);
    for (int q = 0; q < 4; ++q) {
      for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int i = 0; i < 4; ++i) s += (i == q ? a : b) * v[3*i+k];
        pts[3*(4*t+q)+k] = s;
      }
      wts[4*t+q] = 0.25 * vol;
    }
  }
}
void orc_tri_quad(const double *tris, int64_t ntri, double *pts, double *wts) {
  for (int64_t t = 0; t < ntri; ++t) {
    const double *v = tris + 9*t;
    double ar = orc_tri_area(v);
    for (int q = 0; q < 3; ++q) {
      for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int i = 0; i < 3; ++i) s += (i == q ? 2.0/3.0 : 1.0/6.0) * v[3*i+k];
        pts[3*(3*t+q)+k] = s;
      }
      wts[3*t+q] = ar / 3.0;
    }
  }
}

/* ------------------------------------------------------------------ */
/* Near rule: outer composite rule over the target element.             */
/* The target is refined k times (tet: 8 children, the inner octahedron */
/* cut along the x02-x13 diagonal; triangle: 4 midpoint children).  On  */
/* each piece: collapsed-coordinate Gauss-Legendre with n nodes per      */
/* direction (nodes/weights on [0,1] are passed in).                     */
/* ------------------------------------------------------------------ */
typedef struct { const double *x; const double *w; int n; int k; } orc_rule;

static void mid3(const double *a, const double *b, double *o) { for (int k=0;k<3;++k) o[k]=0.5*(a[k]+b[k]); }

static double tet_rule_apply(const double *v, int k, const orc_rule *R,
                             double (*fn)(const double *x, const void *ctx), const void *ctx) {
  if (k > 0) {
    double m[4][4][3];
    for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) mid3(v+3*i, v+3*j, m[i][j]);
    double ch[8][12];
    const double *c[8][4] = {
      { v,       m[0][1], m[0][2], m[0][3] },
      { m[0][1], v+3,     m[1][2], m[1][3] },
      { m[0][2], m[1][2], v+6,     m[2][3] },
      { m[0][3], m[1][3], m[2][3], v+9     },
      { m[0][1], m[0][2], m[0][3], m[1][3] },
      { m[0][1], m[0][2], m[1][2], m[1][3] },
      { m[0][2], m[0][3], m[1][3], m[2][3] },
      { m[0][2], m[1][2], m[1][3], m[2][3] } };
    double s = 0.0;
    for (int q = 0; q < 8; ++q) {
      for (int i = 0; i < 4; ++i) memcpy(ch[q]+3*i, c[q][i], 3*sizeof(double));
      s += tet_rule_apply(ch[q], k-1, R, fn, ctx);
    }
    return s;
  }
  double vol6 = 6.0 * orc_tet_volume(v);
  double s = 0.0;
  for (int a = 0; a < R->n; ++a) for (int b = 0; b < R->n; ++b) for (int c = 0; c < R->n; ++c) {
    double u = R->x[a], vv = R->x[b], ww = R->x[c];
    double x1 = u, x2 = (1-u)*vv, x3 = (1-u)*(1-vv)*ww;
    double jac = (1-u)*(1-u)*(1-vv);
    double p[3];
    for (int q = 0; q < 3; ++q) p[q] = v[q] + x1*(v[3+q]-v[q]) + x2*(v[6+q]-v[q]) + x3*(v[9+q]-v[q]);
    s += R->w[a]*R->w[b]*R->w[c]*jac*vol6 * fn(p, ctx);
  }
  return s;
}

static double tri_rule_apply(const double *v, int k, const orc_rule *R,
                             double (*fn)(const double *x, const void *ctx), const void *ctx) {
  if (k > 0) {
    double m01[3], m12[3], m20[3];
    mid3(v, v+3, m01); mid3(v+3, v+6, m12); mid3(v+6, v, m20);
    const double *c[4][3] = { {v, m01, m20}, {m01, v+3, m12}, {m20, m12, v+6}, {m01, m12, m20} };
    double s = 0.0, ch[9];
    for (int q = 0; q < 4; ++q) {
      for (int i = 0; i < 3; ++i) memcpy(ch+3*i, c[q][i], 3*sizeof(double));
      s += tri_rule_apply(ch, k-1, R, fn, ctx);
    }
    return s;
  }
  double ar2 = 2.0 * orc_tri_area(v);
  double s = 0.0;
  for (int a = 0; a < R->n; ++a) for (int b = 0; b < R->n; ++b) {
    double u = R->x[a], vv = R->x[b];
    double x1 = u, x2 = (1-u)*vv, jac = (1-u);
    double p[3];
    for (int q = 0; q < 3; ++q) p[q] = v[q] + x1*(v[3+q]-v[q]) + x2*(v[6+q]-v[q]);
    s += R->w[a]*R->w[b]*jac*ar2 * fn(p, ctx);
  }
  return s;
}

static double fn_tet_pot(const double *x, const void *ctx) { return orc_tet_potential(x, (const double*)ctx); }
static double fn_tri_pot(const double *x, const void *ctx) { return orc_tri_potential(x, (const double*)ctx); }
static double fn_tri_dl(const double *x, const void *ctx) { return orc_tri_solid_angle(x, (const double*)ctx); }

/* task: 0 = VtV (tet target, tet source), 1 = VtB (tri target, tet source),
 *       2 = BtV (tet target, tri source), 3 = BtV double layer (tet target,
 *       tri source, kernel dG/dn_y).  Returns N_ts (includes 1/(4 pi)). */
double orc_near_pair(int task, const double *tgt, const double *src,
                     const double *glx, const double *glw, int n, int k) {
  orc_rule R = { glx, glw, n, k };
  double s;
  if (task == 0)      s = tet_rule_apply(tgt, k, &R, fn_tet_pot, src);
  else if (task == 1) s = tri_rule_apply(tgt, k, &R, fn_tet_pot, src);
  else if (task == 2) s = tet_rule_apply(tgt, k, &R, fn_tri_pot, src);
  else                s = tet_rule_apply(tgt, k, &R, fn_tri_dl, src);
  return s / FOUR_PI;
}

/* Adaptive reference for pins only: recursive 8-split of the target tet
 * until the rule on a piece and the sum over its children agree to tol. */
static double adapt_tet(const double *v, const orc_rule *R, double (*fn)(const double*, const void*),
                        const void *ctx, double whole, double tol, int depth, int maxdepth) {
  double kids = tet_rule_apply(v, 1, R, fn, ctx);
  if (depth >= maxdepth || fabs(kids - whole) <= tol) return kids;
  double m[4][4][3];
  for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) mid3(v+3*i, v+3*j, m[i][j]);
  const double *c[8][4] = {
    { v,       m[0][1], m[0][2], m[0][3] }, { m[0][1], v+3, m[1][2], m[1][3] },
    { m[0][2], m[1][2], v+6, m[2][3] },     { m[0][3], m[1][3], m[2][3], v+9 },
    { m[0][1], m[0][2], m[0][3], m[1][3] }, { m[0][1], m[0][2], m[1][2], m[1][3] },
    { m[0][2], m[0][3], m[1][3], m[2][3] }, { m[0][2], m[1][2], m[1][3], m[2][3] } };
  double s = 0.0, ch[12];
  for (int q = 0; q < 8; ++q) {
    for (int i = 0; i < 4; ++i) memcpy(ch+3*i, c[q][i], 3*sizeof(double));
    double w0 = tet_rule_apply(ch, 0, R, fn, ctx);
    s += adapt_tet(ch, R, fn, ctx, w0, tol / 8.0 * 2.0, depth+1, maxdepth);
  }
  return s;
}
double orc_adaptive_pair(int task, const double *tgt, const double *src,
                         const double *glx, const double *glw, int n, double tol, int maxdepth) {
  orc_rule R = { glx, glw, n, 0 };
  if (task == 1) return NAN;  /* triangle targets: not needed by the pins */
  double (*fn)(const double*, const void*) = (task == 0) ? fn_tet_pot : (task == 2) ? fn_tri_pot : fn_tri_dl;
  double w0 = tet_rule_apply(tgt, 0, &R, fn, src);
  return adapt_tet(tgt, &R, fn, src, w0, tol, 0, maxdepth) / FOUR_PI;
}

/* ------------------------------------------------------------------ */
/* element geometry for the near test                                  */
/* ------------------------------------------------------------------ */
static void elem_centre_radius(const double *v, int nv, double *c, double *rho) {
  c[0]=c[1]=c[2]=0;
  for (int i = 0; i < nv; ++i) for (int k = 0; k < 3; ++k) c[k] += v[3*i+k] / nv;
  double r = 0;
  for (int i = 0; i < nv; ++i) { double d[3]; sub3(v+3*i, c, d); double l = norm3(d); if (l > r) r = l; }
  *rho = r;
}

/* near iff eta = (rho_t + rho_s)/|x_t - x_s| > eta_ns (eta = inf when the
 * centres coincide). */
int orc_is_near(const double *tv, int ntv, const double *sv, int nsv, double eta_ns) {
  double ct[3], cs[3], rt, rs, d[3];
  elem_centre_radius(tv, ntv, ct, &rt);
  elem_centre_radius(sv, nsv, cs, &rs);
  sub3(ct, cs, d);
  double dist = norm3(d);
  if (dist == 0.0) return 1;
  return (rt + rs) / dist > eta_ns;
}

/* ------------------------------------------------------------------ */
/* O1: direct definition, pair by pair.                                  */
/* tgt_el/src_el: element vertex arrays; nvt/nvs = 4 (tet) or 3 (tri).   */
/* dens: [ndens][nsrc]; out: [ndens][ntargets] (u for target elements    */
/* targets[0..ntargets)).                                                */
/* ------------------------------------------------------------------ */
void orc_direct(int task, const double *tgt_el, int64_t ntgt, const double *src_el, int64_t nsrc,
                const double *dens, int ndens, const int64_t *targets, int64_t ntargets,
                double eta_ns, const double *glx, const double *glw, int n, int k,
                double *out, int nthreads) {
  int nvt = (task == 1) ? 3 : 4, nvs = (task >= 2) ? 3 : 4;
  int nqt = (nvt == 4) ? 4 : 3, nqs = (nvs == 4) ? 4 : 3;
  double *sp = malloc(sizeof(double) * 3 * nqs * nsrc), *sw = malloc(sizeof(double) * nqs * nsrc);
  if (nvs == 4) orc_tet_quad(src_el, nsrc, sp, sw); else orc_tri_quad(src_el, nsrc, sp, sw);
  (void)ntgt;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (int64_t ti = 0; ti < ntargets; ++ti) {
    int64_t t = targets[ti];
    const double *tv = tgt_el + 3*nvt*t;
    double tp[12], tw[4];
    if (nvt == 4) orc_tet_quad(tv, 1, tp, tw); else orc_tri_quad(tv, 1, tp, tw);
    double *acc = calloc(ndens, sizeof(double));
    for (int64_t s = 0; s < nsrc; ++s) {
      const double *sv = src_el + 3*nvs*s;
      double a;
      if (orc_is_near(tv, nvt, sv, nvs, eta_ns)) {
        a = orc_near_pair(task, tv, sv, glx, glw, n, k);
      } else {
        double ns[3] = {0, 0, 0};
        if (task == 3) orc_tri_normal(sv, ns);
        a = 0.0;
        for (int i = 0; i < nqt; ++i) for (int j = 0; j < nqs; ++j) {
          double d[3]; sub3(tp+3*i, sp+3*(nqs*s+j), d);
          double r = norm3(d);
          if (r == 0.0) continue;
          if (task == 3) a += tw[i] * sw[nqs*s+j] * dot3(ns, d) / (FOUR_PI * r * r * r);
          else           a += tw[i] * sw[nqs*s+j] / (FOUR_PI * r);
        }
      }
      for (int q = 0; q < ndens; ++q) acc[q] += a * dens[(int64_t)q*nsrc + s];
    }
    for (int q = 0; q < ndens; ++q) out[(int64_t)q*ntargets + ti] = acc[q];
    free(acc);
  }
  free(sp); free(sw);
}
