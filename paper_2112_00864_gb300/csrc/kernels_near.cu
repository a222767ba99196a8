// Setup kernel: FP64 corrections C_ts = N_ts - Q_ts for near element pairs.
//
// N_ts (near rule) = (1/4pi) int_t psi_s(x) dx with psi_s the closed-form
// potential of the uniform source element, integrated over the target by a
// composite collapsed Gauss-Legendre rule (target refined k times: a tet
// into 8 children with the inner octahedron cut along the x02-x13 diagonal,
// a triangle into its 4 midpoint children).  Q_ts is the product rule the
// point passes apply to the same pair (self point r = 0 skipped).  This is
// the library's own evaluation of the near field of Sec. 3.3; the paper's
// singularity-removing transforms are replaced by the closed-form inner
// integral.
#include "kernels.cuh"

namespace bcfmm {

constexpr double kInv4PiN = 0.079577471545947667884441881686257;

struct V3 { double x, y, z; };
__device__ __forceinline__ V3 vsub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double vdot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 vcross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
__device__ __forceinline__ V3 vscale(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ V3 vmid(V3 a, V3 b) { return {0.5 * (a.x + b.x), 0.5 * (a.y + b.y), 0.5 * (a.z + b.z)}; }

// int_T ds_y / |x - y| over the flat triangle (A, B, C): edge terms
// d_e ln((t2 + R2)/(t1 + R1)) from the in-plane divergence theorem, minus
// |w| times the solid angle (Van Oosterom-Strackee) for the height w.
__device__ double tri_pot(V3 x, const V3* P) {
  V3 n = vcross(vsub(P[1], P[0]), vsub(P[2], P[0]));
  const double nn = sqrt(vdot(n, n));
  n = vscale(n, 1.0 / nn);
  const double w = vdot(vsub(x, P[0]), n);
  const V3 rho = vsub(x, vscale(n, w));
  const double scale = sqrt(nn);
  double acc = 0.0;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const V3 A = P[e], B = P[(e + 1) % 3];
    V3 t = vsub(B, A);
    const double Lt = sqrt(vdot(t, t));
    t = vscale(t, 1.0 / Lt);
    const V3 m = vcross(t, n);
    const double d = vdot(vsub(A, rho), m);
    if (fabs(d) <= 1e-14 * scale) continue;
    const V3 ax = vsub(A, x), bx = vsub(B, x);
    const double t1 = vdot(ax, t), t2 = vdot(bx, t);
    const double R1 = sqrt(vdot(ax, ax)), R2 = sqrt(vdot(bx, bx));
    const double lg = (t1 + t2 >= 0.0) ? log((R2 + t2) / (R1 + t1)) : log((R1 - t1) / (R2 - t2));
    acc += d * lg;
  }
  const V3 r1 = vsub(P[0], x), r2 = vsub(P[1], x), r3 = vsub(P[2], x);
  const double l1 = sqrt(vdot(r1, r1)), l2 = sqrt(vdot(r2, r2)), l3 = sqrt(vdot(r3, r3));
  const double num = vdot(r1, vcross(r2, r3));
  const double den = l1 * l2 * l3 + vdot(r1, r2) * l3 + vdot(r1, r3) * l2 + vdot(r2, r3) * l1;
  const double omega = 2.0 * atan2(num, den);
  return acc - fabs(w) * fabs(omega);
}

// int_T n.(x-y)/|x-y|^3 ds_y over the flat triangle with normal
// n = (P1-P0) x (P2-P0) / |.|: the solid angle T subtends at x, signed
// positive on the side n points to (for y in the plane n.(x-y) is the
// height of x).  Van Oosterom-Strackee: tan(Omega/2) = r1.(r2 x r3) /
// (l1 l2 l3 + (r1.r2) l3 + (r1.r3) l2 + (r2.r3) l1), r_i = P_i - x; the
// triple product is negative for x on the + side, hence the minus sign.
__device__ double tri_solid(V3 x, const V3* P) {
  const V3 r1 = vsub(P[0], x), r2 = vsub(P[1], x), r3 = vsub(P[2], x);
  const double l1 = sqrt(vdot(r1, r1)), l2 = sqrt(vdot(r2, r2)), l3 = sqrt(vdot(r3, r3));
  const double num = vdot(r1, vcross(r2, r3));
  const double den = l1 * l2 * l3 + vdot(r1, r2) * l3 + vdot(r1, r3) * l2 + vdot(r2, r3) * l1;
  return -2.0 * atan2(num, den);
}

// int_tet dy/|x-y| = 1/2 sum_F h_F(x) I_F(x), h_F = n_F.(y_F - x), n_F
// outward, with I_F the flat-triangle integral above.  Everything that does
// not depend on x (face normals, edge directions, in-plane edge normals) is
// prepared once per source tet, and the quantities faces share (vertex
// distances, the log term of each of the 6 edges, which does not depend on
// the face or the edge's direction) are computed once per point.
__device__ constexpr int kTetEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
__device__ constexpr int kTetFace[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
__device__ constexpr int kFaceEdge[4][3] = {{3, 5, 4}, {2, 5, 1}, {0, 4, 2}, {1, 3, 0}};   // edge of (F[j], F[j+1])

struct SrcTet {
  V3 v[4];
  V3 te[6];            // unit direction of edge k (first -> second vertex)
  V3 nout[4];          // outward unit normal of face f
  V3 m[4][3];          // in-plane outward normal of the face's edge j (vertex order of the face)
  double thr[4];       // |d| below this: x on the edge's line within the face plane
};

__device__ void src_tet_prepare(const V3* v, SrcTet& S) {
  V3 cen = {0, 0, 0};
  for (int i = 0; i < 4; ++i) { S.v[i] = v[i]; cen.x += 0.25 * v[i].x; cen.y += 0.25 * v[i].y; cen.z += 0.25 * v[i].z; }
  for (int k = 0; k < 6; ++k) {
    V3 t = vsub(v[kTetEdge[k][1]], v[kTetEdge[k][0]]);
    S.te[k] = vscale(t, 1.0 / sqrt(vdot(t, t)));
  }
  for (int f = 0; f < 4; ++f) {
    const V3 T0 = v[kTetFace[f][0]], T1 = v[kTetFace[f][1]], T2 = v[kTetFace[f][2]];
    V3 n = vcross(vsub(T1, T0), vsub(T2, T0));
    const double nn = sqrt(vdot(n, n));
    n = vscale(n, 1.0 / nn);             // normal of the face's vertex order
    S.thr[f] = 1e-14 * sqrt(nn);
    S.nout[f] = vdot(vsub(T0, cen), n) < 0 ? vscale(n, -1.0) : n;
    for (int j = 0; j < 3; ++j) {
      const int a = kTetFace[f][j], b = kTetFace[f][(j + 1) % 3];
      V3 t = vsub(v[b], v[a]);
      t = vscale(t, 1.0 / sqrt(vdot(t, t)));
      S.m[f][j] = vcross(t, n);
    }
  }
}

__device__ double tet_pot(V3 x, const SrcTet& S) {
  V3 r[4];
  double R[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) { r[i] = vsub(S.v[i], x); R[i] = sqrt(vdot(r[i], r[i])); }
  double L[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int a = kTetEdge[k][0], b = kTetEdge[k][1];
    const double ta = vdot(r[a], S.te[k]), tb = vdot(r[b], S.te[k]);
    L[k] = (ta + tb >= 0.0) ? log((R[b] + tb) / (R[a] + ta)) : log((R[a] - ta) / (R[b] - tb));
  }
  double acc = 0.0;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int i0 = kTetFace[f][0], i1 = kTetFace[f][1], i2 = kTetFace[f][2];
    const double h = vdot(S.nout[f], r[i0]);
    if (h == 0.0) continue;
    double e = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double d = vdot(r[kTetFace[f][j]], S.m[f][j]);
      if (fabs(d) > S.thr[f]) e += d * L[kFaceEdge[f][j]];
    }
    const double num = vdot(r[i0], vcross(r[i1], r[i2]));
    const double den = R[i0] * R[i1] * R[i2] + vdot(r[i0], r[i1]) * R[i2] + vdot(r[i0], r[i2]) * R[i1] +
                       vdot(r[i1], r[i2]) * R[i0];
    const double omega = 2.0 * atan2(num, den);
    acc += 0.5 * h * (e - fabs(h) * fabs(omega));
  }
  return acc;
}

__device__ double tet_vol6(const V3* v) {
  return fabs(vdot(vcross(vsub(v[1], v[0]), vsub(v[2], v[0])), vsub(v[3], v[0])));
}
__device__ double tri_area2(const V3* v) {
  const V3 n = vcross(vsub(v[1], v[0]), vsub(v[2], v[0]));
  return sqrt(vdot(n, n));
}

// children as pairs of parent vertices (i == j: the vertex, else the midpoint)
__constant__ int c_tet_child[8][4][2] = {
    {{0, 0}, {0, 1}, {0, 2}, {0, 3}}, {{0, 1}, {1, 1}, {1, 2}, {1, 3}},
    {{0, 2}, {1, 2}, {2, 2}, {2, 3}}, {{0, 3}, {1, 3}, {2, 3}, {3, 3}},
    {{0, 1}, {0, 2}, {0, 3}, {1, 3}}, {{0, 1}, {0, 2}, {1, 2}, {1, 3}},
    {{0, 2}, {0, 3}, {1, 3}, {2, 3}}, {{0, 2}, {1, 2}, {1, 3}, {2, 3}}};
__constant__ int c_tri_child[4][3][2] = {
    {{0, 0}, {0, 1}, {2, 0}}, {{0, 1}, {1, 1}, {1, 2}}, {{2, 0}, {1, 2}, {2, 2}}, {{0, 1}, {1, 2}, {2, 0}}};

constexpr int kMaxGL = 8;

// One warp per near pair (CSR position k = sel[i], or i without a
// selection list): lanes share the outer points.  The result goes to
// cor_val[k], or to cor_val[i] when compact is set.
__global__ void k_near_rule(int task, int64_t nnz, const int64_t* __restrict__ sel, const int* __restrict__ row,
                            const int* __restrict__ col,
                            const double* __restrict__ tgt_v, const double* __restrict__ src_v,
                            const double* __restrict__ tgt_qp, const double* __restrict__ tgt_qw,
                            const double* __restrict__ src_qp, const double* __restrict__ src_qw,
                            const double* __restrict__ glx, const double* __restrict__ glw, int n, int k,
                            int compact, double* __restrict__ cor_val) {
  const int64_t ii = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (ii >= nnz) return;
  const int64_t kk = sel ? sel[ii] : ii;
  const int t = row[kk], s = col[kk];
  // task 3: BtV double layer, kernel dG/dn_y of the source triangle
  const bool tgt_tet = (task != 1), src_tet = (task != 2 && task != 3), dl = (task == 3);
  const int nvt = tgt_tet ? 4 : 3, nvs = src_tet ? 4 : 3;
  V3 tv[4], sv[4] = {};
  for (int i = 0; i < nvt; ++i) tv[i] = {tgt_v[(int64_t)t * 3 * nvt + 3 * i], tgt_v[(int64_t)t * 3 * nvt + 3 * i + 1], tgt_v[(int64_t)t * 3 * nvt + 3 * i + 2]};
  for (int i = 0; i < nvs; ++i) sv[i] = {src_v[(int64_t)s * 3 * nvs + 3 * i], src_v[(int64_t)s * 3 * nvs + 3 * i + 1], src_v[(int64_t)s * 3 * nvs + 3 * i + 2]};
  double gx[kMaxGL], gw[kMaxGL];
  for (int i = 0; i < n; ++i) { gx[i] = glx[i]; gw[i] = glw[i]; }
  // the source tet's x-independent geometry, prepared once per warp
  __shared__ SrcTet sS[4];
  SrcTet& S = sS[(threadIdx.x >> 5) & 3];
  if (src_tet) {
    if (lane == 0) src_tet_prepare(sv, S);
    __syncwarp();
  }
  const int nch = tgt_tet ? 8 : 4;
  int npc = tgt_tet ? n * n * n : n * n;
  int npieces = 1;
  for (int i = 0; i < k; ++i) npieces *= nch;
  const int total = npieces * npc;
  double sum = 0.0;
  for (int idx = lane; idx < total; idx += 32) {
    int piece = idx / npc, q = idx % npc;
    // descend k levels (most significant digit = first refinement)
    V3 v[4] = {tv[0], tv[1], tv[2], tgt_tet ? tv[3] : tv[0]};
    int div = npieces;
    for (int lev = 0; lev < k; ++lev) {
      div /= nch;
      const int c = (piece / div) % nch;
      V3 w[4];
      for (int i = 0; i < nvt; ++i) {
        const int a = tgt_tet ? c_tet_child[c][i][0] : c_tri_child[c][i][0];
        const int b = tgt_tet ? c_tet_child[c][i][1] : c_tri_child[c][i][1];
        w[i] = (a == b) ? v[a] : vmid(v[a], v[b]);
      }
      for (int i = 0; i < nvt; ++i) v[i] = w[i];
    }
    V3 x;
    double wt;
    if (tgt_tet) {
      const int ia = q / (n * n), ib = (q / n) % n, ic = q % n;
      const double u = gx[ia], vv = gx[ib], ww = gx[ic];
      const double x1 = u, x2 = (1 - u) * vv, x3 = (1 - u) * (1 - vv) * ww;
      const double jac = (1 - u) * (1 - u) * (1 - vv);
      x.x = v[0].x + x1 * (v[1].x - v[0].x) + x2 * (v[2].x - v[0].x) + x3 * (v[3].x - v[0].x);
      x.y = v[0].y + x1 * (v[1].y - v[0].y) + x2 * (v[2].y - v[0].y) + x3 * (v[3].y - v[0].y);
      x.z = v[0].z + x1 * (v[1].z - v[0].z) + x2 * (v[2].z - v[0].z) + x3 * (v[3].z - v[0].z);
      wt = gw[ia] * gw[ib] * gw[ic] * jac * tet_vol6(v);
    } else {
      const int ia = q / n, ib = q % n;
      const double u = gx[ia], vv = gx[ib];
      const double x1 = u, x2 = (1 - u) * vv, jac = 1 - u;
      x.x = v[0].x + x1 * (v[1].x - v[0].x) + x2 * (v[2].x - v[0].x);
      x.y = v[0].y + x1 * (v[1].y - v[0].y) + x2 * (v[2].y - v[0].y);
      x.z = v[0].z + x1 * (v[1].z - v[0].z) + x2 * (v[2].z - v[0].z);
      wt = gw[ia] * gw[ib] * jac * tri_area2(v);
    }
    sum += wt * (src_tet ? tet_pot(x, S) : dl ? tri_solid(x, sv) : tri_pot(x, sv));
  }
  sum *= kInv4PiN;
  V3 ns = {0, 0, 0};
  if (dl) {
    ns = vcross(vsub(sv[1], sv[0]), vsub(sv[2], sv[0]));
    ns = vscale(ns, 1.0 / sqrt(vdot(ns, ns)));
  }
  // product rule of the point passes for this pair
  const int nqt = tgt_tet ? 4 : 3, nqs = src_tet ? 4 : 3;
  double q = 0.0;
  if (lane < nqt * nqs) {
    const int i = lane / nqs, j = lane % nqs;
    const double* xp = tgt_qp + 3 * ((int64_t)t * nqt + i);
    const double* yp = src_qp + 3 * ((int64_t)s * nqs + j);
    const double dx = xp[0] - yp[0], dy = xp[1] - yp[1], dz = xp[2] - yp[2];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    if (r != 0.0) {
      q = tgt_qw[(int64_t)t * nqt + i] * src_qw[(int64_t)s * nqs + j] * kInv4PiN / r;
      if (dl) q *= (ns.x * dx + ns.y * dy + ns.z * dz) / (r * r);
    }
  }
  double c = sum - q;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) cor_val[compact ? ii : kk] = c;
}

cudaError_t launch_near_rule(int task, int64_t nnz, const int64_t* sel, const int* row, const int* col,
                             const double* tgt_v, const double* src_v,
                             const double* tgt_qp, const double* tgt_qw,
                             const double* src_qp, const double* src_qw,
                             const double* glx, const double* glw, int n, int k,
                             int compact, double* cor_val, cudaStream_t st) {
  if (nnz == 0) return cudaSuccess;
  if (n > kMaxGL) return cudaErrorInvalidValue;
  const int64_t threads = nnz * 32;
  k_near_rule<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(task, nnz, sel, row, col, tgt_v, src_v, tgt_qp, tgt_qw,
                                                                src_qp, src_qw, glx, glw, n, k, compact, cor_val);
  return cudaGetLastError();
}

}  // namespace bcfmm
