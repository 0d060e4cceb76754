// sale_ale32.cu -- FP32-mixed kernels of the Eulerian (ALE, remap every
// cycle) cycle.
//
// Field storage and the bulk of the arithmetic are FP32; FP64 is kept for
// the reference hex volumes and corner gradients (computed once in FP64 and
// stored) and the conservation sums (diagnostics).  The conserved cell mass
// and energy and the node mass accumulate in float-float (FP32 hi + lo, about
// 48 bits) instead of FP64, which runs at 1/64 of the FP32 rate on GB300.
//
// Two reformulations keep FP32 accurate where a plain FP32 evaluation
// would cancel:
//  * Reference geometry is never formed from absolute FP32 coordinates:
//    the mesh is the structured box plus per-node jitter offsets, and a
//    coordinate difference is (index difference) * h + (offset difference),
//    exact to FP32 rounding of the difference itself.
//  * Swept volumes (thin hexes between a face's Lagrangian and reference
//    positions) use an expansion of the fan volume formula in the node
//    displacements D = dt * ubar: with E the reference positions relative
//    to the cell's reference node 0, a side quad (L_a, E_a, E_b, L_b) has
//        T = 4 (E_a x E_b) . (D_a + D_b) - 2 (E_a + E_b) . (D_a x D_b)
//    and a Lagrangian face plus the reversed reference face
//        T = S_E . (e1 x d2 + d1 x e2 + d1 x d2) + S_D . ((e1+d1) x (e2+d2))
//    (e = reference diagonals, d = their displacement, S = node sums), so
//    every term is O(h^2 |D|) like the swept volume itself.
//  * The node force vanishes exactly where sigma is uniform: on a jittered
//    mesh it is F_a = sum_c (sigma_c - sigma_ref) G_c(a) over the cached
//    corner gradients (sum_c G_c(a) = 0 in exact arithmetic); on an
//    unjittered one it gathers face terms, F_a = (1/24) sum over the 12 mesh
//    faces at node a of (sigma_low - sigma_high) t_f, t_f = (p1 + 2 p2 + p3)
//    x (p3 - p1) over the face's other nodes relative to a.
#include "sale_device.cuh"

namespace sale {

namespace {

struct F3 {
  float x, y, z;
};
__device__ __forceinline__ F3 operator+(F3 a, F3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ F3 operator-(F3 a, F3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ F3 operator*(float s, F3 a) { return {s * a.x, s * a.y, s * a.z}; }

// The same products with every rounding fixed by intrinsics: the compiler
// may contract a * b + c * d either way, and may choose differently in two
// kernels that inline the same function (a batch block and a single-mesh
// block of the remap + EoS pass); the quantities a batch must reproduce
// bitwise go through these.
__device__ __forceinline__ float dot_rn(F3 a, F3 b) {
  return __fmaf_rn(a.z, b.z, __fmaf_rn(a.y, b.y, __fmul_rn(a.x, b.x)));
}
__device__ __forceinline__ F3 cross_rn(F3 a, F3 b) {
  return {__fmaf_rn(a.y, b.z, -__fmul_rn(a.z, b.y)), __fmaf_rn(a.z, b.x, -__fmul_rn(a.x, b.z)),
          __fmaf_rn(a.x, b.y, -__fmul_rn(a.y, b.x))};
}
// s a + b, fused.  This file is compiled without automatic FMA contraction
// (every tile shape is a separate instantiation of the kernels, and a
// compiler free to fuse differently in each would make results depend on
// the launch shape), so the multiply-adds it wants fused are written so.
__device__ __forceinline__ F3 fma3(float s, F3 a, F3 b) {
  return {__fmaf_rn(s, a.x, b.x), __fmaf_rn(s, a.y, b.y), __fmaf_rn(s, a.z, b.z)};
}

// ---------------------------------------------------------------------------
// Float-float arithmetic for the conserved cell quantities
// ---------------------------------------------------------------------------
// Cell mass and specific internal energy are held as unevaluated sums
// hi + lo of two FP32 numbers (about 48 significant bits).  Plain FP32
// accumulation of the small per-cycle increments these quantities receive
// drifts systematically (round-to-nearest of a slowly varying increment is
// biased); FP64 hardware runs at 1/64 of the FP32 rate on GB300, so the
// extra precision comes from error-free transformations on the FP32 pipe:
// TwoSum (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum and TwoProduct via FMA
// (Dekker, "A floating-point technique for extending the available
// precision", Numer. Math. 18, 1971).  The _rn intrinsics keep the compiler
// from contracting or reordering these sequences.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
  return {s, e};
}

// Requires |a| >= |b| (or a = 0).
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF df_add_f(DF a, float b) {
  const DF s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
  const DF s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ DF df_div(DF a, DF b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const DF p = df_mul(b, DF{q1, 0.f});
  const DF r = df_add(a, DF{-p.hi, -p.lo});
  return fast_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}

__device__ __forceinline__ DF load_df(const float *hi, const float *lo, int c) { return {hi[c], lo[c]}; }

// Jitter offset of a node (one 16-byte load: x, y, z, unused); on an
// unjittered mesh (JIT = false) the offsets are zero and the geometry below
// folds to constants.
template <bool JIT>
__device__ __forceinline__ float4 off_at(const Fields<float> &F, int n) {
  if constexpr (JIT) return __ldg(F.off4 + n);
  return make_float4(0.f, 0.f, 0.f, 0.f);
}

// Position of node nb relative to a base node with offset oa, the two
// differing by the index offset (ox, oy, oz): o * h + (offset - oa).
template <bool JIT>
__device__ __forceinline__ F3 relp(const Fields<float> &F, float4 oa, int nb, int ox, int oy, int oz) {
  const float4 ob = off_at<JIT>(F, nb);
  return {__fmaf_rn((float)ox, F.hx, ob.x - oa.x), __fmaf_rn((float)oy, F.hy, ob.y - oa.y),
          __fmaf_rn((float)oz, F.hz, ob.z - oa.z)};
}

// Reference nodes of the cell whose node 0 is n0 (node strides sy, sz),
// relative to that node.
template <bool JIT>
__device__ __forceinline__ void ref_hex2(const Fields<float> &F, int n0, int sy, int sz, F3 (&E)[8]) {
  const float4 o0 = off_at<JIT>(F, n0);
  E[0] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int a = 1; a < 8; ++a)
    E[a] = relp<JIT>(F, o0, n0 + (a & 1) + ((a >> 1) & 1) * sy + ((a >> 2) & 1) * sz, a & 1, (a >> 1) & 1, (a >> 2) & 1);
}

// sum_a dV/dx_a . U_a for a hex given relative to its node 0, accumulated
// face corner by face corner (the 24-vector gradient is never stored).
__device__ __forceinline__ float grad_dot_f(const F3 (&X)[8], const F3 (&U)[8]) {
  float s = 0.f;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const F3 pa = X[face_node(f, (k + 1) & 3)];
      const F3 pb = X[face_node(f, (k + 2) & 3)];
      const F3 pc = X[face_node(f, (k + 3) & 3)];
      s = __fadd_rn(s, dot_rn(cross_rn(fma3(2.f, pb, pa) + pc, pc - pa), U[face_node(f, k)]));
    }
  }
  return s * (1.f / 24.f);
}

// The same sum from the cached corner gradients of a jittered mesh: 24
// coalesced loads instead of ~480 FP32 operations.
__device__ __forceinline__ float grad_dot_cached(const float *Gc, long long nc, int c, const F3 (&U)[8]) {
  const float *g = Gc + c;
  float s = 0.f;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    s = __fmaf_rn(__ldg(g + (3 * a) * nc), U[a].x, s);
    s = __fmaf_rn(__ldg(g + (3 * a + 1) * nc), U[a].y, s);
    s = __fmaf_rn(__ldg(g + (3 * a + 2) * nc), U[a].z, s);
  }
  return s;
}

// FP32 geometry of a hex given relative to its node 0 (predictor-corrector
// half step, where the nodes are off the reference mesh): volume, corner
// gradients and the largest squared face area, by the same fan formulas as
// the FP64 routines, every multiply-add fused explicitly.
__device__ __forceinline__ float dot_acc(F3 a, F3 b, float s) {
  return __fmaf_rn(a.z, b.z, __fmaf_rn(a.y, b.y, __fmaf_rn(a.x, b.x, s)));
}

__device__ __forceinline__ float hex_volume_f(const F3 (&X)[8]) {
  float s = 0.f;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const F3 p0 = X[face_node(f, 0)], p1 = X[face_node(f, 1)], p2 = X[face_node(f, 2)], p3 = X[face_node(f, 3)];
    s = dot_acc(p0 + p1 + p2 + p3, cross_rn(p2 - p0, p3 - p1), s);
  }
  return s * (1.f / 24.f);
}

// dV/dx_A for one compile-time corner A: the three faces holding A, in
// ascending face order.
template <int A>
__device__ __forceinline__ F3 hex_corner_grad_f(const F3 (&X)[8]) {
  F3 g = {0.f, 0.f, 0.f};
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const int f = 2 * t + ((A >> t) & 1);
    const int k = face_slot(f, A);
    const F3 pa = X[face_node(f, (k + 1) & 3)], pb = X[face_node(f, (k + 2) & 3)], pc = X[face_node(f, (k + 3) & 3)];
    g = g + cross_rn(fma3(2.f, pb, pa) + pc, pc - pa);
  }
  return (1.f / 24.f) * g;
}

template <int A = 0>
__device__ __forceinline__ void hex_grad_f(const F3 (&X)[8], F3 (&G)[8]) {
  G[A] = hex_corner_grad_f<A>(X);
  if constexpr (A < 7) hex_grad_f<A + 1>(X, G);
}

__device__ __forceinline__ float hex_max_face_area2_f(const F3 (&X)[8]) {
  float amax = 0.f;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const F3 p0 = X[face_node(f, 0)], p1 = X[face_node(f, 1)], p2 = X[face_node(f, 2)], p3 = X[face_node(f, 3)];
    const F3 D = cross_rn(p2 - p0, p3 - p1);
    amax = fmaxf(amax, 0.25f * dot_rn(D, D));
  }
  return amax;
}

// FP32 twin of hourglass_store (viscous Flanagan-Belytschko corner forces):
// X relative to node 0, G the corner gradients, U the node velocities.
__device__ __forceinline__ void hourglass_store_f(const F3 (&X)[8], const F3 (&G)[8], const F3 (&U)[8], float V,
                                                  float rho, float cs, float c_hg, float *fh, long long nc, int c) {
  const float iv = 1.f / V;
  F3 hx[4], hu[4];
#pragma unroll
  for (int al = 0; al < 4; ++al) {
    hx[al] = {0.f, 0.f, 0.f};
    hu[al] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const float sg = hg_pattern(al, b);
      hx[al] = fma3(sg, X[b], hx[al]);
      hu[al] = fma3(sg, U[b], hu[al]);
    }
  }
  F3 M[3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    M[0] = fma3(G[b].x, U[b], M[0]);
    M[1] = fma3(G[b].y, U[b], M[1]);
    M[2] = fma3(G[b].z, U[b], M[2]);
  }
  F3 W[3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  F3 q[4];
#pragma unroll
  for (int al = 0; al < 4; ++al) {
    q[al] = fma3(-iv, fma3(hx[al].z, M[2], fma3(hx[al].y, M[1], hx[al].x * M[0])), hu[al]);
    W[0] = fma3(hx[al].x, q[al], W[0]);
    W[1] = fma3(hx[al].y, q[al], W[1]);
    W[2] = fma3(hx[al].z, q[al], W[2]);
  }
  const float cv = cbrtf(V);
  const float kappa = c_hg * rho * cs * cv * cv;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    F3 f = hg_pattern(0, a) * q[0] + hg_pattern(1, a) * q[1] + hg_pattern(2, a) * q[2] + hg_pattern(3, a) * q[3];
    f = fma3(-iv, fma3(G[a].z, W[2], fma3(G[a].y, W[1], G[a].x * W[0])), f);
    fh[(3 * a + 0) * nc + c] = -kappa * f.x;
    fh[(3 * a + 1) * nc + c] = -kappa * f.y;
    fh[(3 * a + 2) * nc + c] = -kappa * f.z;
  }
}

__device__ __forceinline__ F3 hg_corner_f(const float *fh, long long nc, int c, int a) {
  return {__ldg(fh + (3 * a) * nc + c), __ldg(fh + (3 * a + 1) * nc + c), __ldg(fh + (3 * a + 2) * nc + c)};
}

// Side quad (L_a, E_a, E_b, L_b) term, expanded in the displacements.
__device__ __forceinline__ float side_term(const F3 (&E)[8], const F3 (&D)[8], int a, int b) {
  return __fmaf_rn(4.f, dot_rn(cross_rn(E[a], E[b]), D[a] + D[b]),
                   -2.f * dot_rn(E[a] + E[b], cross_rn(D[a], D[b])));
}

// Lagrangian face (p0,p1,p2,p3) plus the reversed reference face, expanded.
__device__ __forceinline__ float pair_term(const F3 (&E)[8], const F3 (&D)[8], int p0, int p1, int p2, int p3) {
  const F3 e1 = E[p2] - E[p0], e2 = E[p3] - E[p1];
  const F3 d1 = D[p2] - D[p0], d2 = D[p3] - D[p1];
  const F3 se = E[p0] + E[p1] + E[p2] + E[p3];
  const F3 sd = D[p0] + D[p1] + D[p2] + D[p3];
  return dot_rn(se, cross_rn(e1, d2) + cross_rn(d1, e2) + cross_rn(d1, d2)) + dot_rn(sd, cross_rn(e1 + d1, e2 + d2));
}

// Swept volumes of the three low faces (see the file comment); E relative
// to the reference node 0 (E[0] = 0), D the node displacements.
__device__ __forceinline__ void swept_low_faces_f(const F3 (&E)[8], const F3 (&D)[8], float &vx, float &vy,
                                                  float &vz) {
  const float t04 = side_term(E, D, 0, 4), t20 = side_term(E, D, 2, 0), t01 = side_term(E, D, 0, 1);
  const float sx = pair_term(E, D, 0, 4, 6, 2) + t04 + side_term(E, D, 6, 2) + t20 + side_term(E, D, 4, 6);
  const float sy = -t04 + side_term(E, D, 1, 5) + pair_term(E, D, 0, 1, 5, 4) + t01 + side_term(E, D, 5, 4);
  const float sz = -t20 + side_term(E, D, 3, 1) - t01 + side_term(E, D, 2, 3) + pair_term(E, D, 0, 2, 3, 1);
  const float s = 1.f / 24.f;
  vx = sx * s;
  vy = sy * s;
  vz = sz * s;
}

__device__ __forceinline__ void wall_bc_f(const Fields<float> &F, int i, int j, int k, float &u, float &v,
                                          float &w) {
  if ((i == 0 && F.reflect[0]) || (i == F.nx && F.reflect[1])) u = 0.f;
  if ((j == 0 && F.reflect[2]) || (j == F.ny && F.reflect[3])) v = 0.f;
  if ((k == 0 && F.reflect[4]) || (k == F.nz && F.reflect[5])) w = 0.f;
}

}  // namespace

// ---------------------------------------------------------------------------
// Initialisation: masses, energies, reference volumes and lengths in FP64
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kBlock) k_m_init_cells(Fields<float> F, DevScalars *S, const double *rho0,
                                                         const double *p0, long long dep_cell, double dep_e,
                                                         float *VE, float *LE, float *Gc) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc) return;
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  P3 X[8];
  load_hex(F.xr, F.yr, F.zr, F.nx, F.ny, i, j, k, X);
  shift0(X);
  const double V = hex_volume_shifted(X);
  if (!(V > 0.0)) set_status(S, SALE_ENEGVOL);
  const double m = rho0[c] * V;
  double e = p0[c] / ((F.gamma - 1.0) * rho0[c]);
  if (c == dep_cell) e = dep_e / m;
  // float-float split: hi = nearest FP32, lo = nearest FP32 to the rest
  F.m[c] = (float)m;
  F.mlo[c] = (float)(m - (double)(float)m);
  F.e[c] = (float)e;
  F.elo[c] = (float)(e - (double)(float)e);
  VE[c] = (float)V;
  LE[c] = (float)(V / sqrt(hex_max_face_area2(X)));
  if (Gc) {  // corner gradients of the reference cell, rounded once from FP64
    P3 g[8];
    hex_grad_shifted(X, g);
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      Gc[(3 * a + 0) * F.nc + c] = (float)g[a].x;
      Gc[(3 * a + 1) * F.nc + c] = (float)g[a].y;
      Gc[(3 * a + 2) * F.nc + c] = (float)g[a].z;
    }
  }
}

// ---------------------------------------------------------------------------
// Lagrangian phase
// ---------------------------------------------------------------------------
//
// Thread layout: blocks of 32 x 8 threads over (i, j) of one k plane; the
// grid is (ceil(n_i / 32), ceil(n_j / 8), n_k) over nodes or cells, so a
// thread's (i, j, k) comes from its block and thread indices (no division)
// and indices stay 32-bit.

// Face term of one mesh face through node (i,j,k): the lower cell across
// the face is SB (bits: cell = node - 1 + bit), the face is normal to D.
template <bool JIT, int SB, int D>
__device__ __forceinline__ void node_face2(const Fields<float> &F, int n, int sy, int sz, float4 oa,
                                           const bool (&lo_ok)[3], const bool (&hi_ok)[3], const float (&sig)[8],
                                           F3 &f) {
  if ((SB >> D) & 1) return;  // the cell must be the lower one across the plane
  constexpr int D1 = (D + 1) % 3, D2 = (D + 2) % 3;
  const bool v1 = ((SB >> D1) & 1) ? hi_ok[D1] : lo_ok[D1];
  const bool v2 = ((SB >> D2) & 1) ? hi_ok[D2] : lo_ok[D2];
  if (!(v1 && v2)) return;  // face outside the mesh
  const float ds = sig[SB] - sig[SB | (1 << D)];
  constexpr int A = 7 - SB;        // local corner of the node in the lower cell
  constexpr int FC = 2 * D + 1;    // the lower cell's high face normal to D
  constexpr int K = face_slot(FC, A);
  constexpr int B1 = face_node(FC, (K + 1) & 3), B2 = face_node(FC, (K + 2) & 3), B3 = face_node(FC, (K + 3) & 3);
  constexpr int X1 = (SB & 1) + (B1 & 1) - 1, Y1 = ((SB >> 1) & 1) + ((B1 >> 1) & 1) - 1,
                Z1 = ((SB >> 2) & 1) + ((B1 >> 2) & 1) - 1;
  constexpr int X2 = (SB & 1) + (B2 & 1) - 1, Y2 = ((SB >> 1) & 1) + ((B2 >> 1) & 1) - 1,
                Z2 = ((SB >> 2) & 1) + ((B2 >> 2) & 1) - 1;
  constexpr int X3 = (SB & 1) + (B3 & 1) - 1, Y3 = ((SB >> 1) & 1) + ((B3 >> 1) & 1) - 1,
                Z3 = ((SB >> 2) & 1) + ((B3 >> 2) & 1) - 1;
  const F3 p1 = relp<JIT>(F, oa, n + X1 + Y1 * sy + Z1 * sz, X1, Y1, Z1);
  const F3 p2 = relp<JIT>(F, oa, n + X2 + Y2 * sy + Z2 * sz, X2, Y2, Z2);
  const F3 p3 = relp<JIT>(F, oa, n + X3 + Y3 * sy + Z3 * sz, X3, Y3, Z3);
  f = fma3(ds, cross_rn(fma3(2.f, p2, p1) + p3, p3 - p1), f);
}

template <bool JIT, int SB>
__device__ __forceinline__ void node_faces2(const Fields<float> &F, int n, int sy, int sz, float4 oa,
                                            const bool (&lo_ok)[3], const bool (&hi_ok)[3], const float (&sig)[8],
                                            F3 &f) {
  node_face2<JIT, SB, 0>(F, n, sy, sz, oa, lo_ok, hi_ok, sig, f);
  node_face2<JIT, SB, 1>(F, n, sy, sz, oa, lo_ok, hi_ok, sig, f);
  node_face2<JIT, SB, 2>(F, n, sy, sz, oa, lo_ok, hi_ok, sig, f);
}

// Kernel bodies: one thread's work for node or cell (i, j, k) of the mesh F.
// The single-mesh kernels and the batched kernels wrap the same bodies, so
// a mesh advanced inside a batch is bitwise equal to the mesh alone.

// OPT: the state may use the predictor-corrector step or hourglass control
// (their branches are compiled out otherwise, as for every batch).
template <bool JIT, bool IN, bool OPT>
__device__ __forceinline__ void m_nodes_body(const Fields<float> &F, DevScalars *S, int i, int j, int k) {
  if ((!IN && (i > F.nx || j > F.ny || k > F.nz)) || !S->next_active) return;
  const float h = S->next_h32;
  const int sy = F.nx + 1, sz = (F.nx + 1) * (F.ny + 1);
  const int n = i + sy * j + sz * k;
  const int csy = F.nx, csz = F.nx * F.ny;
  const int c0 = (i - 1) + csy * (j - 1) + csz * (k - 1);  // cell (i-1, j-1, k-1)
  const bool lo_ok[3] = {IN || i > 0, IN || j > 0, IN || k > 0};
  const bool hi_ok[3] = {IN || i < F.nx, IN || j < F.ny, IN || k < F.nz};
  float sig[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const bool ok = ((s & 1) ? hi_ok[0] : lo_ok[0]) && ((s & 2) ? hi_ok[1] : lo_ok[1]) &&
                    ((s & 4) ? hi_ok[2] : lo_ok[2]);
    sig[s] = ok ? F.sig[c0 + (s & 1) + ((s >> 1) & 1) * csy + ((s >> 2) & 1) * csz] : 0.f;
  }
  F3 f = {0.f, 0.f, 0.f};
  float hm;
  const bool pc = OPT && F.time_order == 2;
  const float *fh = OPT ? F.fh : nullptr;
  if (JIT || pc) {
    // Cached corner gradients (of the reference mesh, or of x^{n+1/2} for
    // the predictor-corrector): F_a = sum_c (sigma_c - sigma_ref) G_c(a).  The
    // dropped sigma_ref sum_c G_c(a) is zero at interior nodes and normal to
    // the (reflecting) walls at boundary nodes, where the wall condition
    // removes it; the differences keep F exactly 0 where sigma is uniform.
    const float *Gsrc = pc ? F.Gh : F.Gc;
    float ref = 0.f;
    bool have = false;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const bool ok = ((q & 1) ? hi_ok[0] : lo_ok[0]) && ((q & 2) ? hi_ok[1] : lo_ok[1]) &&
                      ((q & 4) ? hi_ok[2] : lo_ok[2]);
      if (ok && !have) {
        ref = sig[q];
        have = true;
      }
    }
    const long long nc = F.nc;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const bool ok = ((q & 1) ? hi_ok[0] : lo_ok[0]) && ((q & 2) ? hi_ok[1] : lo_ok[1]) &&
                      ((q & 4) ? hi_ok[2] : lo_ok[2]);
      if (!ok) continue;
      const int c = c0 + (q & 1) + ((q >> 1) & 1) * csy + ((q >> 2) & 1) * csz;
      const float *g = Gsrc + (3 * (7 - q)) * nc + c;  // this node is corner 7 - q of cell q
      const float ds = sig[q] - ref;
      f.x = __fmaf_rn(ds, __ldg(g), f.x);
      f.y = __fmaf_rn(ds, __ldg(g + nc), f.y);
      f.z = __fmaf_rn(ds, __ldg(g + 2 * nc), f.z);
      if (fh) f = f + hg_corner_f(fh, nc, c, 7 - q);
    }
    hm = h / F.mn[n];
  } else {
    const float4 oa = off_at<JIT>(F, n);
    node_faces2<JIT, 0>(F, n, sy, sz, oa, lo_ok, hi_ok, sig, f);
    node_faces2<JIT, 1>(F, n, sy, sz, oa, lo_ok, hi_ok, sig, f);
    node_faces2<JIT, 2>(F, n, sy, sz, oa, lo_ok, hi_ok, sig, f);
    node_faces2<JIT, 3>(F, n, sy, sz, oa, lo_ok, hi_ok, sig, f);
    node_faces2<JIT, 4>(F, n, sy, sz, oa, lo_ok, hi_ok, sig, f);
    node_faces2<JIT, 5>(F, n, sy, sz, oa, lo_ok, hi_ok, sig, f);
    node_faces2<JIT, 6>(F, n, sy, sz, oa, lo_ok, hi_ok, sig, f);
    if (fh) {  // hourglass corner forces, on the face terms' scale of 24
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const bool ok = ((q & 1) ? hi_ok[0] : lo_ok[0]) && ((q & 2) ? hi_ok[1] : lo_ok[1]) &&
                        ((q & 4) ? hi_ok[2] : lo_ok[2]);
        if (ok) f = f + 24.f * hg_corner_f(fh, F.nc, c0 + (q & 1) + ((q >> 1) & 1) * csy + ((q >> 2) & 1) * csz, 7 - q);
      }
    }
    hm = h / (24.f * F.mn[n]);
  }
  const float u0 = F.u[n], v0 = F.v[n], w0 = F.w[n];
  float u1 = __fmaf_rn(hm, f.x, u0), v1 = __fmaf_rn(hm, f.y, v0), w1 = __fmaf_rn(hm, f.z, w0);
  if (!IN) wall_bc_f(F, i, j, k, u1, v1, w1);
  F.u[n] = u1;
  F.v[n] = v1;
  F.w[n] = w1;
  F.ub[n] = 0.5f * (u0 + u1);
  F.vb[n] = 0.5f * (v0 + v1);
  F.wb[n] = 0.5f * (w0 + w1);
}

template <bool JIT, bool IN, bool OPT>
__device__ __forceinline__ void m_cells_body(const Fields<float> &F, DevScalars *S, int i, int j, int k) {
  if ((!IN && (i >= F.nx || j >= F.ny || k >= F.nz)) || !S->next_active) return;
  const float h = S->next_h32;
  const int sy = F.nx + 1, sz = (F.nx + 1) * (F.ny + 1);
  const int n0 = i + sy * j + sz * k;
  const int c = i + F.nx * (j + F.ny * k);
  F3 E[8], ub[8];
  ref_hex2<JIT>(F, n0, sy, sz, E);
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int na = n0 + (a & 1) + ((a >> 1) & 1) * sy + ((a >> 2) & 1) * sz;
    ub[a] = {F.ub[na], F.vb[na], F.wb[na]};
  }
  const float work = (OPT && F.time_order == 2) ? grad_dot_cached(F.Gh, F.nc, c, ub)
                     : JIT              ? grad_dot_cached(F.Gc, F.nc, c, ub)
                                        : grad_dot_f(E, ub);
  // compatible energy update; the increment is FP32, the accumulation
  // float-float
  float de = h * F.sig[c] * work / F.m[c];
  if (OPT && F.fh) {
    float work_hg = 0.f;
#pragma unroll
    for (int a = 0; a < 8; ++a) work_hg = dot_acc(hg_corner_f(F.fh, F.nc, c, a), ub[a], work_hg);
    de += h * work_hg / F.m[c];
  }
  const DF e1 = df_add_f(load_df(F.e, F.elo, c), -de);
  F.e[c] = e1.hi;
  F.elo[c] = e1.lo;
  F3 Dd[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) Dd[a] = h * ub[a];
  float vx, vy, vz;
  swept_low_faces_f(E, Dd, vx, vy, vz);
  F.dvx[c] = IN || i > 0 ? vx : 0.f;
  F.dvy[c] = IN || j > 0 ? vy : 0.f;
  F.dvz[c] = IN || k > 0 ? vz : 0.f;
}

// Hourglass corner forces of cell (i,j,k) on the reference mesh from u^n
// and the state at n (rho = m / V_E; cs from e).
template <bool JIT, bool IN>
__device__ __forceinline__ void m_hourglass_body(const Fields<float> &F, DevScalars *S, int i, int j, int k) {
  if ((!IN && (i >= F.nx || j >= F.ny || k >= F.nz)) || !S->next_active) return;
  const int sy = F.nx + 1, sz = (F.nx + 1) * (F.ny + 1);
  const int n0 = i + sy * j + sz * k;
  const int c = i + F.nx * (j + F.ny * k);
  F3 E[8], U[8], G[8];
  ref_hex2<JIT>(F, n0, sy, sz, E);
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int na = n0 + (a & 1) + ((a >> 1) & 1) * sy + ((a >> 2) & 1) * sz;
    U[a] = {F.u[na], F.v[na], F.w[na]};
  }
  if constexpr (JIT) {
#pragma unroll
    for (int a = 0; a < 8; ++a) G[a] = hg_corner_f(F.Gc, F.nc, c, a);
  } else {
    hex_grad_f(E, G);
  }
  const float e = F.e[c];
  const float g = F.gamma32;
  hourglass_store_f(E, G, U, F.VE[c], F.rho[c], sqrtf(g * (g - 1.f) * fmaxf(e, 0.f)), F.c_hg32, F.fh, F.nc, c);
}

// Corner gradients of the half-step hex, written to Gh, and
// dV/dt = sum_a G_a . u_a accumulated in corner order.  The corner's
// velocity is read again here (a cache hit) rather than held in registers
// through the volume and gradient sums.
template <int A = 0>
__device__ __forceinline__ void predict_corners(const Fields<float> &F, const F3 (&X)[8], int n0, int sy, int sz,
                                                int c, float &dvdt) {
  const F3 g = hex_corner_grad_f<A>(X);
  const int na = n0 + (A & 1) + ((A >> 1) & 1) * sy + ((A >> 2) & 1) * sz;
  dvdt = dot_acc(g, F3{F.u[na], F.v[na], F.w[na]}, dvdt);
  F.Gh[(3 * A + 0) * F.nc + c] = g.x;
  F.Gh[(3 * A + 1) * F.nc + c] = g.y;
  F.Gh[(3 * A + 2) * F.nc + c] = g.z;
  if constexpr (A < 7) predict_corners<A + 1>(F, X, n0, sy, sz, c, dvdt);
}

// Predictor-corrector half step of cell (i,j,k): e^{n+1/2} from sigma^n and
// u^n on the reference mesh, then EoS and viscosity on x_ref + dt/2 u^n;
// sigma^{n+1/2} replaces sigma, the corner gradients there go to Gh.
template <bool JIT, bool IN>
__device__ __forceinline__ void m_predict_body(const Fields<float> &F, DevScalars *S, int i, int j, int k) {
  if ((!IN && (i >= F.nx || j >= F.ny || k >= F.nz)) || !S->next_active) return;
  const float h = S->next_h32;
  const int sy = F.nx + 1, sz = (F.nx + 1) * (F.ny + 1);
  const int n0 = i + sy * j + sz * k;
  const int c = i + F.nx * (j + F.ny * k);
  F3 E[8], U[8];
  ref_hex2<JIT>(F, n0, sy, sz, E);
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int na = n0 + (a & 1) + ((a >> 1) & 1) * sy + ((a >> 2) & 1) * sz;
    U[a] = {F.u[na], F.v[na], F.w[na]};
  }
  const float work = JIT ? grad_dot_cached(F.Gc, F.nc, c, U) : grad_dot_f(E, U);
  const float m = F.m[c];
  float e = F.e[c] - 0.5f * h * F.sig[c] * work / m;
  if (F.fh) {
    float work_hg = 0.f;
#pragma unroll
    for (int a = 0; a < 8; ++a) work_hg = dot_acc(hg_corner_f(F.fh, F.nc, c, a), U[a], work_hg);
    e -= 0.5f * h * work_hg / m;
  }
  F3 X[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) X[a] = fma3(0.5f * h, U[a] - U[0], E[a]);
  const float V = hex_volume_f(X);
  if (!(V > 0.f)) set_status(S, V != V ? SALE_ENAN : SALE_ENEGVOL);
  // one corner gradient live at a time: stored, and its work taken, as made
  float dvdt = 0.f;
  predict_corners(F, X, n0, sy, sz, c, dvdt);
  const float rho = m / V;
  const float g = F.gamma32;
  const float p = (g - 1.f) * rho * e;
  const float cs = sqrtf(g * (g - 1.f) * fmaxf(e, 0.f));
  const float div = dvdt / V;
  const float L = V * rsqrtf(hex_max_face_area2_f(X));
  float q = 0.f;
  if (div < 0.f) {
    const float ld = L * div;
    q = rho * (F.c_q32 * ld * ld + F.c_l32 * cs * L * fabsf(div));
  }
  F.sig[c] = p + q;
}

// Lagrangian volume of a cell by closure: V_E minus its net swept volume.
template <bool IN>
__device__ __forceinline__ float lag_volume(const Fields<float> &F, int c, int i, int j, int k) {
  const int sy = F.nx, sz = F.nx * F.ny;
  float net = -F.dvx[c] - F.dvy[c] - F.dvz[c];
  if (IN || i + 1 < F.nx) net += F.dvx[c + 1];
  if (IN || j + 1 < F.ny) net += F.dvy[c + sy];
  if (IN || k + 1 < F.nz) net += F.dvz[c + sz];
  return F.VE[c] - net;
}

template <int AX, bool IN>
__device__ __forceinline__ void m_face_flux(const Fields<float> &F, int c, int i, int j, int k, float rho_c, float *mu,
                                            float *ep) {
  const int idx = AX == 0 ? i : AX == 1 ? j : k;
  const float *dv = AX == 0 ? F.dvx : AX == 1 ? F.dvy : F.dvz;
  if (!IN && idx == 0) {
    mu[c] = 0.f;
    ep[c] = 0.f;
    return;
  }
  const float v = dv[c];
  float rho_d, e_d;
  if (v > 0.f) {
    rho_d = rho_c;
    e_d = F.e[c];
  } else {
    const int stride = AX == 0 ? 1 : AX == 1 ? F.nx : F.nx * F.ny;
    const int d = c - stride;
    const float VL = lag_volume<IN>(F, d, AX == 0 ? i - 1 : i, AX == 1 ? j - 1 : j, AX == 2 ? k - 1 : k);
    rho_d = F.m[d] / VL;
    e_d = F.e[d];
  }
  const float f = rho_d * v;
  mu[c] = f;
  ep[c] = f * e_d;
}

// Second-order remap: the low-face flux along AX from the donor's limited
// linear profile of rho_L and e (F.vol, F.rho hold V_L and rho_L from the
// density pass), averaged over the swept slab.
template <int AX, bool IN>
__device__ __forceinline__ void m_face_flux2(const Fields<float> &F, int c, int i, int j, int k, float *mu,
                                             float *ep) {
  const int idx = AX == 0 ? i : AX == 1 ? j : k;
  const int n_ax = AX == 0 ? F.nx : AX == 1 ? F.ny : F.nz;
  const float *dv = AX == 0 ? F.dvx : AX == 1 ? F.dvy : F.dvz;
  if (!IN && idx == 0) {
    mu[c] = 0.f;
    ep[c] = 0.f;
    return;
  }
  const int stride = AX == 0 ? 1 : AX == 1 ? F.nx : F.nx * F.ny;
  const float v = dv[c];
  const bool hd = v > 0.f;
  const int d = hd ? c : c - stride;
  const int di = hd ? idx : idx - 1;  // donor index along AX
  const float rho_d = F.rho[d], e_d = F.e[d];
  float sr = 0.f, se = 0.f;
  if (di > 0 && di < n_ax - 1) {
    sr = vanleer_slope_f(rho_d - F.rho[d - stride], F.rho[d + stride] - rho_d);
    se = vanleer_slope_f(e_d - F.e[d - stride], F.e[d + stride] - e_d);
  }
  const float nu = fabsf(v) / F.vol[d];
  const float side = hd ? -1.f : 1.f;
  const float f = slab_average_f(rho_d, sr, nu, side) * v;
  mu[c] = f;
  ep[c] = f * slab_average_f(e_d, se, nu, side);
}

// Lagrangian volume and density of every cell (second-order remap only,
// which needs them at the donor's neighbours too).
template <bool IN>
__device__ __forceinline__ void m_density_body(const Fields<float> &F, DevScalars *S, int i, int j, int k) {
  if ((!IN && (i >= F.nx || j >= F.ny || k >= F.nz)) || !S->next_active || F.remap_order != 2) return;
  const int c = i + F.nx * (j + F.ny * k);
  const float VL = lag_volume<IN>(F, c, i, j, k);
  if (!(VL > 0.f)) set_status(S, VL != VL ? SALE_ENAN : SALE_ENEGVOL);
  F.vol[c] = VL;
  F.rho[c] = F.m[c] / VL;
}

// Lagrangian densities (closure) and donor-cell fluxes of the low faces.
template <bool IN>
__device__ __forceinline__ void m_fluxes_body(const Fields<float> &F, DevScalars *S, int i, int j, int k) {
  if ((!IN && (i >= F.nx || j >= F.ny || k >= F.nz)) || !S->next_active) return;
  const int c = i + F.nx * (j + F.ny * k);
  if (F.remap_order == 2) {
    m_face_flux2<0, IN>(F, c, i, j, k, F.mux, F.epx);
    m_face_flux2<1, IN>(F, c, i, j, k, F.muy, F.epy);
    m_face_flux2<2, IN>(F, c, i, j, k, F.muz, F.epz);
    return;
  }
  const float VL = lag_volume<IN>(F, c, i, j, k);
  if (!(VL > 0.f)) set_status(S, VL != VL ? SALE_ENAN : SALE_ENEGVOL);
  const float rho_c = F.m[c] / VL;
  m_face_flux<0, IN>(F, c, i, j, k, rho_c, F.mux, F.epx);
  m_face_flux<1, IN>(F, c, i, j, k, rho_c, F.muy, F.epy);
  m_face_flux<2, IN>(F, c, i, j, k, rho_c, F.muz, F.epz);
}

// ---------------------------------------------------------------------------
// Node remap (FP32)
// ---------------------------------------------------------------------------

// Whether the edge of node (i,j,k) along AX on side SIDE (0: towards +AX)
// lies in the mesh.
template <int AX, int SIDE>
__device__ __forceinline__ bool m_edge_exists(const Fields<float> &F, int i, int j, int k) {
  const int idx = AX == 0 ? i : AX == 1 ? j : k;
  const int n_ax = AX == 0 ? F.nx : AX == 1 ? F.ny : F.nz;
  return SIDE == 0 ? idx != n_ax : idx != 0;
}

// Momentum, mass and kinetic energy carried into node n through one of its
// edges by the dual flux psi of that edge (positive: towards +AX), upwinded.
template <int AX, int SIDE>
__device__ __forceinline__ void m_edge_apply(const Fields<float> &F, int n, float psi, DF &m, F3 &p, float &ke) {
  const int stride = AX == 0 ? 1 : AX == 1 ? (F.nx + 1) : (F.nx + 1) * (F.ny + 1);
  const int lo = SIDE == 0 ? n : n - stride;
  const int dn = psi > 0.f ? lo + stride : lo;
  const F3 ud = {F.u[dn], F.v[dn], F.w[dn]};
  const float flux = SIDE == 0 ? psi : -psi;
  m = df_add_f(m, flux);  // float-float: the node mass absorbs fluxes ~1% of it every cycle
  p = fma3(flux, ud, p);
  ke = __fmaf_rn(flux * 0.5f, dot_rn(ud, ud), ke);
}

// New node velocity, mass and kinetic-energy defect from the remapped sums.
template <bool IN>
__device__ __forceinline__ void m_remap_node_store(const Fields<float> &F, DevScalars *S, int i, int j, int k, int n,
                                                   DF m, F3 p, float ke) {
  if (!(m.hi > 0.f)) set_status(S, m.hi != m.hi ? SALE_ENAN : SALE_ENEGVOL);
  const float inv_m = 1.f / m.hi;
  float u1 = p.x * inv_m, v1 = p.y * inv_m, w1 = p.z * inv_m;
  if (!IN) wall_bc_f(F, i, j, k, u1, v1, w1);
  F.ub[n] = u1;
  F.vb[n] = v1;
  F.wb[n] = w1;
  F.mn[n] = m.hi;
  F.mnlo[n] = m.lo;
  F.dke[n] = __fmaf_rn(-0.5f * m.hi, dot_rn(F3{u1, v1, w1}, F3{u1, v1, w1}), ke);
}

// The node remap marches in k: a block covers a tile of node columns over
// kRemapChunk node planes.  The dual mass flux of a mesh edge is 1/8 of the
// sum, over the (up to) four cells around the edge, of each cell's pair
// (low-face + high-face mass flux along the edge), added in a fixed cell
// order; cells outside the mesh read as zero.  The pairs of the cell plane
// between two node planes serve the edges of both, and the k-edge below a
// node is the k-edge above the node beneath it, so a column forms each pair
// and each k-edge flux once, and every node sees bitwise the same fluxes as
// its neighbours across the edge.
struct RemapCarry {
  float x0[2], x1[2];  // x-edge pairs of the cell plane below: edges at ci = i, i - 1; cells cj = j - 1, j
  float y0[2], y1[2];  // y-edge pairs: edges at cj = j, j - 1; cells ci = i - 1, i
  float zc[4];         // mu_z of the cells (i - 1 + (s & 1), j - 1 + (s >> 1)) of this node's cell plane
  float psi_below;     // dual flux of the k-edge ending at this node
};

template <bool IN>
__device__ __forceinline__ float mu_at(const float *mu, const Fields<float> &F, int ci, int cj, int ck) {
  if (!IN && (ci < 0 || cj < 0 || ck < 0 || ci >= F.nx || cj >= F.ny || ck >= F.nz)) return 0.f;
  return mu[ci + F.nx * (cj + F.ny * ck)];
}

// The x- and y-edge pairs of the cell plane ck around node column (i, j).
template <bool IN>
__device__ __forceinline__ void remap_plane_pairs(const Fields<float> &F, int i, int j, int ck, float (&x0)[2],
                                                  float (&x1)[2], float (&y0)[2], float (&y1)[2]) {
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    const float a = mu_at<IN>(F.mux, F, i - 1, j - 1 + d, ck), b = mu_at<IN>(F.mux, F, i, j - 1 + d, ck),
                c = mu_at<IN>(F.mux, F, i + 1, j - 1 + d, ck);
    x1[d] = a + b;
    x0[d] = b + c;
    const float e = mu_at<IN>(F.muy, F, i - 1 + d, j - 1, ck), f = mu_at<IN>(F.muy, F, i - 1 + d, j, ck),
                g = mu_at<IN>(F.muy, F, i - 1 + d, j + 1, ck);
    y1[d] = e + f;
    y0[d] = f + g;
  }
}

__device__ __forceinline__ float edge_psi4(float a, float b, float c, float d) {
  float psi = 0.f;
  psi += a;
  psi += b;
  psi += c;
  psi += d;
  return 0.125f * psi;
}

template <bool IN>
__device__ __forceinline__ void m_remap_node_step(const Fields<float> &F, DevScalars *S, int i, int j, int k,
                                                  RemapCarry &cr) {
  float x0[2], x1[2], y0[2], y1[2], zn[4];
  remap_plane_pairs<IN>(F, i, j, k, x0, x1, y0, y1);
#pragma unroll
  for (int s = 0; s < 4; ++s) zn[s] = mu_at<IN>(F.muz, F, i - 1 + (s & 1), j - 1 + (s >> 1), k + 1);
  const float px0 = edge_psi4(cr.x0[0], cr.x0[1], x0[0], x0[1]);
  const float px1 = edge_psi4(cr.x1[0], cr.x1[1], x1[0], x1[1]);
  const float py0 = edge_psi4(cr.y0[0], cr.y0[1], y0[0], y0[1]);
  const float py1 = edge_psi4(cr.y1[0], cr.y1[1], y1[0], y1[1]);
  const float pz0 = edge_psi4(cr.zc[0] + zn[0], cr.zc[1] + zn[1], cr.zc[2] + zn[2], cr.zc[3] + zn[3]);
  const float pz1 = cr.psi_below;
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    cr.x0[d] = x0[d];
    cr.x1[d] = x1[d];
    cr.y0[d] = y0[d];
    cr.y1[d] = y1[d];
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) cr.zc[s] = zn[s];
  cr.psi_below = pz0;

  const int n = i + (F.nx + 1) * (j + (F.ny + 1) * k);
  const float m0 = F.mn[n];
  const F3 u0 = {F.u[n], F.v[n], F.w[n]};
  DF m = {m0, F.mnlo[n]};
  F3 p = m0 * u0;
  float ke = 0.5f * m0 * dot_rn(u0, u0);
  if (IN || m_edge_exists<0, 0>(F, i, j, k)) m_edge_apply<0, 0>(F, n, px0, m, p, ke);
  if (IN || m_edge_exists<0, 1>(F, i, j, k)) m_edge_apply<0, 1>(F, n, px1, m, p, ke);
  if (IN || m_edge_exists<1, 0>(F, i, j, k)) m_edge_apply<1, 0>(F, n, py0, m, p, ke);
  if (IN || m_edge_exists<1, 1>(F, i, j, k)) m_edge_apply<1, 1>(F, n, py1, m, p, ke);
  if (IN || m_edge_exists<2, 0>(F, i, j, k)) m_edge_apply<2, 0>(F, n, pz0, m, p, ke);
  if (IN || m_edge_exists<2, 1>(F, i, j, k)) m_edge_apply<2, 1>(F, n, pz1, m, p, ke);
  m_remap_node_store<IN>(F, S, i, j, k, n, m, p, ke);
}

// Tile (bx, by) of node columns over the node planes of chunk kc.
template <int SH>
__device__ __forceinline__ void m_remap_column(const Fields<float> &F, DevScalars *S, int bx, int by, int kc) {
  const int i = bx * tile_x(SH) + threadIdx.x, j = by * tile_y(SH) + threadIdx.y;
  const int k0 = kc * kRemapChunk;
  const int k1 = min(k0 + kRemapChunk, F.nz + 1);
  if (i > F.nx || j > F.ny) return;
  if (!S->next_active) {  // inactive cycle: velocity carries over unchanged
    for (int k = k0; k < k1; ++k) {
      const int n = i + (F.nx + 1) * (j + (F.ny + 1) * k);
      F.ub[n] = F.u[n];
      F.vb[n] = F.v[n];
      F.wb[n] = F.w[n];
    }
    return;
  }
  // the x/y extent of the tile's cells and neighbours lies in the mesh
  const int i0 = bx * tile_x(SH), j0 = by * tile_y(SH);
  const bool xy_in = i0 >= 1 && i0 + tile_x(SH) <= F.nx - 1 && j0 >= 1 && j0 + tile_y(SH) <= F.ny - 1;
  RemapCarry cr;
  remap_plane_pairs<false>(F, i, j, k0 - 1, cr.x0, cr.x1, cr.y0, cr.y1);
  float zb[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    zb[s] = mu_at<false>(F.muz, F, i - 1 + (s & 1), j - 1 + (s >> 1), k0 - 1);
    cr.zc[s] = mu_at<false>(F.muz, F, i - 1 + (s & 1), j - 1 + (s >> 1), k0);
  }
  cr.psi_below = edge_psi4(zb[0] + cr.zc[0], zb[1] + cr.zc[1], zb[2] + cr.zc[2], zb[3] + cr.zc[3]);
  for (int k = k0; k < k1; ++k) {
    if (xy_in && k >= 1 && k <= F.nz - 2) m_remap_node_step<true>(F, S, i, j, k, cr);
    else m_remap_node_step<false>(F, S, i, j, k, cr);
  }
}

// Threads per SM the single-mesh node remap is compiled to keep resident.
constexpr int kRemapResident = 1024;

template <int SH>
__global__ void __launch_bounds__(tile_x(SH) * tile_y(SH), kRemapResident / (tile_x(SH) * tile_y(SH)))
    k_m_remap_nodes_march(Fields<float> F, DevScalars *S) {
  m_remap_column<SH>(F, S, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ---------------------------------------------------------------------------
// Cell remap, EoS, viscosity, CFL dt (FP32; dt reduced as a double)
// ---------------------------------------------------------------------------

// EoS and viscosity of cell (i,j,k) on the reference mesh; returns its CFL
// step.
template <bool JIT>
__device__ __forceinline__ float m_eos_cell(const Fields<float> &F, int c, int i, int j, int k, float m, float e,
                                            bool store_all) {
  const int sy = F.nx + 1, sz = (F.nx + 1) * (F.ny + 1);
  const int n0 = i + sy * j + sz * k;
  F3 U[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int na = n0 + (a & 1) + ((a >> 1) & 1) * sy + ((a >> 2) & 1) * sz;
    U[a] = {F.u[na], F.v[na], F.w[na]};
  }
  float dvdt;
  if constexpr (JIT) {
    dvdt = grad_dot_cached(F.Gc, F.nc, c, U);
  } else {
    F3 E[8];
    ref_hex2<JIT>(F, n0, sy, sz, E);
    dvdt = grad_dot_f(E, U);
  }
  // every rounding fixed (see dot_rn): sigma and the CFL step feed the
  // next cycle of every kernel that calls this
  const float V = F.VE[c];
  const float inv_v = 1.f / V;
  const float div = __fmul_rn(dvdt, inv_v);
  const float L = F.LE[c];
  const float rho = __fmul_rn(m, inv_v);
  const float g = F.gamma32;
  const float p = __fmul_rn(__fmul_rn(g - 1.f, rho), e);
  const float cs = sqrtf(__fmul_rn(__fmul_rn(g, g - 1.f), fmaxf(e, 0.f)));
  float q_rho = 0.f;
  if (div < 0.f) {
    const float ld = __fmul_rn(L, div);
    q_rho = __fmaf_rn(__fmul_rn(F.c_q32, ld), ld, __fmul_rn(__fmul_rn(__fmul_rn(F.c_l32, cs), L), fabsf(div)));
  }
  const float q = __fmul_rn(rho, q_rho);
  F.rho[c] = rho;
  F.sig[c] = __fadd_rn(p, q);
  if (store_all) {
    F.p[c] = p;
    F.q[c] = q;
    F.cs[c] = cs;
    F.vol[c] = V;
  }
  return __fdiv_rn(__fmul_rn(F.cfl32, L), sqrtf(__fmaf_rn(cs, cs, 2.f * q_rho)));
}

// Cell remap + EoS of cell (i,j,k) in an active cycle; returns its CFL
// step (infinite outside the mesh).
template <bool JIT, bool IN>
__device__ __forceinline__ float m_remap_eos_cell(const Fields<float> &F, DevScalars *S, int i, int j, int k) {
  float dtc = INFINITY;
  if (IN || (i < F.nx && j < F.ny && k < F.nz)) {
    const int sy = F.nx, sz = F.nx * F.ny;
    const int c = i + sy * j + sz * k;
    // float-float: every flux is added to the conserved quantities on its
    // own, so what leaves one cell is exactly what the next one receives
    const DF m0 = load_df(F.m, F.mlo, c);
    DF m1 = df_add_f(m0, -F.mux[c]);
    m1 = df_add_f(m1, -F.muy[c]);
    m1 = df_add_f(m1, -F.muz[c]);
    DF ie = df_mul(m0, load_df(F.e, F.elo, c));
    ie = df_add_f(ie, -F.epx[c]);
    ie = df_add_f(ie, -F.epy[c]);
    ie = df_add_f(ie, -F.epz[c]);
    if (IN || i + 1 < F.nx) { m1 = df_add_f(m1, F.mux[c + 1]); ie = df_add_f(ie, F.epx[c + 1]); }
    if (IN || j + 1 < F.ny) { m1 = df_add_f(m1, F.muy[c + sy]); ie = df_add_f(ie, F.epy[c + sy]); }
    if (IN || k + 1 < F.nz) { m1 = df_add_f(m1, F.muz[c + sz]); ie = df_add_f(ie, F.epz[c + sz]); }
    if (F.ke_fix) {
      const int nsy = F.nx + 1, nsz = (F.nx + 1) * (F.ny + 1);
      const int n0 = i + nsy * j + nsz * k;
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int ni = i + (a & 1), nj = j + ((a >> 1) & 1), nk = k + ((a >> 2) & 1);
        const float share = IN ? 0.125f
                               : ((ni == 0 || ni == F.nx) ? 1.f : 0.5f) * ((nj == 0 || nj == F.ny) ? 1.f : 0.5f) *
                                     ((nk == 0 || nk == F.nz) ? 1.f : 0.5f);
        ie = df_add_f(ie, F.dke[n0 + (a & 1) + ((a >> 1) & 1) * nsy + ((a >> 2) & 1) * nsz] * share);
      }
    }
    if (!(m1.hi > 0.f)) set_status(S, m1.hi != m1.hi ? SALE_ENAN : SALE_ENEGVOL);
    const DF e1 = df_div(ie, m1);
    F.m[c] = m1.hi;
    F.mlo[c] = m1.lo;
    F.e[c] = e1.hi;
    F.elo[c] = e1.lo;
    const float d = m_eos_cell<JIT>(F, c, i, j, k, m1.hi, e1.hi, false);
    dtc = d == d ? d : (set_status(S, SALE_ENAN), INFINITY);
  }
  return dtc;
}

// EoS/viscosity/dt without a remap: kDtInit / kDtPropose, or no dt at all
// (mode < 0: only refresh the derived fields p, q, cs, vol, rho).
template <bool JIT>
__device__ __forceinline__ void m_eos_body(const Fields<float> &F, DevScalars *S, int i, int j, int k, int mode,
                                           unsigned nblk) {
  if (mode >= 0 && S->status != 0) return;
  float dtc = INFINITY;
  if (i < F.nx && j < F.ny && k < F.nz) {
    const int c = i + F.nx * (j + F.ny * k);
    const float d = m_eos_cell<JIT>(F, c, i, j, k, F.m[c], F.e[c], true);
    dtc = d == d ? d : (set_status(S, SALE_ENAN), INFINITY);
  }
  if (mode >= 0) block_min_dt32_and_finalize(F, S, dtc, mode, 0.0, nblk);
}

// ---------------------------------------------------------------------------
// Kernels: tiles of TX x TY threads over one k plane; single mesh (3D grid)
// and batched (table)
// ---------------------------------------------------------------------------

// IN: the block's whole tile lies in 1 <= index <= n - 2 on every axis
// (cells and nodes alike), so every neighbour a body reads exists, no node
// is on a wall and every node is shared by eight cells: the bodies drop
// those tests, with bitwise the same results.
template <bool JIT, bool IN, bool OPT>
__device__ __forceinline__ void run_body(int kid, const Fields<float> &F, DevScalars *S, int i, int j, int k,
                                         unsigned nblk, int mode) {
  switch (kid) {
    case kMixNodes: m_nodes_body<JIT, IN, OPT>(F, S, i, j, k); break;
    case kMixCells: m_cells_body<JIT, IN, OPT>(F, S, i, j, k); break;
    case kMixFluxes: m_fluxes_body<IN>(F, S, i, j, k); break;
    case kMixEos: m_eos_body<JIT>(F, S, i, j, k, mode, nblk); break;
    case kMixDensity: m_density_body<IN>(F, S, i, j, k); break;
    case kMixPredict: m_predict_body<JIT, IN>(F, S, i, j, k); break;
    case kMixHourglass: m_hourglass_body<JIT, IN>(F, S, i, j, k); break;
    default: break;
  }
}

template <int SH>
__device__ __forceinline__ bool tile_interior(const Fields<float> &F, int bx, int by, int k) {
  const int i0 = bx * tile_x(SH), j0 = by * tile_y(SH);
  return i0 >= 1 && i0 + tile_x(SH) <= F.nx - 1 && j0 >= 1 && j0 + tile_y(SH) <= F.ny - 1 && k >= 1 &&
         k <= F.nz - 2;
}

template <int KID, bool JIT, int SH, bool OPT>
__device__ __forceinline__ void run_tile(const Fields<float> &F, DevScalars *S, int bx, int by, int k, unsigned nblk,
                                         int mode) {
  const int i = bx * tile_x(SH) + threadIdx.x, j = by * tile_y(SH) + threadIdx.y;
  if (KID != kMixEos && tile_interior<SH>(F, bx, by, k)) run_body<JIT, true, OPT>(KID, F, S, i, j, k, nblk, mode);
  else run_body<JIT, false, OPT>(KID, F, S, i, j, k, nblk, mode);
}

// Blocks per SM the register budget is held to, per kernel and block size:
// 768 resident threads per SM for the cell pass, 1024 (64 registers) for
// the others; the node gathers lose more to occupancy than they gain from
// the extra loads in flight of an uncapped build.
__host__ __device__ constexpr int min_blocks(int kid, int threads) {
  return (kid == kMixCells || kid == kMixPredict) ? 768 / threads
         : (kid == kMixRemapEos || kid == kMixEos || kid == kMixNodes || kid == kMixRemapNodes) ? 1024 / threads
                                                                                                 : 1;
}

template <int KID, bool JIT, int SH, bool OPT>
__global__ void __launch_bounds__(tile_x(SH) * tile_y(SH), min_blocks(KID, tile_x(SH) * tile_y(SH)))
    k_m(Fields<float> F, DevScalars *S, int mode) {
  const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
  run_tile<KID, JIT, SH, OPT>(F, S, blockIdx.x, blockIdx.y, blockIdx.z, nblk, mode);
}

// Batched: block b works on mesh tab[b].x, tile (tab[b].y, tab[b].z) of
// plane tab[b].w; the part of the mesh's descriptor these kernels read is
// staged in shared memory.  AJ: some mesh of the batch is jittered (each
// block then picks its mesh's body at run time); a batch of unjittered
// meshes runs kernels compiled with that body alone, fewer registers live.
template <int KID, int SH, bool AJ>
__global__ void __launch_bounds__(tile_x(SH) * tile_y(SH), min_blocks(KID, tile_x(SH) * tile_y(SH)))
    kb_m(const BatchItem *items, const int4 *tab) {
  __shared__ BatchItem it;
  const int4 t = tab[blockIdx.x];
  const int tid = threadIdx.x + tile_x(SH) * threadIdx.y;
  const int *src = reinterpret_cast<const int *>(items + t.x);
  int *dst = reinterpret_cast<int *>(&it);
  for (int w = tid; w < (int)(kBatchItemStaged / sizeof(int)); w += tile_x(SH) * tile_y(SH)) dst[w] = src[w];
  __syncthreads();
  // batches take neither the predictor-corrector step nor hourglass control
  if (AJ && it.F.off4) run_tile<KID, true, SH, false>(it.F, it.S, t.y, t.z, t.w, it.nblk_cell, 0);
  else run_tile<KID, false, SH, false>(it.F, it.S, t.y, t.z, t.w, it.nblk_cell, 0);
}

// Threads per SM the remap + EoS pass is compiled to keep resident (its
// register budget), single mesh and batch.
constexpr int kEosResident = 1280;
constexpr int kEosResidentBatch = 1024;  // batch blocks read the descriptor from shared memory: more registers live

// Remap + EoS + dt of tile (bx, by) over the cell planes of chunk kc (of
// kEosPlanes): the blocks' dt minima, two same-address atomics each, are
// kEosPlanes times fewer than with one plane per block, and the minimum is
// exact.  nblk = blocks of this mesh (last-block detection).
template <bool JIT, int SH>
__device__ __forceinline__ void m_remap_eos_column(const Fields<float> &F, DevScalars *S, int bx, int by, int kc,
                                                   unsigned nblk) {
  if (!S->next_active) return;  // uniform over the mesh's blocks: S changes only in its last block
  const int i = bx * tile_x(SH) + threadIdx.x, j = by * tile_y(SH) + threadIdx.y;
  const int k0 = kc * kEosPlanes, k1 = min(k0 + kEosPlanes, F.nz);
  float dtc = INFINITY;
  for (int k = k0; k < k1; ++k) {
    const float d = tile_interior<SH>(F, bx, by, k) ? m_remap_eos_cell<JIT, true>(F, S, i, j, k)
                                                    : m_remap_eos_cell<JIT, false>(F, S, i, j, k);
    dtc = fminf(dtc, d);
  }
  block_min_dt32_and_finalize(F, S, dtc, kDtAdvance, 0.0, nblk);
}

template <bool JIT, int SH>
__global__ void __launch_bounds__(tile_x(SH) * tile_y(SH), kEosResident / (tile_x(SH) * tile_y(SH)))
    k_m_remap_eos_planes(Fields<float> F, DevScalars *S) {
  m_remap_eos_column<JIT, SH>(F, S, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x * gridDim.y * gridDim.z);
}

// Batched remap + EoS + dt: block b covers chunk tab[b].w of tile
// (tab[b].y, tab[b].z) of mesh tab[b].x.
template <int SH, bool AJ>
__global__ void __launch_bounds__(tile_x(SH) * tile_y(SH), kEosResidentBatch / (tile_x(SH) * tile_y(SH)))
    kb_m_remap_eos_planes(const BatchItem *items, const int4 *tab) {
  __shared__ BatchItem it;
  const int4 t = tab[blockIdx.x];
  const int tid = threadIdx.x + tile_x(SH) * threadIdx.y;
  const int *src = reinterpret_cast<const int *>(items + t.x);
  int *dst = reinterpret_cast<int *>(&it);
  for (int w = tid; w < (int)(kBatchItemStaged / sizeof(int)); w += tile_x(SH) * tile_y(SH)) dst[w] = src[w];
  __syncthreads();
  if (AJ && it.F.off4) m_remap_eos_column<true, SH>(it.F, it.S, t.y, t.z, t.w, it.nblk_cell);
  else m_remap_eos_column<false, SH>(it.F, it.S, t.y, t.z, t.w, it.nblk_cell);
}

// Batched node remap: block b marches over chunk tab[b].w of the node
// columns of tile (tab[b].y, tab[b].z) of mesh tab[b].x.
template <int SH>
__global__ void __launch_bounds__(tile_x(SH) * tile_y(SH), 1024 / (tile_x(SH) * tile_y(SH)))
    kb_m_remap_nodes_march(const BatchItem *items, const int4 *tab) {
  __shared__ BatchItem it;
  const int4 t = tab[blockIdx.x];
  const int tid = threadIdx.x + tile_x(SH) * threadIdx.y;
  const int *src = reinterpret_cast<const int *>(items + t.x);
  int *dst = reinterpret_cast<int *>(&it);
  for (int w = tid; w < (int)(kBatchItemStaged / sizeof(int)); w += tile_x(SH) * tile_y(SH)) dst[w] = src[w];
  __syncthreads();
  m_remap_column<SH>(it.F, it.S, t.y, t.z, t.w);
}

// Per mesh of a batch: t_end = inf, cycle_limit = cycle + cycles, decide.
__global__ void kb_set_limits(const BatchItem *items, int n, long long cycles) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  volatile DevScalars *S = items[i].S;
  S->t_end = INFINITY;
  S->cycle_limit = S->cycle + cycles;
  decide_next(S);
}

// Gather (t, dt, cycle, status) of every mesh into one array for the host.
__global__ void kb_gather(const BatchItem *items, int n, BatchStatus *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const DevScalars *S = items[i].S;
  out[i] = {S->t, S->dt, S->cycle, S->status};
}

// Grid of tiles of a shape over an (ni, nj, nk) box of nodes or cells.
dim3 tile_grid(int ni, int nj, int nk, int shape) {
  return dim3((unsigned)((ni + tile_x(shape) - 1) / tile_x(shape)),
              (unsigned)((nj + tile_y(shape) - 1) / tile_y(shape)), (unsigned)nk);
}

void launch_m_init_cells(const Fields<float> &F, DevScalars *S, const double *rho0, const double *p0,
                         long long dep_cell, double dep_e, float *VE, float *LE, float *Gc, cudaStream_t st) {
  k_m_init_cells<<<(unsigned)((F.nc + kBlock - 1) / kBlock), kBlock, 0, st>>>(F, S, rho0, p0, dep_cell, dep_e, VE,
                                                                              LE, Gc);
}

template <int KID, int SH>
static void launch_shaped(const Fields<float> &F, DevScalars *S, int mode, cudaStream_t st) {
  if constexpr (KID == kMixRemapNodes) {
    const dim3 g = tile_grid(F.nx + 1, F.ny + 1, (F.nz + 1 + kRemapChunk - 1) / kRemapChunk, SH);
    k_m_remap_nodes_march<SH><<<g, dim3(tile_x(SH), tile_y(SH)), 0, st>>>(F, S);
    return;
  }
  if constexpr (KID == kMixRemapEos) {
    const dim3 g = tile_grid(F.nx, F.ny, (F.nz + kEosPlanes - 1) / kEosPlanes, SH);
    if (F.off4) k_m_remap_eos_planes<true, SH><<<g, dim3(tile_x(SH), tile_y(SH)), 0, st>>>(F, S);
    else k_m_remap_eos_planes<false, SH><<<g, dim3(tile_x(SH), tile_y(SH)), 0, st>>>(F, S);
    return;
  }
  const bool node = KID == kMixNodes || KID == kMixRemapNodes;
  const dim3 g = node ? tile_grid(F.nx + 1, F.ny + 1, F.nz + 1, SH) : tile_grid(F.nx, F.ny, F.nz, SH);
  const dim3 b(tile_x(SH), tile_y(SH));
  if constexpr (KID == kMixNodes || KID == kMixCells) {
    if (F.time_order == 2 || F.fh) {
      if (F.off4) k_m<KID, true, SH, true><<<g, b, 0, st>>>(F, S, mode);
      else k_m<KID, false, SH, true><<<g, b, 0, st>>>(F, S, mode);
      return;
    }
  }
  if (F.off4) k_m<KID, true, SH, false><<<g, b, 0, st>>>(F, S, mode);
  else k_m<KID, false, SH, false><<<g, b, 0, st>>>(F, S, mode);
}

template <int KID>
static void launch_one(const Fields<float> &F, DevScalars *S, int mode, int shape, cudaStream_t st) {
  switch (shape) {
    case 1: launch_shaped<KID, 1>(F, S, mode, st); break;
    case 2: launch_shaped<KID, 2>(F, S, mode, st); break;
    case 3: launch_shaped<KID, 3>(F, S, mode, st); break;
    case 4: launch_shaped<KID, 4>(F, S, mode, st); break;
    default: launch_shaped<KID, 0>(F, S, mode, st); break;
  }
}

void launch_m_kernel(int kid, const Fields<float> &F, DevScalars *S, int mode, int shape, cudaStream_t st) {
  switch (kid) {
    case kMixNodes: launch_one<kMixNodes>(F, S, mode, shape, st); break;
    case kMixCells: launch_one<kMixCells>(F, S, mode, shape, st); break;
    case kMixFluxes: launch_one<kMixFluxes>(F, S, mode, shape, st); break;
    case kMixRemapNodes: launch_one<kMixRemapNodes>(F, S, mode, shape, st); break;
    case kMixRemapEos: launch_one<kMixRemapEos>(F, S, mode, shape, st); break;
    case kMixEos: launch_one<kMixEos>(F, S, mode, shape, st); break;
    case kMixDensity: launch_one<kMixDensity>(F, S, mode, shape, st); break;
    case kMixPredict: launch_one<kMixPredict>(F, S, mode, shape, st); break;
    case kMixHourglass: launch_one<kMixHourglass>(F, S, mode, shape, st); break;
    default: break;
  }
}

template <int SH, bool AJ>
static void launch_batch_shaped(int kid, const BatchItem *items, const int4 *tab, unsigned nblocks, cudaStream_t st) {
  const dim3 b(tile_x(SH), tile_y(SH));
  switch (kid) {
    case kMixNodes: kb_m<kMixNodes, SH, AJ><<<nblocks, b, 0, st>>>(items, tab); break;
    case kMixCells: kb_m<kMixCells, SH, AJ><<<nblocks, b, 0, st>>>(items, tab); break;
    case kMixFluxes: kb_m<kMixFluxes, SH, AJ><<<nblocks, b, 0, st>>>(items, tab); break;
    case kMixRemapNodes: kb_m_remap_nodes_march<SH><<<nblocks, b, 0, st>>>(items, tab); break;
    case kMixRemapEos: kb_m_remap_eos_planes<SH, AJ><<<nblocks, b, 0, st>>>(items, tab); break;
    case kMixDensity: kb_m<kMixDensity, SH, AJ><<<nblocks, b, 0, st>>>(items, tab); break;
    default: break;
  }
}

template <bool AJ>
static void launch_batch_any(int kid, const BatchItem *items, const int4 *tab, unsigned nblocks, int shape,
                             cudaStream_t st) {
  switch (shape) {
    case 1: launch_batch_shaped<1, AJ>(kid, items, tab, nblocks, st); break;
    case 2: launch_batch_shaped<2, AJ>(kid, items, tab, nblocks, st); break;
    case 3: launch_batch_shaped<3, AJ>(kid, items, tab, nblocks, st); break;
    case 4: launch_batch_shaped<4, AJ>(kid, items, tab, nblocks, st); break;
    default: launch_batch_shaped<0, AJ>(kid, items, tab, nblocks, st); break;
  }
}

void launch_m_batch(int kid, const BatchItem *items, const int4 *tab, unsigned nblocks, int shape, bool any_jit,
                    cudaStream_t st) {
  if (any_jit) launch_batch_any<true>(kid, items, tab, nblocks, shape, st);
  else launch_batch_any<false>(kid, items, tab, nblocks, shape, st);
}

// Field transfers of FP32-mixed states: FP64 values to FP32 (hi, optional lo)
// pairs and back, with the same roundings as the host would take: hi = x
// rounded to FP32, lo = (x - hi) rounded to FP32; x = hi + lo in FP64.
__global__ void k_split64(const double *__restrict__ in, float *__restrict__ hi, float *__restrict__ lo,
                          long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double x = in[i];
    const float h = (float)x;
    hi[i] = h;
    if (lo) lo[i] = (float)(x - (double)h);
  }
}

__global__ void k_join64(const float *__restrict__ hi, const float *__restrict__ lo, double *__restrict__ out,
                         long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = lo ? (double)hi[i] + (double)lo[i] : (double)hi[i];
}

static unsigned grid_stride_blocks(long long n) {
  const long long b = (n + kBlock - 1) / kBlock;
  return (unsigned)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

void launch_split64(const double *in, float *hi, float *lo, long long n, cudaStream_t st) {
  k_split64<<<grid_stride_blocks(n), kBlock, 0, st>>>(in, hi, lo, n);
}

void launch_join64(const float *hi, const float *lo, double *out, long long n, cudaStream_t st) {
  k_join64<<<grid_stride_blocks(n), kBlock, 0, st>>>(hi, lo, out, n);
}

void launch_batch_limits(const BatchItem *items, int n, long long cycles, cudaStream_t st) {
  kb_set_limits<<<(n + 127) / 128, 128, 0, st>>>(items, n, cycles);
}

void launch_batch_gather(const BatchItem *items, int n, BatchStatus *out, cudaStream_t st) {
  kb_gather<<<(n + 127) / 128, 128, 0, st>>>(items, n, out);
}

}  // namespace sale
