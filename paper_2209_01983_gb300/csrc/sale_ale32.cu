// sale_ale32.cu -- FP32-mixed kernels of the Eulerian (ALE, remap every
// cycle) cycle.
//
// Field storage and the bulk of the arithmetic are FP32; FP64 is kept for
// the reference hex volumes (computed once in FP64 and stored), the
// Lagrangian internal-energy update (accumulated in FP64) and the
// conservation sums (diagnostics).  FP64 runs at 1/64 of the FP32 rate on
// GB300, so the FP64 islands are kept to a few operations per cell.
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
//  * The node force gathers face terms: F_a = (1/24) sum over the 12 mesh
//    faces at node a of (sigma_low - sigma_high) t_f, t_f = (p1 + 2 p2 + p3)
//    x (p3 - p1) over the face's other nodes relative to a; it vanishes
//    exactly where sigma is uniform.
#include "sale_device.cuh"

namespace sale {

namespace {

struct F3 {
  float x, y, z;
};
__device__ __forceinline__ F3 operator+(F3 a, F3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ F3 operator-(F3 a, F3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ F3 operator*(float s, F3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ F3 crossf(F3 a, F3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ float dotf(F3 a, F3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Jitter offset of a node (one 16-byte load: x, y, z, unused).
__device__ __forceinline__ float4 node_off(const Fields<float> &F, long long n) {
  return F.off4 ? __ldg(F.off4 + n) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Position of a node relative to a base node with offset oa, the two
// differing by the index offset (ox, oy, oz): o * h + (offset - oa).
__device__ __forceinline__ F3 rel_pos(const Fields<float> &F, float4 oa, long long nb, int ox, int oy, int oz) {
  const float4 ob = node_off(F, nb);
  return {(float)ox * F.hx + (ob.x - oa.x), (float)oy * F.hy + (ob.y - oa.y), (float)oz * F.hz + (ob.z - oa.z)};
}

// Reference nodes of cell (i,j,k) relative to its node 0.
__device__ __forceinline__ void ref_hex(const Fields<float> &F, const long long (&nid)[8], F3 (&E)[8]) {
  const float4 o0 = node_off(F, nid[0]);
  E[0] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int a = 1; a < 8; ++a) E[a] = rel_pos(F, o0, nid[a], a & 1, (a >> 1) & 1, (a >> 2) & 1);
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
      s += dotf(crossf(pa + 2.f * pb + pc, pc - pa), U[face_node(f, k)]);
    }
  }
  return s * (1.f / 24.f);
}

// Side quad (L_a, E_a, E_b, L_b) term, expanded in the displacements.
__device__ __forceinline__ float side_term(const F3 (&E)[8], const F3 (&D)[8], int a, int b) {
  return 4.f * dotf(crossf(E[a], E[b]), D[a] + D[b]) - 2.f * dotf(E[a] + E[b], crossf(D[a], D[b]));
}

// Lagrangian face (p0,p1,p2,p3) plus the reversed reference face, expanded.
__device__ __forceinline__ float pair_term(const F3 (&E)[8], const F3 (&D)[8], int p0, int p1, int p2, int p3) {
  const F3 e1 = E[p2] - E[p0], e2 = E[p3] - E[p1];
  const F3 d1 = D[p2] - D[p0], d2 = D[p3] - D[p1];
  const F3 se = E[p0] + E[p1] + E[p2] + E[p3];
  const F3 sd = D[p0] + D[p1] + D[p2] + D[p3];
  return dotf(se, crossf(e1, d2) + crossf(d1, e2) + crossf(d1, d2)) + dotf(sd, crossf(e1 + d1, e2 + d2));
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
                                                         float *VE, float *LE) {
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
  F.m[c] = (float)m;
  F.e[c] = (float)e;
  VE[c] = (float)V;
  LE[c] = (float)(V / sqrt(hex_max_face_area2(X)));
}

// ---------------------------------------------------------------------------
// Lagrangian phase
// ---------------------------------------------------------------------------

// Face term of one mesh face through node (i,j,k): the lower cell across
// the face is s (bits: cell = node - 1 + bit), the face is normal to D.
template <int SB, int D>
__device__ __forceinline__ void node_face_force(const Fields<float> &F, long long n, float4 oa, int i, int j, int k,
                                                const float (&sig)[8], F3 &f) {
  if ((SB >> D) & 1) return;  // the cell must be the lower one across the plane
  const int c0 = i - 1 + (SB & 1), c1 = j - 1 + ((SB >> 1) & 1), c2 = k - 1 + ((SB >> 2) & 1);
  const int cc[3] = {c0, c1, c2};
  const int nn[3] = {F.nx, F.ny, F.nz};
  constexpr int D1 = (D + 1) % 3, D2 = (D + 2) % 3;
  if (cc[D1] < 0 || cc[D1] >= nn[D1] || cc[D2] < 0 || cc[D2] >= nn[D2]) return;  // face outside the mesh
  const float slo = sig[SB];
  const float shi = sig[SB | (1 << D)];
  constexpr int A = 7 - SB;          // local corner of the node in the lower cell
  constexpr int FACE = 2 * D + 1;    // the lower cell's high face normal to D
  constexpr int K = face_slot(FACE, A);
  constexpr int B1 = face_node(FACE, (K + 1) & 3), B2 = face_node(FACE, (K + 2) & 3),
                B3 = face_node(FACE, (K + 3) & 3);
  const long long sx = 1, sy = F.nx + 1, sz = (long long)(F.nx + 1) * (F.ny + 1);
  // node offsets from (i,j,k): cell offset (bit - 1) plus the local node bits
  constexpr int O1x = (SB & 1) + (B1 & 1) - 1, O1y = ((SB >> 1) & 1) + ((B1 >> 1) & 1) - 1,
                O1z = ((SB >> 2) & 1) + ((B1 >> 2) & 1) - 1;
  constexpr int O2x = (SB & 1) + (B2 & 1) - 1, O2y = ((SB >> 1) & 1) + ((B2 >> 1) & 1) - 1,
                O2z = ((SB >> 2) & 1) + ((B2 >> 2) & 1) - 1;
  constexpr int O3x = (SB & 1) + (B3 & 1) - 1, O3y = ((SB >> 1) & 1) + ((B3 >> 1) & 1) - 1,
                O3z = ((SB >> 2) & 1) + ((B3 >> 2) & 1) - 1;
  const F3 p1 = rel_pos(F, oa, n + O1x * sx + O1y * sy + O1z * sz, O1x, O1y, O1z);
  const F3 p2 = rel_pos(F, oa, n + O2x * sx + O2y * sy + O2z * sz, O2x, O2y, O2z);
  const F3 p3 = rel_pos(F, oa, n + O3x * sx + O3y * sy + O3z * sz, O3x, O3y, O3z);
  f = f + (slo - shi) * crossf(p1 + 2.f * p2 + p3, p3 - p1);
}

template <int SB>
__device__ __forceinline__ void node_cell_faces(const Fields<float> &F, long long n, float4 oa, int i, int j, int k,
                                                const float (&sig)[8], F3 &f) {
  node_face_force<SB, 0>(F, n, oa, i, j, k, sig, f);
  node_face_force<SB, 1>(F, n, oa, i, j, k, sig, f);
  node_face_force<SB, 2>(F, n, oa, i, j, k, sig, f);
}

// Kernel bodies: one thread's work for unit n (node) or c (cell) of the mesh
// F.  The single-mesh kernels and the batched kernels wrap the same bodies,
// so a mesh advanced inside a batch is bitwise equal to the mesh alone.

__device__ __forceinline__ void m_nodes_body(const Fields<float> &F, DevScalars *S, long long n) {
  if (n >= F.nn || !S->next_active) return;
  const float h = S->next_h32;
  int i, j, k;
  node_ijk(n, F.nx, F.ny, i, j, k);
  float sig[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int ci = i - 1 + (s & 1), cj = j - 1 + ((s >> 1) & 1), ck = k - 1 + ((s >> 2) & 1);
    const bool ok = ci >= 0 && cj >= 0 && ck >= 0 && ci < F.nx && cj < F.ny && ck < F.nz;
    sig[s] = ok ? F.sig[cell_index(F.nx, F.ny, ci, cj, ck)] : 0.f;
  }
  F3 f = {0.f, 0.f, 0.f};
  const float4 oa = node_off(F, n);
  node_cell_faces<0>(F, n, oa, i, j, k, sig, f);
  node_cell_faces<1>(F, n, oa, i, j, k, sig, f);
  node_cell_faces<2>(F, n, oa, i, j, k, sig, f);
  node_cell_faces<3>(F, n, oa, i, j, k, sig, f);
  node_cell_faces<4>(F, n, oa, i, j, k, sig, f);
  node_cell_faces<5>(F, n, oa, i, j, k, sig, f);
  node_cell_faces<6>(F, n, oa, i, j, k, sig, f);
  const float hm = h / (24.f * F.mn[n]);
  const float u0 = F.u[n], v0 = F.v[n], w0 = F.w[n];
  float u1 = u0 + hm * f.x, v1 = v0 + hm * f.y, w1 = w0 + hm * f.z;
  wall_bc_f(F, i, j, k, u1, v1, w1);
  F.u[n] = u1;
  F.v[n] = v1;
  F.w[n] = w1;
  F.ub[n] = 0.5f * (u0 + u1);
  F.vb[n] = 0.5f * (v0 + v1);
  F.wb[n] = 0.5f * (w0 + w1);
}

__device__ __forceinline__ void m_cells_body(const Fields<float> &F, DevScalars *S, long long c) {
  if (c >= F.nc || !S->next_active) return;
  const float h = S->next_h32;
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  long long nid[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) nid[a] = node_index(F.nx, F.ny, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
  F3 E[8], ub[8];
  ref_hex(F, nid, E);
#pragma unroll
  for (int a = 0; a < 8; ++a) ub[a] = {F.ub[nid[a]], F.vb[nid[a]], F.wb[nid[a]]};
  const float work = grad_dot_f(E, ub);
  // compatible energy update; the increment is FP32, the accumulation FP64
  const float de = h * F.sig[c] * work / F.m[c];
  F.e[c] = (float)((double)F.e[c] - (double)de);
  F3 Dd[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) Dd[a] = h * ub[a];
  float vx, vy, vz;
  swept_low_faces_f(E, Dd, vx, vy, vz);
  F.dvx[c] = i > 0 ? vx : 0.f;
  F.dvy[c] = j > 0 ? vy : 0.f;
  F.dvz[c] = k > 0 ? vz : 0.f;
}

// Lagrangian volume of a cell by closure: V_E minus its net swept volume.
__device__ __forceinline__ float lag_volume(const Fields<float> &F, long long c, int i, int j, int k) {
  const long long sy = F.nx, sz = (long long)F.nx * F.ny;
  float net = -F.dvx[c] - F.dvy[c] - F.dvz[c];
  if (i + 1 < F.nx) net += F.dvx[c + 1];
  if (j + 1 < F.ny) net += F.dvy[c + sy];
  if (k + 1 < F.nz) net += F.dvz[c + sz];
  return F.VE[c] - net;
}

template <int AX>
__device__ __forceinline__ void m_face_flux(const Fields<float> &F, DevScalars *S, long long c, int i, int j, int k,
                                            float rho_c, float *mu, float *ep) {
  const int idx = AX == 0 ? i : AX == 1 ? j : k;
  const float *dv = AX == 0 ? F.dvx : AX == 1 ? F.dvy : F.dvz;
  if (idx == 0) {
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
    const long long stride = AX == 0 ? 1 : AX == 1 ? (long long)F.nx : (long long)F.nx * F.ny;
    const long long d = c - stride;
    const float VL = lag_volume(F, d, AX == 0 ? i - 1 : i, AX == 1 ? j - 1 : j, AX == 2 ? k - 1 : k);
    rho_d = F.m[d] / VL;
    e_d = F.e[d];
  }
  const float f = rho_d * v;
  mu[c] = f;
  ep[c] = f * e_d;
}

// Lagrangian densities (closure) and donor-cell fluxes of the low faces.
__device__ __forceinline__ void m_fluxes_body(const Fields<float> &F, DevScalars *S, long long c) {
  if (c >= F.nc || !S->next_active) return;
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  const float VL = lag_volume(F, c, i, j, k);
  if (!(VL > 0.f)) set_status(S, VL != VL ? SALE_ENAN : SALE_ENEGVOL);
  const float rho_c = F.m[c] / VL;
  m_face_flux<0>(F, S, c, i, j, k, rho_c, F.mux, F.epx);
  m_face_flux<1>(F, S, c, i, j, k, rho_c, F.muy, F.epy);
  m_face_flux<2>(F, S, c, i, j, k, rho_c, F.muz, F.epz);
}

// ---------------------------------------------------------------------------
// Node remap (FP32)
// ---------------------------------------------------------------------------

template <int AX>
__device__ __forceinline__ float m_edge_psi(const Fields<float> &F, int i, int j, int k) {
  const float *mu = AX == 0 ? F.mux : AX == 1 ? F.muy : F.muz;
  const int n_ax = AX == 0 ? F.nx : AX == 1 ? F.ny : F.nz;
  const long long stride = AX == 0 ? 1 : AX == 1 ? (long long)F.nx : (long long)F.nx * F.ny;
  float psi = 0.f;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    int ci = i, cj = j, ck = k;
    if (AX == 0) { cj = j - 1 + (s & 1); ck = k - 1 + (s >> 1); }
    if (AX == 1) { ci = i - 1 + (s & 1); ck = k - 1 + (s >> 1); }
    if (AX == 2) { ci = i - 1 + (s & 1); cj = j - 1 + (s >> 1); }
    if (ci < 0 || cj < 0 || ck < 0 || ci >= F.nx || cj >= F.ny || ck >= F.nz) continue;
    const long long c = cell_index(F.nx, F.ny, ci, cj, ck);
    const int hi_idx = (AX == 0 ? ci : AX == 1 ? cj : ck) + 1;
    psi += mu[c] + (hi_idx < n_ax ? mu[c + stride] : 0.f);
  }
  return 0.125f * psi;
}

template <int AX, int SIDE>
__device__ __forceinline__ void m_node_edge(const Fields<float> &F, int i, int j, int k, long long n, float &m,
                                            F3 &p, float &ke) {
  const int idx = AX == 0 ? i : AX == 1 ? j : k;
  const int n_ax = AX == 0 ? F.nx : AX == 1 ? F.ny : F.nz;
  if (SIDE == 0 && idx == n_ax) return;
  if (SIDE == 1 && idx == 0) return;
  const float psi = m_edge_psi<AX>(F, (SIDE == 1 && AX == 0) ? i - 1 : i, (SIDE == 1 && AX == 1) ? j - 1 : j,
                                   (SIDE == 1 && AX == 2) ? k - 1 : k);
  const long long stride = AX == 0 ? 1 : AX == 1 ? (long long)(F.nx + 1) : (long long)(F.nx + 1) * (F.ny + 1);
  const long long lo = SIDE == 0 ? n : n - stride;
  const long long dn = psi > 0.f ? lo + stride : lo;
  const F3 ud = {F.u[dn], F.v[dn], F.w[dn]};
  const float flux = SIDE == 0 ? psi : -psi;
  m += flux;
  p = p + flux * ud;
  ke += flux * 0.5f * dotf(ud, ud);
}

__device__ __forceinline__ void m_remap_nodes_body(const Fields<float> &F, DevScalars *S, long long n) {
  if (n >= F.nn) return;
  if (!S->next_active) {  // inactive cycle: velocity carries over unchanged
    F.ub[n] = F.u[n];
    F.vb[n] = F.v[n];
    F.wb[n] = F.w[n];
    return;
  }
  int i, j, k;
  node_ijk(n, F.nx, F.ny, i, j, k);
  const float m0 = F.mn[n];
  const F3 u0 = {F.u[n], F.v[n], F.w[n]};
  float m = m0;
  F3 p = m0 * u0;
  float ke = 0.5f * m0 * dotf(u0, u0);
  m_node_edge<0, 0>(F, i, j, k, n, m, p, ke);
  m_node_edge<0, 1>(F, i, j, k, n, m, p, ke);
  m_node_edge<1, 0>(F, i, j, k, n, m, p, ke);
  m_node_edge<1, 1>(F, i, j, k, n, m, p, ke);
  m_node_edge<2, 0>(F, i, j, k, n, m, p, ke);
  m_node_edge<2, 1>(F, i, j, k, n, m, p, ke);
  if (!(m > 0.f)) set_status(S, m != m ? SALE_ENAN : SALE_ENEGVOL);
  const float inv_m = 1.f / m;
  float u1 = p.x * inv_m, v1 = p.y * inv_m, w1 = p.z * inv_m;
  wall_bc_f(F, i, j, k, u1, v1, w1);
  F.ub[n] = u1;
  F.vb[n] = v1;
  F.wb[n] = w1;
  F.mn[n] = m;
  F.dke[n] = ke - 0.5f * m * (u1 * u1 + v1 * v1 + w1 * w1);
}

// ---------------------------------------------------------------------------
// Cell remap, EoS, viscosity, CFL dt (FP32; dt reduced as a double)
// ---------------------------------------------------------------------------

// EoS and viscosity of a cell on the reference mesh; returns its CFL step.
__device__ __forceinline__ float m_eos_cell(const Fields<float> &F, long long c, int i, int j, int k, float m,
                                            float e, bool store_all) {
  long long nid[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) nid[a] = node_index(F.nx, F.ny, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
  F3 E[8];
  ref_hex(F, nid, E);
  F3 U[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) U[a] = {F.u[nid[a]], F.v[nid[a]], F.w[nid[a]]};
  const float dvdt = grad_dot_f(E, U);
  const float V = F.VE[c];
  const float inv_v = 1.f / V;
  const float div = dvdt * inv_v;
  const float L = F.LE[c];
  const float rho = m * inv_v;
  const float g = F.gamma32;
  const float p = (g - 1.f) * rho * e;
  const float cs = sqrtf(g * (g - 1.f) * fmaxf(e, 0.f));
  float q_rho = 0.f;
  if (div < 0.f) {
    const float ld = L * div;
    q_rho = F.c_q32 * ld * ld + F.c_l32 * cs * L * fabsf(div);
  }
  const float q = rho * q_rho;
  F.rho[c] = rho;
  F.sig[c] = p + q;
  if (store_all) {
    F.p[c] = p;
    F.q[c] = q;
    F.cs[c] = cs;
    F.vol[c] = V;
  }
  return F.cfl32 * L / sqrtf(cs * cs + 2.f * q_rho);
}

// Cell remap + EoS + dt; nblk = blocks of this mesh (last-block detection).
__device__ __forceinline__ void m_remap_eos_body(const Fields<float> &F, DevScalars *S, long long c, unsigned nblk) {
  if (!S->next_active) return;  // uniform over the mesh's blocks: S changes only in its last block
  float dtc = INFINITY;
  if (c < F.nc) {
    int i, j, k;
    cell_ijk(c, F.nx, F.ny, i, j, k);
    const long long sy = F.nx, sz = (long long)F.nx * F.ny;
    float dm = -F.mux[c] - F.muy[c] - F.muz[c];
    float de = -F.epx[c] - F.epy[c] - F.epz[c];
    if (i + 1 < F.nx) { dm += F.mux[c + 1]; de += F.epx[c + 1]; }
    if (j + 1 < F.ny) { dm += F.muy[c + sy]; de += F.epy[c + sy]; }
    if (k + 1 < F.nz) { dm += F.muz[c + sz]; de += F.epz[c + sz]; }
    const float m0 = F.m[c];
    const float m1 = m0 + dm;
    float ie = m0 * F.e[c] + de;
    if (F.ke_fix) {
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int ni = i + (a & 1), nj = j + ((a >> 1) & 1), nk = k + ((a >> 2) & 1);
        const float share = ((ni == 0 || ni == F.nx) ? 1.f : 0.5f) * ((nj == 0 || nj == F.ny) ? 1.f : 0.5f) *
                            ((nk == 0 || nk == F.nz) ? 1.f : 0.5f);
        ie += F.dke[node_index(F.nx, F.ny, ni, nj, nk)] * share;
      }
    }
    if (!(m1 > 0.f)) set_status(S, m1 != m1 ? SALE_ENAN : SALE_ENEGVOL);
    const float e1 = ie / m1;
    F.m[c] = m1;
    F.e[c] = e1;
    const float d = m_eos_cell(F, c, i, j, k, m1, e1, false);
    dtc = d == d ? d : (set_status(S, SALE_ENAN), INFINITY);
  }
  block_min_dt32_and_finalize(F, S, dtc, kDtAdvance, 0.0, nblk);
}

// EoS/viscosity/dt without a remap: kDtInit / kDtPropose, or no dt at all
// (mode < 0: only refresh the derived fields p, q, cs, vol, rho).
__global__ void __launch_bounds__(kBlock, 4) k_m_eos(Fields<float> F, DevScalars *S, int mode) {
  if (mode >= 0 && S->status != 0) return;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  float dtc = INFINITY;
  if (c < F.nc) {
    int i, j, k;
    cell_ijk(c, F.nx, F.ny, i, j, k);
    const float d = m_eos_cell(F, c, i, j, k, F.m[c], F.e[c], true);
    dtc = d == d ? d : (set_status(S, SALE_ENAN), INFINITY);
  }
  if (mode >= 0) block_min_dt32_and_finalize(F, S, dtc, mode, 0.0, gridDim.x);
}

// Single-mesh kernels.
__global__ void __launch_bounds__(kBlock) k_m_nodes(Fields<float> F, DevScalars *S) {
  m_nodes_body(F, S, blockIdx.x * (long long)kBlock + threadIdx.x);
}
__global__ void __launch_bounds__(kBlock) k_m_cells(Fields<float> F, DevScalars *S) {
  m_cells_body(F, S, blockIdx.x * (long long)kBlock + threadIdx.x);
}
__global__ void __launch_bounds__(kBlock) k_m_fluxes(Fields<float> F, DevScalars *S) {
  m_fluxes_body(F, S, blockIdx.x * (long long)kBlock + threadIdx.x);
}
__global__ void __launch_bounds__(kBlock) k_m_remap_nodes(Fields<float> F, DevScalars *S) {
  m_remap_nodes_body(F, S, blockIdx.x * (long long)kBlock + threadIdx.x);
}
__global__ void __launch_bounds__(kBlock, 4) k_m_remap_eos(Fields<float> F, DevScalars *S) {
  m_remap_eos_body(F, S, blockIdx.x * (long long)kBlock + threadIdx.x, gridDim.x);
}

// Batched kernels: one launch covers every mesh of a batch.  Block b works
// on mesh tab[b].x, local block tab[b].y; the mesh's descriptor is staged in
// shared memory once per block.
template <int KID>
__global__ void __launch_bounds__(kBlock, KID == kMixRemapEos ? 4 : 1) kb_m(const BatchItem *items, const int2 *tab) {
  __shared__ BatchItem it;
  const int2 t = tab[blockIdx.x];
  const int *src = reinterpret_cast<const int *>(items + t.x);
  int *dst = reinterpret_cast<int *>(&it);
  for (int w = threadIdx.x; w < (int)(sizeof(BatchItem) / sizeof(int)); w += kBlock) dst[w] = src[w];
  __syncthreads();
  const long long u = (long long)t.y * kBlock + threadIdx.x;
  if constexpr (KID == kMixNodes) m_nodes_body(it.F, it.S, u);
  if constexpr (KID == kMixCells) m_cells_body(it.F, it.S, u);
  if constexpr (KID == kMixFluxes) m_fluxes_body(it.F, it.S, u);
  if constexpr (KID == kMixRemapNodes) m_remap_nodes_body(it.F, it.S, u);
  if constexpr (KID == kMixRemapEos) m_remap_eos_body(it.F, it.S, u, it.nblk_cell);
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

static inline unsigned grid_m(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

void launch_m_batch(int kid, const BatchItem *items, const int2 *tab, unsigned nblocks, cudaStream_t st) {
  switch (kid) {
    case kMixNodes: kb_m<kMixNodes><<<nblocks, kBlock, 0, st>>>(items, tab); break;
    case kMixCells: kb_m<kMixCells><<<nblocks, kBlock, 0, st>>>(items, tab); break;
    case kMixFluxes: kb_m<kMixFluxes><<<nblocks, kBlock, 0, st>>>(items, tab); break;
    case kMixRemapNodes: kb_m<kMixRemapNodes><<<nblocks, kBlock, 0, st>>>(items, tab); break;
    case kMixRemapEos: kb_m<kMixRemapEos><<<nblocks, kBlock, 0, st>>>(items, tab); break;
    default: break;
  }
}

void launch_batch_limits(const BatchItem *items, int n, long long cycles, cudaStream_t st) {
  kb_set_limits<<<(n + 127) / 128, 128, 0, st>>>(items, n, cycles);
}

void launch_batch_gather(const BatchItem *items, int n, BatchStatus *out, cudaStream_t st) {
  kb_gather<<<(n + 127) / 128, 128, 0, st>>>(items, n, out);
}

void launch_m_init_cells(const Fields<float> &F, DevScalars *S, const double *rho0, const double *p0,
                         long long dep_cell, double dep_e, float *VE, float *LE, cudaStream_t st) {
  k_m_init_cells<<<grid_m(F.nc), kBlock, 0, st>>>(F, S, rho0, p0, dep_cell, dep_e, VE, LE);
}

void launch_m_kernel(int kid, const Fields<float> &F, DevScalars *S, int mode, double dt_override, cudaStream_t st) {
  switch (kid) {
    case kMixNodes: k_m_nodes<<<grid_m(F.nn), kBlock, 0, st>>>(F, S); break;
    case kMixCells: k_m_cells<<<grid_m(F.nc), kBlock, 0, st>>>(F, S); break;
    case kMixFluxes: k_m_fluxes<<<grid_m(F.nc), kBlock, 0, st>>>(F, S); break;
    case kMixRemapNodes: k_m_remap_nodes<<<grid_m(F.nn), kBlock, 0, st>>>(F, S); break;
    case kMixRemapEos: k_m_remap_eos<<<grid_m(F.nc), kBlock, 0, st>>>(F, S); break;
    case kMixEos: k_m_eos<<<grid_m(F.nc), kBlock, 0, st>>>(F, S, mode); break;
    default: break;
  }
}

}  // namespace sale
