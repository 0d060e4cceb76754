// sale_ale64.cu -- FP64 kernels of the Eulerian (ALE, remap every cycle)
// cycle.
//
// When every cycle ends with a rezone to the reference mesh, each cycle
// starts with the nodes on the reference mesh, so the reference geometry --
// dV/dx of every cell corner, the reference volume V_E and the length scale
// L_E -- is the same in every cycle.  It is computed once (k_geo_init) and
// read from HBM instead of being recomputed: on GB300 an FP64 corner
// gradient costs ~600 flops at ~1.2 FP64 TFLOP/s, while reading it costs
// 24 doubles at ~6.8 TB/s.
//
// Cycle (ScalSALE Sec. IV, Eulerian rezoning with an advection phase):
//   k_ale_nodes      F_a = sum_c (p+q)_c G_c(a) gathered per node, new
//                    velocity with walls, time-centred velocity ubar
//   k_ale_cells      compatible energy e_L = e - dt/m (p+q) sum_a G(a).ubar_a;
//                    swept volumes of the three low faces between the
//                    Lagrangian face (x_ref + dt ubar) and the reference face
//   k_ale_density    V_L = V_E - (net swept volume): the Lagrangian volume by
//                    closure; rho_L = m / V_L
//   k_ale_fluxes     donor-cell mass and energy fluxes of the low faces
//   k_remap_nodes    (shared with the general path) dual-mesh node remap
//   k_ale_remap_eos  new cell mass/energy + kinetic-energy fix, then EoS,
//                    viscosity, p+q and the CFL dt on the reference mesh
#include "sale_device.cuh"

namespace sale {

namespace {

// Cached corner gradient component: G[(corner*3 + axis) * nc + c].
__device__ __forceinline__ P3 corner_g(const double *G, long long nc, long long c, int corner) {
  const double *g = G + (long long)corner * 3 * nc + c;
  return {g[0], g[nc], g[2 * nc]};
}

// Face term of the fan volume formula for the quad (p0,p1,p2,p3):
// T = (p0+p1+p2+p3) . ((p2-p0) x (p3-p1)); a hex volume is (1/24) times the
// sum of the terms of its six outward faces (same origin for all six).
__device__ __forceinline__ double quad_term(P3 p0, P3 p1, P3 p2, P3 p3) {
  return dot(p0 + p1 + p2 + p3, cross(p2 - p0, p3 - p1));
}

// Swept volumes of the three low faces of a cell (each the volume of the
// hex between the face at its Lagrangian position L and at its reference
// position E; positive when E lies on the high-index side).  All three hexes
// use the cell's reference node 0 as origin, so the side quad along each of
// the three mesh edges at node 0 is shared by two hexes (with opposite
// orientation) and computed once; the three reference-face terms are time
// invariant and come from the cache (TE).  L[a], E[a]: local node a of the
// cell relative to its reference node 0 (E[0] = 0).
__device__ __forceinline__ void swept_low_faces(const P3 (&L)[8], const P3 (&E)[8], const double (&TE)[3],
                                                double &vx, double &vy, double &vz) {
  const double tz0 = quad_term(L[0], E[0], E[4], L[4]);  // edge 0-4
  const double ty0 = quad_term(L[0], L[2], E[2], E[0]);  // edge 0-2
  const double tx0 = quad_term(L[0], E[0], E[1], L[1]);  // edge 0-1
  const double sx = quad_term(L[0], L[4], L[6], L[2]) + TE[0] + tz0 + quad_term(L[2], L[6], E[6], E[2]) + ty0 +
                    quad_term(L[4], E[4], E[6], L[6]);
  const double sy = -tz0 + quad_term(L[1], E[1], E[5], L[5]) + quad_term(L[0], L[1], L[5], L[4]) + TE[1] + tx0 +
                    quad_term(L[4], L[5], E[5], E[4]);
  const double sz = -ty0 + quad_term(L[1], L[3], E[3], E[1]) - tx0 + quad_term(L[2], E[2], E[3], L[3]) +
                    quad_term(L[0], L[2], L[3], L[1]) + TE[2];
  vx = sx * kInvSixth24;
  vy = sy * kInvSixth24;
  vz = sz * kInvSixth24;
}

}  // namespace

// Reference geometry of every cell: corner gradients, volume, length scale.
__global__ void __launch_bounds__(kBlock) k_geo_init(Fields<double> F, DevScalars *S, double *G, double *VE,
                                                     double *LE, double *TE) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc) return;
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  P3 X[8], g[8];
  load_hex(F.xr, F.yr, F.zr, F.nx, F.ny, i, j, k, X);
  shift0(X);
  const double V = hex_volume_shifted(X);
  if (!(V > 0.0)) set_status(S, SALE_ENEGVOL);
  hex_grad_shifted(X, g);
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    G[(3ll * a + 0) * F.nc + c] = g[a].x;
    G[(3ll * a + 1) * F.nc + c] = g[a].y;
    G[(3ll * a + 2) * F.nc + c] = g[a].z;
  }
  VE[c] = V;
  LE[c] = V / sqrt(hex_max_face_area2(X));
  // reference faces of the swept hexes of the low x/y/z faces, origin node 0
  TE[c] = quad_term(X[0], X[2], X[6], X[4]);
  TE[F.nc + c] = quad_term(X[0], X[4], X[5], X[1]);
  TE[2 * F.nc + c] = quad_term(X[0], X[1], X[3], X[2]);
}

__global__ void __launch_bounds__(kBlock) k_ale_nodes(Fields<double> F, DevScalars *S, double dt_override) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= F.nn || !cycle_active(S)) return;
  const double h = step_dt(S, dt_override);
  int i, j, k;
  node_ijk(n, F.nx, F.ny, i, j, k);
  P3 f = {0.0, 0.0, 0.0};
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int ci = i - 1 + (s & 1), cj = j - 1 + ((s >> 1) & 1), ck = k - 1 + ((s >> 2) & 1);
    if (ci < 0 || cj < 0 || ck < 0 || ci >= F.nx || cj >= F.ny || ck >= F.nz) continue;
    const long long c = cell_index(F.nx, F.ny, ci, cj, ck);
    f = f + F.sig[c] * corner_g(F.G, F.nc, c, 7 - s);
  }
  const double hm = h / F.mn[n];
  const double u0 = F.u[n], v0 = F.v[n], w0 = F.w[n];
  double u1 = u0 + hm * f.x, v1 = v0 + hm * f.y, w1 = w0 + hm * f.z;
  wall_bc(F, i, j, k, u1, v1, w1);
  F.u[n] = u1;
  F.v[n] = v1;
  F.w[n] = w1;
  F.ub[n] = 0.5 * (u0 + u1);
  F.vb[n] = 0.5 * (v0 + v1);
  F.wb[n] = 0.5 * (w0 + w1);
}

__global__ void __launch_bounds__(kBlock) k_ale_cells(Fields<double> F, DevScalars *S, double dt_override) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc || !cycle_active(S)) return;
  const double h = step_dt(S, dt_override);
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  long long nid[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) nid[a] = node_index(F.nx, F.ny, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
  // compatible energy update with the cached reference gradient
  P3 ub[8];
  double work = 0.0;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    ub[a] = {F.ub[nid[a]], F.vb[nid[a]], F.wb[nid[a]]};
    work += dot(corner_g(F.G, F.nc, c, a), ub[a]);
  }
  const double m = F.m[c];
  F.e[c] = F.e[c] - h / m * F.sig[c] * work;
  // swept volumes of the three low faces (nodes relative to reference node 0)
  P3 Er[8], Lr[8];
  const P3 o = {F.xr[nid[0]], F.yr[nid[0]], F.zr[nid[0]]};
  Er[0] = {0.0, 0.0, 0.0};
  Lr[0] = h * ub[0];
#pragma unroll
  for (int a = 1; a < 7; ++a) {
    Er[a] = P3{F.xr[nid[a]], F.yr[nid[a]], F.zr[nid[a]]} - o;
    Lr[a] = Er[a] + h * ub[a];
  }
  Er[7] = Lr[7] = {0.0, 0.0, 0.0};  // node 7 is on no low face
  const double TE[3] = {F.TE[c], F.TE[F.nc + c], F.TE[2 * F.nc + c]};
  double vx, vy, vz;
  swept_low_faces(Lr, Er, TE, vx, vy, vz);
  F.dvx[c] = i > 0 ? vx : 0.0;
  F.dvy[c] = j > 0 ? vy : 0.0;
  F.dvz[c] = k > 0 ? vz : 0.0;
}

__global__ void __launch_bounds__(kBlock) k_ale_density(Fields<double> F, DevScalars *S) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc || !cycle_active(S)) return;
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  const long long sy = F.nx, sz = (long long)F.nx * F.ny;
  // V_ref = V_lag + sum over axes of (swept high face - swept low face)
  double net = -F.dvx[c] - F.dvy[c] - F.dvz[c];
  if (i + 1 < F.nx) net += F.dvx[c + 1];
  if (j + 1 < F.ny) net += F.dvy[c + sy];
  if (k + 1 < F.nz) net += F.dvz[c + sz];
  const double VL = F.VE[c] - net;
  if (!(VL > 0.0)) set_status(S, VL != VL ? SALE_ENAN : SALE_ENEGVOL);
  F.vol[c] = VL;
  F.rho[c] = F.m[c] / VL;
}

template <int AX>
__device__ __forceinline__ void ale_face_flux(const Fields<double> &F, long long c, int idx, const double *dv,
                                              double *mu, double *ep) {
  if (idx == 0) {
    mu[c] = 0.0;
    ep[c] = 0.0;
    return;
  }
  const double v = dv[c];
  const long long stride = AX == 0 ? 1 : AX == 1 ? (long long)F.nx : (long long)F.nx * F.ny;
  const long long dn = v > 0.0 ? c : c - stride;
  const double f = F.rho[dn] * v;
  mu[c] = f;
  ep[c] = f * F.e[dn];
}

__global__ void __launch_bounds__(kBlock) k_ale_fluxes(Fields<double> F, DevScalars *S) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc || !cycle_active(S)) return;
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  ale_face_flux<0>(F, c, i, F.dvx, F.mux, F.epx);
  ale_face_flux<1>(F, c, j, F.dvy, F.muy, F.epy);
  ale_face_flux<2>(F, c, k, F.dvz, F.muz, F.epz);
}

__global__ void __launch_bounds__(kBlock) k_ale_remap_eos(Fields<double> F, DevScalars *S, double dt_override) {
  if (!cycle_active(S)) return;  // uniform over the grid: S changes only in the last block
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double dtc = INFINITY;
  if (c < F.nc) {
    int i, j, k;
    cell_ijk(c, F.nx, F.ny, i, j, k);
    const long long sy = F.nx, sz = (long long)F.nx * F.ny;
    double dm = -F.mux[c] - F.muy[c] - F.muz[c];
    double de = -F.epx[c] - F.epy[c] - F.epz[c];
    if (i + 1 < F.nx) { dm += F.mux[c + 1]; de += F.epx[c + 1]; }
    if (j + 1 < F.ny) { dm += F.muy[c + sy]; de += F.epy[c + sy]; }
    if (k + 1 < F.nz) { dm += F.muz[c + sz]; de += F.epz[c + sz]; }
    const double m0 = F.m[c];
    const double m1 = m0 + dm;
    double ie = m0 * F.e[c] + de;
    P3 U[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int ni = i + (a & 1), nj = j + ((a >> 1) & 1), nk = k + ((a >> 2) & 1);
      const long long n = node_index(F.nx, F.ny, ni, nj, nk);
      U[a] = {F.u[n], F.v[n], F.w[n]};
      if (F.ke_fix) {  // share 1/(cells at the node): a power of two, exact
        const double share = ((ni == 0 || ni == F.nx) ? 1.0 : 0.5) * ((nj == 0 || nj == F.ny) ? 1.0 : 0.5) *
                             ((nk == 0 || nk == F.nz) ? 1.0 : 0.5);
        ie += F.dke[n] * share;
      }
    }
    if (!(m1 > 0.0)) set_status(S, m1 != m1 ? SALE_ENAN : SALE_ENEGVOL);
    const double e = ie / m1;
    // EoS and viscosity on the reference mesh
    const double V = F.VE[c];
    const double inv_v = 1.0 / V;
    double dvdt = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) dvdt += dot(corner_g(F.G, F.nc, c, a), U[a]);
    const double div = dvdt * inv_v;
    const double L = F.LE[c];
    const double rho = m1 * inv_v;
    const double p = (F.gamma - 1.0) * rho * e;
    const double cs = sqrt(F.gamma * (F.gamma - 1.0) * fmax(e, 0.0));
    double q_rho = 0.0;  // q / rho
    if (div < 0.0) {
      const double ld = L * div;
      q_rho = F.c_q * ld * ld + F.c_l * cs * L * fabs(div);
    }
    const double q = rho * q_rho;
    F.m[c] = m1;
    F.e[c] = e;
    F.vol[c] = V;
    F.rho[c] = rho;
    F.p[c] = p;
    F.q[c] = q;
    F.cs[c] = cs;
    F.sig[c] = p + q;
    dtc = F.cfl * L / sqrt(cs * cs + 2.0 * q_rho);
    if (dtc != dtc) {
      set_status(S, SALE_ENAN);
      dtc = INFINITY;
    }
  }
  block_min_dt_and_finalize(F, S, dtc, kDtAdvance, dt_override);
}

static inline unsigned grid_ale(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

void launch_geo_init(const Fields<double> &F, DevScalars *S, double *G, double *VE, double *LE, double *TE,
                     cudaStream_t st) {
  k_geo_init<<<grid_ale(F.nc), kBlock, 0, st>>>(F, S, G, VE, LE, TE);
}

void launch_ale_kernel(int kid, const Fields<double> &F, DevScalars *S, double dt_override, cudaStream_t st) {
  switch (kid) {
    case kAleNodes: k_ale_nodes<<<grid_ale(F.nn), kBlock, 0, st>>>(F, S, dt_override); break;
    case kAleCells: k_ale_cells<<<grid_ale(F.nc), kBlock, 0, st>>>(F, S, dt_override); break;
    case kAleDensity: k_ale_density<<<grid_ale(F.nc), kBlock, 0, st>>>(F, S); break;
    case kAleFluxes: k_ale_fluxes<<<grid_ale(F.nc), kBlock, 0, st>>>(F, S); break;
    case kAleRemapEos: k_ale_remap_eos<<<grid_ale(F.nc), kBlock, 0, st>>>(F, S, dt_override); break;
    default: break;
  }
}

}  // namespace sale
