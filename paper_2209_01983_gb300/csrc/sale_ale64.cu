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
//                    velocity with walls, time-centred velocity ubar, and
//                    0.5 |u|^2 for the node remap
//   k_ale_edges      side quads of the swept hexes, one per mesh edge (each
//                    is shared by three cells' swept hexes), with the origin
//                    shifts those cells need, and each cell's Lagrangian
//                    low-face terms, from the cached reference offsets of
//                    every node to its neighbours (k_geo_init_nodes)
//   k_ale_cells      compatible energy e_L = e - dt/m (p+q) sum_a G(a).ubar_a;
//                    swept volumes of the three low faces between the
//                    Lagrangian face (x_ref + dt ubar) and the reference face
//   k_ale_density    V_L = V_E - (net swept volume): the Lagrangian volume by
//                    closure; rho_L = m / V_L
//   k_ale_fluxes     donor-cell mass and energy fluxes of the low faces, and
//                    each cell's dual-mesh flux parts (mu_low + mu_high) / 8
//   k_ale_remap_nodes  dual-mesh node remap from those parts, marching in k
//   k_ale_remap_eos  new cell mass/energy + kinetic-energy fix, then EoS,
//                    viscosity, p+q and the CFL dt on the reference mesh
//
// Every FP64 operation counts on GB300 (one FP64 FMA per 62 FP32 ones), so
// work shared between cells or nodes is done once and passed through HBM,
// which this path leaves mostly idle.
#include "sale_device.cuh"

namespace sale {

namespace {

// Cached corner gradient component: G[(corner*3 + axis) * nc + c].
__device__ __forceinline__ P3 corner_g(const double *G, long long nc, long long c, int corner) {
  const double *g = G + (long long)corner * 3 * nc + c;
  return {g[0], g[nc], g[2 * nc]};
}

// Half the face term of the fan volume formula for the quad (p0,p1,p2,p3):
// T = (p0+p1+p2+p3) . (d1 x d2), d1 = p2 - p0, d2 = p3 - p1; a hex volume is
// (1/24) times the sum of the terms of its six outward faces (same origin
// for all six).  With p2 + p3 = p0 + p1 + d1 + d2 and (d1 + d2) . (d1 x d2)
// = 0 this is T = 2 (p0 + p1) . (d1 x d2), five FP64 operations fewer.  The
// edge pass stores T / 2 (one FP64 multiply fewer per term) and the cell
// pass scales the sums by 1/12: halving is exact in binary floating point
// and commutes with every rounding, and 1/12 = 2 (1/24) exactly, so the
// swept volumes are bitwise those of the full terms scaled by 1/24.
__device__ __forceinline__ double quad_term(P3 p0, P3 p1, P3 p2, P3 p3) {
  return dot(p0 + p1, cross(p2 - p0, p3 - p1));
}
constexpr double kInvTwelfth = 1.0 / 12.0;

}  // namespace

// Reference geometry of every cell: corner gradients, volume, length scale.
__global__ void __launch_bounds__(kBlock) k_geo_init(Fields<double> F, DevScalars *S, double *G, double *VE,
                                                     double *LE, double *TE, double *iVE, double *iL2) {
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
  const double L = V / sqrt(hex_max_face_area2(X));
  LE[c] = L;
  iVE[c] = 1.0 / V;
  const double cl = F.cfl * L;
  iL2[c] = 1.0 / (cl * cl);
  // reference faces of the swept hexes of the low x/y/z faces, origin node 0
  TE[c] = quad_term(X[0], X[2], X[6], X[4]);
  TE[F.nc + c] = quad_term(X[0], X[4], X[5], X[1]);
  TE[2 * F.nc + c] = quad_term(X[0], X[1], X[3], X[2]);
}

// Reference offsets from every node to the six neighbours the edge pass
// reads (+x, +y, +z, yz, xz, xy): the same subtractions it would otherwise
// repeat every cycle.
__global__ void __launch_bounds__(kBlock) k_geo_init_nodes(Fields<double> F, double *rE) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= F.nn) return;
  int i, j, k;
  node_ijk(n, F.nx, F.ny, i, j, k);
  const long long sx = 1, sy = F.nx + 1, sz = (long long)(F.nx + 1) * (F.ny + 1);
  const bool in[6] = {i < F.nx, j < F.ny, k < F.nz, j < F.ny && k < F.nz, i < F.nx && k < F.nz,
                      i < F.nx && j < F.ny};
  const long long b[6] = {n + sx, n + sy, n + sz, n + sy + sz, n + sx + sz, n + sx + sy};
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    const bool ok = in[s];
    rE[(3ll * s + 0) * F.nn + n] = ok ? F.xr[b[s]] - F.xr[n] : 0.0;
    rE[(3ll * s + 1) * F.nn + n] = ok ? F.yr[b[s]] - F.yr[n] : 0.0;
    rE[(3ll * s + 2) * F.nn + n] = ok ? F.zr[b[s]] - F.zr[n] : 0.0;
  }
}

template <bool STR>
__global__ void __launch_bounds__(kBlock) k_ale_nodes(Fields<double> F, DevScalars *S, double dt_override) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= F.nn || !cycle_active(S)) return;
  const double h = step_dt(S, dt_override);
  int i, j, k;
  node_ijk(n, F.nx, F.ny, i, j, k);
  const double *Gs = F.time_order == 2 ? F.Gh : F.G;  // predictor-corrector: gradients at x^{n+1/2}
  P3 f = {0.0, 0.0, 0.0};
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int ci = i - 1 + (s & 1), cj = j - 1 + ((s >> 1) & 1), ck = k - 1 + ((s >> 2) & 1);
    if (ci < 0 || cj < 0 || ck < 0 || ci >= F.nx || cj >= F.ny || ck >= F.nz) continue;
    const long long c = cell_index(F.nx, F.ny, ci, cj, ck);
    const P3 g = corner_g(Gs, F.nc, c, 7 - s);
    P3 cf = F.sig[c] * g;
    if constexpr (STR) cf = cf - stress_apply(F.sdev, F.nc, c, g);  // the deviatoric part of the cell stress
    if (F.fh) cf = cf + hourglass_corner(F.fh, F.nc, c, 7 - s);
    f = f + cf;
  }
  const double hm = h * F.imn[n];
  const double u0 = F.u[n], v0 = F.v[n], w0 = F.w[n];
  double u1 = u0 + hm * f.x, v1 = v0 + hm * f.y, w1 = w0 + hm * f.z;
  wall_bc(F, i, j, k, u1, v1, w1);
  F.u[n] = u1;
  F.v[n] = v1;
  F.w[n] = w1;
  F.ub[n] = 0.5 * (u0 + u1);
  F.vb[n] = 0.5 * (v0 + v1);
  F.wb[n] = 0.5 * (w0 + w1);
  F.kd[n] = 0.5 * (u1 * u1 + v1 * v1 + w1 * w1);
}

// Side quad (L_a, E_a, E_b, L_b) of the swept hexes along the mesh edge from
// node a = n to b = n + e_AX: half its fan term with node n as origin, and
// the same for origin n - e_Q of each other axis Q (the node 0 of the other
// cells whose low faces hold the edge): T(o) / 2 = T(n) / 2 + 2 (x_n - x_o)
// . A, A the quad's diagonal cross product.  ste[(3 AX + v) nn + n], v = 0 for
// origin n, v = 1, 2 for the other two axes in increasing order.  Eb, Lb:
// reference and Lagrangian position of b relative to x_n.
template <int AX>
__device__ __forceinline__ void edge_side_terms(const Fields<double> &F, long long n, const int (&ijk)[3],
                                                const P3 (&back)[3], P3 La, P3 Eb, P3 Lb) {
  const P3 A = cross(Eb - La, Lb);  // diagonals (E_b - L_a) and (L_b - E_a), E_a = 0
  const double T = dot(La, A);  // (L_a + E_a) . A, half the fan term
  F.ste[(3 * AX) * F.nn + n] = T;
  constexpr int Q1 = AX == 0 ? 1 : 0, Q2 = AX == 2 ? 1 : 2;
  if (ijk[Q1] > 0) F.ste[(3 * AX + 1) * F.nn + n] = T + 2.0 * dot(back[Q1], A);
  if (ijk[Q2] > 0) F.ste[(3 * AX + 2) * F.nn + n] = T + 2.0 * dot(back[Q2], A);
}

// Per node n: the side quads of the three mesh edges leaving it and, when n
// is node 0 of a cell, that cell's three low Lagrangian face terms plus their
// reference-face terms (ste[(9 + axis) nn + n]), all with n as origin.  The
// faces use n's +x, +y, +z neighbours (shared with the edges) and three
// diagonal neighbours.
__global__ void __launch_bounds__(kBlock) k_ale_edges(Fields<double> F, DevScalars *S, double dt_override) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= F.nn || !cycle_active(S)) return;
  const double h = step_dt(S, dt_override);
  int i, j, k;
  node_ijk(n, F.nx, F.ny, i, j, k);
  const int ijk[3] = {i, j, k};
  const long long stride[3] = {1, F.nx + 1, (long long)(F.nx + 1) * (F.ny + 1)};
  const P3 La = h * P3{F.ub[n], F.vb[n], F.wb[n]};
  const long long nn = F.nn;
  auto off = [&](int slot, long long m) {  // cached reference offset of node m to its neighbour in slot
    return P3{F.rE[(3ll * slot) * nn + m], F.rE[(3ll * slot + 1) * nn + m], F.rE[(3ll * slot + 2) * nn + m]};
  };
  auto rel = [&](int slot, long long b, P3 &E) {  // reference and Lagrangian position of node b relative to x_n
    E = off(slot, n);
    return E + h * P3{F.ub[b], F.vb[b], F.wb[b]};
  };
  // x_n minus its -x, -y, -z neighbours: the origin shifts of the side quads
  P3 back[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) back[a] = ijk[a] > 0 ? off(a, n - stride[a]) : P3{0.0, 0.0, 0.0};
  P3 Lb[3], Eb;
  if (i < F.nx) { Lb[0] = rel(0, n + stride[0], Eb); edge_side_terms<0>(F, n, ijk, back, La, Eb, Lb[0]); }
  if (j < F.ny) { Lb[1] = rel(1, n + stride[1], Eb); edge_side_terms<1>(F, n, ijk, back, La, Eb, Lb[1]); }
  if (k < F.nz) { Lb[2] = rel(2, n + stride[2], Eb); edge_side_terms<2>(F, n, ijk, back, La, Eb, Lb[2]); }
  if (i < F.nx && j < F.ny && k < F.nz) {
    const P3 Lyz = rel(3, n + stride[1] + stride[2], Eb), Lxz = rel(4, n + stride[0] + stride[2], Eb),
             Lxy = rel(5, n + stride[0] + stride[1], Eb);
    const long long c = cell_index(F.nx, F.ny, i, j, k);
    F.ste[9 * nn + n] = quad_term(La, Lb[2], Lyz, Lb[1]) + F.TE[c];
    F.ste[10 * nn + n] = quad_term(La, Lb[0], Lxz, Lb[2]) + F.TE[F.nc + c];
    F.ste[11 * nn + n] = quad_term(La, Lb[1], Lxy, Lb[0]) + F.TE[2 * F.nc + c];
  }
}

// MAT: several materials; each takes the share alpha_k (p_k + q) of the
// cell's work (uniform strain: the fractions stay), p_k of the state at n on
// the reference mesh.
template <bool STR, bool MAT>
__global__ void __launch_bounds__(kBlock, STR ? 2 : (MAT ? 3 : 4)) k_ale_cells(Fields<double> F, DevScalars *S,
                                                                            double dt_override) {
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
  const double *Gs = F.time_order == 2 ? F.Gh : F.G;  // predictor-corrector: gradients at x^{n+1/2}
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    ub[a] = {F.ub[nid[a]], F.vb[nid[a]], F.wb[nid[a]]};
    work += dot(corner_g(Gs, F.nc, c, a), ub[a]);
  }
  const double im = F.im[c];
  double e1 = F.e[c] - h * im * F.sig[c] * work;
  double work_hg = 0.0;
  if (F.fh) {
#pragma unroll
    for (int a = 0; a < 8; ++a) work_hg += dot(hourglass_corner(F.fh, F.nc, c, a), ub[a]);
    e1 -= h * im * work_hg;
  }
  if constexpr (STR) {
    // the deviatoric forces' work; the stress at n+1 from the time-centred
    // velocity gradient L = (1/V_E) sum_a ubar_a (x) dV/dx_a (x^n is the
    // reference mesh) and G, Y of the state at n, written to the remap's
    // copy, which the remap + EoS pass transports back into sdev
    const long long nc = F.nc;
    double L[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const P3 g = corner_g(Gs, nc, c, a);
      const double ua[3] = {ub[a].x, ub[a].y, ub[a].z}, ga[3] = {g.x, g.y, g.z};
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int q = 0; q < 3; ++q) L[3 * r + q] += ua[r] * ga[q];
    }
    // sum_a (S dV/dx_a) . ubar_a = S : sum_a ubar_a (x) dV/dx_a, the same sum
    // regrouped (S is symmetric)
    const double sxx = F.sdev[c], syy = F.sdev[nc + c], szz = F.sdev[2 * nc + c];
    const double sxy = F.sdev[3 * nc + c], syz = F.sdev[4 * nc + c], szx = F.sdev[5 * nc + c];
    const double work_s = sxx * L[0] + syy * L[4] + szz * L[8] + sxy * (L[1] + L[3]) + syz * (L[5] + L[7]) +
                          szx * (L[2] + L[6]);
    e1 += h * im * work_s;
    const double iv = F.iVE[c];
#pragma unroll
    for (int q = 0; q < 9; ++q) L[q] *= iv;
    // G and Y of the state at n, from the remap + EoS that ended the last cycle
    const double Gm = F.sdev[7 * nc + c], Ym = F.sdev[8 * nc + c];
    double deps, S6[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) S6[q] = F.sdev[q * nc + c];
    stress_update(S6, L, h, Gm, Ym, deps);
#pragma unroll
    for (int q = 0; q < 6; ++q) F.sold[q * nc + c] = S6[q];
    F.sold[6 * nc + c] = F.sdev[6 * nc + c] + deps;
  }
  if constexpr (MAT) {  // x^n is the reference mesh
    const double qc = F.q[c];
    double ie = 0.0;
    for (int km = 0; km < F.nmat; ++km)
      ie += mat_work_share(F, c, km, F.VE[c], F.iVE[c], qc, h, work, work_hg, F.time_order == 2);
    e1 = ie * im;
  }
  F.e[c] = e1;
  // swept volumes of the three low faces, assembled from k_ale_edges: the
  // Lagrangian face plus reference face terms and the side quads (a side
  // quad traversed the other way round changes sign), all with the cell's
  // reference node 0 as origin
  const long long nn = F.nn, n0 = nid[0], n1 = nid[1], n2 = nid[2], n4 = nid[4];
  const double *ste = F.ste;
  const double cx0 = ste[n0], cxy = ste[nn + n2], cxz = ste[2 * nn + n4];
  const double cy0 = ste[3 * nn + n0], cyx = ste[4 * nn + n1], cyz = ste[5 * nn + n4];
  const double cz0 = ste[6 * nn + n0], czx = ste[7 * nn + n1], czy = ste[8 * nn + n2];
  const double sx = ste[9 * nn + n0] + cz0 - czy - cy0 + cyz;
  const double sy = ste[10 * nn + n0] - cz0 + czx + cx0 - cxz;
  const double sz = ste[11 * nn + n0] + cy0 - cyx - cx0 + cxy;
  F.dvx[c] = i > 0 ? sx * kInvTwelfth : 0.0;  // the terms are halves (see quad_term)
  F.dvy[c] = j > 0 ? sy * kInvTwelfth : 0.0;
  F.dvz[c] = k > 0 ? sz * kInvTwelfth : 0.0;
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
  if (!pos_d(VL)) set_status(S, nan_d(VL) ? SALE_ENAN : SALE_ENEGVOL);  // a NaN with the sign clear: caught by the EoS
  F.vol[c] = VL;
  F.rho[c] = F.m[c] / VL;
  if (F.ivl) F.ivl[c] = 1.0 / VL;  // second-order remap and materials: the face fluxes multiply by it
}

// Limited slopes of the Lagrangian density and the specific energy along
// x, y, z of every cell (second-order remap; zero next to a wall).
__global__ void __launch_bounds__(kBlock) k_ale_slopes(Fields<double> F, DevScalars *S) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc || !cycle_active(S)) return;
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  const int idx[3] = {i, j, k}, n_ax[3] = {F.nx, F.ny, F.nz};
  const long long stride[3] = {1, F.nx, (long long)F.nx * F.ny};
  double *sr[3] = {F.srx, F.sry, F.srz}, *se[3] = {F.sex, F.sey, F.sez};
  const double r0 = F.rho[c], e0 = F.e[c];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double s_r = 0.0, s_e = 0.0;
    if (idx[a] > 0 && idx[a] < n_ax[a] - 1) {
      s_r = vanleer_slope(r0 - F.rho[c - stride[a]], F.rho[c + stride[a]] - r0);
      s_e = vanleer_slope(e0 - F.e[c - stride[a]], F.e[c + stride[a]] - e0);
    }
    sr[a][c] = s_r;
    se[a][c] = s_e;
  }
}

// Mass flux through a face with swept volume v whose donor is dn (the
// face is the donor's low face when hi_donates); with O2 the donor density
// and energy are the slab averages of its limited linear profile.  The
// energy flux is returned in ef.
template <bool O2>
__device__ __forceinline__ double ale_donor_flux(const Fields<double> &F, const double *sr, const double *se,
                                                 long long dn, bool hi_donates, double v, double &ef) {
  double rho_f = F.rho[dn], e_f = F.e[dn];
  if (O2) {
    const double nu = fabs(v) * F.ivl[dn];
    const double side = hi_donates ? -1.0 : 1.0;
    rho_f = slab_average(rho_f, sr[dn], nu, side);
    e_f = slab_average(e_f, se[dn], nu, side);
  }
  const double f = rho_f * v;
  ef = f * e_f;
  return f;
}

// Materials: the donor dn's share of the swept volume v for every material
// -- volume alpha_k v, mass (m_k / V_L) v, energy that mass times e_k --
// stored at o + 9 k nc (+ nc, + 2 nc); returns the total mass flux, ef the
// total energy flux.  1 / V_L comes from the density pass (no division).
__device__ __forceinline__ double ale_mat_flux(const Fields<double> &F, long long dn, double v, double &ef,
                                               double *o) {
  const long long nc = F.nc;
  const double sv = v * F.ivl[dn];
  double mu = 0.0, e = 0.0;
  for (int km = 0; km < F.nmat; ++km) {
    const long long ia = 3ll * km * nc + dn;
    const double mf = F.mat[ia + nc] * sv;
    const double efk = mf * F.mat[ia + 2 * nc];
    double *ok = o + 9ll * km * nc;
    ok[0] = F.mat[ia] * v;
    ok[nc] = mf;
    ok[2 * nc] = efk;
    mu += mf;
    e += efk;
  }
  ef = e;
  return mu;
}

// Donor-cell fluxes of the low face normal to AX; also the cell's part of
// the dual-mesh mass flux along AX, (mu_low + mu_high) / 8, mu_high being
// the low-face flux of the +AX neighbour (0 on the high wall).  The node
// remap sums four such parts per mesh edge instead of eight fluxes.
template <int AX, bool O2>
__device__ __forceinline__ void ale_face_flux(const Fields<double> &F, long long c, int idx, int n_ax,
                                              const double *dv, double *mu, double *ep, double *mq) {
  const long long stride = AX == 0 ? 1 : AX == 1 ? (long long)F.nx : (long long)F.nx * F.ny;
  const double *sr = AX == 0 ? F.srx : AX == 1 ? F.sry : F.srz;
  const double *se = AX == 0 ? F.sex : AX == 1 ? F.sey : F.sez;
  double lo = 0.0;
  if (idx == 0) {
    mu[c] = 0.0;
    ep[c] = 0.0;
  } else {
    const double v = dv[c];
    const bool hd = pos_d(v);
    double ef;
    lo = ale_donor_flux<O2>(F, sr, se, hd ? c : c - stride, hd, v, ef);
    mu[c] = lo;
    ep[c] = ef;
  }
  double hi = 0.0;
  if (idx + 1 < n_ax) {
    const double v = dv[c + stride];
    const bool hd = pos_d(v);
    double ef;
    hi = ale_donor_flux<O2>(F, sr, se, hd ? c + stride : c, hd, v, ef);
  }
  mq[c] = (lo + hi) * 0.125;
}

template <bool O2>
__global__ void __launch_bounds__(kBlock) k_ale_fluxes(Fields<double> F, DevScalars *S) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc || !cycle_active(S)) return;
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  ale_face_flux<0, O2>(F, c, i, F.nx, F.dvx, F.mux, F.epx, F.mqx);
  ale_face_flux<1, O2>(F, c, j, F.ny, F.dvy, F.muy, F.epy, F.mqy);
  ale_face_flux<2, O2>(F, c, k, F.nz, F.dvz, F.muz, F.epz, F.mqz);
}

// Materials: every material's fluxes through the three low faces of each
// cell (mfx), their totals (mu, ep) and the cell's dual-mesh parts (mq),
// one axis at a time.  The high face enters the dual part only through its
// total mass flux, the Lagrangian density of its donor times its swept
// volume.
__global__ void __launch_bounds__(kBlock) k_ale_mat_fluxes(Fields<double> F, DevScalars *S) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc || !cycle_active(S)) return;
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  const long long nc = F.nc;
#pragma unroll 1
  for (int ax = 0; ax < 3; ++ax) {
    const int idx = ax == 0 ? i : ax == 1 ? j : k, n_ax = ax == 0 ? F.nx : ax == 1 ? F.ny : F.nz;
    const long long stride = ax == 0 ? 1 : ax == 1 ? (long long)F.nx : (long long)F.nx * F.ny;
    const double *dv = ax == 0 ? F.dvx : ax == 1 ? F.dvy : F.dvz;
    double *o = F.mfx + 3ll * ax * nc + c;
    double lo = 0.0, ef = 0.0;
    if (idx == 0) {
      for (int km = 0; km < F.nmat; ++km) {
        double *ok = o + 9ll * km * nc;
        ok[0] = ok[nc] = ok[2 * nc] = 0.0;
      }
    } else {
      const double v = dv[c];
      lo = ale_mat_flux(F, pos_d(v) ? c : c - stride, v, ef, o);
    }
    (ax == 0 ? F.mux : ax == 1 ? F.muy : F.muz)[c] = lo;
    (ax == 0 ? F.epx : ax == 1 ? F.epy : F.epz)[c] = ef;
    double hi = 0.0;
    if (idx + 1 < n_ax) {
      const double v = dv[c + stride];
      hi = F.rho[pos_d(v) ? c + stride : c] * v;
    }
    (ax == 0 ? F.mqx : ax == 1 ? F.mqy : F.mqz)[c] = (lo + hi) * 0.125;
  }
}

// Upwind transport of mass, momentum and kinetic energy into node n across
// one of its edges, whose dual flux is psi (positive: towards +AX), on the
// low (SIDE = 0: edge from this node to +AX) or high (SIDE = 1: from the
// -AX neighbour) side of the node.
template <int AX, int SIDE>
__device__ __forceinline__ void ale_edge_apply(const Fields<double> &F, long long n, double psi, double &m, P3 &p,
                                               double &ke) {
  const long long stride = AX == 0 ? 1 : AX == 1 ? (long long)(F.nx + 1) : (long long)(F.nx + 1) * (F.ny + 1);
  const long long lo = SIDE == 0 ? n : n - stride;
  // psi > 0 as an integer test of its bits (positive, not zero): the
  // comparison stays off the FP64 pipe, which this kernel keeps ~90% busy
  const long long dn = __double_as_longlong(psi) > 0ll ? lo + stride : lo;
  const double flux = SIDE == 0 ? psi : -psi;
  m += flux;
  p.x += flux * F.u[dn];
  p.y += flux * F.v[dn];
  p.z += flux * F.w[dn];
  ke += flux * F.kd[dn];
}

// Dual-flux part (mu_low + mu_high) / 8 of cell (ci, cj, ck) along one
// axis; zero outside the mesh.
__device__ __forceinline__ double mq_at(const double *mq, const Fields<double> &F, int ci, int cj, int ck) {
  if (ci < 0 || cj < 0 || ck < 0 || ci >= F.nx || cj >= F.ny || ck >= F.nz) return 0.0;
  return mq[cell_index(F.nx, F.ny, ci, cj, ck)];
}

// Node remap marching in k: a block covers a tile of node columns over
// kAleRemapChunk node planes.  The dual flux of a mesh edge is the sum of
// the dual-flux parts of the (up to) four cells around it; for an x- or
// y-edge two of them lie in the cell plane below the node and two above, and
// the pair above one node is the pair below the next, and the k-edge below a
// node is the k-edge above the node beneath it: a column adds each pair and
// each k-edge flux once.
constexpr int kAleRemapChunk = 16;
constexpr int kAleTx = 32, kAleTy = 8;

__global__ void __launch_bounds__(kAleTx * kAleTy) k_ale_remap_nodes(Fields<double> F, DevScalars *S) {
  const int i = blockIdx.x * kAleTx + threadIdx.x, j = blockIdx.y * kAleTy + threadIdx.y;
  const int k0 = blockIdx.z * kAleRemapChunk, k1 = min(k0 + kAleRemapChunk, F.nz + 1);
  if (i > F.nx || j > F.ny) return;
  const long long sz = (long long)(F.nx + 1) * (F.ny + 1);
  const long long n0 = i + (long long)(F.nx + 1) * j;
  if (!cycle_active(S)) {  // inactive cycle: velocity carries over unchanged
    for (int k = k0; k < k1; ++k) {
      const long long n = n0 + sz * k;
      F.ub[n] = F.u[n];
      F.vb[n] = F.v[n];
      F.wb[n] = F.w[n];
    }
    return;
  }
  // pairs of the x-edges (at ci = i, i - 1) and y-edges (at cj = j, j - 1)
  // in cell plane ck, and the k-edge flux through cell plane ck
  auto pairs = [&](int ck, double (&pr)[4]) {
    pr[0] = mq_at(F.mqx, F, i, j - 1, ck) + mq_at(F.mqx, F, i, j, ck);
    pr[1] = mq_at(F.mqx, F, i - 1, j - 1, ck) + mq_at(F.mqx, F, i - 1, j, ck);
    pr[2] = mq_at(F.mqy, F, i - 1, j, ck) + mq_at(F.mqy, F, i, j, ck);
    pr[3] = mq_at(F.mqy, F, i - 1, j - 1, ck) + mq_at(F.mqy, F, i, j - 1, ck);
  };
  auto kflux = [&](int ck) {
    return mq_at(F.mqz, F, i - 1, j - 1, ck) + mq_at(F.mqz, F, i, j - 1, ck) + mq_at(F.mqz, F, i - 1, j, ck) +
           mq_at(F.mqz, F, i, j, ck);
  };
  double below[4];
  pairs(k0 - 1, below);
  double psi_below = kflux(k0 - 1);
  for (int k = k0; k < k1; ++k) {
    double above[4];
    pairs(k, above);
    const double psi_above = kflux(k);
    const long long n = n0 + sz * k;
    const double m0 = F.mn[n];
    double m = m0;
    P3 p = {m0 * F.u[n], m0 * F.v[n], m0 * F.w[n]};
    double ke = m0 * F.kd[n];
    if (i != F.nx) ale_edge_apply<0, 0>(F, n, below[0] + above[0], m, p, ke);
    if (i != 0) ale_edge_apply<0, 1>(F, n, below[1] + above[1], m, p, ke);
    if (j != F.ny) ale_edge_apply<1, 0>(F, n, below[2] + above[2], m, p, ke);
    if (j != 0) ale_edge_apply<1, 1>(F, n, below[3] + above[3], m, p, ke);
    if (k != F.nz) ale_edge_apply<2, 0>(F, n, psi_above, m, p, ke);
    if (k != 0) ale_edge_apply<2, 1>(F, n, psi_below, m, p, ke);
    if (!(m > 0.0)) set_status(S, m != m ? SALE_ENAN : SALE_ENEGVOL);
    const double inv_m = 1.0 / m;
    double u1 = p.x * inv_m, v1 = p.y * inv_m, w1 = p.z * inv_m;
    wall_bc(F, i, j, k, u1, v1, w1);
    F.ub[n] = u1;
    F.vb[n] = v1;
    F.wb[n] = w1;
    F.mn[n] = m;
    F.imn[n] = inv_m;
    F.dke[n] = ke - 0.5 * m * (u1 * u1 + v1 * v1 + w1 * w1);
#pragma unroll
    for (int q = 0; q < 4; ++q) below[q] = above[q];
    psi_below = psi_above;
  }
}

// EoS and viscosity of cell c on the reference mesh (cached gradient,
// 1/V_E, L_E) from its mass, specific energy and node velocities U; writes
// the derived fields and returns the CFL rate (cs^2 + 2 q / rho) / (cfl L)^2
// = 1 / dt_c^2.
template <bool STR = false, bool MAT = false>
__device__ __forceinline__ double ale_eos_cell(const Fields<double> &F, long long c, const P3 (&U)[8], double m,
                                               double e) {
  const double V = F.VE[c];
  const double inv_v = F.iVE[c];
  double dvdt = 0.0;
#pragma unroll
  for (int a = 0; a < 8; ++a) dvdt += dot(corner_g(F.G, F.nc, c, a), U[a]);
  const double div = dvdt * inv_v;
  const double L = F.LE[c];
  const double rho = m * inv_v;
  double p, cs2;
  if constexpr (MAT) {  // the mixture; its sound speed is not a function of e, so it is stored
    mixture_eos(F, c, V, inv_v, F.im[c], p, cs2);
    F.cs[c] = sqrt(cs2);
  } else {
    p = (F.gamma - 1.0) * rho * e;
    cs2 = F.gamma * (F.gamma - 1.0) * max0_d(e);
  }
  double q_rho = 0.0;  // q / rho
  if (sign_d(div)) {   // div < 0 (-0 gives q = 0 either way); the sound speed itself only where the cell compresses
    const double ld = L * div;
    q_rho = F.c_q * ld * ld + F.c_l * sqrt(cs2) * L * fabs(div);
  }
  const double q = rho * q_rho;
  F.vol[c] = V;
  F.rho[c] = rho;
  F.p[c] = p;
  F.q[c] = q;
  F.sig[c] = p + q;  // cs is not stored: it is a function of e (sale_copy_field derives it)
  double c2 = cs2 + 2.0 * q_rho;
  if constexpr (STR) {  // longitudinal elastic wave: K / rho + 4 G / (3 rho); G, Y kept for the next cell pass
    double Gm, Ym;
    steinberg_gy(F.str, p, rho, e, F.sdev[6 * F.nc + c], Gm, Ym);
    F.sdev[7 * F.nc + c] = Gm;
    F.sdev[8 * F.nc + c] = Ym;
    c2 += 4.0 * Gm / (3.0 * rho);
  }
  return c2 * F.iL2[c];
}

__device__ __forceinline__ void ale_cell_velocities(const Fields<double> &F, int i, int j, int k, P3 (&U)[8]) {
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const long long n = node_index(F.nx, F.ny, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
    U[a] = {F.u[n], F.v[n], F.w[n]};
  }
}

// Projected hourglass shape vectors of every reference cell (Flanagan &
// Belytschko 1981): gamma_alpha(a) = h_alpha(a) - hx_alpha . b_a with
// b_a = G_a / V_E and hx_alpha = sum_b h_alpha(b) x_b.  They depend on the
// reference mesh alone, so the Eulerian cycle reads them instead of
// rebuilding them (about 350 FP64 operations per cell every cycle).  Stored
// scaled by V_E^(1/3): the forces carry V^(2/3) = (V^(1/3))^2 through the
// two products with gamma.
__global__ void __launch_bounds__(kBlock) k_geo_init_hg(Fields<double> F, double *HG) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc) return;
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  P3 X[8];
  load_hex(F.xr, F.yr, F.zr, F.nx, F.ny, i, j, k, X);
  shift0(X);
  const double V = F.VE[c];
  const double iv = 1.0 / V, s = cbrt(V);
#pragma unroll
  for (int al = 0; al < 4; ++al) {
    P3 hx = {0.0, 0.0, 0.0};
#pragma unroll
    for (int b = 0; b < 8; ++b) hx = hx + (double)hg_pattern(al, b) * X[b];
#pragma unroll
    for (int a = 0; a < 8; ++a)
      HG[(8ll * al + a) * F.nc + c] = ((double)hg_pattern(al, a) - iv * dot(hx, corner_g(F.G, F.nc, c, a))) * s;
  }
}

// Hourglass corner forces on the reference mesh from u^n and the state at
// n: q_alpha = sum_a gamma_alpha(a) u_a, f_a = -kappa sum_alpha
// gamma_alpha(a) q_alpha, kappa = c_hg rho cs V^(2/3), with the cached
// scaled shape vectors (k_geo_init_hg).
// MAT: several materials, the mixture's sound speed (stored by the EoS) in kappa.
template <bool MAT>
__global__ void __launch_bounds__(kBlock, 2) k_ale_hourglass(Fields<double> F, DevScalars *S) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc || !cycle_active(S)) return;
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  const double *hg = F.HG + c;
  const long long nc = F.nc;
  P3 q[4];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const long long n = node_index(F.nx, F.ny, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
    const P3 u = {F.u[n], F.v[n], F.w[n]};
#pragma unroll
    for (int al = 0; al < 4; ++al) q[al] = a == 0 ? hg[(8ll * al) * nc] * u : q[al] + hg[(8ll * al + a) * nc] * u;
  }
  const double cs = MAT ? F.cs[c] : sqrt(F.gamma * (F.gamma - 1.0) * fmax(F.e[c], 0.0));
  const double kappa = F.c_hg * F.rho[c] * cs;
#pragma unroll
  for (int al = 0; al < 4; ++al) q[al] = -kappa * q[al];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    P3 f = hg[a * nc] * q[0];
#pragma unroll
    for (int al = 1; al < 4; ++al) f = f + hg[(8ll * al + a) * nc] * q[al];
    F.fh[(3ll * a + 0) * nc + c] = f.x;
    F.fh[(3ll * a + 1) * nc + c] = f.y;
    F.fh[(3ll * a + 2) * nc + c] = f.z;
  }
}

// Predictor-corrector half step on the reference mesh: e^{n+1/2} with the
// cached gradient and u^n, then the EoS and viscosity on x_ref + dt/2 u^n.
// sigma^{n+1/2} replaces sigma; the corner gradients at x^{n+1/2} go to Gh
// for the corrector's node and cell passes.
// MAT: several materials (see mat_predict); their half-step shares of
// sigma are kept for the corrector's cell pass.
template <bool MAT>
__global__ void __launch_bounds__(kBlock, 2) k_ale_predict(Fields<double> F, DevScalars *S, double dt_override) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc || !cycle_active(S)) return;
  const double h = step_dt(S, dt_override);
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  const long long n0 = node_index(F.nx, F.ny, i, j, k);
  const long long sy = F.nx + 1, sz = sy * (F.ny + 1);
  P3 X[8];
  double work = 0.0, work_hg = 0.0;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const long long n = n0 + (a & 1) + ((a >> 1) & 1) * sy + ((a >> 2) & 1) * sz;
    const P3 u = {F.u[n], F.v[n], F.w[n]};
    work += dot(corner_g(F.G, F.nc, c, a), u);
    if (F.fh) work_hg += dot(hourglass_corner(F.fh, F.nc, c, a), u);
    X[a] = {F.xr[n] + 0.5 * h * u.x, F.yr[n] + 0.5 * h * u.y, F.zr[n] + 0.5 * h * u.z};
  }
  const double m = F.m[c];
  const double hm = 0.5 * h * F.im[c];
  double e = F.e[c] - hm * F.sig[c] * work;
  if (F.fh) e -= hm * work_hg;
  // x^{n+1/2} relative to node 0
#pragma unroll
  for (int a = 1; a < 8; ++a) X[a] = X[a] - X[0];
  X[0] = {0.0, 0.0, 0.0};
  P3 R[8];
  double a2max;
  const double V = hex_geometry_rel0(X, R, a2max);
  if (!(V > 0.0)) set_status(S, V != V ? SALE_ENAN : SALE_ENEGVOL);
  double dvdt = 0.0;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const P3 g = kInvSixth24 * R[a];
    F.Gh[(3ll * a + 0) * F.nc + c] = g.x;
    F.Gh[(3ll * a + 1) * F.nc + c] = g.y;
    F.Gh[(3ll * a + 2) * F.nc + c] = g.z;
    const long long n = n0 + (a & 1) + ((a >> 1) & 1) * sy + ((a >> 2) & 1) * sz;
    dvdt += dot(g, P3{F.u[n], F.v[n], F.w[n]});
  }
  const double rho = m / V;
  double p, cs;
  double aph[kMaxMat];
  if constexpr (MAT) {  // x^n is the reference mesh
    double cs2;
    mat_predict(F, c, F.iVE[c], F.q[c], 0.5 * h, work, work_hg, V, 1.0 / V, F.im[c], aph, p, cs2);
    cs = sqrt(cs2);
  } else {
    p = (F.gamma - 1.0) * rho * e;
    cs = sqrt(F.gamma * (F.gamma - 1.0) * fmax(e, 0.0));
  }
  // L div = (V / max_f |A_f / 2|) (dvdt / V) = 2 dvdt / sqrt(max_f |A_f|^2)
  double q = 0.0;
  if (dvdt < 0.0) {
    const double ld = 2.0 * dvdt * rsqrt(a2max);
    q = rho * (F.c_q * ld * ld + F.c_l * cs * fabs(ld));
  }
  F.sig[c] = p + q;
  if constexpr (MAT) mat_store_shares(F, c, aph, q);
}

// Cell remap + EoS of cell c; returns its CFL rate 1 / dt_c^2 (0 outside
// the mesh).
template <bool STR, bool MAT>
__device__ __forceinline__ double ale_remap_eos_cell(const Fields<double> &F, DevScalars *S, long long c) {
  double rate = 0.0;
  if constexpr (MAT) {  // the materials' remap (V_L from the density pass), then the mixture's EoS
    if (c < F.nc) {
      int i, j, k;
      cell_ijk(c, F.nx, F.ny, i, j, k);
      mat_remap_cell(F, S, c, i, j, k);
      P3 U[8];
      ale_cell_velocities(F, i, j, k, U);
      rate = ale_eos_cell<false, true>(F, c, U, F.m[c], F.e[c]);
      if (nan_d(rate)) {
        set_status(S, SALE_ENAN);
        rate = 0.0;
      }
    }
    return rate;
  }
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
    ale_cell_velocities(F, i, j, k, U);
    if (F.ke_fix) {
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        // share 1/(cells at the node) = 2^-(interior axes), built from its bits
        const int ni = i + (a & 1), nj = j + ((a >> 1) & 1), nk = k + ((a >> 2) & 1);
        const int interior = (ni != 0 && ni != F.nx) + (nj != 0 && nj != F.ny) + (nk != 0 && nk != F.nz);
        const double share = __longlong_as_double((long long)(1023 - interior) << 52);
        ie += F.dke[node_index(F.nx, F.ny, ni, nj, nk)] * share;
      }
    }
    // (a NaN mass with the sign bit clear passes here and makes the rate NaN)
    if (!pos_d(m1)) set_status(S, nan_d(m1) ? SALE_ENAN : SALE_ENEGVOL);
    const double r = 1.0 / m1;
    double e = ie * r;
    // The second-order remap's limiter divides only where neighbouring
    // values differ: one residual step (Markstein, IBM J. Res. Dev. 34,
    // 1990) makes e the correctly rounded ie / m1 in nearly every cell, so
    // a quiescent region stays bitwise uniform instead of carrying the
    // product's last-bit noise into the slopes.
    if (F.remap_order == 2) e = fma(r, fma(-m1, e, ie), e);
    F.m[c] = m1;
    F.im[c] = r;
    F.e[c] = e;
    if constexpr (STR) {
      // deviatoric stress and plastic strain per unit mass, carried by each
      // face's mass flux from its donor (mu > 0: the high cell), from the
      // Lagrangian values the cell pass left in sold
      const long long nc = F.nc;
      double ms[7];
#pragma unroll
      for (int q = 0; q < 7; ++q) ms[q] = m0 * F.sold[q * nc + c];
      auto face = [&](double mu, long long lo, long long hi, double sign) {
        const long long dn = mu > 0.0 ? hi : lo;
#pragma unroll
        for (int q = 0; q < 7; ++q) ms[q] += sign * mu * F.sold[q * nc + dn];
      };
      if (i > 0) face(F.mux[c], c - 1, c, -1.0);
      if (i + 1 < F.nx) face(F.mux[c + 1], c, c + 1, 1.0);
      if (j > 0) face(F.muy[c], c - sy, c, -1.0);
      if (j + 1 < F.ny) face(F.muy[c + sy], c, c + sy, 1.0);
      if (k > 0) face(F.muz[c], c - sz, c, -1.0);
      if (k + 1 < F.nz) face(F.muz[c + sz], c, c + sz, 1.0);
#pragma unroll
      for (int q = 0; q < 7; ++q) F.sdev[q * nc + c] = ms[q] * r;
    }
    rate = ale_eos_cell<STR>(F, c, U, m1, e);
    if (nan_d(rate)) {
      set_status(S, SALE_ENAN);
      rate = 0.0;
    }
  }
  return rate;
}

// A thread takes kEosCellsPerThread cells, kBlock apart, so the blocks' dt
// minima (two same-address atomics each) are that many times fewer; the
// largest rate is exact, and dt with it.
constexpr int kEosCellsPerThread = 4;

template <bool STR, bool MAT>
__global__ void __launch_bounds__(kBlock, STR || MAT ? 2 : 3) k_ale_remap_eos(Fields<double> F, DevScalars *S,
                                                                             double dt_override) {
  if (!cycle_active(S)) return;  // uniform over the grid: S changes only in the last block
  const long long c0 = blockIdx.x * (long long)(kBlock * kEosCellsPerThread) + threadIdx.x;
  double rate = 0.0;  // CFL rate 1 / dt_c^2
#pragma unroll 1
  for (int r = 0; r < kEosCellsPerThread; ++r)
    rate = max_nonneg_d(rate, ale_remap_eos_cell<STR, MAT>(F, S, c0 + (long long)r * kBlock));  // rates are >= 0, not NaN
  block_min_dt_and_finalize<double, true>(F, S, rate, kDtAdvance, dt_override);
}

// EoS, viscosity and a proposed dt on the reference mesh without a remap
// (refresh after fields were set from the host).
__global__ void __launch_bounds__(kBlock) k_ale_eos(Fields<double> F, DevScalars *S, int mode) {
  if (S->status != 0) return;  // uniform over the grid
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double rate = 0.0;
  if (c < F.nc) {
    int i, j, k;
    cell_ijk(c, F.nx, F.ny, i, j, k);
    P3 U[8];
    ale_cell_velocities(F, i, j, k, U);
    rate = ale_eos_cell(F, c, U, F.m[c], F.e[c]);
    if (rate != rate) {
      set_status(S, SALE_ENAN);
      rate = 0.0;
    }
  }
  block_min_dt_and_finalize<double, true>(F, S, rate, mode, 0.0);
}

static inline unsigned grid_ale(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

void launch_geo_init_hg(const Fields<double> &F, double *HG, cudaStream_t st) {
  k_geo_init_hg<<<grid_ale(F.nc), kBlock, 0, st>>>(F, HG);
}

void launch_geo_init_nodes(const Fields<double> &F, double *rE, cudaStream_t st) {
  k_geo_init_nodes<<<grid_ale(F.nn), kBlock, 0, st>>>(F, rE);
}

void launch_geo_init(const Fields<double> &F, DevScalars *S, double *G, double *VE, double *LE, double *TE,
                     double *iVE, double *iL2, cudaStream_t st) {
  k_geo_init<<<grid_ale(F.nc), kBlock, 0, st>>>(F, S, G, VE, LE, TE, iVE, iL2);
}

void launch_ale_kernel(int kid, const Fields<double> &F, DevScalars *S, double dt_override, cudaStream_t st) {
  switch (kid) {
    case kAleNodes:
      if (F.sdev) k_ale_nodes<true><<<grid_ale(F.nn), kBlock, 0, st>>>(F, S, dt_override);
      else k_ale_nodes<false><<<grid_ale(F.nn), kBlock, 0, st>>>(F, S, dt_override);
      break;
    case kAleEdges: k_ale_edges<<<grid_ale(F.nn), kBlock, 0, st>>>(F, S, dt_override); break;
    case kAlePredict:
      if (F.mat) k_ale_predict<true><<<grid_ale(F.nc), kBlock, 0, st>>>(F, S, dt_override);
      else k_ale_predict<false><<<grid_ale(F.nc), kBlock, 0, st>>>(F, S, dt_override);
      break;
    case kAleHourglass:
      if (F.mat) k_ale_hourglass<true><<<grid_ale(F.nc), kBlock, 0, st>>>(F, S);
      else k_ale_hourglass<false><<<grid_ale(F.nc), kBlock, 0, st>>>(F, S);
      break;
    case kAleCells:
      if (F.mat) k_ale_cells<false, true><<<grid_ale(F.nc), kBlock, 0, st>>>(F, S, dt_override);
      else if (F.sdev) k_ale_cells<true, false><<<grid_ale(F.nc), kBlock, 0, st>>>(F, S, dt_override);
      else k_ale_cells<false, false><<<grid_ale(F.nc), kBlock, 0, st>>>(F, S, dt_override);
      break;
    case kAleDensity: k_ale_density<<<grid_ale(F.nc), kBlock, 0, st>>>(F, S); break;
    case kAleSlopes: k_ale_slopes<<<grid_ale(F.nc), kBlock, 0, st>>>(F, S); break;
    case kAleFluxes:
      if (F.mat) k_ale_mat_fluxes<<<grid_ale(F.nc), kBlock, 0, st>>>(F, S);
      else if (F.remap_order == 2) k_ale_fluxes<true><<<grid_ale(F.nc), kBlock, 0, st>>>(F, S);
      else k_ale_fluxes<false><<<grid_ale(F.nc), kBlock, 0, st>>>(F, S);
      break;
    case kAleRemapNodes: {
      const dim3 g((unsigned)((F.nx + kAleTx) / kAleTx), (unsigned)((F.ny + kAleTy) / kAleTy),
                   (unsigned)((F.nz + kAleRemapChunk) / kAleRemapChunk));
      k_ale_remap_nodes<<<g, dim3(kAleTx, kAleTy), 0, st>>>(F, S);
      break;
    }
    case kAleEos: k_ale_eos<<<grid_ale(F.nc), kBlock, 0, st>>>(F, S, kDtPropose); break;
    case kAleRemapEos: {
      const unsigned g = grid_ale((F.nc + kEosCellsPerThread - 1) / kEosCellsPerThread);
      if (F.mat) k_ale_remap_eos<false, true><<<g, kBlock, 0, st>>>(F, S, dt_override);
      else if (F.sdev) k_ale_remap_eos<true, false><<<g, kBlock, 0, st>>>(F, S, dt_override);
      else k_ale_remap_eos<false, false><<<g, kBlock, 0, st>>>(F, S, dt_override);
      break;
    }
    default: break;
  }
}

}  // namespace sale
