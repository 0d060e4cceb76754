// sale_kernels.cu -- sm_103a kernels of the SALE hydro cycle (general path:
// positions may be anywhere; geometry is recomputed from the node
// coordinates every time it is needed).
//
// Cycle (ScalSALE Sec. IV: Lagrangian phase, then Eulerian rezoning with
// an advection phase when the run is Eulerian):
//   k_lagrange_nodes  corner forces gathered per node (no atomics), new
//                     velocity (walls reflect), time-centred velocity,
//                     new positions                  ("Update_acceleration")
//   k_lagrange_cells  compatible internal-energy update, new density
//                     ("Calculate_density")
//   k_remap_faces     swept volumes of the three low faces of each cell,
//                     donor-cell mass and energy fluxes
//   k_remap_nodes     dual-mesh mass, momentum and kinetic-energy fluxes,
//                     new node velocity and mass, lost kinetic energy
//   k_remap_cells     new cell mass and energy (plus the kinetic-energy fix)
//   k_eos_dt          EoS, sound speed, viscosity, p+q, CFL dt (warp-shuffle
//                     min, one atomicMin per block on the bits of a positive
//                     double, last block finalises time and dt)
// With several materials (FP64, nmat >= 2) the EoS pass evaluates the
// mixture, the cell pass splits the compatible work among the materials
// (uniform strain) and the face and cell remap passes move each material's
// volume, mass and energy (separate instantiations: the single-material
// kernels are unchanged).
#include <cfloat>
#include <cmath>
#include <type_traits>

#include "sale_device.cuh"

namespace sale {


// ---------------------------------------------------------------------------
// Initialisation
// ---------------------------------------------------------------------------

// m = rho0 V, e = p0 / ((gamma-1) rho0); the deposit cell gets e = E / m.
// Materials: cell (i,j,k) is pure material 1 when i >= mat_i0, else 0, its e
// from that material's stiffened-gas EoS at (rho0, p0).
template <typename R>
__global__ void k_init_cells(Fields<R> F, DevScalars *S, const double *rho0, const double *p0,
                             long long dep_cell, double dep_e, int mat_i0) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc) return;
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  P3 X[8];
  load_hex(F.x, F.y, F.z, F.nx, F.ny, i, j, k, X);
  shift0(X);
  const double V = hex_volume_shifted(X);
  if (!(V > 0.0)) set_status(S, SALE_ENEGVOL);
  const double r0 = rho0[c];
  const double m = r0 * V;
  double e;
  if (F.mat) {
    const int km = i >= mat_i0 ? 1 : 0;
    const double g = F.mgam[km];
    e = (p0[c] + g * F.mpinf[km]) / ((g - 1.0) * r0);
    if (c == dep_cell) e = dep_e / m;
    for (int q = 0; q < F.nmat; ++q) {
      F.mat[(3ll * q + 0) * F.nc + c] = (R)(q == km ? 1.0 : 0.0);
      F.mat[(3ll * q + 1) * F.nc + c] = (R)(q == km ? m : 0.0);
      F.mat[(3ll * q + 2) * F.nc + c] = (R)(q == km ? e : 0.0);
    }
  } else {
    e = p0[c] / ((F.gamma - 1.0) * r0);
    if (c == dep_cell) e = dep_e / m;
  }
  F.m[c] = (R)m;
  F.e[c] = (R)e;
  if (F.im) F.im[c] = (R)(1.0 / m);
}

// Cell totals from the materials (after a host upload of material fields):
// m = sum_k m_k, e = sum_k m_k e_k / m.
template <typename R>
__global__ void k_mat_totals(Fields<R> F) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc) return;
  double m = 0.0, ie = 0.0;
  for (int k = 0; k < F.nmat; ++k) {
    const double mk = (double)F.mat[(3ll * k + 1) * F.nc + c];
    m += mk;
    ie += mk * (double)F.mat[(3ll * k + 2) * F.nc + c];
  }
  F.m[c] = (R)m;
  F.e[c] = (R)(ie / m);
  if (F.im) F.im[c] = (R)(1.0 / m);
}

// Node mass = sum of m_c / 8 over the cells holding the node; u = 0.
template <typename R>
__global__ void k_init_nodes(Fields<R> F) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= F.nn) return;
  int i, j, k;
  node_ijk(n, F.nx, F.ny, i, j, k);
  double mn = 0.0;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int ci = i - 1 + (s & 1), cj = j - 1 + ((s >> 1) & 1), ck = k - 1 + ((s >> 2) & 1);
    if (ci < 0 || cj < 0 || ck < 0 || ci >= F.nx || cj >= F.ny || ck >= F.nz) continue;
    const long long c = cell_index(F.nx, F.ny, ci, cj, ck);
    mn += ((double)F.m[c] + (F.mlo ? (double)F.mlo[c] : 0.0)) / 8.0;
  }
  F.mn[n] = (R)mn;
  if (F.imn) F.imn[n] = (R)(1.0 / mn);
  if (F.mnlo) F.mnlo[n] = (R)(mn - (double)(R)mn);  // float-float node mass of the mixed path
  F.u[n] = F.v[n] = F.w[n] = (R)0;
}

__global__ void k_set_limits(DevScalars *S, double t_end, long long cycle_limit) {
  S->t_end = t_end;
  S->cycle_limit = cycle_limit;
  decide_next(S);
}

__global__ void k_reset_scalars(DevScalars *S) {
  S->t = 0.0;
  S->dt = 0.0;
  S->dt_last = 0.0;
  S->t_end = INFINITY;
  S->cycle = 0;
  S->cycle_limit = 0x7FFFFFFFFFFFFFFFll;
  S->dtmin_bits = kInfBits;
  S->blocks_done = 0;
  S->status = 0;
  decide_next(S);
}

// ---------------------------------------------------------------------------
// EoS, viscosity, CFL dt
// ---------------------------------------------------------------------------

// Corner a's gradient from the current-position cache Gn[(3 a + axis) nc + c].
template <typename R>
__device__ __forceinline__ P3 gn_corner(const R *Gn, long long nc, long long c, int a) {
  const R *g = Gn + 3ll * a * nc + c;
  return {(double)g[0], (double)g[nc], (double)g[2 * nc]};
}

// STR: the state carries material strength (a separate instantiation, so
// the stress module's registers do not weigh on the plain kernels).
template <typename R, bool STR, bool MAT>
__global__ void __launch_bounds__(kBlock, STR ? 1 : 2) k_eos_dt(Fields<R> F, DevScalars *S, int mode,
                                                              double dt_override) {
  const bool active = (mode == kDtAdvance) ? cycle_active(S) : (S->status == 0);
  if (!active) return;  // uniform over the grid: S changes only in the last block
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double rate = 0.0;  // CFL rate (c / (cfl L))^2; 0 without a cell
  if (c < F.nc) {
    int i, j, k;
    cell_ijk(c, F.nx, F.ny, i, j, k);
    P3 X[8], Rs[8];
    load_hex(F.x, F.y, F.z, F.nx, F.ny, i, j, k, X);
    // the geometry once, face by face (volume by Euler's relation), and
    // the corner gradients kept for the next Lagrangian step
#pragma unroll
    for (int a = 1; a < 8; ++a) X[a] = X[a] - X[0];
    X[0] = {0.0, 0.0, 0.0};
    double a2max;
    const double V = hex_geometry_rel0(X, Rs, a2max);
    if (!(V > 0.0)) set_status(S, V != V ? SALE_ENAN : SALE_ENEGVOL);
    double dvdt = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const P3 g = kInvSixth24 * Rs[a];
      if (F.Gn) {
        F.Gn[(3ll * a + 0) * F.nc + c] = (R)g.x;
        F.Gn[(3ll * a + 1) * F.nc + c] = (R)g.y;
        F.Gn[(3ll * a + 2) * F.nc + c] = (R)g.z;
      }
      const long long n = node_index(F.nx, F.ny, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
      dvdt += dot(g, P3{(double)F.u[n], (double)F.v[n], (double)F.w[n]});
    }
    // with L = V / max_f |A_f / 2|: L div = 2 dvdt / sqrt(max_f |A_f|^2) and
    // 1 / L^2 = max_f |A_f|^2 / (4 V^2), so neither L nor a division by V is
    // formed beyond 1 / V
    const double iv = 1.0 / V;
    const double m = (double)F.m[c], e = (double)F.e[c];
    const double rho = m * iv;
    double p, cs2;
    if constexpr (MAT) {
      mixture_eos(F, c, V, iv, (double)F.im[c], p, cs2);
    } else {
      p = (F.gamma - 1.0) * rho * e;
      cs2 = F.gamma * (F.gamma - 1.0) * max0_d(e);
    }
    const double cs = sqrt(cs2);
    double q = 0.0, q_rho = 0.0;
    if (dvdt < 0.0) {  // div < 0 (V > 0)
      const double ld = 2.0 * dvdt * rsqrt(a2max);
      q_rho = F.c_q * ld * ld + F.c_l * cs * fabs(ld);
      q = rho * q_rho;
    }
    F.vol[c] = (R)V;
    F.rho[c] = (R)rho;
    F.p[c] = (R)p;
    F.q[c] = (R)q;
    F.cs[c] = (R)cs;
    F.sig[c] = (R)(p + q);
    double c2 = cs2 + 2.0 * q_rho;
    if constexpr (STR) {  // longitudinal elastic wave: K / rho + 4 G / (3 rho); G, Y kept for the next cell pass
      double Gm, Ym;
      steinberg_gy(F.str, p, rho, e, (double)F.sdev[6 * F.nc + c], Gm, Ym);
      F.sdev[7 * F.nc + c] = (R)Gm;
      F.sdev[8 * F.nc + c] = (R)Ym;
      c2 += 4.0 * Gm / (3.0 * rho);
    }
    rate = c2 * (0.25 * a2max) * (iv * iv) / (F.cfl * F.cfl);
    if (rate != rate) {
      set_status(S, SALE_ENAN);
      rate = 0.0;
    }
  }
  block_min_dt_and_finalize<R, true>(F, S, rate, mode, dt_override);
}

// ---------------------------------------------------------------------------
// Lagrangian step
// ---------------------------------------------------------------------------

// One corner of the hex around a node: accumulate sigma_c dV_c/dx_node,
// the gradient taken at the positions (gx, gy, gz).
template <int S8, typename R>
__device__ __forceinline__ void add_corner_force(const Fields<R> &F, const R *gx, const R *gy, const R *gz, int i,
                                                 int j, int k, bool cached, P3 &f) {
  const int ci = i - 1 + (S8 & 1), cj = j - 1 + ((S8 >> 1) & 1), ck = k - 1 + ((S8 >> 2) & 1);
  if (ci < 0 || cj < 0 || ck < 0 || ci >= F.nx || cj >= F.ny || ck >= F.nz) return;
  const long long c = cell_index(F.nx, F.ny, ci, cj, ck);
  P3 g;
  if (cached) {  // this node is corner 7 - S8 of the cell; its gradient at x^n from the EoS pass
    g = gn_corner(F.Gn, F.nc, c, 7 - S8);
  } else {
    P3 X[8];
    load_hex(gx, gy, gz, F.nx, F.ny, ci, cj, ck, X);
    shift0(X);
    g = hex_corner_grad_shifted<7 - S8>(X);
  }
  const double sig = (double)F.sig[c];
  P3 cf = sig * g;
  if (F.sdev) cf = cf - stress_apply(F.sdev, F.nc, c, g);  // the deviatoric part of the cell stress
  if (F.fh) cf = cf + hourglass_corner(F.fh, F.nc, c, 7 - S8);
  f = f + cf;
}

// Hourglass corner forces of every cell from x^n, u^n and the state at n
// (c_hg > 0), held for the node and cell passes of the step.
template <typename R>
__global__ void __launch_bounds__(kBlock) k_hourglass(Fields<R> F, DevScalars *S) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc || !cycle_active(S)) return;
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  P3 X[8], U[8], G[8];
  load_hex(F.x, F.y, F.z, F.nx, F.ny, i, j, k, X);
  load_hex(F.u, F.v, F.w, F.nx, F.ny, i, j, k, U);
  shift0(X);
  if (F.Gn) {  // the gradients of x^n, kept by the EoS pass
#pragma unroll
    for (int a = 0; a < 8; ++a) G[a] = gn_corner(F.Gn, F.nc, c, a);
  } else {
    hex_grad_shifted(X, G);
  }
  // cs from e (the Eulerian kernels do not store it); with materials the
  // mixture's, stored by the EoS
  const double cs = F.mat ? (double)F.cs[c] : sqrt(F.gamma * (F.gamma - 1.0) * fmax((double)F.e[c], 0.0));
  hourglass_store(X, G, U, (double)F.vol[c], (double)F.rho[c], cs, F.c_hg, F.fh, F.nc, c);
}

// Predictor-corrector (time_order 2) half step: x^{n+1/2} = x^n + dt/2 u^n
// of every node, into the next-position buffer.
template <typename R>
__global__ void __launch_bounds__(kBlock) k_pc_positions(Fields<R> F, DevScalars *S, double dt_override) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= F.nn || !cycle_active(S)) return;
  const double h = step_dt(S, dt_override);
  F.xn[n] = (R)((double)F.x[n] + 0.5 * h * (double)F.u[n]);
  F.yn[n] = (R)((double)F.y[n] + 0.5 * h * (double)F.v[n]);
  F.zn[n] = (R)((double)F.z[n] + 0.5 * h * (double)F.w[n]);
}

// Predictor of every cell: e^{n+1/2} = e^n - dt/(2m) sigma^n sum_a
// dV/dx_a(x^n).u^n_a, then the EoS and viscosity on x^{n+1/2} with u^n;
// sigma^{n+1/2} replaces sigma (read only by this cell's thread).
// MAT: several materials, each with its own half-step energy; their
// half-step shares of sigma are kept for the corrector.
template <typename R, bool MAT>
__global__ void __launch_bounds__(kBlock, 2) k_pc_predict(Fields<R> F, DevScalars *S, double dt_override) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc || !cycle_active(S)) return;
  const double h = step_dt(S, dt_override);
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  P3 X[8], U[8], G[8];
  load_hex(F.u, F.v, F.w, F.nx, F.ny, i, j, k, U);
  if (F.Gn) {  // the gradients of x^n, kept by the EoS pass
#pragma unroll
    for (int a = 0; a < 8; ++a) G[a] = gn_corner(F.Gn, F.nc, c, a);
  } else {
    load_hex(F.x, F.y, F.z, F.nx, F.ny, i, j, k, X);
    shift0(X);
    hex_grad_shifted(X, G);
  }
  double work = 0.0;
#pragma unroll
  for (int a = 0; a < 8; ++a) work += dot(G[a], U[a]);
  const double m = (double)F.m[c];
  double e = (double)F.e[c] - 0.5 * h / m * (double)F.sig[c] * work;
  double work_hg = 0.0;
  if (F.fh) {
#pragma unroll
    for (int a = 0; a < 8; ++a) work_hg += dot(hourglass_corner(F.fh, F.nc, c, a), U[a]);
    e -= 0.5 * h / m * work_hg;
  }
  load_hex(F.xn, F.yn, F.zn, F.nx, F.ny, i, j, k, X);
  shift0(X);
  const double V = hex_volume_shifted(X);
  if (!(V > 0.0)) set_status(S, V != V ? SALE_ENAN : SALE_ENEGVOL);
  hex_grad_shifted(X, G);
  double dvdt = 0.0;
#pragma unroll
  for (int a = 0; a < 8; ++a) dvdt += dot(G[a], U[a]);
  const double rho = m / V;
  double p, cs;
  double aph[kMaxMat];
  if constexpr (MAT) {
    double cs2;
    mat_predict(F, c, 1.0 / (double)F.vol[c], (double)F.q[c], 0.5 * h, work, work_hg, V, 1.0 / V, (double)F.im[c],
                aph, p, cs2);
    cs = sqrt(cs2);
  } else {
    p = (F.gamma - 1.0) * rho * e;
    cs = sqrt(F.gamma * (F.gamma - 1.0) * fmax(e, 0.0));
  }
  const double div = dvdt / V;
  const double L = V / sqrt(hex_max_face_area2(X));
  double q = 0.0;
  if (div < 0.0) {
    const double ld = L * div;
    q = rho * (F.c_q * ld * ld + F.c_l * cs * L * fabs(div));
  }
  F.sig[c] = (R)(p + q);
  if constexpr (MAT) mat_store_shares(F, c, aph, q);
}

// Lagrangian node pass.  Single stage: corner forces of x^n, new positions
// into the next-position buffer.  Predictor-corrector: corner forces of
// x^{n+1/2} (next-position buffer), new positions in place.
template <typename R>
__global__ void __launch_bounds__(kBlock) k_lagrange_nodes(Fields<R> F, DevScalars *S, double dt_override) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= F.nn) return;
  const bool pc = F.time_order == 2;
  if (!cycle_active(S)) {  // inactive cycle: positions carry over unchanged
    if (!pc) {
      F.xn[n] = F.x[n];
      F.yn[n] = F.y[n];
      F.zn[n] = F.z[n];
    }
    return;
  }
  const double h = step_dt(S, dt_override);
  int i, j, k;
  node_ijk(n, F.nx, F.ny, i, j, k);
  const R *gx = pc ? F.xn : F.x, *gy = pc ? F.yn : F.y, *gz = pc ? F.zn : F.z;
  const bool cached = !pc && F.Gn;  // single stage: the gradients of x^n are kept
  P3 f = {0.0, 0.0, 0.0};
  add_corner_force<0>(F, gx, gy, gz, i, j, k, cached, f);
  add_corner_force<1>(F, gx, gy, gz, i, j, k, cached, f);
  add_corner_force<2>(F, gx, gy, gz, i, j, k, cached, f);
  add_corner_force<3>(F, gx, gy, gz, i, j, k, cached, f);
  add_corner_force<4>(F, gx, gy, gz, i, j, k, cached, f);
  add_corner_force<5>(F, gx, gy, gz, i, j, k, cached, f);
  add_corner_force<6>(F, gx, gy, gz, i, j, k, cached, f);
  add_corner_force<7>(F, gx, gy, gz, i, j, k, cached, f);
  const double mn = (double)F.mn[n];
  const double u0 = (double)F.u[n], v0 = (double)F.v[n], w0 = (double)F.w[n];
  double u1 = u0 + h * f.x / mn, v1 = v0 + h * f.y / mn, w1 = w0 + h * f.z / mn;
  wall_bc(F, i, j, k, u1, v1, w1);
  const double ub = 0.5 * (u0 + u1), vb = 0.5 * (v0 + v1), wb = 0.5 * (w0 + w1);
  F.u[n] = (R)u1;
  F.v[n] = (R)v1;
  F.w[n] = (R)w1;
  F.ub[n] = (R)ub;
  F.vb[n] = (R)vb;
  F.wb[n] = (R)wb;
  R *ox = pc ? F.x : F.xn, *oy = pc ? F.y : F.yn, *oz = pc ? F.z : F.zn;
  ox[n] = (R)((double)F.x[n] + h * ub);
  oy[n] = (R)((double)F.y[n] + h * vb);
  oz[n] = (R)((double)F.z[n] + h * wb);
}

// MAT: several materials (the predictor-corrector's corrector: each takes
// its half-step share of sigma from the predictor).
template <typename R, bool STR, bool MAT>
__global__ void __launch_bounds__(kBlock, STR ? 1 : 2) k_lagrange_cells(Fields<R> F, DevScalars *S,
                                                                       double dt_override) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc || !cycle_active(S)) return;
  const double h = step_dt(S, dt_override);
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  const bool pc = F.time_order == 2;  // gradient at x^{n+1/2}, new positions in place
  P3 X[8], UB[8], G[8];
  double work = 0.0, work_hg = 0.0;
  load_hex(F.ub, F.vb, F.wb, F.nx, F.ny, i, j, k, UB);
  if (!pc && F.Gn) {  // the gradients of x^n, kept by the EoS pass
#pragma unroll
    for (int a = 0; a < 8; ++a) G[a] = gn_corner(F.Gn, F.nc, c, a);
  } else {
    if (pc) load_hex(F.xn, F.yn, F.zn, F.nx, F.ny, i, j, k, X);
    else load_hex(F.x, F.y, F.z, F.nx, F.ny, i, j, k, X);
    shift0(X);
    hex_grad_shifted(X, G);
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) work += dot(G[a], UB[a]);
  if (F.fh)
#pragma unroll
    for (int a = 0; a < 8; ++a) work_hg += dot(hourglass_corner(F.fh, F.nc, c, a), UB[a]);
  const double m = (double)F.m[c];
  double e1 = (double)F.e[c] - h / m * (double)F.sig[c] * work;
  if (F.fh) e1 -= h / m * work_hg;
  if constexpr (MAT) {
    const double V0 = (double)F.vol[c], qc = (double)F.q[c];
    double ie = 0.0;
    for (int km = 0; km < F.nmat; ++km) ie += mat_work_share(F, c, km, V0, 1.0 / V0, qc, h, work, work_hg, pc);
    e1 = ie / m;
  }
  if constexpr (STR) {
    // the deviatoric forces' work, then the stress at n+1 from the
    // time-centred velocity gradient L = (1/V^n) sum_a ubar_a (x) dV/dx_a and
    // G, Y of the state at n (single-stage step: X is x^n here)
    double work_s = 0.0, L[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      work_s += dot(stress_apply(F.sdev, F.nc, c, G[a]), UB[a]);
      const double ua[3] = {UB[a].x, UB[a].y, UB[a].z}, ga[3] = {G[a].x, G[a].y, G[a].z};
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int q = 0; q < 3; ++q) L[3 * r + q] += ua[r] * ga[q];
    }
    e1 += h / m * work_s;
    const double Vn = (double)F.vol[c];
#pragma unroll
    for (int q = 0; q < 9; ++q) L[q] /= Vn;
    const long long nc = F.nc;
    // G and Y of the state at n, from the EoS that ended the last cycle
    const double Gm = (double)F.sdev[7 * nc + c], Ym = (double)F.sdev[8 * nc + c];
    double deps, S6[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) S6[q] = (double)F.sdev[q * nc + c];
    stress_update(S6, L, h, Gm, Ym, deps);
#pragma unroll
    for (int q = 0; q < 6; ++q) F.sdev[q * nc + c] = (R)S6[q];
    F.sdev[6 * nc + c] = (R)((double)F.sdev[6 * nc + c] + deps);
  }
  if (pc) load_hex(F.x, F.y, F.z, F.nx, F.ny, i, j, k, X);
  else load_hex(F.xn, F.yn, F.zn, F.nx, F.ny, i, j, k, X);
  shift0(X);
  const double V1 = hex_volume_shifted(X);
  if (!(V1 > 0.0)) set_status(S, V1 != V1 ? SALE_ENAN : SALE_ENEGVOL);
  F.e[c] = (R)e1;
  F.vol[c] = (R)V1;
  F.rho[c] = (R)(m / V1);
}

// The Lagrangian cell pass of the common case -- single-stage step, the
// gradients of x^n kept by the EoS pass, no material strength -- with one
// corner at a time live: the compatible energy update, then the volume and
// density at x^{n+1} (the remap's donor density).
// MAT: several materials; each takes the share alpha_k (p_k + q) of the
// cell's work (uniform strain: the fractions stay), p_k at the state of x^n.
template <typename R, bool MAT>
__global__ void __launch_bounds__(kBlock, 3) k_lagrange_cells_cached(Fields<R> F, DevScalars *S,
                                                                    double dt_override) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc || !cycle_active(S)) return;
  const double h = step_dt(S, dt_override);
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  double work = 0.0, work_hg = 0.0;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const long long n = node_index(F.nx, F.ny, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
    const P3 ub = {(double)F.ub[n], (double)F.vb[n], (double)F.wb[n]};
    work += dot(gn_corner(F.Gn, F.nc, c, a), ub);
    if (F.fh) work_hg += dot(hourglass_corner(F.fh, F.nc, c, a), ub);
  }
  const double m = (double)F.m[c];
  double e1 = (double)F.e[c] - h / m * (double)F.sig[c] * work;
  if (F.fh) e1 -= h / m * work_hg;
  if constexpr (MAT) {
    const double V0 = (double)F.vol[c], qc = (double)F.q[c], iv0 = 1.0 / V0;
    double ie = 0.0;
    for (int km = 0; km < F.nmat; ++km) ie += mat_work_share(F, c, km, V0, iv0, qc, h, work, work_hg, false);
    e1 = ie / m;
  }
  P3 X[8];
  load_hex(F.xn, F.yn, F.zn, F.nx, F.ny, i, j, k, X);
  shift0(X);
  const double V1 = hex_volume_shifted(X);
  if (!(V1 > 0.0)) set_status(S, V1 != V1 ? SALE_ENAN : SALE_ENEGVOL);
  F.e[c] = (R)e1;
  F.vol[c] = (R)V1;
  F.rho[c] = (R)(m / V1);
}

// ---------------------------------------------------------------------------
// Remap (Eulerian rezone to the reference mesh + donor-cell advection)
// ---------------------------------------------------------------------------

// Swept hex of the low face of cell (i,j,k) normal to axis AX: local node
// with bit AX = 0 at the current position, = 1 at the reference position,
// other bits picking the face node.  Positive volume: the reference face
// lies on the high-index side, so the high cell donates.
template <int AX, typename R>
__device__ __forceinline__ double swept_volume(const Fields<R> &F, int i, int j, int k) {
  P3 X[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int b0 = (AX == 0) ? 0 : (a & 1);
    const int b1 = (AX == 1) ? 0 : ((a >> 1) & 1);
    const int b2 = (AX == 2) ? 0 : ((a >> 2) & 1);
    const long long n = node_index(F.nx, F.ny, i + b0, j + b1, k + b2);
    const bool ref = (a >> AX) & 1;
    X[a] = ref ? P3{F.xr[n], F.yr[n], F.zr[n]} : P3{(double)F.x[n], (double)F.y[n], (double)F.z[n]};
  }
  shift0(X);
  return hex_volume_shifted(X);
}

template <int AX, typename R>
__device__ __forceinline__ void face_flux(const Fields<R> &F, long long c, int i, int j, int k, R *mu,
                                          R *ep) {
  const int idx = AX == 0 ? i : AX == 1 ? j : k;
  if (idx == 0) {
    mu[c] = (R)0;
    ep[c] = (R)0;
    return;
  }
  const double dv = swept_volume<AX>(F, i, j, k);
  const long long stride = AX == 0 ? 1 : AX == 1 ? (long long)F.nx : (long long)F.nx * F.ny;
  const bool hi_donates = dv > 0.0;
  const long long dn = hi_donates ? c : c - stride;
  double rho_f = (double)F.rho[dn], e_f = (double)F.e[dn];
  if (F.remap_order == 2) {  // F.rho, F.vol hold the Lagrangian density and volume here
    const int n_ax = AX == 0 ? F.nx : AX == 1 ? F.ny : F.nz;
    const int di = hi_donates ? idx : idx - 1;  // donor index along AX
    double sr = 0.0, se = 0.0;
    if (di > 0 && di < n_ax - 1) {
      sr = vanleer_slope(rho_f - (double)F.rho[dn - stride], (double)F.rho[dn + stride] - rho_f);
      se = vanleer_slope(e_f - (double)F.e[dn - stride], (double)F.e[dn + stride] - e_f);
    }
    const double nu = fabs(dv) / (double)F.vol[dn];
    const double side = hi_donates ? -1.0 : 1.0;
    rho_f = slab_average(rho_f, sr, nu, side);
    e_f = slab_average(e_f, se, nu, side);
  }
  const double f = rho_f * dv;
  mu[c] = (R)f;
  ep[c] = (R)(f * e_f);
}

// Materials: the low face along AX moves each material's share of its
// swept volume dv out of the donor -- volume alpha_k dv, mass (m_k / V_L) dv
// (the partial density of the Lagrangian donor), energy that mass times
// e_k -- into mfx; mu and ep get the totals over the materials.
template <int AX, typename R>
__device__ __forceinline__ void mat_face_flux(const Fields<R> &F, long long c, int i, int j, int k, R *mu,
                                              R *ep) {
  const int idx = AX == 0 ? i : AX == 1 ? j : k;
  const long long nc = F.nc;
  if (idx == 0) {
    mu[c] = (R)0;
    ep[c] = (R)0;
    for (int km = 0; km < F.nmat; ++km) {
      R *o = F.mfx + (9ll * km + 3 * AX) * nc + c;
      o[0] = o[nc] = o[2 * nc] = (R)0;
    }
    return;
  }
  const double dv = swept_volume<AX>(F, i, j, k);
  const long long stride = AX == 0 ? 1 : AX == 1 ? (long long)F.nx : (long long)F.nx * F.ny;
  const long long dn = dv > 0.0 ? c : c - stride;
  const double sv = dv / (double)F.vol[dn];
  double mu_t = 0.0, ef_t = 0.0;
  for (int km = 0; km < F.nmat; ++km) {
    const long long ia = 3ll * km * nc + dn;
    const double vf = (double)F.mat[ia] * dv;
    const double mf = (double)F.mat[ia + nc] * sv;
    const double ef = mf * (double)F.mat[ia + 2 * nc];
    R *o = F.mfx + (9ll * km + 3 * AX) * nc + c;
    o[0] = (R)vf;
    o[nc] = (R)mf;
    o[2 * nc] = (R)ef;
    mu_t += mf;
    ef_t += ef;
  }
  mu[c] = (R)mu_t;
  ep[c] = (R)ef_t;
}

template <typename R, bool MAT>
__global__ void __launch_bounds__(kBlock) k_remap_faces(Fields<R> F, DevScalars *S) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc || !cycle_active(S)) return;
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  if constexpr (MAT) {
    mat_face_flux<0>(F, c, i, j, k, F.mux, F.epx);
    mat_face_flux<1>(F, c, i, j, k, F.muy, F.epy);
    mat_face_flux<2>(F, c, i, j, k, F.muz, F.epz);
    return;
  }
  face_flux<0>(F, c, i, j, k, F.mux, F.epx);
  face_flux<1>(F, c, i, j, k, F.muy, F.epy);
  face_flux<2>(F, c, i, j, k, F.muz, F.epz);
  if (F.sdev)  // the cell remap reads the donors' stress from this copy while it writes the new one
    for (int q = 0; q < 7; ++q) F.sold[q * F.nc + c] = F.sdev[q * F.nc + c];
}

// Dual mass flux along the mesh edge from node (i,j,k) to its +AX
// neighbour: sum over the (up to four) cells around the edge of
// (mu_low_face + mu_high_face) / 8.  Positive: mass moves to the low node.
template <int AX, typename R>
__device__ __forceinline__ double edge_psi(const Fields<R> &F, int i, int j, int k) {
  const R *mu = AX == 0 ? F.mux : AX == 1 ? F.muy : F.muz;
  double psi = 0.0;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    int ci = i, cj = j, ck = k;
    if (AX == 0) { cj = j - 1 + (s & 1); ck = k - 1 + (s >> 1); }
    if (AX == 1) { ci = i - 1 + (s & 1); ck = k - 1 + (s >> 1); }
    if (AX == 2) { ci = i - 1 + (s & 1); cj = j - 1 + (s >> 1); }
    if (ci < 0 || cj < 0 || ck < 0 || ci >= F.nx || cj >= F.ny || ck >= F.nz) continue;
    const long long c = cell_index(F.nx, F.ny, ci, cj, ck);
    const double lo = (double)mu[c];
    const int hi_idx = (AX == 0 ? ci : AX == 1 ? cj : ck) + 1;
    const int n_ax = AX == 0 ? F.nx : AX == 1 ? F.ny : F.nz;
    const long long stride = AX == 0 ? 1 : AX == 1 ? (long long)F.nx : (long long)F.nx * F.ny;
    const double hi = hi_idx < n_ax ? (double)mu[c + stride] : 0.0;
    psi += (lo + hi) * 0.125;
  }
  return psi;
}

// Apply the flux of the edge along AX on the low (SIDE = 0: edge from this
// node to +AX) or high (SIDE = 1: edge from the -AX neighbour) side.
template <int AX, int SIDE, typename R>
__device__ __forceinline__ void node_edge(const Fields<R> &F, int i, int j, int k, long long n, double &m,
                                          P3 &p, double &ke) {
  const int idx = AX == 0 ? i : AX == 1 ? j : k;
  const int n_ax = AX == 0 ? F.nx : AX == 1 ? F.ny : F.nz;
  if (SIDE == 0 && idx == n_ax) return;
  if (SIDE == 1 && idx == 0) return;
  const int li = (SIDE == 1 && AX == 0) ? i - 1 : i;
  const int lj = (SIDE == 1 && AX == 1) ? j - 1 : j;
  const int lk = (SIDE == 1 && AX == 2) ? k - 1 : k;
  const double psi = edge_psi<AX>(F, li, lj, lk);
  const long long stride = AX == 0 ? 1 : AX == 1 ? (long long)(F.nx + 1) : (long long)(F.nx + 1) * (F.ny + 1);
  const long long lo = SIDE == 0 ? n : n - stride;
  const long long dn = psi > 0.0 ? lo + stride : lo;
  const double ud = (double)F.u[dn], vd = (double)F.v[dn], wd = (double)F.w[dn];
  const double kd = 0.5 * (ud * ud + vd * vd + wd * wd);
  const double sgn = SIDE == 0 ? 1.0 : -1.0;
  m += sgn * psi;
  p.x += sgn * psi * ud;
  p.y += sgn * psi * vd;
  p.z += sgn * psi * wd;
  ke += sgn * psi * kd;
}

template <typename R>
__global__ void __launch_bounds__(kBlock) k_remap_nodes(Fields<R> F, DevScalars *S) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= F.nn) return;
  if (!cycle_active(S)) {  // inactive cycle: velocity carries over unchanged
    F.ub[n] = F.u[n];
    F.vb[n] = F.v[n];
    F.wb[n] = F.w[n];
    return;
  }
  int i, j, k;
  node_ijk(n, F.nx, F.ny, i, j, k);
  const double m0 = (double)F.mn[n];
  const double u0 = (double)F.u[n], v0 = (double)F.v[n], w0 = (double)F.w[n];
  double m = m0;
  P3 p = {m0 * u0, m0 * v0, m0 * w0};
  double ke = 0.5 * m0 * (u0 * u0 + v0 * v0 + w0 * w0);
  node_edge<0, 0>(F, i, j, k, n, m, p, ke);
  node_edge<0, 1>(F, i, j, k, n, m, p, ke);
  node_edge<1, 0>(F, i, j, k, n, m, p, ke);
  node_edge<1, 1>(F, i, j, k, n, m, p, ke);
  node_edge<2, 0>(F, i, j, k, n, m, p, ke);
  node_edge<2, 1>(F, i, j, k, n, m, p, ke);
  if (!(m > 0.0)) set_status(S, m != m ? SALE_ENAN : SALE_ENEGVOL);
  const double inv_m = 1.0 / m;
  double u1 = p.x * inv_m, v1 = p.y * inv_m, w1 = p.z * inv_m;
  wall_bc(F, i, j, k, u1, v1, w1);
  F.ub[n] = (R)u1;
  F.vb[n] = (R)v1;
  F.wb[n] = (R)w1;
  F.mn[n] = (R)m;
  if (F.imn) F.imn[n] = (R)inv_m;
  F.dke[n] = (R)(ke - 0.5 * m * (u1 * u1 + v1 * v1 + w1 * w1));
  if (F.remap_sets_x) {
    F.x[n] = (R)F.xr[n];
    F.y[n] = (R)F.yr[n];
    F.z[n] = (R)F.zr[n];
  }
}

template <typename R, bool MAT>
__global__ void __launch_bounds__(kBlock) k_remap_cells(Fields<R> F, DevScalars *S) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= F.nc || !cycle_active(S)) return;
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  if constexpr (MAT) {
    mat_remap_cell(F, S, c, i, j, k);
    return;
  }
  const long long sy = F.nx, sz = (long long)F.nx * F.ny;
  double dm = -(double)F.mux[c] - (double)F.muy[c] - (double)F.muz[c];
  double de = -(double)F.epx[c] - (double)F.epy[c] - (double)F.epz[c];
  if (i + 1 < F.nx) { dm += (double)F.mux[c + 1]; de += (double)F.epx[c + 1]; }
  if (j + 1 < F.ny) { dm += (double)F.muy[c + sy]; de += (double)F.epy[c + sy]; }
  if (k + 1 < F.nz) { dm += (double)F.muz[c + sz]; de += (double)F.epz[c + sz]; }
  const double m0 = (double)F.m[c];
  const double m1 = m0 + dm;
  double ie = m0 * (double)F.e[c] + de;
  if (F.ke_fix) {
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int ni = i + (a & 1), nj = j + ((a >> 1) & 1), nk = k + ((a >> 2) & 1);
      const int cnt = ((ni == 0 || ni == F.nx) ? 1 : 2) * ((nj == 0 || nj == F.ny) ? 1 : 2) *
                      ((nk == 0 || nk == F.nz) ? 1 : 2);
      ie += (double)F.dke[node_index(F.nx, F.ny, ni, nj, nk)] / (double)cnt;
    }
  }
  if (!(m1 > 0.0)) set_status(S, m1 != m1 ? SALE_ENAN : SALE_ENEGVOL);
  F.m[c] = (R)m1;
  F.e[c] = (R)(ie / m1);
  if (F.im) F.im[c] = (R)(1.0 / m1);
  if (F.sdev) {
    // deviatoric stress and plastic strain per unit mass, carried by each
    // face's mass flux from its donor (mu > 0: the high cell), first-order
    // donor cell; low faces take mass from this cell, high faces give it
    const long long nc = F.nc;
    double ms[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) ms[q] = m0 * (double)F.sold[q * nc + c];
    auto face = [&](double mu, long long lo, long long hi, double sign) {
      const long long dn = mu > 0.0 ? hi : lo;
#pragma unroll
      for (int q = 0; q < 7; ++q) ms[q] += sign * mu * (double)F.sold[q * nc + dn];
    };
    if (i > 0) face((double)F.mux[c], c - 1, c, -1.0);
    if (i + 1 < F.nx) face((double)F.mux[c + 1], c, c + 1, 1.0);
    if (j > 0) face((double)F.muy[c], c - sy, c, -1.0);
    if (j + 1 < F.ny) face((double)F.muy[c + sy], c, c + sy, 1.0);
    if (k > 0) face((double)F.muz[c], c - sz, c, -1.0);
    if (k + 1 < F.nz) face((double)F.muz[c + sz], c, c + sz, 1.0);
#pragma unroll
    for (int q = 0; q < 7; ++q) F.sdev[q * nc + c] = (R)(ms[q] / m1);
  }
}

// ---------------------------------------------------------------------------
// Diagnostics: fixed-order FP64 reduction (deterministic)
// ---------------------------------------------------------------------------

constexpr int kDiagBlocks = 512;
constexpr int kDiagQ = 6;  // mass, mom x, mom y, mom z, ie, ke

template <typename R>
__global__ void __launch_bounds__(kBlock) k_diag_partial(Fields<R> F, double *partial) {
  double acc[kDiagQ] = {0, 0, 0, 0, 0, 0};
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < F.nc; c += stride) {
    double m = (double)F.m[c], e = (double)F.e[c];
    if (F.mlo) {  // float-float cell quantities of the mixed path
      m += (double)F.mlo[c];
      e += (double)F.elo[c];
    }
    acc[0] += m;
    acc[4] += m * e;
  }
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < F.nn; n += stride) {
    const double m = (double)F.mn[n], u = (double)F.u[n], v = (double)F.v[n], w = (double)F.w[n];
    acc[1] += m * u;
    acc[2] += m * v;
    acc[3] += m * w;
    acc[5] += 0.5 * m * (u * u + v * v + w * w);
  }
  __shared__ double sm[kDiagQ][kBlock / 32];
#pragma unroll
  for (int q = 0; q < kDiagQ; ++q) {
    const double v = warp_sum(acc[q]);
    if ((threadIdx.x & 31) == 0) sm[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < kDiagQ) {
    double s = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) s += sm[threadIdx.x][w];
    partial[threadIdx.x * kDiagBlocks + blockIdx.x] = s;
  }
}

__global__ void k_diag_final(const double *partial, double *out) {
  __shared__ double sm[kDiagQ][kDiagBlocks / 32];
  for (int q = 0; q < kDiagQ; ++q) {
    double v = partial[q * kDiagBlocks + threadIdx.x];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sm[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < kDiagQ) {
    double s = 0.0;
    for (int w = 0; w < kDiagBlocks / 32; ++w) s += sm[threadIdx.x][w];
    out[threadIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// Host launchers (one per kernel, indexed by KernelId)
// ---------------------------------------------------------------------------

static inline unsigned grid_for(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

void launch_reset(DevScalars *S, cudaStream_t st) { k_reset_scalars<<<1, 1, 0, st>>>(S); }

void launch_set_limits(DevScalars *S, double t_end, long long cycle_limit, cudaStream_t st) {
  k_set_limits<<<1, 1, 0, st>>>(S, t_end, cycle_limit);
}

// r = 1 / a elementwise (the reciprocal masses after a host upload).
__global__ void k_recip(const double *__restrict__ a, double *__restrict__ r, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) r[i] = 1.0 / a[i];
}

void launch_recip(const double *a, double *r, long long n, cudaStream_t st) {
  if (n > 0) k_recip<<<grid_for(n), kBlock, 0, st>>>(a, r, n);
}

template <typename R>
void launch_init_cells(const Fields<R> &F, DevScalars *S, const double *rho0, const double *p0,
                       long long dep_cell, double dep_e, int mat_i0, cudaStream_t st) {
  k_init_cells<R><<<grid_for(F.nc), kBlock, 0, st>>>(F, S, rho0, p0, dep_cell, dep_e, mat_i0);
}

void launch_mat_totals(const Fields<double> &F, cudaStream_t st) {
  k_mat_totals<double><<<grid_for(F.nc), kBlock, 0, st>>>(F);
}

void launch_ale_kernel(int kid, const Fields<double> &F, DevScalars *S, double dt_override, cudaStream_t st);

template <typename R>
void launch_kernel(int kid, const Fields<R> &F, DevScalars *S, int mode, double dt_override, double *partial,
                   double *out, cudaStream_t st) {
  if ((kid >= kAleNodes && kid <= kAleRemapEos) || kid == kAleEdges || kid == kAleRemapNodes || kid == kAleEos ||
      kid == kAleSlopes || kid == kAlePredict || kid == kAleHourglass) {
    if constexpr (std::is_same<R, double>::value) launch_ale_kernel(kid, F, S, dt_override, st);
    return;
  }
  // materials run on FP64 states only (the instantiations for float are never launched)
  constexpr bool kFp64 = std::is_same<R, double>::value;
  const bool mat = kFp64 && F.mat != nullptr;
  switch (kid) {
    case kInitNodes: k_init_nodes<R><<<grid_for(F.nn), kBlock, 0, st>>>(F); break;
    case kEos:
      if (mat) {
        if constexpr (kFp64) k_eos_dt<R, false, true><<<grid_for(F.nc), kBlock, 0, st>>>(F, S, mode, dt_override);
      } else if (F.sdev) k_eos_dt<R, true, false><<<grid_for(F.nc), kBlock, 0, st>>>(F, S, mode, dt_override);
      else k_eos_dt<R, false, false><<<grid_for(F.nc), kBlock, 0, st>>>(F, S, mode, dt_override);
      break;
    case kLagNodes: k_lagrange_nodes<R><<<grid_for(F.nn), kBlock, 0, st>>>(F, S, dt_override); break;
    case kLagCells:
      // materials: a state carries the gradient cache and takes the single-stage step
      if (mat) {
        if constexpr (kFp64) {
          if (F.time_order == 2) k_lagrange_cells<R, false, true><<<grid_for(F.nc), kBlock, 0, st>>>(F, S, dt_override);
          else k_lagrange_cells_cached<R, true><<<grid_for(F.nc), kBlock, 0, st>>>(F, S, dt_override);
        }
      } else if (F.sdev) k_lagrange_cells<R, true, false><<<grid_for(F.nc), kBlock, 0, st>>>(F, S, dt_override);
      else if (F.Gn && F.time_order != 2)
        k_lagrange_cells_cached<R, false><<<grid_for(F.nc), kBlock, 0, st>>>(F, S, dt_override);
      else k_lagrange_cells<R, false, false><<<grid_for(F.nc), kBlock, 0, st>>>(F, S, dt_override);
      break;
    case kPcPositions: k_pc_positions<R><<<grid_for(F.nn), kBlock, 0, st>>>(F, S, dt_override); break;
    case kHourglass: k_hourglass<R><<<grid_for(F.nc), kBlock, 0, st>>>(F, S); break;
    case kPcPredict:
      if (mat) {
        if constexpr (kFp64) k_pc_predict<R, true><<<grid_for(F.nc), kBlock, 0, st>>>(F, S, dt_override);
      } else k_pc_predict<R, false><<<grid_for(F.nc), kBlock, 0, st>>>(F, S, dt_override);
      break;
    case kRemapFaces:
      if (mat) {
        if constexpr (kFp64) k_remap_faces<R, true><<<grid_for(F.nc), kBlock, 0, st>>>(F, S);
      } else k_remap_faces<R, false><<<grid_for(F.nc), kBlock, 0, st>>>(F, S);
      break;
    case kRemapNodes: k_remap_nodes<R><<<grid_for(F.nn), kBlock, 0, st>>>(F, S); break;
    case kRemapCells:
      if (mat) {
        if constexpr (kFp64) k_remap_cells<R, true><<<grid_for(F.nc), kBlock, 0, st>>>(F, S);
      } else k_remap_cells<R, false><<<grid_for(F.nc), kBlock, 0, st>>>(F, S);
      break;
    case kDiag:
      k_diag_partial<R><<<kDiagBlocks, kBlock, 0, st>>>(F, partial);
      k_diag_final<<<1, kDiagBlocks, 0, st>>>(partial, out);
      break;
    default: break;
  }
}

template void launch_init_cells<double>(const Fields<double> &, DevScalars *, const double *, const double *,
                                        long long, double, int, cudaStream_t);
template void launch_kernel<double>(int, const Fields<double> &, DevScalars *, int, double, double *, double *,
                                    cudaStream_t);
template void launch_kernel<float>(int, const Fields<float> &, DevScalars *, int, double, double *, double *,
                                   cudaStream_t);

}  // namespace sale
