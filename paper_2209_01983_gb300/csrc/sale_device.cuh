// sale_device.cuh -- device helpers shared by the kernel translation units
// of the GB300 SALE library: index maps, hex gathers, wall conditions, warp
// reductions and the end-of-step dt reduction.
#pragma once

#include <cmath>

#include "sale_internal.cuh"

namespace sale {

constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;

// Sign, clamp, maximum and NaN tests of doubles as integer operations on
// their bits.  The FP64 kernels keep GB300's FP64 pipe about 90% busy, and
// each comparison, min/max or NaN test there takes a slot of that pipe;
// these take integer slots instead and give the same result for every
// non-NaN value (NaNs are still caught: see each use).
__device__ __forceinline__ bool pos_d(double x) { return __double_as_longlong(x) > 0ll; }     // x > 0
__device__ __forceinline__ bool sign_d(double x) { return __double_as_longlong(x) < 0ll; }    // sign bit set
__device__ __forceinline__ double max0_d(double x) { return sign_d(x) ? 0.0 : x; }           // max(x, 0)
__device__ __forceinline__ bool nan_d(double x) {
  return (unsigned long long)(__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll) > kInfBits;
}
// max(a, b) of two non-negative doubles: their bits order like the values.
__device__ __forceinline__ double max_nonneg_d(double a, double b) {
  return __double_as_longlong(a) >= __double_as_longlong(b) ? a : b;
}

template <typename R>
__device__ __forceinline__ void load_hex(const R *px, const R *py, const R *pz, int nx, int ny, int i,
                                         int j, int k, P3 (&X)[8]) {
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const long long n = node_index(nx, ny, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
    X[a] = {(double)px[n], (double)py[n], (double)pz[n]};
  }
}

__device__ __forceinline__ void cell_ijk(long long c, int nx, int ny, int &i, int &j, int &k) {
  const long long nxy = (long long)nx * ny;
  k = (int)(c / nxy);
  const long long r = c - (long long)k * nxy;
  j = (int)(r / nx);
  i = (int)(r - (long long)j * nx);
}

__device__ __forceinline__ void node_ijk(long long n, int nx, int ny, int &i, int &j, int &k) {
  const long long sx = nx + 1, sxy = sx * (ny + 1);
  k = (int)(n / sxy);
  const long long r = n - (long long)k * sxy;
  j = (int)(r / sx);
  i = (int)(r - (long long)j * sx);
}

template <typename R>
__device__ __forceinline__ void wall_bc(const Fields<R> &F, int i, int j, int k, double &u, double &v,
                                        double &w) {
  if ((i == 0 && F.reflect[0]) || (i == F.nx && F.reflect[1])) u = 0.0;
  if ((j == 0 && F.reflect[2]) || (j == F.ny && F.reflect[3])) v = 0.0;
  if ((k == 0 && F.reflect[4]) || (k == F.nz && F.reflect[5])) w = 0.0;
}

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Second-order cell remap (van Leer 1977): the limited slope of a cell
// quantity along one axis is the harmonic mean of its two one-sided
// differences when they agree in sign, else 0; a face carries the average
// of the donor's linear profile over the slab of relative thickness nu it
// sweeps, side = +1 at the donor's high face, -1 at its low face.
__host__ __device__ __forceinline__ double vanleer_slope(double dm, double dp) {
  return dm * dp > 0.0 ? 2.0 * dm * dp / (dm + dp) : 0.0;
}
__host__ __device__ __forceinline__ double slab_average(double q, double slope, double nu, double side) {
  return q + side * 0.5 * slope * (1.0 - fmin(nu, 1.0));
}
__device__ __forceinline__ float vanleer_slope_f(float dm, float dp) {
  return dm * dp > 0.f ? 2.f * dm * dp / (dm + dp) : 0.f;
}
__device__ __forceinline__ float slab_average_f(float q, float slope, float nu, float side) {
  return q + side * 0.5f * slope * (1.f - fminf(nu, 1.f));
}

// Face F's contributions to the corner sums R_a = 24 dV/dx_a of a hex given
// relative to its node 0 (X[0] = 0), and to max_f |A_f|^2 with the face
// vector A_f = d02 x d13 (twice the face's vector area).  A corner's fan
// term, (p_next + 2 p_opposite + p_prev) x (p_prev - p_next) over the
// face's cycle q0..q3, shares the face's diagonals d02 = q2 - q0 and
// d13 = q3 - q1 with its neighbours, and opposite corners' terms add up to
// 2 A_f: t0 = (q1 + q3 + 2 q2) x d13, t1 = d02 x (q0 + q2 + 2 q3),
// t2 = 2 A_f - t0, t3 = 2 A_f - t1.  The faces through node 0 start at it
// (q0 = 0).  Every corner's x face (F = 0 or 1) comes first and sets its sum.
template <int F>
__device__ __forceinline__ void face_fan(const P3 (&X)[8], P3 (&R)[8], double &a2max) {
  constexpr int n0 = face_node(F, 0), n1 = face_node(F, 1), n2 = face_node(F, 2), n3 = face_node(F, 3);
  const P3 q1 = X[n1], q2 = X[n2], q3 = X[n3];
  const P3 d02 = n0 == 0 ? q2 : q2 - X[n0];
  const P3 s02 = n0 == 0 ? q2 : X[n0] + q2;
  const P3 d13 = q3 - q1;
  const P3 A = cross(d02, d13);
  const double aa = dot(A, A);
  a2max = F == 0 ? aa : max_nonneg_d(a2max, aa);
  const P3 t0 = cross((q1 + q3) + 2.0 * q2, d13);
  const P3 t1 = cross(d02, s02 + 2.0 * q3);
  const P3 A2 = 2.0 * A;
  const P3 t2 = A2 - t0, t3 = A2 - t1;
  if constexpr (F < 2) {
    R[n0] = t0;
    R[n1] = t1;
    R[n2] = t2;
    R[n3] = t3;
  } else {
    R[n0] = R[n0] + t0;
    R[n1] = R[n1] + t1;
    R[n2] = R[n2] + t2;
    R[n3] = R[n3] + t3;
  }
}

// The geometry of a hex given relative to its node 0 (X[0] = 0), face by
// face: the corner sums R_a = 24 dV/dx_a, max_f |A_f|^2 (A_f twice the
// face's vector area) and the volume by Euler's relation for the cubic V,
// 3 V = sum_a x_a . dV/dx_a = sum_a x_a . R_a / 24 (x_0 = 0).
__device__ __forceinline__ double hex_geometry_rel0(const P3 (&X)[8], P3 (&R)[8], double &a2max) {
  face_fan<0>(X, R, a2max);
  face_fan<1>(X, R, a2max);
  face_fan<2>(X, R, a2max);
  face_fan<3>(X, R, a2max);
  face_fan<4>(X, R, a2max);
  face_fan<5>(X, R, a2max);
  double v72 = dot(X[1], R[1]);
#pragma unroll
  for (int a = 2; a < 8; ++a) v72 += dot(X[a], R[a]);
  return v72 * (1.0 / 72.0);
}

// Corner A's gradient of a shifted hex, stored to G[(3A + axis) nc + c]
// and dotted with U[A] into dvdt (one corner at a time keeps the full
// 24-value gradient out of registers).
template <int A, typename R>
__device__ __forceinline__ void corner_grad_store(const P3 (&X)[8], const P3 (&U)[8], R *G, long long nc,
                                                  long long c, double &dvdt) {
  const P3 g = hex_corner_grad_shifted<A>(X);
  dvdt += dot(g, U[A]);
  G[(3ll * A + 0) * nc + c] = (R)g.x;
  G[(3ll * A + 1) * nc + c] = (R)g.y;
  G[(3ll * A + 2) * nc + c] = (R)g.z;
}

template <typename R>
__device__ __forceinline__ double grad_store_dot(const P3 (&X)[8], const P3 (&U)[8], R *G, long long nc, long long c) {
  double dvdt = 0.0;
  corner_grad_store<0>(X, U, G, nc, c, dvdt);
  corner_grad_store<1>(X, U, G, nc, c, dvdt);
  corner_grad_store<2>(X, U, G, nc, c, dvdt);
  corner_grad_store<3>(X, U, G, nc, c, dvdt);
  corner_grad_store<4>(X, U, G, nc, c, dvdt);
  corner_grad_store<5>(X, U, G, nc, c, dvdt);
  corner_grad_store<6>(X, U, G, nc, c, dvdt);
  corner_grad_store<7>(X, U, G, nc, c, dvdt);
  return dvdt;
}

// Viscous hourglass corner forces of a cell (Flanagan-Belytschko): X its
// nodes relative to node 0, G = dV/dx of its corners, U its node
// velocities; with b = G / V, gamma_alpha(a) = h_alpha(a) - hx_alpha . b_a
// (hx_alpha = sum_b h_alpha(b) x_b), q_alpha = sum_a gamma_alpha(a) u_a,
// f_a = -kappa sum_alpha gamma_alpha(a) q_alpha, kappa = c_hg rho cs V^(2/3).
// Evaluated through M_i = sum_b b_b,i u_b and W_i = sum_alpha hx_alpha,i
// q_alpha / V, so gamma is never formed; stored to fh[(3a + axis) nc + c].
template <typename R>
__device__ __forceinline__ void hourglass_store(const P3 (&X)[8], const P3 (&G)[8], const P3 (&U)[8], double V,
                                                double rho, double cs, double c_hg, R *fh, long long nc,
                                                long long c) {
  const double iv = 1.0 / V;
  P3 hx[4], hu[4];
#pragma unroll
  for (int al = 0; al < 4; ++al) {
    hx[al] = {0.0, 0.0, 0.0};
    hu[al] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const double sg = hg_pattern(al, b);
      hx[al] = hx[al] + sg * X[b];
      hu[al] = hu[al] + sg * U[b];
    }
  }
  P3 M[3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    M[0] = M[0] + G[b].x * U[b];
    M[1] = M[1] + G[b].y * U[b];
    M[2] = M[2] + G[b].z * U[b];
  }
  P3 W[3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
  P3 q[4];
#pragma unroll
  for (int al = 0; al < 4; ++al) {
    q[al] = hu[al] - iv * (hx[al].x * M[0] + hx[al].y * M[1] + hx[al].z * M[2]);
    W[0] = W[0] + hx[al].x * q[al];
    W[1] = W[1] + hx[al].y * q[al];
    W[2] = W[2] + hx[al].z * q[al];
  }
  const double cv = cbrt(V);
  const double kappa = c_hg * rho * cs * cv * cv;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    P3 f = hg_pattern(0, a) * q[0] + hg_pattern(1, a) * q[1] + hg_pattern(2, a) * q[2] + hg_pattern(3, a) * q[3];
    f = f - iv * (G[a].x * W[0] + G[a].y * W[1] + G[a].z * W[2]);
    fh[(3ll * a + 0) * nc + c] = (R)(-kappa * f.x);
    fh[(3ll * a + 1) * nc + c] = (R)(-kappa * f.y);
    fh[(3ll * a + 2) * nc + c] = (R)(-kappa * f.z);
  }
}

template <typename R>
__device__ __forceinline__ P3 hourglass_corner(const R *fh, long long nc, long long c, int a) {
  return {(double)fh[(3ll * a + 0) * nc + c], (double)fh[(3ll * a + 1) * nc + c], (double)fh[(3ll * a + 2) * nc + c]};
}

// ---------------------------------------------------------------------------
// Material strength: the stress module (Steinberg-Guinan shear modulus and
// yield, Wilkins deviatoric stress update)
// ---------------------------------------------------------------------------

// Steinberg, Cochran, Guinan (J. Appl. Phys. 51, 1498, 1980): G grows with
// the pressure scaled by the cube root of eta = rho_ref / rho and falls
// with the temperature T - T_ref = (e - e_ref) / cv, clamped at 0; the yield
// stress work-hardens, Y0 (1 + beta eps_p)^n up to Ymax, and follows G / G0.
__device__ __forceinline__ void steinberg_gy(const Strength &s, double p, double rho, double e, double eps_p,
                                             double &G, double &Y) {
  double g = s.shear0 + s.shear_dp * p * cbrt(s.rho_ref / rho) + s.shear_dt * (e - s.e_ref) * s.inv_cv;
  if (!(g > 0.0)) g = 0.0;
  // a cell that never yielded (eps_p exactly 0, which the remap keeps exact
  // where every donor has it) takes Y0 itself, the value pow(1, n) gives
  double y = eps_p > 0.0 ? s.yield0 * pow(1.0 + s.hard_beta * eps_p, s.hard_n) : s.yield0;
  if (y > s.yield_max) y = s.yield_max;
  G = g;
  Y = y * g * s.inv_shear0;
}

// S_c g for the deviatoric stress of cell c (sdev[q nc + c], q = xx, yy,
// zz, xy, yz, zx).
template <typename R>
__device__ __forceinline__ P3 stress_apply(const R *sd, long long nc, long long c, P3 g) {
  const double sxx = (double)sd[c], syy = (double)sd[nc + c], szz = (double)sd[2 * nc + c];
  const double sxy = (double)sd[3 * nc + c], syz = (double)sd[4 * nc + c], szx = (double)sd[5 * nc + c];
  return {sxx * g.x + sxy * g.y + szx * g.z, sxy * g.x + syy * g.y + syz * g.z, szx * g.x + syz * g.y + szz * g.z};
}

// Wilkins (1963): with the velocity gradient L[3 i + j] = du_i/dx_j, the
// strain rate deviator D' and the spin W, the trial stress
// S* = S + dt (2 G D' + W S - S W) (Jaumann rate); above the von Mises
// surface sqrt(3/2 S*:S*) = Y it is scaled back onto it (radial return)
// and the plastic strain grows by (J - Y) / (3 G).  S6 = (xx, yy, zz, xy,
// yz, zx) in place.
__device__ __forceinline__ void stress_update(double (&S6)[6], const double (&L)[9], double dt, double G, double Y,
                                              double &deps) {
  const double S[3][3] = {{S6[0], S6[3], S6[5]}, {S6[3], S6[1], S6[4]}, {S6[5], S6[4], S6[2]}};
  double D[3][3], W[3][3], T[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      D[i][j] = 0.5 * (L[3 * i + j] + L[3 * j + i]);
      W[i][j] = 0.5 * (L[3 * i + j] - L[3 * j + i]);
    }
  const double tr = (D[0][0] + D[1][1] + D[2][2]) / 3.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) D[i][i] -= tr;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double ws = 0.0, sw = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        ws += W[i][k] * S[k][j];
        sw += S[i][k] * W[k][j];
      }
      T[i][j] = S[i][j] + dt * (2.0 * G * D[i][j] + ws - sw);
    }
  double ss = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) ss += T[i][j] * T[i][j];
  double scale = 1.0;
  deps = 0.0;
  if (1.5 * ss > Y * Y) {  // J > Y, the square root and division only where the cell yields
    const double J = sqrt(1.5 * ss);
    scale = Y / J;
    if (G > 0.0) deps = (J - Y) / (3.0 * G);
  }
  S6[0] = scale * T[0][0];
  S6[1] = scale * T[1][1];
  S6[2] = scale * T[2][2];
  S6[3] = scale * 0.5 * (T[0][1] + T[1][0]);
  S6[4] = scale * 0.5 * (T[1][2] + T[2][1]);
  S6[5] = scale * 0.5 * (T[2][0] + T[0][2]);
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// End of a step: the block's minimum CFL step goes to one atomicMin on the
// bits of a positive double (order of positive doubles = order of their
// bits), then the last block to finish sets the next dt (and advances t by
// the step just taken in kDtAdvance mode).  Every thread of the block must
// call this; dtc = +inf for threads without a cell.
// RATE: the threads pass the CFL rate r = 1 / dt^2 instead (0 without a
// cell); the block takes the maximum and converts it once, dt = 1 / sqrt(r),
// which saves a square root and a division per cell on the FP64 pipe.
template <typename R, bool RATE = false>
__device__ __forceinline__ void block_min_dt_and_finalize(const Fields<R> &F, DevScalars *S, double dtc,
                                                          int mode, double dt_override) {
  __shared__ double smin[kBlock / 32];
  bool last = false;  // set in thread 0 only: no second barrier needed
  dtc = RATE ? warp_max(dtc) : warp_min(dtc);
  if ((threadIdx.x & 31) == 0) smin[threadIdx.x >> 5] = dtc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kBlock / 32 ? smin[threadIdx.x] : (RATE ? 0.0 : INFINITY);
    if (RATE) {
      v = warp_max(v);
      v = v > 0.0 ? 1.0 / sqrt(v) : INFINITY;
    } else {
      v = warp_min(v);
    }
    if (threadIdx.x == 0) {
      atomicMin(&S->dtmin_bits, (unsigned long long)__double_as_longlong(v));
      __threadfence();
      const unsigned int done = atomicAdd(&S->blocks_done, 1u);
      last = (done == gridDim.x - 1);
    }
  }
  if (!last || threadIdx.x != 0) return;
  // Last block: every other block has published its minimum.
  __threadfence();
  volatile DevScalars *VS = S;
  const double dtcfl = __longlong_as_double((long long)atomicAdd(&S->dtmin_bits, 0ull));
  double dt;
  if (mode == kDtInit) {
    dt = dtcfl;
    if (F.dt_init > 0.0 && F.dt_init < dt) dt = F.dt_init;
    VS->dt_last = dt;
  } else {
    if (mode == kDtAdvance) {
      const double h = step_dt(S, dt_override);
      const bool clamp = dt_override <= 0.0 && (VS->t_end - VS->t) < VS->dt;
      VS->t = clamp ? VS->t_end : VS->t + h;
      VS->dt_last = h;
      VS->cycle = VS->cycle + 1;
    }
    dt = fmin(dtcfl, F.growth * VS->dt_last);
  }
  if (!(dt > 0.0) || dt == INFINITY) set_status(S, SALE_EDT);
  else VS->dt = dt;
  VS->dtmin_bits = kInfBits;
  VS->blocks_done = 0;
  decide_next(VS);
  __threadfence();
}

// FP32 variant: the block minimum is taken in FP32 and converted once per
// block (the minimum of FP32 values is exact in either precision).
__device__ __forceinline__ float warp_min_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <typename R>
__device__ __forceinline__ void block_min_dt32_and_finalize(const Fields<R> &F, DevScalars *S, float dtc, int mode,
                                                            double dt_override, unsigned nblk) {
  __shared__ float smin32[kMaxWarpsPerBlock];
  bool last32 = false;  // set in thread 0 only: no second barrier needed
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nwarps = (int)((blockDim.x * blockDim.y * blockDim.z + 31) / 32);
  dtc = warp_min_f32(dtc);
  if ((tid & 31) == 0) smin32[tid >> 5] = dtc;
  __syncthreads();
  if (tid < 32) {
    float v = tid < nwarps ? smin32[tid] : INFINITY;
    v = warp_min_f32(v);
    if (tid == 0) {
      atomicMin(&S->dtmin_bits, (unsigned long long)__double_as_longlong((double)v));
      __threadfence();
      const unsigned int done = atomicAdd(&S->blocks_done, 1u);
      last32 = (done == nblk - 1);
    }
  }
  if (!last32 || tid != 0) return;
  __threadfence();
  volatile DevScalars *VS = S;
  const double dtcfl = __longlong_as_double((long long)atomicAdd(&S->dtmin_bits, 0ull));
  double dt;
  if (mode == kDtInit) {
    dt = dtcfl;
    if (F.dt_init > 0.0 && F.dt_init < dt) dt = F.dt_init;
    VS->dt_last = dt;
  } else {
    if (mode == kDtAdvance) {
      const double h = step_dt(S, dt_override);
      const bool clamp = dt_override <= 0.0 && (VS->t_end - VS->t) < VS->dt;
      VS->t = clamp ? VS->t_end : VS->t + h;
      VS->dt_last = h;
      VS->cycle = VS->cycle + 1;
    }
    dt = fmin(dtcfl, F.growth * VS->dt_last);
  }
  if (!(dt > 0.0) || dt == INFINITY) set_status(S, SALE_EDT);
  else VS->dt = dt;
  VS->dtmin_bits = kInfBits;
  VS->blocks_done = 0;
  decide_next(VS);
  __threadfence();
}

// ---------------------------------------------------------------------------
// Materials (several per cell, FP64 states)
// ---------------------------------------------------------------------------

// Predictor of the materials (predictor-corrector step): each material's
// half-step internal energy m_k e_k - dt/2 (alpha_k (p_k + q0) W + alpha_k
// W_hg), p_k at the state of x^n (volume V0, iv0 = 1/V0, viscosity q0), and
// the mixture at x^{n+1/2} (volume Vh, ivh = 1/Vh, im = 1/m): p and the
// mass-weighted c^2 as in mixture_eos; alpha_k p_k of the half step is left
// in aph[k] (0 for an absent material).
template <typename R>
__device__ __forceinline__ void mat_predict(const Fields<R> &F, long long c, double iv0, double q0, double hh,
                                            double work, double work_hg, double Vh, double ivh, double im,
                                            double (&aph)[kMaxMat], double &p, double &cs2) {
  double ps = 0.0, cm = 0.0;
  for (int k = 0; k < F.nmat; ++k) {
    const long long ia = 3ll * k * F.nc + c;
    const double a = (double)F.mat[ia];
    aph[k] = 0.0;
    if (!(a > 0.0)) continue;
    const double ie = (double)F.mat[ia + F.nc] * (double)F.mat[ia + 2 * F.nc];
    const double g = F.mgam[k], pinf = F.mpinf[k];
    const double apk = (g - 1.0) * ie * iv0 - g * pinf * a;
    const double ieh = ie - hh * ((apk + a * q0) * work + a * work_hg);
    aph[k] = (g - 1.0) * ieh * ivh - g * pinf * a;
    ps += aph[k];
    const double mc2 = g * (g - 1.0) * (ieh - pinf * a * Vh);
    cm += mc2 > 0.0 ? mc2 : 0.0;
  }
  p = ps;
  cs2 = cm * im;
}

// The predictor's shares alpha_k (p_k + q) of the half step, for the corrector.
template <typename R>
__device__ __forceinline__ void mat_store_shares(const Fields<R> &F, long long c, const double (&aph)[kMaxMat],
                                                 double q) {
  for (int k = 0; k < F.nmat; ++k)
    F.msh[k * F.nc + c] = (R)(aph[k] + (double)F.mat[3ll * k * F.nc + c] * q);
}

// Material k is a stiffened gas: p = (g - 1) rho e - g p_inf, c^2 = g (g - 1)
// (e - p_inf / rho) floored at 0 (p_inf = 0: ideal gas).
// Mixed cell c of volume V (iv = 1/V) and mass m (im = 1/m): materials
// present (alpha_k > 0) at density rho_k = m_k / (alpha_k V); p = sum_k
// alpha_k p_k, c^2 = sum_k m_k c_k^2 / m.  Written without a division, in
// the material's internal energy ie_k = m_k e_k: alpha_k p_k = (g - 1) ie_k / V
// - g p_inf alpha_k and m_k c_k^2 = g (g - 1) (ie_k - p_inf alpha_k V), floored
// at 0 (the FP64 pipe bounds these kernels, and a division takes about ten
// of its instructions).
template <typename R>
__device__ __forceinline__ void mixture_eos(const Fields<R> &F, long long c, double V, double iv, double im,
                                            double &p, double &cs2) {
  double ps = 0.0, cm = 0.0;
  for (int k = 0; k < F.nmat; ++k) {
    const long long ia = 3ll * k * F.nc + c;
    const double a = (double)F.mat[ia];
    if (!(a > 0.0)) continue;
    const double ie = (double)F.mat[ia + F.nc] * (double)F.mat[ia + 2 * F.nc];
    const double g = F.mgam[k], pinf = F.mpinf[k];
    ps += (g - 1.0) * ie * iv - g * pinf * a;
    const double mc2 = g * (g - 1.0) * (ie - pinf * a * V);
    cm += mc2 > 0.0 ? mc2 : 0.0;
  }
  p = ps;
  cs2 = cm * im;
}

// The cell pass's share of the compatible work for material k of cell c
// (uniform strain): e_k -= dt (alpha_k (p_k + q) W + alpha_k W_hg) / m_k,
// with W = sum_a dV/dx_a . ubar_a, W_hg the hourglass forces' work (0
// without control) and p_k at the state of x^n (volume V0, iv0 = 1/V0);
// with the predictor-corrector (pc) alpha_k (p_k + q) is the predictor's,
// from msh.  Returns m_k e_k of the new state (0 for an absent material).
template <typename R>
__device__ __forceinline__ double mat_work_share(const Fields<R> &F, long long c, int k, double V0, double iv0,
                                                 double q, double h, double work, double work_hg, bool pc) {
  const long long ia = 3ll * k * F.nc + c;
  const double a = (double)F.mat[ia];
  if (!(a > 0.0)) return 0.0;
  const double mk = (double)F.mat[ia + F.nc];
  double ek = (double)F.mat[ia + 2 * F.nc];
  const double g = F.mgam[k];
  const double sh = pc ? (double)F.msh[k * F.nc + c]
                       : (g - 1.0) * (mk * ek) * iv0 - g * F.mpinf[k] * a + a * q;  // alpha_k (p_k + q)
  ek -= h * (sh * work + a * work_hg) / mk;
  F.mat[ia + 2 * F.nc] = (R)ek;
  return mk * ek;
}

// Materials: each material's volume, mass and energy after the fluxes of
// the cell's six faces (mfx, written by a face pass; the cell's Lagrangian
// volume in F.vol); the kinetic-energy fix shared by mass; a material
// at or below kAlphaMin of the cell's new volume, or with no positive mass
// or volume, leaves the cell, its mass and energy going to the remaining
// materials by mass; fractions = remaining volumes over their sum.
template <typename R>
__device__ __forceinline__ void mat_remap_cell(const Fields<R> &F, DevScalars *S, long long c, int i, int j,
                                               int k) {
  const long long nc = F.nc, sy = F.nx, sz = (long long)F.nx * F.ny;
  double fix = 0.0;
  if (F.ke_fix) {
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      // share 1/(cells at the node) = 2^-(interior axes), exact, built from its bits
      const int ni = i + (a & 1), nj = j + ((a >> 1) & 1), nk = k + ((a >> 2) & 1);
      const int interior = (ni != 0 && ni != F.nx) + (nj != 0 && nj != F.ny) + (nk != 0 && nk != F.nz);
      fix += (double)F.dke[node_index(F.nx, F.ny, ni, nj, nk)] *
             __longlong_as_double((long long)(1023 - interior) << 52);
    }
  }
  const double vl = (double)F.vol[c];
  double mv[kMaxMat], mk[kMaxMat], me[kMaxMat];
  double m1 = 0.0, vtot = 0.0;
  for (int km = 0; km < F.nmat; ++km) {
    const R *f = F.mfx + 9ll * km * nc;  // f[(3 axis + q) nc + cell]
    double d[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      double v = -(double)f[q * nc + c] - (double)f[(3 + q) * nc + c] - (double)f[(6 + q) * nc + c];
      if (i + 1 < F.nx) v += (double)f[q * nc + c + 1];
      if (j + 1 < F.ny) v += (double)f[(3 + q) * nc + c + sy];
      if (k + 1 < F.nz) v += (double)f[(6 + q) * nc + c + sz];
      d[q] = v;
    }
    const long long ia = 3ll * km * nc + c;
    const double m0 = (double)F.mat[ia + nc];
    mv[km] = (double)F.mat[ia] * vl + d[0];
    mk[km] = m0 + d[1];
    me[km] = m0 * (double)F.mat[ia + 2 * nc] + d[2];
    m1 += mk[km];
    vtot += mv[km];
  }
  // the kinetic-energy share goes into me; one reciprocal per sum (the same
  // sum when no material leaves), one division per material for its
  // specific energy
  const double r1 = 1.0 / m1;
  const double fix_m = fix * r1;
  bool keep[kMaxMat];
  double mkeep = 0.0, mdrop = 0.0, iedrop = 0.0, vkeep = 0.0;
  for (int km = 0; km < F.nmat; ++km) {
    keep[km] = mk[km] > 0.0 && mv[km] > kAlphaMin * vtot;
    me[km] += mk[km] * fix_m;
    if (keep[km]) {
      mkeep += mk[km];
      vkeep += mv[km];
    } else {
      mdrop += mk[km];
      iedrop += me[km];
    }
  }
  const double imkeep = mkeep == m1 ? r1 : 1.0 / mkeep, ivkeep = 1.0 / vkeep;
  double msum = 0.0, iesum = 0.0;
  for (int km = 0; km < F.nmat; ++km) {
    const long long ia = 3ll * km * nc + c;
    if (keep[km]) {
      const double w = mk[km] * imkeep;
      const double mnew = mk[km] + w * mdrop;
      const double ie = me[km] + w * iedrop;
      F.mat[ia] = (R)(mv[km] * ivkeep);
      F.mat[ia + nc] = (R)mnew;
      F.mat[ia + 2 * nc] = (R)(ie / mnew);
      msum += mnew;
      iesum += ie;
    } else {
      F.mat[ia] = F.mat[ia + nc] = F.mat[ia + 2 * nc] = (R)0;
    }
  }
  if (!(msum > 0.0)) set_status(S, msum != msum ? SALE_ENAN : SALE_ENEGVOL);
  const double r = msum == m1 ? r1 : 1.0 / msum;
  F.m[c] = (R)msum;
  F.e[c] = (R)(iesum * r);
  if (F.im) F.im[c] = (R)r;
}

}  // namespace sale
