/*
 * sale_oracle.c -- plain serial FP64 reference of the SALE hydro cycle.
 *
 * TEST INFRASTRUCTURE (see sale_oracle.h).  Written for a reader checking
 * it against the method by eye: one loop per step, no blocking, no fusion.
 * Build with -O2 -ffp-contract=off so that no FMA contraction happens.
 *
 * The paper (ScalSALE, arXiv 2209.01983) names the physics steps -- ideal
 * gas EoS (Sec. I-D), Update_acceleration (Sec. III-D), Calculate_density
 * in Hydro (Sec. III-A), Lagrangian and Eulerian rezoning with an advection
 * phase (Table I, Sec. IV) -- and the scheme (SALE) without printing its
 * equations.  The formulas here are the standard ones:
 *
 *  Geometry:   V = (1/24) sum_f S_f . ((p2-p0) x (p3-p1)), S_f = p0+p1+p2+p3
 *              over the 6 outward faces (p0..p3) of the hex.  This is the
 *              divergence theorem over faces fanned from their node mean
 *              and equals the exact volume of the trilinear hex.
 *  EoS:        p = (g-1) rho e,  cs^2 = g (g-1) max(e,0).
 *  Viscosity:  div = sum_a gradV_a . u_a / V;  if div < 0
 *              q = rho (c_q (L div)^2 + c_l cs L |div|), else q = 0,
 *              L = V / max_f |A_f|.
 *  Lagrange:   sigma = p + q; F_a = sum_c sigma_c gradV_a(c);
 *              u+ = u + dt F/m_n (normal part zeroed on walls);
 *              ubar = (u + u+)/2; x+ = x + dt ubar;
 *              e+ = e - dt/m_c sigma_c sum_a gradV_a(c).ubar_a
 *              (compatible update: total energy conserved to roundoff).
 *  dt:         dt = min(cfl min_c L/sqrt(cs^2 + 2 q/rho), growth * dt_last).
 *  Remap:      rezone to the reference mesh; face swept volumes dV as hex
 *              volumes; mass flux mu = rho_donor dV (upwind); energy flux
 *              mu e_donor; node mass/momentum/KE fluxes on the dual mesh
 *              psi = sum_{cells at edge} (mu_lo + mu_hi)/8, upwind by node;
 *              KE lost by the momentum remap returned to the cells.
 *  Strength:   (optional, shear0 > 0) deviatoric stress S per cell after
 *              Wilkins (1963): L = (1/V) sum_a ubar_a (x) dV/dx_a,
 *              D' = sym(L) - tr(L)/3 I, W = skew(L),
 *              S* = S + dt (2 G D' + W S - S W), radial return to the von
 *              Mises surface sqrt(3/2 S:S) <= Y; G and Y from the
 *              Steinberg-Guinan model (Steinberg, Cochran, Guinan 1980);
 *              corner forces (p + q) dV/dx_a - S dV/dx_a, used in both the
 *              velocity and the compatible energy update; the CFL speed
 *              includes 4 G / (3 rho); S and the plastic strain are
 *              remapped like e (donor cell, per unit mass).
 */
#include "sale_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Hex geometry                                                        */
/* ------------------------------------------------------------------ */

/* Outward-oriented faces of the hex, local node ids in cyclic order. */
static const int FACE[6][4] = {
    {0, 4, 6, 2}, /* x-lo */
    {1, 3, 7, 5}, /* x-hi */
    {0, 1, 5, 4}, /* y-lo */
    {2, 6, 7, 3}, /* y-hi */
    {0, 2, 3, 1}, /* z-lo */
    {4, 5, 7, 6}, /* z-hi */
};

static void cross3(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* Coordinates relative to local node 0 (the volume and its gradient are
 * translation invariant; the shift only reduces cancellation). */
static void shift_to_node0(const double *X, double *Y) {
  for (int a = 0; a < 8; ++a)
    for (int d = 0; d < 3; ++d) Y[a * 3 + d] = X[a * 3 + d] - X[d];
}

double oracle_hex_volume(const double *X) {
  double Y[24];
  shift_to_node0(X, Y);
  double sum = 0.0;
  for (int f = 0; f < 6; ++f) {
    const double *p0 = &Y[FACE[f][0] * 3], *p1 = &Y[FACE[f][1] * 3];
    const double *p2 = &Y[FACE[f][2] * 3], *p3 = &Y[FACE[f][3] * 3];
    double d1[3], d2[3], D[3], S[3];
    for (int d = 0; d < 3; ++d) {
      d1[d] = p2[d] - p0[d];
      d2[d] = p3[d] - p1[d];
      S[d] = p0[d] + p1[d] + p2[d] + p3[d];
    }
    cross3(d1, d2, D);
    sum += dot3(S, D);
  }
  return sum / 24.0;
}

/* dV/dp_k of one face term T = S.((p2-p0)x(p3-p1)) is
 * (p_{k+1} + 2 p_{k+2} + p_{k+3}) x (p_{k+3} - p_{k+1})  (indices mod 4);
 * V = (1/24) sum_f T_f, so dV/dx_a sums this over the 3 faces holding a. */
void oracle_hex_volume_grad(const double *X, double *G) {
  double Y[24];
  shift_to_node0(X, Y);
  for (int i = 0; i < 24; ++i) G[i] = 0.0;
  for (int f = 0; f < 6; ++f) {
    for (int k = 0; k < 4; ++k) {
      const double *pa = &Y[FACE[f][(k + 1) & 3] * 3];
      const double *pb = &Y[FACE[f][(k + 2) & 3] * 3];
      const double *pc = &Y[FACE[f][(k + 3) & 3] * 3];
      double r[3], b[3], t[3];
      for (int d = 0; d < 3; ++d) {
        r[d] = pa[d] + 2.0 * pb[d] + pc[d];
        b[d] = pc[d] - pa[d];
      }
      cross3(r, b, t);
      double *g = &G[FACE[f][k] * 3];
      for (int d = 0; d < 3; ++d) g[d] += t[d];
    }
  }
  for (int i = 0; i < 24; ++i) G[i] /= 24.0;
}

/* Face vector area A_f = (1/2) (p2-p0) x (p3-p1), outward. */
void oracle_hex_face_areas(const double *X, double *A) {
  for (int f = 0; f < 6; ++f) {
    const double *p0 = &X[FACE[f][0] * 3], *p1 = &X[FACE[f][1] * 3];
    const double *p2 = &X[FACE[f][2] * 3], *p3 = &X[FACE[f][3] * 3];
    double d1[3], d2[3], D[3];
    for (int d = 0; d < 3; ++d) {
      d1[d] = p2[d] - p0[d];
      d2[d] = p3[d] - p1[d];
    }
    cross3(d1, d2, D);
    for (int d = 0; d < 3; ++d) A[f * 3 + d] = 0.5 * D[d];
  }
}

/* L = V / max_f |A_f|  (= min edge length on a box). */
double oracle_hex_char_length(const double *X) {
  double A[18];
  oracle_hex_face_areas(X, A);
  double amax2 = 0.0;
  for (int f = 0; f < 6; ++f) {
    double a2 = dot3(&A[f * 3], &A[f * 3]);
    if (a2 > amax2) amax2 = a2;
  }
  return oracle_hex_volume(X) / sqrt(amax2);
}

/* ------------------------------------------------------------------ */
/* Indexing                                                            */
/* ------------------------------------------------------------------ */

static long long cell_id(const oracle_state *s, int i, int j, int k) {
  return (long long)i + (long long)s->nx * ((long long)j + (long long)s->ny * k);
}

static long long node_id(const oracle_state *s, int i, int j, int k) {
  return (long long)i +
         (long long)(s->nx + 1) * ((long long)j + (long long)(s->ny + 1) * k);
}

/* Gather the 8 node coordinates of cell (i,j,k) from arrays px,py,pz. */
static void gather_hex(const oracle_state *s, int i, int j, int k,
                       const double *px, const double *py, const double *pz,
                       double *X) {
  for (int a = 0; a < 8; ++a) {
    long long n = node_id(s, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
    X[a * 3 + 0] = px[n];
    X[a * 3 + 1] = py[n];
    X[a * 3 + 2] = pz[n];
  }
}

/* Number of cells that contain node (i,j,k). */
static int node_cell_count(const oracle_state *s, int i, int j, int k) {
  int c = 1;
  c *= (i == 0 || i == s->nx) ? 1 : 2;
  c *= (j == 0 || j == s->ny) ? 1 : 2;
  c *= (k == 0 || k == s->nz) ? 1 : 2;
  return c;
}

/* Zero the velocity components normal to the reflecting walls the node
 * lies on (all walls are axis-aligned planes). */
static void apply_wall_bc(const oracle_state *s, int i, int j, int k,
                          double *uu, double *vv, double *ww) {
  if ((i == 0 && s->prm.reflect[0]) || (i == s->nx && s->prm.reflect[1])) *uu = 0.0;
  if ((j == 0 && s->prm.reflect[2]) || (j == s->ny && s->prm.reflect[3])) *vv = 0.0;
  if ((k == 0 && s->prm.reflect[4]) || (k == s->nz && s->prm.reflect[5])) *ww = 0.0;
}

/* ------------------------------------------------------------------ */
/* State                                                               */
/* ------------------------------------------------------------------ */

static double *alloc_zero(long long n) {
  return (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
}

oracle_state *oracle_create(int nx, int ny, int nz, const double *xn,
                            const double *yn, const double *zn,
                            const oracle_params *prm) {
  if (nx < 1 || ny < 1 || nz < 1 || !xn || !yn || !zn || !prm) return NULL;
  oracle_state *s = (oracle_state *)calloc(1, sizeof(oracle_state));
  if (!s) return NULL;
  s->nx = nx;
  s->ny = ny;
  s->nz = nz;
  s->nc = (long long)nx * ny * nz;
  s->nn = (long long)(nx + 1) * (ny + 1) * (nz + 1);
  s->prm = *prm;
  double **node_arrays[] = {&s->x, &s->y, &s->z, &s->xr, &s->yr,
                            &s->zr, &s->u, &s->v, &s->w, &s->mn};
  for (size_t i = 0; i < sizeof(node_arrays) / sizeof(node_arrays[0]); ++i) {
    *node_arrays[i] = alloc_zero(s->nn);
    if (!*node_arrays[i]) { oracle_destroy(s); return NULL; }
  }
  double **cell_arrays[] = {&s->m, &s->e, &s->vol, &s->rho, &s->p, &s->q, &s->cs, &s->len,
                            &s->sxx, &s->syy, &s->szz, &s->sxy, &s->syz, &s->szx, &s->eps_p};
  for (size_t i = 0; i < sizeof(cell_arrays) / sizeof(cell_arrays[0]); ++i) {
    *cell_arrays[i] = alloc_zero(s->nc);
    if (!*cell_arrays[i]) { oracle_destroy(s); return NULL; }
  }
  if (prm->nmat > ORACLE_MAX_MAT) { oracle_destroy(s); return NULL; }
  if (prm->nmat >= 2) {
    double **mat_arrays[] = {&s->alpha, &s->mm, &s->me};
    for (size_t i = 0; i < 3; ++i) {
      *mat_arrays[i] = alloc_zero(prm->nmat * s->nc);
      if (!*mat_arrays[i]) { oracle_destroy(s); return NULL; }
    }
  }
  memcpy(s->x, xn, sizeof(double) * s->nn);
  memcpy(s->y, yn, sizeof(double) * s->nn);
  memcpy(s->z, zn, sizeof(double) * s->nn);
  memcpy(s->xr, xn, sizeof(double) * s->nn);
  memcpy(s->yr, yn, sizeof(double) * s->nn);
  memcpy(s->zr, zn, sizeof(double) * s->nn);
  return s;
}

void oracle_destroy(oracle_state *s) {
  if (!s) return;
  double *arrays[] = {s->x, s->y, s->z, s->xr, s->yr, s->zr, s->u, s->v, s->w,
                      s->mn, s->m, s->e, s->vol, s->rho, s->p, s->q, s->cs, s->len,
                      s->sxx, s->syy, s->szz, s->sxy, s->syz, s->szx, s->eps_p, s->alpha, s->mm, s->me};
  for (size_t i = 0; i < sizeof(arrays) / sizeof(arrays[0]); ++i) free(arrays[i]);
  free(s);
}

/* Node mass m_n = sum over the cells holding the node of m_c / 8. */
static void node_masses_from_cells(oracle_state *s) {
  for (long long n = 0; n < s->nn; ++n) s->mn[n] = 0.0;
  for (int k = 0; k < s->nz; ++k)
    for (int j = 0; j < s->ny; ++j)
      for (int i = 0; i < s->nx; ++i) {
        double share = s->m[cell_id(s, i, j, k)] / 8.0;
        for (int a = 0; a < 8; ++a)
          s->mn[node_id(s, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1))] += share;
      }
}

/* ------------------------------------------------------------------ */
/* Material strength (R17)                                             */
/* ------------------------------------------------------------------ */

/* Steinberg-Guinan (J. Appl. Phys. 51, 1498, 1980): the shear modulus
 * grows with pressure, scaled by the cube root of the volume ratio
 * eta = rho_ref / rho, and falls with temperature, T - T_ref =
 * (e - e_ref) / cv:  G = G0 + G_p p eta^(1/3) + G_T (T - T_ref),  clamped
 * at 0 (melt).  The yield stress work-hardens up to a cap and follows G:
 * Y = min(Y0 (1 + beta eps_p)^n, Ymax) G / G0. */
void oracle_steinberg(const oracle_params *prm, double p, double rho, double e, double eps_p, double *G,
                      double *Y) {
  const double eta = prm->rho_ref / rho;
  double g = prm->shear0 + prm->shear_dp * p * cbrt(eta) + prm->shear_dt * (e - prm->e_ref) / prm->cv;
  if (!(g > 0.0)) g = 0.0;
  double y = prm->yield0 * pow(1.0 + prm->hard_beta * eps_p, prm->hard_n);
  if (y > prm->yield_max) y = prm->yield_max;
  *G = g;
  *Y = y * g / prm->shear0;
}

/* One Wilkins (1963) update of the deviatoric stress.  With the strain
 * rate D = (L + L^T)/2, its deviator D' = D - tr(D)/3 I and the spin
 * W = (L - L^T)/2, the trial stress is S* = S + dt (2 G D' + W S - S W)
 * (the Jaumann rate, which rotates S with the material).  Von Mises:
 * J = sqrt(3/2 S*:S*); above the yield stress the trial stress is scaled
 * back onto the surface J = Y (radial return) and the equivalent plastic
 * strain grows by (J - Y) / (3 G). */
void oracle_stress_update(const double *S6, const double *L, double dt, double G, double Y, double *S_out,
                          double *deps) {
  double S[3][3] = {{S6[0], S6[3], S6[5]}, {S6[3], S6[1], S6[4]}, {S6[5], S6[4], S6[2]}};
  double D[3][3], W[3][3], T[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      D[i][j] = 0.5 * (L[3 * i + j] + L[3 * j + i]);
      W[i][j] = 0.5 * (L[3 * i + j] - L[3 * j + i]);
    }
  const double tr = (D[0][0] + D[1][1] + D[2][2]) / 3.0;
  for (int i = 0; i < 3; ++i) D[i][i] -= tr;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double ws = 0.0, sw = 0.0;
      for (int k = 0; k < 3; ++k) {
        ws += W[i][k] * S[k][j];
        sw += S[i][k] * W[k][j];
      }
      T[i][j] = S[i][j] + dt * (2.0 * G * D[i][j] + ws - sw);
    }
  double ss = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) ss += T[i][j] * T[i][j];
  const double J = sqrt(1.5 * ss);
  double scale = 1.0;
  *deps = 0.0;
  if (J > Y) {
    scale = Y / J;
    if (G > 0.0) *deps = (J - Y) / (3.0 * G);
  }
  S_out[0] = scale * T[0][0];
  S_out[1] = scale * T[1][1];
  S_out[2] = scale * T[2][2];
  S_out[3] = scale * 0.5 * (T[0][1] + T[1][0]);
  S_out[4] = scale * 0.5 * (T[1][2] + T[2][1]);
  S_out[5] = scale * 0.5 * (T[2][0] + T[0][2]);
}

static int strength_on(const oracle_state *s) { return s->prm.shear0 > 0.0; }

/* out = S_c g: the deviatoric stress of cell c applied to a 3-vector. */
static void stress_apply(const oracle_state *s, long long c, const double *g, double *out) {
  out[0] = s->sxx[c] * g[0] + s->sxy[c] * g[1] + s->szx[c] * g[2];
  out[1] = s->sxy[c] * g[0] + s->syy[c] * g[1] + s->syz[c] * g[2];
  out[2] = s->szx[c] * g[0] + s->syz[c] * g[1] + s->szz[c] * g[2];
}

/* ------------------------------------------------------------------ */
/* Materials (R18)                                                     */
/* ------------------------------------------------------------------ */

static int mm_on(const oracle_state *s) { return s->prm.nmat >= 2; }

/* Stiffened-gas EoS of material k: p = (g - 1) rho e - g p_inf; its sound
 * speed c^2 = g (p + p_inf) / rho = g (g - 1) (e - p_inf / rho), floored
 * at 0 like the single gas's.  p_inf = 0 is the ideal gas. */
static double mat_pressure(const oracle_state *s, int k, double rho, double e) {
  const double g = s->prm.mat_gamma[k];
  return (g - 1.0) * rho * e - g * s->prm.mat_pinf[k];
}

static double mat_cs2(const oracle_state *s, int k, double rho, double e) {
  const double g = s->prm.mat_gamma[k];
  const double c2 = g * (g - 1.0) * (e - s->prm.mat_pinf[k] / rho);
  return c2 > 0.0 ? c2 : 0.0;
}

/* Mixed cell c of volume V and mass m: the materials present (alpha_k > 0)
 * have density rho_k = m_k / (alpha_k V); the cell pressure is
 * sum_k alpha_k p_k and the squared sound speed the mass-weighted
 * sum_k m_k c_k^2 / m.  me holds the materials' specific energies
 * ([k * nc + c]: the state's, or the predictor's half-step ones). */
static void mixture_eos(const oracle_state *s, long long c, double V, double m, const double *me, double *p,
                        double *cs2) {
  double ps = 0.0, cm = 0.0;
  for (int k = 0; k < s->prm.nmat; ++k) {
    const long long kc = k * s->nc + c;
    const double a = s->alpha[kc];
    if (!(a > 0.0)) continue;
    const double rk = s->mm[kc] / (a * V);
    ps += a * mat_pressure(s, k, rk, me[kc]);
    cm += s->mm[kc] * mat_cs2(s, k, rk, me[kc]);
  }
  *p = ps;
  *cs2 = cm / m;
}

/* Cell totals from the materials: m = sum_k m_k, e = sum_k m_k e_k / m. */
static void mm_totals(oracle_state *s, long long c) {
  double m = 0.0, ie = 0.0;
  for (int k = 0; k < s->prm.nmat; ++k) {
    m += s->mm[k * s->nc + c];
    ie += s->mm[k * s->nc + c] * s->me[k * s->nc + c];
  }
  s->m[c] = m;
  s->e[c] = ie / m;
}

/* EoS (R2), sound speed and artificial viscosity (R3) of cell c with node
 * positions X and velocities U (24 values each), mass m and specific
 * internal energy e (with materials, the EoS is the mixture's of the
 * material energies me, R18).  Returns a status. */
static int cell_state(const oracle_state *s, long long c, const double *X, const double *U, double m, double e,
                      const double *me, double *V_out, double *rho_out, double *p_out, double *q_out,
                      double *cs_out, double *L_out) {
  const double g = s->prm.gamma;
  double G[24];
  double V = oracle_hex_volume(X);
  if (!(V > 0.0)) return isnan(V) ? ORACLE_ENAN : ORACLE_ENEGVOL;
  double rho = m / V;
  double p, cs;
  if (mm_on(s)) {
    double cs2;
    mixture_eos(s, c, V, m, me, &p, &cs2);
    cs = sqrt(cs2);
  } else {
    p = (g - 1.0) * rho * e;
    cs = sqrt(g * (g - 1.0) * (e > 0.0 ? e : 0.0));
  }
  oracle_hex_volume_grad(X, G);
  double dvdt = 0.0;
  for (int a = 0; a < 8; ++a) dvdt += dot3(&G[a * 3], &U[a * 3]);
  double div = dvdt / V;
  double L = oracle_hex_char_length(X);
  double q = 0.0;
  if (div < 0.0) {
    double ld = L * div;
    q = rho * (s->prm.c_q * ld * ld + s->prm.c_l * cs * L * fabs(div));
  }
  if (isnan(p) || isnan(q) || isnan(cs)) return ORACLE_ENAN;
  *V_out = V;
  *rho_out = rho;
  *p_out = p;
  *q_out = q;
  *cs_out = cs;
  *L_out = L;
  return ORACLE_OK;
}

/* EoS, sound speed, artificial viscosity and length scale at the current
 * positions and velocities. */
int oracle_eos(oracle_state *s) {
  for (int k = 0; k < s->nz; ++k)
    for (int j = 0; j < s->ny; ++j)
      for (int i = 0; i < s->nx; ++i) {
        long long c = cell_id(s, i, j, k);
        double X[24], U[24];
        gather_hex(s, i, j, k, s->x, s->y, s->z, X);
        gather_hex(s, i, j, k, s->u, s->v, s->w, U);
        int rc = cell_state(s, c, X, U, s->m[c], s->e[c], s->me, &s->vol[c], &s->rho[c], &s->p[c], &s->q[c],
                            &s->cs[c], &s->len[c]);
        if (rc) return s->status = rc;
      }
  return ORACLE_OK;
}

double oracle_cfl_dt(const oracle_state *s) {
  double dt = INFINITY;
  for (long long c = 0; c < s->nc; ++c) {
    double c2 = s->cs[c] * s->cs[c] + 2.0 * s->q[c] / s->rho[c];
    if (strength_on(s)) {  /* longitudinal elastic wave: K/rho + 4 G / (3 rho) */
      double G, Y;
      oracle_steinberg(&s->prm, s->p[c], s->rho[c], s->e[c], s->eps_p[c], &G, &Y);
      c2 += 4.0 * G / (3.0 * s->rho[c]);
    }
    double ceff = sqrt(c2);
    double dtc = s->prm.cfl * s->len[c] / ceff;
    if (dtc < dt) dt = dtc;
  }
  return dt;
}

/* Proposed next dt: min(CFL limit, growth * last dt used). */
static int propose_dt(oracle_state *s) {
  double dt = oracle_cfl_dt(s);
  double cap = s->prm.dt_growth * s->dt_last;
  if (cap < dt) dt = cap;
  if (!(dt > 0.0) || isinf(dt)) {
    s->status = ORACLE_EDT;
    return s->status;
  }
  s->dt = dt;
  return ORACLE_OK;
}

/* The rest of an initial state once m and e are set: u = 0, node masses,
 * derived fields and the first dt (capped by dt_init). */
static int init_finish(oracle_state *s) {
  for (long long n = 0; n < s->nn; ++n) s->u[n] = s->v[n] = s->w[n] = 0.0;
  node_masses_from_cells(s);
  s->t = 0.0;
  s->cycle = 0;
  s->status = ORACLE_OK;
  int rc = oracle_eos(s);
  if (rc) return rc;
  double dt = oracle_cfl_dt(s);
  if (s->prm.dt_init > 0.0 && s->prm.dt_init < dt) dt = s->prm.dt_init;
  if (!(dt > 0.0) || isinf(dt)) return s->status = ORACLE_EDT;
  s->dt = dt;
  s->dt_last = dt;
  return ORACLE_OK;
}

int oracle_init_prim(oracle_state *s, const double *rho0, const double *p0,
                     long long deposit_cell, double deposit_energy) {
  if (mm_on(s)) return s->status = ORACLE_EINVAL;  /* materials: oracle_init_materials */
  const double g = s->prm.gamma;
  for (int k = 0; k < s->nz; ++k)
    for (int j = 0; j < s->ny; ++j)
      for (int i = 0; i < s->nx; ++i) {
        long long c = cell_id(s, i, j, k);
        double X[24];
        gather_hex(s, i, j, k, s->x, s->y, s->z, X);
        double V = oracle_hex_volume(X);
        s->m[c] = rho0[c] * V;
        s->e[c] = p0[c] / ((g - 1.0) * rho0[c]);
      }
  if (deposit_cell >= 0 && deposit_cell < s->nc)
    s->e[deposit_cell] = deposit_energy / s->m[deposit_cell];
  return init_finish(s);
}

/* The materials of the multi-material scheme (R18) take neither strength
 * nor the second-order remap (the predictor-corrector and hourglass
 * control, yes). */
static int mm_options_ok(const oracle_state *s) {
  const oracle_params *p = &s->prm;
  if (p->nmat < 2 || p->nmat > ORACLE_MAX_MAT) return 0;
  if (strength_on(s) || p->remap_order == 2) return 0;
  for (int k = 0; k < p->nmat; ++k)
    if (!(p->mat_gamma[k] > 1.0) || !(p->mat_pinf[k] >= 0.0) || isinf(p->mat_gamma[k]) || isinf(p->mat_pinf[k]))
      return 0;
  return 1;
}

int oracle_init_materials(oracle_state *s, const double *rho0, const double *p0, const int *mat,
                          long long deposit_cell, double deposit_energy) {
  if (!mm_options_ok(s)) return s->status = ORACLE_EINVAL;
  const long long nc = s->nc;
  for (long long c = 0; c < nc; ++c)
    if (mat[c] < 0 || mat[c] >= s->prm.nmat) return s->status = ORACLE_EINVAL;
  for (int k = 0; k < s->nz; ++k)
    for (int j = 0; j < s->ny; ++j)
      for (int i = 0; i < s->nx; ++i) {
        long long c = cell_id(s, i, j, k);
        double X[24];
        gather_hex(s, i, j, k, s->x, s->y, s->z, X);
        const int mk = mat[c];
        const double g = s->prm.mat_gamma[mk];
        double m = rho0[c] * oracle_hex_volume(X);
        /* the EoS solved for e at (rho0, p0) */
        double e = (p0[c] + g * s->prm.mat_pinf[mk]) / ((g - 1.0) * rho0[c]);
        if (c == deposit_cell) e = deposit_energy / m;
        for (int q = 0; q < s->prm.nmat; ++q) {
          s->alpha[q * nc + c] = q == mk ? 1.0 : 0.0;
          s->mm[q * nc + c] = q == mk ? m : 0.0;
          s->me[q * nc + c] = q == mk ? e : 0.0;
        }
        s->m[c] = m;
        s->e[c] = e;
      }
  return init_finish(s);
}

int oracle_set_materials(oracle_state *s, const double *alpha, const double *mm, const double *me) {
  if (!mm_options_ok(s)) return s->status = ORACLE_EINVAL;
  const long long nc = s->nc;
  for (long long c = 0; c < nc; ++c) {
    double asum = 0.0;
    for (int k = 0; k < s->prm.nmat; ++k) {
      const long long kc = k * nc + c;
      if (!(alpha[kc] >= 0.0) || !(mm[kc] >= 0.0) || (alpha[kc] > 0.0) != (mm[kc] > 0.0) || isnan(me[kc]))
        return s->status = ORACLE_EINVAL;
      asum += alpha[kc];
    }
    if (!(fabs(asum - 1.0) <= 1e-12)) return s->status = ORACLE_EINVAL;
  }
  const size_t b = sizeof(double) * (size_t)(s->prm.nmat * nc);
  memcpy(s->alpha, alpha, b);
  memcpy(s->mm, mm, b);
  memcpy(s->me, me, b);
  for (long long c = 0; c < nc; ++c) mm_totals(s, c);
  s->status = ORACLE_OK;
  int rc = oracle_eos(s);
  if (rc) return rc;
  return propose_dt(s);
}

int oracle_set_state(oracle_state *s, const double *x, const double *y,
                     const double *z, const double *u, const double *v,
                     const double *w, const double *mn, const double *m,
                     const double *e, double t, double dt_last) {
  size_t nb = sizeof(double) * (size_t)s->nn, cb = sizeof(double) * (size_t)s->nc;
  memcpy(s->x, x, nb);
  memcpy(s->y, y, nb);
  memcpy(s->z, z, nb);
  memcpy(s->u, u, nb);
  memcpy(s->v, v, nb);
  memcpy(s->w, w, nb);
  memcpy(s->mn, mn, nb);
  memcpy(s->m, m, cb);
  memcpy(s->e, e, cb);
  s->t = t;
  s->dt_last = dt_last;
  s->status = ORACLE_OK;
  int rc = oracle_eos(s);
  if (rc) return rc;
  return propose_dt(s);
}

/* ------------------------------------------------------------------ */
/* Lagrangian step                                                     */
/* ------------------------------------------------------------------ */

/* Viscous hourglass corner forces of one cell (reading R16, Flanagan and
 * Belytschko 1981).  With local node a = di + 2 dj + 4 dk and signs
 * s = 2 d - 1, the four hourglass patterns are h_1 = s_x s_y, h_2 = s_y s_z,
 * h_3 = s_z s_x, h_4 = s_x s_y s_z.  With b_a = dV/dx_a / V (the mean shape
 * function gradients) the hourglass shape vectors are
 *     gamma_alpha(a) = h_alpha(a) - sum_i (sum_b h_alpha(b) x_b,i) b_a,i,
 * which vanish on every linear field; the hourglass rates are
 * q_alpha = sum_a gamma_alpha(a) u_a and the corner forces
 *     f_a = -kappa sum_alpha gamma_alpha(a) q_alpha,
 * kappa = c_hg rho cs V^(2/3).  X, U: the cell's 8 nodes (24 values). */
static void hourglass_forces(const double *X, const double *U, double V, double rho, double cs, double c_hg,
                             double *fh) {
  double G[24];
  oracle_hex_volume_grad(X, G);
  double h[4][8];
  for (int a = 0; a < 8; ++a) {
    const double sx = (a & 1) ? 1.0 : -1.0, sy = (a & 2) ? 1.0 : -1.0, sz = (a & 4) ? 1.0 : -1.0;
    h[0][a] = sx * sy;
    h[1][a] = sy * sz;
    h[2][a] = sz * sx;
    h[3][a] = sx * sy * sz;
  }
  double gam[4][8];
  for (int al = 0; al < 4; ++al) {
    double hx[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < 8; ++b)
      for (int i = 0; i < 3; ++i) hx[i] += h[al][b] * X[b * 3 + i];
    for (int a = 0; a < 8; ++a) gam[al][a] = h[al][a] - dot3(hx, &G[a * 3]) / V;
  }
  const double kappa = c_hg * rho * cs * cbrt(V) * cbrt(V);
  for (int a = 0; a < 24; ++a) fh[a] = 0.0;
  for (int al = 0; al < 4; ++al) {
    double q[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < 8; ++b)
      for (int i = 0; i < 3; ++i) q[i] += gam[al][b] * U[b * 3 + i];
    for (int a = 0; a < 8; ++a)
      for (int i = 0; i < 3; ++i) fh[a * 3 + i] -= kappa * gam[al][a] * q[i];
  }
}

/* Lagrangian step (R4).  Single stage: corner forces sigma^n dV/dx(x^n).
 * Predictor-corrector (R15, time_order = 2): a half step of dt/2 first
 * moves the nodes to x^{n+1/2} = x^n + dt/2 u^n and the cells to
 * e^{n+1/2} = e^n - dt/(2m) sigma^n sum_a dV/dx_a(x^n).u^n_a, where the EoS
 * and viscosity (with u^n) give sigma^{n+1/2}; the full step then uses the
 * corner forces sigma^{n+1/2} dV/dx(x^{n+1/2}) for both the velocity and
 * the compatible energy update, so total energy stays exact. */
int oracle_lagrange_step(oracle_state *s, double dt) {
  if (s->status) return s->status;
  if (!(dt > 0.0)) return s->status = ORACLE_EDT;
  const long long nn = s->nn, nc = s->nc;
  const int pc = s->prm.time_order == 2;
  const int str = strength_on(s);
  if (str && pc) return s->status = ORACLE_EINVAL;  /* strength takes the single-stage step */
  const int mm = mm_on(s);
  if (mm && !mm_options_ok(s)) return s->status = ORACLE_EINVAL;
  double *fx = alloc_zero(nn), *fy = alloc_zero(nn), *fz = alloc_zero(nn);
  double *ubx = alloc_zero(nn), *uby = alloc_zero(nn), *ubz = alloc_zero(nn);
  double *e_new = alloc_zero(nc), *sig = alloc_zero(nc);
  double *xh = alloc_zero(nn), *yh = alloc_zero(nn), *zh = alloc_zero(nn);
  const int hg = s->prm.c_hg > 0.0;
  double *fh = hg ? alloc_zero(24 * nc) : NULL;
  double *s_new = str ? alloc_zero(7 * nc) : NULL;  /* S (6) and eps_p at n+1 */
  /* materials with the predictor: half-step specific energies, and each
   * material's half-step share alpha_k (p_k + q) of the cell's sigma */
  const int mmpc = mm && pc;
  double *meh = mmpc ? alloc_zero(s->prm.nmat * nc) : NULL, *share = mmpc ? alloc_zero(s->prm.nmat * nc) : NULL;
  if (!fx || !fy || !fz || !ubx || !uby || !ubz || !e_new || !sig || !xh || !yh || !zh || (hg && !fh) ||
      (str && !s_new) || (mmpc && (!meh || !share))) {
    free(fx); free(fy); free(fz); free(ubx); free(uby); free(ubz); free(e_new); free(sig);
    free(xh); free(yh); free(zh); free(fh); free(s_new); free(meh); free(share);
    return s->status = ORACLE_ENOMEM;
  }

  /* Hourglass corner forces of x^n, u^n (R16), held for the whole step. */
  if (hg)
    for (int k = 0; k < s->nz; ++k)
      for (int j = 0; j < s->ny; ++j)
        for (int i = 0; i < s->nx; ++i) {
          long long c = cell_id(s, i, j, k);
          double X[24], U[24];
          gather_hex(s, i, j, k, s->x, s->y, s->z, X);
          gather_hex(s, i, j, k, s->u, s->v, s->w, U);
          hourglass_forces(X, U, s->vol[c], s->rho[c], s->cs[c], s->prm.c_hg, &fh[24 * c]);
        }

  /* Stress of every cell and the positions its corner forces are taken at. */
  const double *gx = s->x, *gy = s->y, *gz = s->z;
  for (long long c = 0; c < nc; ++c) sig[c] = s->p[c] + s->q[c];
  if (pc) {
    for (long long n = 0; n < nn; ++n) {
      xh[n] = s->x[n] + 0.5 * dt * s->u[n];
      yh[n] = s->y[n] + 0.5 * dt * s->v[n];
      zh[n] = s->z[n] + 0.5 * dt * s->w[n];
    }
    for (int k = 0; k < s->nz; ++k)
      for (int j = 0; j < s->ny; ++j)
        for (int i = 0; i < s->nx; ++i) {
          long long c = cell_id(s, i, j, k);
          double X[24], G[24], U[24], XH[24];
          gather_hex(s, i, j, k, s->x, s->y, s->z, X);
          gather_hex(s, i, j, k, s->u, s->v, s->w, U);
          oracle_hex_volume_grad(X, G);
          double work = 0.0, work_hg = 0.0;
          for (int a = 0; a < 8; ++a) work += dot3(&G[a * 3], &U[a * 3]);
          if (hg)
            for (int a = 0; a < 8; ++a) work_hg += dot3(&fh[24 * c + a * 3], &U[a * 3]);
          double e_half = s->e[c] - 0.5 * dt / s->m[c] * sig[c] * work;
          if (hg) e_half -= 0.5 * dt / s->m[c] * work_hg;
          if (mmpc)  /* each material's half step, its share of the work as in the corrector below */
            for (int kk = 0; kk < s->prm.nmat; ++kk) {
              const long long kc = kk * nc + c;
              const double a = s->alpha[kc];
              meh[kc] = 0.0;
              if (!(a > 0.0)) continue;
              const double mk = s->mm[kc];
              const double pk = mat_pressure(s, kk, mk / (a * s->vol[c]), s->me[kc]);
              meh[kc] = s->me[kc] - 0.5 * dt / mk * (a * (pk + s->q[c]) * work + (hg ? a * work_hg : 0.0));
            }
          gather_hex(s, i, j, k, xh, yh, zh, XH);
          double V, rho, p, q, cs, L;
          int rc = cell_state(s, c, XH, U, s->m[c], e_half, meh, &V, &rho, &p, &q, &cs, &L);
          if (rc) {
            free(fx); free(fy); free(fz); free(ubx); free(uby); free(ubz); free(e_new); free(sig);
            free(xh); free(yh); free(zh); free(fh); free(meh); free(share);
            return s->status = rc;
          }
          e_new[c] = p + q;  /* sigma^{n+1/2}, moved into sig below */
          if (mmpc)
            for (int kk = 0; kk < s->prm.nmat; ++kk) {
              const long long kc = kk * nc + c;
              const double a = s->alpha[kc];
              share[kc] = a > 0.0 ? a * (mat_pressure(s, kk, s->mm[kc] / (a * V), meh[kc]) + q) : 0.0;
            }
        }
    memcpy(sig, e_new, sizeof(double) * (size_t)nc);
    gx = xh;
    gy = yh;
    gz = zh;
  }

  /* Corner forces F_a += sigma_c dV_c/dx_a, gathered to nodes. */
  for (int k = 0; k < s->nz; ++k)
    for (int j = 0; j < s->ny; ++j)
      for (int i = 0; i < s->nx; ++i) {
        long long c = cell_id(s, i, j, k);
        double sigma = sig[c];
        double X[24], G[24];
        gather_hex(s, i, j, k, gx, gy, gz, X);
        oracle_hex_volume_grad(X, G);
        for (int a = 0; a < 8; ++a) {
          long long n = node_id(s, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
          double cf[3] = {sigma * G[a * 3 + 0], sigma * G[a * 3 + 1], sigma * G[a * 3 + 2]};
          if (str) {  /* the deviatoric part of the cell stress, -S dV/dx_a */
            double sg[3];
            stress_apply(s, c, &G[a * 3], sg);
            for (int d = 0; d < 3; ++d) cf[d] -= sg[d];
          }
          if (hg)
            for (int d = 0; d < 3; ++d) cf[d] += fh[24 * c + a * 3 + d];
          fx[n] += cf[0];
          fy[n] += cf[1];
          fz[n] += cf[2];
        }
      }

  /* Velocity update with wall conditions; time-centred velocity. */
  for (int k = 0; k <= s->nz; ++k)
    for (int j = 0; j <= s->ny; ++j)
      for (int i = 0; i <= s->nx; ++i) {
        long long n = node_id(s, i, j, k);
        double un = s->u[n] + dt * fx[n] / s->mn[n];
        double vn = s->v[n] + dt * fy[n] / s->mn[n];
        double wn = s->w[n] + dt * fz[n] / s->mn[n];
        apply_wall_bc(s, i, j, k, &un, &vn, &wn);
        ubx[n] = 0.5 * (s->u[n] + un);
        uby[n] = 0.5 * (s->v[n] + vn);
        ubz[n] = 0.5 * (s->w[n] + wn);
        s->u[n] = un;
        s->v[n] = vn;
        s->w[n] = wn;
      }

  /* Compatible internal-energy update with the same corner forces. */
  for (int k = 0; k < s->nz; ++k)
    for (int j = 0; j < s->ny; ++j)
      for (int i = 0; i < s->nx; ++i) {
        long long c = cell_id(s, i, j, k);
        double sigma = sig[c];
        double X[24], G[24], UB[24];
        gather_hex(s, i, j, k, gx, gy, gz, X);
        gather_hex(s, i, j, k, ubx, uby, ubz, UB);
        oracle_hex_volume_grad(X, G);
        double work = 0.0, work_hg = 0.0;
        for (int a = 0; a < 8; ++a) work += dot3(&G[a * 3], &UB[a * 3]);
        if (hg)
          for (int a = 0; a < 8; ++a) work_hg += dot3(&fh[24 * c + a * 3], &UB[a * 3]);
        e_new[c] = s->e[c] - dt / s->m[c] * sigma * work;
        if (hg) e_new[c] -= dt / s->m[c] * work_hg;
        if (mm) {
          /* uniform strain (R18): each material takes the cell's volume
           * change in proportion to its fraction, so material k does the
           * share alpha_k (p_k + q) of the cell's sigma work; the sum over
           * k is the cell's work since sum_k alpha_k p_k = p.  The
           * hourglass forces' work, a dissipation like q's, is shared by
           * fraction too. */
          const double V0 = s->vol[c];
          double ie = 0.0;
          for (int kk = 0; kk < s->prm.nmat; ++kk) {
            const long long kc = kk * nc + c;
            const double a = s->alpha[kc];
            if (!(a > 0.0)) continue;
            const double mk = s->mm[kc];
            /* the predictor-corrector's share is that of the half step */
            const double sh = pc ? share[kc] : a * (mat_pressure(s, kk, mk / (a * V0), s->me[kc]) + s->q[c]);
            s->me[kc] -= dt / mk * (sh * work + (hg ? a * work_hg : 0.0));
            ie += mk * s->me[kc];
          }
          e_new[c] = ie / s->m[c];
        }
        if (str) {
          /* the deviatoric forces' work, then the stress at n+1 from the
           * time-centred velocity gradient and G, Y of the state at n */
          double work_s = 0.0, Lg[9] = {0.0};
          for (int a = 0; a < 8; ++a) {
            double sg[3];
            stress_apply(s, c, &G[a * 3], sg);
            work_s += dot3(sg, &UB[a * 3]);
            for (int i2 = 0; i2 < 3; ++i2)
              for (int j2 = 0; j2 < 3; ++j2) Lg[3 * i2 + j2] += UB[a * 3 + i2] * G[a * 3 + j2];
          }
          e_new[c] += dt / s->m[c] * work_s;
          for (int q9 = 0; q9 < 9; ++q9) Lg[q9] /= s->vol[c];
          double Gm, Ym, deps;
          oracle_steinberg(&s->prm, s->p[c], s->rho[c], s->e[c], s->eps_p[c], &Gm, &Ym);
          const double S6[6] = {s->sxx[c], s->syy[c], s->szz[c], s->sxy[c], s->syz[c], s->szx[c]};
          oracle_stress_update(S6, Lg, dt, Gm, Ym, &s_new[7 * c], &deps);
          s_new[7 * c + 6] = s->eps_p[c] + deps;
        }
      }

  /* Move the mesh with the time-centred velocity. */
  for (long long n = 0; n < nn; ++n) {
    s->x[n] += dt * ubx[n];
    s->y[n] += dt * uby[n];
    s->z[n] += dt * ubz[n];
  }
  memcpy(s->e, e_new, sizeof(double) * (size_t)nc);
  if (str)
    for (long long c = 0; c < nc; ++c) {
      s->sxx[c] = s_new[7 * c + 0];
      s->syy[c] = s_new[7 * c + 1];
      s->szz[c] = s_new[7 * c + 2];
      s->sxy[c] = s_new[7 * c + 3];
      s->syz[c] = s_new[7 * c + 4];
      s->szx[c] = s_new[7 * c + 5];
      s->eps_p[c] = s_new[7 * c + 6];
    }
  free(fx); free(fy); free(fz); free(ubx); free(uby); free(ubz); free(e_new); free(sig);
  free(xh); free(yh); free(zh); free(fh); free(s_new); free(meh); free(share);

  s->t += dt;
  s->dt_last = dt;
  s->cycle += 1;
  int rc = oracle_eos(s);
  if (rc) return rc;
  return propose_dt(s);
}

/* ------------------------------------------------------------------ */
/* Remap                                                               */
/* ------------------------------------------------------------------ */

/* Swept hex of a face normal to axis `ax`: local node (di,dj,dk) of the
 * hex takes the face node given by the two other bits, at the current
 * (Lagrangian) position when the bit along `ax` is 0 and at the reference
 * position when it is 1.  Its volume is positive when the reference face
 * lies on the high-index side of the current face. */
static double swept_volume(const oracle_state *s, int ax, int i, int j, int k) {
  double X[24];
  for (int a = 0; a < 8; ++a) {
    int b[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
    int ref = b[ax];
    b[ax] = 0;
    long long n = node_id(s, i + b[0], j + b[1], k + b[2]);
    X[a * 3 + 0] = ref ? s->xr[n] : s->x[n];
    X[a * 3 + 1] = ref ? s->yr[n] : s->y[n];
    X[a * 3 + 2] = ref ? s->zr[n] : s->z[n];
  }
  return oracle_hex_volume(X);
}

void oracle_swept_volumes(const oracle_state *s, double *dvx, double *dvy,
                          double *dvz) {
  const int nx = s->nx, ny = s->ny, nz = s->nz;
  /* Faces on the domain boundary are walls: no flux. */
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i <= nx; ++i)
        dvx[i + (long long)(nx + 1) * (j + (long long)ny * k)] =
            (i == 0 || i == nx) ? 0.0 : swept_volume(s, 0, i, j, k);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i < nx; ++i)
        dvy[i + (long long)nx * (j + (long long)(ny + 1) * k)] =
            (j == 0 || j == ny) ? 0.0 : swept_volume(s, 1, i, j, k);
  for (int k = 0; k <= nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        dvz[i + (long long)nx * (j + (long long)ny * k)] =
            (k == 0 || k == nz) ? 0.0 : swept_volume(s, 2, i, j, k);
}

/* Second-order cell remap (reading: van Leer 1977).  In every cell and along
 * every logical axis the density and specific energy get the limited slope
 * of van Leer: the harmonic mean of the two one-sided differences when they
 * have the same sign, else zero (also zero next to a wall, where one
 * difference is missing).  A face then carries the average of the donor's
 * linear profile q(xi) = q_d + s_d xi, xi in [-1/2, 1/2] across the donor,
 * over the slab of relative thickness nu = |dV| / V_d that the face sweeps
 * out of the donor:  q_d + side * s_d (1 - nu) / 2,  side = +1 when the
 * slab lies at the donor's high face, -1 at its low face (nu capped at 1). */
static double vanleer_slope(double dm, double dp) {
  return dm * dp > 0.0 ? 2.0 * dm * dp / (dm + dp) : 0.0;
}

static double slab_average(double q, double slope, double nu, double side) {
  return q + side * 0.5 * slope * (1.0 - (nu < 1.0 ? nu : 1.0));
}

/* Slope of field q (cells) at cell (i,j,k) along axis ax. */
static double cell_slope(const oracle_state *s, const double *q, int i, int j, int k, int ax) {
  const int n_ax = ax == 0 ? s->nx : ax == 1 ? s->ny : s->nz;
  const int idx = ax == 0 ? i : ax == 1 ? j : k;
  if (idx == 0 || idx == n_ax - 1) return 0.0;
  const int di = ax == 0, dj = ax == 1, dk = ax == 2;
  const double qm = q[cell_id(s, i - di, j - dj, k - dk)];
  const double q0 = q[cell_id(s, i, j, k)];
  const double qp = q[cell_id(s, i + di, j + dj, k + dk)];
  return vanleer_slope(q0 - qm, qp - q0);
}

/* Mass and energy flux of the face between cells lo and hi along ax with
 * swept volume dv (> 0: hi donates). */
static void face_fluxes(const oracle_state *s, const double *rho_l, const double *vol_l, int lo_i, int lo_j,
                        int lo_k, int ax, double dv, double *mu, double *eflux) {
  const int di = ax == 0, dj = ax == 1, dk = ax == 2;
  const long long lo = cell_id(s, lo_i, lo_j, lo_k), hi = cell_id(s, lo_i + di, lo_j + dj, lo_k + dk);
  const int hi_donates = dv > 0.0;
  const long long dn = hi_donates ? hi : lo;
  double rho_f = rho_l[dn], e_f = s->e[dn];
  if (s->prm.remap_order == 2) {
    const int di_ = hi_donates ? lo_i + di : lo_i, dj_ = hi_donates ? lo_j + dj : lo_j,
              dk_ = hi_donates ? lo_k + dk : lo_k;
    const double nu = fabs(dv) / vol_l[dn];
    const double side = hi_donates ? -1.0 : 1.0;
    rho_f = slab_average(rho_l[dn], cell_slope(s, rho_l, di_, dj_, dk_, ax), nu, side);
    e_f = slab_average(s->e[dn], cell_slope(s, s->e, di_, dj_, dk_, ax), nu, side);
  }
  *mu = rho_f * dv;
  *eflux = *mu * e_f;
}

/* Strength (R17): the deviatoric stress and plastic strain are carried per
 * unit mass with the face's mass flux mu from the same donor cell as e
 * (first-order donor cell): ms[7 c + q] holds m S_q (q < 6) and m eps_p. */
static void advect_strength(const oracle_state *s, double *ms, long long lo, long long hi, double mu, double dv) {
  const long long dn = dv > 0.0 ? hi : lo;
  const double q[7] = {s->sxx[dn], s->syy[dn], s->szz[dn], s->sxy[dn], s->syz[dn], s->szx[dn], s->eps_p[dn]};
  for (int k = 0; k < 7; ++k) {
    ms[7 * lo + k] += mu * q[k];
    ms[7 * hi + k] -= mu * q[k];
  }
}

/* Materials (R18): the face's swept volume dv leaves its donor (dv > 0:
 * the high cell) as each material's share of the donor: volume
 * alpha_k dv, mass (m_k / V_L) dv -- the material's partial density in
 * the Lagrangian donor -- and energy that mass times e_k.  mv, mk, me hold
 * each material's volume, mass and energy at [k * nc + c].  *mu and *ef
 * get the face's total mass and energy fluxes. */
static void mm_face(const oracle_state *s, const double *vol_l, long long lo, long long hi, double dv,
                    double *mv, double *mk, double *me, double *mu, double *ef) {
  const long long nc = s->nc, dn = dv > 0.0 ? hi : lo;
  double mu_t = 0.0, ef_t = 0.0;
  for (int k = 0; k < s->prm.nmat; ++k) {
    const long long d = k * nc + dn;
    const double vf = s->alpha[d] * dv;
    const double mf = s->mm[d] / vol_l[dn] * dv;
    const double eflux = mf * s->me[d];
    mv[k * nc + lo] += vf;
    mv[k * nc + hi] -= vf;
    mk[k * nc + lo] += mf;
    mk[k * nc + hi] -= mf;
    me[k * nc + lo] += eflux;
    me[k * nc + hi] -= eflux;
    mu_t += mf;
    ef_t += eflux;
  }
  *mu = mu_t;
  *ef = ef_t;
}

/* New material state of cell c after the fluxes (R18).  fix is the
 * kinetic energy the node remap returns to the cell, shared among the
 * materials by mass.  Donor-cell upwinding leaves geometric tails of a
 * material ahead of its front, and a fragment's specific energy is the
 * ratio of two roundoff-sized numbers: a material whose new volume is
 * at most ORACLE_ALPHA_MIN of the cell's, or whose mass or volume is not
 * positive, leaves the cell, its mass and energy going to the remaining
 * materials in proportion to their masses (the cell's mass and energy
 * stay as the fluxes left them).  The fractions are the remaining volumes
 * over their sum. */
static void mm_cell_update(oracle_state *s, long long c, const double *mv, const double *mk, const double *me,
                           double fix) {
  const long long nc = s->nc;
  const int nm = s->prm.nmat;
  double m1 = 0.0, vtot = 0.0;
  for (int k = 0; k < nm; ++k) {
    m1 += mk[k * nc + c];
    vtot += mv[k * nc + c];
  }
  int keep[ORACLE_MAX_MAT];
  double mkeep = 0.0, mdrop = 0.0, iedrop = 0.0, vkeep = 0.0;
  for (int k = 0; k < nm; ++k) {
    const long long kc = k * nc + c;
    keep[k] = mk[kc] > 0.0 && mv[kc] > ORACLE_ALPHA_MIN * vtot;
    const double ie = me[kc] + mk[kc] / m1 * fix;
    if (keep[k]) {
      mkeep += mk[kc];
      vkeep += mv[kc];
    } else {
      mdrop += mk[kc];
      iedrop += ie;
    }
  }
  double msum = 0.0, iesum = 0.0;
  for (int k = 0; k < nm; ++k) {
    const long long kc = k * nc + c;
    if (keep[k]) {
      const double w = mk[kc] / mkeep;
      const double mnew = mk[kc] + w * mdrop;
      const double ie = me[kc] + mk[kc] / m1 * fix + w * iedrop;
      s->alpha[kc] = mv[kc] / vkeep;
      s->mm[kc] = mnew;
      s->me[kc] = ie / mnew;
      msum += mnew;
      iesum += ie;
    } else {
      s->alpha[kc] = 0.0;
      s->mm[kc] = 0.0;
      s->me[kc] = 0.0;
    }
  }
  s->m[c] = msum;
  s->e[c] = iesum / msum;
}

int oracle_remap_step(oracle_state *s) {
  if (s->status) return s->status;
  const int nx = s->nx, ny = s->ny, nz = s->nz;
  const long long nc = s->nc, nn = s->nn;
  const long long nfx = (long long)(nx + 1) * ny * nz;
  const long long nfy = (long long)nx * (ny + 1) * nz;
  const long long nfz = (long long)nx * ny * (nz + 1);
  double *dvx = alloc_zero(nfx), *dvy = alloc_zero(nfy), *dvz = alloc_zero(nfz);
  double *mux = alloc_zero(nfx), *muy = alloc_zero(nfy), *muz = alloc_zero(nfz);
  double *rho_l = alloc_zero(nc), *m_new = alloc_zero(nc), *ie_new = alloc_zero(nc), *vol_l = alloc_zero(nc);
  double *mn_new = alloc_zero(nn), *px = alloc_zero(nn), *py = alloc_zero(nn);
  double *pz = alloc_zero(nn), *ke = alloc_zero(nn), *dke = alloc_zero(nn);
  const int str = strength_on(s);
  double *ms_new = alloc_zero(str ? 7 * nc : 1);
  const int mm = mm_on(s);
  if (mm && !mm_options_ok(s)) {
    free(dvx); free(dvy); free(dvz); free(mux); free(muy); free(muz); free(rho_l); free(m_new); free(ie_new);
    free(vol_l); free(mn_new); free(px); free(py); free(pz); free(ke); free(dke); free(ms_new);
    return s->status = ORACLE_EINVAL;
  }
  const long long nmc = mm ? s->prm.nmat * nc : 1;
  double *mv = alloc_zero(nmc), *mk = alloc_zero(nmc), *me = alloc_zero(nmc);
  double *all[] = {dvx, dvy, dvz, mux, muy, muz, rho_l, m_new, ie_new,
                   mn_new, px, py, pz, ke, dke, vol_l, ms_new, mv, mk, me};
  const size_t nall = sizeof(all) / sizeof(all[0]);
  for (size_t i = 0; i < nall; ++i)
    if (!all[i]) {
      for (size_t j = 0; j < nall; ++j) free(all[j]);
      return s->status = ORACLE_ENOMEM;
    }

  /* Lagrangian density of every cell (donor density). */
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long long c = cell_id(s, i, j, k);
        double X[24];
        gather_hex(s, i, j, k, s->x, s->y, s->z, X);
        vol_l[c] = oracle_hex_volume(X);
        rho_l[c] = s->m[c] / vol_l[c];
      }

  /* 1. Swept volumes of every face. */
  oracle_swept_volumes(s, dvx, dvy, dvz);

  /* 2. Donor-cell mass and energy fluxes.  dV > 0: the swept region lies
   *    in the high-index cell, which donates to the low-index one. */
  if (mm)
    for (int k = 0; k < s->prm.nmat; ++k)
      for (long long c = 0; c < nc; ++c) {
        mv[k * nc + c] = s->alpha[k * nc + c] * vol_l[c];
        mk[k * nc + c] = s->mm[k * nc + c];
        me[k * nc + c] = s->mm[k * nc + c] * s->me[k * nc + c];
      }
  for (long long c = 0; c < nc; ++c) {
    m_new[c] = s->m[c];
    ie_new[c] = s->m[c] * s->e[c];
    if (str) {
      const double q[7] = {s->sxx[c], s->syy[c], s->szz[c], s->sxy[c], s->syz[c], s->szx[c], s->eps_p[c]};
      for (int k = 0; k < 7; ++k) ms_new[7 * c + k] = s->m[c] * q[k];
    }
  }
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 1; i < nx; ++i) {
        long long f = i + (long long)(nx + 1) * (j + (long long)ny * k);
        long long lo = cell_id(s, i - 1, j, k), hi = cell_id(s, i, j, k);
        double mu, ef;
        if (mm) mm_face(s, vol_l, lo, hi, dvx[f], mv, mk, me, &mu, &ef);
        else face_fluxes(s, rho_l, vol_l, i - 1, j, k, 0, dvx[f], &mu, &ef);
        if (str) advect_strength(s, ms_new, lo, hi, mu, dvx[f]);
        mux[f] = mu;
        m_new[lo] += mu;
        m_new[hi] -= mu;
        ie_new[lo] += ef;
        ie_new[hi] -= ef;
      }
  for (int k = 0; k < nz; ++k)
    for (int j = 1; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long long f = i + (long long)nx * (j + (long long)(ny + 1) * k);
        long long lo = cell_id(s, i, j - 1, k), hi = cell_id(s, i, j, k);
        double mu, ef;
        if (mm) mm_face(s, vol_l, lo, hi, dvy[f], mv, mk, me, &mu, &ef);
        else face_fluxes(s, rho_l, vol_l, i, j - 1, k, 1, dvy[f], &mu, &ef);
        if (str) advect_strength(s, ms_new, lo, hi, mu, dvy[f]);
        muy[f] = mu;
        m_new[lo] += mu;
        m_new[hi] -= mu;
        ie_new[lo] += ef;
        ie_new[hi] -= ef;
      }
  for (int k = 1; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long long f = i + (long long)nx * (j + (long long)ny * k);
        long long lo = cell_id(s, i, j, k - 1), hi = cell_id(s, i, j, k);
        double mu, ef;
        if (mm) mm_face(s, vol_l, lo, hi, dvz[f], mv, mk, me, &mu, &ef);
        else face_fluxes(s, rho_l, vol_l, i, j, k - 1, 2, dvz[f], &mu, &ef);
        if (str) advect_strength(s, ms_new, lo, hi, mu, dvz[f]);
        muz[f] = mu;
        m_new[lo] += mu;
        m_new[hi] -= mu;
        ie_new[lo] += ef;
        ie_new[hi] -= ef;
      }

  /* 3. Node (dual-mesh) fluxes along every mesh edge (a -> b = a + e_ax).
   *    psi = sum over the cells around the edge of (mu_lo + mu_hi)/8, the
   *    quarter of the mass crossing the cell mid-plane normal to ax next
   *    to the edge.  psi > 0 moves mass from b to a.  Momentum and kinetic
   *    energy are carried with the donor node's velocity. */
  for (long long n = 0; n < nn; ++n) {
    double uu = s->u[n], vv = s->v[n], ww = s->w[n];
    mn_new[n] = s->mn[n];
    px[n] = s->mn[n] * uu;
    py[n] = s->mn[n] * vv;
    pz[n] = s->mn[n] * ww;
    ke[n] = 0.5 * s->mn[n] * (uu * uu + vv * vv + ww * ww);
  }
  for (int ax = 0; ax < 3; ++ax) {
    const int ex = ax == 0, ey = ax == 1, ez = ax == 2;
    for (int k = 0; k <= nz - ez; ++k)
      for (int j = 0; j <= ny - ey; ++j)
        for (int i = 0; i <= nx - ex; ++i) {
          /* the (up to) four cells around the edge */
          double psi = 0.0;
          for (int s1 = 0; s1 < 2; ++s1)
            for (int s2 = 0; s2 < 2; ++s2) {
              int ci = i, cj = j, ck = k;
              if (ax == 0) { cj = j - 1 + s1; ck = k - 1 + s2; }
              if (ax == 1) { ci = i - 1 + s1; ck = k - 1 + s2; }
              if (ax == 2) { ci = i - 1 + s1; cj = j - 1 + s2; }
              if (ci < 0 || ci >= nx || cj < 0 || cj >= ny || ck < 0 || ck >= nz)
                continue;
              double mu_lo, mu_hi;
              if (ax == 0) {
                mu_lo = mux[ci + (long long)(nx + 1) * (cj + (long long)ny * ck)];
                mu_hi = mux[ci + 1 + (long long)(nx + 1) * (cj + (long long)ny * ck)];
              } else if (ax == 1) {
                mu_lo = muy[ci + (long long)nx * (cj + (long long)(ny + 1) * ck)];
                mu_hi = muy[ci + (long long)nx * (cj + 1 + (long long)(ny + 1) * ck)];
              } else {
                mu_lo = muz[ci + (long long)nx * (cj + (long long)ny * ck)];
                mu_hi = muz[ci + (long long)nx * (cj + (long long)ny * (ck + 1))];
              }
              psi += (mu_lo + mu_hi) / 8.0;
            }
          long long a = node_id(s, i, j, k);
          long long b = node_id(s, i + ex, j + ey, k + ez);
          long long dn = psi > 0.0 ? b : a;
          double ud = s->u[dn], vd = s->v[dn], wd = s->w[dn];
          double kd = 0.5 * (ud * ud + vd * vd + wd * wd);
          mn_new[a] += psi;
          mn_new[b] -= psi;
          px[a] += psi * ud;
          px[b] -= psi * ud;
          py[a] += psi * vd;
          py[b] -= psi * vd;
          pz[a] += psi * wd;
          pz[b] -= psi * wd;
          ke[a] += psi * kd;
          ke[b] -= psi * kd;
        }
  }

  /* 4. New node velocity (walls reflect), and the kinetic energy that the
   *    momentum remap did not keep. */
  for (int k = 0; k <= nz; ++k)
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i <= nx; ++i) {
        long long n = node_id(s, i, j, k);
        double uu = px[n] / mn_new[n], vv = py[n] / mn_new[n], ww = pz[n] / mn_new[n];
        apply_wall_bc(s, i, j, k, &uu, &vv, &ww);
        dke[n] = ke[n] - 0.5 * mn_new[n] * (uu * uu + vv * vv + ww * ww);
        s->u[n] = uu;
        s->v[n] = vv;
        s->w[n] = ww;
        s->mn[n] = mn_new[n];
      }

  /* 5. Kinetic-energy fix: each node's lost KE goes in equal shares to
   *    the internal energy of the cells around it (with materials, shared
   *    among the cell's materials in step 6). */
  if (s->prm.ke_fix && !mm)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          long long c = cell_id(s, i, j, k);
          for (int a = 0; a < 8; ++a) {
            int ni = i + (a & 1), nj = j + ((a >> 1) & 1), nk = k + ((a >> 2) & 1);
            ie_new[c] += dke[node_id(s, ni, nj, nk)] / node_cell_count(s, ni, nj, nk);
          }
        }

  /* 6. New cell state on the reference mesh. */
  if (mm)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          long long c = cell_id(s, i, j, k);
          double fix = 0.0;
          if (s->prm.ke_fix)
            for (int a = 0; a < 8; ++a) {
              int ni = i + (a & 1), nj = j + ((a >> 1) & 1), nk = k + ((a >> 2) & 1);
              fix += dke[node_id(s, ni, nj, nk)] / node_cell_count(s, ni, nj, nk);
            }
          mm_cell_update(s, c, mv, mk, me, fix);
        }
  for (long long c = 0; c < nc && !mm; ++c) {
    s->m[c] = m_new[c];
    s->e[c] = ie_new[c] / m_new[c];
    if (str) {
      double *q[7] = {s->sxx, s->syy, s->szz, s->sxy, s->syz, s->szx, s->eps_p};
      for (int k = 0; k < 7; ++k) q[k][c] = ms_new[7 * c + k] / m_new[c];
    }
  }
  memcpy(s->x, s->xr, sizeof(double) * (size_t)nn);
  memcpy(s->y, s->yr, sizeof(double) * (size_t)nn);
  memcpy(s->z, s->zr, sizeof(double) * (size_t)nn);
  for (size_t i = 0; i < nall; ++i) free(all[i]);

  int rc = oracle_eos(s);
  if (rc) return rc;
  return propose_dt(s);
}

/* ------------------------------------------------------------------ */
/* Driver and diagnostics                                              */
/* ------------------------------------------------------------------ */

int oracle_run(oracle_state *s, double t_end, long long max_cycles,
               int remap_every, long long *done) {
  long long n = 0;
  while (n < max_cycles && s->t < t_end && s->status == ORACLE_OK) {
    double dt = s->dt;
    int clamp = 0;
    if (t_end - s->t < dt) {
      dt = t_end - s->t;
      clamp = 1;
    }
    int rc = oracle_lagrange_step(s, dt);
    if (rc) break;
    if (clamp) s->t = t_end;
    if (remap_every > 0 && s->cycle % remap_every == 0) {
      rc = oracle_remap_step(s);
      if (rc) break;
    }
    ++n;
  }
  if (done) *done = n;
  return s->status;
}

void oracle_diagnostics(const oracle_state *s, double *out) {
  double mass = 0, mx = 0, my = 0, mz = 0, ie = 0, ke = 0;
  for (long long c = 0; c < s->nc; ++c) {
    mass += s->m[c];
    ie += s->m[c] * s->e[c];
  }
  for (long long n = 0; n < s->nn; ++n) {
    mx += s->mn[n] * s->u[n];
    my += s->mn[n] * s->v[n];
    mz += s->mn[n] * s->w[n];
    ke += 0.5 * s->mn[n] * (s->u[n] * s->u[n] + s->v[n] * s->v[n] + s->w[n] * s->w[n]);
  }
  out[0] = mass;
  out[1] = mx;
  out[2] = my;
  out[3] = mz;
  out[4] = ie;
  out[5] = ke;
  out[6] = ie + ke;
}
