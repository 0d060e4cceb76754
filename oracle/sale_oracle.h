/*
 * sale_oracle.h -- plain serial FP64 reference of the SALE staggered-grid
 * hydro cycle (ScalSALE, arXiv 2209.01983: SALE scheme of Sec. I-D, the
 * Lagrangian/Eulerian rezoning + advection rows of Table I, Sec. IV).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this library.  It shares no code
 * with the CUDA library; it is slow on purpose and is never tuned.
 *
 * The paper names the scheme (SALE, Amsden-Ruppel-Hirt) but prints none of
 * its formulas.  Every formula below is a standard published form, written
 * out in full in sale_oracle.c next to the loop that evaluates it:
 *   - hex volume: exact trilinear-hex volume, as the divergence-theorem sum
 *     over the six faces, each face fanned into four triangles from its
 *     node mean;
 *   - compatible energy update (Caramana, Burton, Shashkov, Whalen 1998),
 *     single stage or with a midpoint predictor for second order in time;
 *   - optional viscous hourglass control (Flanagan, Belytschko, "A uniform
 *     strain hexahedron and quadrilateral with orthogonal hourglass
 *     control", IJNME 17, 1981);
 *   - donor-cell (upwind) remap of mass, energy, momentum (Amsden et al.
 *     1980, "SALE"), with kinetic-energy fix-up;
 *   - optionally, second-order cell remap: van Leer's limited
 *     piecewise-linear profile in the donor cell (van Leer 1977, "Towards
 *     the ultimate conservative difference scheme IV"), averaged over the
 *     slab the face sweeps;
 *   - optionally, material strength, the stress module of the paper's
 *     case study (Sec. III-D): deviatoric stress with the Jaumann rate and
 *     von Mises radial return (Wilkins 1963, "Calculation of elastic-plastic
 *     flow"), shear modulus and yield from the Steinberg-Guinan model
 *     (Steinberg, Cochran, Guinan, J. Appl. Phys. 51, 1980);
 *   - optionally, several materials with their own equations of state (the
 *     multi-material SALE scheme of Sec. I-D and Table I): per-material
 *     volume fraction, mass and energy in every cell; stiffened-gas EoS
 *     (ideal gas when p_inf = 0); mixed cells closed by uniform strain (the
 *     materials of a cell share its volume change, so the fractions do not
 *     change in the Lagrangian phase; one of the closures surveyed by
 *     Benson, "Computational methods in Lagrangian and Eulerian
 *     hydrocodes", CMAME 99, 1992), cell
 *     pressure sum_k alpha_k p_k; donor-cell remap of each material's
 *     volume, mass and energy.
 *
 * Layout: SoA, x index fastest.  Cell c = i + nx*(j + ny*k); node
 * n = i + (nx+1)*(j + (ny+1)*k).  Local node a = di + 2*dj + 4*dk of cell
 * (i,j,k) is node (i+di, j+dj, k+dk).
 */
#ifndef SALE_ORACLE_H
#define SALE_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORACLE_OK = 0,
  ORACLE_EINVAL = -1,
  ORACLE_ENOMEM = -2,
  ORACLE_ENEGVOL = -4,
  ORACLE_EDT = -5,
  ORACLE_ENAN = -6
};

typedef struct oracle_params {
  double gamma;      /* ideal-gas ratio of specific heats                 */
  double cfl;        /* Courant number                                    */
  double c_q;        /* quadratic artificial-viscosity coefficient        */
  double c_l;        /* linear artificial-viscosity coefficient           */
  double dt_growth;  /* max ratio dt_{n+1}/dt_n                           */
  double dt_init;    /* cap on the first dt (<=0 or inf: none)            */
  int ke_fix;        /* 1: remap returns lost kinetic energy to cells     */
  int reflect[6];    /* x-lo,x-hi,y-lo,y-hi,z-lo,z-hi: 1 = reflecting wall */
  int remap_order;   /* cell remap: 2 = van Leer piecewise linear, else first-order donor cell */
  int time_order;    /* Lagrange step: 2 = predictor-corrector, else single stage */
  double c_hg;       /* Flanagan-Belytschko viscous hourglass coefficient (0: none) */
  /* Material strength (Steinberg-Guinan shear modulus and yield, Wilkins
   * deviatoric stress); shear0 = 0: none, the pure hydro scheme.          */
  double shear0;     /* G0, shear modulus at the reference state          */
  double shear_dp;   /* dG/dp                                             */
  double shear_dt;   /* dG/dT                                             */
  double cv;         /* specific heat: T - T_ref = (e - e_ref) / cv       */
  double e_ref;      /* specific internal energy at the reference T       */
  double rho_ref;    /* reference density                                 */
  double yield0;     /* Y0                                                */
  double yield_max;  /* Ymax                                              */
  double hard_beta;  /* work-hardening coefficient beta                   */
  double hard_n;     /* work-hardening exponent n                         */
  /* Materials: nmat <= 1 is the single ideal gas of `gamma` above; with
   * 2 <= nmat <= ORACLE_MAX_MAT every cell holds per-material fractions
   * and material k has the stiffened-gas EoS (mat_gamma[k], mat_pinf[k]). */
  int nmat;
  double mat_gamma[4];
  double mat_pinf[4];
} oracle_params;

#define ORACLE_MAX_MAT 4
/* a material whose volume fraction falls to this or below in a remap
 * leaves the cell (its mass and energy go to the cell's other materials) */
#define ORACLE_ALPHA_MIN 1e-8

typedef struct oracle_state {
  int nx, ny, nz;
  long long nc, nn;
  oracle_params prm;
  double *x, *y, *z;       /* node position                                */
  double *xr, *yr, *zr;    /* reference mesh = Eulerian rezone target      */
  double *u, *v, *w;       /* node velocity                                */
  double *mn;              /* node mass                                    */
  double *m, *e;           /* cell mass, specific internal energy          */
  double *vol, *rho, *p, *q, *cs, *len; /* derived cell quantities         */
  double *sxx, *syy, *szz, *sxy, *syz, *szx; /* deviatoric stress (strength) */
  double *eps_p;           /* equivalent plastic strain (strength)         */
  double t, dt, dt_last;   /* time, proposed next dt, last dt used         */
  long long cycle;
  int status;
  /* materials (nmat >= 2): volume fraction, mass and specific internal
   * energy of material k in cell c at [k * nc + c]; m and e above are the
   * cell totals sum_k m_k and sum_k m_k e_k / m */
  double *alpha, *mm, *me;
} oracle_state;

/* ---- single-hex geometry; X[a*3+d] = coordinate d of local node a ---- */
double oracle_hex_volume(const double *X);
void oracle_hex_volume_grad(const double *X, double *G); /* G[a*3+d] = dV/dX */
/* face vector areas A[f*3+d], faces ordered x-lo,x-hi,y-lo,y-hi,z-lo,z-hi */
void oracle_hex_face_areas(const double *X, double *A);
double oracle_hex_char_length(const double *X);

/* ---- material strength (single cell) ----
 * Steinberg-Guinan shear modulus G and yield stress Y of a cell with EoS
 * pressure p, density rho, specific energy e, plastic strain eps_p. */
void oracle_steinberg(const oracle_params *prm, double p, double rho, double e, double eps_p, double *G,
                      double *Y);
/* Wilkins deviatoric stress update with von Mises radial return.  S[6] =
 * (xx, yy, zz, xy, yz, zx), L[9] the velocity gradient L[3*i + j] =
 * du_i/dx_j; S_out gets the new stress, *deps the plastic strain added. */
void oracle_stress_update(const double *S, const double *L, double dt, double G, double Y, double *S_out,
                          double *deps);

/* ---- state ---- */
oracle_state *oracle_create(int nx, int ny, int nz, const double *xn,
                            const double *yn, const double *zn,
                            const oracle_params *prm);
void oracle_destroy(oracle_state *s);
/* Initial state from per-cell primitive rho0, p0 (u = 0).  If
 * deposit_cell >= 0 its specific energy is replaced by
 * deposit_energy / m_cell.  Computes derived fields and the first dt. */
int oracle_init_prim(oracle_state *s, const double *rho0, const double *p0,
                     long long deposit_cell, double deposit_energy);
/* Overwrite the evolving fields (positions, velocities, node mass, cell
 * mass, energy, time and last dt), then recompute derived fields and the
 * proposed dt.  Used to restart the oracle from an arbitrary state.  The
 * deviatoric stress and plastic strain (strength) are kept as they are. */
int oracle_set_state(oracle_state *s, const double *x, const double *y,
                     const double *z, const double *u, const double *v,
                     const double *w, const double *mn, const double *m,
                     const double *e, double t, double dt_last);
/* Multi-material initial state (nmat >= 2): cell c is pure material
 * mat[c] with primitive rho0, p0, its specific energy from that
 * material's EoS; the deposit as in oracle_init_prim.  EINVAL for a
 * material index out of range, an invalid EoS, or an option the
 * multi-material scheme does not take (strength, second-order remap). */
int oracle_init_materials(oracle_state *s, const double *rho0, const double *p0, const int *mat,
                          long long deposit_cell, double deposit_energy);
/* Overwrite the per-material fields ([k * nc + c] layout), recompute the
 * cell totals m and e, the derived fields and the proposed dt.  Each cell
 * needs alpha_k >= 0 summing to 1 (to 1e-12), m_k >= 0, and alpha_k > 0
 * exactly where m_k > 0; EINVAL otherwise. */
int oracle_set_materials(oracle_state *s, const double *alpha, const double *mm, const double *me);
int oracle_eos(oracle_state *s);            /* vol, rho, p, cs, q, len     */
double oracle_cfl_dt(const oracle_state *s); /* min over cells (uses eos)  */

/* One Lagrangian step with the given dt (> 0); then eos and dt proposal. */
int oracle_lagrange_step(oracle_state *s, double dt);
/* Eulerian rezone to the reference mesh + donor-cell advection; then eos
 * and dt proposal. */
int oracle_remap_step(oracle_state *s);
/* Signed swept volumes of every face between the current and reference
 * mesh.  dvx has (nx+1)*ny*nz entries (index i + (nx+1)*(j + ny*k)),
 * dvy nx*(ny+1)*nz (i + nx*(j + (ny+1)*k)), dvz nx*ny*(nz+1). */
void oracle_swept_volumes(const oracle_state *s, double *dvx, double *dvy,
                          double *dvz);
/* Cycles until t >= t_end or max_cycles; remap after every remap_every-th
 * cycle (0 = never).  Returns status; *done = cycles run. */
int oracle_run(oracle_state *s, double t_end, long long max_cycles,
               int remap_every, long long *done);
/* out: mass, mom_x, mom_y, mom_z, internal E, kinetic E, total E */
void oracle_diagnostics(const oracle_state *s, double *out);

#ifdef __cplusplus
}
#endif
#endif
