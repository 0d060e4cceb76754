/*
 * sale.h -- C ABI of the GB300 SALE hydro library (libsale_gb300.so).
 *
 * The library advances the staggered-grid hydrodynamics cycle of the SALE
 * scheme on a structured hexahedral mesh, on one GPU, in hand-written
 * sm_103a CUDA kernels.  ScalSALE (arXiv 2209.01983) defines the problem:
 * 3D structured grid (Table I "Mesh: Structured"), ideal-gas equation of
 * state (Sec. I-D), the SALE hydrodynamic scheme (Sec. I-D), Lagrangian and
 * Eulerian rezoning with an advection phase (Table I "Numerical kernels";
 * Sec. IV), slip (reflecting) cell boundary conditions per mesh edge
 * (Sec. III-A, Polymorphism), and the Sod and Sedov-Taylor problems
 * (Sec. I-D, Sec. IV).  The paper prints no equations; the library
 * implements these standard forms:
 *
 *   EoS            p = (gamma-1) rho e,  cs^2 = gamma (gamma-1) max(e,0)
 *   viscosity      q = rho (c_q (L div)^2 + c_l cs L |div|) when div < 0
 *   corner force   F_a = sum_c (p_c + q_c) dV_c/dx_a   (node gather)
 *   kinematics     u+ = u + dt F/m_n;  x+ = x + dt (u + u+)/2
 *   energy         e+ = e - dt/m_c (p+q) sum_a dV_c/dx_a . (u_a + u+_a)/2
 *   time step      dt = min(cfl min_c L_c / sqrt(cs^2 + 2q/rho), g dt_prev)
 *   remap          donor-cell advection of mass, internal energy, node
 *                  momentum and kinetic energy to the reference mesh
 *
 * Conventions
 *  - Every call returns a sale_status (0 = OK, negative = error) and never
 *    aborts the process.  sale_last_error() gives a message for the last
 *    non-OK status of the calling thread.
 *  - Device errors (non-positive volume, NaN, dt underflow, wait timeout)
 *    are recorded in a status word on the GPU and reported by the next call
 *    that synchronises (run_to_time, diagnostics, copy_field).  After that
 *    the state refuses further steps (SALE_ESTATE).
 *  - Field memory belongs to the caller: sale_state_bytes() says how much
 *    device memory a state needs; sale_state_init() carves it out of the
 *    caller's buffer, which must stay alive until sale_state_destroy().
 *    Handles (mesh/state metadata) belong to the library.
 *  - A state runs on the CUDA stream given at init; handles are not
 *    thread-safe.
 *  - Layout: structure of arrays, x index fastest.  Cell (i,j,k) is
 *    c = i + nx*(j + ny*k); node (i,j,k) is n = i + (nx+1)*(j + (ny+1)*k).
 */
#ifndef SALE_H
#define SALE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SALE_OK = 0,
  SALE_EINVAL = -1,   /* bad argument                                  */
  SALE_ENOMEM = -2,   /* host allocation failed or device buffer small */
  SALE_ECUDA = -3,    /* CUDA runtime error                            */
  SALE_ENEGVOL = -4,  /* a cell volume became non-positive (tangling)  */
  SALE_EDT = -5,      /* time step not positive / not finite           */
  SALE_ENAN = -6,     /* NaN in a field                                */
  SALE_ETIMEOUT = -7, /* a bounded device-side wait ran out            */
  SALE_ESTATE = -8    /* state is in an error state or wrong mode      */
} sale_status;

typedef enum {
  SALE_FP64 = 0,       /* FP64 storage and arithmetic                   */
  SALE_FP32_MIXED = 1  /* FP32 storage, FP64 volumes/energy/sums        */
} sale_precision;

enum { SALE_PROB_SOD_X = 0, SALE_PROB_SEDOV = 1, SALE_PROB_UNIFORM = 2 };

typedef struct sale_mesh sale_mesh;
typedef struct sale_state sale_state;

/* Structured mesh on the box [lo, hi].  Node (i,j,k) sits at
 * lo + (i,j,k) * h with h = (hi - lo) / (nx,ny,nz), plus, when jitter > 0,
 * an offset ((2u - 1) * jitter) * h per axis, u = top 53 bits of the
 * SplitMix64 draw number 3*node + axis of stream `seed` divided by 2^53.
 * Nodes get no offset normal to a boundary plane they lie on.
 * reflect[6] (x-lo, x-hi, y-lo, y-hi, z-lo, z-hi) must all be 1: every wall
 * is a reflecting (slip / symmetry) plane. */
typedef struct {
  int nx, ny, nz;
  double lo[3], hi[3];
  double jitter;
  unsigned long long seed;
  int reflect[6];
} sale_mesh_desc;

/* Initial state and scheme parameters.
 *  SOD_X:   cell on the left state (rho_l, p_l) when its logical centre
 *           lo_x + (i + 0.5) h_x < x_split, else (rho_r, p_r).
 *  SEDOV:   background (rho_bg, p_bg); the origin cell (0,0,0) gets the
 *           specific energy e_deposit / m_cell when e_deposit > 0, else the
 *           primitive state (rho_blast, p_blast).
 *  UNIFORM: (rho_bg, p_bg) everywhere.
 * Velocities start at zero.  cfl: Courant number; c_q, c_l: quadratic and
 * linear viscosity coefficients; dt_init: cap on the first step (<= 0 or
 * inf: none); dt_growth: max ratio of successive steps; ke_fix: return the
 * kinetic energy lost in the momentum remap to the cells (1) or not (0);
 * remap_order: cell remap of density and specific energy, 1 (or 0) the
 * first-order donor cell, 2 van Leer's limited piecewise-linear profile in
 * the donor averaged over the swept slab (the node remap stays donor
 * node); time_order: Lagrangian step, 1 (or 0) single stage with the
 * corner forces of x^n, 2 predictor-corrector: a half step to
 * x^n + dt/2 u^n gives sigma^{n+1/2}, and the corner forces there move the
 * nodes and update the energy (second order in time, energy exact);
 * c_hg: viscous hourglass control (Flanagan-Belytschko) with corner forces
 * -c_hg rho cs V^(2/3) sum_alpha gamma_alpha (gamma_alpha . u) from the
 * start of the step, in both the velocity and the energy update (0: none).
 * Material strength, the stress module of ScalSALE's case study (Sec.
 * III-D; shear0 = 0: none, the pure hydro scheme; FP64 states, single-stage
 * step): a deviatoric stress S per cell, advanced by the Jaumann rate with
 * von Mises radial return (Wilkins 1963) from the time-centred velocity
 * gradient; shear modulus and yield from the Steinberg-Guinan model,
 * G = shear0 + shear_dp p (rho_ref / rho)^(1/3) + shear_dt (e - e_ref) / cv
 * (clamped at 0) and Y = min(yield0 (1 + hard_beta eps_p)^hard_n,
 * yield_max) G / shear0; the corner forces gain -S dV/dx_a (velocity and
 * energy update alike, so total energy stays exact), the CFL speed
 * 4 G / (3 rho), and the remap carries S and the plastic strain eps_p per
 * unit mass with the donor cell's mass flux.  The fields "sxx", "syy",
 * "szz", "sxy", "syz", "szx" and "eps_p" then exist.
 * Materials, the multi-material scheme of ScalSALE (Sec. I-D, Table I:
 * "multi-material, multiple EoS"; nmat = 0 or 1: one ideal gas of
 * `gamma`).  With 2 <= nmat <= SALE_MAX_MAT (FP64 states; first-order
 * remap, no strength) material k has
 * the stiffened-gas EoS p = (mat_gamma[k] - 1) rho e - mat_gamma[k]
 * mat_pinf[k] (mat_pinf[k] = 0: ideal gas; `gamma` is unused) and every
 * cell holds each material's volume fraction alpha_k, mass m_k and
 * specific energy e_k.  Initially a cell is pure: material 1 where its
 * logical centre lo_x + (i + 0.5) h_x >= x_split (the right state of
 * SOD_X), material 0 elsewhere, its e_k from its own EoS at the cell's
 * (rho, p).  Mixed cells are closed by uniform strain: the materials share
 * the cell's volume change in proportion to their fractions, so the
 * fractions do not change in the Lagrangian step, and material k takes the
 * share alpha_k (p_k + q) of the cell's compatible work; the cell pressure
 * is sum_k alpha_k p_k(m_k / (alpha_k V), e_k), its sound speed squared
 * sum_k m_k c_k^2 / m with c_k^2 = gamma_k (gamma_k - 1) (e_k - p_inf_k /
 * rho_k) floored at 0.  The remap moves each material's volume
 * (alpha_k dV), mass ((m_k / V_L) dV) and energy (mass times e_k) out of
 * the donor of every face, shares the cell's kinetic-energy fix by mass,
 * and drops a material whose new fraction is at most SALE_MAT_ALPHA_MIN
 * (its mass and energy go to the cell's other materials by mass).  With
 * hourglass control the materials share its work by fraction and its
 * coefficient takes the mixture's sound speed; with the predictor-corrector
 * each material's half step follows from its share of the predictor's work
 * and its half-step share alpha_k (p_k + q) enters the corrector.  Fields
 * "alpha<k>", "m<k>", "e<k>" (k = 0 .. nmat-1) then exist; "m" and "e"
 * are the cell totals sum_k m_k and sum_k m_k e_k / m.
 * Options other than the defaults may need more device memory: size the
 * buffer with sale_state_bytes_for().  Batches take only the default
 * time_order, c_hg, shear0 and nmat. */
typedef struct {
  int kind;
  double gamma;
  double rho_l, p_l, rho_r, p_r, x_split;
  double rho_bg, p_bg, rho_blast, p_blast, e_deposit;
  double cfl, c_q, c_l, dt_init, dt_growth;
  int ke_fix;
  int remap_order;
  int time_order;
  double c_hg;
  double shear0, shear_dp, shear_dt, cv, e_ref, rho_ref;
  double yield0, yield_max, hard_beta, hard_n;
  int nmat;
  double mat_gamma[4], mat_pinf[4];
} sale_problem_desc;

#define SALE_MAX_MAT 4
#define SALE_MAT_ALPHA_MIN 1e-8

/* Diagnostics (FP64 sums in a fixed reduction order). */
typedef struct {
  double t;        /* simulated time                                    */
  double dt;       /* proposed next time step                           */
  long long cycle; /* Lagrangian steps taken                            */
  double mass;     /* sum_c m_c                                         */
  double mom[3];   /* sum_n m_n u_n                                     */
  double ie;       /* sum_c m_c e_c                                     */
  double ke;       /* sum_n m_n |u_n|^2 / 2                             */
  double etot;     /* ie + ke                                           */
  int status;      /* device status word (sale_status)                  */
} sale_diag;

/* Build the mesh (host coordinates, library-owned).  EINVAL for sizes < 1,
 * hi <= lo, jitter outside [0, 0.45], non-reflecting walls. */
int sale_mesh_create(const sale_mesh_desc *desc, sale_mesh **out);
void sale_mesh_destroy(sale_mesh *mesh);
/* Host copy of the mesh node coordinates: xyz holds 3 * nnodes doubles,
 * all x, then all y, then all z. */
int sale_mesh_nodes(const sale_mesh *mesh, double *xyz, size_t n);

/* Device bytes a state of this mesh and precision needs with the default
 * scheme options (0 on bad args, and for FP32-mixed meshes of more than
 * 2^31 - 1 nodes, which its 32-bit indexing does not reach). */
size_t sale_state_bytes(const sale_mesh *mesh, int precision);
/* Device bytes for this mesh, problem and precision: includes the scratch
 * of the second-order remap (FP64), of the predictor-corrector step
 * (half-step corner gradients), of the hourglass control (corner forces),
 * of material strength (stress, plastic strain, G, Y and the remap's copy)
 * and of several materials (each material's fraction, mass and energy, its
 * face fluxes, 1 / V_L, and with the predictor-corrector its half-step
 * share of sigma) when the problem asks for them. */
size_t sale_state_bytes_for(const sale_mesh *mesh, const sale_problem_desc *prob, int precision);
/* Initialise a state in the caller's device buffer (>= sale_state_bytes_for,
 * 256-byte aligned) on `cuda_stream` (a cudaStream_t; NULL = legacy
 * default stream).  Computes volumes, masses, energies, node masses, the
 * EoS/viscosity state and the first dt.  The mesh may be destroyed after. */
int sale_state_init(const sale_mesh *mesh, const sale_problem_desc *prob,
                    int precision, void *device_buf, size_t bytes,
                    void *cuda_stream, sale_state **out);
void sale_state_destroy(sale_state *st);

/* One Lagrangian step (force gather, velocity/position update, compatible
 * energy update, new EoS/viscosity state, next dt).  dt > 0 uses that
 * step; dt <= 0 uses the on-device CFL step.  Asynchronous. */
int sale_lagrange_step(sale_state *st, double dt);
/* Eulerian rezone to the initial mesh plus donor-cell advection of mass,
 * energy, momentum and kinetic energy (Table I "Eulerian rezoning,
 * Advection"); then EoS/viscosity state and next dt.  Asynchronous. */
int sale_remap_step(sale_state *st);
/* Cycle until t >= t_end or max_cycles cycles: each cycle is a Lagrangian
 * step with the on-device dt (clamped to land on t_end) followed by a remap
 * when remap_every > 0 and the cycle count is a multiple of it.  Runs as
 * replays of a captured CUDA graph; synchronises; *cycles_done (may be
 * NULL) gets the number of cycles run. */
int sale_run_to_time(sale_state *st, double t_end, long long max_cycles,
                     int remap_every, long long *cycles_done);
/* Synchronising FP64 reductions of the conserved quantities. */
int sale_diagnostics(const sale_state *st, sale_diag *out);

/* Synchronising copy of a field to host FP64.  Names: node fields "x",
 * "y", "z", "u", "v", "w", "mn", "xref", "yref", "zref" (n = nnodes); cell
 * fields "m", "e", "rho", "p", "q", "cs", "vol" (n = ncells), and with
 * materials "alpha<k>", "m<k>", "e<k>".  FP32-mixed fields are widened on
 * the device (hi + lo for the float-float m, e, mn); FP64 "cs" of a
 * single-material state is formed from e as sqrt(gamma (gamma - 1)
 * max(e, 0)), the formula the kernels use. */
int sale_copy_field(const sale_state *st, const char *name, double *host_out,
                    size_t n);
/* Overwrite an evolving field from host FP64 (same names as copy_field for
 * "x","y","z","u","v","w","mn","m","e", and with materials "alpha<k>",
 * "m<k>", "e<k>" in place of "m" and "e"); call sale_refresh() after the
 * last one to recompute derived fields and dt (with materials, refresh
 * first forms the cell totals m and e from the material fields; each cell
 * must have fractions >= 0 summing to 1 and alpha_k > 0 exactly where
 * m_k > 0, which is not checked).  FP32-mixed states split each
 * value on the device into hi = fl32(x) and, for m, e and mn, lo =
 * fl32(x - hi).  Asynchronous with respect to the host only when host_in is
 * pinned memory (which must then stay unchanged until the state's stream
 * has passed the copy). */
int sale_set_field(sale_state *st, const char *name, const double *host_in,
                   size_t n);
int sale_refresh(sale_state *st);

/* Sizes of a state: ncells, nnodes. */
int sale_state_dims(const sale_state *st, long long *ncells, long long *nnodes);

/* Remap step without any device allocation.  The paper has no counterpart
 * of this call; it serves callers that cannot allocate device memory:
 * plug-ins whose host program owns every device allocation and hands them
 * only their field arrays, and loops that must not call an allocator
 * (cudaMalloc and cudaFree can synchronise the device).  It does what
 * sale_remap_step does -- face swept volumes, donor-cell mass and energy
 * fluxes, dual-mesh node momentum and kinetic-energy fluxes, new node
 * velocity and mass, cell mass and energy with the kinetic-energy fix --
 * on a mesh held entirely in the caller's device arrays (FP64, SoA, layout
 * as above), without EoS or dt.  Arguments:
 *   nx, ny, nz   cells per axis; at most SALE_STATIC_MAX_CELLS cells and
 *                SALE_STATIC_MAX_NODES nodes, else SALE_EINVAL
 *   reflect[6]   host array, 1 = reflecting wall (x-lo,x-hi,..,z-hi), 0 = none
 *   ke_fix       return the remap's kinetic-energy loss to the cells (1)
 *   xref         3*nnodes reference (rezone target) positions, x then y then z
 *   x            3*nnodes Lagrangian positions in; the reference positions out
 *   u_in         3*nnodes node velocity before the remap (not modified)
 *   u_out        3*nnodes node velocity after the remap (must not alias u_in)
 *   mn           nnodes node mass, in/out
 *   m, e         ncells cell mass and specific internal energy, in/out
 *   rho          ncells cell density on the Lagrangian mesh, m / V(x)
 *   cuda_stream  stream to run on (NULL = legacy default stream)
 * Scratch (status word, face fluxes, node energy losses) lives in one fixed
 * static device array of the library (about 4 MB at the limits below),
 * present on every GPU that loads the library until the process exits.
 * Every call shares it and it keeps the last call's contents (the status
 * word is cleared at the start of each call; the flux arrays are written in
 * full before they are read), so calls that overlap on the GPU (other
 * streams, other host threads) race: serialise them.  The first call on a
 * device looks up the array's device address (and may load the library's
 * GPU code); make that first call before any stream capture.  After a
 * device reset (cudaDeviceReset) that address is stale: do not call this
 * entry point again in a process that has reset the device.  Calls no
 * device or host allocator.  Synchronises the stream and returns the
 * device status (SALE_ENEGVOL when a node or cell mass is not positive). */
#define SALE_STATIC_MAX_CELLS 65536
#define SALE_STATIC_MAX_NODES 131072
int sale_remap_static(int nx, int ny, int nz, const int *reflect, int ke_fix,
                      const double *xref, double *x, const double *u_in,
                      double *u_out, double *mn, double *m, double *e,
                      const double *rho, void *cuda_stream);

/* Batches: n independent meshes (each its own problem, size and dt)
 * advanced together.  Every cycle of every mesh runs in the same five
 * kernel launches (a block-to-mesh table maps each block to its mesh), and
 * a sale_batch_run replays captured CUDA graphs of up to 64 cycles of
 * every mesh (at most 64 graphs are kept per batch).  Batches run the
 * FP32-mixed Eulerian cycle (precision SALE_FP32_MIXED, remap every
 * cycle).  Memory: sale_batch_bytes() bytes of caller device memory
 * (256-byte aligned), alive until sale_batch_destroy(); meshes[i] follow
 * the sale_mesh_desc rules, probs[i] the sale_problem_desc rules; the
 * stream must not be the legacy default stream. */
typedef struct sale_batch sale_batch;
size_t sale_batch_bytes(int n, const sale_mesh_desc *meshes, int precision);
int sale_batch_create(int n, const sale_mesh_desc *meshes,
                      const sale_problem_desc *probs, int precision,
                      void *device_buf, size_t bytes, void *cuda_stream,
                      sale_batch **out);
/* Advance every mesh by `cycles` cycles, each with its own on-device dt;
 * remap_every must be 1.  Synchronises; reports the first mesh with a
 * device error.  *cycles_done (may be NULL) gets the cycles run. */
int sale_batch_run(sale_batch *b, long long cycles, int remap_every,
                   long long *cycles_done);
/* Borrowed handle of mesh i (diagnostics, copy_field, set_field, refresh,
 * run_to_time); valid until sale_batch_destroy().  NULL when out of range. */
sale_state *sale_batch_state(sale_batch *b, int i);
void sale_batch_destroy(sale_batch *b);

/* Tuning knobs of the FP32-mixed kernels (no effect on results: every
 * thread's work is independent of the tiling and the dt minimum is exact).
 * Shapes 0..4 are thread tiles of tx x ty threads over one k plane:
 * (32,8), (32,4), (64,4), (128,2), (16,8).  sale_set_tiling applies to an
 * FP32-mixed state (EINVAL otherwise); sale_batch_set_schedule sets the
 * shape of a batch and the order of its meshes' tiles in a launch
 * (0: input order, 1: largest mesh first).  Both synchronise and drop
 * captured graphs. */
int sale_tile_shape(int shape, int *tx, int *ty);
int sale_set_tiling(sale_state *st, int shape);
int sale_batch_set_schedule(sale_batch *b, int shape, int order);

/* Launch-time profile.  While on, every kernel launch of the state's steps
 * is bracketed by CUDA events on the state's stream (inside captured
 * graphs as event nodes); device times accumulate on the host at each
 * synchronising call.  sale_profile_read() synchronises, copies the
 * per-kernel totals (milliseconds, launches) for kernel ids [0, n) and
 * optionally resets them.  Kernel ids name the kernels of the cycle in
 * sale_kernel_name(id), 0 <= id < sale_kernel_count(). */
int sale_profile(sale_state *st, int on);
int sale_profile_read(sale_state *st, double *ms, long long *launches, int n,
                      int reset);
int sale_kernel_count(void);
const char *sale_kernel_name(int id);

/* Measured fused multiply-add rate of the current GPU, for the roofline of
 * the FP64 cycle (which is bound by the FP64 vector pipe rather than by
 * HBM).  The paper has no counterpart of this call.  precision SALE_FP64
 * times FP64 FMAs, SALE_FP32_MIXED FP32 ones: eight independent FMA chains
 * per thread, 8 blocks of 256 threads per SM, best of three timed launches
 * (CUDA events on cuda_stream, after one untimed launch).  device_buf
 * (caller-owned device memory, at least 8 * 256 * SMs * sizeof(value)
 * bytes) receives the chains' sums.  *flop_per_s = 2 x FMAs / second.
 * Synchronises the stream.  SALE_ENOMEM when the buffer is too small. */
int sale_fma_probe(int precision, void *device_buf, size_t bytes, void *cuda_stream, double *flop_per_s);

const char *sale_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SALE_H */
