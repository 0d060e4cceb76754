// sale_internal.cuh -- device-side data structures and hex geometry of the
// GB300 SALE library.  Shared by the kernel and host translation units of
// the library only.
//
// Geometry (structured hex mesh, ScalSALE Table I "Mesh: Structured").
// The hex volume is the divergence-theorem sum over the six outward faces,
// each face fanned into four triangles from its node mean:
//     V = (1/24) sum_f S_f . ((p2 - p0) x (p3 - p1)),  S_f = p0+p1+p2+p3,
// which is the exact volume of the trilinear hex.  Its derivative with
// respect to node p_k of face f is
//     dT_f/dp_k = (p_{k+1} + 2 p_{k+2} + p_{k+3}) x (p_{k+3} - p_{k+1}),
// and dV/dx_a = (1/24) sum over the three faces holding a.  Coordinates
// are taken relative to local node 0 of the hex (translation invariance)
// to limit cancellation.
#pragma once

#include <cstddef>
#include <cstdint>

#include "sale.h"

namespace sale {

constexpr int kBlock = 256;           // threads per block of the 1D kernels
constexpr double kInvSixth24 = 1.0 / 24.0;

// Device scalars of one state (one cache line group, device memory).
struct DevScalars {
  double t;          // simulated time
  double dt;         // proposed next time step
  double dt_last;    // last time step taken
  double t_end;      // cycles stop once t >= t_end
  long long cycle;   // Lagrangian steps taken
  long long cycle_limit;  // cycles stop once cycle >= cycle_limit
  unsigned long long dtmin_bits;  // running CFL minimum (bits of a double)
  unsigned int blocks_done;       // last-block counter of the dt kernel
  int status;        // first device error (sale_status), 0 = OK
  // The next cycle, decided whenever t, dt or the limits change, so that
  // FP32 kernels read one flag and one step instead of comparing doubles
  // per thread (FP64 runs at 1/64 rate on GB300).
  int next_active;   // 1 while status == 0, t < t_end, cycle < cycle_limit
  float next_h32;    // min(dt, t_end - t) as FP32
  double next_h;     // min(dt, t_end - t)
  double pad[6];
};

// Kernels of the cycle, in the order of their launch-time profile slots.
enum KernelId : int {
  kInitNodes = 0,
  kEos,
  kLagNodes,
  kLagCells,
  kRemapFaces,
  kRemapNodes,
  kRemapCells,
  kDiag,
  kAleNodes,     // ALE path (positions start each cycle on the reference mesh)
  kAleCells,
  kAleDensity,
  kAleFluxes,
  kAleRemapEos,
  kGeoInit,
  kMixNodes,     // FP32-mixed Eulerian path
  kMixCells,
  kMixFluxes,
  kMixRemapNodes,
  kMixRemapEos,
  kMixEos,
  kAleEdges,     // ALE path: side-quad terms of the swept hexes, per mesh edge
  kAleRemapNodes,
  kAleEos,       // ALE path: EoS + dt on the reference mesh (refresh)
  kAleSlopes,    // ALE path, second-order remap: limited slopes of rho_L and e
  kMixDensity,   // FP32-mixed path, second-order remap: V_L and rho_L
  kPcPositions,  // predictor-corrector (general path): half-step positions
  kPcPredict,    //   half-step energy, EoS, viscosity: sigma^{n+1/2}
  kAlePredict,   // predictor-corrector, FP64 Eulerian path
  kMixPredict,   // predictor-corrector, FP32-mixed path
  kHourglass,    // hourglass corner forces: general path
  kAleHourglass, //   FP64 Eulerian path
  kMixHourglass, //   FP32-mixed path
  kNumKernels
};

// Modes of the kernel that ends a step and proposes the next dt.
enum DtMode : int {
  kDtPropose = 0,  // dt = min(cfl, growth * dt_last)
  kDtAdvance = 1,  // advance t and cycle by the step just taken, then propose
  kDtInit = 2      // dt = min(cfl, dt_init); dt_last = dt
};

// Device pointers and constants of one state (passed by value).
// Steinberg-Guinan parameters (the problem descriptor's strength fields).
struct Strength {
  double shear0, shear_dp, shear_dt, cv, e_ref, rho_ref, yield0, yield_max, hard_beta, hard_n;
  double inv_cv, inv_shear0;  // 1 / cv, 1 / shear0
};

template <typename R>
struct Fields {
  // --- read by the FP32-mixed kernels (a batch stages this prefix, up to
  // xr, in shared memory) ---
  int nx, ny, nz;
  long long nc, nn;
  R *u, *v, *w;                // node velocity
  R *ub, *vb, *wb;             // time-centred / remapped node velocity
  // Material strength (Steinberg-Guinan G and Y, Wilkins deviatoric
  // stress), FP64 states with shear0 > 0: sdev[q nc + c], q = xx, yy, zz,
  // xy, yz, zx, then the equivalent plastic strain (q = 6), and G, Y of the
  // current state (q = 7, 8: written by the EoS that ends every cycle, read
  // by the next cell pass); sold the first seven, the copy the cell remap
  // reads its donors from.  Null: no strength.
  R *sdev, *sold;
  Strength str;
  R *mn;                       // node mass
  R *dke;                      // kinetic energy lost by the node remap
  R *m, *e;                    // cell mass, specific internal energy
  // FP64 states: 1 / m and 1 / mn, written by every pass that writes m or mn
  // (and after a host upload of either), so the force and energy updates
  // multiply instead of dividing; null elsewhere
  R *im, *imn;
  R *mlo, *elo;                // FP32-mixed path: low parts of m and e (float-float); null otherwise
  R *mnlo;                     // FP32-mixed path: low part of the node mass (float-float); null otherwise
  R *sig;                      // p + q
  R *rho, *p, *q, *cs, *vol;   // derived cell fields
  R *mux, *muy, *muz;          // mass flux through the low x/y/z face
  R *epx, *epy, *epz;          // internal-energy flux through those faces
  const R *VE, *LE;            // reference volume and length scale
  R *dvx, *dvy, *dvz;          // swept volumes of the low x/y/z faces
  // Structured reference mesh of the FP32-mixed path: node (i,j,k) sits at
  // lo + (i,j,k) * h + off[node]; coordinate differences are formed as
  // index difference * h + offset difference (no absolute coordinates).
  float hx, hy, hz;
  const float4 *off4;          // per-node jitter offsets x, y, z (w unused); null: none
  // Jittered FP32-mixed meshes: dV/dx of the 8 corners of every reference
  // cell, Gc[(3 * corner + axis) * nc + c] (coalesced across a row of cells
  // and across a row of nodes); null on unjittered meshes, where the
  // gradient folds to constants.
  const float *Gc;
  R *Gh;                       // predictor-corrector: corner gradients at x^{n+1/2}, Gh[(3 a + axis) nc + c]
  // FP64 states: corner gradients at the current positions, Gn[(3 a + axis)
  // nc + c], written by the general EoS pass (which runs after every change
  // of the positions: each cycle, each remap, state creation and refresh)
  // and read by the next Lagrangian step; null elsewhere
  R *Gn;
  R *fh;                       // hourglass corner forces of the step, fh[(3 a + axis) nc + c]; null: no control
  double gamma, growth, dt_init;
  float gamma32, cfl32, c_q32, c_l32, c_hg32;  // FP32 copies of the constants
  int ke_fix;
  int remap_order;             // cell remap: 1 donor cell, 2 van Leer piecewise linear
  int time_order;              // Lagrangian step: 1 single stage, 2 predictor-corrector
  int reflect[6];
  // --- FP64 paths only ---
  const double *xr, *yr, *zr;  // reference mesh (Eulerian rezone target)
  R *x, *y, *z;                // current node positions
  R *xn, *yn, *zn;             // next node positions (written by the step)
  // Cached reference-mesh geometry (ALE path): dV/dx of every cell corner,
  // G[(corner*3 + axis) * nc + c].
  const R *G;
  const R *TE;                 // reference-face terms of the low-face swept hexes (3 per cell)
  // FP64 Eulerian path: 1 / V_E and 1 / (cfl L_E)^2 of the reference mesh,
  // the side-quad terms of the swept hexes along every mesh edge (nine node
  // arrays, ste[slot * nn + n], slot = 3 * axis + origin variant) and the
  // Lagrangian + reference low-face terms of the cell whose node 0 is n
  // (slots 9, 10, 11 for x, y, z), each cell's dual-mesh flux part
  // (mu_low + mu_high) / 8 along x/y/z, and the node kinetic energy per
  // unit mass 0.5 |u|^2 after the Lagrangian step.
  const R *iVE, *iL2;
  // FP64 Eulerian path with hourglass control: the four projected hourglass
  // shape vectors of every reference cell, scaled by V_E^(1/3),
  // HG[(8 alpha + a) nc + c] = (h_alpha(a) - hx_alpha . G_a / V_E) V_E^(1/3);
  // null without control
  const R *HG;
  // FP64 Eulerian path: reference offsets x_ref[b] - x_ref[n] from every
  // node n to its +x, +y, +z neighbours and its yz, xz, xy face-diagonal
  // neighbours, rE[(3 * slot + axis) * nn + n] (zero where b is off the mesh)
  const R *rE;
  R *ste;
  R *mqx, *mqy, *mqz;
  R *kd;
  double cfl, c_q, c_l, c_hg;
  R *srx, *sry, *srz, *sex, *sey, *sez;  // FP64 Eulerian path: slopes of rho_L and e along x, y, z
  R *ivl;                      // FP64 Eulerian path, second-order remap or materials: 1 / V_L (null otherwise)
  int remap_sets_x;            // node remap writes the reference positions to x
  // Materials (FP64 general path, nmat >= 2; null mat: one ideal gas):
  // mat[(3 k + q) nc + c] holds material k's volume fraction (q = 0), mass
  // (q = 1) and specific internal energy (q = 2) in cell c; m and e above
  // are the cell totals.  mfx[(9 k + 3 axis + q) nc + c] holds the
  // material's volume (q = 0), mass (1) and energy (2) flux through the
  // cell's low face along axis, written by the face pass of a remap.
  R *mat, *mfx;
  R *msh;                      // materials with the predictor-corrector: alpha_k (p_k + q) of the half step, msh[k nc + c]
  int nmat;
  double mgam[4], mpinf[4];    // stiffened-gas gamma and p_inf of every material
};

constexpr int kMaxMat = 4;
constexpr double kAlphaMin = 1e-8;  // a material at or below this fraction after a remap leaves the cell

// Hourglass patterns of the hex (local node a = di + 2 dj + 4 dk, signs
// s = 2 d - 1): s_x s_y, s_y s_z, s_z s_x, s_x s_y s_z.
__host__ __device__ constexpr float hg_pattern(int alpha, int a) {
  return (alpha == 0   ? (((a & 1) != 0) == ((a & 2) != 0))
          : alpha == 1 ? (((a & 2) != 0) == ((a & 4) != 0))
          : alpha == 2 ? (((a & 4) != 0) == ((a & 1) != 0))
                       : ((((a & 1) != 0) + ((a & 2) != 0) + ((a & 4) != 0)) % 2 == 1))
             ? 1.f
             : -1.f;
}

// Thread-tile shapes of the FP32-mixed kernels (x by y threads over one k
// plane); the autotuner picks one per state or batch.
constexpr int kNumTileShapes = 5;
// Node planes one block of the FP32-mixed node remap marches over, and cell
// planes one block of its remap + EoS + dt pass covers.
constexpr int kRemapChunk = 16;
constexpr int kEosPlanes = 8;

__host__ __device__ constexpr int tile_x(int shape) {
  return shape == 0 ? 32 : shape == 1 ? 32 : shape == 2 ? 64 : shape == 3 ? 128 : 16;
}
__host__ __device__ constexpr int tile_y(int shape) {
  return shape == 0 ? 8 : shape == 1 ? 4 : shape == 2 ? 4 : shape == 3 ? 2 : 8;
}
constexpr int kMaxWarpsPerBlock = 16;

// One mesh of a batch, as seen by the batched kernels.
struct BatchItem {
  DevScalars *S;
  unsigned nblk_cell;  // blocks of this mesh in the remap + EoS pass (last-block detection of its dt)
  unsigned pad;
  Fields<float> F;
};

// Bytes of a BatchItem the FP32-mixed kernels read: its header and the
// mixed prefix of F (everything before the FP64-only xr).
constexpr size_t kBatchItemStaged = offsetof(BatchItem, F) + offsetof(Fields<float>, xr);

// Per-mesh summary the host reads after a batched run.
struct BatchStatus {
  double t, dt;
  long long cycle;
  long long status;
};

struct P3 {
  double x, y, z;
};

__host__ __device__ __forceinline__ P3 operator+(P3 a, P3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__host__ __device__ __forceinline__ P3 operator-(P3 a, P3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__host__ __device__ __forceinline__ P3 operator*(double s, P3 a) { return {s * a.x, s * a.y, s * a.z}; }
__host__ __device__ __forceinline__ P3 cross(P3 a, P3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__host__ __device__ __forceinline__ double dot(P3 a, P3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Outward faces of the hex (local node a = di + 2 dj + 4 dk), cyclic order:
// x-lo {0,4,6,2}, x-hi {1,3,7,5}, y-lo {0,1,5,4}, y-hi {2,6,7,3},
// z-lo {0,2,3,1}, z-hi {4,5,7,6}.
__host__ __device__ constexpr int face_node(int f, int k) {
  return f == 0   ? (k == 0 ? 0 : k == 1 ? 4 : k == 2 ? 6 : 2)
         : f == 1 ? (k == 0 ? 1 : k == 1 ? 3 : k == 2 ? 7 : 5)
         : f == 2 ? (k == 0 ? 0 : k == 1 ? 1 : k == 2 ? 5 : 4)
         : f == 3 ? (k == 0 ? 2 : k == 1 ? 6 : k == 2 ? 7 : 3)
         : f == 4 ? (k == 0 ? 0 : k == 1 ? 2 : k == 2 ? 3 : 1)
                  : (k == 0 ? 4 : k == 1 ? 5 : k == 2 ? 7 : 6);
}

// Position of local node a in the cycle of face f (f must hold a).
__host__ __device__ constexpr int face_slot(int f, int a) {
  return face_node(f, 0) == a ? 0 : face_node(f, 1) == a ? 1 : face_node(f, 2) == a ? 2 : 3;
}

// Shift hex coordinates so local node 0 is the origin.
__device__ __forceinline__ void shift0(P3 (&X)[8]) {
  const P3 o = X[0];
#pragma unroll
  for (int a = 0; a < 8; ++a) X[a] = X[a] - o;
}

// Volume of a hex whose coordinates are already shifted (X[0] = 0).
__device__ __forceinline__ double hex_volume_shifted(const P3 (&X)[8]) {
  double s = 0.0;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const P3 p0 = X[face_node(f, 0)], p1 = X[face_node(f, 1)];
    const P3 p2 = X[face_node(f, 2)], p3 = X[face_node(f, 3)];
    s += dot(p0 + p1 + p2 + p3, cross(p2 - p0, p3 - p1));
  }
  return s * kInvSixth24;
}

// Full volume gradient of a shifted hex: G[a] = dV/dx_a.
__device__ __forceinline__ void hex_grad_shifted(const P3 (&X)[8], P3 (&G)[8]) {
#pragma unroll
  for (int a = 0; a < 8; ++a) G[a] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int f = 0; f < 6; ++f) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const P3 pa = X[face_node(f, (k + 1) & 3)];
      const P3 pb = X[face_node(f, (k + 2) & 3)];
      const P3 pc = X[face_node(f, (k + 3) & 3)];
      G[face_node(f, k)] = G[face_node(f, k)] + cross(pa + 2.0 * pb + pc, pc - pa);
    }
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) G[a] = kInvSixth24 * G[a];
}

// dV/dx_A for one compile-time corner A of a shifted hex.
template <int A>
__device__ __forceinline__ P3 hex_corner_grad_shifted(const P3 (&X)[8]) {
  P3 g = {0.0, 0.0, 0.0};
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const int f = 2 * t + ((A >> t) & 1);
    const int k = face_slot(f, A);
    const P3 pa = X[face_node(f, (k + 1) & 3)];
    const P3 pb = X[face_node(f, (k + 2) & 3)];
    const P3 pc = X[face_node(f, (k + 3) & 3)];
    g = g + cross(pa + 2.0 * pb + pc, pc - pa);
  }
  return kInvSixth24 * g;
}

// max_f |A_f|^2 of the face vector areas A_f = (1/2)(p2-p0) x (p3-p1).
__device__ __forceinline__ double hex_max_face_area2(const P3 (&X)[8]) {
  double amax = 0.0;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const P3 p0 = X[face_node(f, 0)], p1 = X[face_node(f, 1)];
    const P3 p2 = X[face_node(f, 2)], p3 = X[face_node(f, 3)];
    const P3 D = cross(p2 - p0, p3 - p1);
    amax = fmax(amax, 0.25 * dot(D, D));
  }
  return amax;
}

__device__ __forceinline__ long long node_index(int nx, int ny, int i, int j, int k) {
  return (long long)i + (long long)(nx + 1) * ((long long)j + (long long)(ny + 1) * k);
}

__device__ __forceinline__ long long cell_index(int nx, int ny, int i, int j, int k) {
  return (long long)i + (long long)nx * ((long long)j + (long long)ny * k);
}

// Record the first device error.
__device__ __forceinline__ void set_status(DevScalars *S, int code) {
  atomicCAS(&S->status, 0, code);
}

// True while the current cycle should run.
__device__ __forceinline__ bool cycle_active(const DevScalars *S) {
  return S->status == 0 && S->t < S->t_end && S->cycle < S->cycle_limit;
}

// Refresh the next-cycle decision (single thread; after t/dt/limits change).
__device__ __forceinline__ void decide_next(volatile DevScalars *S) {
  const bool act = S->status == 0 && S->t < S->t_end && S->cycle < S->cycle_limit;
  const double rem = S->t_end - S->t;
  const double h = rem < S->dt ? rem : S->dt;
  S->next_h = h;
  S->next_h32 = (float)h;
  S->next_active = act ? 1 : 0;
}

// The time step of the cycle in flight: an explicit dt > 0, else the
// proposed dt clamped so the step lands on t_end.
__device__ __forceinline__ double step_dt(const DevScalars *S, double dt_override) {
  if (dt_override > 0.0) return dt_override;
  const double rem = S->t_end - S->t;
  return rem < S->dt ? rem : S->dt;
}

}  // namespace sale
