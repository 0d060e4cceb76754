// sale_capi.cu -- host side of the C ABI declared in include/sale.h.
//
// Owns handles, validates arguments, generates the mesh and the primitive
// initial state on the host, carves the caller's device buffer into the
// structure-of-arrays fields, orders the kernels of a cycle on the state's
// stream and replays captured CUDA graphs of whole cycles.  Time, dt and the
// error status stay on the device; the host reads them back only in the
// synchronising calls.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "sale_internal.cuh"

namespace sale {
void launch_reset(DevScalars *, cudaStream_t);
void launch_set_limits(DevScalars *, double, long long, cudaStream_t);
template <typename R>
void launch_init_cells(const Fields<R> &, DevScalars *, const double *, const double *, long long, double, int,
                       cudaStream_t);
template <typename R>
void launch_kernel(int kid, const Fields<R> &, DevScalars *, int mode, double dt_override, double *partial,
                   double *out, cudaStream_t);
void launch_geo_init_nodes(const Fields<double> &F, double *rE, cudaStream_t st);
void launch_geo_init_hg(const Fields<double> &F, double *HG, cudaStream_t st);
void launch_recip(const double *a, double *r, long long n, cudaStream_t st);
void launch_mat_totals(const Fields<double> &F, cudaStream_t st);
void launch_geo_init(const Fields<double> &F, DevScalars *S, double *G, double *VE, double *LE, double *TE,
                     double *iVE, double *iL2, cudaStream_t st);
void launch_m_init_cells(const Fields<float> &F, DevScalars *S, const double *rho0, const double *p0,
                         long long dep_cell, double dep_e, float *VE, float *LE, float *Gc, cudaStream_t st);
void launch_m_kernel(int kid, const Fields<float> &F, DevScalars *S, int mode, int shape, cudaStream_t st);
void launch_split64(const double *in, float *hi, float *lo, long long n, cudaStream_t st);
void launch_join64(const float *hi, const float *lo, double *out, long long n, cudaStream_t st);
}  // namespace sale

using namespace sale;

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------

static thread_local std::string g_last_error;

static int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

namespace sale {
// Error reporting shared with the library's other host translation units.
int report_error(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}
}  // namespace sale

static int cuda_fail(cudaError_t e, const char *where) {
  return fail(SALE_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CUDA_TRY(expr)                                \
  do {                                                \
    cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr); \
  } while (0)

static const char *status_name(int s) {
  switch (s) {
    case SALE_ENEGVOL: return "non-positive cell volume or node mass (mesh tangled)";
    case SALE_EDT: return "time step not positive or not finite";
    case SALE_ENAN: return "NaN in a field";
    case SALE_ETIMEOUT: return "bounded device wait ran out";
    default: return "device error";
  }
}

// ---------------------------------------------------------------------------
// Mesh (host)
// ---------------------------------------------------------------------------

struct sale_mesh {
  sale_mesh_desc d;
  long long nc, nn;
  std::vector<double> x, y, z;
};

static uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

extern "C" int sale_mesh_create(const sale_mesh_desc *desc, sale_mesh **out) {
  if (!desc || !out) return fail(SALE_EINVAL, "sale_mesh_create: null argument");
  *out = nullptr;
  const sale_mesh_desc &d = *desc;
  if (d.nx < 1 || d.ny < 1 || d.nz < 1) return fail(SALE_EINVAL, "sale_mesh_create: cell counts must be >= 1");
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  if (nn > (1ll << 33)) return fail(SALE_EINVAL, "sale_mesh_create: mesh too large");
  for (int a = 0; a < 3; ++a)
    if (!(d.hi[a] > d.lo[a]) || !std::isfinite(d.lo[a]) || !std::isfinite(d.hi[a]))
      return fail(SALE_EINVAL, "sale_mesh_create: need finite lo < hi on every axis");
  if (!(d.jitter >= 0.0 && d.jitter <= 0.45)) return fail(SALE_EINVAL, "sale_mesh_create: jitter must be in [0, 0.45]");
  for (int f = 0; f < 6; ++f)
    if (d.reflect[f] != 1) return fail(SALE_EINVAL, "sale_mesh_create: every wall must be reflecting (reflect[f] = 1)");
  sale_mesh *m = new (std::nothrow) sale_mesh;
  if (!m) return fail(SALE_ENOMEM, "sale_mesh_create: out of host memory");
  m->d = d;
  m->nc = (long long)d.nx * d.ny * d.nz;
  m->nn = nn;
  try {
    m->x.resize(nn);
    m->y.resize(nn);
    m->z.resize(nn);
  } catch (...) {
    delete m;
    return fail(SALE_ENOMEM, "sale_mesh_create: out of host memory");
  }
  const int n[3] = {d.nx, d.ny, d.nz};
  double h[3];
  for (int a = 0; a < 3; ++a) h[a] = (d.hi[a] - d.lo[a]) / n[a];
  std::vector<double> *dst[3] = {&m->x, &m->y, &m->z};
  for (int k = 0; k <= d.nz; ++k)
    for (int j = 0; j <= d.ny; ++j)
      for (int i = 0; i <= d.nx; ++i) {
        const long long node = i + (long long)(d.nx + 1) * (j + (long long)(d.ny + 1) * k);
        const int idx[3] = {i, j, k};
        for (int a = 0; a < 3; ++a) {
          double c = d.lo[a] + (double)idx[a] * h[a];
          if (d.jitter > 0.0 && idx[a] > 0 && idx[a] < n[a]) {
            const uint64_t r = splitmix64_at(d.seed, (uint64_t)node * 3u + (uint64_t)a);
            const double u = (double)(r >> 11) * 0x1p-53;
            const double off = ((2.0 * u - 1.0) * d.jitter) * h[a];
            c = c + off;
          }
          (*dst[a])[node] = c;
        }
      }
  *out = m;
  return SALE_OK;
}

extern "C" void sale_mesh_destroy(sale_mesh *mesh) { delete mesh; }

extern "C" int sale_mesh_nodes(const sale_mesh *mesh, double *xyz, size_t n) {
  if (!mesh || !xyz) return fail(SALE_EINVAL, "sale_mesh_nodes: null argument");
  if (n != (size_t)(3 * mesh->nn)) return fail(SALE_EINVAL, "sale_mesh_nodes: need 3*nnodes = %lld doubles", 3 * mesh->nn);
  memcpy(xyz, mesh->x.data(), sizeof(double) * mesh->nn);
  memcpy(xyz + mesh->nn, mesh->y.data(), sizeof(double) * mesh->nn);
  memcpy(xyz + 2 * mesh->nn, mesh->z.data(), sizeof(double) * mesh->nn);
  return SALE_OK;
}


// ---------------------------------------------------------------------------
// State layout
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kAlign = 256;
constexpr int kDiagBlocks = 512;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Hands out 256-byte aligned pieces of one buffer (or, with base == null,
// only counts the bytes: the same code sizes and carves a state).
struct Carver {
  char *base;
  size_t off = 0;
  void *take(size_t bytes) {
    off = align_up(off);
    void *p = base ? base + off : nullptr;
    off += bytes;
    return p;
  }
};

}  // namespace

struct GraphKey {
  int k, remap_every, xpar, upar, flags;
  bool operator<(const GraphKey &o) const {
    return std::tie(k, remap_every, xpar, upar, flags) < std::tie(o.k, o.remap_every, o.xpar, o.upar, o.flags);
  }
};

struct ProfEvent {
  int kid;
  cudaEvent_t a, b;
};

struct sale_state {
  int nx, ny, nz;
  long long nc, nn;
  int precision;       // SALE_FP64 or SALE_FP32_MIXED
  size_t elem;         // bytes of one stored value
  cudaStream_t stream;
  DevScalars *S;
  double *diag_partial, *diag_out;
  double *xr[3];       // reference mesh, FP64 in every precision
  void *xs[2][3];      // two position buffers (FP64 path)
  void *us[2][3];      // two velocity buffers
  void *mn, *dke;
  void *m, *e, *sig, *rho, *p, *q, *cs, *vol, *mu[3], *ep[3], *dv[3];
  double *geoG, *geoVE, *geoLE, *geoTE;  // FP64 path: cached reference geometry
  double *geoIVE, *geoIL2;               //   1 / V_E, 1 / (cfl L_E)^2
  double *geoHG;                         //   hourglass shape vectors (32 per cell; control on)
  double *im, *imn;                      //   1 / m per cell, 1 / mn per node
  double *sdev, *sold;                   //   strength: stress, plastic strain, G, Y (9 per cell); remap copy (7)
  double *Gn;                            //   corner gradients at the current positions (24 per cell)
  double *mat, *mfx;                     //   materials: fraction, mass, energy (3 per material per cell); face fluxes (9)
  double *msh;                           //   materials with the predictor-corrector: half-step shares (1 per material)
  double *ste, *mq[3], *kd;              // FP64 path: Eulerian-cycle working arrays
  double *relE;                          // FP64 path: reference offsets to 6 neighbours (18 per node)
  double *slope[7];                      // FP64 path, second-order remap: slopes of rho_L and e along x, y, z; 1/V_L
  float4 *off4;                          // FP32-mixed path: jitter offsets
  float *mlo, *elo;                      // FP32-mixed path: low parts of m, e
  float *mnlo;                           // FP32-mixed path: low part of the node mass
  float *VE32, *LE32;                    // FP32-mixed path: V_E, L_E
  float *Gc;                             // FP32-mixed path, jittered mesh: corner gradients
  void *Gh;                              // predictor-corrector: half-step corner gradients (24 per cell)
  void *fh;                              // hourglass control: corner forces of the step (24 per cell)
  bool jit = false;                      // the mesh is jittered
  bool o2 = false;                       // second-order remap scratch carved (FP64)
  bool pc = false;                       // predictor-corrector scratch carved
  bool hg = false;                       // hourglass scratch carved
  bool str = false;                      // material strength (FP64): deviatoric stress carved
  int nmat = 0;                          // materials (FP64, >= 2), 0: one ideal gas
  float h32[3];
  int xpar, upar;
  bool x_is_ref;       // current positions are the reference mesh
  int tile_shape = 0;  // thread-tile shape of the FP32-mixed kernels
  int remap_sets_x;    // flag passed to the node remap kernel
  double lim_t_end;
  long long lim_cycles;
  bool failed;
  int fail_code;
  sale_problem_desc prob;
  int reflect[6];
  std::map<GraphKey, cudaGraphExec_t> graphs;
  // launch-time profile: CUDA events around every kernel of the cycle
  bool prof_on = false;
  bool capturing = false;
  std::vector<cudaEvent_t> ev_pool;                  // free events
  std::vector<ProfEvent> pending;                    // direct launches not yet read
  std::vector<ProfEvent> capture_events;             // events of the graph being captured
  std::map<GraphKey, std::vector<ProfEvent>> graph_events;
  std::vector<const std::vector<ProfEvent> *> pending_graphs;  // replays not yet read
  double prof_ms[kNumKernels] = {};
  long long prof_n[kNumKernels] = {};
};

// Carve (or, with base == null, size) the device fields of a state.
static size_t carve(sale_state *st, char *base) {
  Carver cv{base};
  const size_t E = st->elem, nn = (size_t)st->nn, nc = (size_t)st->nc;
  const bool fp64 = st->precision == SALE_FP64;
  st->S = (DevScalars *)cv.take(sizeof(DevScalars));
  st->diag_partial = (double *)cv.take(sizeof(double) * 6 * kDiagBlocks);
  st->diag_out = (double *)cv.take(sizeof(double) * 8);
  for (int d = 0; d < 3; ++d) st->xr[d] = (double *)cv.take(sizeof(double) * nn);
  for (int b = 0; b < 2; ++b)
    for (int d = 0; d < 3; ++d) {
      st->xs[b][d] = fp64 ? cv.take(E * nn) : nullptr;  // the mixed path keeps positions implicit
      st->us[b][d] = cv.take(E * nn);
    }
  st->mn = cv.take(E * nn);
  st->dke = cv.take(E * nn);
  void **cells[] = {&st->m, &st->e, &st->sig, &st->rho, &st->p, &st->q, &st->cs, &st->vol};
  for (void **c : cells) *c = cv.take(E * nc);
  for (int d = 0; d < 3; ++d) {
    st->mu[d] = cv.take(E * nc);
    st->ep[d] = cv.take(E * nc);
    st->dv[d] = cv.take(E * nc);
  }
  st->geoG = st->geoVE = st->geoLE = st->geoTE = st->geoIVE = st->geoIL2 = st->geoHG = nullptr;
  st->im = st->imn = nullptr;
  st->sdev = st->sold = nullptr;
  st->Gn = nullptr;
  st->mat = st->mfx = st->msh = nullptr;
  st->ste = st->kd = st->mq[0] = st->mq[1] = st->mq[2] = nullptr;
  st->relE = nullptr;
  for (int d = 0; d < 7; ++d) st->slope[d] = nullptr;
  st->off4 = nullptr;
  st->VE32 = st->LE32 = st->mlo = st->elo = st->mnlo = nullptr;
  st->Gc = nullptr;
  st->Gh = nullptr;
  st->fh = nullptr;
  if (fp64) {
    // one block, the corner gradients indexed with stride nc
    st->geoG = (double *)cv.take(sizeof(double) * 31 * nc);
    if (base) {
      st->geoVE = st->geoG + 24 * nc;
      st->geoLE = st->geoVE + nc;
      st->geoTE = st->geoLE + nc;
      st->geoIVE = st->geoTE + 3 * nc;
      st->geoIL2 = st->geoIVE + nc;
    }
    st->ste = (double *)cv.take(sizeof(double) * 12 * nn);
    st->relE = (double *)cv.take(sizeof(double) * 18 * nn);
    for (int d = 0; d < 3; ++d) st->mq[d] = (double *)cv.take(sizeof(double) * nc);
    st->kd = (double *)cv.take(sizeof(double) * nn);
    st->im = (double *)cv.take(sizeof(double) * nc);
    st->imn = (double *)cv.take(sizeof(double) * nn);
    st->Gn = (double *)cv.take(sizeof(double) * 24 * nc);
    if (st->o2)
      for (int d = 0; d < 7; ++d) st->slope[d] = (double *)cv.take(sizeof(double) * nc);
    else if (st->nmat >= 2)  // materials: 1 / V_L for the flux pass
      st->slope[6] = (double *)cv.take(sizeof(double) * nc);
    if (st->hg) st->geoHG = (double *)cv.take(sizeof(double) * 32 * nc);
    if (st->str) {
      st->sdev = (double *)cv.take(sizeof(double) * 9 * nc);
      st->sold = (double *)cv.take(sizeof(double) * 7 * nc);
    }
    if (st->nmat >= 2) {
      st->mat = (double *)cv.take(sizeof(double) * 3 * (size_t)st->nmat * nc);
      st->mfx = (double *)cv.take(sizeof(double) * 9 * (size_t)st->nmat * nc);
      if (st->pc) st->msh = (double *)cv.take(sizeof(double) * (size_t)st->nmat * nc);
    }
  } else {
    st->off4 = (float4 *)cv.take(sizeof(float4) * nn);
    st->VE32 = (float *)cv.take(sizeof(float) * nc);
    st->LE32 = (float *)cv.take(sizeof(float) * nc);
    st->mlo = (float *)cv.take(sizeof(float) * nc);
    st->elo = (float *)cv.take(sizeof(float) * nc);
    st->mnlo = (float *)cv.take(sizeof(float) * nn);
    if (st->jit) st->Gc = (float *)cv.take(sizeof(float) * 24 * nc);
  }
  if (st->pc) st->Gh = cv.take(E * 24 * nc);
  if (st->hg) st->fh = cv.take(E * 24 * nc);
  return align_up(cv.off);
}

template <typename R>
static Fields<R> fields_t(const sale_state *st) {
  Fields<R> F = {};
  F.nx = st->nx;
  F.ny = st->ny;
  F.nz = st->nz;
  F.nc = st->nc;
  F.nn = st->nn;
  F.xr = st->xr[0];
  F.yr = st->xr[1];
  F.zr = st->xr[2];
  F.x = (R *)st->xs[st->xpar][0];
  F.y = (R *)st->xs[st->xpar][1];
  F.z = (R *)st->xs[st->xpar][2];
  F.xn = (R *)st->xs[st->xpar ^ 1][0];
  F.yn = (R *)st->xs[st->xpar ^ 1][1];
  F.zn = (R *)st->xs[st->xpar ^ 1][2];
  F.u = (R *)st->us[st->upar][0];
  F.v = (R *)st->us[st->upar][1];
  F.w = (R *)st->us[st->upar][2];
  F.ub = (R *)st->us[st->upar ^ 1][0];
  F.vb = (R *)st->us[st->upar ^ 1][1];
  F.wb = (R *)st->us[st->upar ^ 1][2];
  F.mn = (R *)st->mn;
  F.dke = (R *)st->dke;
  F.m = (R *)st->m;
  F.e = (R *)st->e;
  F.sig = (R *)st->sig;
  F.rho = (R *)st->rho;
  F.p = (R *)st->p;
  F.q = (R *)st->q;
  F.cs = (R *)st->cs;
  F.vol = (R *)st->vol;
  F.mux = (R *)st->mu[0];
  F.muy = (R *)st->mu[1];
  F.muz = (R *)st->mu[2];
  F.epx = (R *)st->ep[0];
  F.epy = (R *)st->ep[1];
  F.epz = (R *)st->ep[2];
  F.dvx = (R *)st->dv[0];
  F.dvy = (R *)st->dv[1];
  F.dvz = (R *)st->dv[2];
  if (st->precision == SALE_FP64) {
    F.G = (const R *)st->geoG;
    F.VE = (const R *)st->geoVE;
    F.LE = (const R *)st->geoLE;
    F.TE = (const R *)st->geoTE;
    F.iVE = (const R *)st->geoIVE;
    F.iL2 = (const R *)st->geoIL2;
    F.HG = (const R *)st->geoHG;
    F.sdev = (R *)st->sdev;
    F.sold = (R *)st->sold;
    F.Gn = (R *)st->Gn;
    F.ste = (R *)st->ste;
    F.rE = (const R *)st->relE;
    F.mqx = (R *)st->mq[0];
    F.mqy = (R *)st->mq[1];
    F.mqz = (R *)st->mq[2];
    F.kd = (R *)st->kd;
    F.im = (R *)st->im;
    F.imn = (R *)st->imn;
  } else {
    F.VE = (const R *)st->VE32;
    F.LE = (const R *)st->LE32;
  }
  F.mlo = (R *)st->mlo;
  F.elo = (R *)st->elo;
  F.mnlo = (R *)st->mnlo;
  F.hx = st->h32[0];
  F.hy = st->h32[1];
  F.hz = st->h32[2];
  F.off4 = st->off4;
  F.Gc = st->Gc;
  F.remap_sets_x = st->remap_sets_x;
  F.gamma = st->prob.gamma;
  F.cfl = st->prob.cfl;
  F.c_q = st->prob.c_q;
  F.c_l = st->prob.c_l;
  F.growth = st->prob.dt_growth;
  F.dt_init = std::isfinite(st->prob.dt_init) ? st->prob.dt_init : 0.0;
  F.gamma32 = (float)F.gamma;
  F.cfl32 = (float)F.cfl;
  F.c_q32 = (float)F.c_q;
  F.c_l32 = (float)F.c_l;
  F.ke_fix = st->prob.ke_fix;
  F.remap_order = st->prob.remap_order == 2 ? 2 : 1;
  F.time_order = st->prob.time_order == 2 ? 2 : 1;
  F.Gh = (R *)st->Gh;
  F.fh = (R *)st->fh;
  F.c_hg = st->prob.c_hg;
  F.c_hg32 = (float)st->prob.c_hg;
  F.str = {st->prob.shear0,  st->prob.shear_dp,  st->prob.shear_dt,  st->prob.cv,        st->prob.e_ref,
           st->prob.rho_ref, st->prob.yield0,    st->prob.yield_max, st->prob.hard_beta, st->prob.hard_n,
           st->prob.cv > 0.0 ? 1.0 / st->prob.cv : 0.0, st->prob.shear0 > 0.0 ? 1.0 / st->prob.shear0 : 0.0};
  F.srx = (R *)st->slope[0];
  F.sry = (R *)st->slope[1];
  F.srz = (R *)st->slope[2];
  F.sex = (R *)st->slope[3];
  F.sey = (R *)st->slope[4];
  F.sez = (R *)st->slope[5];
  F.ivl = (R *)st->slope[6];
  for (int f = 0; f < 6; ++f) F.reflect[f] = st->reflect[f];
  F.mat = (R *)st->mat;
  F.mfx = (R *)st->mfx;
  F.msh = (R *)st->msh;
  F.nmat = st->nmat;
  for (int k = 0; k < kMaxMat; ++k) {
    F.mgam[k] = st->prob.mat_gamma[k];
    F.mpinf[k] = st->prob.mat_pinf[k];
  }
  return F;
}

static size_t state_bytes(long long nc, long long nn, int precision, bool jit, bool o2 = false, bool pc = false,
                          bool hg = false, bool str = false, int nmat = 0) {
  sale_state tmp;
  tmp.nc = nc;
  tmp.nn = nn;
  tmp.precision = precision;
  tmp.jit = jit;
  tmp.o2 = o2 && precision == SALE_FP64;
  tmp.pc = pc;
  tmp.hg = hg;
  tmp.str = str && precision == SALE_FP64;
  tmp.nmat = nmat >= 2 && precision == SALE_FP64 ? nmat : 0;
  tmp.elem = precision == SALE_FP64 ? sizeof(double) : sizeof(float);
  return carve(&tmp, nullptr);
}

// The FP32-mixed kernels index cells and nodes with 32-bit integers.
static bool mixed_fits(const sale_mesh *mesh, int precision) {
  return precision != SALE_FP32_MIXED || mesh->nn <= 0x7FFFFFFFll;
}

extern "C" size_t sale_state_bytes(const sale_mesh *mesh, int precision) {
  if (!mesh || (precision != SALE_FP64 && precision != SALE_FP32_MIXED) || !mixed_fits(mesh, precision)) return 0;
  return state_bytes(mesh->nc, mesh->nn, precision, mesh->d.jitter > 0.0);
}

extern "C" size_t sale_state_bytes_for(const sale_mesh *mesh, const sale_problem_desc *prob, int precision) {
  if (!mesh || !prob || (precision != SALE_FP64 && precision != SALE_FP32_MIXED) || !mixed_fits(mesh, precision))
    return 0;
  return state_bytes(mesh->nc, mesh->nn, precision, mesh->d.jitter > 0.0, prob->remap_order == 2,
                     prob->time_order == 2, prob->c_hg > 0.0, prob->shear0 > 0.0, prob->nmat);
}

static int validate_problem(const sale_problem_desc &p) {
  if (p.kind < SALE_PROB_SOD_X || p.kind > SALE_PROB_UNIFORM) return fail(SALE_EINVAL, "problem: unknown kind %d", p.kind);
  if (!(p.gamma > 1.0) || !std::isfinite(p.gamma)) return fail(SALE_EINVAL, "problem: gamma must be > 1");
  if (!(p.cfl > 0.0 && p.cfl <= 1.0)) return fail(SALE_EINVAL, "problem: cfl must be in (0, 1]");
  if (!(p.c_q >= 0.0) || !(p.c_l >= 0.0)) return fail(SALE_EINVAL, "problem: viscosity coefficients must be >= 0");
  if (!(p.dt_growth >= 1.0) || !std::isfinite(p.dt_growth)) return fail(SALE_EINVAL, "problem: dt_growth must be >= 1");
  const double dens[] = {p.rho_l, p.rho_r, p.rho_bg, p.rho_blast};
  const double pres[] = {p.p_l, p.p_r, p.p_bg, p.p_blast};
  for (int i = 0; i < 4; ++i) {
    if (!(dens[i] > 0.0) || !std::isfinite(dens[i])) return fail(SALE_EINVAL, "problem: densities must be finite and > 0");
    if (!(pres[i] >= 0.0) || !std::isfinite(pres[i])) return fail(SALE_EINVAL, "problem: pressures must be finite and >= 0");
  }
  if (!std::isfinite(p.e_deposit) || p.e_deposit < 0.0) return fail(SALE_EINVAL, "problem: e_deposit must be finite and >= 0");
  if (p.remap_order < 0 || p.remap_order > 2) return fail(SALE_EINVAL, "problem: remap_order must be 0, 1 or 2");
  if (p.time_order < 0 || p.time_order > 2) return fail(SALE_EINVAL, "problem: time_order must be 0, 1 or 2");
  if (!(p.c_hg >= 0.0) || !std::isfinite(p.c_hg)) return fail(SALE_EINVAL, "problem: c_hg must be finite and >= 0");
  if (!(p.shear0 >= 0.0) || !std::isfinite(p.shear0)) return fail(SALE_EINVAL, "problem: shear0 must be finite and >= 0");
  if (p.nmat < 0 || p.nmat > SALE_MAX_MAT) return fail(SALE_EINVAL, "problem: nmat must be in [0, %d]", SALE_MAX_MAT);
  if (p.nmat >= 2) {
    for (int k = 0; k < p.nmat; ++k)
      if (!(p.mat_gamma[k] > 1.0) || !std::isfinite(p.mat_gamma[k]) || !(p.mat_pinf[k] >= 0.0) ||
          !std::isfinite(p.mat_pinf[k]))
        return fail(SALE_EINVAL, "problem: material %d needs mat_gamma > 1 and a finite mat_pinf >= 0", k);
    if (p.shear0 > 0.0 || p.remap_order == 2)
      return fail(SALE_EINVAL, "problem: materials take the first-order remap, without strength");
  }
  if (p.shear0 > 0.0) {
    const double fin[] = {p.shear_dp, p.shear_dt, p.e_ref, p.yield0, p.yield_max, p.hard_beta, p.hard_n};
    for (double v : fin)
      if (!std::isfinite(v)) return fail(SALE_EINVAL, "problem: strength parameters must be finite");
    if (!(p.cv > 0.0) || !(p.rho_ref > 0.0) || !std::isfinite(p.cv) || !std::isfinite(p.rho_ref))
      return fail(SALE_EINVAL, "problem: strength needs cv > 0 and rho_ref > 0");
    if (p.yield0 < 0.0 || p.yield_max < 0.0 || p.hard_beta < 0.0 || p.hard_n < 0.0)
      return fail(SALE_EINVAL, "problem: yield0, yield_max, hard_beta, hard_n must be >= 0");
    if (p.time_order == 2)
      return fail(SALE_EINVAL, "problem: material strength takes the single-stage step (time_order 1)");
  }
  return SALE_OK;
}

// Per-cell primitive initial state (same definition as the Python inputs
// module: logical cell centres for the Sod split, origin cell for Sedov).
static void host_primitives(const sale_mesh &mesh, const sale_problem_desc &p, std::vector<double> &rho0,
                            std::vector<double> &p0, long long &dep_cell, double &dep_e) {
  const sale_mesh_desc &d = mesh.d;
  rho0.assign(mesh.nc, p.rho_bg);
  p0.assign(mesh.nc, p.p_bg);
  dep_cell = -1;
  dep_e = 0.0;
  if (p.kind == SALE_PROB_SOD_X) {
    const double hx = (d.hi[0] - d.lo[0]) / d.nx;
    for (long long c = 0; c < mesh.nc; ++c) {
      const int i = (int)(c % d.nx);
      const bool left = (d.lo[0] + ((double)i + 0.5) * hx) < p.x_split;
      rho0[c] = left ? p.rho_l : p.rho_r;
      p0[c] = left ? p.p_l : p.p_r;
    }
  } else if (p.kind == SALE_PROB_SEDOV) {
    if (p.e_deposit > 0.0) {
      dep_cell = 0;
      dep_e = p.e_deposit;
    } else {
      rho0[0] = p.rho_blast;
      p0[0] = p.p_blast;
    }
  }
}

static void collect_profile(sale_state *st);

static int sync_scalars(const sale_state *cst, DevScalars *h) {
  sale_state *st = const_cast<sale_state *>(cst);
  CUDA_TRY(cudaMemcpyAsync(h, st->S, sizeof(DevScalars), cudaMemcpyDeviceToHost, st->stream));
  CUDA_TRY(cudaStreamSynchronize(st->stream));
  if (!st->pending.empty() || !st->pending_graphs.empty()) collect_profile(st);
  return SALE_OK;
}

// Mark the state failed if the device reported an error.
static int check_device_status(sale_state *st, const DevScalars &h) {
  if (h.status != 0) {
    st->failed = true;
    st->fail_code = h.status;
    return fail(h.status, "device: %s (t = %.17g, cycle %lld)", status_name(h.status), h.t, h.cycle);
  }
  return SALE_OK;
}

// ---------------------------------------------------------------------------
// Launch with optional profiling events
// ---------------------------------------------------------------------------

static cudaEvent_t take_event(sale_state *st) {
  if (!st->ev_pool.empty()) {
    cudaEvent_t e = st->ev_pool.back();
    st->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// During stream capture an event record becomes a graph node only with
// cudaEventRecordExternal (a plain record is a capture-internal join point).
static void record(sale_state *st, cudaEvent_t ev) {
  if (st->capturing) cudaEventRecordWithFlags(ev, st->stream, cudaEventRecordExternal);
  else cudaEventRecord(ev, st->stream);
}

static void dispatch(sale_state *st, int kid, int mode, double dt_override) {
  if (st->precision == SALE_FP64) {
    launch_kernel(kid, fields_t<double>(st), st->S, mode, dt_override, st->diag_partial, st->diag_out, st->stream);
  } else if ((kid >= kMixNodes && kid <= kMixEos) || kid == kMixDensity || kid == kMixPredict ||
             kid == kMixHourglass) {
    launch_m_kernel(kid, fields_t<float>(st), st->S, mode, st->tile_shape, st->stream);
  } else {
    launch_kernel(kid, fields_t<float>(st), st->S, mode, dt_override, st->diag_partial, st->diag_out, st->stream);
  }
}

static void launch_k(sale_state *st, int kid, int mode = 0, double dt_override = 0.0) {
  cudaEvent_t a = nullptr;
  if (st->prof_on) {
    a = take_event(st);
    record(st, a);
  }
  dispatch(st, kid, mode, dt_override);
  if (st->prof_on) {
    cudaEvent_t b = take_event(st);
    record(st, b);
    (st->capturing ? st->capture_events : st->pending).push_back({kid, a, b});
  }
}

// Accumulate the profile of launches that completed (stream synchronised).
static void collect_profile(sale_state *st) {
  for (auto &pe : st->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) {
      st->prof_ms[pe.kid] += ms;
      st->prof_n[pe.kid] += 1;
    }
    st->ev_pool.push_back(pe.a);
    st->ev_pool.push_back(pe.b);
  }
  st->pending.clear();
  for (auto *list : st->pending_graphs)
    for (auto &pe : *list) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) {
        st->prof_ms[pe.kid] += ms;
        st->prof_n[pe.kid] += 1;
      }
    }
  st->pending_graphs.clear();
  cudaGetLastError();  // a never-recorded event is not an error of the state
}

// ---------------------------------------------------------------------------
// Initialisation
// ---------------------------------------------------------------------------

// Check a caller-provided device buffer: non-null, 256-byte aligned, large
// enough, device (or managed) memory.
static int check_device_buffer(const char *who, void *device_buf, size_t bytes, size_t need) {
  if (!device_buf) return fail(SALE_EINVAL, "%s: null device buffer", who);
  if ((uintptr_t)device_buf % kAlign) return fail(SALE_EINVAL, "%s: device buffer must be 256-byte aligned", who);
  if (bytes < need) return fail(SALE_ENOMEM, "%s: buffer has %zu bytes, need %zu", who, bytes, need);
  cudaPointerAttributes attr;
  CUDA_TRY(cudaPointerGetAttributes(&attr, device_buf));
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    return fail(SALE_EINVAL, "%s: buffer is not device memory", who);
  return SALE_OK;
}

static int state_init_at(const sale_mesh *mesh, const sale_problem_desc *prob, int precision, void *device_buf,
                         void *cuda_stream, sale_state **out);

extern "C" int sale_state_init(const sale_mesh *mesh, const sale_problem_desc *prob, int precision,
                               void *device_buf, size_t bytes, void *cuda_stream, sale_state **out) {
  if (!mesh || !prob || !out) return fail(SALE_EINVAL, "sale_state_init: null argument");
  *out = nullptr;
  if (precision != SALE_FP64 && precision != SALE_FP32_MIXED)
    return fail(SALE_EINVAL, "sale_state_init: unknown precision %d", precision);
  int rc = validate_problem(*prob);
  if (rc) return rc;
  if (prob->shear0 > 0.0 && precision != SALE_FP64)
    return fail(SALE_EINVAL, "sale_state_init: material strength runs on FP64 states");
  if (prob->nmat >= 2 && precision != SALE_FP64)
    return fail(SALE_EINVAL, "sale_state_init: several materials run on FP64 states");
  if (!mixed_fits(mesh, precision))
    return fail(SALE_EINVAL, "sale_state_init: FP32-mixed states index nodes in 32 bits (at most 2^31 - 1 nodes)");
  rc = check_device_buffer("sale_state_init", device_buf, bytes, sale_state_bytes_for(mesh, prob, precision));
  if (rc) return rc;
  return state_init_at(mesh, prob, precision, device_buf, cuda_stream, out);
}

// Initialise a state in an already checked region of device memory.
static int state_init_at(const sale_mesh *mesh, const sale_problem_desc *prob, int precision, void *device_buf,
                         void *cuda_stream, sale_state **out) {
  int rc = SALE_OK;
  sale_state *st = new (std::nothrow) sale_state;
  if (!st) return fail(SALE_ENOMEM, "sale_state_init: out of host memory");
  st->nx = mesh->d.nx;
  st->ny = mesh->d.ny;
  st->nz = mesh->d.nz;
  st->nc = mesh->nc;
  st->nn = mesh->nn;
  st->precision = precision;
  st->jit = mesh->d.jitter > 0.0;
  st->o2 = precision == SALE_FP64 && prob->remap_order == 2;
  st->pc = prob->time_order == 2;
  st->hg = prob->c_hg > 0.0;
  st->str = precision == SALE_FP64 && prob->shear0 > 0.0;
  st->nmat = precision == SALE_FP64 && prob->nmat >= 2 ? prob->nmat : 0;
  st->elem = precision == SALE_FP64 ? sizeof(double) : sizeof(float);
  st->stream = (cudaStream_t)cuda_stream;
  st->prob = *prob;
  for (int f = 0; f < 6; ++f) st->reflect[f] = mesh->d.reflect[f];
  for (int a = 0; a < 3; ++a) {
    const int n = a == 0 ? mesh->d.nx : a == 1 ? mesh->d.ny : mesh->d.nz;
    st->h32[a] = (float)((mesh->d.hi[a] - mesh->d.lo[a]) / n);
  }
  st->xpar = st->upar = 0;
  st->x_is_ref = true;
  st->remap_sets_x = 1;
  st->lim_t_end = INFINITY;
  st->lim_cycles = 0x7FFFFFFFFFFFFFFFll;
  st->failed = false;
  st->fail_code = 0;
  carve(st, (char *)device_buf);

  std::vector<double> rho0, p0;
  std::vector<float> offs;
  long long dep_cell;
  double dep_e;
  const bool mixed = precision == SALE_FP32_MIXED;
  try {
    host_primitives(*mesh, *prob, rho0, p0, dep_cell, dep_e);
    if (mixed && mesh->d.jitter > 0.0) {
      // per-node offset from the structured position lo + i*h, as FP32
      offs.assign(4 * (size_t)mesh->nn, 0.0f);
      const int n[3] = {mesh->d.nx, mesh->d.ny, mesh->d.nz};
      const std::vector<double> *src[3] = {&mesh->x, &mesh->y, &mesh->z};
      for (int a = 0; a < 3; ++a) {
        const double h = (mesh->d.hi[a] - mesh->d.lo[a]) / n[a];
        for (long long nd = 0; nd < mesh->nn; ++nd) {
          const long long sx = mesh->d.nx + 1, sxy = sx * (mesh->d.ny + 1);
          const long long idx = a == 0 ? nd % sx : a == 1 ? (nd / sx) % (mesh->d.ny + 1) : nd / sxy;
          offs[4 * nd + a] = (float)((*src[a])[nd] - (mesh->d.lo[a] + (double)idx * h));
        }
      }
    }
  } catch (...) {
    delete st;
    return fail(SALE_ENOMEM, "sale_state_init: out of host memory");
  }
  const size_t nb = sizeof(double) * mesh->nn, cb = sizeof(double) * mesh->nc;
  cudaError_t e = cudaSuccess;
  const std::vector<double> *src[3] = {&mesh->x, &mesh->y, &mesh->z};
  for (int d = 0; d < 3 && e == cudaSuccess; ++d) {
    e = cudaMemcpyAsync(st->xr[d], src[d]->data(), nb, cudaMemcpyHostToDevice, st->stream);
    if (e == cudaSuccess && !mixed)
      e = cudaMemcpyAsync(st->xs[0][d], src[d]->data(), nb, cudaMemcpyHostToDevice, st->stream);
  }
  if (mixed && !offs.empty() && e == cudaSuccess)
    e = cudaMemcpyAsync(st->off4, offs.data(), sizeof(float4) * mesh->nn, cudaMemcpyHostToDevice, st->stream);
  if (mixed && offs.empty()) st->off4 = nullptr;  // unjittered: offsets are zero
  // The per-cell FP64 primitives are staged in scratch that init does not
  // otherwise touch: FP64 p and q arrays, or (mixed) the second-role
  // velocity arrays (carved back to back: >= 12 bytes per node) and the
  // flux / swept-volume arrays from mu[0] on (36 bytes per cell).
  double *stage_rho = mixed ? (double *)st->us[1][0] : (double *)st->p;
  double *stage_p = mixed ? (double *)st->mu[0] : (double *)st->q;
  if (e == cudaSuccess) e = cudaMemcpyAsync(stage_rho, rho0.data(), cb, cudaMemcpyHostToDevice, st->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(stage_p, p0.data(), cb, cudaMemcpyHostToDevice, st->stream);
  if (e != cudaSuccess) {
    delete st;
    return cuda_fail(e, "sale_state_init: upload");
  }
  launch_reset(st->S, st->stream);
  if (st->sdev && e == cudaSuccess)  // strength: unstressed, no plastic strain
    e = cudaMemsetAsync(st->sdev, 0, sizeof(double) * 9 * (size_t)st->nc, st->stream);
  if (!mixed) {
    const Fields<double> F = fields_t<double>(st);
    // materials: the first cell index whose logical centre is at or past x_split holds material 1
    int mat_i0 = mesh->d.nx;
    const double hx = (mesh->d.hi[0] - mesh->d.lo[0]) / mesh->d.nx;
    for (int i = mesh->d.nx - 1; i >= 0 && !(mesh->d.lo[0] + ((double)i + 0.5) * hx < prob->x_split); --i) mat_i0 = i;
    launch_init_cells(F, st->S, stage_rho, stage_p, dep_cell, dep_e, mat_i0, st->stream);
    launch_kernel(kInitNodes, F, st->S, 0, 0.0, nullptr, nullptr, st->stream);
    launch_kernel(kEos, F, st->S, kDtInit, 0.0, nullptr, nullptr, st->stream);
    launch_geo_init(F, st->S, st->geoG, st->geoVE, st->geoLE, st->geoTE, st->geoIVE, st->geoIL2, st->stream);
    launch_geo_init_nodes(F, st->relE, st->stream);
    if (st->geoHG) launch_geo_init_hg(F, st->geoHG, st->stream);
  } else {
    const Fields<float> F = fields_t<float>(st);
    launch_m_init_cells(F, st->S, stage_rho, stage_p, dep_cell, dep_e, st->VE32, st->LE32, st->Gc, st->stream);
    launch_kernel(kInitNodes, F, st->S, 0, 0.0, nullptr, nullptr, st->stream);
    launch_m_kernel(kMixEos, F, st->S, kDtInit, st->tile_shape, st->stream);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);  // host vectors die here
  if (e != cudaSuccess) {
    delete st;
    return cuda_fail(e, "sale_state_init: init kernels");
  }
  DevScalars h;
  rc = sync_scalars(st, &h);
  if (rc == SALE_OK) rc = check_device_status(st, h);
  if (rc) {
    delete st;
    return rc;
  }
  *out = st;
  return SALE_OK;
}

extern "C" void sale_state_destroy(sale_state *st) {
  if (!st) return;
  cudaStreamSynchronize(st->stream);
  for (auto &kv : st->graphs) cudaGraphExecDestroy(kv.second);
  for (auto &kv : st->graph_events)
    for (auto &pe : kv.second) {
      cudaEventDestroy(pe.a);
      cudaEventDestroy(pe.b);
    }
  for (auto &pe : st->pending) {
    cudaEventDestroy(pe.a);
    cudaEventDestroy(pe.b);
  }
  for (auto ev : st->ev_pool) cudaEventDestroy(ev);
  delete st;
}

// ---------------------------------------------------------------------------
// Stepping
// ---------------------------------------------------------------------------

static int ready(const sale_state *st, const char *who) {
  if (!st) return fail(SALE_EINVAL, "%s: null state", who);
  if (st->failed) return fail(SALE_ESTATE, "%s: state failed earlier (%s)", who, status_name(st->fail_code));
  return SALE_OK;
}

static int fp64_only(const sale_state *st, const char *who) {
  if (st->precision != SALE_FP64)
    return fail(SALE_ESTATE,
                "%s: FP32-mixed states run only Eulerian cycles (sale_run_to_time with remap_every = 1)", who);
  return SALE_OK;
}

static void set_limits(sale_state *st, double t_end, long long cycles) {
  if (st->lim_t_end != t_end || st->lim_cycles != cycles) {
    launch_set_limits(st->S, t_end, cycles, st->stream);
    st->lim_t_end = t_end;
    st->lim_cycles = cycles;
  }
}

static void launch_remap(sale_state *st) {
  launch_k(st, kRemapFaces);
  launch_k(st, kRemapNodes);
  st->upar ^= 1;
  launch_k(st, kRemapCells);
}

// Eulerian cycle starting on the reference mesh: the Lagrangian positions
// stay implicit (x_ref + dt ubar) and are never written.
static void launch_ale_cycle(sale_state *st, double dt_override) {
  if (st->precision == SALE_FP32_MIXED) {
    if (st->hg) launch_k(st, kMixHourglass);
    if (st->prob.time_order == 2) launch_k(st, kMixPredict, 0, dt_override);
    launch_k(st, kMixNodes, 0, dt_override);
    launch_k(st, kMixCells, 0, dt_override);
    if (st->prob.remap_order == 2) launch_k(st, kMixDensity);
    launch_k(st, kMixFluxes);
    launch_k(st, kMixRemapNodes);
    st->upar ^= 1;
    launch_k(st, kMixRemapEos, kDtAdvance, dt_override);
    return;
  }
  if (st->hg) launch_k(st, kAleHourglass);
  if (st->prob.time_order == 2) launch_k(st, kAlePredict, 0, dt_override);
  launch_k(st, kAleNodes, 0, dt_override);
  launch_k(st, kAleEdges, 0, dt_override);
  launch_k(st, kAleCells, 0, dt_override);
  launch_k(st, kAleDensity);
  if (st->prob.remap_order == 2) launch_k(st, kAleSlopes);
  launch_k(st, kAleFluxes);
  launch_k(st, kAleRemapNodes);
  st->upar ^= 1;
  launch_k(st, kAleRemapEos, kDtAdvance, dt_override);
}

static void launch_cycle(sale_state *st, bool remap, double dt_override) {
  if (remap && st->x_is_ref) {
    launch_ale_cycle(st, dt_override);
    return;
  }
  const bool pc = st->prob.time_order == 2;
  if (st->hg) launch_k(st, kHourglass);  // hourglass corner forces of x^n, u^n
  if (pc) {  // half step: positions x^{n+1/2} (next-position buffer), then sigma^{n+1/2}
    launch_k(st, kPcPositions, 0, dt_override);
    launch_k(st, kPcPredict, 0, dt_override);
  }
  launch_k(st, kLagNodes, 0, dt_override);
  launch_k(st, kLagCells, 0, dt_override);
  if (!pc) st->xpar ^= 1;  // the corrector moves the nodes in place
  if (remap) launch_remap(st);
  launch_k(st, kEos, kDtAdvance, dt_override);
  st->x_is_ref = remap;
}

extern "C" int sale_lagrange_step(sale_state *st, double dt) {
  int rc = ready(st, "sale_lagrange_step");
  if (rc || (rc = fp64_only(st, "sale_lagrange_step"))) return rc;
  if (!std::isfinite(dt)) return fail(SALE_EINVAL, "sale_lagrange_step: dt must be finite");
  set_limits(st, INFINITY, 0x7FFFFFFFFFFFFFFFll);
  launch_cycle(st, false, dt > 0.0 ? dt : 0.0);  // leaves x off the reference mesh
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SALE_OK : cuda_fail(e, "sale_lagrange_step");
}

extern "C" int sale_remap_step(sale_state *st) {
  int rc = ready(st, "sale_remap_step");
  if (rc || (rc = fp64_only(st, "sale_remap_step"))) return rc;
  set_limits(st, INFINITY, 0x7FFFFFFFFFFFFFFFll);
  launch_remap(st);
  st->x_is_ref = true;
  launch_k(st, kEos, kDtPropose);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SALE_OK : cuda_fail(e, "sale_remap_step");
}

// Capture `k` cycles (remap after cycle j when (j+1) % remap_every == 0,
// the first cycle being aligned to the remap cadence) as one graph.
static int get_graph(sale_state *st, int k, int remap_every, cudaGraphExec_t *out) {
  GraphKey key{k, remap_every, st->xpar, st->upar, (st->prof_on ? 1 : 0) | (st->x_is_ref ? 2 : 0)};
  auto it = st->graphs.find(key);
  if (it != st->graphs.end()) {
    *out = it->second;
    if (st->prof_on) st->pending_graphs.push_back(&st->graph_events[key]);
    for (int j = 0; j < k; ++j) {  // replay the buffer-role toggles of launch_cycle
      const bool remap = remap_every > 0 && (j + 1) % remap_every == 0;
      if (remap && st->x_is_ref) {
        st->upar ^= 1;
        continue;
      }
      if (st->prob.time_order != 2) st->xpar ^= 1;
      if (remap) st->upar ^= 1;
      st->x_is_ref = remap;
    }
    return SALE_OK;
  }
  cudaGraph_t g;
  CUDA_TRY(cudaStreamBeginCapture(st->stream, cudaStreamCaptureModeThreadLocal));
  st->capturing = true;
  st->capture_events.clear();
  for (int j = 0; j < k; ++j) launch_cycle(st, remap_every > 0 && (j + 1) % remap_every == 0, 0.0);
  st->capturing = false;
  cudaError_t e = cudaStreamEndCapture(st->stream, &g);
  if (e != cudaSuccess) return cuda_fail(e, "graph capture");
  if (st->prof_on) {
    st->graph_events[key] = st->capture_events;
    st->pending_graphs.push_back(&st->graph_events[key]);
  }
  st->capture_events.clear();
  cudaGraphExec_t ge;
  e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
  st->graphs[key] = ge;
  *out = ge;
  return SALE_OK;
}

extern "C" int sale_run_to_time(sale_state *st, double t_end, long long max_cycles, int remap_every,
                                long long *cycles_done) {
  int rc = ready(st, "sale_run_to_time");
  if (rc) return rc;
  if (cycles_done) *cycles_done = 0;
  if (std::isnan(t_end) || max_cycles < 0 || remap_every < 0)
    return fail(SALE_EINVAL, "sale_run_to_time: need t_end not NaN, max_cycles >= 0, remap_every >= 0");
  if (st->precision == SALE_FP32_MIXED && remap_every != 1) return fp64_only(st, "sale_run_to_time");
  DevScalars h;
  if ((rc = sync_scalars(st, &h))) return rc;
  if ((rc = check_device_status(st, h))) return rc;
  const long long c0 = h.cycle;
  const long long limit = max_cycles > 0x7FFFFFFFFFFFFFFFll - c0 ? 0x7FFFFFFFFFFFFFFFll : c0 + max_cycles;
  set_limits(st, t_end, limit);
  const bool graphs = st->stream != nullptr;
  int chunk = remap_every > 0 ? remap_every : 1;
  while (chunk < 16) chunk += remap_every > 0 ? remap_every : 1;
  if (chunk % 2) chunk *= 2;
  while (h.t < t_end && h.cycle < limit) {
    const bool aligned = remap_every == 0 || h.cycle % remap_every == 0;
    // a graph only when a whole chunk of cycles is within the cycle budget
    // (cycles past t_end inside a replay are cheap no-ops)
    if (graphs && aligned && limit - h.cycle >= chunk) {
      cudaGraphExec_t ge;
      if ((rc = get_graph(st, chunk, remap_every, &ge))) return rc;
      CUDA_TRY(cudaGraphLaunch(ge, st->stream));
    } else {
      const bool remap = remap_every > 0 && (h.cycle + 1) % remap_every == 0;
      launch_cycle(st, remap, 0.0);
      CUDA_TRY(cudaGetLastError());
    }
    if ((rc = sync_scalars(st, &h))) return rc;
    if ((rc = check_device_status(st, h))) return rc;
  }
  if (cycles_done) *cycles_done = h.cycle - c0;
  return SALE_OK;
}

// ---------------------------------------------------------------------------
// Diagnostics and field access
// ---------------------------------------------------------------------------

extern "C" int sale_diagnostics(const sale_state *cst, sale_diag *out) {
  sale_state *st = const_cast<sale_state *>(cst);
  if (!st || !out) return fail(SALE_EINVAL, "sale_diagnostics: null argument");
  dispatch(st, kDiag, 0, 0.0);
  CUDA_TRY(cudaGetLastError());
  double q[8];
  CUDA_TRY(cudaMemcpyAsync(q, st->diag_out, sizeof(double) * 6, cudaMemcpyDeviceToHost, st->stream));
  DevScalars h;
  int rc = sync_scalars(st, &h);
  if (rc) return rc;
  out->t = h.t;
  out->dt = h.dt;
  out->cycle = h.cycle;
  out->mass = q[0];
  out->mom[0] = q[1];
  out->mom[1] = q[2];
  out->mom[2] = q[3];
  out->ie = q[4];
  out->ke = q[5];
  out->etot = q[4] + q[5];
  out->status = h.status;
  return check_device_status(st, h);
}

// Device array of a named field; *elem = bytes per value (8 or 4).
static void *field_ptr(const sale_state *st, const char *name, bool *node, bool *writable, size_t *elem) {
  *writable = true;
  *node = true;
  *elem = st->elem;
  const int xp = st->xpar, up = st->upar;
  const bool mixed = st->precision == SALE_FP32_MIXED;
  if (!strcmp(name, "x") || !strcmp(name, "y") || !strcmp(name, "z")) {
    const int d = name[0] - 'x';
    if (mixed) {  // positions are always the reference mesh after a cycle
      *writable = false;
      *elem = sizeof(double);
      return st->xr[d];
    }
    return st->xs[xp][d];
  }
  if (!strcmp(name, "u")) return st->us[up][0];
  if (!strcmp(name, "v")) return st->us[up][1];
  if (!strcmp(name, "w")) return st->us[up][2];
  if (!strcmp(name, "mn")) return st->mn;
  *writable = false;
  *elem = sizeof(double);
  if (!strcmp(name, "xref")) return st->xr[0];
  if (!strcmp(name, "yref")) return st->xr[1];
  if (!strcmp(name, "zref")) return st->xr[2];
  *node = false;
  *writable = true;
  *elem = st->elem;
  if (st->nmat) {  // materials: fraction, mass, energy of each; the cell totals m, e are derived
    const char *pre[3] = {"alpha", "m", "e"};
    for (int q = 0; q < 3; ++q) {
      const size_t l = strlen(pre[q]);
      if (!strncmp(name, pre[q], l) && name[l] >= '0' && name[l] < '0' + st->nmat && name[l + 1] == 0)
        return st->mat + (size_t)(3 * (name[l] - '0') + q) * (size_t)st->nc;
    }
    *writable = false;
  }
  if (!strcmp(name, "m")) return st->m;
  if (!strcmp(name, "e")) return st->e;
  *writable = true;
  if (st->sdev) {  // strength: deviatoric stress components and plastic strain
    static const char *const snames[7] = {"sxx", "syy", "szz", "sxy", "syz", "szx", "eps_p"};
    for (int q = 0; q < 7; ++q)
      if (!strcmp(name, snames[q])) return st->sdev + (size_t)q * (size_t)st->nc;
  }
  *writable = false;
  if (!strcmp(name, "rho")) return st->rho;
  if (!strcmp(name, "p")) return st->p;
  if (!strcmp(name, "q")) return st->q;
  if (!strcmp(name, "cs")) return st->cs;
  if (!strcmp(name, "vol")) return st->vol;
  return nullptr;
}

// FP32-mixed states: the per-face flux and swept-volume arrays (mu, ep, dv;
// carved back to back, >= 36 bytes per cell) hold nothing between cycles, so
// field transfers stage FP64 values there and convert them on the device.
static void mixed_stage(const sale_state *st, double **buf, size_t *cap) {
  char *b = (char *)st->mu[0];
  char *e = (char *)st->dv[2] + sizeof(float) * (size_t)st->nc;
  *buf = (double *)b;
  *cap = (size_t)(e - b) / sizeof(double);
}

static float *mixed_lo(const sale_state *st, const char *name) {
  return !strcmp(name, "m") ? st->mlo : !strcmp(name, "e") ? st->elo : !strcmp(name, "mn") ? st->mnlo : nullptr;
}

extern "C" int sale_copy_field(const sale_state *cst, const char *name, double *host_out, size_t n) {
  sale_state *st = const_cast<sale_state *>(cst);
  if (!st || !name || !host_out) return fail(SALE_EINVAL, "sale_copy_field: null argument");
  bool node, wr;
  size_t elem;
  void *p = field_ptr(st, name, &node, &wr, &elem);
  if (!p) return fail(SALE_EINVAL, "sale_copy_field: unknown field '%s'", name);
  const size_t want = (size_t)(node ? st->nn : st->nc);
  if (n != want) return fail(SALE_EINVAL, "sale_copy_field: '%s' has %zu values, got n = %zu", name, want, n);
  if (st->precision == SALE_FP32_MIXED && !node && !st->failed &&
      (!strcmp(name, "p") || !strcmp(name, "q") || !strcmp(name, "cs") || !strcmp(name, "vol")))
    dispatch(st, kMixEos, -1, 0.0);  // the mixed cycle stores only rho and p+q
  const bool cs_from_e = st->precision == SALE_FP64 && !st->nmat && !strcmp(name, "cs");
  if (cs_from_e) {
    // FP64: the sound speed is a function of e, sqrt(gamma (gamma - 1)
    // max(e, 0)), which the Eulerian kernels do not store; the same IEEE
    // operations on the host give the device's value bit for bit
    CUDA_TRY(cudaMemcpyAsync(host_out, st->e, sizeof(double) * n, cudaMemcpyDeviceToHost, st->stream));
    CUDA_TRY(cudaStreamSynchronize(st->stream));
    const double g = st->prob.gamma;
    for (size_t i = 0; i < n; ++i) host_out[i] = std::sqrt(g * (g - 1.0) * std::fmax(host_out[i], 0.0));
  } else if (elem == sizeof(double)) {
    CUDA_TRY(cudaMemcpyAsync(host_out, p, sizeof(double) * n, cudaMemcpyDeviceToHost, st->stream));
  } else {
    // FP32 field (plus its low part for float-float quantities): widened to
    // FP64 on the device in staging-sized chunks, then copied out
    double *stage;
    size_t cap;
    mixed_stage(st, &stage, &cap);
    const float *lo = mixed_lo(st, name);
    for (size_t off = 0; off < n; off += cap) {
      const size_t k = std::min(cap, n - off);
      launch_join64((const float *)p + off, lo ? lo + off : nullptr, stage, (long long)k, st->stream);
      CUDA_TRY(cudaGetLastError());
      CUDA_TRY(cudaMemcpyAsync(host_out + off, stage, sizeof(double) * k, cudaMemcpyDeviceToHost, st->stream));
    }
  }
  DevScalars h;
  int rc = sync_scalars(st, &h);
  if (rc) return rc;
  return check_device_status(st, h);
}

extern "C" int sale_set_field(sale_state *st, const char *name, const double *host_in, size_t n) {
  int rc = ready(st, "sale_set_field");
  if (rc) return rc;
  if (!name || !host_in) return fail(SALE_EINVAL, "sale_set_field: null argument");
  bool node, wr;
  size_t elem;
  void *p = field_ptr(st, name, &node, &wr, &elem);
  if (!p || !wr) return fail(SALE_EINVAL, "sale_set_field: '%s' is not a settable field", name);
  const size_t want = (size_t)(node ? st->nn : st->nc);
  if (n != want) return fail(SALE_EINVAL, "sale_set_field: '%s' has %zu values, got n = %zu", name, want, n);
  if (elem == sizeof(double)) {
    CUDA_TRY(cudaMemcpyAsync(p, host_in, sizeof(double) * n, cudaMemcpyHostToDevice, st->stream));
    double *inv = !strcmp(name, "m") ? st->im : !strcmp(name, "mn") ? st->imn : nullptr;
    if (inv) {
      launch_recip((const double *)p, inv, (long long)n, st->stream);
      CUDA_TRY(cudaGetLastError());
    }
  } else {
    // FP32 field: FP64 values staged on the device in chunks and split there
    // into the FP32 value and, for float-float quantities, its low part
    double *stage;
    size_t cap;
    mixed_stage(st, &stage, &cap);
    float *lo = mixed_lo(st, name);
    for (size_t off = 0; off < n; off += cap) {
      const size_t k = std::min(cap, n - off);
      CUDA_TRY(cudaMemcpyAsync(stage, host_in + off, sizeof(double) * k, cudaMemcpyHostToDevice, st->stream));
      launch_split64(stage, (float *)p + off, lo ? lo + off : nullptr, (long long)k, st->stream);
      CUDA_TRY(cudaGetLastError());
    }
  }
  if (!strcmp(name, "x") || !strcmp(name, "y") || !strcmp(name, "z")) st->x_is_ref = false;
  return SALE_OK;
}

extern "C" int sale_refresh(sale_state *st) {
  int rc = ready(st, "sale_refresh");
  if (rc) return rc;
  // on the reference mesh the FP64 refresh reads the cached geometry
  if (st->nmat) launch_mat_totals(fields_t<double>(st), st->stream);  // m, e from the uploaded materials
  launch_k(st, st->precision == SALE_FP64 ? (st->x_is_ref && !st->str && !st->nmat ? kAleEos : kEos) : kMixEos,
           kDtPropose);
  CUDA_TRY(cudaGetLastError());
  return SALE_OK;
}

extern "C" int sale_tile_shape(int shape, int *tx, int *ty) {
  if (shape < 0 || shape >= kNumTileShapes) return fail(SALE_EINVAL, "sale_tile_shape: shape in [0, %d)", kNumTileShapes);
  if (tx) *tx = tile_x(shape);
  if (ty) *ty = tile_y(shape);
  return SALE_OK;
}

extern "C" int sale_set_tiling(sale_state *st, int shape) {
  if (!st) return fail(SALE_EINVAL, "sale_set_tiling: null state");
  if (st->precision != SALE_FP32_MIXED) return fail(SALE_EINVAL, "sale_set_tiling: applies to FP32-mixed states");
  if (shape < 0 || shape >= kNumTileShapes) return fail(SALE_EINVAL, "sale_set_tiling: shape in [0, %d)", kNumTileShapes);
  if (shape == st->tile_shape) return SALE_OK;
  CUDA_TRY(cudaStreamSynchronize(st->stream));
  for (auto &kv : st->graphs) cudaGraphExecDestroy(kv.second);  // captured with the old launch shapes
  st->graphs.clear();
  st->graph_events.clear();
  st->pending_graphs.clear();
  st->tile_shape = shape;
  return SALE_OK;
}

extern "C" int sale_state_dims(const sale_state *st, long long *ncells, long long *nnodes) {
  if (!st) return fail(SALE_EINVAL, "sale_state_dims: null state");
  if (ncells) *ncells = st->nc;
  if (nnodes) *nnodes = st->nn;
  return SALE_OK;
}

// ---------------------------------------------------------------------------
// Batches: many independent meshes advanced by one graph launch
// ---------------------------------------------------------------------------

namespace sale {
void launch_m_batch(int kid, const BatchItem *items, const int4 *tab, unsigned nblocks, int shape, bool any_jit,
                    cudaStream_t st);
void launch_batch_limits(const BatchItem *items, int n, long long cycles, cudaStream_t st);
void launch_batch_gather(const BatchItem *items, int n, BatchStatus *out, cudaStream_t st);
}  // namespace sale

struct sale_batch {
  int n;
  cudaStream_t stream;
  std::vector<sale_state *> st;     // one state per mesh, carved from the batch buffer
  BatchItem *items[2];              // per velocity-buffer parity
  int4 *tab_cell, *tab_node;        // block -> (mesh, tile x, tile y, plane)
  int4 *tab_chunk;                  // node remap: block -> (mesh, tile x, tile y, chunk of kRemapChunk planes)
  int4 *tab_eos;                    // remap + EoS: block -> (mesh, tile x, tile y, chunk of kEosPlanes planes)
  unsigned nb_cell, nb_node, nb_chunk, nb_eos;
  BatchStatus *status;              // device gather area
  std::vector<int> item_upar;       // each mesh's velocity parity when the descriptors were built
  std::vector<sale_mesh_desc> meshes;
  int shape = 0;                    // thread-tile shape
  bool any_order2 = false;          // some mesh uses the second-order remap
  bool any_jit = false;             // some mesh is jittered (its kernels carry both bodies)
  int order = 0;                    // 0: meshes in input order, 1: largest mesh first
  std::map<long long, cudaGraphExec_t> graphs;
};

// Tiles of a thread-tile shape per plane, as the mixed kernels lay threads out.
static unsigned tiles_of(int ni, int nj, int nk, int shape) {
  const int tx = tile_x(shape), ty = tile_y(shape);
  return (unsigned)(((ni + tx - 1) / tx) * ((nj + ty - 1) / ty) * nk);
}
static unsigned cell_tiles(const sale_mesh_desc &d, int shape) { return tiles_of(d.nx, d.ny, d.nz, shape); }
static unsigned node_tiles(const sale_mesh_desc &d, int shape) { return tiles_of(d.nx + 1, d.ny + 1, d.nz + 1, shape); }
static void append_tiles(std::vector<int4> &tab, int mesh, int ni, int nj, int nk, int shape) {
  const int tx = tile_x(shape), ty = tile_y(shape);
  for (int k = 0; k < nk; ++k)  // k: plane, or chunk of planes
    for (int by = 0; by < (nj + ty - 1) / ty; ++by)
      for (int bx = 0; bx < (ni + tx - 1) / tx; ++bx) tab.push_back(make_int4(mesh, bx, by, k));
}

// Layout of a batch buffer: header (descriptors, block tables, status
// gather area) then one state region per mesh.
static size_t batch_layout(int n, const sale_mesh_desc *meshes, int precision, size_t *state_off, size_t *hdr_parts) {
  long long nbc = 0, nbn = 0;  // the largest tables over the tile shapes
  for (int sh = 0; sh < kNumTileShapes; ++sh) {
    long long c = 0, nd = 0;
    for (int i = 0; i < n; ++i) {
      c += cell_tiles(meshes[i], sh);
      nd += node_tiles(meshes[i], sh);
    }
    nbc = std::max(nbc, c);
    nbn = std::max(nbn, nd);
  }
  size_t off = 0;
  hdr_parts[0] = off;  // descriptors, two parities
  off = align_up(off + 2 * sizeof(BatchItem) * n);
  hdr_parts[1] = off;  // cell block table
  off = align_up(off + sizeof(int4) * nbc);
  hdr_parts[2] = off;  // node block table
  off = align_up(off + sizeof(int4) * nbn);
  hdr_parts[4] = off;  // node-remap chunk table (no larger than the node table)
  off = align_up(off + sizeof(int4) * nbn);
  hdr_parts[5] = off;  // remap + EoS chunk table (no larger than the cell table)
  off = align_up(off + sizeof(int4) * nbc);
  hdr_parts[3] = off;  // status gather
  off = align_up(off + sizeof(BatchStatus) * n);
  for (int i = 0; i < n; ++i) {
    const sale_mesh_desc &d = meshes[i];
    const long long nc = (long long)d.nx * d.ny * d.nz, nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    if (state_off) state_off[i] = off;
    off = align_up(off + state_bytes(nc, nn, precision, d.jitter > 0.0));
  }
  return off;
}

extern "C" size_t sale_batch_bytes(int n, const sale_mesh_desc *meshes, int precision) {
  if (n < 1 || !meshes || precision != SALE_FP32_MIXED) return 0;
  for (int i = 0; i < n; ++i) {
    if (meshes[i].nx < 1 || meshes[i].ny < 1 || meshes[i].nz < 1) return 0;
    if ((long long)(meshes[i].nx + 1) * (meshes[i].ny + 1) * (meshes[i].nz + 1) > 0x7FFFFFFFll) return 0;
  }
  size_t parts[6];
  return batch_layout(n, meshes, precision, nullptr, parts);
}

extern "C" void sale_batch_destroy(sale_batch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
  for (auto *st : b->st) sale_state_destroy(st);
  delete b;
}

// Descriptors relative to each mesh's current velocity-buffer parity:
// items[0] as the buffers are now, items[1] with the two roles swapped.
static int upload_batch_items(sale_batch *b) {
  std::vector<BatchItem> h((size_t)b->n);
  for (int rel = 0; rel < 2; ++rel) {
    for (int i = 0; i < b->n; ++i) {
      sale_state *st = b->st[i];
      const int keep = st->upar;
      st->upar = keep ^ rel;
      h[i].F = fields_t<float>(st);
      st->upar = keep;
      h[i].S = st->S;
      h[i].nblk_cell = tiles_of(st->nx, st->ny, (st->nz + kEosPlanes - 1) / kEosPlanes, b->shape);
      h[i].pad = 0;
    }
    CUDA_TRY(cudaMemcpyAsync(b->items[rel], h.data(), sizeof(BatchItem) * b->n, cudaMemcpyHostToDevice, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));  // h is rewritten next
  }
  b->item_upar.resize(b->n);
  for (int i = 0; i < b->n; ++i) b->item_upar[i] = b->st[i]->upar;
  return SALE_OK;
}

// Block tables for the batch's tile shape and mesh order.
static int upload_batch_tables(sale_batch *b) {
  std::vector<int> ord((size_t)b->n);
  for (int i = 0; i < b->n; ++i) ord[i] = i;
  if (b->order == 1)  // largest meshes first: their blocks start early, the short tail is small meshes
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) { return b->st[a]->nc > b->st[c]->nc; });
  std::vector<int4> tc, tn, tk, te;
  try {
    for (int i : ord) {
      const sale_mesh_desc &d = b->meshes[i];
      append_tiles(tc, i, d.nx, d.ny, d.nz, b->shape);
      append_tiles(tn, i, d.nx + 1, d.ny + 1, d.nz + 1, b->shape);
      append_tiles(tk, i, d.nx + 1, d.ny + 1, (d.nz + 1 + kRemapChunk - 1) / kRemapChunk, b->shape);
      append_tiles(te, i, d.nx, d.ny, (d.nz + kEosPlanes - 1) / kEosPlanes, b->shape);
    }
  } catch (...) {
    return fail(SALE_ENOMEM, "batch: out of host memory");
  }
  b->nb_cell = (unsigned)tc.size();
  b->nb_node = (unsigned)tn.size();
  b->nb_chunk = (unsigned)tk.size();
  b->nb_eos = (unsigned)te.size();
  CUDA_TRY(cudaMemcpyAsync(b->tab_cell, tc.data(), sizeof(int4) * tc.size(), cudaMemcpyHostToDevice, b->stream));
  CUDA_TRY(cudaMemcpyAsync(b->tab_node, tn.data(), sizeof(int4) * tn.size(), cudaMemcpyHostToDevice, b->stream));
  CUDA_TRY(cudaMemcpyAsync(b->tab_chunk, tk.data(), sizeof(int4) * tk.size(), cudaMemcpyHostToDevice, b->stream));
  CUDA_TRY(cudaMemcpyAsync(b->tab_eos, te.data(), sizeof(int4) * te.size(), cudaMemcpyHostToDevice, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));  // tc, tn, tk, te die here
  return SALE_OK;
}

extern "C" int sale_batch_create(int n, const sale_mesh_desc *meshes, const sale_problem_desc *probs,
                                 int precision, void *device_buf, size_t bytes, void *cuda_stream,
                                 sale_batch **out) {
  if (!out) return fail(SALE_EINVAL, "sale_batch_create: null out");
  *out = nullptr;
  if (n < 1 || !meshes || !probs) return fail(SALE_EINVAL, "sale_batch_create: need n >= 1, meshes, problems");
  if (precision != SALE_FP32_MIXED)
    return fail(SALE_EINVAL, "sale_batch_create: batches run the FP32-mixed Eulerian cycle (precision %d)",
                SALE_FP32_MIXED);
  if (!cuda_stream) return fail(SALE_EINVAL, "sale_batch_create: a non-default stream is required (graph capture)");
  for (int i = 0; i < n; ++i) {
    int rc = validate_problem(probs[i]);
    if (rc) return fail(rc, "sale_batch_create: mesh %d: %s", i, sale_last_error());
    if (probs[i].time_order == 2 || probs[i].c_hg > 0.0 || probs[i].shear0 > 0.0 || probs[i].nmat >= 2)
      return fail(SALE_EINVAL,
                  "sale_batch_create: mesh %d: batches run the single-stage step of one material without hourglass "
                  "control or strength",
                  i);
  }
  std::vector<size_t> soff((size_t)n);
  size_t parts[6];
  const size_t need = batch_layout(n, meshes, precision, soff.data(), parts);
  int rc = check_device_buffer("sale_batch_create", device_buf, bytes, need);
  if (rc) return rc;
  sale_batch *b = new (std::nothrow) sale_batch;
  if (!b) return fail(SALE_ENOMEM, "sale_batch_create: out of host memory");
  char *base = (char *)device_buf;
  b->n = n;
  b->stream = (cudaStream_t)cuda_stream;
  b->items[0] = (BatchItem *)(base + parts[0]);
  b->items[1] = b->items[0] + n;
  b->tab_cell = (int4 *)(base + parts[1]);
  b->tab_node = (int4 *)(base + parts[2]);
  b->tab_chunk = (int4 *)(base + parts[4]);
  b->tab_eos = (int4 *)(base + parts[5]);
  b->status = (BatchStatus *)(base + parts[3]);
  for (int i = 0; i < n; ++i) {
    sale_mesh *m = nullptr;
    sale_state *sti = nullptr;
    rc = sale_mesh_create(&meshes[i], &m);
    if (rc == SALE_OK) rc = state_init_at(m, &probs[i], precision, base + soff[i], cuda_stream, &sti);
    sale_mesh_destroy(m);
    if (rc) {
      const std::string msg = sale_last_error();
      sale_batch_destroy(b);
      return fail(rc, "sale_batch_create: mesh %d: %s", i, msg.c_str());
    }
    b->st.push_back(sti);
  }
  b->meshes.assign(meshes, meshes + n);
  for (int i = 0; i < n; ++i) b->any_order2 = b->any_order2 || probs[i].remap_order == 2;
  for (int i = 0; i < n; ++i) b->any_jit = b->any_jit || meshes[i].jitter > 0.0;
  rc = upload_batch_tables(b);
  if (rc == SALE_OK) rc = upload_batch_items(b);
  if (rc) {
    sale_batch_destroy(b);
    return rc;
  }
  *out = b;
  return SALE_OK;
}

extern "C" sale_state *sale_batch_state(sale_batch *b, int i) {
  if (!b || i < 0 || i >= b->n) return nullptr;
  return b->st[i];
}

// One cycle of every mesh: the four kernels before the velocity-buffer
// toggle read descriptors of parity p, the fused remap/EoS/dt one p ^ 1.
static void launch_batch_cycle(sale_batch *b, int p) {
  launch_m_batch(kMixNodes, b->items[p], b->tab_node, b->nb_node, b->shape, b->any_jit, b->stream);
  launch_m_batch(kMixCells, b->items[p], b->tab_cell, b->nb_cell, b->shape, b->any_jit, b->stream);
  if (b->any_order2)  // first-order meshes leave this pass at once
    launch_m_batch(kMixDensity, b->items[p], b->tab_cell, b->nb_cell, b->shape, b->any_jit, b->stream);
  launch_m_batch(kMixFluxes, b->items[p], b->tab_cell, b->nb_cell, b->shape, b->any_jit, b->stream);
  launch_m_batch(kMixRemapNodes, b->items[p], b->tab_chunk, b->nb_chunk, b->shape, b->any_jit, b->stream);
  launch_m_batch(kMixRemapEos, b->items[p ^ 1], b->tab_eos, b->nb_eos, b->shape, b->any_jit, b->stream);
}

extern "C" int sale_batch_set_schedule(sale_batch *b, int shape, int order) {
  if (!b) return fail(SALE_EINVAL, "sale_batch_set_schedule: null batch");
  if (shape < 0 || shape >= kNumTileShapes || (order != 0 && order != 1))
    return fail(SALE_EINVAL, "sale_batch_set_schedule: shape in [0, %d), order 0 or 1", kNumTileShapes);
  if (shape == b->shape && order == b->order) return SALE_OK;
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);  // they bake in the old tables
  b->graphs.clear();
  b->shape = shape;
  b->order = order;
  for (auto *st : b->st) st->tile_shape = shape;
  int rc = upload_batch_tables(b);
  if (rc == SALE_OK) rc = upload_batch_items(b);
  return rc;
}

// Cycles per replayed batch graph (even; see sale_batch_run).
constexpr long long kBatchChunk = 64;
static_assert(kBatchChunk % 2 == 0, "a batch chunk must keep the velocity roles");

// The instantiated graph of n cycles of every mesh (captured on first use).
static int batch_graph(sale_batch *b, long long n, cudaGraphExec_t *out) {
  auto it = b->graphs.find(n);
  if (it != b->graphs.end()) {
    *out = it->second;
    return SALE_OK;
  }
  cudaGraph_t g;
  CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  int p = 0;
  for (long long j = 0; j < n; ++j, p ^= 1) launch_batch_cycle(b, p);
  cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (e != cudaSuccess) return cuda_fail(e, "sale_batch_run: graph capture");
  cudaGraphExec_t ge;
  e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "sale_batch_run: graph instantiate");
  b->graphs[n] = ge;
  *out = ge;
  return SALE_OK;
}

extern "C" int sale_batch_run(sale_batch *b, long long cycles, int remap_every, long long *cycles_done) {
  if (!b) return fail(SALE_EINVAL, "sale_batch_run: null batch");
  if (cycles_done) *cycles_done = 0;
  if (cycles < 0 || cycles > (1ll << 20)) return fail(SALE_EINVAL, "sale_batch_run: cycles must be in [0, 2^20]");
  if (remap_every != 1)
    return fail(SALE_EINVAL, "sale_batch_run: batches run Eulerian cycles (remap_every = 1)");
  for (auto *st : b->st) {
    int rc = ready(st, "sale_batch_run");
    if (rc) return rc;
    st->lim_t_end = NAN;  // the batch sets the device limits; force a reset on the next single-mesh call
  }
  if (cycles == 0) return SALE_OK;
  for (int i = 0; i < b->n; ++i)
    if (b->st[i]->upar != b->item_upar[i]) {  // a mesh was advanced on its own since
      int rc = upload_batch_items(b);
      if (rc) return rc;
      break;
    }
  launch_batch_limits(b->items[0], b->n, cycles, b->stream);
  // Replays of a graph of kBatchChunk cycles of every mesh, then one graph
  // of the remaining cycles: at most kBatchChunk graphs are ever kept, and
  // an even chunk leaves every mesh's velocity roles as they were, so each
  // graph starts from the same descriptors.
  const long long full = cycles / kBatchChunk, rest = cycles % kBatchChunk;
  cudaGraphExec_t ge;
  if (full > 0) {
    int rc = batch_graph(b, kBatchChunk, &ge);
    if (rc) return rc;
    for (long long r = 0; r < full; ++r) CUDA_TRY(cudaGraphLaunch(ge, b->stream));
  }
  if (rest > 0) {
    int rc = batch_graph(b, rest, &ge);
    if (rc) return rc;
    CUDA_TRY(cudaGraphLaunch(ge, b->stream));
  }
  if (cycles & 1)  // odd run: every mesh's velocity roles swapped
    for (auto *st : b->st) st->upar ^= 1;
  launch_batch_gather(b->items[0], b->n, b->status, b->stream);
  std::vector<BatchStatus> hs((size_t)b->n);
  CUDA_TRY(cudaMemcpyAsync(hs.data(), b->status, sizeof(BatchStatus) * b->n, cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  if (cycles & 1) {  // descriptors follow the swapped roles (graphs keep their array pointers)
    int rc = upload_batch_items(b);
    if (rc) return rc;
  }
  for (int i = 0; i < b->n; ++i) {
    if (hs[i].status != 0) {
      b->st[i]->failed = true;
      b->st[i]->fail_code = (int)hs[i].status;
      return fail((int)hs[i].status, "sale_batch_run: mesh %d: %s (t = %.17g, cycle %lld)", i,
                  status_name((int)hs[i].status), hs[i].t, hs[i].cycle);
    }
  }
  if (cycles_done) *cycles_done = cycles;
  return SALE_OK;
}

// ---------------------------------------------------------------------------
// Launch-time profile
// ---------------------------------------------------------------------------

static const char *const kKernelNames[kNumKernels] = {
    "init_nodes",   "eos_dt",    "lagrange_nodes", "lagrange_cells", "remap_faces",     "remap_nodes",
    "remap_cells",  "diagnostics", "ale_nodes",    "ale_cells",      "ale_density",     "ale_fluxes",
    "ale_remap_eos", "geo_init",  "mix_nodes",     "mix_cells",      "mix_fluxes",      "mix_remap_nodes",
    "mix_remap_eos", "mix_eos",   "ale_edges",   "ale_remap_nodes", "ale_eos",     "ale_slopes",
    "mix_density",  "pc_positions", "pc_predict", "ale_predict", "mix_predict", "hourglass",
    "ale_hourglass", "mix_hourglass"};

extern "C" int sale_kernel_count(void) { return kNumKernels; }

extern "C" const char *sale_kernel_name(int id) {
  return (id >= 0 && id < kNumKernels) ? kKernelNames[id] : nullptr;
}

extern "C" int sale_profile(sale_state *st, int on) {
  if (!st) return fail(SALE_EINVAL, "sale_profile: null state");
  st->prof_on = on != 0;
  return SALE_OK;
}

extern "C" int sale_profile_read(sale_state *st, double *ms, long long *launches, int n, int reset) {
  if (!st) return fail(SALE_EINVAL, "sale_profile_read: null state");
  if (n < 0 || n > kNumKernels) return fail(SALE_EINVAL, "sale_profile_read: n must be in [0, %d]", kNumKernels);
  DevScalars h;
  int rc = sync_scalars(st, &h);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    if (ms) ms[i] = st->prof_ms[i];
    if (launches) launches[i] = st->prof_n[i];
  }
  if (reset)
    for (int i = 0; i < kNumKernels; ++i) {
      st->prof_ms[i] = 0.0;
      st->prof_n[i] = 0;
    }
  return SALE_OK;
}

extern "C" const char *sale_last_error(void) { return g_last_error.c_str(); }
