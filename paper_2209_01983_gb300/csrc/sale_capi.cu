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
void launch_init_cells(const Fields<R> &, DevScalars *, const double *, const double *, long long, double,
                       cudaStream_t);
template <typename R>
void launch_kernel(int kid, const Fields<R> &, DevScalars *, int mode, double dt_override, double *partial,
                   double *out, cudaStream_t);
void launch_geo_init(const Fields<double> &F, DevScalars *S, double *G, double *VE, double *LE, double *TE,
                     cudaStream_t st);
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
constexpr int kNodeArrays = 17;  // xr,yr,zr, x(2x3), u(2x3), mn, dke
constexpr int kCellArrays = 17;  // m,e,sig,rho,p,q,cs,vol, mu(3), ep(3), dv(3)
constexpr int kGeoPerCell = 29;  // cached reference geometry: 24 corner gradients, V_E, L_E, 3 face terms
constexpr int kDiagBlocks = 512;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t scalars, diag_partial, diag_out, node[kNodeArrays], cell[kCellArrays], geo, total;
};

Layout make_layout(long long nc, long long nn, size_t elem) {
  Layout L;
  size_t off = 0;
  L.scalars = off;
  off = align_up(off + sizeof(DevScalars));
  L.diag_partial = off;
  off = align_up(off + sizeof(double) * 6 * kDiagBlocks);
  L.diag_out = off;
  off = align_up(off + sizeof(double) * 8);
  for (int a = 0; a < kNodeArrays; ++a) {
    L.node[a] = off;
    // the reference mesh is FP64 in every precision
    off = align_up(off + (a < 3 ? sizeof(double) : elem) * (size_t)nn);
  }
  for (int a = 0; a < kCellArrays; ++a) {
    L.cell[a] = off;
    off = align_up(off + elem * (size_t)nc);
  }
  // one contiguous block: the corner gradients are indexed with stride nc
  L.geo = off;
  off = align_up(off + elem * (size_t)kGeoPerCell * (size_t)nc);
  L.total = off;
  return L;
}

}  // namespace

struct GraphKey {
  int k, remap_every, xpar, upar, prof;
  bool operator<(const GraphKey &o) const {
    return std::tie(k, remap_every, xpar, upar, prof) < std::tie(o.k, o.remap_every, o.xpar, o.upar, o.prof);
  }
};

struct ProfEvent {
  int kid;
  cudaEvent_t a, b;
};

struct sale_state {
  int nx, ny, nz;
  long long nc, nn;
  int precision;
  cudaStream_t stream;
  char *base;
  DevScalars *S;
  double *diag_partial, *diag_out;
  double *xr[3];
  double *xs[2][3];  // two position buffers
  double *us[2][3];  // two velocity buffers
  double *mn, *dke;
  double *m, *e, *sig, *rho, *p, *q, *cs, *vol, *mu[3], *ep[3], *dv[3];
  double *geoG, *geoVE, *geoLE, *geoTE;  // cached reference geometry
  int xpar, upar;
  bool x_is_ref;       // current positions are the reference mesh
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

static Fields<double> fields(const sale_state *st) {
  Fields<double> F;
  F.nx = st->nx;
  F.ny = st->ny;
  F.nz = st->nz;
  F.nc = st->nc;
  F.nn = st->nn;
  F.xr = st->xr[0];
  F.yr = st->xr[1];
  F.zr = st->xr[2];
  F.x = st->xs[st->xpar][0];
  F.y = st->xs[st->xpar][1];
  F.z = st->xs[st->xpar][2];
  F.xn = st->xs[st->xpar ^ 1][0];
  F.yn = st->xs[st->xpar ^ 1][1];
  F.zn = st->xs[st->xpar ^ 1][2];
  F.u = st->us[st->upar][0];
  F.v = st->us[st->upar][1];
  F.w = st->us[st->upar][2];
  F.ub = st->us[st->upar ^ 1][0];
  F.vb = st->us[st->upar ^ 1][1];
  F.wb = st->us[st->upar ^ 1][2];
  F.mn = st->mn;
  F.dke = st->dke;
  F.m = st->m;
  F.e = st->e;
  F.sig = st->sig;
  F.rho = st->rho;
  F.p = st->p;
  F.q = st->q;
  F.cs = st->cs;
  F.vol = st->vol;
  F.mux = st->mu[0];
  F.muy = st->mu[1];
  F.muz = st->mu[2];
  F.epx = st->ep[0];
  F.epy = st->ep[1];
  F.epz = st->ep[2];
  F.dvx = st->dv[0];
  F.dvy = st->dv[1];
  F.dvz = st->dv[2];
  F.G = st->geoG;
  F.VE = st->geoVE;
  F.LE = st->geoLE;
  F.TE = st->geoTE;
  F.remap_sets_x = st->remap_sets_x;
  F.gamma = st->prob.gamma;
  F.cfl = st->prob.cfl;
  F.c_q = st->prob.c_q;
  F.c_l = st->prob.c_l;
  F.growth = st->prob.dt_growth;
  F.dt_init = std::isfinite(st->prob.dt_init) ? st->prob.dt_init : 0.0;
  F.ke_fix = st->prob.ke_fix;
  for (int f = 0; f < 6; ++f) F.reflect[f] = st->reflect[f];
  return F;
}

extern "C" size_t sale_state_bytes(const sale_mesh *mesh, int precision) {
  if (!mesh || precision != SALE_FP64) return 0;
  return make_layout(mesh->nc, mesh->nn, sizeof(double)).total;
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

extern "C" int sale_state_init(const sale_mesh *mesh, const sale_problem_desc *prob, int precision,
                               void *device_buf, size_t bytes, void *cuda_stream, sale_state **out) {
  if (!mesh || !prob || !out) return fail(SALE_EINVAL, "sale_state_init: null argument");
  *out = nullptr;
  if (precision != SALE_FP64) return fail(SALE_EINVAL, "sale_state_init: precision %d not supported", precision);
  int rc = validate_problem(*prob);
  if (rc) return rc;
  const Layout L = make_layout(mesh->nc, mesh->nn, sizeof(double));
  if (!device_buf) return fail(SALE_EINVAL, "sale_state_init: null device buffer");
  if ((uintptr_t)device_buf % kAlign) return fail(SALE_EINVAL, "sale_state_init: device buffer must be 256-byte aligned");
  if (bytes < L.total) return fail(SALE_ENOMEM, "sale_state_init: buffer has %zu bytes, need %zu", bytes, L.total);
  cudaPointerAttributes attr;
  CUDA_TRY(cudaPointerGetAttributes(&attr, device_buf));
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    return fail(SALE_EINVAL, "sale_state_init: buffer is not device memory");

  sale_state *st = new (std::nothrow) sale_state;
  if (!st) return fail(SALE_ENOMEM, "sale_state_init: out of host memory");
  st->nx = mesh->d.nx;
  st->ny = mesh->d.ny;
  st->nz = mesh->d.nz;
  st->nc = mesh->nc;
  st->nn = mesh->nn;
  st->precision = precision;
  st->stream = (cudaStream_t)cuda_stream;
  st->prob = *prob;
  for (int f = 0; f < 6; ++f) st->reflect[f] = mesh->d.reflect[f];
  st->xpar = st->upar = 0;
  st->lim_t_end = INFINITY;
  st->lim_cycles = 0x7FFFFFFFFFFFFFFFll;
  st->failed = false;
  st->fail_code = 0;
  char *b = (char *)device_buf;
  st->base = b;
  st->S = (DevScalars *)(b + L.scalars);
  st->diag_partial = (double *)(b + L.diag_partial);
  st->diag_out = (double *)(b + L.diag_out);
  double *na[kNodeArrays];
  for (int a = 0; a < kNodeArrays; ++a) na[a] = (double *)(b + L.node[a]);
  double *ca[kCellArrays];
  for (int a = 0; a < kCellArrays; ++a) ca[a] = (double *)(b + L.cell[a]);
  for (int d = 0; d < 3; ++d) {
    st->xr[d] = na[d];
    st->xs[0][d] = na[3 + d];
    st->xs[1][d] = na[6 + d];
    st->us[0][d] = na[9 + d];
    st->us[1][d] = na[12 + d];
  }
  st->mn = na[15];
  st->dke = na[16];
  st->m = ca[0];
  st->e = ca[1];
  st->sig = ca[2];
  st->rho = ca[3];
  st->p = ca[4];
  st->q = ca[5];
  st->cs = ca[6];
  st->vol = ca[7];
  for (int d = 0; d < 3; ++d) {
    st->mu[d] = ca[8 + d];
    st->ep[d] = ca[11 + d];
    st->dv[d] = ca[14 + d];
  }
  st->geoG = (double *)(b + L.geo);
  st->geoVE = st->geoG + 24 * mesh->nc;
  st->geoLE = st->geoVE + mesh->nc;
  st->geoTE = st->geoLE + mesh->nc;
  st->x_is_ref = true;
  st->remap_sets_x = 1;

  std::vector<double> rho0, p0;
  long long dep_cell;
  double dep_e;
  try {
    host_primitives(*mesh, *prob, rho0, p0, dep_cell, dep_e);
  } catch (...) {
    delete st;
    return fail(SALE_ENOMEM, "sale_state_init: out of host memory");
  }
  const size_t nb = sizeof(double) * mesh->nn, cb = sizeof(double) * mesh->nc;
  cudaError_t e = cudaSuccess;
  const std::vector<double> *src[3] = {&mesh->x, &mesh->y, &mesh->z};
  for (int d = 0; d < 3 && e == cudaSuccess; ++d) {
    e = cudaMemcpyAsync(st->xr[d], src[d]->data(), nb, cudaMemcpyHostToDevice, st->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(st->xs[0][d], src[d]->data(), nb, cudaMemcpyHostToDevice, st->stream);
  }
  // primitives are staged in the p and q arrays, which the EoS overwrites
  if (e == cudaSuccess) e = cudaMemcpyAsync(st->p, rho0.data(), cb, cudaMemcpyHostToDevice, st->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(st->q, p0.data(), cb, cudaMemcpyHostToDevice, st->stream);
  if (e != cudaSuccess) {
    delete st;
    return cuda_fail(e, "sale_state_init: upload");
  }
  {
    const Fields<double> F = fields(st);
    launch_reset(st->S, st->stream);
    launch_init_cells(F, st->S, st->p, st->q, dep_cell, dep_e, st->stream);
    launch_kernel(kInitNodes, F, st->S, 0, 0.0, nullptr, nullptr, st->stream);
    launch_kernel(kEos, F, st->S, kDtInit, 0.0, nullptr, nullptr, st->stream);
    launch_geo_init(F, st->S, st->geoG, st->geoVE, st->geoLE, st->geoTE, st->stream);
  }
  e = cudaGetLastError();
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

static void launch_k(sale_state *st, int kid, int mode = 0, double dt_override = 0.0) {
  cudaEvent_t a = nullptr;
  if (st->prof_on) {
    a = take_event(st);
    record(st, a);
  }
  launch_kernel(kid, fields(st), st->S, mode, dt_override, st->diag_partial, st->diag_out, st->stream);
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
// Stepping
// ---------------------------------------------------------------------------

static int ready(const sale_state *st, const char *who) {
  if (!st) return fail(SALE_EINVAL, "%s: null state", who);
  if (st->failed) return fail(SALE_ESTATE, "%s: state failed earlier (%s)", who, status_name(st->fail_code));
  return SALE_OK;
}

static void set_limits(sale_state *st, double t_end, long long cycles) {
  if (st->lim_t_end != t_end || st->lim_cycles != cycles) {
    launch_set_limits(st->S, t_end, cycles, st->stream);
    st->lim_t_end = t_end;
    st->lim_cycles = cycles;
  }
}

// Kernels of one cycle on the state's stream; toggles the host's record of
// which buffers hold the current positions and velocities.
static void launch_remap(sale_state *st) {
  launch_k(st, kRemapFaces);
  launch_k(st, kRemapNodes);
  st->upar ^= 1;
  launch_k(st, kRemapCells);
}

// Eulerian cycle starting on the reference mesh: cached geometry, the
// Lagrangian positions stay implicit (x_ref + dt ubar), no position writes.
static void launch_ale_cycle(sale_state *st, double dt_override) {
  launch_k(st, kAleNodes, 0, dt_override);
  launch_k(st, kAleCells, 0, dt_override);
  launch_k(st, kAleDensity);
  launch_k(st, kAleFluxes);
  st->remap_sets_x = 0;
  launch_k(st, kRemapNodes);
  st->remap_sets_x = 1;
  st->upar ^= 1;
  launch_k(st, kAleRemapEos, kDtAdvance, dt_override);
}

static void launch_cycle(sale_state *st, bool remap, double dt_override) {
  if (remap && st->x_is_ref) {
    launch_ale_cycle(st, dt_override);
    return;
  }
  launch_k(st, kLagNodes, 0, dt_override);
  launch_k(st, kLagCells, 0, dt_override);
  st->xpar ^= 1;
  if (remap) launch_remap(st);
  launch_k(st, kEos, kDtAdvance, dt_override);
  st->x_is_ref = remap;
}

extern "C" int sale_lagrange_step(sale_state *st, double dt) {
  int rc = ready(st, "sale_lagrange_step");
  if (rc) return rc;
  if (!std::isfinite(dt)) return fail(SALE_EINVAL, "sale_lagrange_step: dt must be finite");
  set_limits(st, INFINITY, 0x7FFFFFFFFFFFFFFFll);
  launch_cycle(st, false, dt > 0.0 ? dt : 0.0);  // leaves x off the reference mesh
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SALE_OK : cuda_fail(e, "sale_lagrange_step");
}

extern "C" int sale_remap_step(sale_state *st) {
  int rc = ready(st, "sale_remap_step");
  if (rc) return rc;
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
      st->xpar ^= 1;
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
  launch_kernel(kDiag, fields(st), st->S, 0, 0.0, st->diag_partial, st->diag_out, st->stream);
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

static double *field_ptr(const sale_state *st, const char *name, bool *node, bool *writable) {
  *writable = true;
  *node = true;
  const int xp = st->xpar, up = st->upar;
  if (!strcmp(name, "x")) return st->xs[xp][0];
  if (!strcmp(name, "y")) return st->xs[xp][1];
  if (!strcmp(name, "z")) return st->xs[xp][2];
  if (!strcmp(name, "u")) return st->us[up][0];
  if (!strcmp(name, "v")) return st->us[up][1];
  if (!strcmp(name, "w")) return st->us[up][2];
  if (!strcmp(name, "mn")) return st->mn;
  *writable = false;
  if (!strcmp(name, "xref")) return st->xr[0];
  if (!strcmp(name, "yref")) return st->xr[1];
  if (!strcmp(name, "zref")) return st->xr[2];
  *node = false;
  *writable = true;
  if (!strcmp(name, "m")) return st->m;
  if (!strcmp(name, "e")) return st->e;
  *writable = false;
  if (!strcmp(name, "rho")) return st->rho;
  if (!strcmp(name, "p")) return st->p;
  if (!strcmp(name, "q")) return st->q;
  if (!strcmp(name, "cs")) return st->cs;
  if (!strcmp(name, "vol")) return st->vol;
  return nullptr;
}

extern "C" int sale_copy_field(const sale_state *st, const char *name, double *host_out, size_t n) {
  if (!st || !name || !host_out) return fail(SALE_EINVAL, "sale_copy_field: null argument");
  bool node, wr;
  double *p = field_ptr(st, name, &node, &wr);
  if (!p) return fail(SALE_EINVAL, "sale_copy_field: unknown field '%s'", name);
  const size_t want = (size_t)(node ? st->nn : st->nc);
  if (n != want) return fail(SALE_EINVAL, "sale_copy_field: '%s' has %zu values, got n = %zu", name, want, n);
  CUDA_TRY(cudaMemcpyAsync(host_out, p, sizeof(double) * n, cudaMemcpyDeviceToHost, st->stream));
  DevScalars h;
  int rc = sync_scalars(st, &h);
  if (rc) return rc;
  return check_device_status(const_cast<sale_state *>(st), h);
}

extern "C" int sale_set_field(sale_state *st, const char *name, const double *host_in, size_t n) {
  int rc = ready(st, "sale_set_field");
  if (rc) return rc;
  if (!name || !host_in) return fail(SALE_EINVAL, "sale_set_field: null argument");
  bool node, wr;
  double *p = field_ptr(st, name, &node, &wr);
  if (!p || !wr) return fail(SALE_EINVAL, "sale_set_field: '%s' is not a settable field", name);
  const size_t want = (size_t)(node ? st->nn : st->nc);
  if (n != want) return fail(SALE_EINVAL, "sale_set_field: '%s' has %zu values, got n = %zu", name, want, n);
  CUDA_TRY(cudaMemcpyAsync(p, host_in, sizeof(double) * n, cudaMemcpyHostToDevice, st->stream));
  if (!strcmp(name, "x") || !strcmp(name, "y") || !strcmp(name, "z")) st->x_is_ref = false;
  return SALE_OK;
}

extern "C" int sale_refresh(sale_state *st) {
  int rc = ready(st, "sale_refresh");
  if (rc) return rc;
  launch_k(st, kEos, kDtPropose);
  CUDA_TRY(cudaGetLastError());
  return SALE_OK;
}

extern "C" int sale_state_dims(const sale_state *st, long long *ncells, long long *nnodes) {
  if (!st) return fail(SALE_EINVAL, "sale_state_dims: null state");
  if (ncells) *ncells = st->nc;
  if (nnodes) *nnodes = st->nn;
  return SALE_OK;
}

// ---------------------------------------------------------------------------
// Launch-time profile
// ---------------------------------------------------------------------------

static const char *const kKernelNames[kNumKernels] = {
    "init_nodes", "eos_dt",    "lagrange_nodes", "lagrange_cells", "remap_faces",   "remap_nodes", "remap_cells",
    "diagnostics", "ale_nodes", "ale_cells",      "ale_density",    "ale_fluxes", "ale_remap_eos", "geo_init"};

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
