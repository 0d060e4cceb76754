// sale_static.cu -- remap step for callers that cannot allocate device
// memory (see sale_remap_static in include/sale.h).
//
// Some callers have no way to call cudaMalloc: plug-ins whose host
// application owns every device allocation and hands them only the arrays
// they work on, and loops that must not call an allocator (cudaMalloc and
// cudaFree can synchronise the device and stall every other stream).  They
// already hold their field arrays; what the remap additionally needs is
// scratch for the face fluxes, the node kinetic-energy losses and a device
// status word.  Here that scratch is one fixed file-scope device array,
// sized for at most SALE_STATIC_MAX_CELLS cells and SALE_STATIC_MAX_NODES
// nodes; it exists on every GPU that loads the library, from module load
// until process exit.
//
// Host code cannot use the array's name as a device address (it denotes a
// host-side shadow), so the device address is looked up once per device
// with cudaGetSymbolAddress, on the first call on that device, and passed
// to the kernels.  A device reset (cudaDeviceReset) unloads the module and
// leaves that address stale: the entry point is not for processes that
// reset a device they have called it on.
#include <cmath>
#include <mutex>

#include "sale_internal.cuh"

namespace sale {
template <typename R>
void launch_kernel(int kid, const Fields<R> &, DevScalars *, int mode, double dt_override, double *partial,
                   double *out, cudaStream_t);
void launch_reset(DevScalars *, cudaStream_t);
int report_error(int code, const char *fmt, ...);
}  // namespace sale

using namespace sale;

namespace {

constexpr long long kMaxCells = SALE_STATIC_MAX_CELLS;
constexpr long long kMaxNodes = SALE_STATIC_MAX_NODES;
constexpr size_t kScalarBytes = 256;  // DevScalars, padded to the alignment
static_assert(sizeof(DevScalars) <= kScalarBytes, "status block too large");
// layout: [status block][6 face-flux arrays of kMaxCells][dKE of kMaxNodes]
constexpr size_t kScratchBytes = kScalarBytes + sizeof(double) * (6 * kMaxCells + kMaxNodes);

static __device__ __align__(256) unsigned char g_remap_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
char *g_scratch[kMaxDevices] = {};  // device address of g_remap_scratch, per device

// Device address of the scratch on the current device (looked up on the
// first call for that device).
int scratch_address(char **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report_error(SALE_ECUDA, "sale_remap_static: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return report_error(SALE_EINVAL, "sale_remap_static: device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_lock);
  if (!g_scratch[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_remap_scratch);
    if (e != cudaSuccess || !p)
      return report_error(SALE_ECUDA, "sale_remap_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_scratch[dev] = (char *)p;
  }
  *out = g_scratch[dev];
  return SALE_OK;
}

}  // namespace

extern "C" int sale_remap_static(int nx, int ny, int nz, const int *reflect, int ke_fix, const double *xref,
                                 double *x, const double *u_in, double *u_out, double *mn, double *m, double *e,
                                 const double *rho, void *cuda_stream) {
  if (nx < 1 || ny < 1 || nz < 1) return report_error(SALE_EINVAL, "sale_remap_static: cell counts must be >= 1");
  const long long nc = (long long)nx * ny * nz;
  const long long nn = (long long)(nx + 1) * (ny + 1) * (nz + 1);
  if (nc > kMaxCells || nn > kMaxNodes)
    return report_error(SALE_EINVAL,
                        "sale_remap_static: mesh %dx%dx%d has %lld cells / %lld nodes; the static scratch holds at "
                        "most %lld cells and %lld nodes",
                        nx, ny, nz, nc, nn, kMaxCells, kMaxNodes);
  if (!reflect || !xref || !x || !u_in || !u_out || !mn || !m || !e || !rho)
    return report_error(SALE_EINVAL, "sale_remap_static: null argument");
  if (u_out == u_in) return report_error(SALE_EINVAL, "sale_remap_static: u_out must not alias u_in");
  for (int f = 0; f < 6; ++f)
    if (reflect[f] != 0 && reflect[f] != 1) return report_error(SALE_EINVAL, "sale_remap_static: reflect[] must be 0 or 1");

  char *base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  DevScalars *S = (DevScalars *)base;
  double *flux = (double *)(base + kScalarBytes);

  Fields<double> F = {};
  F.nx = nx;
  F.ny = ny;
  F.nz = nz;
  F.nc = nc;
  F.nn = nn;
  F.xr = xref;
  F.yr = xref + nn;
  F.zr = xref + 2 * nn;
  F.x = x;
  F.y = x + nn;
  F.z = x + 2 * nn;
  F.u = const_cast<double *>(u_in);
  F.v = const_cast<double *>(u_in) + nn;
  F.w = const_cast<double *>(u_in) + 2 * nn;
  F.ub = u_out;
  F.vb = u_out + nn;
  F.wb = u_out + 2 * nn;
  F.mn = mn;
  F.m = m;
  F.e = e;
  F.rho = const_cast<double *>(rho);
  F.mux = flux;
  F.muy = flux + kMaxCells;
  F.muz = flux + 2 * kMaxCells;
  F.epx = flux + 3 * kMaxCells;
  F.epy = flux + 4 * kMaxCells;
  F.epz = flux + 5 * kMaxCells;
  F.dke = flux + 6 * kMaxCells;
  F.ke_fix = ke_fix ? 1 : 0;
  F.remap_sets_x = 1;  // x leaves holding the reference positions
  for (int f = 0; f < 6; ++f) F.reflect[f] = reflect[f];

  // The status block starts from zero on every call (a previous call's
  // error must not leak in); the flux and dKE arrays are written in full
  // by the kernels before they are read.
  launch_reset(S, stream);
  launch_kernel(kRemapFaces, F, S, 0, 0.0, nullptr, nullptr, stream);
  launch_kernel(kRemapNodes, F, S, 0, 0.0, nullptr, nullptr, stream);
  launch_kernel(kRemapCells, F, S, 0, 0.0, nullptr, nullptr, stream);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return report_error(SALE_ECUDA, "sale_remap_static: launch: %s", cudaGetErrorString(err));
  int status = 0;
  err = cudaMemcpyAsync(&status, &S->status, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(stream);
  if (err != cudaSuccess) return report_error(SALE_ECUDA, "sale_remap_static: %s", cudaGetErrorString(err));
  if (status != 0) return report_error(status, "sale_remap_static: device reported status %d", status);
  return SALE_OK;
}
