// fit_apply_noalloc: the operator apply without any device allocation.
//
// fit_apply keeps the per-system angular frequencies in a device buffer owned by the grid handle
// and grows that buffer with cudaMalloc whenever a call brings a larger batch.  Some callers must
// not allocate: a host thread driving a latency-critical loop (cudaMalloc / cudaFree may
// synchronise the whole device and stall it), or a framework that owns all device memory through
// its own pool and must not see raw allocations behind its back.  This entry point keeps the
// frequencies in a fixed static device array instead, so it never allocates.
#include <mutex>

#include "fit_internal.cuh"

// Static scratch for the frequencies: FIT_NOALLOC_MAX_BATCH doubles (32 KiB), resident on every
// device that loads the library until the process exits.  In host code the symbol is only a
// stand-in: its device address comes from cudaGetSymbolAddress.
#define FIT_NOALLOC_MAX_BATCH 4096
static __device__ __align__(256) double g_noalloc_omega[FIT_NOALLOC_MAX_BATCH];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_addr[kMaxDevices] = {};

// once per device, with that device current: look up the array's device address.  The cached address
// belongs to the device's primary context; a cudaDeviceReset of the device would make it stale, which is
// why the header rules out calls after such a reset.
fit_status noalloc_scratch(int device, double** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (device < 0 || device >= kMaxDevices) {
    fit_set_error("fit_apply_noalloc: device index out of range");
    return FIT_EINVAL;
  }
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_omega);
    if (e != cudaSuccess || !p) {
      fit_set_error(std::string("fit_apply_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return FIT_ECUDA;
    }
    g_noalloc_addr[device] = (double*)p;
  }
  *out = g_noalloc_addr[device];
  return FIT_OK;
}
}  // namespace

// launch without the autotuner (defined with the fused kernels)
fit_status fit_launch_apply_fixed(fit_grid* g, int nbatch, const double* omega_dev, const void* x, void* y,
                                  fit_prec prec, double out_scale, cudaStream_t s);

extern "C" fit_status fit_apply_noalloc(fit_grid* g, int nbatch, const double* omega, const void* x, void* y,
                                        fit_prec prec, void* stream) {
  FIT_REQUIRE(g && omega && x && y, "fit_apply_noalloc: null argument");
  FIT_REQUIRE(nbatch >= 1, "fit_apply_noalloc: nbatch must be >= 1");
  FIT_REQUIRE(nbatch <= FIT_NOALLOC_MAX_BATCH,
              "fit_apply_noalloc: nbatch exceeds the static frequency scratch (4096 systems per call)");
  FIT_REQUIRE(prec == FIT_C64 || prec == FIT_C128, "fit_apply_noalloc: unknown precision");
  FIT_REQUIRE(g->has_materials, "fit_apply_noalloc: materials not set");
  for (int b = 0; b < nbatch; ++b) FIT_REQUIRE(isfinite(omega[b]), "fit_apply_noalloc: omega must be finite");
  if (fit_check_abort(g, "fit_apply_noalloc") != FIT_OK) return FIT_ETIMEOUT;
  const size_t vbytes = (size_t)g->ne * (prec == FIT_C64 ? sizeof(float2) : sizeof(double2)) * nbatch;
  const char* xb = (const char*)x;
  const char* yb = (const char*)y;
  FIT_REQUIRE(xb + vbytes <= yb || yb + vbytes <= xb, "fit_apply_noalloc: x and y overlap");
  FIT_CHECK_CUDA(cudaSetDevice(g->device));
  double* om = nullptr;
  fit_status st = noalloc_scratch(g->device, &om);
  if (st != FIT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // every call overwrites the nbatch entries it uses, so nothing has to start at zero
  FIT_CHECK_CUDA(cudaMemcpyAsync(om, omega, nbatch * sizeof(double), cudaMemcpyHostToDevice, s));
  const double out_scale = prec == FIT_C64 ? 1.0 / g->coef_scale : 1.0;
  return fit_launch_apply_fixed(g, nbatch, om, x, y, prec, out_scale, s);
}
