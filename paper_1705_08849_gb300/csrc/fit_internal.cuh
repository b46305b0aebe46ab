// Internal definitions shared by the translation units of the FIT library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/fit.h"

// Physical constants: mu0 = 4 pi 1e-7 H/m, c exact, eps0 = 1 / (mu0 c^2).
#define FIT_MU0 (4.0e-7 * 3.141592653589793)
#define FIT_C0 299792458.0
#define FIT_EPS0 (1.0 / (FIT_MU0 * FIT_C0 * FIT_C0))

// Row pitch (in cells) of the library's internal per-cell arrays is a multiple of this, so that
// every row starts on a 16-byte boundary for the bulk tensor copies (TMA) of the fused kernel.
#define FIT_PITCH_ALIGN 16

struct fit_grid {
  int nx = 0, ny = 0, nz = 0;
  int nxp = 0;             // padded row pitch of internal arrays (cells)
  long long ncell = 0;     // nx*ny*nz
  long long ncellp = 0;    // nxp*ny*nz
  long long ne = 0;        // 3*ncell
  int device = 0;
  double* dx = nullptr;    // device copies of the cell widths
  double* dy = nullptr;
  double* dz = nullptr;
  // Material coefficients, padded layout: internal cell index cp = i + nxp*(j + ny*k).
  double* nu64 = nullptr;  // [ncellp*3] M_nu facet values (SI)
  double* ek64 = nullptr;  // [ncellp*6] M_eps (x,y,z) then M_kappa (x,y,z) edge values (SI)
  float* nu32 = nullptr;   // [ncellp*3] coef_scale * M_nu
  float* ek32 = nullptr;   // [ncellp*6] coef_scale * (M_eps, M_kappa)
  uint8_t* mask = nullptr; // [ncellp] bit w set = w-edge of the cell is masked (PEC/wall)
  double coef_scale = 1.0; // c64 coefficients are coef_scale * SI values (1 / max M_nu)
  bool has_materials = false;
  bool eps_positive = false;  // M_eps > 0 and finite on every unmasked edge (the symmetrised form divides by it)
  double* omega_dev = nullptr;  // per-batch angular frequencies for fit_apply
  int omega_cap = 0;
  size_t bytes_held = 0;
  size_t budget = 0;       // 0 = unlimited
  // autotuned apply kernel per (batch, precision): -1 = generic kernel, k >= 0 = fused variant k
  std::map<long long, int> tuned;
  int* err_dev = nullptr;  // device error word: 1 = a bounded wait in a kernel ran out, 2 = aborted
  int* abort_host = nullptr;       // abort word in pinned, mapped host memory (fit_set_abort)
  const int* abort_dev = nullptr;  // its device alias, polled by the kernels' bounded waits and the solver
  int* abort_mirror = nullptr;     // a device-memory copy of the word, for the fused kernels' first check
  cudaStream_t side = nullptr;     // non-blocking stream that carries the copy while other work runs
  void* mat16 = nullptr;   // [ncell][4] bf16 material channels of the learned preconditioner
  struct fit_unet* unet = nullptr;  // attached learned preconditioner (not owned)
};

struct fit_unet;
// z = scale_out * U(scale_in * v) for one complex64 vector of the grid (x16: [ncell][16] bf16 scratch),
// plus jac_scale * dinv (.) jac_v when dinv is given (a multiple of a Jacobi direction)
fit_status fit_unet_apply_vec(fit_unet* u, const fit_grid* g, const void* v, void* z, float scale_in, float scale_out,
                              void* x16, const void* dinv, const void* jac_v, float jac_scale, cudaStream_t s);
// size the network's activations for the grid and refresh its bf16 weights (call before capture)
fit_status fit_unet_prepare(fit_unet* u, const fit_grid* g, cudaStream_t s);

// Reads and clears the grid's device error word (synchronous); FIT_ETIMEOUT with a message if a bounded
// wait ran out or the abort word stopped a kernel since the last check, else FIT_OK.
fit_status fit_take_device_error(fit_grid* g);
// Reads and clears the network kernels' timeout word on the current device (synchronous): 1 if a bounded
// wait of a tensor-core convolution ran out since the last call.
int fit_unet_take_timeout();
// FIT_ETIMEOUT (with a message) if the grid's abort word is set, else FIT_OK: checked on the host before
// a call enqueues any work.
fit_status fit_check_abort(const fit_grid* g, const char* what);

// Thread-local last-error message.
void fit_set_error(const std::string& msg);
const char* fit_get_error();

#define FIT_CHECK_CUDA(call)                                                          \
  do {                                                                                \
    cudaError_t err__ = (call);                                                       \
    if (err__ != cudaSuccess) {                                                       \
      fit_set_error(std::string(#call) + ": " + cudaGetErrorString(err__));           \
      return FIT_ECUDA;                                                               \
    }                                                                                 \
  } while (0)

#define FIT_REQUIRE(cond, msg)      \
  do {                              \
    if (!(cond)) {                  \
      fit_set_error(msg);           \
      return FIT_EINVAL;            \
    }                               \
  } while (0)

// Device allocation accounted against the handle's budget.
fit_status fit_dev_alloc(fit_grid* g, void** p, size_t bytes);
void fit_dev_free(fit_grid* g, void* p, size_t bytes);

// Transient device buffers of one call, counted against the handle's budget and freed when the
// object goes out of scope (on every return path).
struct FitDevTmp {
  fit_grid* g;
  std::vector<std::pair<void*, size_t>> held;
  explicit FitDevTmp(fit_grid* gg) : g(gg) {}
  FitDevTmp(const FitDevTmp&) = delete;
  FitDevTmp& operator=(const FitDevTmp&) = delete;
  ~FitDevTmp() {
    for (auto& h : held) fit_dev_free(g, h.first, h.second);
  }
  fit_status alloc(void** dst, size_t bytes) {
    fit_status st = fit_dev_alloc(g, dst, bytes);
    if (st == FIT_OK && *dst) held.push_back({*dst, bytes});
    return st;
  }
  // allocate and copy a host array in (stream-ordered on s)
  fit_status copy(void** dst, const void* src, size_t bytes, cudaStream_t s) {
    fit_status st = alloc(dst, bytes);
    if (st != FIT_OK) return st;
    if (bytes) FIT_CHECK_CUDA(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, s));
    return FIT_OK;
  }
};

// Fused epilogues of the operator apply (all per system b of the batch; sums are written as
// per-block partials part[(b*nblk + block)*4 + q], reduced later in a fixed order):
//   FIT_EPI_NONE    y = out_scale * A x
//   FIT_EPI_DOT_U   y = A x;  q0,q1 = sum conj(u) * y           (BiCGStab <r^, v>)
//   FIT_EPI_DOT_TS  y = A x;  q0,q1 = sum conj(y) * x, q2 = sum |y|^2   (<t, s>, <t, t>)
//   FIT_EPI_RESID   y = u - A x (u = b);  q2 = sum |y|^2        (true residual and its norm)
//   FIT_EPI_DOT_XY  y = A x;  q0,q1 = sum x * y (unconjugated)  (COCG (p, A p))
// Systems whose status[b] != 0 are skipped entirely (no write, no partial).
enum { FIT_EPI_NONE = 0, FIT_EPI_DOT_U = 1, FIT_EPI_DOT_TS = 2, FIT_EPI_RESID = 3, FIT_EPI_DOT_XY = 4 };
struct fit_epi {
  int mode = FIT_EPI_NONE;
  const void* u = nullptr;
  double* part = nullptr;
  const int* status = nullptr;
  long long nslots = 0;  // set by the launcher: partial slots per system this launch writes
};

// Launch the operator apply: y_b = out_scale * A(omega_b) x_b (+ epilogue).  omega_dev is a
// device array of nbatch angular frequencies.  x/y are float2 (FIT_C64) or double2 (FIT_C128).
fit_status fit_launch_apply(fit_grid* g, int nbatch, const double* omega_dev, const void* x, void* y,
                            fit_prec prec, double out_scale, cudaStream_t stream, fit_epi* epi = nullptr);
// the symmetrised operator of Eq. e2s (generic kernel), omega already on the device
fit_status fit_launch_apply_sym(fit_grid* g, int nbatch, const double* omega_dev, const void* x, void* y,
                                fit_prec prec, cudaStream_t s);
// Time the apply variants for (nbatch, prec) on the given buffers and cache the fastest; no-op if
// already tuned.  Must not be called while the stream is being captured.
fit_status fit_tune_apply(fit_grid* g, int nbatch, const double* omega_dev, const void* x, void* y, fit_prec prec,
                          cudaStream_t s);
// The cached choice: out7 = {choice (-1 generic, -2 untuned, >= 0 fused variant), TX, TY, TZ,
// ring stages, warp-specialised (0/1), L2 prefetch distance in planes}.
int fit_tuned_choice(const fit_grid* g, fit_prec prec, int nbatch, int* out7);
// name (blanks replaced) and SM count of the current device: the device part of a tuning-cache key
fit_status fit_tuning_device_key(std::string* name, int* sm_count);
// cuTensorMapEncodeTiled through the runtime's driver entry point (no swizzle, no interleave, zero fill
// outside the tensor, unit element strides); false if the entry point or the encoding fails
bool fit_tmap_encode(CUtensorMap* m, CUtensorMapDataType dt, int rank, const void* base, const cuuint64_t* dims,
                     const cuuint64_t* strides, const cuuint32_t* box);
// Number of partial-sum slots per system that the apply writes for an epilogue.
long long fit_apply_partials(const fit_grid* g, fit_prec prec);

// ------------------------------------------------------------------------------------------------
// complex helpers
// ------------------------------------------------------------------------------------------------
template <typename T> struct cplx;
template <> struct cplx<float> { using t = float2; };
template <> struct cplx<double> { using t = double2; };

__host__ __device__ inline float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__host__ __device__ inline double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

template <typename V> __host__ __device__ inline V czero();
template <> __host__ __device__ inline float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __host__ __device__ inline double2 czero<double2>() { return make_double2(0.0, 0.0); }

// diag(A(w)) of one unmasked edge w of cell (i, j, k) (Eq. Precond construction on the unsymmetrised
// operator): the sum of M_nu over the four facets that contain the edge (zero beyond the low walls),
// minus w^2 M_eps, plus j w M_kappa; coefficients in the padded per-cell layout (row pitch nxp).
template <typename T>
__device__ inline double2 fit_jacobi_diag(const T* __restrict__ nu, const T* __restrict__ ek, int i, int j, int k,
                                          int w, int nxp, int ny, double omega) {
  auto NU = [&](int a, int bb, int cc, int q) -> double {
    if (a < 0 || bb < 0 || cc < 0) return 0.0;
    return (double)nu[3 * (a + (long long)nxp * (bb + (long long)ny * cc)) + q];
  };
  double ns;
  if (w == 0) ns = NU(i, j, k, 1) + NU(i, j, k - 1, 1) + NU(i, j, k, 2) + NU(i, j - 1, k, 2);
  else if (w == 1) ns = NU(i, j, k, 0) + NU(i, j, k - 1, 0) + NU(i, j, k, 2) + NU(i - 1, j, k, 2);
  else ns = NU(i, j, k, 0) + NU(i, j - 1, k, 0) + NU(i, j, k, 1) + NU(i - 1, j, k, 1);
  const long long cp = i + (long long)nxp * (j + (long long)ny * k);
  return make_double2(ns - omega * omega * (double)ek[6 * cp + w], omega * (double)ek[6 * cp + 3 + w]);
}

// ------------------------------------------------------------------------------------------------
// Block sum of NQ per-thread values.  Each thread's value is in T (float for the complex64 path,
// whose products are exact enough per cell, double for complex128); warps reduce with shuffles
// in T, then thread 0 adds the warp sums in double in a fixed order (deterministic).  GB300 runs
// FP64 at about 1/58 of the FP32 rate, so FP64 is kept to the per-warp level and above.
// All threads of the block must call it; out[0..NQ-1] is written by thread 0.
// ------------------------------------------------------------------------------------------------
template <typename T, int NQ>
__device__ inline void fit_block_sum(T (&v)[NQ], double* out) {
  __shared__ double red[32][NQ > 0 ? NQ : 1];
  int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  int nthreads = blockDim.x * blockDim.y * blockDim.z;
  int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) red[warp][q] = (double)v[q];
  }
  __syncthreads();
  if (tid == 0) {
    int nw = (nthreads + 31) >> 5;
    for (int q = 0; q < NQ; ++q) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += red[w][q];
      out[q] = s;
    }
  }
  __syncthreads();
}
