// Grid handle, material assembly (Sec. II, Eq. Material) and the public apply entry point.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda_bf16.h>

#include "fit_internal.cuh"

static thread_local std::string g_last_error;

void fit_set_error(const std::string& msg) { g_last_error = msg; }
const char* fit_get_error() { return g_last_error.c_str(); }

fit_status fit_dev_alloc(fit_grid* g, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return FIT_OK;
  if (g->budget && g->bytes_held + bytes > g->budget) {
    fit_set_error("device allocation of " + std::to_string(bytes) + " bytes exceeds the HBM budget");
    return FIT_EBUDGET;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    (void)cudaGetLastError();
    fit_set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return FIT_ENOMEM;
  }
  g->bytes_held += bytes;
  return FIT_OK;
}

void fit_dev_free(fit_grid* g, void* p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  g->bytes_held -= std::min(g->bytes_held, bytes);
}

// ------------------------------------------------------------------------------------------------
// Material assembly.  One thread per cell (i, j, k) gathers, for the x-, y- and z-edge leaving its
// low node, the (up to) four cells that share the edge, and for its three primal facets the two
// half cells on the dual edge through the facet.  Cells beyond a wall contribute nothing.
//   M_eps  = eps0 * sum_c eps_r(c) * (h_u(c)/2)(h_v(c)/2) / h_w        (dual-facet average)
//   M_kap  =        sum_c sigma(c) * (h_u(c)/2)(h_v(c)/2) / h_w
//   M_nu   = sum_halves (h_w/2) inv_mu_r / mu0 / (h_u h_v)              (dual-edge average)
// An edge is masked if it lies in a low wall plane or any cell sharing it is PEC.
// ------------------------------------------------------------------------------------------------
struct CellField {
  const float* a;
  int nx, ny, nz;
  __device__ double at(int i, int j, int k) const {
    if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) return 0.0;
    return (double)a[i + (long long)nx * (j + (long long)ny * k)];
  }
};

__device__ inline double width(const double* d, int n, int i) { return (i >= 0 && i < n) ? d[i] : 0.0; }

__global__ void assemble_kernel(const double* __restrict__ dx, const double* __restrict__ dy,
                                const double* __restrict__ dz, const float* __restrict__ eps_r,
                                const float* __restrict__ sigma, const float* __restrict__ inv_mu_r,
                                const uint8_t* __restrict__ pec, int nx, int ny, int nz, int nxp,
                                double* __restrict__ nu64, double* __restrict__ ek64, uint8_t* __restrict__ mask) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long ncell = (long long)nx * ny * nz;
  if (t >= ncell) return;
  int i = (int)(t % nx);
  int j = (int)((t / nx) % ny);
  int k = (int)(t / ((long long)nx * ny));
  CellField E{eps_r, nx, ny, nz}, S{sigma, nx, ny, nz}, M{inv_mu_r, nx, ny, nz};
  auto is_pec = [&](int a, int b, int c) -> bool {
    if (!pec || a < 0 || b < 0 || c < 0 || a >= nx || b >= ny || c >= nz) return false;
    return pec[a + (long long)nx * (b + (long long)ny * c)] != 0;
  };
  long long cp = i + (long long)nxp * (j + (long long)ny * k);
  double eps[3], kap[3];
  uint8_t m = 0;
  // x-edge: cells (i, j-1..j, k-1..k)
  {
    double se = 0, sk = 0;
    bool p = false;
    for (int dj = -1; dj <= 0; ++dj)
      for (int dk = -1; dk <= 0; ++dk) {
        double a = 0.25 * width(dy, ny, j + dj) * width(dz, nz, k + dk);
        se += E.at(i, j + dj, k + dk) * a;
        sk += S.at(i, j + dj, k + dk) * a;
        p = p || is_pec(i, j + dj, k + dk);
      }
    eps[0] = FIT_EPS0 * se / dx[i];
    kap[0] = sk / dx[i];
    if (j == 0 || k == 0 || p) m |= 1;
  }
  // y-edge: cells (i-1..i, j, k-1..k)
  {
    double se = 0, sk = 0;
    bool p = false;
    for (int di = -1; di <= 0; ++di)
      for (int dk = -1; dk <= 0; ++dk) {
        double a = 0.25 * width(dx, nx, i + di) * width(dz, nz, k + dk);
        se += E.at(i + di, j, k + dk) * a;
        sk += S.at(i + di, j, k + dk) * a;
        p = p || is_pec(i + di, j, k + dk);
      }
    eps[1] = FIT_EPS0 * se / dy[j];
    kap[1] = sk / dy[j];
    if (i == 0 || k == 0 || p) m |= 2;
  }
  // z-edge: cells (i-1..i, j-1..j, k)
  {
    double se = 0, sk = 0;
    bool p = false;
    for (int di = -1; di <= 0; ++di)
      for (int dj = -1; dj <= 0; ++dj) {
        double a = 0.25 * width(dx, nx, i + di) * width(dy, ny, j + dj);
        se += E.at(i + di, j + dj, k) * a;
        sk += S.at(i + di, j + dj, k) * a;
        p = p || is_pec(i + di, j + dj, k);
      }
    eps[2] = FIT_EPS0 * se / dz[k];
    kap[2] = sk / dz[k];
    if (i == 0 || j == 0 || p) m |= 4;
  }
  double nux = (0.5 * width(dx, nx, i - 1) * M.at(i - 1, j, k) + 0.5 * dx[i] * M.at(i, j, k)) / (FIT_MU0 * dy[j] * dz[k]);
  double nuy = (0.5 * width(dy, ny, j - 1) * M.at(i, j - 1, k) + 0.5 * dy[j] * M.at(i, j, k)) / (FIT_MU0 * dx[i] * dz[k]);
  double nuz = (0.5 * width(dz, nz, k - 1) * M.at(i, j, k - 1) + 0.5 * dz[k] * M.at(i, j, k)) / (FIT_MU0 * dx[i] * dy[j]);
  nu64[3 * cp + 0] = nux;
  nu64[3 * cp + 1] = nuy;
  nu64[3 * cp + 2] = nuz;
  for (int w = 0; w < 3; ++w) {
    ek64[6 * cp + w] = eps[w];
    ek64[6 * cp + 3 + w] = kap[w];
  }
  mask[cp] = m;
}

// Material channels of the learned preconditioner per cell (bf16): eps_r / 10, log10(1 + sigma) / 8,
// 1 / mu_r, and the cell size (dx dy dz)^(1/3) in millimetres.
__global__ void mat16_kernel(const float* __restrict__ eps_r, const float* __restrict__ sigma,
                             const float* __restrict__ inv_mu_r, const double* __restrict__ dx,
                             const double* __restrict__ dy, const double* __restrict__ dz, int nx, int ny, int nz,
                             __nv_bfloat16* out) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= (long long)nx * ny * nz) return;
  int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
  out[4 * c + 0] = __float2bfloat16(eps_r[c] / 10.f);
  out[4 * c + 1] = __float2bfloat16((float)(log10(1.0 + (double)sigma[c]) / 8.0));
  out[4 * c + 2] = __float2bfloat16(inv_mu_r[c]);
  out[4 * c + 3] = __float2bfloat16((float)(cbrt(dx[i] * dy[j] * dz[k]) * 1e3));
}

// max over facets of M_nu (positive doubles order like their bit patterns)
__global__ void max_nu_kernel(const double* __restrict__ nu, long long n, unsigned long long* out) {
  unsigned long long best = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double v = nu[t];
    if (v > 0.0) best = max(best, (unsigned long long)__double_as_longlong(v));
  }
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

__global__ void to_c64_kernel(const double* __restrict__ nu64, const double* __restrict__ ek64, long long ncellp,
                              double scale, float* __restrict__ nu32, float* __restrict__ ek32) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ncellp; t += (long long)gridDim.x * blockDim.x) {
    for (int w = 0; w < 3; ++w) nu32[3 * t + w] = (float)(scale * nu64[3 * t + w]);
    for (int w = 0; w < 6; ++w) ek32[6 * t + w] = (float)(scale * ek64[6 * t + w]);
  }
}

static fit_status finish_coefficients(fit_grid* g) {
  unsigned long long* dmax = nullptr;
  FIT_CHECK_CUDA(cudaMalloc(&dmax, sizeof(unsigned long long)));
  cudaMemset(dmax, 0, sizeof(unsigned long long));
  max_nu_kernel<<<1024, 256>>>(g->nu64, 3 * g->ncellp, dmax);
  unsigned long long bits = 0;
  cudaError_t e = cudaMemcpy(&bits, dmax, sizeof(bits), cudaMemcpyDeviceToHost);
  cudaFree(dmax);
  FIT_CHECK_CUDA(e);
  double mx;
  memcpy(&mx, &bits, sizeof(mx));
  if (!(mx > 0.0) || !isfinite(mx)) {
    fit_set_error("material matrices have no positive finite M_nu entry");
    return FIT_EINVAL;
  }
  g->coef_scale = 1.0 / mx;
  to_c64_kernel<<<1024, 256>>>(g->nu64, g->ek64, g->ncellp, g->coef_scale, g->nu32, g->ek32);
  FIT_CHECK_CUDA(cudaGetLastError());
  FIT_CHECK_CUDA(cudaDeviceSynchronize());
  g->has_materials = true;
  return FIT_OK;
}

// ------------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------------
fit_status fit_check_abort(const fit_grid* g, const char* what) {
  if (g->abort_host && __atomic_load_n(g->abort_host, __ATOMIC_SEQ_CST)) {
    fit_set_error(std::string(what) + ": the grid's abort word is set (fit_set_abort)");
    return FIT_ETIMEOUT;
  }
  return FIT_OK;
}

fit_status fit_take_device_error(fit_grid* g) {
  int code = 0;
  FIT_CHECK_CUDA(cudaMemcpy(&code, g->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
  if (code == 0) return FIT_OK;
  FIT_CHECK_CUDA(cudaMemset(g->err_dev, 0, sizeof(int)));
  fit_set_error(code == 2 ? "a kernel of this grid stopped early: the abort word was set"
                          : "a bounded wait in a kernel of this grid ran out; its output is incomplete");
  return FIT_ETIMEOUT;
}

extern "C" {

const char* fit_status_str(fit_status s) {
  switch (s) {
    case FIT_OK: return "FIT_OK";
    case FIT_NOT_CONVERGED: return "FIT_NOT_CONVERGED";
    case FIT_BREAKDOWN: return "FIT_BREAKDOWN";
    case FIT_EINVAL: return "FIT_EINVAL";
    case FIT_ENOMEM: return "FIT_ENOMEM";
    case FIT_ECUDA: return "FIT_ECUDA";
    case FIT_ETIMEOUT: return "FIT_ETIMEOUT";
    case FIT_EBUDGET: return "FIT_EBUDGET";
    case FIT_ENAN: return "FIT_ENAN";
  }
  return "FIT_UNKNOWN";
}

const char* fit_last_error(void) { return fit_get_error(); }

void fit_grid_destroy(fit_grid* g) {
  if (!g) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(g->device);
  void* ptrs[] = {g->dx,       g->dy,      g->dz,      g->nu64,  g->ek64,        g->nu32,
                  g->ek32,     g->mask,    g->omega_dev, g->err_dev, g->mat16,     g->abort_mirror};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (g->abort_host) cudaFreeHost(g->abort_host);
  if (g->side) cudaStreamDestroy(g->side);
  cudaSetDevice(cur);
  delete g;
}

fit_status fit_grid_create(int nx, int ny, int nz, const double* dx, const double* dy, const double* dz,
                           unsigned bc_flags, fit_grid** out) {
  FIT_REQUIRE(out != nullptr, "fit_grid_create: out is NULL");
  *out = nullptr;
  FIT_REQUIRE(nx >= 1 && ny >= 1 && nz >= 1, "fit_grid_create: nx, ny, nz must be >= 1");
  FIT_REQUIRE((long long)nx * ny * nz <= (1LL << 33), "fit_grid_create: grid too large");
  FIT_REQUIRE(dx && dy && dz, "fit_grid_create: null cell-width array");
  FIT_REQUIRE(bc_flags == FIT_BC_PEC_ALL, "fit_grid_create: only PEC walls (FIT_BC_PEC_ALL) are supported");
  for (int i = 0; i < nx; ++i) FIT_REQUIRE(dx[i] > 0 && isfinite(dx[i]), "fit_grid_create: dx must be positive");
  for (int i = 0; i < ny; ++i) FIT_REQUIRE(dy[i] > 0 && isfinite(dy[i]), "fit_grid_create: dy must be positive");
  for (int i = 0; i < nz; ++i) FIT_REQUIRE(dz[i] > 0 && isfinite(dz[i]), "fit_grid_create: dz must be positive");
  fit_grid* g = new fit_grid();
  FIT_CHECK_CUDA(cudaGetDevice(&g->device));
  g->nx = nx;
  g->ny = ny;
  g->nz = nz;
  g->nxp = (nx + FIT_PITCH_ALIGN - 1) / FIT_PITCH_ALIGN * FIT_PITCH_ALIGN;
  g->ncell = (long long)nx * ny * nz;
  g->ncellp = (long long)g->nxp * ny * nz;
  g->ne = 3 * g->ncell;
  fit_status st = FIT_OK;
  size_t np = (size_t)g->ncellp;
  if ((st = fit_dev_alloc(g, (void**)&g->dx, nx * sizeof(double))) ||
      (st = fit_dev_alloc(g, (void**)&g->dy, ny * sizeof(double))) ||
      (st = fit_dev_alloc(g, (void**)&g->dz, nz * sizeof(double))) ||
      (st = fit_dev_alloc(g, (void**)&g->nu64, np * 3 * sizeof(double))) ||
      (st = fit_dev_alloc(g, (void**)&g->ek64, np * 6 * sizeof(double))) ||
      (st = fit_dev_alloc(g, (void**)&g->nu32, np * 3 * sizeof(float))) ||
      (st = fit_dev_alloc(g, (void**)&g->ek32, np * 6 * sizeof(float))) ||
      (st = fit_dev_alloc(g, (void**)&g->mask, np)) ||
      (st = fit_dev_alloc(g, (void**)&g->err_dev, sizeof(int))) ||
      (st = fit_dev_alloc(g, (void**)&g->abort_mirror, sizeof(int))) ||
      (st = fit_dev_alloc(g, (void**)&g->mat16, (size_t)g->ncell * 4 * 2))) {
    fit_grid_destroy(g);
    return st;
  }
  // the abort word: pinned host memory mapped into the device's address space, so that a kernel that
  // is already running sees the host's write
  {
    void* hp = nullptr;
    void* dp = nullptr;
    cudaError_t e = cudaHostAlloc(&hp, sizeof(int), cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaSuccess) {
      g->abort_host = (int*)hp;
      *g->abort_host = 0;
      e = cudaHostGetDevicePointer(&dp, hp, 0);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      fit_set_error(std::string("fit_grid_create: abort word: ") + cudaGetErrorString(e));
      fit_grid_destroy(g);
      return FIT_ECUDA;
    }
    g->abort_dev = (const int*)dp;
  }
  cudaMemcpy(g->dx, dx, nx * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(g->dy, dy, ny * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(g->dz, dz, nz * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemset(g->nu64, 0, np * 3 * sizeof(double));
  cudaMemset(g->ek64, 0, np * 6 * sizeof(double));
  cudaMemset(g->nu32, 0, np * 3 * sizeof(float));
  cudaMemset(g->ek32, 0, np * 6 * sizeof(float));
  cudaMemset(g->mask, 0, np);
  cudaMemset(g->err_dev, 0, sizeof(int));
  cudaMemset(g->abort_mirror, 0, sizeof(int));
  cudaMemset(g->mat16, 0, (size_t)g->ncell * 4 * 2);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    fit_set_error(std::string("fit_grid_create: ") + cudaGetErrorString(e));
    fit_grid_destroy(g);
    return FIT_ECUDA;
  }
  *out = g;
  return FIT_OK;
}

fit_status fit_set_materials(fit_grid* g, const float* eps_r, const float* sigma, const float* inv_mu_r,
                             const unsigned char* pec_cell) {
  FIT_REQUIRE(g && eps_r && sigma && inv_mu_r, "fit_set_materials: null argument");
  size_t n = (size_t)g->ncell;
  for (size_t c = 0; c < n; ++c) {
    FIT_REQUIRE(std::isfinite(eps_r[c]) && eps_r[c] > 0.0f, "fit_set_materials: eps_r must be finite and > 0");
    FIT_REQUIRE(std::isfinite(sigma[c]) && sigma[c] >= 0.0f, "fit_set_materials: sigma must be finite and >= 0");
    FIT_REQUIRE(std::isfinite(inv_mu_r[c]) && inv_mu_r[c] > 0.0f, "fit_set_materials: inv_mu_r must be finite and > 0");
  }
  FIT_CHECK_CUDA(cudaSetDevice(g->device));
  FitDevTmp tmp(g);  // the per-cell inputs live only for this call
  void *d_eps = nullptr, *d_sig = nullptr, *d_imu = nullptr, *d_pec = nullptr;
  fit_status st;
  if ((st = tmp.copy(&d_eps, eps_r, n * sizeof(float), nullptr)) != FIT_OK) return st;
  if ((st = tmp.copy(&d_sig, sigma, n * sizeof(float), nullptr)) != FIT_OK) return st;
  if ((st = tmp.copy(&d_imu, inv_mu_r, n * sizeof(float), nullptr)) != FIT_OK) return st;
  if (pec_cell && (st = tmp.copy(&d_pec, pec_cell, n, nullptr)) != FIT_OK) return st;
  int threads = 256;
  long long blocks = ((long long)n + threads - 1) / threads;
  const float *pe = (const float*)d_eps, *ps = (const float*)d_sig, *pm = (const float*)d_imu;
  assemble_kernel<<<(unsigned)blocks, threads>>>(g->dx, g->dy, g->dz, pe, ps, pm, (const uint8_t*)d_pec, g->nx,
                                                 g->ny, g->nz, g->nxp, g->nu64, g->ek64, g->mask);
  mat16_kernel<<<(unsigned)blocks, threads>>>(pe, ps, pm, g->dx, g->dy, g->dz, g->nx, g->ny, g->nz,
                                              (__nv_bfloat16*)g->mat16);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    fit_set_error(std::string("fit_set_materials: ") + cudaGetErrorString(e));
    return FIT_ECUDA;
  }
  g->eps_positive = true;  // positive cell permittivities and widths give a positive M_eps on every edge
  return finish_coefficients(g);
}

fit_status fit_set_material_matrices(fit_grid* g, const double* m_eps, const double* m_kappa, const double* m_nu,
                                     const unsigned char* edge_mask) {
  FIT_REQUIRE(g && m_eps && m_kappa && m_nu, "fit_set_material_matrices: null argument");
  FIT_CHECK_CUDA(cudaSetDevice(g->device));
  bool eps_pos = true;
  for (long long e = 0; e < g->ne; ++e)
    if (!(edge_mask && edge_mask[e]) && !(std::isfinite(m_eps[e]) && m_eps[e] > 0.0)) eps_pos = false;
  g->eps_positive = eps_pos;
  size_t np = (size_t)g->ncellp;
  std::vector<double> nu(np * 3, 0.0), ek(np * 6, 0.0);
  std::vector<uint8_t> mk(np, 0);
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        size_t c = i + (size_t)g->nx * (j + (size_t)g->ny * k);
        size_t cp = i + (size_t)g->nxp * (j + (size_t)g->ny * k);
        uint8_t m = 0;
        for (int w = 0; w < 3; ++w) {
          nu[3 * cp + w] = m_nu[3 * c + w];
          ek[6 * cp + w] = m_eps[3 * c + w];
          ek[6 * cp + 3 + w] = m_kappa[3 * c + w];
          if (edge_mask && edge_mask[3 * c + w]) m |= (uint8_t)(1u << w);
        }
        mk[cp] = m;
      }
  FIT_CHECK_CUDA(cudaMemcpy(g->nu64, nu.data(), np * 3 * sizeof(double), cudaMemcpyHostToDevice));
  FIT_CHECK_CUDA(cudaMemcpy(g->ek64, ek.data(), np * 6 * sizeof(double), cudaMemcpyHostToDevice));
  FIT_CHECK_CUDA(cudaMemcpy(g->mask, mk.data(), np, cudaMemcpyHostToDevice));
  return finish_coefficients(g);
}

fit_status fit_coef_scale(const fit_grid* g, double* s) {
  FIT_REQUIRE(g && s && g->has_materials, "fit_coef_scale: null argument or materials not set");
  *s = g->coef_scale;
  return FIT_OK;
}

fit_status fit_set_hbm_budget(fit_grid* g, size_t bytes) {
  FIT_REQUIRE(g, "fit_set_hbm_budget: null grid");
  g->budget = bytes;
  return FIT_OK;
}

fit_status fit_grid_info(const fit_grid* g, long long* out6) {
  FIT_REQUIRE(g && out6, "fit_grid_info: null argument");
  out6[0] = g->nx;
  out6[1] = g->ny;
  out6[2] = g->nz;
  out6[3] = g->ne;
  out6[4] = (long long)g->bytes_held;
  out6[5] = (long long)g->budget;
  return FIT_OK;
}

// the batch's frequencies into the handle's device buffer (grown on demand, counted in the budget)
static fit_status stage_omega(fit_grid* g, int nbatch, const double* omega, cudaStream_t s) {
  if (nbatch > g->omega_cap) {
    if (g->omega_dev) fit_dev_free(g, g->omega_dev, g->omega_cap * sizeof(double));
    g->omega_dev = nullptr;
    g->omega_cap = 0;
    int cap = std::max(nbatch, 64);
    fit_status st = fit_dev_alloc(g, (void**)&g->omega_dev, cap * sizeof(double));
    if (st != FIT_OK) return st;
    g->omega_cap = cap;
  }
  FIT_CHECK_CUDA(cudaMemcpyAsync(g->omega_dev, omega, nbatch * sizeof(double), cudaMemcpyHostToDevice, s));
  return FIT_OK;
}

fit_status fit_apply(fit_grid* g, int nbatch, const double* omega, const void* x, void* y, fit_prec prec,
                     void* stream) {
  FIT_REQUIRE(g && omega && x && y, "fit_apply: null argument");
  FIT_REQUIRE(nbatch >= 1, "fit_apply: nbatch must be >= 1");
  FIT_REQUIRE(prec == FIT_C64 || prec == FIT_C128, "fit_apply: unknown precision");
  FIT_REQUIRE(g->has_materials, "fit_apply: materials not set");
  for (int b = 0; b < nbatch; ++b) FIT_REQUIRE(isfinite(omega[b]), "fit_apply: omega must be finite");
  size_t esz = prec == FIT_C64 ? sizeof(float2) : sizeof(double2);
  size_t vbytes = (size_t)g->ne * esz * nbatch;
  const char* xb = (const char*)x;
  const char* yb = (const char*)y;
  FIT_REQUIRE(xb + vbytes <= yb || yb + vbytes <= xb, "fit_apply: x and y overlap");
  if (fit_check_abort(g, "fit_apply") != FIT_OK) return FIT_ETIMEOUT;
  FIT_CHECK_CUDA(cudaSetDevice(g->device));
  cudaStream_t s = (cudaStream_t)stream;
  fit_status st = stage_omega(g, nbatch, omega, s);
  if (st != FIT_OK) return st;
  double out_scale = prec == FIT_C64 ? 1.0 / g->coef_scale : 1.0;
  return fit_launch_apply(g, nbatch, g->omega_dev, x, y, prec, out_scale, s);
}

fit_status fit_set_abort(fit_grid* g, int value) {
  FIT_REQUIRE(g && g->abort_host, "fit_set_abort: null grid");
  FIT_REQUIRE(value == 0 || value == 1, "fit_set_abort: value must be 0 or 1");
  __atomic_store_n(g->abort_host, value, __ATOMIC_SEQ_CST);
  // the device-memory copy the fused kernels read first: a copy on the grid's non-blocking side stream,
  // which the copy engine carries out while kernels of other streams run
  FIT_CHECK_CUDA(cudaSetDevice(g->device));
  static thread_local int staged = 0;
  staged = value;
  FIT_CHECK_CUDA(cudaMemcpyAsync(g->abort_mirror, &staged, sizeof(int), cudaMemcpyHostToDevice, g->side));
  FIT_CHECK_CUDA(cudaStreamSynchronize(g->side));
  return FIT_OK;
}

fit_status fit_sync(fit_grid* g, void* stream) {
  FIT_REQUIRE(g, "fit_sync: null grid");
  FIT_CHECK_CUDA(cudaSetDevice(g->device));
  FIT_CHECK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  fit_status st = fit_take_device_error(g);
  if (fit_unet_take_timeout() && st == FIT_OK) {
    fit_set_error("fit_sync: a bounded wait in a learned-preconditioner convolution ran out");
    st = FIT_ETIMEOUT;
  }
  return st;
}

fit_status fit_apply_sym(fit_grid* g, int nbatch, const double* omega, const void* x, void* y, fit_prec prec,
                         void* stream) {
  FIT_REQUIRE(g && omega && x && y, "fit_apply_sym: null argument");
  FIT_REQUIRE(nbatch >= 1, "fit_apply_sym: nbatch must be >= 1");
  FIT_REQUIRE(prec == FIT_C64 || prec == FIT_C128, "fit_apply_sym: unknown precision");
  FIT_REQUIRE(g->has_materials, "fit_apply_sym: materials not set");
  FIT_REQUIRE(g->eps_positive, "fit_apply_sym: M_eps must be finite and > 0 on every unmasked edge");
  for (int b = 0; b < nbatch; ++b) FIT_REQUIRE(isfinite(omega[b]), "fit_apply_sym: omega must be finite");
  size_t esz = prec == FIT_C64 ? sizeof(float2) : sizeof(double2);
  size_t vbytes = (size_t)g->ne * esz * nbatch;
  const char* xb = (const char*)x;
  const char* yb = (const char*)y;
  FIT_REQUIRE(xb + vbytes <= yb || yb + vbytes <= xb, "fit_apply_sym: x and y overlap");
  if (fit_check_abort(g, "fit_apply_sym") != FIT_OK) return FIT_ETIMEOUT;
  FIT_CHECK_CUDA(cudaSetDevice(g->device));
  cudaStream_t s = (cudaStream_t)stream;
  fit_status st = stage_omega(g, nbatch, omega, s);
  if (st != FIT_OK) return st;
  return fit_launch_apply_sym(g, nbatch, g->omega_dev, x, y, prec, s);
}

}  // extern "C"
