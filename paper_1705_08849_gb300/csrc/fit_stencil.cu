// Matrix-free FIT operator apply (Sec. III, Eq. e2t fused into one pass):
//     y = out_scale * [ C^T M_nu C x - w^2 M_eps x + j w M_kappa x ]   on unmasked edges,
//     y = x                                                            on masked edges,
// where C^T M_nu C acts on the masked-out (zeroed) copy of x.  The curl of Eq. CP per facet:
//     b_x(i,j,k) = e_y(i,j,k) - e_y(i,j,k+1) + e_z(i,j+1,k) - e_z(i,j,k)
//     b_y(i,j,k) = e_z(i,j,k) - e_z(i+1,j,k) + e_x(i,j,k+1) - e_x(i,j,k)
//     b_z(i,j,k) = e_x(i,j,k) - e_x(i,j+1,k) + e_y(i+1,j,k) - e_y(i,j,k)
// h = M_nu b, and the dual curl C^T h per edge:
//     (C^T h)_x = h_y(i,j,k-1) - h_y(i,j,k) + h_z(i,j,k) - h_z(i,j-1,k)
//     (C^T h)_y = h_z(i-1,j,k) - h_z(i,j,k) + h_x(i,j,k) - h_x(i,j,k-1)
//     (C^T h)_z = h_x(i,j-1,k) - h_x(i,j,k) + h_y(i,j,k) - h_y(i-1,j,k)
// Values beyond the grid are zero (truncated forward differences, PEC high walls).
//
// This file holds the generic kernel: one thread per cell, operands read straight from global
// memory (through L1), any grid size and batch.  It is the reference launch for the fused
// shared-memory kernels in fit_fused.cu and the fallback for shapes they do not take.
//
// With SYM it applies the symmetrised operator of Eq. e2s instead (D = M_eps^{-1/2} per edge):
//     y' = D C^T M_nu C (D x') - w^2 x' + j w (M_kappa / M_eps) x'   on unmasked edges, y' = x' on masked,
// i.e. D A(w) D x' with the unsymmetrised A above.  D is formed from M_eps as it is read, so a common
// scale of the coefficients cancels and no output scale applies.
#include "fit_internal.cuh"

template <typename T>
struct ApplyArgs {
  using V = typename cplx<T>::t;
  const V* __restrict__ x;
  V* __restrict__ y;
  const T* __restrict__ nu;  // [ncellp*3]
  const T* __restrict__ ek;  // [ncellp*6]
  const uint8_t* __restrict__ mask;
  const double* __restrict__ omega;
  int nx, ny, nz, nxp;
  long long ne;
  int nbatch;
  T out_scale;
};

template <typename T, bool SYM = false>
struct GenericView {
  using V = typename cplx<T>::t;
  const ApplyArgs<T>& a;
  const V* x;
  __device__ bool inside(int i, int j, int k) const {
    return i >= 0 && j >= 0 && k >= 0 && i < a.nx && j < a.ny && k < a.nz;
  }
  // masked-out voltage: zero beyond the grid and on masked edges
  __device__ V e(int i, int j, int k, int w) const {
    if (!inside(i, j, k)) return czero<V>();
    long long cp = i + (long long)a.nxp * (j + (long long)a.ny * k);
    if ((a.mask[cp] >> w) & 1) return czero<V>();
    V v = x[3 * (i + (long long)a.nx * (j + (long long)a.ny * k)) + w];
    if constexpr (SYM) {
      const T d = T(1) / sqrt(a.ek[6 * cp + w]);  // D = M_eps^{-1/2}
      v.x *= d;
      v.y *= d;
    }
    return v;
  }
  __device__ T nu(int i, int j, int k, int w) const {
    if (!inside(i, j, k)) return T(0);
    return a.nu[3 * (i + (long long)a.nxp * (j + (long long)a.ny * k)) + w];
  }
  // facet fluxes times M_nu, per component
  __device__ V hx(int i, int j, int k) const {
    return nu(i, j, k, 0) * (e(i, j, k, 1) - e(i, j, k + 1, 1) + e(i, j + 1, k, 2) - e(i, j, k, 2));
  }
  __device__ V hy(int i, int j, int k) const {
    return nu(i, j, k, 1) * (e(i, j, k, 2) - e(i + 1, j, k, 2) + e(i, j, k + 1, 0) - e(i, j, k, 0));
  }
  __device__ V hz(int i, int j, int k) const {
    return nu(i, j, k, 2) * (e(i, j, k, 0) - e(i, j + 1, k, 0) + e(i + 1, j, k, 1) - e(i, j, k, 1));
  }
};

template <typename T, int EPI, bool SYM = false>
__global__ void __launch_bounds__(256) apply_generic_kernel(ApplyArgs<T> a, fit_epi epi) {
  using V = typename cplx<T>::t;
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y;
  const bool valid = i < a.nx && j < a.ny;
  for (long long zb = blockIdx.z; zb < (long long)a.nz * a.nbatch; zb += gridDim.z) {
    const int k = (int)(zb % a.nz);
    const int b = (int)(zb / a.nz);
    if (epi.status && epi.status[b] != 0) continue;  // uniform over the block
    const V* x = a.x + (long long)b * a.ne;
    V* y = a.y + (long long)b * a.ne;
    T acc[3] = {T(0), T(0), T(0)};
    if (valid) {
      GenericView<T, SYM> g{a, x};
      V hx = g.hx(i, j, k), hy = g.hy(i, j, k), hz = g.hz(i, j, k);
      V cx = g.hy(i, j, k - 1) - hy + hz - g.hz(i, j - 1, k);
      V cy = g.hz(i - 1, j, k) - hz + hx - g.hx(i, j, k - 1);
      V cz = g.hx(i, j - 1, k) - hx + hy - g.hy(i - 1, j, k);
      long long c = i + (long long)a.nx * (j + (long long)a.ny * k);
      long long cp = i + (long long)a.nxp * (j + (long long)a.ny * k);
      uint8_t m = a.mask[cp];
      T w = (T)a.omega[b];
      T w2 = w * w;
      V curl[3] = {cx, cy, cz};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        V xv = x[3 * c + q];
        V out;
        if ((m >> q) & 1) {
          out = xv;
        } else if constexpr (SYM) {
          const T eps = a.ek[6 * cp + q];
          const T d = T(1) / sqrt(eps);
          const T ai = w * (a.ek[6 * cp + 3 + q] / eps);  // w M_kappa / M_eps
          out.x = d * curl[q].x - w2 * xv.x - ai * xv.y;
          out.y = d * curl[q].y - w2 * xv.y + ai * xv.x;
        } else {
          T ar = -w2 * a.ek[6 * cp + q];    // -w^2 M_eps
          T ai = w * a.ek[6 * cp + 3 + q];  // w M_kappa
          out.x = a.out_scale * (curl[q].x + ar * xv.x - ai * xv.y);
          out.y = a.out_scale * (curl[q].y + ar * xv.y + ai * xv.x);
        }
        if (EPI == FIT_EPI_DOT_U) {
          V u = ((const V*)epi.u)[(long long)b * a.ne + 3 * c + q];
          acc[0] += u.x * out.x + u.y * out.y;  // conj(u) * y
          acc[1] += u.x * out.y - u.y * out.x;
        } else if (EPI == FIT_EPI_DOT_TS) {
          acc[0] += out.x * xv.x + out.y * xv.y;  // conj(t) * s
          acc[1] += out.x * xv.y - out.y * xv.x;
          acc[2] += out.x * out.x + out.y * out.y;
        } else if (EPI == FIT_EPI_RESID) {
          V u = ((const V*)epi.u)[(long long)b * a.ne + 3 * c + q];
          out = u - out;
          acc[2] += out.x * out.x + out.y * out.y;
        } else if (EPI == FIT_EPI_DOT_XY) {
          acc[0] += xv.x * out.x - xv.y * out.y;  // x * y, unconjugated
          acc[1] += xv.x * out.y + xv.y * out.x;
        }
        y[3 * c + q] = out;
      }
    }
    if (EPI != FIT_EPI_NONE) {
      long long nblk = (long long)gridDim.x * gridDim.y * a.nz;
      long long blk = ((long long)k * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      fit_block_sum<T, 3>(acc, epi.part + ((long long)b * nblk + blk) * 4);
    }
  }
}

template <typename T>
static fit_status launch_generic(fit_grid* g, int nbatch, const double* omega_dev, const void* x, void* y,
                                 const T* nu, const T* ek, double out_scale, cudaStream_t s, const fit_epi* epi) {
  ApplyArgs<T> a;
  a.x = (const typename cplx<T>::t*)x;
  a.y = (typename cplx<T>::t*)y;
  a.nu = nu;
  a.ek = ek;
  a.mask = g->mask;
  a.omega = omega_dev;
  a.nx = g->nx;
  a.ny = g->ny;
  a.nz = g->nz;
  a.nxp = g->nxp;
  a.ne = g->ne;
  a.nbatch = nbatch;
  a.out_scale = (T)out_scale;
  fit_epi e;
  if (epi) e = *epi;
  dim3 block(32, 8, 1);
  long long gz = (long long)g->nz * nbatch;
  dim3 grid((g->nx + 31) / 32, (g->ny + 7) / 8, (unsigned)(gz < 65535 ? gz : 65535));
  switch (e.mode) {
    case FIT_EPI_NONE: apply_generic_kernel<T, FIT_EPI_NONE><<<grid, block, 0, s>>>(a, e); break;
    case FIT_EPI_DOT_U: apply_generic_kernel<T, FIT_EPI_DOT_U><<<grid, block, 0, s>>>(a, e); break;
    case FIT_EPI_DOT_TS: apply_generic_kernel<T, FIT_EPI_DOT_TS><<<grid, block, 0, s>>>(a, e); break;
    case FIT_EPI_RESID: apply_generic_kernel<T, FIT_EPI_RESID><<<grid, block, 0, s>>>(a, e); break;
    case FIT_EPI_DOT_XY: apply_generic_kernel<T, FIT_EPI_DOT_XY><<<grid, block, 0, s>>>(a, e); break;
    default: fit_set_error("unknown apply epilogue"); return FIT_EINVAL;
  }
  FIT_CHECK_CUDA(cudaGetLastError());
  return FIT_OK;
}

template <typename T>
static fit_status launch_sym(fit_grid* g, int nbatch, const double* omega_dev, const void* x, void* y, const T* nu,
                             const T* ek, cudaStream_t s) {
  ApplyArgs<T> a;
  a.x = (const typename cplx<T>::t*)x;
  a.y = (typename cplx<T>::t*)y;
  a.nu = nu;
  a.ek = ek;
  a.mask = g->mask;
  a.omega = omega_dev;
  a.nx = g->nx;
  a.ny = g->ny;
  a.nz = g->nz;
  a.nxp = g->nxp;
  a.ne = g->ne;
  a.nbatch = nbatch;
  a.out_scale = T(1);
  fit_epi e;
  dim3 block(32, 8, 1);
  long long gz = (long long)g->nz * nbatch;
  dim3 grid((g->nx + 31) / 32, (g->ny + 7) / 8, (unsigned)(gz < 65535 ? gz : 65535));
  apply_generic_kernel<T, FIT_EPI_NONE, true><<<grid, block, 0, s>>>(a, e);
  FIT_CHECK_CUDA(cudaGetLastError());
  return FIT_OK;
}

fit_status fit_launch_apply_sym(fit_grid* g, int nbatch, const double* omega_dev, const void* x, void* y,
                                fit_prec prec, cudaStream_t s) {
  if (prec == FIT_C64) return launch_sym<float>(g, nbatch, omega_dev, x, y, g->nu32, g->ek32, s);
  return launch_sym<double>(g, nbatch, omega_dev, x, y, g->nu64, g->ek64, s);
}

long long fit_apply_partials_generic(const fit_grid* g) {
  return (long long)((g->nx + 31) / 32) * ((g->ny + 7) / 8) * g->nz;
}

fit_status fit_launch_apply_generic(fit_grid* g, int nbatch, const double* omega_dev, const void* x, void* y,
                                    fit_prec prec, double out_scale, cudaStream_t s, fit_epi* epi) {
  if (epi) epi->nslots = fit_apply_partials_generic(g);
  if (prec == FIT_C64)
    return launch_generic<float>(g, nbatch, omega_dev, x, y, g->nu32, g->ek32, out_scale, s, epi);
  return launch_generic<double>(g, nbatch, omega_dev, x, y, g->nu64, g->ek64, out_scale, s, epi);
}

