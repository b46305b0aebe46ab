// Port excitation and probe read-out (Sec. IV): currents impressed on the edges of input ports
// drive the system, the voltages along the edges of probes are summed as outputs, and impedance
// parameters Z_ij = V_i / I_j follow; S parameters use a source impedance Z0 (50 Ohm in the paper).
//   port / probe: a list of public edge indices 3*(i + nx*(j + ny*k)) + w with orientations s = +-1
//   right-hand side of a port excited with current I: b = -j w (I s) on its unmasked edges (Eq. e2)
//   probe voltage:  V = - sum_k s_k x[edge_k]  (against the current's direction, so that the power a
//                   source delivers, Re(V conj(I)) / 2, is >= 0 for a passive structure)
//   S = (Z - Z0 1)(Z + Z0 1)^{-1}
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "fit_internal.cuh"

namespace {

// b[f][e] += -j w_f * current * s for the listed edges (b is zeroed before); masked edges keep 0
__global__ void k_port_rhs(const double* __restrict__ omega, int nfreq, const long long* __restrict__ edges,
                           const double* __restrict__ signs, int nedge, double current,
                           const uint8_t* __restrict__ mask, int nx, int ny, int nxp, long long ne, double2* b) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nfreq * nedge) return;
  const int f = (int)(t / nedge), q = (int)(t % nedge);
  const long long e = edges[q];
  const long long cell = e / 3;
  const int w = (int)(e % 3);
  const int i = (int)(cell % nx), j = (int)((cell / nx) % ny);
  const long long k = cell / ((long long)nx * ny);
  if ((mask[i + (long long)nxp * (j + (long long)ny * k)] >> w) & 1) return;
  const double v = -omega[f] * (current * signs[q]);  // -j w (I s): purely imaginary
  atomicAdd(&b[(long long)f * ne + e].y, v);
}

// V[f][q] = - sum over the edges of probe q of s_k x_f[edge_k]; one CTA per (probe, system), FP64
__global__ void __launch_bounds__(256) k_probe(const double2* __restrict__ x, long long ne,
                                               const int* __restrict__ off, const long long* __restrict__ edges,
                                               const double* __restrict__ signs, int nprobe, double2* V) {
  const int q = (int)(blockIdx.x % nprobe), f = (int)(blockIdx.x / nprobe);
  __shared__ double red[2][256];
  double sr = 0.0, si = 0.0;
  for (int k = off[q] + threadIdx.x; k < off[q + 1]; k += 256) {
    const double2 v = x[(long long)f * ne + edges[k]];
    sr -= signs[k] * v.x;
    si -= signs[k] * v.y;
  }
  red[0][threadIdx.x] = sr;
  red[1][threadIdx.x] = si;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {  // fixed-order tree: the same sum on every run
    if ((int)threadIdx.x < h) {
      red[0][threadIdx.x] += red[0][threadIdx.x + h];
      red[1][threadIdx.x] += red[1][threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) V[(long long)f * nprobe + q] = make_double2(red[0][0], red[1][0]);
}

}  // namespace

extern "C" {

fit_status fit_port_rhs(fit_grid* g, int nfreq, const double* omega, int nedge, const long long* edges,
                        const double* signs, double current, void* b, void* stream) {
  FIT_REQUIRE(g && omega && b && nfreq >= 1 && nedge >= 0, "fit_port_rhs: bad argument");
  FIT_REQUIRE(nedge == 0 || (edges && signs), "fit_port_rhs: null edge list");
  FIT_REQUIRE(g->has_materials, "fit_port_rhs: materials not set");
  FIT_REQUIRE(std::isfinite(current), "fit_port_rhs: current must be finite");
  for (int f = 0; f < nfreq; ++f) FIT_REQUIRE(std::isfinite(omega[f]), "fit_port_rhs: omega must be finite");
  for (int q = 0; q < nedge; ++q) FIT_REQUIRE(edges[q] >= 0 && edges[q] < g->ne, "fit_port_rhs: edge out of range");
  FIT_CHECK_CUDA(cudaSetDevice(g->device));  // temporaries and kernels on the grid's device
  cudaStream_t s = (cudaStream_t)stream;
  FIT_CHECK_CUDA(cudaMemsetAsync(b, 0, (size_t)nfreq * g->ne * sizeof(double2), s));
  if (nedge == 0) {
    FIT_CHECK_CUDA(cudaStreamSynchronize(s));
    return FIT_OK;
  }
  FitDevTmp tmp(g);
  void *d_om, *d_e, *d_s;
  fit_status st;
  if ((st = tmp.copy(&d_om, omega, nfreq * sizeof(double), s)) != FIT_OK) return st;
  if ((st = tmp.copy(&d_e, edges, nedge * sizeof(long long), s)) != FIT_OK) return st;
  if ((st = tmp.copy(&d_s, signs, nedge * sizeof(double), s)) != FIT_OK) return st;
  const long long n = (long long)nfreq * nedge;
  k_port_rhs<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const double*)d_om, nfreq, (const long long*)d_e,
                                                          (const double*)d_s, nedge, current, g->mask, g->nx, g->ny,
                                                          g->nxp, g->ne, (double2*)b);
  FIT_CHECK_CUDA(cudaGetLastError());
  FIT_CHECK_CUDA(cudaStreamSynchronize(s));  // the temporaries are freed on return
  return FIT_OK;
}

fit_status fit_probe_voltages(fit_grid* g, int nfreq, const void* x, int nprobe, const int* off,
                              const long long* edges, const double* signs, double* V, void* stream) {
  FIT_REQUIRE(g && x && V && nfreq >= 1 && nprobe >= 1 && off, "fit_probe_voltages: bad argument");
  FIT_REQUIRE(off[0] == 0, "fit_probe_voltages: off[0] must be 0");
  for (int q = 0; q < nprobe; ++q) FIT_REQUIRE(off[q + 1] >= off[q], "fit_probe_voltages: off must not decrease");
  FIT_REQUIRE((long long)nfreq * nprobe <= 0x7fffffffLL, "fit_probe_voltages: too many (probe, system) pairs");
  const int nedge = off[nprobe];
  FIT_REQUIRE(nedge == 0 || (edges && signs), "fit_probe_voltages: null edge list");
  for (int k = 0; k < nedge; ++k)
    FIT_REQUIRE(edges[k] >= 0 && edges[k] < g->ne, "fit_probe_voltages: edge out of range");
  FIT_CHECK_CUDA(cudaSetDevice(g->device));  // temporaries and kernels on the grid's device
  cudaStream_t s = (cudaStream_t)stream;
  FitDevTmp tmp(g);
  void *d_off, *d_e, *d_s, *d_v;
  fit_status st;
  if ((st = tmp.copy(&d_off, off, (nprobe + 1) * sizeof(int), s)) != FIT_OK) return st;
  if ((st = tmp.copy(&d_e, edges, nedge * sizeof(long long), s)) != FIT_OK) return st;
  if ((st = tmp.copy(&d_s, signs, nedge * sizeof(double), s)) != FIT_OK) return st;
  if ((st = tmp.alloc(&d_v, (size_t)nfreq * nprobe * sizeof(double2))) != FIT_OK) return st;
  k_probe<<<(unsigned)((long long)nfreq * nprobe), 256, 0, s>>>((const double2*)x, g->ne, (const int*)d_off, (const long long*)d_e,
                                               (const double*)d_s, nprobe, (double2*)d_v);
  FIT_CHECK_CUDA(cudaGetLastError());
  FIT_CHECK_CUDA(cudaMemcpyAsync(V, d_v, (size_t)nfreq * nprobe * sizeof(double2), cudaMemcpyDeviceToHost, s));
  FIT_CHECK_CUDA(cudaStreamSynchronize(s));
  return FIT_OK;
}

fit_status fit_z_to_s(int P, const double* Z, double z0, double* S) {
  FIT_REQUIRE(P >= 1 && Z && S && z0 > 0 && std::isfinite(z0), "fit_z_to_s: bad argument");
  // S (Z + z0 1) = Z - z0 1, i.e. (Z + z0 1)^T S^T = (Z - z0 1)^T: Gauss-Jordan with partial pivoting
  // on M = (Z + z0 1)^T, right-hand sides R = (Z - z0 1)^T (complex, row-major, P x P)
  std::vector<double> M(2 * P * P), R(2 * P * P);
  for (int r = 0; r < P; ++r)
    for (int c = 0; c < P; ++c) {
      const double zr = Z[2 * (c * P + r)], zi = Z[2 * (c * P + r) + 1];  // (Z^T)[r][c] = Z[c][r]
      const double d = r == c ? z0 : 0.0;
      M[2 * (r * P + c)] = zr + d;
      M[2 * (r * P + c) + 1] = zi;
      R[2 * (r * P + c)] = zr - d;
      R[2 * (r * P + c) + 1] = zi;
    }
  for (int c = 0; c < P; ++c) {
    int piv = c;
    double best = -1.0;
    for (int r = c; r < P; ++r) {
      const double a = std::hypot(M[2 * (r * P + c)], M[2 * (r * P + c) + 1]);
      if (a > best) {
        best = a;
        piv = r;
      }
    }
    FIT_REQUIRE(best > 0.0 && std::isfinite(best), "fit_z_to_s: Z + z0 1 is singular");
    if (piv != c)
      for (int k = 0; k < P; ++k)
        for (int h = 0; h < 2; ++h) {
          std::swap(M[2 * (c * P + k) + h], M[2 * (piv * P + k) + h]);
          std::swap(R[2 * (c * P + k) + h], R[2 * (piv * P + k) + h]);
        }
    const double pr = M[2 * (c * P + c)], pi = M[2 * (c * P + c) + 1], den = pr * pr + pi * pi;
    const double ir = pr / den, ii = -pi / den;  // 1 / pivot
    for (int k = 0; k < P; ++k) {
      double a = M[2 * (c * P + k)], b = M[2 * (c * P + k) + 1];
      M[2 * (c * P + k)] = a * ir - b * ii;
      M[2 * (c * P + k) + 1] = a * ii + b * ir;
      a = R[2 * (c * P + k)];
      b = R[2 * (c * P + k) + 1];
      R[2 * (c * P + k)] = a * ir - b * ii;
      R[2 * (c * P + k) + 1] = a * ii + b * ir;
    }
    for (int r = 0; r < P; ++r) {
      if (r == c) continue;
      const double fr = M[2 * (r * P + c)], fi = M[2 * (r * P + c) + 1];
      if (fr == 0.0 && fi == 0.0) continue;
      for (int k = 0; k < P; ++k) {
        const double mr = M[2 * (c * P + k)], mi = M[2 * (c * P + k) + 1];
        M[2 * (r * P + k)] -= fr * mr - fi * mi;
        M[2 * (r * P + k) + 1] -= fr * mi + fi * mr;
        const double rr = R[2 * (c * P + k)], ri = R[2 * (c * P + k) + 1];
        R[2 * (r * P + k)] -= fr * rr - fi * ri;
        R[2 * (r * P + k) + 1] -= fr * ri + fi * rr;
      }
    }
  }
  // R now holds S^T
  for (int r = 0; r < P; ++r)
    for (int c = 0; c < P; ++c) {
      S[2 * (r * P + c)] = R[2 * (c * P + r)];
      S[2 * (r * P + c) + 1] = R[2 * (c * P + r) + 1];
    }
  return FIT_OK;
}

fit_status fit_z_parameters(fit_grid* g, int nfreq, const double* omega, int nport, const int* off,
                            const long long* edges, const double* signs, double current, double tol,
                            const fit_solve_opts* opts, double* Z, fit_solve_report* report) {
  FIT_REQUIRE(g && omega && off && Z && nfreq >= 1 && nport >= 1, "fit_z_parameters: bad argument");
  FIT_REQUIRE(current != 0.0 && std::isfinite(current), "fit_z_parameters: current must be finite and nonzero");
  for (int f = 0; f < nfreq; ++f) FIT_REQUIRE(std::isfinite(omega[f]), "fit_z_parameters: omega must be finite");
  FIT_REQUIRE(off[0] == 0, "fit_z_parameters: off[0] must be 0");
  for (int q = 0; q < nport; ++q) FIT_REQUIRE(off[q + 1] >= off[q], "fit_z_parameters: off must not decrease");
  FIT_REQUIRE(off[nport] == 0 || (edges && signs), "fit_z_parameters: null edge list");
  for (int k = 0; k < off[nport]; ++k)
    FIT_REQUIRE(edges[k] >= 0 && edges[k] < g->ne, "fit_z_parameters: edge out of range");
  FIT_REQUIRE(g->has_materials, "fit_z_parameters: materials not set");
  const long long nsys = (long long)nport * nfreq;
  FIT_REQUIRE(nsys <= (1 << 20), "fit_z_parameters: too many (port, frequency) systems");
  fit_solve_opts o;
  if (opts)
    o = *opts;
  else
    fit_solve_opts_default(&o);
  FIT_CHECK_CUDA(cudaSetDevice(g->device));
  // one batch of nport * nfreq systems: system (j, f) at j * nfreq + f is port j excited alone at omega_f
  const size_t vbytes = (size_t)nsys * g->ne * sizeof(double2);
  FitDevTmp tmp(g);
  void *d_b, *d_x;
  fit_status st;
  if ((st = tmp.alloc(&d_b, vbytes)) != FIT_OK) return st;
  if ((st = tmp.alloc(&d_x, vbytes)) != FIT_OK) return st;
  std::vector<double> om((size_t)nsys);
  for (int j = 0; j < nport; ++j) {
    for (int f = 0; f < nfreq; ++f) om[(size_t)j * nfreq + f] = omega[f];
    const int n = off[j + 1] - off[j];
    if ((st = fit_port_rhs(g, nfreq, omega, n, n ? edges + off[j] : nullptr, n ? signs + off[j] : nullptr, current,
                           (double2*)d_b + (size_t)j * nfreq * g->ne, o.stream)) != FIT_OK)
      return st;
  }
  std::vector<fit_solve_report> rep((size_t)nsys);
  const fit_status solved = fit_solve(g, (int)nsys, om.data(), d_b, d_x, tol, &o, rep.data());
  if (report)  // per-system outcomes are reported on every path that reached the solve
    for (long long t = 0; t < nsys; ++t) report[t] = rep[(size_t)t];
  if (solved < 0) return solved;
  std::vector<double> V((size_t)nsys * nport * 2);
  if ((st = fit_probe_voltages(g, (int)nsys, d_x, nport, off, edges, signs, V.data(), o.stream)) != FIT_OK)
    return st;
  // Z[f][i][j] = V_i / I with port j excited at omega_f
  for (int j = 0; j < nport; ++j)
    for (int f = 0; f < nfreq; ++f)
      for (int i = 0; i < nport; ++i) {
        const size_t src = 2 * (((size_t)j * nfreq + f) * nport + i), dst = 2 * (((size_t)f * nport + i) * nport + j);
        Z[dst] = V[src] / current;
        Z[dst + 1] = V[src + 1] / current;
      }
  return solved;
}

}  // extern "C"
