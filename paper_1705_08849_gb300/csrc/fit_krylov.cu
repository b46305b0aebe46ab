// Krylov solvers on the fused FIT operator (Sec. IV: the short-listed bcgs and gmres family).
//
// Structure of fit_solve for a batch of B systems A(w_b) x_b = b_b sharing one geometry:
//
//   outer loop (FP64 iterative refinement; the true residual judges convergence):
//       r = b - A x            (complex128 apply with a fused residual epilogue, FP64 norm)
//       stop if ||r|| <= tol ||b||
//       r~ = r / ||r||         (to complex64 for FIT_SOLVE_MIXED, complex128 for FIT_SOLVE_C128)
//       inner Krylov solve  A_in d = r~  to a relative tolerance (BiCGStab, or one FGMRES(m) cycle)
//       x += s_in ||r|| d      (A_in = s_in A: the complex64 coefficients are scaled by s_in)
//
// With FIT_SOLVE_C128 the same loop is plain complex128 Krylov restarted from the true residual.
// Every kernel is predicated on a per-system status word, so converged systems stop updating while
// the rest of the batch continues.  Scalars (rho, alpha, omega, Hessenberg, Givens) live on the
// device; with opts->use_graph the whole solve is one CUDA graph: a WHILE node for the outer loop
// holding the inner loop (a nested WHILE node for BiCGStab, m unrolled steps for FGMRES), with
// device-side conditions.  Every loop has a device-side iteration guard, so it always ends.
//
// Inner products: per-thread partial sums in the vector precision, warp shuffles, then FP64
// from the warp level up, in a fixed order (deterministic run to run).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "fit_internal.cuh"

namespace {

enum { SYS_RUN = 0, SYS_CONV = 1, SYS_BREAK = 2, SYS_MAXIT = 3, SYS_NAN = 4 };

struct Sys {
  double bnorm2;       // ||b||^2
  double rnorm2;       // ||b - A x||^2 of the current x
  double tol2;         // (tol ||b||)^2
  double rscale;       // ||r|| at the start of the current inner solve
  double corr;         // s_in * rscale: x += corr * d
  double inner_tol2;   // inner stop threshold on ||r_in||^2
  double rin2;         // inner recurrence residual ||r_in||^2
  double best2;        // smallest true residual seen (stagnation test)
  double2 rho, alpha, omega, beta;
  double inv_hn;       // FGMRES: 1 / h_{j+1,j}
  int outer_status;    // SYS_*
  int outer;           // refinement steps done
  int iters;           // inner iterations summed over refinement steps
  int inner_status;    // SYS_RUN while the inner solve of this system is active
  int inner_it;        // iterations of the current inner solve
  int stagn;           // consecutive refinement steps without residual decrease
  int jlast;           // FGMRES: Arnoldi steps done in the current cycle
  int max_inner;       // inner iteration cap of the current inner solve
  double rin_min2;     // smallest inner recurrence residual of the current inner solve
  double rin0;         // inner residual at the start of the current inner solve
  int hist;            // history snapshots written
  int hist_pad;
  int rin_min_it;      // iteration at which it was reached
  int mr;              // 1: the step length amr of this refinement step is still to be applied
  int replay;          // > 0: the last inner solve failed; stop the next one at this iteration
  double2 amr;         // minimal-residual step length along this step's correction
};

struct Ctl {
  int inner_guard;
  int outer_guard;
  int cond;
  int pad;
};

struct P {
  int B;
  long long ne;
  int nblk;          // blocks per system of the vector kernels
  int pstride;       // doubles per partial slot of the vector kernels
  int m;             // FGMRES restart length
  int max_iter, max_outer;
  double tol, inner_tol;
  int mixed;         // inner precision is complex64
  double s_in;       // A_in = s_in * A
  double tiny;       // breakdown threshold for the inner precision
  int stall;         // inner solve stops after this many iterations without a new minimum
  int precond;       // right preconditioner of the inner solve (FIT_PC_*)
  int pc_every;      // FIT_PC_UNET: Arnoldi steps j with (j + 1) % pc_every == 0 take the network's direction
  const volatile int* abort;  // the grid's abort word (pinned host memory), polled by the loop conditions
  int* err;                   // the grid's error word: set to 2 when the abort word ends the loops
};

__device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ inline double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ inline double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ inline double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ inline double2 cdiv(double2 a, double2 b) {
  double d = cabs2(b);
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ inline bool cfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }

template <typename T> __device__ inline typename cplx<T>::t mkc(double re, double im);
template <> __device__ inline float2 mkc<float>(double re, double im) { return make_float2((float)re, (float)im); }
template <> __device__ inline double2 mkc<double>(double re, double im) { return make_double2(re, im); }

// ------------------------------------------------------------------------------------------------
// Fixed-order reduction of the per-block partials of one system, then a scalar operation.
// ------------------------------------------------------------------------------------------------
// All 256 threads of the block call it; thread 0 receives out[0..NQ-1] = sum over the nslots
// partials pb[s * stride + q] in a fixed order (threads take slots t, t + 256, ..., then a tree).
// The partials are read through L2 (another block of the same kernel may just have written them).
template <int NQ>
__device__ inline void reduce_slots(const double* pb, long long nslots, int stride, double* out) {
  __shared__ double red[256][NQ];
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  for (long long s = threadIdx.x; s < nslots; s += 256)
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] += __ldcg(pb + s * stride + q);
#pragma unroll
  for (int q = 0; q < NQ; ++q) red[threadIdx.x][q] = acc[q];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
#pragma unroll
      for (int q = 0; q < NQ; ++q) red[threadIdx.x][q] += red[threadIdx.x + h][q];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < NQ; ++q) out[q] = red[0][q];
}

template <int NQ, class Op>
__global__ void __launch_bounds__(256) fin_kernel(const double* __restrict__ part, long long nslots, int stride,
                                                  Sys* sys, P p, Op op) {
  const int b = blockIdx.x;
  if (!op.active(sys[b])) return;
  double s[NQ];
  reduce_slots<NQ>(part + (long long)b * nslots * stride, nslots, stride, s);
  if (threadIdx.x == 0) op.apply(sys[b], s, p, b);
}

// The last block of a vector kernel to finish (per system) reduces the partial sums of all blocks and
// applies the scalar operation, in place of a separate fin_kernel launch.  Every block calls it after
// fit_block_sum has written its partials; cnt[b] counts the finished blocks of system b and is reset by
// the last one, so it is zero again for the next launch.
template <int NQ, class Op>
__device__ inline void last_block_fin(const double* part, unsigned* cnt, Sys* sys, const P& p, int b, Op op) {
  __shared__ int last;
  if (threadIdx.x == 0) {
    __threadfence();  // this block's partials are visible before its arrival is counted
    last = atomicAdd(&cnt[b], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s[NQ];
  reduce_slots<NQ>(part + (long long)b * p.nblk * p.pstride, p.nblk, p.pstride, s);
  if (threadIdx.x == 0) {
    op.apply(sys[b], s, p, b);
    cnt[b] = 0u;
  }
}

// ---- outer-loop operations --------------------------------------------------------------------
struct OpOuterInit {  // q2 = ||b||^2
  __device__ bool active(const Sys&) const { return true; }
  __device__ void apply(Sys& s, const double* q, const P& p, int) const {
    s.bnorm2 = q[2];
    s.rnorm2 = q[2];
    s.best2 = q[2];
    s.tol2 = p.tol * p.tol * q[2];
    s.rscale = sqrt(q[2]);
    s.outer = 0;
    s.iters = 0;
    s.stagn = 0;
    s.mr = 0;
    s.replay = 0;
    s.inner_status = SYS_CONV;
    s.inner_it = 0;
    if (!isfinite(q[2])) s.outer_status = SYS_NAN;
    else if (q[2] == 0.0) s.outer_status = SYS_CONV;
    else s.outer_status = SYS_RUN;
  }
};

// After the correction c d: with r0 = b - A x (before) and r1 = b - A (x + c d) (after, both
// computed in FP64), u = r0 - r1 = A c d.  The step length along the correction that minimises
// the true residual, amr = <u, r0> / <u, u>, gives x + amr c d with residual (1 - amr) r0 + amr r1
// (linear in the step, so again b - A x exactly up to rounding), whose norm never exceeds that of
// r0 or r1: a correction that would raise the residual is shortened instead, down to none.
// q0 = ||r0||^2, q1, q2 = Re, Im <r1, r0>, q3 = ||r1||^2.
struct OpOuter {
  __device__ bool active(const Sys& s) const { return s.outer_status == SYS_RUN; }
  __device__ void apply(Sys& s, const double* q, const P& p, int) const {
    const double a = q[0], c = q[3];
    const double2 bb = make_double2(q[1], q[2]);
    s.outer += 1;
    s.iters += s.inner_it;
    s.mr = 1;
    double2 al = make_double2(0.0, 0.0);
    double r2 = a;
    const double den = a - 2.0 * bb.x + c;  // ||u||^2
    // a dropped correction (corr = 0) keeps r = r0 bit for bit, so that a replayed inner solve
    // starts from exactly the residual the failed one started from
    if (s.corr != 0.0 && isfinite(c) && cfinite(bb) && den > 0.0) {
      al = make_double2((a - bb.x) / den, -bb.y / den);  // <u, r0> / ||u||^2
      // ||(1 - amr) r0 + amr r1||^2 = a - |a - bb|^2 / den = c - |c - bb|^2 / den; evaluated from the
      // smaller of a and c, so that its rounding error is relative to the smaller residual
      const double base = fmin(a, c);
      r2 = fmax(0.0, base - ((base - bb.x) * (base - bb.x) + bb.y * bb.y) / den);
    }
    s.amr = al;
    if (!isfinite(a)) { s.outer_status = SYS_NAN; return; }
    if (s.corr != 0.0) {  // a dropped step leaves the residual and its scale exactly as they were
      s.rnorm2 = r2;
      s.rscale = sqrt(r2);
    } else {
      r2 = s.rnorm2;
    }
    if (r2 <= s.tol2) { s.outer_status = SYS_CONV; return; }
    if (r2 < 0.99 * s.best2) { s.best2 = r2; s.stagn = 0; }
    else s.stagn += 1;
    if (s.outer >= p.max_outer || s.iters >= p.max_iter || s.stagn >= 5) s.outer_status = SYS_MAXIT;
  }
};

// inner start: q0 = ||r~||^2 (for BiCGStab rho = <r^, r> = ||r~||^2)
struct OpInnerStart {
  __device__ bool active(const Sys&) const { return true; }
  __device__ void apply(Sys& s, const double* q, const P& p, int) const {
    if (s.outer_status != SYS_RUN) { s.inner_status = SYS_CONV; return; }
    s.inner_status = SYS_RUN;
    s.inner_it = 0;
    s.jlast = 0;
    s.rho = make_double2(q[0], 0.0);
    s.alpha = make_double2(1.0, 0.0);
    s.omega = make_double2(1.0, 0.0);
    s.beta = make_double2(0.0, 0.0);
    s.rin2 = q[0];
    s.rin_min2 = q[0];
    s.rin0 = q[0];
    s.rin_min_it = 0;
    s.corr = p.s_in * s.rscale;
    // relative target of this inner solve: no tighter than needed for the outer tolerance
    double need = 0.5 * sqrt(s.tol2) / s.rscale;
    double it = p.mixed ? fmax(p.inner_tol, need) : fmax(need, 1e-15);
    s.inner_tol2 = it * it * q[0];
    s.max_inner = max(1, p.max_iter - s.iters);
    // The previous inner solve ended above its start and its correction was dropped.  This one
    // starts from the same residual (x and r are unchanged) and runs the same kernels, so it retraces
    // the same iterates: stop it where the last one had its smallest residual and keep that iterate.
    if (s.replay > 0) {
      s.max_inner = min(s.max_inner, s.replay);
      s.replay = 0;
    }
  }
};

// ---- COCG operations ---------------------------------------------------------------------------
// Conjugate orthogonal CG for the complex symmetric A (A^T = A): CG with the unconjugated bilinear
// form (u, v) = sum_i u_i v_i in place of the inner product, right/left-symmetric Jacobi
// preconditioner z = D^-1 r.  Per iteration: q = A p, alpha = rho / (p, q), d += alpha p,
// r -= alpha q, rho' = (r, D^-1 r), beta = rho' / rho, p = D^-1 r + beta p.
struct OpCocgStart {  // q0,q1 = (r~, D^-1 r~), q2 = ||r~||^2
  __device__ bool active(const Sys&) const { return true; }
  __device__ void apply(Sys& s, const double* q, const P& p, int b) const {
    const double qq[3] = {q[2], 0.0, 0.0};
    OpInnerStart{}.apply(s, qq, p, b);
    s.rho = make_double2(q[0], q[1]);
    if (s.inner_status == SYS_RUN && !cfinite(s.rho)) s.inner_status = SYS_NAN;
  }
};

struct OpCocgAlpha {  // q0,q1 = (p, A p)
  __device__ bool active(const Sys& s) const { return s.inner_status == SYS_RUN; }
  __device__ void apply(Sys& s, const double* q, const P& p, int) const {
    double2 sig = make_double2(q[0], q[1]);
    if (!cfinite(sig)) { s.inner_status = SYS_NAN; return; }
    if (sqrt(cabs2(sig)) < p.tiny) { s.inner_status = SYS_BREAK; return; }
    s.alpha = cdiv(s.rho, sig);
  }
};

struct OpCocgRho {  // q0,q1 = (r, D^-1 r), q2 = ||r||^2
  __device__ bool active(const Sys& s) const { return s.inner_status == SYS_RUN; }
  __device__ void apply(Sys& s, const double* q, const P& p, int) const {
    double2 rn = make_double2(q[0], q[1]);
    double rr = q[2];
    s.inner_it += 1;
    s.rin2 = rr;
    if (!cfinite(rn) || !isfinite(rr)) { s.inner_status = SYS_NAN; return; }
    if (rr <= s.inner_tol2) { s.inner_status = SYS_CONV; return; }
    if (s.inner_it >= s.max_inner) { s.inner_status = SYS_MAXIT; return; }
    if (rr < s.rin_min2) { s.rin_min2 = rr; s.rin_min_it = s.inner_it; }
    // a stalled or diverging inner solve hands back to the refinement loop (as for BiCGStab)
    if (s.inner_it - s.rin_min_it > p.stall || rr > 1e8 * s.rin_min2) {
      s.inner_status = SYS_MAXIT;
      if (rr > s.rin0) {
        s.corr = 0.0;
        s.replay = s.rin_min_it;
      }
      return;
    }
    if (sqrt(cabs2(rn)) < p.tiny) { s.inner_status = SYS_BREAK; return; }
    s.beta = cdiv(rn, s.rho);
    s.rho = rn;
  }
};

// ---- COCR operations ---------------------------------------------------------------------------
// Conjugate orthogonal conjugate residual for the complex symmetric A: the conjugate-residual
// recurrences with the unconjugated bilinear form and a symmetric diagonal preconditioner M = D^-1
// (COCR on M^{1/2} A M^{1/2}, written in the original variables).  The start sets z = M r~, p = q = 0;
// every iteration then runs
//   w = A z;  rho' = (z, w);  beta = rho' / rho (0 on the first);  p = z + beta p;  q = w + beta q;
//   alpha = rho' / (q, M q);  d += alpha p;  r -= alpha q;  z = M r
// so that q = A p throughout and each iteration costs one apply.
struct OpCocrStart {  // q2 = ||r~||^2
  __device__ bool active(const Sys&) const { return true; }
  __device__ void apply(Sys& s, const double* q, const P& p, int b) const {
    const double qq[3] = {q[2], 0.0, 0.0};
    OpInnerStart{}.apply(s, qq, p, b);
    s.beta = make_double2(0.0, 0.0);
  }
};

struct OpCocrBeta {  // q0,q1 = (z, A z)
  __device__ bool active(const Sys& s) const { return s.inner_status == SYS_RUN; }
  __device__ void apply(Sys& s, const double* q, const P& p, int) const {
    const double2 rn = make_double2(q[0], q[1]);
    if (!cfinite(rn)) { s.inner_status = SYS_NAN; return; }
    if (sqrt(cabs2(rn)) < p.tiny) { s.inner_status = SYS_BREAK; return; }
    s.beta = s.inner_it == 0 ? make_double2(0.0, 0.0) : cdiv(rn, s.rho);
    s.rho = rn;
  }
};

struct OpCocrAlpha {  // q0,q1 = (q, M q)
  __device__ bool active(const Sys& s) const { return s.inner_status == SYS_RUN; }
  __device__ void apply(Sys& s, const double* q, const P& p, int) const {
    const double2 sig = make_double2(q[0], q[1]);
    if (!cfinite(sig)) { s.inner_status = SYS_NAN; return; }
    if (sqrt(cabs2(sig)) < p.tiny) { s.inner_status = SYS_BREAK; return; }
    s.alpha = cdiv(s.rho, sig);
  }
};

struct OpCocrRes {  // q2 = ||r||^2 after the update
  __device__ bool active(const Sys& s) const { return s.inner_status == SYS_RUN; }
  __device__ void apply(Sys& s, const double* q, const P& p, int) const {
    const double rr = q[2];
    s.inner_it += 1;
    s.rin2 = rr;
    if (!isfinite(rr)) { s.inner_status = SYS_NAN; return; }
    if (rr <= s.inner_tol2) { s.inner_status = SYS_CONV; return; }
    if (s.inner_it >= s.max_inner) { s.inner_status = SYS_MAXIT; return; }
    if (rr < s.rin_min2) { s.rin_min2 = rr; s.rin_min_it = s.inner_it; }
    if (s.inner_it - s.rin_min_it > p.stall || rr > 1e8 * s.rin_min2) {  // as for COCG
      s.inner_status = SYS_MAXIT;
      if (rr > s.rin0) {
        s.corr = 0.0;
        s.replay = s.rin_min_it;
      }
    }
  }
};

// ---- BiCGStab operations -----------------------------------------------------------------------
struct OpAlpha {  // q0,q1 = <r^, v>
  __device__ bool active(const Sys& s) const { return s.inner_status == SYS_RUN; }
  __device__ void apply(Sys& s, const double* q, const P& p, int) const {
    double2 sig = make_double2(q[0], q[1]);
    if (!cfinite(sig)) { s.inner_status = SYS_NAN; return; }
    if (sqrt(cabs2(sig)) < p.tiny) { s.inner_status = SYS_BREAK; return; }
    s.alpha = cdiv(s.rho, sig);
  }
};

struct OpOmega {  // q0,q1 = <t, s>, q2 = <t, t>
  __device__ bool active(const Sys& s) const { return s.inner_status == SYS_RUN; }
  __device__ void apply(Sys& s, const double* q, const P&, int) const {
    double tt = q[2];
    if (!isfinite(tt)) { s.inner_status = SYS_NAN; return; }
    s.omega = tt > 0.0 ? make_double2(q[0] / tt, q[1] / tt) : make_double2(0.0, 0.0);
  }
};

struct OpRho {  // q0,q1 = <r^, r_new>, q2 = ||r_new||^2
  __device__ bool active(const Sys& s) const { return s.inner_status == SYS_RUN; }
  __device__ void apply(Sys& s, const double* q, const P& p, int) const {
    double2 rn = make_double2(q[0], q[1]);
    double rr = q[2];
    s.inner_it += 1;
    s.rin2 = rr;
    if (!cfinite(rn) || !isfinite(rr)) { s.inner_status = SYS_NAN; return; }
    if (rr <= s.inner_tol2) { s.inner_status = SYS_CONV; return; }
    if (s.inner_it >= s.max_inner) { s.inner_status = SYS_MAXIT; return; }
    if (rr < s.rin_min2) { s.rin_min2 = rr; s.rin_min_it = s.inner_it; }
    // a stalled or diverging inner solve hands back to the refinement loop, which restarts it
    // from the true residual
    if (s.inner_it - s.rin_min_it > p.stall || rr > 1e8 * s.rin_min2) {  // 1e4 in norm
      s.inner_status = SYS_MAXIT;
      // an inner solve that ends above its starting residual would make x worse: drop it
      if (rr > s.rin0) {
        s.corr = 0.0;
        s.replay = s.rin_min_it;
      }
      return;
    }
    if (sqrt(cabs2(rn)) < p.tiny || sqrt(cabs2(s.omega)) < p.tiny) { s.inner_status = SYS_BREAK; return; }
    s.beta = cmul(cdiv(rn, s.rho), cdiv(s.alpha, s.omega));
    s.rho = rn;
  }
};

// ------------------------------------------------------------------------------------------------
// Vector kernels.  Grid (nblk, B); thread t of block k of system b owns the elements
// e = k*256 + t + n*nblk*256 (fixed assignment, so partial sums are reproducible).
// ------------------------------------------------------------------------------------------------
#define VEC_LOOP(p) for (long long e = blockIdx.x * 256LL + threadIdx.x; e < (p).ne; e += (long long)gridDim.x * 256)
#define PSLOT(p, b) ((((long long)(b) * (p).nblk + blockIdx.x)) * (p).pstride)

__global__ void __launch_bounds__(256) k_outer_init(const double2* __restrict__ rhs, double2* __restrict__ x,
                                                    double2* __restrict__ r, double* part, P p) {
  const int b = blockIdx.y;
  const long long off = (long long)b * p.ne;
  double acc[3] = {0, 0, 0};
  VEC_LOOP(p) {
    double2 v = rhs[off + e];
    x[off + e] = make_double2(0.0, 0.0);
    r[off + e] = v;
    acc[2] += v.x * v.x + v.y * v.y;
  }
  fit_block_sum<double, 3>(acc, part + PSLOT(p, b));
}

// r~ = r / ||r|| in the inner precision; BiCGStab: r^ = r~, p = v = d = 0; FGMRES: V0 = r~, d = 0
template <typename T, bool BICG>
__global__ void __launch_bounds__(256) k_inner_start(const double2* __restrict__ r128, const Sys* __restrict__ sys,
                                                     typename cplx<T>::t* rin, typename cplx<T>::t* rhat,
                                                     typename cplx<T>::t* pv, typename cplx<T>::t* v,
                                                     typename cplx<T>::t* d, double* part, P p) {
  using V = typename cplx<T>::t;
  const int b = blockIdx.y;
  T acc[3] = {T(0), T(0), T(0)};
  if (sys[b].outer_status == SYS_RUN) {
    const long long off = (long long)b * p.ne;
    const double sc = 1.0 / sys[b].rscale;
    VEC_LOOP(p) {
      double2 r = r128[off + e];
      V z = mkc<T>(r.x * sc, r.y * sc);
      rin[off + e] = z;
      d[off + e] = czero<V>();
      if (BICG) {
        rhat[off + e] = z;
        pv[off + e] = czero<V>();
        v[off + e] = czero<V>();
      }
      acc[0] += z.x * z.x + z.y * z.y;
    }
  }
  fit_block_sum<T, 3>(acc, part + PSLOT(p, b));
}

template <typename V>
__device__ inline V cmulv(V a, V b) {
  V o;
  o.x = a.x * b.x - a.y * b.y;
  o.y = a.x * b.y + a.y * b.x;
  return o;
}

// BiCGStab: p = r + beta (p - omega v); with a right preconditioner also p^ = D^-1 p
template <typename T>
__global__ void __launch_bounds__(256) k_bicg_p(const typename cplx<T>::t* __restrict__ r, typename cplx<T>::t* pv,
                                                const typename cplx<T>::t* __restrict__ v,
                                                const typename cplx<T>::t* __restrict__ dinv,
                                                typename cplx<T>::t* phat, const Sys* __restrict__ sys, P p) {
  using V = typename cplx<T>::t;
  const int b = blockIdx.y;
  if (sys[b].inner_status != SYS_RUN) return;
  const long long off = (long long)b * p.ne;
  const double2 bd = sys[b].beta, od = sys[b].omega;
  const T br = (T)bd.x, bi = (T)bd.y, orr = (T)od.x, oi = (T)od.y;
  VEC_LOOP(p) {
    V rr = r[off + e], pp = pv[off + e], vv = v[off + e];
    V t;  // p - omega v
    t.x = pp.x - (orr * vv.x - oi * vv.y);
    t.y = pp.y - (orr * vv.y + oi * vv.x);
    V o;
    o.x = rr.x + br * t.x - bi * t.y;
    o.y = rr.y + br * t.y + bi * t.x;
    pv[off + e] = o;
    if (dinv) phat[off + e] = cmulv(dinv[off + e], o);
  }
}

// BiCGStab: s = r - alpha v (in place in r); with a right preconditioner also s^ = D^-1 s
template <typename T>
__global__ void __launch_bounds__(256) k_bicg_s(typename cplx<T>::t* r, const typename cplx<T>::t* __restrict__ v,
                                                const typename cplx<T>::t* __restrict__ dinv,
                                                typename cplx<T>::t* shat, const Sys* __restrict__ sys, P p) {
  using V = typename cplx<T>::t;
  const int b = blockIdx.y;
  if (sys[b].inner_status != SYS_RUN) return;
  const long long off = (long long)b * p.ne;
  const T ar = (T)sys[b].alpha.x, ai = (T)sys[b].alpha.y;
  VEC_LOOP(p) {
    V rr = r[off + e], vv = v[off + e];
    rr.x -= ar * vv.x - ai * vv.y;
    rr.y -= ar * vv.y + ai * vv.x;
    r[off + e] = rr;
    if (dinv) shat[off + e] = cmulv(dinv[off + e], rr);
  }
}

// D^-1 of the diagonal preconditioner per system; masked edges: 1.  Jacobi: diag(A_in(w_b)) =
// nusum - w^2 M_eps + j w M_kappa (the Eq. Precond column-sum construction on the unsymmetrised
// operator).  eps_only: w^2 M_eps, the change of variable e' = M_eps^{1/2} e of the symmetrised form
// (Eq. e2s) applied as a split diagonal preconditioner (nusum is not read).  The constant factor w^2
// leaves the Krylov iterates unchanged and makes the preconditioned operator K / (w^2 M_eps) - 1 of
// order one: with M_eps^-1 alone the complex64 vectors reach ~1e20 and their products overflow FP32.
template <typename T>
__global__ void __launch_bounds__(256) k_dinv(const T* __restrict__ nusum, const T* __restrict__ ek,
                                              const uint8_t* __restrict__ mask, const double* __restrict__ omega,
                                              int nx, int ny, int nxp, typename cplx<T>::t* dinv, P p,
                                              int eps_only) {
  using V = typename cplx<T>::t;
  const int b = blockIdx.y;
  const double w = omega[b];
  const long long off = (long long)b * p.ne;
  VEC_LOOP(p) {
    long long c = e / 3;
    int q = (int)(e - 3 * c);
    long long i = c % nx, jj = (c / nx) % ny, k = c / ((long long)nx * ny);
    long long cp = i + (long long)nxp * (jj + (long long)ny * k);
    V o;
    if ((mask[cp] >> q) & 1) {
      o.x = T(1);
      o.y = T(0);
    } else if (eps_only) {
      const double me = (double)ek[6 * cp + q], wme = w * w * me;
      o.x = (T)(1.0 / (wme > 0.0 ? wme : me));  // w = 0: M_eps^-1 itself
      o.y = T(0);
    } else {
      double dr = (double)nusum[e] - w * w * (double)ek[6 * cp + q];
      double di = w * (double)ek[6 * cp + 3 + q];
      double den = dr * dr + di * di;
      o.x = (T)(dr / den);
      o.y = (T)(-di / den);
    }
    dinv[off + e] = o;
  }
}

// z = D^-1 v for FGMRES basis vector j
template <typename T>
__global__ void __launch_bounds__(256) k_fg_precond_diag(const typename cplx<T>::t* __restrict__ Vb,
                                                         typename cplx<T>::t* Zb, int j,
                                                         const typename cplx<T>::t* __restrict__ dinv,
                                                         const Sys* __restrict__ sys, P p) {
  const int b = blockIdx.y;
  if (sys[b].inner_status != SYS_RUN) return;
  const long long vs = (long long)p.B * p.ne;
  const long long off = (long long)b * p.ne;
  VEC_LOOP(p) { Zb[(long long)j * vs + off + e] = cmulv(dinv[off + e], Vb[(long long)j * vs + off + e]); }
}

// BiCGStab: d += alpha p + omega s; r = s - omega t; q0,q1 = <r^, r>, q2 = ||r||^2
template <typename T>
__global__ void __launch_bounds__(256) k_bicg_xr(typename cplx<T>::t* d, const typename cplx<T>::t* __restrict__ pv,
                                                 typename cplx<T>::t* r, const typename cplx<T>::t* __restrict__ t,
                                                 const typename cplx<T>::t* __restrict__ shat,
                                                 const typename cplx<T>::t* __restrict__ rhat, const Sys* __restrict__ sys,
                                                 double* part, P p) {
  using V = typename cplx<T>::t;
  const int b = blockIdx.y;
  if (sys[b].inner_status != SYS_RUN) return;
  const long long off = (long long)b * p.ne;
  const T ar = (T)sys[b].alpha.x, ai = (T)sys[b].alpha.y, orr = (T)sys[b].omega.x, oi = (T)sys[b].omega.y;
  T acc[3] = {T(0), T(0), T(0)};
  VEC_LOOP(p) {
    V s = r[off + e], pp = pv[off + e], tt = t[off + e], dd = d[off + e], rh = rhat[off + e];
    const V sx = shat ? shat[off + e] : s;  // the update uses the preconditioned s
    dd.x += (ar * pp.x - ai * pp.y) + (orr * sx.x - oi * sx.y);
    dd.y += (ar * pp.y + ai * pp.x) + (orr * sx.y + oi * sx.x);
    V rn;
    rn.x = s.x - (orr * tt.x - oi * tt.y);
    rn.y = s.y - (orr * tt.y + oi * tt.x);
    d[off + e] = dd;
    r[off + e] = rn;
    acc[0] += rh.x * rn.x + rh.y * rn.y;
    acc[1] += rh.x * rn.y - rh.y * rn.x;
    acc[2] += rn.x * rn.x + rn.y * rn.y;
  }
  fit_block_sum<T, 3>(acc, part + PSLOT(p, b));
}

// q0,q1 = <t, s>, q2 = <t, t> (BiCGStab omega with a right preconditioner)
template <typename T>
__global__ void __launch_bounds__(256) k_dots_ts(const typename cplx<T>::t* __restrict__ t,
                                                 const typename cplx<T>::t* __restrict__ sv, const Sys* __restrict__ sys,
                                                 double* part, P p) {
  using V = typename cplx<T>::t;
  const int b = blockIdx.y;
  if (sys[b].inner_status != SYS_RUN) return;
  const long long off = (long long)b * p.ne;
  T acc[3] = {T(0), T(0), T(0)};
  VEC_LOOP(p) {
    V tt = t[off + e], ss = sv[off + e];
    acc[0] += tt.x * ss.x + tt.y * ss.y;
    acc[1] += tt.x * ss.y - tt.y * ss.x;
    acc[2] += tt.x * tt.x + tt.y * tt.y;
  }
  fit_block_sum<T, 3>(acc, part + PSLOT(p, b));
}

// history snapshot of x after an outer step: slot sys.hist when outer % every == 0 (copy), then
// k_history_count advances the slot (a separate launch, so every copy block has read the old slot)
__global__ void __launch_bounds__(256) k_history(const double2* __restrict__ x, double2* hist, const Sys* __restrict__ sys,
                                                 int every, int len, P p) {
  const int b = blockIdx.y;
  const Sys& s = sys[b];
  if (s.outer == 0 || s.outer % every != 0 || s.hist >= len || s.hist_pad == s.outer) return;
  const long long off = (long long)b * p.ne;
  double2* dst = hist + ((long long)s.hist * p.B + b) * p.ne;
  VEC_LOOP(p) { dst[e] = x[off + e]; }
}
__global__ void k_history_count(Sys* sys, int every, int len, P p) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= p.B) return;
  Sys& s = sys[b];
  if (s.outer == 0 || s.outer % every != 0 || s.hist >= len || s.hist_pad == s.outer) return;
  s.hist += 1;
  s.hist_pad = s.outer;  // one snapshot per outer step
}

// x128 += corr * d (only systems still in the outer loop)
template <typename T>
__global__ void __launch_bounds__(256) k_update_x(double2* x, const typename cplx<T>::t* __restrict__ d,
                                                  const Sys* __restrict__ sys, P p) {
  const int b = blockIdx.y;
  if (sys[b].outer_status != SYS_RUN) return;
  const long long off = (long long)b * p.ne;
  const double c = sys[b].corr;
  if (c == 0.0) return;  // a dropped correction: 0 * d would turn an overflowed d into NaN
  VEC_LOOP(p) {
    auto dd = d[off + e];
    double2 xx = x[off + e];
    xx.x += c * (double)dd.x;
    xx.y += c * (double)dd.y;
    x[off + e] = xx;
  }
}

// r_prev = r before a correction is tried
__global__ void __launch_bounds__(256) k_copy_r(const double2* __restrict__ r, double2* __restrict__ rprev,
                                                const Sys* __restrict__ sys, P p) {
  const int b = blockIdx.y;
  if (sys[b].outer_status != SYS_RUN) return;
  const long long off = (long long)b * p.ne;
  VEC_LOOP(p) rprev[off + e] = r[off + e];
}

// partials ||r0||^2, Re <r1, r0>, Im <r1, r0>, ||r1||^2 (r0 = r before the correction, r1 after)
__global__ void __launch_bounds__(256) k_mr_dots(const double2* __restrict__ r0, const double2* __restrict__ r1,
                                                 const Sys* __restrict__ sys, double* part, P p) {
  const int b = blockIdx.y;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if (sys[b].outer_status == SYS_RUN) {
    const long long off = (long long)b * p.ne;
    VEC_LOOP(p) {
      const double2 u = r0[off + e], v = r1[off + e];
      acc[0] += u.x * u.x + u.y * u.y;
      acc[1] += v.x * u.x + v.y * u.y;
      acc[2] += v.x * u.y - v.y * u.x;
      acc[3] += v.x * v.x + v.y * v.y;
    }
  }
  fit_block_sum<double, 4>(acc, part + PSLOT(p, b));
}

// apply the step length: x += (amr - 1) corr d, r = (1 - amr) r0 + amr r1 (r holds r1)
template <typename T>
__global__ void __launch_bounds__(256) k_mr_combine(double2* x, const typename cplx<T>::t* __restrict__ d,
                                                    double2* r, const double2* __restrict__ r0,
                                                    const Sys* __restrict__ sys, P p) {
  const int b = blockIdx.y;
  if (!sys[b].mr) return;
  const long long off = (long long)b * p.ne;
  const double2 al = sys[b].amr;
  const double c = sys[b].corr;
  const double2 f = make_double2(c * (al.x - 1.0), c * al.y);  // (amr - 1) corr
  const double2 g = make_double2(1.0 - al.x, -al.y);          // 1 - amr
  VEC_LOOP(p) {
    if (c != 0.0) {
      const auto dd = d[off + e];
      const double dx = (double)dd.x, dy = (double)dd.y;
      double2 xx = x[off + e];
      xx.x += f.x * dx - f.y * dy;
      xx.y += f.x * dy + f.y * dx;
      x[off + e] = xx;
    }
    const double2 u = r0[off + e], v = r[off + e];
    if (al.x == 0.0 && al.y == 0.0) r[off + e] = u;  // no step: r0 bit for bit
    else
      r[off + e] = make_double2(g.x * u.x - g.y * u.y + al.x * v.x - al.y * v.y,
                                g.x * u.y + g.y * u.x + al.x * v.y + al.y * v.x);
  }
}

// COCG start: r~ = r / ||r|| (vector precision), d = 0, p = z = D^-1 r~; partials (r~, z), ||r~||^2
template <typename T>
__global__ void __launch_bounds__(256) k_cocg_start(const double2* __restrict__ r128, const Sys* __restrict__ sys,
                                                    typename cplx<T>::t* rin, typename cplx<T>::t* pv,
                                                    typename cplx<T>::t* d, const typename cplx<T>::t* __restrict__ dinv,
                                                    double* part, P p) {
  using V = typename cplx<T>::t;
  const int b = blockIdx.y;
  T acc[3] = {T(0), T(0), T(0)};
  if (sys[b].outer_status == SYS_RUN) {
    const long long off = (long long)b * p.ne;
    const double sc = 1.0 / sys[b].rscale;
    VEC_LOOP(p) {
      const double2 r = r128[off + e];
      const V rz = mkc<T>(r.x * sc, r.y * sc);
      const V z = dinv ? cmulv(dinv[off + e], rz) : rz;
      rin[off + e] = rz;
      pv[off + e] = z;
      d[off + e] = czero<V>();
      acc[0] += rz.x * z.x - rz.y * z.y;
      acc[1] += rz.x * z.y + rz.y * z.x;
      acc[2] += rz.x * rz.x + rz.y * rz.y;
    }
  }
  fit_block_sum<T, 3>(acc, part + PSLOT(p, b));
}

// COCG: d += alpha p, r -= alpha q; partials (r, D^-1 r), ||r||^2; the last block applies OpCocgRho
template <typename T>
__global__ void __launch_bounds__(256) k_cocg_xr(typename cplx<T>::t* d, const typename cplx<T>::t* __restrict__ pv,
                                                 typename cplx<T>::t* r, const typename cplx<T>::t* __restrict__ q,
                                                 const typename cplx<T>::t* __restrict__ dinv, Sys* sys,
                                                 double* part, unsigned* cnt, P p) {
  using V = typename cplx<T>::t;
  const int b = blockIdx.y;
  if (sys[b].inner_status != SYS_RUN) return;
  const long long off = (long long)b * p.ne;
  const T ar = (T)sys[b].alpha.x, ai = (T)sys[b].alpha.y;
  T acc[3] = {T(0), T(0), T(0)};
  VEC_LOOP(p) {
    const V pp = pv[off + e], qq = q[off + e];
    V dd = d[off + e], rr = r[off + e];
    dd.x += ar * pp.x - ai * pp.y;
    dd.y += ar * pp.y + ai * pp.x;
    rr.x -= ar * qq.x - ai * qq.y;
    rr.y -= ar * qq.y + ai * qq.x;
    d[off + e] = dd;
    r[off + e] = rr;
    const V z = dinv ? cmulv(dinv[off + e], rr) : rr;
    acc[0] += rr.x * z.x - rr.y * z.y;
    acc[1] += rr.x * z.y + rr.y * z.x;
    acc[2] += rr.x * rr.x + rr.y * rr.y;
  }
  fit_block_sum<T, 3>(acc, part + PSLOT(p, b));
  last_block_fin<3>(part, cnt, sys, p, b, OpCocgRho{});
}

// COCG: p = D^-1 r + beta p
template <typename T>
__global__ void __launch_bounds__(256) k_cocg_p(const typename cplx<T>::t* __restrict__ r, typename cplx<T>::t* pv,
                                                const typename cplx<T>::t* __restrict__ dinv, const Sys* __restrict__ sys,
                                                P p) {
  using V = typename cplx<T>::t;
  const int b = blockIdx.y;
  if (sys[b].inner_status != SYS_RUN) return;
  const long long off = (long long)b * p.ne;
  const T br = (T)sys[b].beta.x, bi = (T)sys[b].beta.y;
  VEC_LOOP(p) {
    const V rr = r[off + e], pp = pv[off + e];
    const V z = dinv ? cmulv(dinv[off + e], rr) : rr;
    V o;
    o.x = z.x + br * pp.x - bi * pp.y;
    o.y = z.y + br * pp.y + bi * pp.x;
    pv[off + e] = o;
  }
}

// COCR start: r~ = r / ||r|| (vector precision), z = D^-1 r~, p = q = d = 0; partials ||r~||^2
template <typename T>
__global__ void __launch_bounds__(256) k_cocr_start(const double2* __restrict__ r128, const Sys* __restrict__ sys,
                                                    typename cplx<T>::t* rin, typename cplx<T>::t* z,
                                                    typename cplx<T>::t* pv, typename cplx<T>::t* q,
                                                    typename cplx<T>::t* d, const typename cplx<T>::t* __restrict__ dinv,
                                                    double* part, P p) {
  using V = typename cplx<T>::t;
  const int b = blockIdx.y;
  T acc[3] = {T(0), T(0), T(0)};
  if (sys[b].outer_status == SYS_RUN) {
    const long long off = (long long)b * p.ne;
    const double sc = 1.0 / sys[b].rscale;
    VEC_LOOP(p) {
      const double2 r = r128[off + e];
      const V rz = mkc<T>(r.x * sc, r.y * sc);
      rin[off + e] = rz;
      z[off + e] = dinv ? cmulv(dinv[off + e], rz) : rz;
      pv[off + e] = czero<V>();
      q[off + e] = czero<V>();
      d[off + e] = czero<V>();
      acc[2] += rz.x * rz.x + rz.y * rz.y;
    }
  }
  fit_block_sum<T, 3>(acc, part + PSLOT(p, b));
}

// COCR: partials of (z, w) with w = A z (unconjugated)
template <typename T>
__global__ void __launch_bounds__(256) k_cocr_rho(const typename cplx<T>::t* __restrict__ z,
                                                  const typename cplx<T>::t* __restrict__ wv, const Sys* __restrict__ sys,
                                                  double* part, P p) {
  using V = typename cplx<T>::t;
  const int b = blockIdx.y;
  if (sys[b].inner_status != SYS_RUN) return;
  const long long off = (long long)b * p.ne;
  T acc[3] = {T(0), T(0), T(0)};
  VEC_LOOP(p) {
    const V a = z[off + e], c = wv[off + e];
    acc[0] += a.x * c.x - a.y * c.y;
    acc[1] += a.x * c.y + a.y * c.x;
  }
  fit_block_sum<T, 3>(acc, part + PSLOT(p, b));
}

// COCR: p = z + beta p, q = w + beta q; partials (q, D^-1 q) (unconjugated)
template <typename T>
__global__ void __launch_bounds__(256) k_cocr_pq(const typename cplx<T>::t* __restrict__ z,
                                                 const typename cplx<T>::t* __restrict__ wv, typename cplx<T>::t* pv,
                                                 typename cplx<T>::t* q, const typename cplx<T>::t* __restrict__ dinv,
                                                 const Sys* __restrict__ sys, double* part, P p) {
  using V = typename cplx<T>::t;
  const int b = blockIdx.y;
  if (sys[b].inner_status != SYS_RUN) return;
  const long long off = (long long)b * p.ne;
  const T br = (T)sys[b].beta.x, bi = (T)sys[b].beta.y;
  T acc[3] = {T(0), T(0), T(0)};
  VEC_LOOP(p) {
    const V zz = z[off + e], ww = wv[off + e];
    V pp = pv[off + e], qq = q[off + e];
    pp = V{zz.x + br * pp.x - bi * pp.y, zz.y + br * pp.y + bi * pp.x};
    qq = V{ww.x + br * qq.x - bi * qq.y, ww.y + br * qq.y + bi * qq.x};
    pv[off + e] = pp;
    q[off + e] = qq;
    const V mq = dinv ? cmulv(dinv[off + e], qq) : qq;
    acc[0] += qq.x * mq.x - qq.y * mq.y;
    acc[1] += qq.x * mq.y + qq.y * mq.x;
  }
  fit_block_sum<T, 3>(acc, part + PSLOT(p, b));
}

// COCR: d += alpha p, r -= alpha q, z = D^-1 r; partials ||r||^2
template <typename T>
__global__ void __launch_bounds__(256) k_cocr_xr(typename cplx<T>::t* d, const typename cplx<T>::t* __restrict__ pv,
                                                 typename cplx<T>::t* r, const typename cplx<T>::t* __restrict__ q,
                                                 typename cplx<T>::t* z, const typename cplx<T>::t* __restrict__ dinv,
                                                 const Sys* __restrict__ sys, double* part, P p) {
  using V = typename cplx<T>::t;
  const int b = blockIdx.y;
  if (sys[b].inner_status != SYS_RUN) return;
  const long long off = (long long)b * p.ne;
  const T ar = (T)sys[b].alpha.x, ai = (T)sys[b].alpha.y;
  T acc[3] = {T(0), T(0), T(0)};
  VEC_LOOP(p) {
    const V pp = pv[off + e], qq = q[off + e];
    V dd = d[off + e], rr = r[off + e];
    dd.x += ar * pp.x - ai * pp.y;
    dd.y += ar * pp.y + ai * pp.x;
    rr.x -= ar * qq.x - ai * qq.y;
    rr.y -= ar * qq.y + ai * qq.x;
    d[off + e] = dd;
    r[off + e] = rr;
    z[off + e] = dinv ? cmulv(dinv[off + e], rr) : rr;
    acc[2] += rr.x * rr.x + rr.y * rr.y;
  }
  fit_block_sum<T, 3>(acc, part + PSLOT(p, b));
}

// the step length of this refinement step is applied: no later step may apply it again (the loop
// keeps running while any system of the batch is active)
__global__ void k_clear_mr(Sys* sys, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) sys[b].mr = 0;
}

// ---- FGMRES(m) vector kernels ---------------------------------------------------------------
// Arnoldi step j works on the basis V[0..j] (vector i of system b at V + (i*B + b)*ne) and the
// new vector w = V[j+1].  Partial slot layout: 2*(j+1) doubles (re, im of <V_i, w>) per block.
template <typename T>
__device__ inline void warp_accum(T re, T im, double* slot_re, double* slot_im) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    *slot_re += (double)re;
    *slot_im += (double)im;
  }
}

#define FG_MAXV 65  // m + 1 <= 65

// The last block of an orthogonalisation kernel to finish (per system b; cnt counts the finished blocks
// and is reset by the last one) sums the nq per-block partials in a fixed order:
// one warp per coefficient q, its lanes taking blocks lane, lane + 32, ..., then a shuffle tree.
// Returns true in the last block (all of its threads), with hout[b][0 .. nq-1] written.
__device__ inline bool fg_last_block_fin(const double* part, int nq, double* hout, unsigned* cnt, int b, const P& p) {
  __shared__ int last;
  __threadfence();  // every thread's partials are visible before the block's arrival is counted
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&cnt[b], 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return false;
  __threadfence();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const double* pb = part + (long long)b * p.nblk * p.pstride;
  for (int q = warp; q < nq; q += nw) {
    double sum = 0.0;
    for (int k = lane; k < p.nblk; k += 32) sum += __ldcg(pb + (long long)k * p.pstride + q);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) hout[(long long)b * 2 * FG_MAXV + q] = sum;
  }
  __threadfence_block();
  __syncthreads();
  if (threadIdx.x == 0) cnt[b] = 0u;
  return true;
}

// Hessenberg column j = h + h2, h_{j+1,j} = ||w||; Givens rotations; residual estimate |g_{j+1}|
__device__ inline void fg_givens(int b, const double* __restrict__ hn2, int j, const double* __restrict__ h1,
                                 const double* __restrict__ h2, double* H, double* G, double* CS, double* SN, Sys* sys,
                                 const P& p) {
  Sys& s = sys[b];
  if (s.inner_status != SYS_RUN) return;
  const double nrm2 = hn2[(long long)b * 2 * FG_MAXV];  // ||w||^2, reduced by the last block
  const int m = p.m;
  double2* Hc = (double2*)(H + (long long)b * 2 * (m + 1) * m) + (long long)j * (m + 1);  // column j
  double2* g = (double2*)(G + (long long)b * 2 * (m + 1));
  double2* cs = (double2*)(CS + (long long)b * 2 * m);
  double2* sn = (double2*)(SN + (long long)b * 2 * m);
  const double2* a1 = (const double2*)(h1 + (long long)b * 2 * FG_MAXV);
  const double2* a2 = (const double2*)(h2 + (long long)b * 2 * FG_MAXV);
  for (int i = 0; i <= j; ++i) Hc[i] = cadd(a1[i], a2[i]);
  const double hn = sqrt(nrm2);
  Hc[j + 1] = make_double2(hn, 0.0);
  if (!isfinite(hn) || !cfinite(Hc[j])) { s.inner_status = SYS_NAN; return; }
  for (int i = 0; i < j; ++i) {
    double2 hi = Hc[i], hi1 = Hc[i + 1];
    Hc[i] = cadd(cmul(cconj(cs[i]), hi), cmul(cconj(sn[i]), hi1));
    Hc[i + 1] = csub(cmul(cs[i], hi1), cmul(sn[i], hi));
  }
  double2 a = Hc[j], c = Hc[j + 1];
  double den = sqrt(cabs2(a) + cabs2(c));
  if (den > 0.0) {
    cs[j] = make_double2(a.x / den, a.y / den);
    sn[j] = make_double2(c.x / den, c.y / den);
  } else {
    cs[j] = make_double2(1.0, 0.0);
    sn[j] = make_double2(0.0, 0.0);
  }
  Hc[j] = make_double2(den, 0.0);
  Hc[j + 1] = make_double2(0.0, 0.0);
  double2 gj = g[j];
  g[j + 1] = make_double2(-(sn[j].x * gj.x - sn[j].y * gj.y), -(sn[j].x * gj.y + sn[j].y * gj.x));
  g[j] = cmul(cconj(cs[j]), gj);
  s.jlast = j + 1;
  s.inner_it += 1;
  s.inv_hn = hn > 0.0 ? 1.0 / hn : 0.0;
  double res2 = cabs2(g[j + 1]);
  s.rin2 = res2;
  if (res2 <= s.inner_tol2) s.inner_status = SYS_CONV;
  else if (hn == 0.0 || den == 0.0) s.inner_status = SYS_CONV;  // exact invariant subspace
  else if (j + 1 >= m || s.inner_it >= s.max_inner) s.inner_status = SYS_MAXIT;
}

// Arnoldi coefficient vectors of the orthogonalisation passes and the Hessenberg workspace, for the
// last block's reduction and Givens step
struct FgOut {
  double *h1, *h2, *hn2, *H, *G, *CS, *SN;
  unsigned* cnt;
};

// The three CGS2 passes.  They work on chunks of CH elements (one per thread, CH = 256 for complex64
// and 128 for complex128) and keep only a few values per thread in registers:
//   k_fg_dots:         h_i = <V_i, w>                   (2(j+1) partials per block)
//   k_fg_update_dots:  w -= sum_i h_i V_i, then h2_i = <V_i, w>
//   k_fg_update_norm:  w -= sum_i h2_i V_i, then ||w||^2 (partial slot 0)
// The dots are a tall-skinny product: the chunk of w sits in shared memory and each warp streams
// whole basis vectors (i = warp, warp + nwarps, ...) over it, summing in the vector precision within
// the chunk and in FP64 across chunks, in a fixed order.  k_fg_update_dots keeps the chunk of every
// V_i it reads for the update in shared memory, so V is read from HBM once for both halves.
template <typename T>
struct FgChunk {
  static constexpr int CH = sizeof(T) == 4 ? 256 : 128;
};

template <typename T>
__device__ inline void fg_chunk_dots(const typename cplx<T>::t* vchunk, long long vstride, bool vglobal,
                                     const typename cplx<T>::t* ws, int nv, int nvalid, double* acc) {
  constexpr int CH = FgChunk<T>::CH;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = CH / 32;
  for (int i = warp; i < nv; i += nw) {
    const auto* vi = vchunk + (vglobal ? (long long)i * vstride : (long long)i * CH);
    T sr = T(0), si = T(0);
#pragma unroll
    for (int q0 = 0; q0 < CH; q0 += 32) {
      const int q = q0 + lane;
      if (q < nvalid) {
        const auto a = vi[q], b = ws[q];
        sr += a.x * b.x + a.y * b.y;
        si += a.x * b.y - a.y * b.x;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane == 0) {
      acc[2 * i] += (double)sr;
      acc[2 * i + 1] += (double)si;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_fg_dots(const typename cplx<T>::t* __restrict__ Vb, int j,
                                                 const Sys* __restrict__ sys, double* part, FgOut fo, P p) {
  using V = typename cplx<T>::t;
  constexpr int CH = FgChunk<T>::CH;
  const int b = blockIdx.y;
  if (sys[b].inner_status != SYS_RUN) return;
  __shared__ V ws[CH];
  __shared__ double acc[2 * FG_MAXV];
  const int nv = j + 1, tid = threadIdx.x;
  const long long vs = (long long)p.B * p.ne, off = (long long)b * p.ne;
  const V* w = Vb + (long long)(j + 1) * vs + off;
  for (int q = tid; q < 2 * nv; q += CH) acc[q] = 0.0;
  for (long long c0 = (long long)blockIdx.x * CH; c0 < p.ne; c0 += (long long)gridDim.x * CH) {
    const int nvalid = (int)min((long long)CH, p.ne - c0);
    __syncthreads();  // the previous chunk's dots are done with ws
    ws[tid] = tid < nvalid ? w[c0 + tid] : czero<V>();
    __syncthreads();
    fg_chunk_dots<T>(Vb + off + c0, vs, true, ws, nv, nvalid, acc);
  }
  __syncthreads();
  double* out = part + PSLOT(p, b);
  for (int q = tid; q < 2 * nv; q += CH) out[q] = acc[q];
  fg_last_block_fin(part, 2 * nv, fo.h1, fo.cnt, b, p);
}

template <typename T>
__global__ void __launch_bounds__(256) k_fg_update_dots(const typename cplx<T>::t* __restrict__ Vb, int j,
                                                        const double* __restrict__ hcoef,
                                                        const Sys* __restrict__ sys, double* part, FgOut fo, P p) {
  using V = typename cplx<T>::t;
  constexpr int CH = FgChunk<T>::CH;
  const int b = blockIdx.y;
  if (sys[b].inner_status != SYS_RUN) return;
  extern __shared__ __align__(16) unsigned char fg_smem[];
  V* vsm = (V*)fg_smem;                 // [nv][CH]
  const int nv = j + 1, tid = threadIdx.x;
  V* ws = vsm + (long long)nv * CH;     // [CH]
  double* acc = (double*)(ws + CH);     // [2 nv]
  T* hs = (T*)(acc + 2 * nv);           // [2 nv]
  const long long vs = (long long)p.B * p.ne, off = (long long)b * p.ne;
  V* w = (V*)(Vb + (long long)(j + 1) * vs + off);
  const double* hc = hcoef + (long long)b * 2 * FG_MAXV;
  for (int q = tid; q < 2 * nv; q += CH) {
    acc[q] = 0.0;
    hs[q] = (T)hc[q];
  }
  for (long long c0 = (long long)blockIdx.x * CH; c0 < p.ne; c0 += (long long)gridDim.x * CH) {
    const int nvalid = (int)min((long long)CH, p.ne - c0);
    const bool valid = tid < nvalid;
    __syncthreads();  // hs is set; the previous chunk's dots are done with vsm and ws
    V wv = valid ? w[c0 + tid] : czero<V>();
    const V* vcol = Vb + off + c0 + tid;
#pragma unroll 8
    for (int i = 0; i < nv; ++i) {
      const V a = valid ? vcol[(long long)i * vs] : czero<V>();
      vsm[i * CH + tid] = a;
      const T hr = hs[2 * i], hi = hs[2 * i + 1];
      wv.x -= hr * a.x - hi * a.y;
      wv.y -= hr * a.y + hi * a.x;
    }
    if (valid) w[c0 + tid] = wv;
    ws[tid] = wv;
    __syncthreads();
    fg_chunk_dots<T>(vsm, 0, false, ws, nv, nvalid, acc);
  }
  __syncthreads();
  double* out = part + PSLOT(p, b);
  for (int q = tid; q < 2 * nv; q += CH) out[q] = acc[q];
  fg_last_block_fin(part, 2 * nv, fo.h2, fo.cnt, b, p);
}

template <typename T>
__global__ void __launch_bounds__(256) k_fg_update_norm(const typename cplx<T>::t* __restrict__ Vb, int j,
                                                        const double* __restrict__ hcoef,
                                                        Sys* sys, double* part, FgOut fo, P p) {
  using V = typename cplx<T>::t;
  constexpr int CH = FgChunk<T>::CH;
  const int b = blockIdx.y;
  if (sys[b].inner_status != SYS_RUN) return;
  __shared__ T hs[2 * FG_MAXV];
  const int nv = j + 1, tid = threadIdx.x;
  const long long vs = (long long)p.B * p.ne, off = (long long)b * p.ne;
  V* w = (V*)(Vb + (long long)(j + 1) * vs + off);
  const double* hc = hcoef + (long long)b * 2 * FG_MAXV;
  for (int q = tid; q < 2 * nv; q += CH) hs[q] = (T)hc[q];
  __syncthreads();
  T nrm[1] = {T(0)};
  for (long long e = (long long)blockIdx.x * CH + tid; e < p.ne; e += (long long)gridDim.x * CH) {
    V wv = w[e];
    const V* vcol = Vb + off + e;
#pragma unroll 8
    for (int i = 0; i < nv; ++i) {
      const V a = vcol[(long long)i * vs];
      const T hr = hs[2 * i], hi = hs[2 * i + 1];
      wv.x -= hr * a.x - hi * a.y;
      wv.y -= hr * a.y + hi * a.x;
    }
    w[e] = wv;
    nrm[0] += wv.x * wv.x + wv.y * wv.y;
  }
  fit_block_sum<T, 1>(nrm, part + PSLOT(p, b));
  // the last block reduces ||w||^2 and takes the Givens step of this system
  if (fg_last_block_fin(part, 1, fo.hn2, fo.cnt, b, p) && threadIdx.x == 0) {
    __threadfence_block();
    fg_givens(b, fo.hn2, j, fo.h1, fo.h2, fo.H, fo.G, fo.CS, fo.SN, sys, p);
  }
}


// ---- the three CGS2 passes with bulk copies -----------------------------------------------------
// The same passes and per-block partial layout as k_fg_dots / k_fg_update_dots / k_fg_update_norm, but
// the block's chunk of every basis vector and of w arrives in shared memory by a bulk copy engine
// transfer (cp.async.bulk, one 2 KB copy per vector and chunk), S chunks in flight, completed on one
// mbarrier per stage.  The copy engine keeps the loads streaming while the threads update w and take
// the dot products from shared memory, so V is read from HBM once per pass at close to copy speed.
// Dot products: warp q of NW owns the basis vectors i = q, q + NW, ...; each lane accumulates its share over
// all of the block's chunks in the vector precision, and the warp's shuffle sum goes to the block's
// partial slot in FP64.  Needs 16-byte aligned chunks: complex128, or complex64 with an even n_e.
// Every wait on a stage is bounded (2^22 polls, the grid's abort word read every 4096): on a timeout the
// block records it in the grid's error word, lets its own copies land and leaves.
__device__ inline uint32_t kr_smem(const void* q) { return (uint32_t)__cvta_generic_to_shared(q); }
__device__ inline bool kr_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(kr_smem(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ inline bool kr_wait(uint64_t* bar, uint32_t parity, const volatile int* abort) {
  for (int it = 0; it < (1 << 22); ++it) {
    if (kr_try_wait(bar, parity)) return true;
    if (it > 32) __nanosleep(32);
    if ((it & 4095) == 4095 && abort && *abort) return false;
  }
  return false;
}

template <typename T, int MODE, int S>
__global__ void __launch_bounds__(256) k_fg_cgs_bulk(const typename cplx<T>::t* __restrict__ Vb, int j,
                                                     const double* __restrict__ hcoef, Sys* sys, double* part,
                                                     FgOut fo, P p) {
  using V = typename cplx<T>::t;
  constexpr int CH = FgChunk<T>::CH;
  constexpr int NW = CH / 32;       // warps per block (one thread per chunk element)
  constexpr int SLOTS = 64 / NW;    // basis vectors per warp: nv <= 64
  const int b = blockIdx.y;
  if (sys[b].inner_status != SYS_RUN) return;
  extern __shared__ __align__(128) unsigned char fg_bulk_smem[];
  const int nv = j + 1, nrow = nv + 1, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const size_t stage_vals = (size_t)nrow * CH;
  V* stg = (V*)fg_bulk_smem;
  uint64_t* bar = (uint64_t*)(stg + S * stage_vals);
  T* hs = (T*)(bar + S);                 // [2 nv]
  double* red = (double*)(hs + 2 * FG_MAXV);  // [2 nv] per-vector block sums
  __shared__ int bad;
  const long long vs = (long long)p.B * p.ne, off = (long long)b * p.ne;
  V* w = (V*)(Vb + (long long)(j + 1) * vs + off);
  const long long first = (long long)blockIdx.x * CH, step = (long long)gridDim.x * CH;
  const int nch = first < p.ne ? (int)((p.ne - first + step - 1) / step) : 0;
  if (tid == 0) {
    for (int q = 0; q < S; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(kr_smem(&bar[q])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    bad = 0;
  }
  if (MODE >= 1) {
    const double* hc = hcoef + (long long)b * 2 * FG_MAXV;
    for (int q = tid; q < 2 * nv; q += blockDim.x) hs[q] = (T)hc[q];
  }
  __syncthreads();
  auto issue = [&](int n) {  // thread 0: every row of chunk n into stage n % S
    const long long c0 = first + (long long)n * step;
    const uint32_t bytes = (uint32_t)(min((long long)CH, p.ne - c0) * (long long)sizeof(V));
    V* dst = stg + (size_t)(n % S) * stage_vals;
    uint64_t* br = &bar[n % S];
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(kr_smem(br)), "r"(bytes * nrow)
                 : "memory");
    for (int r = 0; r < nrow; ++r) {
      const V* src = (r < nv ? Vb + (long long)r * vs + off : w) + c0;
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       kr_smem(dst + (size_t)r * CH)),
                   "l"(src), "r"(bytes), "r"(kr_smem(br))
                   : "memory");
    }
  };
  int issued = 0;
  if (tid == 0)
    for (; issued < min(S, nch); ++issued) issue(issued);
  T ar[SLOTS], ai[SLOTS], nrm = T(0);
#pragma unroll
  for (int q = 0; q < SLOTS; ++q) ar[q] = ai[q] = T(0);
  int n = 0;
  for (; n < nch; ++n) {
    const bool ok = kr_wait(&bar[n % S], (uint32_t)((n / S) & 1), p.abort);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        bad = 1;
        atomicMax(p.err, (p.abort && *p.abort) ? 2 : 1);
      }
      break;
    }
    V* sv = stg + (size_t)(n % S) * stage_vals;
    const long long c0 = first + (long long)n * step;
    const int nvalid = (int)min((long long)CH, p.ne - c0);
    if (MODE >= 1 && tid < nvalid) {  // w -= sum_i h_i V_i for this thread's element
      V wv = sv[(size_t)nv * CH + tid];
      for (int i = 0; i < nv; ++i) {
        const V a = sv[(size_t)i * CH + tid];
        const T hr = hs[2 * i], hi = hs[2 * i + 1];
        wv.x -= hr * a.x - hi * a.y;
        wv.y -= hr * a.y + hi * a.x;
      }
      w[c0 + tid] = wv;
      if (MODE == 1) sv[(size_t)nv * CH + tid] = wv;
      else nrm += wv.x * wv.x + wv.y * wv.y;
    }
    if (MODE <= 1) {
      if (MODE == 1) __syncthreads();  // the updated w of the chunk is in shared memory
      const V* wsm = sv + (size_t)nv * CH;
#pragma unroll
      for (int q = 0; q < SLOTS; ++q) {
        const int i = warp + NW * q;
        if (i < nv) {
          const V* vi = sv + (size_t)i * CH;
          for (int e = lane; e < nvalid; e += 32) {
            const V a = vi[e], c = wsm[e];
            ar[q] += a.x * c.x + a.y * c.y;  // conj(V_i) w
            ai[q] += a.x * c.y - a.y * c.x;
          }
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes before the stage's refill
    __syncthreads();  // the stage is consumed
    if (tid == 0 && issued < nch) issue(issued++);
  }
  if (bad) {  // let this block's copies land before it leaves (bounded; no early exit on abort)
    if (tid == 0)
      for (int q = n; q < issued; ++q) (void)kr_wait(&bar[q % S], (uint32_t)((q / S) & 1), nullptr);
    __syncthreads();
    return;
  }
  double* out = part + PSLOT(p, b);
  if (MODE == 2) {
    T v1[1] = {nrm};
    fit_block_sum<T, 1>(v1, out);
    if (fg_last_block_fin(part, 1, fo.hn2, fo.cnt, b, p) && tid == 0) {
      __threadfence_block();
      fg_givens(b, fo.hn2, j, fo.h1, fo.h2, fo.H, fo.G, fo.CS, fo.SN, sys, p);
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < SLOTS; ++q) {
    const int i = warp + NW * q;
    T r = ar[q], m = ai[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      r += __shfl_xor_sync(0xffffffffu, r, o);
      m += __shfl_xor_sync(0xffffffffu, m, o);
    }
    if (lane == 0 && i < nv) {
      red[2 * i] = (double)r;
      red[2 * i + 1] = (double)m;
    }
  }
  __syncthreads();
  for (int q = tid; q < 2 * nv; q += blockDim.x) out[q] = red[q];
  fg_last_block_fin(part, 2 * nv, MODE == 0 ? fo.h1 : fo.h2, fo.cnt, b, p);
}

// v_{j+1} = w / h_{j+1,j}
template <typename T>
__global__ void __launch_bounds__(256) k_fg_scale(typename cplx<T>::t* Vb, int j, const Sys* __restrict__ sys, P p) {
  const int b = blockIdx.y;
  if (sys[b].inner_status != SYS_RUN) return;
  const long long vs = (long long)p.B * p.ne;
  auto* w = Vb + (long long)(j + 1) * vs + (long long)b * p.ne;
  const T sc = (T)sys[b].inv_hn;
  VEC_LOOP(p) {
    auto v = w[e];
    v.x *= sc;
    v.y *= sc;
    w[e] = v;
  }
}

// back substitution H y = g on the rotated (upper triangular) Hessenberg, then d = sum y_i Z_i
__global__ void k_fg_solve(const double* __restrict__ H, const double* __restrict__ G, double* Y, const Sys* sys, P p) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= p.B) return;
  const Sys& s = sys[b];
  if (s.outer_status != SYS_RUN) return;
  const int m = p.m, n = s.jlast;
  const double2* Hb = (const double2*)(H + (long long)b * 2 * (m + 1) * m);
  const double2* g = (const double2*)(G + (long long)b * 2 * (m + 1));
  double2* y = (double2*)(Y + (long long)b * 2 * FG_MAXV);
  for (int i = n - 1; i >= 0; --i) {
    double2 acc = g[i];
    for (int k = i + 1; k < n; ++k) acc = csub(acc, cmul(Hb[(long long)k * (m + 1) + i], y[k]));
    double2 hii = Hb[(long long)i * (m + 1) + i];
    y[i] = cabs2(hii) > 0.0 ? cdiv(acc, hii) : make_double2(0.0, 0.0);
  }
  for (int i = n; i < m; ++i) y[i] = make_double2(0.0, 0.0);
}

template <typename T, int MAXV>
__global__ void __launch_bounds__(256) k_fg_combine(const typename cplx<T>::t* __restrict__ Zb, typename cplx<T>::t* d,
                                                    const double* __restrict__ Y, const Sys* __restrict__ sys, P p) {
  using V = typename cplx<T>::t;
  const int b = blockIdx.y;
  if (sys[b].outer_status != SYS_RUN) return;
  const int n = sys[b].jlast;
  const long long vs = (long long)p.B * p.ne;
  const long long off = (long long)b * p.ne;
  const double* y = Y + (long long)b * 2 * FG_MAXV;
  T yr[MAXV], yi[MAXV];
#pragma unroll
  for (int i = 0; i < MAXV; ++i) {
    yr[i] = i < n ? (T)y[2 * i] : T(0);
    yi[i] = i < n ? (T)y[2 * i + 1] : T(0);
  }
  VEC_LOOP(p) {
    V acc = czero<V>();
#pragma unroll
    for (int i = 0; i < MAXV; ++i) {
      if (i < n) {
        V zi = Zb[(long long)i * vs + off + e];
        acc.x += yr[i] * zi.x - yi[i] * zi.y;
        acc.y += yr[i] * zi.y + yi[i] * zi.x;
      }
    }
    d[off + e] = acc;
  }
}

// FGMRES inner start: g = (1, 0, ...), rotations cleared
__global__ void k_fg_reset(double* G, const Sys* sys, P p) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= p.B) return;
  double2* g = (double2*)(G + (long long)b * 2 * (p.m + 1));
  g[0] = make_double2(sqrt(sys[b].rin2), 0.0);
  for (int i = 1; i <= p.m; ++i) g[i] = make_double2(0.0, 0.0);
}

// sum over facets containing each edge of M_nu (the C^T M_nu C diagonal; Eq. Precond construction)
template <typename T>
__global__ void k_nusum(const T* __restrict__ nu, int nx, int ny, int nz, int nxp, T* out) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= (long long)nx * ny * nz) return;
  int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
  auto NU = [&](int a, int bb, int cc, int w) -> T {
    if (a < 0 || bb < 0 || cc < 0) return T(0);
    return nu[3 * (a + (long long)nxp * (bb + (long long)ny * cc)) + w];
  };
  out[3 * c + 0] = NU(i, j, k, 1) + NU(i, j, k - 1, 1) + NU(i, j, k, 2) + NU(i, j - 1, k, 2);
  out[3 * c + 1] = NU(i, j, k, 0) + NU(i, j, k - 1, 0) + NU(i, j, k, 2) + NU(i - 1, j, k, 2);
  out[3 * c + 2] = NU(i, j, k, 0) + NU(i, j - 1, k, 0) + NU(i, j, k, 1) + NU(i - 1, j, k, 1);
}

// ---- loop conditions -------------------------------------------------------------------------
// (it also refreshes the mirrored per-system status words the apply's predicate reads)
__global__ void k_cond(const Sys* __restrict__ sys, Ctl* ctl, P p, int which, int guard_max,
                       cudaGraphConditionalHandle h, int use_handle, int* mirror_inner, int* mirror_outer) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < p.B; b += blockDim.x) {
    const int si = sys[b].inner_status, so = sys[b].outer_status;
    mirror_inner[b] = si;
    mirror_outer[b] = so;
    if ((which == 0 ? si : so) == SYS_RUN) any = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int* guard = which == 0 ? &ctl->inner_guard : &ctl->outer_guard;
    *guard += 1;
    // the host's abort word ends both loops: read at every outer step and every 64th inner step (a
    // read of pinned host memory costs about a microsecond)
    bool stop = false;
    if (p.abort && (which == 1 || (*guard & 63) == 1) && *p.abort) {
      stop = true;
      atomicMax(p.err, 2);
    }
    int v = (!stop && any && *guard < guard_max) ? 1 : 0;
    ctl->cond = v;
    if (use_handle) cudaGraphSetConditional(h, v);
  }
}

// Resets a loop guard and, inside a graph, re-arms the loop's WHILE handle: the default value of a
// handle is applied once per graph launch, so a nested loop that is entered again (the inner loop
// of every refinement step) must be set to 1 explicitly before its node is reached.
__global__ void k_reset_guard(Ctl* ctl, int which, cudaGraphConditionalHandle h, int use_handle) {
  if (which == 0) ctl->inner_guard = 0;
  else ctl->outer_guard = 0;
  if (use_handle) cudaGraphSetConditional(h, 1);
}

}  // namespace

// ================================================================================================
// Host side: workspace, launch sequence, graph capture and the solve loop
// ================================================================================================
namespace {

struct Work {
  fit_grid* g = nullptr;
  int B = 0, m = 30, method = FIT_BICGSTAB, mixed = 1, pc = FIT_PC_NONE;
  fit_prec inner = FIT_C64;
  size_t esz = 8;         // bytes per complex inner element
  P p{};
  // device buffers
  double2* r128 = nullptr;
  double2* rprev = nullptr;  // r before the current correction (true-residual acceptance test)
  double* omega = nullptr;
  void *rin = nullptr, *rhat = nullptr, *pv = nullptr, *v = nullptr, *t = nullptr, *d = nullptr;
  void* Vb = nullptr;     // FGMRES basis (m+1 vectors)
  void* Zb = nullptr;     // FGMRES preconditioned vectors (m), or aliases Vb
  void* nusum = nullptr;
  void* dinv = nullptr;   // Jacobi D^-1 per system (inner precision)
  void *phat = nullptr, *shat = nullptr;  // BiCGStab: preconditioned p and s
  void* x16 = nullptr;   // U-Net input scratch ([ncell][16] bf16)
  double *part_apply = nullptr, *part_vec = nullptr;
  long long napply = 0;
  double *h1 = nullptr, *h2 = nullptr, *hn2 = nullptr, *H = nullptr, *G = nullptr, *CS = nullptr, *SN = nullptr, *Y = nullptr;
  Sys* sys = nullptr;
  Ctl* ctl = nullptr;
  unsigned* cnt = nullptr;  // per system: blocks of a vector kernel finished (last-block reductions)
  std::vector<std::pair<void*, size_t>> allocs;
  ~Work() {
    for (auto& a : allocs) fit_dev_free(g, a.first, a.second);
  }
  fit_status alloc(void** ptr, size_t bytes) {
    fit_status st = fit_dev_alloc(g, ptr, bytes);
    if (st == FIT_OK && *ptr) allocs.push_back({*ptr, bytes});
    return st;
  }
};

size_t workspace_bytes(const fit_grid* g, int B, int method, int m, int mixed, int pc) {
  size_t ne = (size_t)g->ne;
  size_t esz = mixed ? 8 : 16;
  size_t vec = ne * B * esz;
  size_t bytes = ne * B * 32;  // r128 and r_prev
  if (method == FIT_BICGSTAB) bytes += 6 * vec + (pc != FIT_PC_NONE ? 2 * vec : 0);
  else if (method == FIT_COCG) bytes += 4 * vec;
  else if (method == FIT_COCR) bytes += 6 * vec;
  else bytes += (size_t)(m + 1) * vec + (pc != FIT_PC_NONE ? (size_t)m * vec : 0) + 2 * vec;
  if (pc == FIT_PC_JACOBI || pc == FIT_PC_UNET) bytes += ne * esz / 2 + vec;
  else if (pc == FIT_PC_EPS) bytes += vec;
  size_t napply = (size_t)std::max(fit_apply_partials(g, FIT_C64), fit_apply_partials(g, FIT_C128));
  bytes += (size_t)B * napply * 4 * 8;
  bytes += (size_t)B * 1216 * 2 * FG_MAXV * 8;
  bytes += (size_t)B * (3 * 2 * FG_MAXV + 2 * (m + 1) * m * 2 + 2 * (m + 1) * 2 + 2 * 2 * m + 2 * FG_MAXV) * 8;
  return bytes + (size_t)B * (sizeof(Sys) + sizeof(unsigned)) + 4096;
}

fit_status setup(Work& w, int B) {
  fit_grid* g = w.g;
  w.B = B;
  w.esz = w.mixed ? sizeof(float2) : sizeof(double2);
  w.inner = w.mixed ? FIT_C64 : FIT_C128;
  size_t ne = (size_t)g->ne;
  size_t vec = ne * B * w.esz;
  fit_status st;
#define ALLOC(ptr, bytes) \
  if ((st = w.alloc((void**)&(ptr), (bytes))) != FIT_OK) return st
  ALLOC(w.r128, ne * B * sizeof(double2));
  ALLOC(w.rprev, ne * B * sizeof(double2));
  ALLOC(w.omega, B * sizeof(double));
  if (w.method == FIT_BICGSTAB) {
    ALLOC(w.rin, vec);
    ALLOC(w.rhat, vec);
    ALLOC(w.pv, vec);
    ALLOC(w.v, vec);
    ALLOC(w.t, vec);
    ALLOC(w.d, vec);
    if (w.pc != FIT_PC_NONE) {
      ALLOC(w.phat, vec);
      ALLOC(w.shat, vec);
    }
  } else if (w.method == FIT_COCG) {
    ALLOC(w.rin, vec);
    ALLOC(w.pv, vec);
    ALLOC(w.v, vec);
    ALLOC(w.d, vec);
  } else if (w.method == FIT_COCR) {  // r, z (in t), p, q (in rhat), w = A z (in v), the correction d
    ALLOC(w.rin, vec);
    ALLOC(w.t, vec);
    ALLOC(w.pv, vec);
    ALLOC(w.rhat, vec);
    ALLOC(w.v, vec);
    ALLOC(w.d, vec);
  } else {
    ALLOC(w.Vb, (size_t)(w.m + 1) * vec);
    if (w.pc != FIT_PC_NONE) {
      ALLOC(w.Zb, (size_t)w.m * vec);
    } else {
      w.Zb = w.Vb;
    }
    ALLOC(w.d, vec);
    w.rin = w.Vb;  // V0 holds r~
  }
  if (w.pc == FIT_PC_JACOBI || w.pc == FIT_PC_UNET) {  // the learned preconditioner adds to Jacobi
    ALLOC(w.nusum, ne * w.esz / 2);
    ALLOC(w.dinv, vec);
  } else if (w.pc == FIT_PC_EPS) {
    ALLOC(w.dinv, vec);
  }
  if (w.pc == FIT_PC_UNET) {
    ALLOC(w.x16, (size_t)g->ncell * 16 * 2);
    if ((st = fit_unet_prepare(g->unet, g, 0)) != FIT_OK) return st;
  }
  w.napply = std::max(fit_apply_partials(g, FIT_C64), fit_apply_partials(g, FIT_C128));
  ALLOC(w.part_apply, (size_t)B * w.napply * 4 * sizeof(double));
  int nblk = std::max(8, std::min(1216, (int)((ne + 255) / 256)));
  nblk = std::max(1, std::min(nblk, 1216 / std::max(1, std::min(B, 8)) * 1));
  int pstride = w.method == FIT_FGMRES ? 2 * (w.m + 1) : 4;
  if (pstride < 4) pstride = 4;
  ALLOC(w.part_vec, (size_t)B * nblk * pstride * sizeof(double));
  if (w.method == FIT_FGMRES) {
    ALLOC(w.h1, (size_t)B * 2 * FG_MAXV * sizeof(double));
    ALLOC(w.h2, (size_t)B * 2 * FG_MAXV * sizeof(double));
    ALLOC(w.hn2, (size_t)B * 2 * FG_MAXV * sizeof(double));
    ALLOC(w.H, (size_t)B * 2 * (w.m + 1) * w.m * sizeof(double));
    ALLOC(w.G, (size_t)B * 2 * (w.m + 1) * sizeof(double));
    ALLOC(w.CS, (size_t)B * 2 * w.m * sizeof(double));
    ALLOC(w.SN, (size_t)B * 2 * w.m * sizeof(double));
    ALLOC(w.Y, (size_t)B * 2 * FG_MAXV * sizeof(double));
  }
  ALLOC(w.sys, (size_t)B * sizeof(Sys));
  ALLOC(w.ctl, sizeof(Ctl));
  ALLOC(w.cnt, (size_t)B * sizeof(unsigned));
#undef ALLOC
  FIT_CHECK_CUDA(cudaMemset(w.sys, 0, (size_t)B * sizeof(Sys)));
  FIT_CHECK_CUDA(cudaMemset(w.ctl, 0, sizeof(Ctl)));
  FIT_CHECK_CUDA(cudaMemset(w.cnt, 0, (size_t)B * sizeof(unsigned)));
  w.p.B = B;
  w.p.ne = g->ne;
  w.p.nblk = nblk;
  w.p.pstride = pstride;
  w.p.m = w.m;
  w.p.mixed = w.mixed;
  w.p.s_in = w.mixed ? g->coef_scale : 1.0;
  w.p.tiny = w.mixed ? 1e-30 : 1e-300;
  // iterations without a new smallest inner residual before the inner solve hands back: COCG's
  // residual norm is not monotone (A is complex symmetric, not Hermitian) and can wander above its
  // minimum for thousands of iterations before it falls again, so it gets a far longer window
  w.p.stall = (w.method == FIT_COCG || w.method == FIT_COCR) ? 20000 : 1000;
  w.p.precond = w.pc;
  w.p.abort = g->abort_dev;
  w.p.err = g->err_dev;
  if (w.pc == FIT_PC_JACOBI || w.pc == FIT_PC_UNET) {
    long long nc = g->ncell;
    if (w.mixed)
      k_nusum<float><<<(unsigned)((nc + 255) / 256), 256>>>(g->nu32, g->nx, g->ny, g->nz, g->nxp, (float*)w.nusum);
    else
      k_nusum<double><<<(unsigned)((nc + 255) / 256), 256>>>(g->nu64, g->nx, g->ny, g->nz, g->nxp, (double*)w.nusum);
    FIT_CHECK_CUDA(cudaGetLastError());
  }
  return FIT_OK;
}

// ---- the launch sequence (used directly, or captured into a graph) ------------------------------
struct Seq {
  Work& w;
  const double2* rhs;
  double2* x;
  cudaStream_t s;
  fit_status st = FIT_OK;

  dim3 vgrid() const { return dim3(w.p.nblk, w.p.B); }
  void check() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess && st == FIT_OK) {
      fit_set_error(std::string("fit_solve kernel launch: ") + cudaGetErrorString(e));
      st = FIT_ECUDA;
    }
  }
  template <int NQ, class Op>
  void fin(const double* part, long long nslots, int stride, Op op) {
    fin_kernel<NQ, Op><<<w.p.B, 256, 0, s>>>(part, nslots, stride, w.sys, w.p, op);
    check();
  }
  // launches the apply and returns the number of partial slots per system it writes
  long long apply(const void* xin, void* yout, int mode, const void* u, fit_prec prec, const int* status_field) {
    fit_epi e;
    e.mode = mode;
    e.u = u;
    e.part = w.part_apply;
    e.status = status_field;
    fit_status r = fit_launch_apply(w.g, w.p.B, w.omega, xin, yout, prec, 1.0, s, &e);
    if (r != FIT_OK && st == FIT_OK) st = r;
    if (e.nslots > w.napply && st == FIT_OK) {
      fit_set_error("fit_solve: apply wrote more partial slots than were allocated");
      st = FIT_ECUDA;
    }
    return e.nslots;
  }
  cudaGraphConditionalHandle h_inner = 0;  // set when the inner loop is a graph WHILE node
  int use_h_inner = 0;

  void outer_init() {
    k_reset_guard<<<1, 1, 0, s>>>(w.ctl, 1, 0, 0);
    k_outer_init<<<vgrid(), 256, 0, s>>>(rhs, x, w.r128, w.part_vec, w.p);
    check();
    fin<3>(w.part_vec, w.p.nblk, w.p.pstride, OpOuterInit{});
  }

  template <typename T>
  void inner_start() {
    using V = typename cplx<T>::t;
    k_reset_guard<<<1, 1, 0, s>>>(w.ctl, 0, h_inner, use_h_inner);
    if (w.method == FIT_COCG) {
      k_cocg_start<T><<<vgrid(), 256, 0, s>>>(w.r128, w.sys, (V*)w.rin, (V*)w.pv, (V*)w.d, (const V*)w.dinv,
                                              w.part_vec, w.p);
      check();
      fin<3>(w.part_vec, w.p.nblk, w.p.pstride, OpCocgStart{});
      return;
    }
    if (w.method == FIT_COCR) {
      k_cocr_start<T><<<vgrid(), 256, 0, s>>>(w.r128, w.sys, (V*)w.rin, (V*)w.t, (V*)w.pv, (V*)w.rhat, (V*)w.d,
                                              (const V*)w.dinv, w.part_vec, w.p);
      check();
      fin<3>(w.part_vec, w.p.nblk, w.p.pstride, OpCocrStart{});
      return;
    }
    bool bicg = w.method == FIT_BICGSTAB;
    if (bicg)
      k_inner_start<T, true><<<vgrid(), 256, 0, s>>>(w.r128, w.sys, (V*)w.rin, (V*)w.rhat, (V*)w.pv, (V*)w.v,
                                                      (V*)w.d, w.part_vec, w.p);
    else
      k_inner_start<T, false><<<vgrid(), 256, 0, s>>>(w.r128, w.sys, (V*)w.rin, nullptr, nullptr, nullptr, (V*)w.d,
                                                       w.part_vec, w.p);
    check();
    fin<3>(w.part_vec, w.p.nblk, w.p.pstride, OpInnerStart{});
    if (!bicg) {
      k_fg_reset<<<(w.p.B + 127) / 128, 128, 0, s>>>(w.G, w.sys, w.p);
      check();
    }
  }

  // one COCG iteration (predicated on inner status): q = A p with (p, q) from the apply's epilogue,
  // alpha, the x/r update (its last block computes rho and beta), then p
  template <typename T>
  void cocg_iter(const int* st_inner) {
    using V = typename cplx<T>::t;
    long long n1 = apply(w.pv, w.v, FIT_EPI_DOT_XY, nullptr, w.inner, st_inner);
    fin<3>(w.part_apply, n1, 4, OpCocgAlpha{});
    k_cocg_xr<T><<<vgrid(), 256, 0, s>>>((V*)w.d, (const V*)w.pv, (V*)w.rin, (const V*)w.v, (const V*)w.dinv, w.sys,
                                         w.part_vec, w.cnt, w.p);
    check();
    k_cocg_p<T><<<vgrid(), 256, 0, s>>>((const V*)w.rin, (V*)w.pv, (const V*)w.dinv, w.sys, w.p);
    check();
  }

  // one COCR iteration (predicated on inner status): w = A z, beta, p and q, alpha, the x/r/z update
  template <typename T>
  void cocr_iter(const int* st_inner) {
    using V = typename cplx<T>::t;
    apply(w.t, w.v, FIT_EPI_NONE, nullptr, w.inner, st_inner);
    k_cocr_rho<T><<<vgrid(), 256, 0, s>>>((const V*)w.t, (const V*)w.v, w.sys, w.part_vec, w.p);
    check();
    fin<3>(w.part_vec, w.p.nblk, w.p.pstride, OpCocrBeta{});
    k_cocr_pq<T><<<vgrid(), 256, 0, s>>>((const V*)w.t, (const V*)w.v, (V*)w.pv, (V*)w.rhat, (const V*)w.dinv,
                                         w.sys, w.part_vec, w.p);
    check();
    fin<3>(w.part_vec, w.p.nblk, w.p.pstride, OpCocrAlpha{});
    k_cocr_xr<T><<<vgrid(), 256, 0, s>>>((V*)w.d, (const V*)w.pv, (V*)w.rin, (const V*)w.rhat, (V*)w.t,
                                         (const V*)w.dinv, w.sys, w.part_vec, w.p);
    check();
    fin<3>(w.part_vec, w.p.nblk, w.p.pstride, OpCocrRes{});
  }

  // one iteration of the single-vector methods (BiCGStab, COCG or COCR)
  template <typename T>
  void loop_iter(const int* st_inner) {
    if (w.method == FIT_COCG) cocg_iter<T>(st_inner);
    else if (w.method == FIT_COCR) cocr_iter<T>(st_inner);
    else bicg_iter<T>(st_inner);
  }

  // one BiCGStab iteration (predicated on inner status)
  template <typename T>
  void bicg_iter(const int* st_inner) {
    using V = typename cplx<T>::t;
    const bool pc = w.dinv != nullptr;
    k_bicg_p<T><<<vgrid(), 256, 0, s>>>((const V*)w.rin, (V*)w.pv, (const V*)w.v, (const V*)w.dinv, (V*)w.phat,
                                        w.sys, w.p);
    check();
    long long n1 = apply(pc ? w.phat : w.pv, w.v, FIT_EPI_DOT_U, w.rhat, w.inner, st_inner);
    fin<3>(w.part_apply, n1, 4, OpAlpha{});
    k_bicg_s<T><<<vgrid(), 256, 0, s>>>((V*)w.rin, (const V*)w.v, (const V*)w.dinv, (V*)w.shat, w.sys, w.p);
    check();
    // <t, s> and <t, t> with t = A s^: the epilogue's <y, x> uses the apply input, so with a
    // preconditioner the dots are taken in k_bicg_dots_ts instead
    long long n2 = apply(pc ? w.shat : w.rin, w.t, pc ? FIT_EPI_NONE : FIT_EPI_DOT_TS, nullptr, w.inner, st_inner);
    if (pc) {
      k_dots_ts<T><<<vgrid(), 256, 0, s>>>((const V*)w.t, (const V*)w.rin, w.sys, w.part_vec, w.p);
      check();
      fin<3>(w.part_vec, w.p.nblk, w.p.pstride, OpOmega{});
    } else {
      fin<3>(w.part_apply, n2, 4, OpOmega{});
    }
    k_bicg_xr<T><<<vgrid(), 256, 0, s>>>((V*)w.d, (const V*)(pc ? w.phat : w.pv), (V*)w.rin, (const V*)w.t,
                                         (const V*)(pc ? w.shat : nullptr), (const V*)w.rhat, w.sys, w.part_vec, w.p);
    check();
    fin<3>(w.part_vec, w.p.nblk, w.p.pstride, OpRho{});
  }

  // the three CGS2 passes over V[0..j] (mode 0: dots; 1: update with h, dots; 2: update with h2, norm)
  FgOut fg_out() const { return FgOut{w.h1, w.h2, w.hn2, w.H, w.G, w.CS, w.SN, w.cnt}; }
  template <typename T, int MODE, int S>
  void ortho_bulk(int j, const double* h) {
    using V = typename cplx<T>::t;
    constexpr int CH = FgChunk<T>::CH;
    const size_t smem = (size_t)S * (j + 2) * CH * sizeof(V) + S * 8 + 2 * FG_MAXV * sizeof(T) +
                        2 * FG_MAXV * sizeof(double);
    auto kern = k_fg_cgs_bulk<T, MODE, S>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<vgrid(), CH, smem, s>>>((const V*)w.Vb, j, h, w.sys, w.part_vec, fg_out(), w.p);
    check();
  }
  // the bulk-copy passes need 16-byte aligned chunks of every vector
  bool bulk_ok() const { return w.esz == 16 || (w.p.ne % 2) == 0; }
  template <typename T, int MODE>
  void ortho(int j, const double* h) {
    using V = typename cplx<T>::t;
    constexpr int CH = FgChunk<T>::CH;
    const int nv = j + 1;
    if (bulk_ok()) {  // three stages while they fit two blocks per SM, else two
      if ((size_t)3 * (j + 2) * CH * sizeof(V) <= 100 * 1024) ortho_bulk<T, MODE, 3>(j, h);
      else ortho_bulk<T, MODE, 2>(j, h);
      return;
    }
    if (MODE == 0) {
      k_fg_dots<T><<<vgrid(), CH, 0, s>>>((const V*)w.Vb, j, w.sys, w.part_vec, fg_out(), w.p);
    } else if (MODE == 1) {
      const size_t smem = (size_t)(nv + 1) * CH * sizeof(V) + (size_t)2 * nv * sizeof(double) +
                          (size_t)2 * nv * sizeof(T);
      auto kern = k_fg_update_dots<T>;
      if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      kern<<<vgrid(), CH, smem, s>>>((const V*)w.Vb, j, h, w.sys, w.part_vec, fg_out(), w.p);
    } else {
      k_fg_update_norm<T><<<vgrid(), CH, 0, s>>>((const V*)w.Vb, j, h, w.sys, w.part_vec, fg_out(), w.p);
    }
    check();
  }

  // Arnoldi step j of FGMRES (predicated on inner status)
  template <typename T>
  void fg_step(int j, const int* st_inner) {
    using V = typename cplx<T>::t;
    size_t vecb = (size_t)w.p.ne * w.p.B * w.esz;
    const char* vj = (const char*)w.Vb + (size_t)j * vecb;
    char* wj1 = (char*)w.Vb + (size_t)(j + 1) * vecb;
    const void* zin = vj;
    if (w.pc == FIT_PC_JACOBI || w.pc == FIT_PC_EPS) {
      k_fg_precond_diag<T><<<vgrid(), 256, 0, s>>>((const V*)w.Vb, (V*)w.Zb, j, (const V*)w.dinv, w.sys, w.p);
      check();
      zin = (const char*)w.Zb + (size_t)j * vecb;
    } else if (w.pc == FIT_PC_UNET && ((j + 1) % w.p.pc_every) != 0) {
      // every other step of the cycle: the Jacobi term
      k_fg_precond_diag<T><<<vgrid(), 256, 0, s>>>((const V*)w.Vb, (V*)w.Zb, j, (const V*)w.dinv, w.sys, w.p);
      check();
      zin = (const char*)w.Zb + (size_t)j * vecb;
    } else if (w.pc == FIT_PC_UNET) {
      // The network's direction: z_j = U(v_i) / sqrt(n_e) + 1e-3 D^-1 v_j with i = j + 1 - pc_every and
      // v_i of unit norm (the network sees v / rms(v) = sqrt(n_e) v).  By default pc_every = m: the last
      // step of the cycle takes the network's answer for the cycle's first vector, the normalised true
      // residual, which U (trained on residual -> error-direction pairs) maps to the direction of the
      // current error.  Every earlier step is a Jacobi step, so the cycle's subspace is the Jacobi
      // Krylov subspace of m - 1 steps plus the network's direction: flexible GMRES minimises the
      // residual over whatever directions z_j it is given (their scale is immaterial), and a poor
      // network costs one direction, not the cycle.  The small Jacobi term keeps z_j a usable direction
      // when the network outputs zero (an untrained network, whose head starts at zero, then gives
      // exactly Jacobi FGMRES).
      const float sin = (float)sqrt((double)w.p.ne), sout = 1.0f / sin;
      const char* vin = (const char*)w.Vb + (size_t)(j + 1 - w.p.pc_every) * vecb;
      for (int b = 0; b < w.p.B; ++b) {
        const size_t off = (size_t)b * w.p.ne * w.esz;
        fit_status r = fit_unet_apply_vec(w.g->unet, w.g, vin + off, (char*)w.Zb + (size_t)j * vecb + off, sin,
                                          sout, w.x16, (const char*)w.dinv + off, vj + off, 1e-3f, s);
        if (r != FIT_OK && st == FIT_OK) st = r;
      }
      zin = (const char*)w.Zb + (size_t)j * vecb;
    }
    apply(zin, wj1, FIT_EPI_NONE, nullptr, w.inner, st_inner);
    // CGS2: each pass's last block reduces its partial sums (h, h2, then ||w||^2 and the Givens step)
    ortho<T, 0>(j, nullptr);
    ortho<T, 1>(j, w.h1);
    ortho<T, 2>(j, w.h2);
    k_fg_scale<T><<<vgrid(), 256, 0, s>>>((V*)w.Vb, j, w.sys, w.p);
    check();
  }

  template <typename T>
  void fg_finish() {
    using V = typename cplx<T>::t;
    k_fg_solve<<<(w.p.B + 127) / 128, 128, 0, s>>>(w.H, w.G, w.Y, w.sys, w.p);
    check();
    if (w.m <= 16) k_fg_combine<T, 16><<<vgrid(), 256, 0, s>>>((const V*)w.Zb, (V*)w.d, w.Y, w.sys, w.p);
    else if (w.m <= 32) k_fg_combine<T, 32><<<vgrid(), 256, 0, s>>>((const V*)w.Zb, (V*)w.d, w.Y, w.sys, w.p);
    else k_fg_combine<T, 64><<<vgrid(), 256, 0, s>>>((const V*)w.Zb, (V*)w.d, w.Y, w.sys, w.p);
    check();
  }

  double2* hist = nullptr;
  int hist_len = 0, hist_every = 1;

  template <typename T>
  void outer_tail(const int* st_outer) {
    using V = typename cplx<T>::t;
    k_copy_r<<<vgrid(), 256, 0, s>>>(w.r128, w.rprev, w.sys, w.p);
    k_update_x<T><<<vgrid(), 256, 0, s>>>(x, (const V*)w.d, w.sys, w.p);
    check();
    apply(x, w.r128, FIT_EPI_RESID, rhs, FIT_C128, st_outer);
    k_mr_dots<<<vgrid(), 256, 0, s>>>(w.rprev, w.r128, w.sys, w.part_vec, w.p);
    check();
    fin<4>(w.part_vec, w.p.nblk, w.p.pstride, OpOuter{});
    k_mr_combine<T><<<vgrid(), 256, 0, s>>>(x, (const V*)w.d, w.r128, w.rprev, w.sys, w.p);
    k_clear_mr<<<(w.p.B + 127) / 128, 128, 0, s>>>(w.sys, w.p.B);
    check();
    if (hist) {
      k_history<<<vgrid(), 256, 0, s>>>(x, hist, w.sys, hist_every, hist_len, w.p);
      k_history_count<<<(w.p.B + 127) / 128, 128, 0, s>>>(w.sys, hist_every, hist_len, w.p);
      check();
    }
  }

  int* mirror_inner = nullptr;  // per-system status words for the apply's predicate
  int* mirror_outer = nullptr;
  void cond(int which, int guard_max, cudaGraphConditionalHandle h, int use_handle) {
    k_cond<<<1, 256, 0, s>>>(w.sys, w.ctl, w.p, which, guard_max, h, use_handle, mirror_inner, mirror_outer);
    check();
  }
};

// The apply's status predicate reads an int per system with stride 1; the Sys struct is larger, so
// keep small mirrored status arrays instead.
__global__ void k_mirror_status(const Sys* __restrict__ sys, int* inner, int* outer, int B) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) {
    inner[b] = sys[b].inner_status;
    outer[b] = sys[b].outer_status;
  }
}

template <typename T>
fit_status run_batch(Work& w, const double2* rhs, double2* x, cudaStream_t s, int use_graph, int max_outer_guard,
                     int max_inner_guard, double2* hist, int hist_len, int hist_every) {
  int* st_inner = nullptr;
  int* st_outer = nullptr;
  fit_status st;
  if ((st = w.alloc((void**)&st_inner, w.p.B * sizeof(int))) != FIT_OK) return st;
  if ((st = w.alloc((void**)&st_outer, w.p.B * sizeof(int))) != FIT_OK) return st;
  Seq q{w, rhs, x, s};
  q.mirror_inner = st_inner;
  q.mirror_outer = st_outer;
  q.hist = hist;
  q.hist_len = hist_len;
  q.hist_every = hist_every;
  if (w.pc == FIT_PC_JACOBI || w.pc == FIT_PC_UNET || w.pc == FIT_PC_EPS) {  // D^-1 per system, once per solve
    const fit_grid* g = w.g;
    k_dinv<T><<<dim3(w.p.nblk, w.p.B), 256, 0, s>>>((const T*)w.nusum, w.mixed ? (const T*)g->ek32 : (const T*)g->ek64,
                                                     g->mask, w.omega, g->nx, g->ny, g->nxp,
                                                     (typename cplx<T>::t*)w.dinv, w.p, w.pc == FIT_PC_EPS);
    FIT_CHECK_CUDA(cudaGetLastError());
  }
  // pick the apply kernels (autotuner) now: timing cannot run inside a stream capture
  {
    void* ti = w.method == FIT_FGMRES ? w.Vb : w.pv;
    void* to = w.method == FIT_FGMRES ? w.d : w.v;
    FIT_CHECK_CUDA(cudaMemsetAsync(ti, 0, (size_t)w.p.ne * w.p.B * w.esz, s));
    fit_status ts = fit_tune_apply(w.g, w.p.B, w.omega, ti, to, w.inner, s);
    if (ts == FIT_OK) ts = fit_tune_apply(w.g, w.p.B, w.omega, rhs, w.r128, FIT_C128, s);
    if (ts != FIT_OK) return ts;
  }
  auto mirror = [&](cudaStream_t ss) {
    k_mirror_status<<<(w.p.B + 127) / 128, 128, 0, ss>>>(w.sys, st_inner, st_outer, w.p.B);
  };
  const bool bicg = w.method == FIT_BICGSTAB || w.method == FIT_COCG || w.method == FIT_COCR;  // single-vector loops

  // FIT_TRACE_SOLVE=1 prints the scalars of system 0 after every host-loop step (stderr)
  const char* tr = getenv("FIT_TRACE_SOLVE");
  const bool trace = tr && tr[0] == '1';
  auto dump = [&](const char* what, int k) {
    if (!trace) return;
    Sys h;
    cudaStreamSynchronize(s);
    cudaMemcpy(&h, w.sys, sizeof(Sys), cudaMemcpyDeviceToHost);
    fprintf(stderr, "[fit trace] %s %d: outer=%d st=%d/%d it=%d jl=%d rin=%.3e relres=%.3e inv_hn=%.3e iters=%d\n", what,
            k, h.outer, h.outer_status, h.inner_status, h.inner_it, h.jlast, sqrt(h.rin2),
            h.bnorm2 > 0 ? sqrt(h.rnorm2 / h.bnorm2) : 0.0, h.inv_hn, h.iters);
  };
  if (!use_graph) {
    q.outer_init();
    mirror(s);
    dump("init", 0);
    Ctl hc;
    for (int outer = 0; outer < max_outer_guard; ++outer) {
      q.inner_start<T>();
      mirror(s);
      if (bicg) {
        for (int it = 0; it < max_inner_guard; ++it) {
          q.loop_iter<T>(st_inner);
          if (it % 100 == 99) dump("bicg it", it + 1);
          q.cond(0, max_inner_guard, 0, 0);
          FIT_CHECK_CUDA(cudaMemcpyAsync(&hc, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
          FIT_CHECK_CUDA(cudaStreamSynchronize(s));
          if (q.st != FIT_OK) return q.st;
          if (!hc.cond) break;
        }
      } else {
        for (int j = 0; j < w.m; ++j) {
          q.fg_step<T>(j, st_inner);
          dump("fg step", j);
          q.cond(0, max_inner_guard, 0, 0);
          FIT_CHECK_CUDA(cudaMemcpyAsync(&hc, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
          FIT_CHECK_CUDA(cudaStreamSynchronize(s));
          if (q.st != FIT_OK) return q.st;
          if (!hc.cond) break;
        }
        q.fg_finish<T>();
      }
      q.outer_tail<T>(st_outer);
      dump("outer", outer);
      q.cond(1, max_outer_guard, 0, 0);
      FIT_CHECK_CUDA(cudaMemcpyAsync(&hc, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
      FIT_CHECK_CUDA(cudaStreamSynchronize(s));
      if (q.st != FIT_OK) return q.st;
      if (!hc.cond) break;
    }
    return q.st;
  }

  // ---- graph mode: one launch for the whole batch solve --------------------------------------
  // Capture runs on private streams (the caller's stream may be the legacy default stream, which
  // cannot be captured); the instantiated graph is launched on the caller's stream.
  cudaStream_t s_top = nullptr, s_outer = nullptr, s_inner = nullptr;
  FIT_CHECK_CUDA(cudaStreamCreateWithFlags(&s_top, cudaStreamNonBlocking));
  FIT_CHECK_CUDA(cudaStreamCreateWithFlags(&s_outer, cudaStreamNonBlocking));
  FIT_CHECK_CUDA(cudaStreamCreateWithFlags(&s_inner, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  fit_status result = FIT_OK;
  auto fail = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && result == FIT_OK) {
      fit_set_error(std::string("fit_solve graph: ") + what + ": " + cudaGetErrorString(e));
      result = FIT_ECUDA;
    }
  };
  do {
    FIT_CHECK_CUDA(cudaGraphCreate(&graph, 0));
    // top level: outer init, then the outer WHILE node
    fail(cudaStreamBeginCaptureToGraph(s_top, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
         "capture top");
    if (result != FIT_OK) break;
    q.s = s_top;
    q.outer_init();
    mirror(s_top);
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edata = nullptr;
    size_t ndeps = 0;
    cudaGraph_t capg = nullptr;
    fail(cudaStreamGetCaptureInfo(s_top, &cst, nullptr, &capg, &deps, &edata, &ndeps), "capture info");
    cudaGraphConditionalHandle h_outer;
    fail(cudaGraphConditionalHandleCreate(&h_outer, capg, 1, cudaGraphCondAssignDefault), "outer handle");
    cudaGraphNodeParams cp_outer = {};
    cp_outer.type = cudaGraphNodeTypeConditional;
    cp_outer.conditional.handle = h_outer;
    cp_outer.conditional.type = cudaGraphCondTypeWhile;
    cp_outer.conditional.size = 1;
    cudaGraphNode_t n_outer;
    fail(cudaGraphAddNode(&n_outer, capg, deps, edata, ndeps, &cp_outer), "outer node");
    fail(cudaStreamUpdateCaptureDependencies(s_top, &n_outer, nullptr, 1, cudaStreamSetCaptureDependencies), "deps");
    cudaGraph_t body_outer = cp_outer.conditional.phGraph_out[0];
    cudaGraphConditionalHandle h_inner = 0;
    if (bicg) {
      fail(cudaGraphConditionalHandleCreate(&h_inner, body_outer, 1, cudaGraphCondAssignDefault), "inner handle");
      q.h_inner = h_inner;
      q.use_h_inner = 1;
    }
    // outer body
    fail(cudaStreamBeginCaptureToGraph(s_outer, body_outer, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
         "capture outer body");
    if (result != FIT_OK) break;
    q.s = s_outer;
    q.inner_start<T>();
    mirror(s_outer);
    if (bicg) {
      cudaGraph_t capo = nullptr;
      fail(cudaStreamGetCaptureInfo(s_outer, &cst, nullptr, &capo, &deps, &edata, &ndeps), "capture info 2");
      cudaGraphNodeParams cp_inner = {};
      cp_inner.type = cudaGraphNodeTypeConditional;
      cp_inner.conditional.handle = h_inner;
      cp_inner.conditional.type = cudaGraphCondTypeWhile;
      cp_inner.conditional.size = 1;
      cudaGraphNode_t n_inner;
      fail(cudaGraphAddNode(&n_inner, capo, deps, edata, ndeps, &cp_inner), "inner node");
      fail(cudaStreamUpdateCaptureDependencies(s_outer, &n_inner, nullptr, 1, cudaStreamSetCaptureDependencies), "deps2");
      cudaGraph_t body_inner = cp_inner.conditional.phGraph_out[0];
      fail(cudaStreamBeginCaptureToGraph(s_inner, body_inner, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
           "capture inner body");
      if (result != FIT_OK) break;
      q.s = s_inner;
      q.loop_iter<T>(st_inner);
      q.cond(0, max_inner_guard, h_inner, 1);
      cudaGraph_t tmp;
      fail(cudaStreamEndCapture(s_inner, &tmp), "end inner");
      q.s = s_outer;
    } else {
      for (int j = 0; j < w.m; ++j) {
        q.fg_step<T>(j, st_inner);
        mirror(s_outer);
      }
      q.fg_finish<T>();
    }
    q.outer_tail<T>(st_outer);
    q.cond(1, max_outer_guard, h_outer, 1);
    cudaGraph_t tmp2;
    fail(cudaStreamEndCapture(s_outer, &tmp2), "end outer");
    cudaGraph_t tmp3;
    fail(cudaStreamEndCapture(s_top, &tmp3), "end top");
    if (result != FIT_OK || q.st != FIT_OK) break;
    fail(cudaGraphInstantiate(&exec, graph, 0), "instantiate");
    if (result != FIT_OK) break;
    fail(cudaGraphLaunch(exec, s), "launch");
    fail(cudaStreamSynchronize(s), "run");
  } while (0);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(s_top);
  cudaStreamDestroy(s_outer);
  cudaStreamDestroy(s_inner);
  if (q.st != FIT_OK) return q.st;
  return result;
}

}  // namespace

namespace {
// y = D(w)^-1 x with D = diag(A(w)) = sum of M_nu over the facets containing the edge - w^2 M_eps
// + j w M_kappa (Eq. Precond construction); masked edges: y = x
template <typename T>
__global__ void k_jacobi_apply(const typename cplx<T>::t* __restrict__ x, typename cplx<T>::t* y, const T* __restrict__ nu,
                               const T* __restrict__ ek, const uint8_t* __restrict__ mask, const double* __restrict__ omega,
                               int nx, int ny, int nz, int nxp, long long ne, int nbatch, double out_scale) {
  const long long n = ne * nbatch;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / ne);
    const long long e = t - (long long)b * ne;
    const long long c = e / 3;
    const int q = (int)(e - 3 * c);
    const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
    const long long cp = i + (long long)nxp * (j + (long long)ny * k);
    const auto xv = x[t];
    typename cplx<T>::t o;
    if ((mask[cp] >> q) & 1) {
      o = xv;
    } else {
      const double2 dg = fit_jacobi_diag<T>(nu, ek, i, j, k, q, nxp, ny, omega[b]);
      const double dr = dg.x, di = dg.y;
      const double den = (dr * dr + di * di) / out_scale;
      o.x = (T)((xv.x * dr + xv.y * di) / den);
      o.y = (T)((xv.y * dr - xv.x * di) / den);
    }
    y[t] = o;
  }
}
}  // namespace

extern "C" {

fit_status fit_jacobi(fit_grid* g, int nbatch, const double* omega, const void* x, void* y, fit_prec prec,
                      void* stream) {
  FIT_REQUIRE(g && omega && x && y && nbatch >= 1, "fit_jacobi: bad argument");
  FIT_REQUIRE(g->has_materials, "fit_jacobi: materials not set");
  FIT_CHECK_CUDA(cudaSetDevice(g->device));
  cudaStream_t s = (cudaStream_t)stream;
  double* om = nullptr;
  FIT_CHECK_CUDA(cudaMallocAsync((void**)&om, nbatch * sizeof(double), s));
  FIT_CHECK_CUDA(cudaMemcpyAsync(om, omega, nbatch * sizeof(double), cudaMemcpyHostToDevice, s));
  const long long n = g->ne * nbatch;
  const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 32);
  if (prec == FIT_C64)  // scaled coefficients: D_s = s D, so D^-1 = s D_s^-1
    k_jacobi_apply<float><<<blocks, 256, 0, s>>>((const float2*)x, (float2*)y, g->nu32, g->ek32, g->mask, om, g->nx,
                                                 g->ny, g->nz, g->nxp, g->ne, nbatch, g->coef_scale);
  else
    k_jacobi_apply<double><<<blocks, 256, 0, s>>>((const double2*)x, (double2*)y, g->nu64, g->ek64, g->mask, om, g->nx,
                                                  g->ny, g->nz, g->nxp, g->ne, nbatch, 1.0);
  FIT_CHECK_CUDA(cudaGetLastError());
  FIT_CHECK_CUDA(cudaFreeAsync(om, s));
  return FIT_OK;
}

void fit_solve_opts_default(fit_solve_opts* o) {
  if (!o) return;
  o->method = FIT_BICGSTAB;
  o->restart = 30;
  o->precision = FIT_SOLVE_MIXED;
  o->max_iter = 20000;
  o->max_outer = 30;
  o->inner_tol = 1e-4;
  o->batch = 0;
  o->use_graph = 1;
  o->precond = FIT_PC_NONE;
  o->stream = nullptr;
  o->history = nullptr;
  o->history_len = 0;
  o->history_every = 1;
  o->pc_every = 0;
}

fit_status fit_solve(fit_grid* g, int nfreq, const double* omega, const void* rhs, void* x, double tol,
                     const fit_solve_opts* opts, fit_solve_report* report) {
  FIT_REQUIRE(g && omega && rhs && x, "fit_solve: null argument");
  FIT_REQUIRE(nfreq >= 1, "fit_solve: nfreq must be >= 1");
  FIT_REQUIRE(tol > 0 && isfinite(tol), "fit_solve: tol must be positive");
  FIT_REQUIRE(g->has_materials, "fit_solve: materials not set");
  fit_solve_opts o;
  fit_solve_opts_default(&o);
  if (opts) o = *opts;
  FIT_REQUIRE(o.method == FIT_BICGSTAB || o.method == FIT_FGMRES || o.method == FIT_COCG || o.method == FIT_COCR,
              "fit_solve: unknown method");
  FIT_REQUIRE(o.precision == FIT_SOLVE_C128 || o.precision == FIT_SOLVE_MIXED, "fit_solve: unknown precision");
  FIT_REQUIRE(o.method != FIT_FGMRES || (o.restart >= 1 && o.restart <= FG_MAXV - 1),
              "fit_solve: FGMRES restart must be in 1..64");
  FIT_REQUIRE(o.precond != FIT_PC_EPS || g->eps_positive,
              "fit_solve: FIT_PC_EPS needs M_eps finite and > 0 on every unmasked edge");
  FIT_REQUIRE(o.precond == FIT_PC_NONE || o.precond == FIT_PC_JACOBI || o.precond == FIT_PC_UNET ||
                  o.precond == FIT_PC_EPS,
              "fit_solve: unknown preconditioner");
  FIT_REQUIRE(o.precond != FIT_PC_UNET || g->unet != nullptr,
              "fit_solve: FIT_PC_UNET needs a network attached with fit_set_preconditioner");
  FIT_REQUIRE(o.precond != FIT_PC_UNET || (o.method == FIT_FGMRES && o.precision == FIT_SOLVE_MIXED),
              "fit_solve: the learned preconditioner runs inside complex64 FGMRES (FIT_SOLVE_MIXED)");
  FIT_REQUIRE(o.max_iter >= 1 && o.max_outer >= 1, "fit_solve: iteration caps must be >= 1");
  FIT_REQUIRE(o.inner_tol > 0 && o.inner_tol < 1, "fit_solve: inner_tol must be in (0, 1)");
  FIT_REQUIRE(!o.history || (o.history_len >= 1 && o.history_every >= 1), "fit_solve: bad history options");
  FIT_REQUIRE(o.pc_every >= 0, "fit_solve: pc_every must be >= 0");
  FIT_REQUIRE(!o.history || o.batch == 0 || o.batch >= nfreq, "fit_solve: history needs all systems in one batch");
  for (int f = 0; f < nfreq; ++f) FIT_REQUIRE(isfinite(omega[f]), "fit_solve: omega must be finite");
  if (fit_check_abort(g, "fit_solve") != FIT_OK) return FIT_ETIMEOUT;
  FIT_CHECK_CUDA(cudaSetDevice(g->device));
  cudaStream_t s = (cudaStream_t)o.stream;
  const int mixed = o.precision == FIT_SOLVE_MIXED;
  const int m = o.method == FIT_FGMRES ? o.restart : 0;

  // HBM admission: the largest batch whose workspace fits the budget
  int B = o.batch > 0 ? std::min(o.batch, nfreq) : nfreq;
  size_t held = g->bytes_held;
  while (B > 1 && g->budget && held + workspace_bytes(g, B, o.method, m, mixed, o.precond) > g->budget) B = (B + 1) / 2;
  if (g->budget && held + workspace_bytes(g, B, o.method, m, mixed, o.precond) > g->budget) {
    fit_set_error("fit_solve: the Krylov workspace of one system exceeds the HBM budget");
    return FIT_EBUDGET;
  }

  fit_status overall = FIT_OK;
  std::vector<Sys> hs;
  for (int f0 = 0; f0 < nfreq; f0 += B) {
    int nb = std::min(B, nfreq - f0);
    Work w;
    w.g = g;
    w.method = o.method;
    w.m = m > 0 ? m : 30;
    w.mixed = mixed;
    w.pc = o.precond;
    fit_status st = setup(w, nb);
    if (st != FIT_OK) return st;
    w.p.tol = tol;
    w.p.inner_tol = o.inner_tol;
    w.p.max_iter = o.max_iter;
    w.p.max_outer = o.max_outer;
    w.p.pc_every = o.pc_every > 0 ? o.pc_every : w.m;  // 0: once per cycle, at its last step
    FIT_CHECK_CUDA(cudaMemcpyAsync(w.omega, omega + f0, nb * sizeof(double), cudaMemcpyHostToDevice, s));
    const double2* rb = (const double2*)rhs + (size_t)f0 * g->ne;
    double2* xb = (double2*)x + (size_t)f0 * g->ne;
    FIT_CHECK_CUDA(cudaStreamSynchronize(s));
    auto t0 = std::chrono::steady_clock::now();
    int outer_guard = o.max_outer + 1;
    int inner_guard = o.max_iter + 1;
    double2* hist = (double2*)o.history;
    if (hist && nb != nfreq) {
      fit_set_error("fit_solve: history needs all systems in one batch (raise the HBM budget)");
      return FIT_EBUDGET;
    }
    st = mixed ? run_batch<float>(w, rb, xb, s, o.use_graph, outer_guard, inner_guard, hist, o.history_len,
                                  o.history_every)
               : run_batch<double>(w, rb, xb, s, o.use_graph, outer_guard, inner_guard, hist, o.history_len,
                                   o.history_every);
    if (st != FIT_OK) return st;
    FIT_CHECK_CUDA(cudaStreamSynchronize(s));
    double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    // a bounded wait that ran out (apply or network kernels) or the abort word ends the solve: the
    // reports of this batch are still filled, later batches are not run
    fit_status dev_err = fit_take_device_error(g);
    if (dev_err == FIT_OK && w.pc == FIT_PC_UNET && fit_unet_take_timeout()) {
      fit_set_error("fit_solve: a bounded wait in a learned-preconditioner convolution ran out");
      dev_err = FIT_ETIMEOUT;
    }
    hs.resize(nb);
    FIT_CHECK_CUDA(cudaMemcpy(hs.data(), w.sys, nb * sizeof(Sys), cudaMemcpyDeviceToHost));
    for (int b = 0; b < nb; ++b) {
      const Sys& y = hs[b];
      fit_status ps = FIT_OK;
      switch (y.outer_status) {
        case SYS_CONV: ps = FIT_OK; break;
        case SYS_NAN: ps = FIT_ENAN; break;
        case SYS_BREAK: ps = FIT_BREAKDOWN; break;
        default: ps = FIT_NOT_CONVERGED; break;
      }
      if (ps != FIT_OK && overall == FIT_OK) overall = ps;
      if (report) {
        fit_solve_report& r = report[f0 + b];
        r.status = ps;
        r.iterations = y.iters;
        r.outer = y.outer;
        r.relres = y.bnorm2 > 0 ? sqrt(y.rnorm2 / y.bnorm2) : 0.0;
        r.seconds = secs;
        r.snapshots = y.hist;
      }
    }
    if (dev_err != FIT_OK) return dev_err;
  }
  return overall;
}

}  // extern "C"
