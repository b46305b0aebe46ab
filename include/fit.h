/*
 * fit.h -- C ABI of the GB300 (sm_103a) matrix-free FIT operator and its Krylov solvers.
 *
 * The library implements the frequency-domain finite integration technique of
 * A. Geranmayeh, "Parallel Matrix-Free Implementation of Frequency-Domain Finite Difference
 * Methods for Cluster Computing" (arXiv 1705.08849):
 *
 *     A(w) e = (C^T M_nu C - w^2 M_eps + j w M_kappa) e = b                 (Sec. II, Eq. e2)
 *
 * on a staggered Cartesian grid of nx * ny * nz cells.  C is the primal curl (Eq. CP), never
 * stored; M_nu = M_mu^{-1}, M_eps, M_kappa are diagonal material matrices (Eq. Material).
 *
 * Conventions shared by every call
 *  - Unknown layout (Eq. e12Nxyz, cell-by-cell): cell (i, j, k), 0 <= i < nx, ..., has linear
 *    index c = i + nx*(j + ny*k) and owns the x-, y- and z-edge leaving its low node; the
 *    unknown index is 3*c + w, w = 0, 1, 2 for x, y, z.  n_e = 3 * nx * ny * nz.  Complex values
 *    are interleaved (re, im): a FIT_C64 vector is n_e float2, a FIT_C128 vector n_e double2.
 *    A batch of B vectors is B such vectors back to back (vector b starts at b * n_e).
 *  - Boundaries: all six walls are PEC.  Edges lying in a low wall plane and all 12 edges of a
 *    PEC cell are "masked": their rows and columns of A are the identity (E_tan = 0, Sec. II).
 *    Entities on the high walls are not stored (identically zero).
 *  - Memory: vectors (x, y, rhs, solutions) are DEVICE pointers owned by the caller, on the
 *    device that was current at fit_grid_create.  Geometry and material inputs are HOST
 *    pointers, copied in before the call returns.  The handle owns every derived device array.
 *  - Devices: every call that takes a grid makes the grid's device current (cudaSetDevice) before
 *    its first device allocation or launch, and leaves it current on return; the caller's stream
 *    must belong to that device.
 *  - Errors: every call returns a fit_status and never throws across the ABI.  Negative values
 *    are errors that leave outputs unspecified; FIT_NOT_CONVERGED / FIT_BREAKDOWN still fill
 *    the solution and the report.  fit_last_error() gives a message for the calling thread.
 *  - Threads/streams: a handle is used by one host thread at a time.  Kernels run on the stream
 *    the caller passes (a cudaStream_t cast to void*, NULL = legacy default stream).
 */
#ifndef FIT_GB300_H
#define FIT_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fit_grid fit_grid; /* opaque, library-owned */

typedef enum {
  FIT_OK = 0,
  FIT_NOT_CONVERGED = 1, /* iteration cap reached; x holds the last iterate */
  FIT_BREAKDOWN = 2,     /* Krylov breakdown (|rho| or |omega| underflow, zero Hessenberg) */
  FIT_EINVAL = -1,       /* bad argument (null pointer, size, unsupported option) */
  FIT_ENOMEM = -2,       /* device allocation failed */
  FIT_ECUDA = -3,        /* a CUDA runtime/driver call failed */
  FIT_ETIMEOUT = -4,     /* a bounded device-side wait ran out */
  FIT_EBUDGET = -5,      /* the request exceeds the handle's HBM budget; nothing was allocated */
  FIT_ENAN = -6          /* a NaN/Inf appeared in the right-hand side or an iterate */
} fit_status;

typedef enum { FIT_C64 = 0, FIT_C128 = 1 } fit_prec;

#define FIT_BC_PEC_ALL 0x3Fu /* one bit per wall (x-, x+, y-, y+, z-, z+); only PEC is supported */

/* fit_grid_create -- allocate a grid handle on the current CUDA device.
 * Sec. II (primal/dual grid pair G, G~ with edge lengths L and facet areas A).
 *   nx, ny, nz   cells per axis, each >= 1
 *   dx, dy, dz   host arrays of the nx / ny / nz primal cell widths [m], all > 0
 *   bc_flags     must be FIT_BC_PEC_ALL
 *   out          receives the handle (NULL on error)
 * Returns FIT_EINVAL on bad sizes/widths/flags, FIT_ENOMEM / FIT_ECUDA on device failure. */
fit_status fit_grid_create(int nx, int ny, int nz, const double* dx, const double* dy,
                           const double* dz, unsigned bc_flags, fit_grid** out);

/* fit_set_materials -- build M_eps, M_kappa, M_nu and the edge mask on the device from per-cell
 * materials (Sec. II, Eq. Material: eps averaged over the dual facet, 1/mu along the dual edge,
 * times the grid metric; PEC folded in as the edge mask, Sec. II end).
 *   eps_r, sigma, inv_mu_r   host float arrays of nx*ny*nz cells, index i + nx*(j + ny*k):
 *                            relative permittivity (> 0), conductivity [S/m] (>= 0), 1/mu_r (> 0)
 *   pec_cell                 host uint8 array of nx*ny*nz (nonzero = PEC cell) or NULL
 * Synchronous.  FIT_EINVAL on null pointers or a value outside its range (checked on the host before
 * anything is copied). */
fit_status fit_set_materials(fit_grid* g, const float* eps_r, const float* sigma,
                             const float* inv_mu_r, const unsigned char* pec_cell);

/* fit_set_material_matrices -- load the diagonals directly (Eq. Material, already assembled):
 *   m_eps, m_kappa   host double arrays of n_e edge values (interleaved ordering)
 *   m_nu             host double array of n_e facet values (facet w of cell c at 3*c + w)
 *   edge_mask        host uint8 array of n_e (nonzero = masked edge) or NULL (no mask)
 * Replaces whatever fit_set_materials built.  Synchronous.  fit_apply_sym and FIT_PC_EPS additionally
 * need m_eps finite and > 0 on every unmasked edge; they return FIT_EINVAL otherwise. */
fit_status fit_set_material_matrices(fit_grid* g, const double* m_eps, const double* m_kappa,
                                     const double* m_nu, const unsigned char* edge_mask);

/* fit_apply -- y_b = A(omega_b) x_b for b = 0 .. nbatch-1 (Eq. e2 operator, matrix-free as in
 * Sec. III / Eq. e2t, fused into one stencil pass): masked rows return y = x.
 *   nbatch   >= 1 systems in the batch
 *   omega    HOST array of nbatch angular frequencies [rad/s]
 *   x, y     DEVICE arrays of nbatch * n_e complex values of precision prec; must not overlap
 *   prec     FIT_C64 (float2 vectors, FP32 arithmetic) or FIT_C128 (double2, FP64 arithmetic)
 *   stream   cudaStream_t (as void*) on which the kernel is enqueued; asynchronous
 * FIT_EINVAL on bad arguments. */
fit_status fit_apply(fit_grid* g, int nbatch, const double* omega, const void* x, void* y,
                     fit_prec prec, void* stream);

/* fit_apply_sym -- y'_b = A_s(omega_b) x'_b with the symmetrised operator of Eq. e2s (Sec. II,
 * change of variable e' = M_eps^{1/2} e; Eq. e2tt writes the same operator as cal_A^T cal_A - w^2 I
 * with cal_A = M_mu^{-1/2} C M_eps^{-1/2}):
 *     A_s(w) = D C^T M_nu C D - w^2 I + j w M_kappa / M_eps,   D = M_eps^{-1/2},   = D A(w) D,
 * on unmasked edges; masked rows return y' = x'.  A solution e' of A_s e' = D b gives e = D e'.
 * Same arguments and conventions as fit_apply.  One generic (L1-cached, untiled) kernel pass: this
 * is the operator for callers that work in the symmetrised variable; fit_solve reaches the same
 * Krylov iterates with FIT_PC_EPS on the fused apply. */
fit_status fit_apply_sym(fit_grid* g, int nbatch, const double* omega, const void* x, void* y,
                         fit_prec prec, void* stream);

/* fit_apply_noalloc -- the same operator apply as fit_apply, for callers that must not allocate
 * device memory (the paper has no counterpart).  fit_apply keeps the batch's frequencies in a buffer
 * owned by the handle and may cudaMalloc a larger one on a call with a larger batch; a host thread
 * driving a latency-critical loop (where cudaMalloc / cudaFree can synchronise the device) or a
 * framework whose device memory is entirely managed by its own pool cannot allow that.  This call
 * keeps the frequencies in a static device array of 4096 doubles (32 KiB, held by every device that
 * loads the library until the process exits) and never allocates, never frees and never runs the
 * autotuner: it uses the kernel the autotuner already picked for (prec, nbatch) on this handle, or
 * the first fused variant.
 *   nbatch   1 .. 4096; larger batches return FIT_EINVAL
 *   other arguments as for fit_apply (host omega, device x and y, stream)
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before anything that must not see CUDA runtime set-up work,
 * and before any stream capture.  The address is kept for the life of the process: it belongs to the
 * device's primary context, so after a cudaDeviceReset of that device this call must not be used
 * again in the process.
 * All calls share the one array and each overwrites the entries it uses, so calls whose work may
 * overlap on the GPU (different streams, or different host threads) race on it: serialise them. */
fit_status fit_apply_noalloc(fit_grid* g, int nbatch, const double* omega, const void* x, void* y,
                             fit_prec prec, void* stream);

/* fit_set_abort -- set (value 1) or clear (value 0) the grid's abort word (not in the paper: failure
 * detection of the runtime).  The word lives in pinned host memory mapped into the device, so kernels
 * that are already queued or running see the host's write:
 *   - while it is set, every call on this grid that enqueues device work (fit_apply, fit_apply_sym,
 *     fit_apply_noalloc, fit_solve) returns FIT_ETIMEOUT at once without enqueuing anything;
 *   - a fused apply kernel that starts while it is set leaves at once, and one that is running gives up
 *     at its next bounded wait; either writes no further output and records the abort in the grid's
 *     error word, which fit_sync reports;
 *   - a running fit_solve ends its Krylov loops at the next loop test (every outer step, every 64th inner
 *     step) and returns FIT_ETIMEOUT with x holding the last iterate and the reports filled.
 * The untiled generic kernel has no waits and does not poll the word.  Host only; thread-safe (an
 * atomic store), so another host thread may call it while a solve runs.  FIT_EINVAL for value not 0/1. */
fit_status fit_set_abort(fit_grid* g, int value);

/* fit_sync -- synchronise stream (a cudaStream_t as void*, NULL = legacy default stream), then read and
 * clear the grid's device error word and the learned preconditioner's convolution timeout word.
 * Returns FIT_ETIMEOUT (with fit_last_error saying which) if, since the last check, a bounded wait in a
 * kernel of this grid ran out (about 0.5 s for the fused apply's hand-offs between warps, 2^22 polls
 * for a copy) or the abort word stopped a kernel: the output of that kernel is incomplete.  FIT_OK
 * otherwise; FIT_ECUDA if the synchronisation itself fails.  fit_solve performs the same check before
 * it returns. */
fit_status fit_sync(fit_grid* g, void* stream);

/* Krylov methods (Sec. IV lists the PETSc solvers tried; bcgs and the gmres family are kept, and
 * "cg" and "cr" on this complex symmetric system (A^T = A, Eq. e2) are read as CG and CR with the
 * unconjugated bilinear form, i.e. COCG and COCR):
 *   FIT_BICGSTAB  BiCGStab, r^ = r0, conjugated inner products
 *   FIT_FGMRES    restarted flexible GMRES(restart), CGS2 orthogonalisation, Givens least squares
 *   FIT_COCG      conjugate orthogonal CG: one apply and three fused vector passes per iteration,
 *                 no stored basis; preconditioner none, Jacobi or eps (diagonal, so A stays symmetric)
 *   FIT_COCR      conjugate orthogonal conjugate residual: one apply and three fused vector passes per
 *                 iteration over six vectors; the same preconditioners.  Its residual recurrence is
 *                 fragile in complex64: prefer FIT_SOLVE_C128 */
typedef enum { FIT_BICGSTAB = 0, FIT_FGMRES = 1, FIT_COCG = 2, FIT_COCR = 3 } fit_method;
typedef enum { FIT_SOLVE_C128 = 0, FIT_SOLVE_MIXED = 1 } fit_solve_precision;
/* FIT_PC_EPS: the diagonal (w^2 M_eps)^-1 (1 on masked edges), a constant multiple of M_eps^-1.  It is the
 * change of variable e' = M_eps^{1/2} e of the symmetrised form (Eq. e2s): COCG with FIT_PC_EPS takes
 * exactly the iterates of COCG on M_eps^{-1/2} A M_eps^{-1/2} e' = M_eps^{-1/2} b, mapped back by
 * e = M_eps^{-1/2} e' (the constant w^2 changes no iterate; it keeps the complex64 inner vectors of order
 * one).  With BiCGStab and FGMRES it is a right preconditioner like Jacobi. */
typedef enum { FIT_PC_NONE = 0, FIT_PC_JACOBI = 1, FIT_PC_UNET = 2, FIT_PC_EPS = 3 } fit_pc_kind;

typedef struct fit_solve_opts {
  int method;        /* fit_method: BiCGStab, FGMRES(restart) or COCG (Sec. IV, Fig. Iterative) */
  int restart;       /* FGMRES restart length m (1..64); default 30 */
  int precision;     /* fit_solve_precision: plain complex128 Krylov, or complex64 inner Krylov
                        inside FP64 iterative refinement (true residual b - A x in FP64) */
  int max_iter;      /* cap on Krylov iterations per system (summed over refinement steps) */
  int max_outer;     /* cap on outer steps (refinement steps, or true-residual restarts of a
                        complex128 solve); default 30 */
  double inner_tol;  /* relative tolerance of each inner complex64 solve; default 1e-4 */
  int batch;         /* systems solved together in one batched launch; 0 = all nfreq */
  int use_graph;     /* nonzero: run the Krylov loop as one CUDA graph with a device-side loop */
  int precond;       /* fit_pc_kind applied as the right preconditioner (BiCGStab and COCG: none,
                        Jacobi or eps; the learned one needs FGMRES with FIT_SOLVE_MIXED) */
  void* stream;      /* cudaStream_t (as void*) for all work; NULL = legacy default stream */
  void* history;     /* optional DEVICE buffer of history_len * nfreq * n_e double2: the iterate x
                        after every history_every-th outer step, slot h of system f at
                        (h * nfreq + f) * n_e (used to harvest training pairs); NULL = off */
  int history_len;   /* slots in history (per system) */
  int history_every; /* outer steps between snapshots (>= 1) */
  int pc_every;      /* FIT_PC_UNET: the Arnoldi steps j = 0 .. m-1 of a cycle with (j + 1) % pc_every == 0
                        take the network's direction z_j = U(v_{j+1-pc_every}) (see fit_set_preconditioner),
                        all others the Jacobi term z_j = D^-1 v_j; 0 (the default) means pc_every = m: once
                        per cycle, at its last step, where the network's input is the cycle's first vector,
                        the normalised true residual it was trained on.  0 or >= 2 */
} fit_solve_opts;

typedef struct fit_solve_report {
  int status;        /* fit_status of this system */
  int iterations;    /* Krylov iterations (inner iterations summed over refinement steps) */
  int outer;         /* outer steps taken (refinement steps / true-residual restarts) */
  double relres;     /* final true relative residual ||b - A x||_2 / ||b||_2, computed in FP64 */
  double seconds;    /* wall time of the batch this system was solved in */
  int snapshots;     /* history slots written for this system */
} fit_solve_report;

/* fit_solve_opts_default -- fill opts with the defaults named above. */
void fit_solve_opts_default(fit_solve_opts* opts);

/* fit_solve -- solve A(omega_f) x_f = rhs_f for f = 0 .. nfreq-1 to ||b - A x|| <= tol ||b||
 * (Sec. IV stop criterion on the relative residual; the test is on the true residual).
 *   nfreq    >= 1 systems (frequencies, right-hand sides) on this geometry
 *   omega    HOST array of nfreq angular frequencies [rad/s]
 *   rhs      DEVICE array of nfreq * n_e double2 (b = -j w j for an impressed current j, Eq. e2)
 *   x        DEVICE array of nfreq * n_e double2, overwritten with the solutions (x0 = 0)
 *   tol      relative residual target (> 0)
 *   opts     NULL for defaults
 *   report   HOST array of nfreq reports (may be NULL)
 * Refinement: every outer step solves A d = r approximately (complex64 inner solve in
 * FIT_SOLVE_MIXED) and recomputes the true residual in FP64.  x then moves along d by the complex
 * step length that minimises ||b - A x||, so the true residual never grows.  An inner solve that
 * ends above its starting residual gives no step, and the next one (from the same residual, so
 * along the same iterates) stops where that one was smallest.
 * Returns FIT_OK if every system converged, else the first non-OK per-system status, or an
 * error; FIT_ETIMEOUT if the abort word (fit_set_abort) ended the solve or a bounded device wait ran
 * out (the reports of the systems that ran are filled).  Synchronous on opts->stream.  FIT_EBUDGET if the Krylov workspace for the batch does
 * not fit the handle's HBM budget (checked before any allocation). */
fit_status fit_solve(fit_grid* g, int nfreq, const double* omega, const void* rhs, void* x,
                     double tol, const fit_solve_opts* opts, fit_solve_report* report);

/* fit_set_hbm_budget -- cap (bytes) on the device memory the handle may hold; 0 = no cap. */
fit_status fit_set_hbm_budget(fit_grid* g, size_t bytes);

/* fit_grid_info -- sizes: out[0..5] = nx, ny, nz, n_e, bytes held on the device, budget. */
fit_status fit_grid_info(const fit_grid* g, long long* out6);

/* fit_apply_variant_count -- number of launch shapes of the fused TMA stencil kernel for a precision
 * (the candidates the autotuner times; see fit_apply_tuned). */
int fit_apply_variant_count(fit_prec prec);

/* fit_apply_tuned -- the apply kernel the autotuner picked for (prec, nbatch) on this grid:
 *   out7[0] = -2 not tuned yet, -1 generic kernel, k >= 0 fused variant k
 *   out7[1..3] = tile TX, TY and planes per CTA (TZ; 0 = chosen at launch so that the tiles fill
 *               the resident CTAs in one balanced wave; -1 = one system's (column, plane) pairs
 *               split evenly over the resident CTAs) of that kernel
 *   out7[4] = shared-memory ring stages (0 for the generic kernel)
 *   out7[5] = 0 generic or CTA-synchronous fused kernel, 1 warp-specialised fused kernel
 *             (a copy-issuing warp and a masking warp feed the ring, one consumer warp per row)
 *   out7[6] = L2 prefetch distance: planes of the tile requested into L2 this far ahead of
 *             their copy into shared memory (0: none).
 * The autotuner runs on the first fit_apply / fit_solve with a new (prec, nbatch); it times every
 * candidate on the caller's stream (synchronising it) and caches the fastest in the handle.
 * Candidates are timed from a cold L2: for the duration of the tuning the handle holds a scratch
 * buffer of twice the L2 size (counted against fit_set_hbm_budget; if it does not fit, candidates
 * are timed back to back instead).
 * Tests and experiments can force a kernel with the environment variable
 * FIT_APPLY_KERNEL=generic or FIT_APPLY_KERNEL=fused:<k>.
 * Persistence (opt-in): with FIT_TUNE_CACHE=<file> set, the autotuner first looks the key up in that
 * file (fit_tuning_lookup) and uses a recorded choice without timing anything; after a search it
 * appends its result (fit_tuning_record).  The key is the device name and SM count, the grid size, the
 * precision and the batch. */
fit_status fit_apply_tuned(const fit_grid* g, fit_prec prec, int nbatch, int* out7);

/* fit_tuning_record -- append one autotuner result to the text cache file at path (created if
 * missing): key (device name, SM count, nx, ny, nz, prec, nbatch), the number of fused variants this
 * build has for prec, and choice (-1 generic kernel, k >= 0 fused variant k; see fit_apply_tuned).
 * Host only.  FIT_EINVAL on a null or out-of-range argument or if the file cannot be written. */
fit_status fit_tuning_record(const char* path, const char* device, int sm_count, int nx, int ny, int nz,
                             fit_prec prec, int nbatch, int choice);

/* fit_tuning_lookup -- *choice = the last choice recorded in path for this key by a build with the
 * same variant table, or -2 if there is none (a missing file is not an error).  Malformed lines and
 * lines of other keys or builds are skipped.  Host only.  FIT_EINVAL on a null argument. */
fit_status fit_tuning_lookup(const char* path, const char* device, int sm_count, int nx, int ny, int nz,
                             fit_prec prec, int nbatch, int* choice);

/* ---- learned right preconditioner (3-level 3D U-Net) ---------------------------------------------
 * Not in the paper: its matrix-free operator "cannot use black-box preconditioners" (Sec. I), and
 * Sec. III builds only the diagonal one (Eq. Precond).  The network maps a residual to a correction:
 * z = rms(v) U(v / rms(v)) approximates A_in^{-1} v for the scaled complex64 operator of the inner
 * FGMRES.  Layers: two 3x3x3 convs + ReLU per level (16, 32, 64 channels), 2x average pooling,
 * 2x2x2 transposed convs up, skip concatenation, 1x1x1 head to 6 channels.  Activations and conv
 * weights are bf16 with FP32 accumulation on the tensor cores; master weights and Adam are FP32.
 * Tensors are NDHWC on the device (voxel x + nx*(y + ny*z), channels innermost); grid sizes must be
 * multiples of 4.  Input: 16 bf16 channels (Re/Im of the three residual components, then eps_r/10,
 * log10(1+sigma)/8, 1/mu_r, cell size [mm], then 6 zero channels).  Output: 6 FP32 channels. */
typedef struct fit_unet fit_unet;

/* fit_unet_create -- network with He-initialised weights drawn from a counter-based generator. */
fit_status fit_unet_create(unsigned long long seed, fit_unet** out);
void fit_unet_destroy(fit_unet* net);
/* number of FP32 parameters; get/set copy them to/from a HOST array (checkpointing, tests) */
long long fit_unet_param_count(void);
fit_status fit_unet_get_params(const fit_unet* net, float* host, long long n);
fit_status fit_unet_set_params(fit_unet* net, const float* host, long long n);
/* forward: in16 (device bf16 [N][16]) -> out6 (device float [N][6]) */
fit_status fit_unet_forward(fit_unet* net, int nx, int ny, int nz, const void* in16, float* out6, void* stream);
/* loss L = ||U(in) - t||^2 / ||t||^2 (host *loss, synchronising) and its gradient w.r.t. every
 * parameter (device float [param_count], may be NULL) */
fit_status fit_unet_backward(fit_unet* net, int nx, int ny, int nz, const void* in16, const float* target6,
                             float* grad, double* loss, void* stream);
/* one Adam step (beta 0.9 / 0.999, eps 1e-8) on that loss */
fit_status fit_unet_train_step(fit_unet* net, int nx, int ny, int nz, const void* in16, const float* target6,
                               float lr, double* loss, void* stream);
/* pack a complex64 residual r (device, n_e) times scale, plus the grid's material channels, into
 * the network input (device bf16 [ncell][16]) */
fit_status fit_unet_pack(const fit_grid* g, const void* r, double scale, void* out16, void* stream);
/* pack a complex128 correction e (device, n_e) times scale into a training target
 * (device float [ncell][6]); masked edges are zero */
fit_status fit_unet_pack_target(const fit_grid* g, const void* e, double scale, float* out6, void* stream);
/* z = scale * (network output as complex64, n_e), zero on masked edges */
fit_status fit_unet_unpack(const fit_grid* g, const float* y6, double scale, void* z, void* stream);
/* Single layers of the network: the kernels fit_unet_forward and fit_unet_backward run, one call per
 * layer, for per-layer checks and tools.  All tensors are DEVICE pointers in NDHWC layout (voxel
 * x + nx*(y + ny*z), channels innermost); activations are bf16, weights, biases and weight gradients
 * FP32.  Asynchronous on stream.  The convolution calls convert the FP32 weights to the layer's bf16
 * copies in stream-ordered scratch (cudaMallocAsync / cudaFreeAsync) exactly as the network does.
 * FIT_EINVAL for a (cin, cout) that is not a layer shape of the network. */
/* fit_unet_conv3 -- 3x3x3 convolution, stride 1, zero padding 1, on the tensor cores (bf16 operands, FP32
 * accumulation, bf16 result):  out[v][co] = act(bias[co] + sum_{tap, ci} in[v + off(tap)][ci] W[tap][co][ci])
 * with tap = dz*9 + dy*3 + dx, off(tap) = (dx-1, dy-1, dz-1), act = ReLU if relu != 0.
 *   nx, ny, nz >= 1 (any sizes); (cin, cout) in {(16,16), (16,32), (32,32), (32,64), (64,64), (64,32), (32,16)}
 *   in [N][cin] bf16; w [27][cout][cin] FP32 (rounded to bf16 for the MMAs); bias [cout] FP32 or NULL;
 *   out [N][cout] bf16 */
fit_status fit_unet_conv3(int nx, int ny, int nz, int cin, int cout, const void* in, const float* w,
                          const float* bias, int relu, void* out, void* stream);
/* fit_unet_conv3_dgrad -- its data gradient (the same convolution kernel on flipped, transposed weights):
 *   din[v][ci] = sum_{tap, co} dout[v - off(tap)][co] W[tap][co][ci];  dout [N][cout] bf16, din [N][cin] bf16 */
fit_status fit_unet_conv3_dgrad(int nx, int ny, int nz, int cin, int cout, const void* dout, const float* w,
                                void* din, void* stream);
/* fit_unet_conv3_wgrad -- its weight gradient (a GEMM over voxels per tap on the tensor cores, bf16 operands,
 * FP32 accumulation), overwritten:
 *   dw[tap][co][ci] = sum_v dout[v][co] in[v + off(tap)][ci],  db[co] = sum_v dout[v][co] (db may be NULL) */
fit_status fit_unet_conv3_wgrad(int nx, int ny, int nz, int cin, int cout, const void* in, const void* dout,
                                float* dw, float* db, void* stream);
/* fit_unet_tconv -- 2x2x2 transposed convolution, stride 2, from an mx x my x mz grid to the 2x finer one:
 *   out[X][co] = b[co] + sum_ci in[X / 2][ci] W[k][co][ci], k = X_x%2 + 2 (X_y%2) + 4 (X_z%2);
 *   (cin, cout) = (64, 32) or (32, 16); in [mx*my*mz][cin] bf16, w [8][cout][cin] FP32 master weights that
 *   enter as their bf16 rounding (as in the network), FP32 accumulation, out bf16 */
fit_status fit_unet_tconv(int mx, int my, int mz, int cin, int cout, const void* in, const float* w,
                          const float* b, void* out, void* stream);
/* fit_unet_tconv_backward -- din[V][ci] = sum_{k, co} dout[child(V, k)][co] W[k][co][ci] (bf16, W as its bf16
 * rounding), and, overwritten,
 * dw[k][co][ci] = sum_V in[V][ci] dout[child(V, k)][co], db[co] = sum dout[.][co] (FP32) */
fit_status fit_unet_tconv_backward(int mx, int my, int mz, int cin, int cout, const void* in, const void* dout,
                                   const float* w, void* din, float* dw, float* db, void* stream);
/* fit_unet_head -- the 1x1x1 head, 16 -> 6 channels: out[v][o] = b[o] + sum_c in[v][c] W[o][c] (FP32 out) */
fit_status fit_unet_head(long long nvox, const void* in, const float* w, const float* b, float* out, void* stream);
/* fit_unet_head_backward -- din[v][c] = sum_o dout[v][o] W[o][c] (bf16); overwritten dw[o][c] = sum_v dout[v][o]
 * in[v][c], db[o] = sum_v dout[v][o] (FP32) */
fit_status fit_unet_head_backward(long long nvox, const void* in, const float* dout, const float* w, void* din,
                                  float* dw, float* db, void* stream);

/* fit_unet_training_pair -- one training pair of the learned preconditioner from an iterate x_k of a solve
 * of A(omega) x = b whose solution is x* (the harvest step of the training data):
 *     r = b - A(omega) x_k  (FP64 apply),   e = x* - x_k  (the error of the iterate, A e = r),
 *     pair[c][0..5]  = bf16 of r / rms(r)     (Re, Im of the x, y, z edges of cell c)
 *     pair[c][6..11] = bf16 of e / rms(e)     (the direction of the error)
 * with rms(v) = ||v||_2 / sqrt(n_e) over the unmasked edges; masked edges are zero in both halves.  Both
 * halves have unit rms whatever the iterate, so pairs from early and late iterates weigh alike in the
 * loss.  x_k, x_star, b: DEVICE complex128 [n_e];  pair: DEVICE bf16 [ncell][12] (4-byte aligned);
 * rms_out: HOST, may be NULL: receives rms(r) (the call synchronises on stream either way).  Holds two
 * temporary device vectors (counted against the HBM budget) while it runs. */
fit_status fit_unet_training_pair(fit_grid* g, double omega, const void* xk, const void* xstar, const void* b,
                                  void* pair, double* rms_out, void* stream);
/* fit_unet_pair_sample -- network input and target of a stored pair: in16[c] = base16[c] with channels
 * 0..5 replaced by pair[c][0..5]; target6[c] = FP32 of pair[c][6..11].  base16 is the geometry's packed
 * input of a zero residual (fit_unet_pack), which carries its material channels.  DEVICE pointers,
 * base16 and in16 16-byte aligned; asynchronous. */
fit_status fit_unet_pair_sample(long long ncell, const void* pair, const void* base16, void* in16, float* target6,
                                void* stream);

/* fit_unet_train_step_residual -- one Adam step of the network on the residual-angle loss of one input:
 * with r^ the normalised residual in the input's first six channels (in16 as fit_unet_pair_sample builds
 * it, on this grid), z = U(in16) as a complex64 vector (zero on masked edges) and w = A_in(omega) z (the
 * scaled complex64 operator the network serves),
 *     L = 1 - |<w, r^>|^2 / (||w||^2 ||r^||^2),
 * the fraction of the residual that the direction z cannot remove: what flexible GMRES gains from the
 * network's direction, which it may scale freely.  The gradient goes through the apply's adjoint
 * (A^H = conj(A), A complex symmetric).  *loss receives L before the step (the call synchronises).
 * The network keeps four complex64 work vectors of the grid's size between calls. */
fit_status fit_unet_train_step_residual(fit_unet* net, fit_grid* g, double omega, const void* in16, float lr,
                                        double* loss, void* stream);
/* fit_unet_residual_loss -- that loss without a step (validation); synchronising. */
fit_status fit_unet_residual_loss(fit_unet* net, fit_grid* g, double omega, const void* in16, double* loss,
                                  void* stream);

/* attach a network to the grid; fit_solve with precond = FIT_PC_UNET (FGMRES, FIT_SOLVE_MIXED) then
 * gives flexible GMRES one direction from the network per restart cycle by default (see
 * fit_solve_opts.pc_every): at the cycle's last Arnoldi step j = m-1,
 *     z_j = U(v_0) / sqrt(n_e) + 1e-3 D^-1 v_j,
 * v_0 the normalised residual of the cycle, which the network maps to a correction direction
 * (fit_unet_training_pair, fit_unet_train_step_residual); every other step takes the Jacobi direction
 * D^-1 v_j.  The cycle's subspace is thus the Jacobi Krylov subspace of m-1 steps plus the network's
 * direction.  The small Jacobi term keeps z_j usable if the network outputs zero (an untrained network,
 * whose head starts at zero, gives exactly Jacobi FGMRES).  The residual minimisation decides how much of
 * the network's direction to use, so a poor network costs its application time but cannot stop the
 * Jacobi directions from converging.  The grid does not own the network. */
fit_status fit_set_preconditioner(fit_grid* g, int kind, fit_unet* net);

/* fit_jacobi -- y_b = D(omega_b)^-1 x_b with D = diag(A(omega)): for an unmasked edge the sum of M_nu
 * over the four facets containing it (the column sums of squares of the weighted curl, Eq. Precond)
 * minus w^2 M_eps plus j w M_kappa; masked edges are left unchanged.  Same argument conventions as
 * fit_apply.  Allocates a few bytes with cudaMallocAsync on the stream. */
fit_status fit_jacobi(fit_grid* g, int nbatch, const double* omega, const void* x, void* y, fit_prec prec,
                      void* stream);

/* fit_coef_scale -- s such that the complex64 coefficients (and the inner complex64 operator) are
 * s * (SI values): s = 1 / max M_nu.  Materials must be set. */
fit_status fit_coef_scale(const fit_grid* g, double* s);

/* Ports (Sec. IV: structures are driven by time-harmonic currents impressed on the edges of input
 * ports; the edge voltages along a probe are summed; impedance parameters follow, and S parameters
 * with a 50 Ohm source impedance).  A port (or probe) is a list of public edge indices
 * 3*(i + nx*(j + ny*k)) + w, each with an orientation s_k = +1 or -1 relative to the port's
 * reference direction.  Exciting a port with current I impresses the edge currents I s_k; its
 * voltage is V = - sum_k s_k x[edge_k], counted against the current so that the power a source
 * delivers, Re(V conj(I)) / 2, is >= 0 for a passive structure.  Z_ij = V_i / I_j with port j
 * excited alone. */

/* fit_port_rhs -- b_f = -j omega_f (I s) on the port's unmasked edges, zero elsewhere (Eq. e2), for
 * f = 0 .. nfreq-1: the right-hand sides of one port excited at nfreq frequencies.
 *   omega    HOST array of nfreq angular frequencies [rad/s]
 *   nedge    edges in the port (>= 0); edges / signs: HOST arrays of nedge indices in [0, n_e) and
 *            orientations (an edge listed twice adds up)
 *   current  impressed current I [A]
 *   b        DEVICE array of nfreq * n_e double2, overwritten
 * Materials must be set (they fix the mask).  FIT_EINVAL on a null pointer, an edge out of range or
 * a non-finite frequency or current, checked before anything is written.  Synchronous on the stream. */
fit_status fit_port_rhs(fit_grid* g, int nfreq, const double* omega, int nedge, const long long* edges,
                        const double* signs, double current, void* b, void* stream);

/* fit_probe_voltages -- V[f][q] = - sum over the edges of probe q of s_k x_f[edge_k], summed in FP64
 * in a fixed order (the same bits on every run).
 *   x        DEVICE array of nfreq * n_e double2 (solutions of fit_solve)
 *   nprobe   >= 1 probes; off: HOST array of nprobe + 1 offsets (off[0] = 0, non-decreasing): the
 *            edges of probe q are edges[off[q] .. off[q+1]-1], with orientations signs[...]
 *   V        HOST array of nfreq * nprobe (re, im) double pairs, probe fastest
 * FIT_EINVAL on bad offsets or an edge out of range.  Synchronous on the stream. */
fit_status fit_probe_voltages(fit_grid* g, int nfreq, const void* x, int nprobe, const int* off,
                              const long long* edges, const double* signs, double* V, void* stream);

/* fit_z_to_s -- S = (Z - z0 1)(Z + z0 1)^{-1} for a P x P complex impedance matrix (Sec. IV, z0 = 50
 * Ohm in the paper).  Z and S are HOST arrays of P * P (re, im) double pairs, row-major; S may not
 * alias Z.  Host computation (Gauss-Jordan with partial pivoting), no device work.  FIT_EINVAL if
 * z0 <= 0 or Z + z0 1 is singular. */
fit_status fit_z_to_s(int P, const double* Z, double z0, double* S);

/* fit_z_parameters -- the impedance matrices of nport ports at nfreq frequencies (Sec. IV: one
 * right-hand side per excited port and frequency, all solved together).  Builds the nport * nfreq
 * right-hand sides with fit_port_rhs (system j * nfreq + f: port j excited alone with current I at
 * omega_f), solves them as one fit_solve batch, reads every port's voltage with fit_probe_voltages
 * and returns Z[f][i][j] = V_i / I.
 *   omega      HOST array of nfreq angular frequencies
 *   nport, off, edges, signs   the ports, laid out as in fit_probe_voltages (each port is also the
 *              probe that reads its own voltage)
 *   current    I [A], finite and nonzero (Z does not depend on it up to the solver's tolerance)
 *   tol, opts  passed to fit_solve (opts NULL = defaults; opts->stream carries all the work)
 *   Z          HOST array of nfreq * nport * nport (re, im) double pairs: Z[f] is row-major P x P
 *   report     HOST array of nport * nfreq reports in system order j * nfreq + f (may be NULL)
 * Holds 2 * nport * nfreq * n_e double2 of device memory (right-hand sides and solutions) plus the
 * Krylov workspace while it runs, all counted against the HBM budget and freed before return.
 * Returns what fit_solve returns (Z is filled for FIT_NOT_CONVERGED / FIT_BREAKDOWN too; the reports
 * are filled whenever the solve ran, errors included), or an error; FIT_EINVAL on bad ports, a
 * non-finite frequency or current, checked before any device work. */
fit_status fit_z_parameters(fit_grid* g, int nfreq, const double* omega, int nport, const int* off,
                            const long long* edges, const double* signs, double current, double tol,
                            const fit_solve_opts* opts, double* Z, fit_solve_report* report);

/* fit_grid_destroy -- free the handle and all its device memory (NULL is a no-op). */
void fit_grid_destroy(fit_grid* g);

/* fit_status_str -- static English name of a status code. */
const char* fit_status_str(fit_status s);

/* fit_last_error -- message describing the last error on the calling host thread ("" if none). */
const char* fit_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FIT_GB300_H */
