// Krylov solvers on the fused operator (Sec. IV: BiCGStab and the GMRES family).
#include "fit_internal.cuh"

extern "C" {

void fit_solve_opts_default(fit_solve_opts* o) {
  if (!o) return;
  o->method = FIT_BICGSTAB;
  o->restart = 30;
  o->precision = FIT_SOLVE_MIXED;
  o->max_iter = 20000;
  o->max_outer = 20;
  o->inner_tol = 1e-4;
  o->batch = 0;
  o->use_graph = 1;
  o->precond = FIT_PC_NONE;
  o->stream = nullptr;
}

fit_status fit_solve(fit_grid* g, int nfreq, const double* omega, const void* rhs, void* x, double tol,
                     const fit_solve_opts* opts, fit_solve_report* report) {
  (void)g; (void)nfreq; (void)omega; (void)rhs; (void)x; (void)tol; (void)opts; (void)report;
  fit_set_error("fit_solve: not available in this build");
  return FIT_EINVAL;
}

}  // extern "C"
