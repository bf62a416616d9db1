// Internal interface of the batched BiCGSTAB solver.
#pragma once

#include <cmath>

#include "operator.cuh"

namespace dbi {

// Per-problem solver state (FP64 scalars of the BiCGSTAB recurrences).
struct KState {
  double rho_re, rho_im;      // <rhat, r> of the current residual
  double alpha_re, alpha_im;  // alpha of the current iteration
  double om_re, om_im;        // omega of the last completed iteration
  double beta_re, beta_im;    // beta for the next direction update
  double bnorm2, rnorm2, snorm2, rhatnorm2;  // of the scaled system
  double scale;                              // power of two applied to rhs and x
  int iters, code, restart, half;
  int zero_rhs, restarts, pad[2];  // restarts: breakdown restarts so far
};

// A value that is neither NaN nor infinite (host and device).
__host__ __device__ __forceinline__ bool finite_value(double x) { return isfinite(x); }

// End-of-iteration decision of BiCGSTAB for one problem (host and device, so that its branches are
// testable without a GPU). q = (Re, Im <rhat, r>, ||r||^2) of the new residual r of the scaled
// system. In order: a non-finite q or scalar stops the problem (DBI_NONFINITE: NaN or infinity in
// the data, the model or the iteration); convergence (the half step already met tol, or ||r|| <=
// tol ||b||); the iteration limit; a breakdown (omega = 0, or <rhat, r> negligible against
// ||rhat|| ||r||) restarts from the current iterate with rhat := r; otherwise beta for the next
// direction. Returns 1 while the problem stays active.
__host__ __device__ inline int bicgstab_decide(KState &k, const double q[3], double tol, int max_iter) {
  k.iters += 1;
  k.rnorm2 = q[2];
  k.restart = 0;
  if (!finite_value(q[0]) || !finite_value(q[1]) || !finite_value(q[2]) || !finite_value(k.om_re) || !finite_value(k.om_im) ||
      !finite_value(k.alpha_re) || !finite_value(k.alpha_im)) {
    k.code = DBI_NONFINITE;
    return 0;
  }
  if (k.half || q[2] <= tol * tol * k.bnorm2) {
    k.code = DBI_CONVERGED;
    return 0;
  }
  if (k.iters >= max_iter) {
    k.code = DBI_NOT_CONVERGED;
    return 0;
  }
  const double rho_abs = sqrt(q[0] * q[0] + q[1] * q[1]);
  const bool om_zero = k.om_re == 0.0 && k.om_im == 0.0;
  if (om_zero || rho_abs <= 1e-14 * sqrt(k.rhatnorm2 * q[2])) {  // restart: rhat := r, p := r
    k.restart = 1;
    k.restarts += 1;
    k.code = DBI_BREAKDOWN;
    k.rho_re = q[2]; k.rho_im = 0.0;  // <rhat, r> = ||r||^2
    k.alpha_re = 1.0; k.alpha_im = 0.0;
    k.om_re = 1.0; k.om_im = 0.0;
    k.beta_re = 0.0; k.beta_im = 0.0;
    k.rhatnorm2 = q[2];
    return 1;
  }
  // beta = (rho_new / rho) (alpha / omega), complex
  const double rr = k.rho_re * k.rho_re + k.rho_im * k.rho_im;
  const double r1 = (q[0] * k.rho_re + q[1] * k.rho_im) / rr, i1 = (q[1] * k.rho_re - q[0] * k.rho_im) / rr;
  const double oo = k.om_re * k.om_re + k.om_im * k.om_im;
  const double r2 = (k.alpha_re * k.om_re + k.alpha_im * k.om_im) / oo;
  const double i2 = (k.alpha_im * k.om_re - k.alpha_re * k.om_im) / oo;
  k.beta_re = r1 * r2 - i1 * i2;
  k.beta_im = r1 * i2 + i1 * r2;
  k.rho_re = q[0]; k.rho_im = q[1];
  k.code = DBI_NOT_CONVERGED;
  return 1;
}

struct SolverBufs {
  void *r, *rhat, *p, *v, *s, *t;  // [B][2][nz][nx] complex
  KState *st;                      // [B]
  int *active;                     // [B]
  int *counters;                   // [4]: active counts by iteration parity, compaction count
  int *plist;                      // [B] active problems, compacted
  double *partA, *partS, *partB, *partC;  // [B][kRedBlocks][kRedSlots]
};

size_t bytes_solver(const dbi_grid *g, int B, int precision);
SolverBufs carve_solver(Arena &ar, const dbi_grid *g, int B, int precision);
// The same for fields of field_bytes bytes in all (uneven batches).
size_t bytes_solver_fields(size_t field_bytes, int B);
SolverBufs carve_solver_fields(Arena &ar, size_t field_bytes, int B);

// Solves A x = rhs for every problem of `op` (op.in / op.out / op.ident are set internally).
// x_zero: the initial guess is zero (x is overwritten without being read). The iteration runs on
// rhs scaled by a power of two per problem (KState::scale, max |scaled rhs| in [1, 2)); with
// unscale = false the returned x stays in that scaled system (x = scale * A^{-1} rhs).
// Validates Krylov options (tol >= 0, max_iter >= 0, check_every >= 0).
int check_krylov(const dbi_krylov_opts *o);

// Restarted GMRES(m) (gmres.cu) on the operator `op` (2D or 3D): the basis and the cycle state are
// carved from `ar`; field_bytes = bytes of one field of the whole batch (256-aligned).
constexpr int kGmresMaxRestart = 64;
size_t gmres_bytes_fields(size_t field_bytes, int B, int m);
int run_gmres(const OpArgs &op, Arena &ar, size_t field_bytes, int m, const void *rhs, void *x, bool x_zero,
              const dbi_krylov_opts &o, const dbi_status *status, cudaStream_t s);

// plist = the problems b < B with active[b] != 0 in ascending order, *count = how many (device).
int compact_active(int B, const int *active, int *plist, int *count, cudaStream_t s);

// use_graph (uneven batches only): the iterations between two host checks are captured once as
// a CUDA graph and replayed.
int run_bicgstab(OpArgs op, const SolverBufs &sb, const void *rhs, void *x, bool x_zero,
                 const dbi_krylov_opts &opts, const dbi_status *status, cudaStream_t s, bool unscale,
                 bool use_graph = false);

}  // namespace dbi
