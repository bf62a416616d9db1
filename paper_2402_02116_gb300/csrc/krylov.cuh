// Internal interface of the batched BiCGSTAB solver.
#pragma once

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
  int zero_rhs, pad[3];
};

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
