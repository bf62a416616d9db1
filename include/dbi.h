/*
 * dbi.h -- C ABI of the GB300 library for the 2D elastic Lippmann-Schwinger (LS) operator and
 * the matrix-free distorted-Born (DBI) products of Xiang, Jakobsen, Shekhar, Eikrem and Naevdal,
 * "Efficient scattering approach to seismic full-waveform inversion in anisotropic elastic media
 * with variable density" (arXiv 2402.02116).
 *
 * Discrete problem (2D P-SV, x1 horizontal, x3 depth, Voigt indices {1, 3, 5}):
 *   grid D of nz x nx square cells of size h, cell (iz, ix) centred at (x1, x3) = (ix h, iz h);
 *   reference medium homogeneous isotropic (rho0, alpha0, beta0) (Eq. 4);
 *   model per cell (rho, C11, C13, C33, C55) (the VTI stiffness of Eq. 39 restricted to 2D);
 *   A u = u - h^2 sum_{x' in D} G_h(x - x') s(x'),  s = w^2 drho u + div(dC : eps(u))   (Eq. 6, 10)
 *   with central differences (fields zero outside D) for eps and div, G_h the closed-form Green's
 *   tensor of Appendix A (Eq. A-3, A-4) at cell-centre offsets and its disk average on the self
 *   cell, and the convolution done by FFT on an lz x lx zero-padded grid (Eq. 12).
 *
 * Conventions shared by every call
 *   - Pointers marked "device" are CUDA device pointers owned by the caller; the library never
 *     allocates, frees or keeps them. Scratch memory comes from the caller's `work` buffer of
 *     `work_bytes` bytes, sized by dbi_workspace_bytes(). A call may use all of it.
 *   - Complex arrays hold interleaved (re, im) pairs: float2 for DBI_C64, double2 for DBI_C128.
 *     Real model-space arrays (m, dm, g) are float for DBI_C64 and double for DBI_C128.
 *   - Complex arrays and the work buffer must start on a 16-byte boundary (cudaMalloc gives 256):
 *     the kernels move complex64 values in 16-byte pairs and Green's tables by 16-byte loads and
 *     copies. The library does not check this; a misaligned start is a device fault.
 *   - Wavefields are C-contiguous [B][2][nz][nx] (component 0 = u1, 1 = u3); receiver data are
 *     [B][n_rec][2]; model-space arrays are [5][nz][nx] in the order rho, C11, C13, C33, C55.
 *   - Problem b has angular frequency omega[fidx[b]] and uses Green's table fidx[b].
 *   - Calls are asynchronous on `stream` unless stated otherwise; inputs must stay valid until the
 *     work completes. Calls that overlap on the GPU must not share output or work buffers.
 *   - Every call returns 0 (DBI_OK) or a negative dbi_code; it then records a message that
 *     dbi_last_error() returns (per host thread). Per-problem numerical outcomes (convergence,
 *     breakdown) are reported in dbi_status arrays, not in the return code.
 */
#ifndef DBI_H
#define DBI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *dbi_stream; /* a cudaStream_t; NULL is the legacy default stream */

enum dbi_precision { DBI_C64 = 0, DBI_C128 = 1 };

enum dbi_code {
  DBI_OK = 0,
  DBI_ERR_ARG = -1,         /* a null pointer, a non-positive size, an index out of range */
  DBI_ERR_UNSUPPORTED = -2, /* an FFT length or precision this build does not provide */
  DBI_ERR_WORKSPACE = -3,   /* work_bytes smaller than dbi_workspace_bytes() */
  DBI_ERR_CUDA = -4         /* a CUDA launch or copy failed; the message names it */
};

/* Per-problem outcome of a Krylov solve. DBI_BREAKDOWN: the last BiCGSTAB step broke down and the
 * problem restarted from its iterate (a later step overwrites it). DBI_NONFINITE: a NaN or an
 * infinity appeared in the right-hand side, the model or an inner product; the problem stopped at
 * once (its iterate is not meaningful). */
enum dbi_problem_code { DBI_CONVERGED = 0, DBI_NOT_CONVERGED = 1, DBI_BREAKDOWN = 2, DBI_NONFINITE = 3 };

enum dbi_op {
  DBI_OP_GREENS = 0,
  DBI_OP_CONVOLVE = 1,
  DBI_OP_APPLY = 2,
  DBI_OP_SOLVE = 3,
  DBI_OP_FRECHET = 4,
  DBI_OP_ADJOINT = 5,
  DBI_OP_NORMAL_CG = 6,
  DBI_OP_GREENS_K = 7, /* greens_tabulate_k (B counts frequencies) */
  DBI_OP_APPLY_K = 8,  /* ls_apply_k */
  DBI_OP_SOLVE_K = 9   /* ls_solve_k */
};

typedef struct dbi_grid {
  int nz, nx; /* cells of the domain D (rows: depth x3; columns: x1) */
  int lz, lx; /* FFT grid; lz >= 2 nz - 1, lx >= 2 nx - 1, each a power of two in [16, 1024]; with
               * complex64, 768 is also taken (3 x 256: Eq. 12 holds for any lengths >= 2n - 1) by
               * the Green's tables, the incident field, the operator and everything built on it
               * (not by the paper-literal form K entry points, which return DBI_ERR_UNSUPPORTED) */
  double h;   /* cell size in metres */
} dbi_grid;

typedef struct dbi_medium {
  double rho0, alpha0, beta0; /* homogeneous isotropic reference (kg/m^3, m/s, m/s) */
  /* homogeneous VTI reference stiffness (Pa), used instead of alpha0, beta0 when c11 > 0 (an
   * extension: the paper's reference is isotropic); all zero for an isotropic reference */
  double c11, c13, c33, c55;
} dbi_medium;

typedef struct dbi_model {
  dbi_grid grid;
  dbi_medium ref;
  const void *m; /* device [5][nz][nx] real: absolute rho, C11, C13, C33, C55 of each cell */
} dbi_model;

typedef struct dbi_batch {
  int B;               /* number of (source, frequency) problems */
  int nf;              /* number of frequencies in the Green's tables */
  const double *omega; /* device [nf] angular frequencies (rad/s) */
  const int *fidx;     /* device [B] frequency index of every problem, in [0, nf) */
} dbi_batch;

typedef struct dbi_receivers {
  int n;            /* number of receivers */
  const int *cells; /* device [n][2] (iz, ix) receiver cells */
} dbi_receivers;

typedef struct dbi_krylov_opts {
  double tol;      /* stop problem b when ||rhs - A u|| / ||rhs|| <= tol (recursive residual) */
  int max_iter;    /* BiCGSTAB iterations per problem at most (two operator applies each) */
  int check_every; /* host checks for "all converged" every this many iterations (a stream
                      synchronisation each time); 0 runs max_iter iterations without checking */
  int zero_guess;  /* ls_solve only: 1 = start from u = 0 without reading u (saves one operator
                      pass); 0 = u holds the initial guess */
} dbi_krylov_opts;

typedef struct dbi_status { /* device arrays of length B; each pointer may be NULL */
  int *iters;               /* BiCGSTAB iterations taken */
  double *relres;           /* final recursive relative residual */
  int *code;                /* dbi_problem_code */
} dbi_status;

typedef struct dbi_cg_opts {
  int iters;          /* CG iterations on the normal equation */
  double lambda;      /* Tikhonov weight (> 0), or <= 0 to use lambda_rel * lambda_max */
  double lambda_rel;  /* multiple of the power-iteration estimate of lambda_max(Re J~^H J~) */
  int power_iters;    /* power iterations for the estimate */
} dbi_cg_opts;

/* Message of the last failing call on this host thread ("" if none). */
const char *dbi_last_error(void);

/* Library version (major * 10000 + minor * 100 + patch). */
int dbi_version(void);

/* Bytes of `work` that call `op` needs for B problems on grid g in `precision`; 0 if the grid or
 * precision is invalid. */
size_t dbi_workspace_bytes(const dbi_grid *g, int B, int precision, int op);

/*
 * greens_tabulate -- Green's tensor tables for nf frequencies (Appendix A, Eq. A-3, A-4; Eq. 12).
 *   Evaluates G_h in FP64 at every cell-centre offset y = (dx h, dz h), |dz| < nz, |dx| < nx
 *   (the self cell gets the disk average of radius h / sqrt(pi)), places offset d at slot d mod L of
 *   the lz x lx grid (other slots 0), and takes the FP64 2D FFT.
 *   omega  device [nf] angular frequencies.
 *   Ghat   device [nf][3][lx][lz] complex out: h^2 / (lz lx) * FFT(G) for components 11, 13, 33,
 *          stored column-major: entry [f][c][kx][kz] holds wavenumber (kz, kx). At lz = 768 the kz
 *          entries of a column are residue-major: entry [f][c][kx][(kz mod 3) 256 + kz / 3] holds
 *          wavenumber (kz, kx), the order in which the length-768 column stage reads them.
 *   Gspace device [nf][3][lz][lx] complex out (may be NULL): the spatial G_h on the same slots.
 *   Work: DBI_OP_GREENS bytes.
 */
int greens_tabulate(const dbi_grid *g, const dbi_medium *ref, const double *omega, int nf,
                    int precision, void *Ghat, void *Gspace, void *work, size_t work_bytes,
                    dbi_stream stream);

/*
 * incident_field -- u0(x) = G_h(x - x_s) f for a point force f at cell x_s (Eq. 7).
 *   Gspace    device [nf][3][lz][lx] spatial table from greens_tabulate.
 *   src_cells device [B][2] (iz, ix) source cell of every problem.
 *   forces    device [B][2] double (f1, f3) force of every problem.
 *   u0        device [B][2][nz][nx] complex out.
 */
int incident_field(const dbi_grid *g, const dbi_batch *batch, const void *Gspace,
                   const int *src_cells, const double *forces, void *u0, int precision,
                   dbi_stream stream);

/*
 * green_convolve -- out = h^2 sum_{x' in D} G_h(x - x') src(x') for every problem (the integrals
 *   of Eq. 6 / Eq. 31 / Eq. 35 evaluated by Eq. 12). src, out: device [B][2][nz][nx] complex
 *   (distinct buffers). Work: DBI_OP_CONVOLVE bytes.
 */
int green_convolve(const dbi_grid *g, const dbi_batch *batch, const void *Ghat, const void *src,
                   void *out, int precision, void *work, size_t work_bytes, dbi_stream stream);

/*
 * ls_apply -- out = A u = u - h^2 G * (w^2 drho u + div(dC : eps(u))) for every problem (Eq. 10),
 *   with drho, dC = model - reference (Eq. 4). u, out: device [B][2][nz][nx] complex (distinct).
 *   Work: DBI_OP_APPLY bytes.
 */
int ls_apply(const dbi_model *model, const dbi_batch *batch, const void *Ghat, const void *u,
             void *out, int precision, void *work, size_t work_bytes, dbi_stream stream);

/*
 * ls_solve -- solves A u = rhs (Eq. 11) for every problem by BiCGSTAB (the paper's Krylov
 *   forward solver), complex inner product sum conj(a) b, shadow residual = initial residual;
 *   vectors in the precision's complex type, inner products, norms and scalar recurrences in
 *   FP64. On breakdown (rho or omega zero) the problem restarts from its current iterate.
 *   rhs device [B][2][nz][nx] complex; u device same shape, in: initial guess, out: solution.
 *   Synchronises the stream every opts->check_every iterations. Work: DBI_OP_SOLVE bytes.
 */
int ls_solve(const dbi_model *model, const dbi_batch *batch, const void *Ghat, const void *rhs,
             void *u, const dbi_krylov_opts *opts, const dbi_status *status, int precision,
             void *work, size_t work_bytes, dbi_stream stream);

/*
 * dbi_gmres_workspace_bytes -- work-buffer size of ls_solve_gmres for B problems on grid g with
 *   restart length `restart` (1..64): the operator scratch plus restart + 1 basis vectors per
 *   problem. Returns 0 for invalid arguments.
 */
size_t dbi_gmres_workspace_bytes(const dbi_grid *g, int B, int precision, int restart);

/*
 * ls_solve_gmres -- solves A u = rhs (Eq. 11) for every problem by restarted GMRES(restart), the
 *   Krylov method of the paper's experiments: Arnoldi basis by classical Gram-Schmidt with one
 *   re-orthogonalisation, complex plane rotations on the Hessenberg matrix, minimal-residual
 *   iterate at the end of each cycle. Basis vectors in the precision's complex type; Hessenberg
 *   matrix, rotations, inner products and norms in FP64. A problem stops when the minimal
 *   residual of its cycle is <= opts->tol ||rhs||, when its new basis vector vanishes, or after
 *   opts->max_iter Arnoldi steps in all. rhs, u: device [B][2][nz][nx] complex (distinct); u holds
 *   the initial guess unless opts->zero_guess. status: iters = Arnoldi steps (operator passes
 *   inside the cycles), relres = the last minimal residual / ||rhs||, code. Synchronises the
 *   stream every opts->check_every steps and at every restart. Work: dbi_gmres_workspace_bytes.
 */
int ls_solve_gmres(const dbi_model *model, const dbi_batch *batch, const void *Ghat, const void *rhs,
                   void *u, const dbi_krylov_opts *opts, int restart, const dbi_status *status,
                   int precision, void *work, size_t work_bytes, dbi_stream stream);

/* ---------------------------------------------------------------------------------------------
 * 3D extension (the paper's 3D examples and Eq. A-1): fields [B][3][nz][ny][nx] complex
 * (u1, u2, u3 along x1, x2, x3; x3 the depth), models [6][nz][ny][nx] real
 * (rho, C11, C13, C33, C55, C66 of a VTI medium; C12 = C11 - 2 C66, C44 = C55), cubic cells of
 * side h, an isotropic reference. Tables [nf][6][lz][ly][lx] (components 11, 12, 13, 22, 23, 33).
 * ------------------------------------------------------------------------------------------- */
typedef struct dbi_grid3 {
  int nz, ny, nx; /* cells */
  int lz, ly, lx; /* FFT grid, powers of two in [16, 1024], each >= 2 n - 1 */
  double h;
} dbi_grid3;

typedef struct dbi_model3 {
  dbi_grid3 grid;
  dbi_medium ref; /* isotropic (rho0, alpha0, beta0) */
  const void *m;  /* device [6][nz][ny][nx] real of the precision */
} dbi_model3;

/* dbi_workspace_bytes_3d -- work-buffer size for op DBI_OP_GREENS (B = nf), DBI_OP_APPLY or
 * DBI_OP_SOLVE (GMRES with `restart`); 0 for invalid arguments. */
size_t dbi_workspace_bytes_3d(const dbi_grid3 *g, int B, int precision, int op, int restart);

/* greens_tabulate_3d -- the 3D isotropic Green's tensor (Eq. A-1, written for the exp(+i w t)
 * convention of the 2D tensor, i.e. its complex conjugate; outgoing exp(-i k r)) at the offsets
 * |d| < n, the self cell as the mean over the ball of volume h^3, FP64 3D FFT, scaled by
 * h^3 / (lz ly lx) into Ghat (natural [kz][ky][kx] order); Gspace (may be NULL) the spatial table. */
int greens_tabulate_3d(const dbi_grid3 *g, const dbi_medium *ref, const double *omega, int nf,
                       int precision, void *Ghat, void *Gspace, void *work, size_t work_bytes,
                       dbi_stream stream);

/* incident_field_3d -- u0(x) = G_h(x - x_s) f (Eq. 7 in 3D). src_cells device [B][3] (iz, iy, ix),
 * forces device [B][3] double (f1, f2, f3), u0 device [B][3][nz][ny][nx] out. */
int incident_field_3d(const dbi_grid3 *g, const dbi_batch *batch, const void *Gspace,
                      const int *src_cells, const double *forces, void *u0, int precision,
                      dbi_stream stream);

/* ls_apply_3d -- out = A u = u - h^3 G * (w^2 drho u + div(dC : eps(u))) in 3D (central
 * differences, fields zero outside the grid). Work: dbi_workspace_bytes_3d(..., DBI_OP_APPLY). */
int ls_apply_3d(const dbi_model3 *model, const dbi_batch *batch, const void *Ghat, const void *u,
                void *out, int precision, void *work, size_t work_bytes, dbi_stream stream);

/* dbi_products_workspace_bytes_3d -- work-buffer size of frechet_apply_3d / adjoint_apply_3d. */
size_t dbi_products_workspace_bytes_3d(const dbi_grid3 *g, int B, int precision, int restart);

/* frechet_apply_3d -- d = J dm in 3D (Eq. 20, 26-31): the virtual source
 * w^2 dm_rho u_b + div(dC(dm) : eps(u_b)) convolved with G, solved in the background by
 * GMRES(restart), sampled at the receivers. u_b device [B][3][nz][ny][nx]; rec_cells device
 * [n_rec][3] int (iz, iy, ix); dm device [6][nz][ny][nx] real of the precision; d device
 * [B][n_rec][3] complex out. */
int frechet_apply_3d(const dbi_model3 *background, const dbi_batch *batch, const void *Ghat,
                     const void *u_b, const int *rec_cells, int n_rec, const void *dm, void *d,
                     const dbi_krylov_opts *opts, int restart, const dbi_status *status, int precision,
                     void *work, size_t work_bytes, dbi_stream stream);

/* adjoint_apply_3d -- g = Re J^H r summed over the problems (Eq. 25, 32-35 in 3D): conj(r)
 * injected at the receivers, convolved with G, solved in the background, imaged against u_b:
 * g_rho = sum Re(w^2 u_a . u_b), g_p = -sum Re(eps(u_a)^T B_p eps(u_b)) with the derivatives B_p
 * of the 3D VTI stiffness (C11, C13, C33, C55, C66). r device [B][n_rec][3] complex; g device
 * [6][nz][ny][nx] real of the precision out (FP64 accumulation). */
int adjoint_apply_3d(const dbi_model3 *background, const dbi_batch *batch, const void *Ghat,
                     const void *u_b, const int *rec_cells, int n_rec, const void *r, void *g,
                     const dbi_krylov_opts *opts, int restart, const dbi_status *status, int precision,
                     void *work, size_t work_bytes, dbi_stream stream);

/* sample_3d -- d[b][r][c] = u[b][c] at receiver cell r (the sampling P of Eq. 27 in 3D); u device
 * [B][3][nz][ny][nx], rec_cells device [n_rec][3] int, d device [B][n_rec][3] complex out. */
int sample_3d(const dbi_grid3 *g, int B, const int *rec_cells, int n_rec, const void *u, void *d,
              int precision, dbi_stream stream);

/* dbi_normal_cg_workspace_bytes_3d -- work-buffer size of normal_cg_3d. */
size_t dbi_normal_cg_workspace_bytes_3d(const dbi_grid3 *g, int B, int precision, int restart, int n_rec,
                                        int iters);

/* normal_cg_3d -- the Tikhonov normal equation (Eq. 23, 24) in 3D, as normal_cg: CG on the
 * relative unknowns x_p = dm_p / s_p, s = (rho0, rho0 alpha0^2 for C11, C13 and C33,
 * rho0 beta0^2 for C55 and C66), (Re J~^H J~ + lambda I) x = Re J~^H dd from x = 0, every product
 * through frechet_apply_3d / adjoint_apply_3d (GMRES(restart) solves). dd device [B][n_rec][3];
 * power_start device [6][nz][ny][nx] real (when lambda is estimated); dm device [6][nz][ny][nx]
 * real out; lambda_out, hist_out (iters + 1 norms of the normal residual) host. */
int normal_cg_3d(const dbi_model3 *background, const dbi_batch *batch, const void *Ghat, const void *u_b,
                 const int *rec_cells, int n_rec, const void *dd, const dbi_cg_opts *cg,
                 const void *power_start, void *dm, double *lambda_out, double *hist_out,
                 const dbi_krylov_opts *opts, int restart, const dbi_status *status, int precision,
                 void *work, size_t work_bytes, dbi_stream stream);

/* ls_solve_3d -- A u = rhs in 3D by restarted GMRES(restart) (as ls_solve_gmres). */
int ls_solve_3d(const dbi_model3 *model, const dbi_batch *batch, const void *Ghat, const void *rhs,
                void *u, const dbi_krylov_opts *opts, int restart, const dbi_status *status,
                int precision, void *work, size_t work_bytes, dbi_stream stream);

/*
 * greens_tabulate_k -- the derivative tables of the paper-literal form of the LS equation (Eq. 9,
 *   the gradient acting on the Green's tensor instead of on the stress): central differences
 *   (D_k G)(y) = [G_h(y + h e_k) - G_h(y - h e_k)] / 2h of the same lattice G_h as greens_tabulate
 *   (self cell = disk average), at every offset |dz| < nz, |dx| < nx, placed at slot d mod L and
 *   transformed by the FP64 2D FFT. Six entries per frequency, the kernel entries of the stress
 *   components: e = D1G11, D1G13 (sigma11), D3G11 + D1G13, D3G13 + D1G33 (sigma13),
 *   D3G13, D3G33 (sigma33).
 *   omega device [nf]. Dhat device [nf][6][lx][lz] complex out, h^2 / (lz lx) * FFT, stored
 *   column-major like Ghat. Work: DBI_OP_GREENS_K bytes (B = nf).
 */
int greens_tabulate_k(const dbi_grid *g, const dbi_medium *ref, const double *omega, int nf,
                      int precision, void *Dhat, void *work, size_t work_bytes, dbi_stream stream);

/*
 * ls_apply_k -- out = u - h^2 [ G * (w^2 drho u) + sum_jk (D_k G_ij) * sigma_jk ], sigma = dC : eps(u)
 *   (Eq. 9 discretised with the quadrature of Eq. 10 and evaluated by Eq. 12), eps by central
 *   differences of u (zero outside D). Equals ls_apply exactly when dC vanishes on the outer ring
 *   of cells of D (summation by parts); otherwise the two differ by the convolution of G with the
 *   ring's boundary sources. Ghat from greens_tabulate, Dhat from greens_tabulate_k (same grid,
 *   medium, frequencies, precision). u, out: device [B][2][nz][nx] complex (distinct).
 *   Work: DBI_OP_APPLY_K bytes.
 */
int ls_apply_k(const dbi_model *model, const dbi_batch *batch, const void *Ghat, const void *Dhat,
               const void *u, void *out, int precision, void *work, size_t work_bytes, dbi_stream stream);

/*
 * ls_solve_k -- ls_solve with the operator of ls_apply_k (BiCGSTAB, same options, status and
 *   FP64 scalars). Work: DBI_OP_SOLVE_K bytes.
 */
int ls_solve_k(const dbi_model *model, const dbi_batch *batch, const void *Ghat, const void *Dhat,
               const void *rhs, void *u, const dbi_krylov_opts *opts, const dbi_status *status,
               int precision, void *work, size_t work_bytes, dbi_stream stream);

/*
 * frechet_apply -- d = J dm (Eq. 20, 26-31): the virtual source w^2 dm_rho u_b + div(dC(dm) :
 *   eps(u_b)) (Y and M of Eq. 26 in one field), convolved with G, solved in the background
 *   model (Eq. 30), sampled at the receivers (Eq. 27).
 *   background: model of the background (its drho, dC define A_b). u_b: device [B][2][nz][nx]
 *   background wavefields. dm: device [5][nz][nx] real perturbation. d: device [B][n_rec][2]
 *   complex out. Work: DBI_OP_FRECHET bytes.
 */
int frechet_apply(const dbi_model *background, const dbi_batch *batch, const void *Ghat,
                  const void *u_b, const dbi_receivers *rec, const void *dm, void *d,
                  const dbi_krylov_opts *opts, const dbi_status *status, int precision,
                  void *work, size_t work_bytes, dbi_stream stream);

/*
 * adjoint_apply -- g = Re J^H r summed over the problems (Eq. 25, 32-35): conj(r) injected at
 *   the receivers, convolved with G, solved in the background (Eq. 34), imaged against u_b:
 *   g_rho = sum Re(w^2 u_a . u_b), g_p = -sum Re(eps(u_a)^T B_p eps(u_b)) (Appendix C B matrices
 *   restricted to 2D). Accumulated in FP64. r: device [B][n_rec][2] complex. g: device
 *   [5][nz][nx] real out (overwritten). Work: DBI_OP_ADJOINT bytes.
 */
int adjoint_apply(const dbi_model *background, const dbi_batch *batch, const void *Ghat,
                  const void *u_b, const dbi_receivers *rec, const void *r, void *g,
                  const dbi_krylov_opts *opts, const dbi_status *status, int precision,
                  void *work, size_t work_bytes, dbi_stream stream);

/*
 * data_residual -- r = P u - d_obs at the receivers and phi = 1/2 sum |r|^2 (the L2 data misfit;
 *   Eq. 23 without the regularisation term). u: device [B][2][nz][nx]; d_obs, r: device
 *   [B][n_rec][2] complex; phi: device double[1] out (may be NULL).
 */
int data_residual(const dbi_grid *g, const dbi_batch *batch, const dbi_receivers *rec,
                  const void *u, const void *d_obs, void *r, double *phi, int precision,
                  dbi_stream stream);

/*
 * normal_cg -- Tikhonov-regularised normal equation (Eq. 23, 24) on relative unknowns
 *   x_p = dm_p / s_p (s = rho0, rho0 alpha0^2 for C11, C13, C33, rho0 beta0^2 for C55):
 *   (Re J~^H J~ + lambda I) x = Re J~^H dd, J~ = J diag(s), solved by cg->iters CG steps from
 *   x = 0 with FP64 vectors and scalars. If cg->lambda <= 0, lambda = cg->lambda_rel times the
 *   Rayleigh quotient after cg->power_iters power steps from `power_start` (device [5][nz][nx]
 *   real). dd: device [B][n_rec][2] complex data residual. dm: device [5][nz][nx] real out.
 *   lambda_out: host double (may be NULL). hist: host double[cg->iters + 1] (may be NULL) gets
 *   ||normal residual|| after each step. Synchronises the stream before returning.
 *   Work: DBI_OP_NORMAL_CG bytes.
 */
int normal_cg(const dbi_model *background, const dbi_batch *batch, const void *Ghat,
              const void *u_b, const dbi_receivers *rec, const void *dd,
              const dbi_cg_opts *cg, const void *power_start, void *dm, double *lambda_out,
              double *hist, const dbi_krylov_opts *opts, const dbi_status *status,
              int precision, void *work, size_t work_bytes, dbi_stream stream);

/*
 * ls_apply_noalloc -- the same operator pass as ls_apply (same kernels, same result) for callers
 *   that cannot pass a work buffer because they must not allocate device memory while running
 *   (a plugin whose host application owns all device allocations, a loop with a memory budget
 *   fixed at start-up). No counterpart in the paper: it only changes where the scratch lives.
 *   The scratch is one fixed device array inside this library of dbi_noalloc_scratch_bytes()
 *   bytes (32 MiB), held by every GPU that loads the library until the process exits. The call
 *   allocates and frees nothing. A batch whose DBI_OP_APPLY workspace exceeds the array is
 *   rejected with DBI_ERR_WORKSPACE before any GPU work. The first call on a device looks up the
 *   array's device address (once per device, with that device current); make that first call
 *   before any stream capture. All calls share the array, so calls that overlap on the GPU (other
 *   streams, other host threads) race and must be serialised by the caller; nothing in the array
 *   needs to start at zero (each call writes all the scratch it reads).
 */
int ls_apply_noalloc(const dbi_model *model, const dbi_batch *batch, const void *Ghat,
                     const void *u, void *out, int precision, dbi_stream stream);

/* Size in bytes of the fixed scratch array of ls_apply_noalloc. */
size_t dbi_noalloc_scratch_bytes(void);

/*
 * Diagnostics (no counterpart in the paper).
 *
 * dbi_kernel_launches -- number of kernels this library has launched in the process so far
 *   (host-side counter; the difference across a region counts the region's launches).
 * dbi_profile_begin -- start timing one stage of every LS-operator pass with CUDA events recorded
 *   on the launching stream: 1 = stencil + forward row FFTs, 2 = column FFTs with the Green's
 *   multiply, 3 = inverse row FFTs + epilogue, 4 = the whole three-kernel pass, 0 = off.
 *   Process-wide; a second begin restarts the count.
 * dbi_profile_end -- wait for the recorded events and return the summed duration (ms) and the
 *   number of timed launches since dbi_profile_begin; stops timing.
 */
unsigned long long dbi_kernel_launches(void);
int dbi_profile_begin(int stage);
int dbi_profile_end(double *total_ms, long long *launches);

/*
 * dbi_fma_probe -- launch `blocks` CTAs of 256 threads that issue nothing but FP32 fused
 *   multiply-adds (8 independent chains per thread, `iters` steps each) on `stream`, to measure
 *   the FP32 arithmetic peak that bounds the FFT-bound operator kernels (time it with events on the
 *   same stream). out: device float[blocks * 256], written (the chains' sums). Returns the number
 *   of floating-point operations launched (2 per FMA), or a negative dbi_code.
 */
long long dbi_fma_probe(int blocks, int iters, float *out, dbi_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* DBI_H */
