// Internal interface of the LS operator pipeline (Eq. 6, 10, 12) shared by the library's TUs.
#pragma once

#include "common.cuh"

namespace dbi {

// Per-problem extent of a batched array: problem b holds elements [offset(b), offset(b) +
// count(b)). A batch on one grid has n elements per problem; an uneven batch passes prefix
// offsets offs[B + 1] (device memory).
struct Span {
  size_t n;
  const long long *offs;
  __host__ __device__ __forceinline__ size_t offset(int b) const { return offs ? size_t(offs[b]) : size_t(b) * n; }
  __host__ __device__ __forceinline__ size_t count(int b) const {
    return offs ? size_t(offs[b + 1] - offs[b]) : n;
  }
};

struct GroupLaunch;  // launch description of an uneven batch (group.cuh)

// One batched pass  out = ident - K(src)  or  out = K(src), where K(src) = h^2 G * src and src
// is either the contrast source w^2 drho u + div(dC : eps(u)) of `in` (stencil = true) or `in`
// itself (stencil = false).
struct OpArgs {
  int precision;
  int nz, nx, lz, lx;
  double h;
  int B;
  int nf;               // frequencies in the tables
  const double *omega;  // device [nf]
  const int *fidx;      // device [B]
  const void *m;        // device [5][nz][nx] real (stencil mode): model or perturbation
  double ref[6];        // subtracted from m per cell (the reference medium, or zeros; [5]: C66 in 3D)
  bool stencil;
  const void *in;       // device [B][2][nz][nx] complex
  const void *ident;    // device [B][2][nz][nx] complex or NULL
  void *out;            // device [B][2][nz][nx] complex
  void *T;              // device [B][2][lx][nz] complex scratch (column-major spectra)
  const void *Ghat;     // device [nf][3][lx][lz] complex (column-major)
  const void *Dhat;     // device [nf][6][lx][lz] derivative tables: the paper-literal form (Eq. 9)
                        // replaces the stencil pass (form_k.cu; T then holds [B][7][lx][nz])
  const void *tw;       // device twiddle table of the precision
  const int *active;    // device [B] (0 = skip the problem) or NULL
  const int *plist;     // device [nb]: the problems to run (launch slot -> problem), or NULL
  int nb;               // launch slots (problems run); B when plist is NULL
  // Exact power-of-two scalings that keep FP32 intermediates in range (each may be NULL):
  const double *in_scale;   // device [B]: the input field is multiplied by in_scale[b]
  const double *m_scale;    // device [1]: the contrast (m - ref) is multiplied by m_scale[0]
  const double *out_scale;  // device [B]: the convolution result is multiplied by out_scale[b]
  // Inner products fused into the last kernel's epilogue (krylov.cu); 0 / NULL for a plain pass.
  //   epi = 1: partials of <rhat, out> (rhat = krhat); epi = 2: partials of <out, ident>, <out, out>.
  //   part_out: [B][operator_parts][kRedSlots].
  int epi;
  const void *krhat;
  double *part_out;
  // Uneven batch: problems on different grids (nz, nx, lz, lx, m, Ghat, omega, ref above are then
  // unused and come from the group's member descriptors). offs: field offsets per problem.
  const GroupLaunch *group;
  const long long *offs;
  // 3D grids (ls3d.cu): ny > 0; fields [B][3][nz][ny][nx], m [6][nz][ny][nx]; T holds the spectra
  // [B][3][nz][ly][lx] and T2 the stress [B][6][nz][ny][nx]; Ghat [nf][6][lz][ly][lx].
  int ny, ly;
  void *T2;
};

// Partials per problem written by the operator kernels (one per CTA row block): the single-grid
// divergence form (operator_parts) and the paper-literal form (operator_parts_k, whose row stages
// keep 2048 / L rows per tile at every length).
int operator_parts(int nz, int lx, int precision);
int operator_parts_k(int nz, int lx, int precision);

int run_operator(const OpArgs &a, cudaStream_t s);
int run_form_k(const OpArgs &a, cudaStream_t s);
int run_operator_3d(const OpArgs &a, cudaStream_t s);

// Field elements per problem: 2 nz nx in 2D, 3 nz ny nx in 3D.
inline size_t field_elems(const OpArgs &a) {
  return a.ny > 0 ? size_t(3) * a.nz * a.ny * a.nx : size_t(2) * a.nz * a.nx;
}

// In-place FP64 FFTs of the Green's tables (greens.cu): nlines contiguous lines of length L, or
// the columns of nmat row-major [L][width] matrices.
int fft_rows_fp64(double2 *W, long nlines, int L, const double2 *tw, cudaStream_t s);
int fft_cols_fp64(double2 *W, int nmat, int L, int width, const double2 *tw, cudaStream_t s);

// Per-problem power-of-two normalisers of B arrays of n elements each (or of the extents offs
// gives, when non-NULL; complex of the precision, or real when `real` is set): scale[b] = 2^-e
// with max |x_b| (largest real or imaginary part) in [2^e, 2^(e+1)), 1 for a zero array. If inv is
// non-NULL, inv[b] = 1 / (scale[b] * (extra ? extra[0] : 1)). part: bytes_partials(B).
struct Scales {
  double *scale, *inv, *aux, *mscale, *part;
};
inline Scales carve_scales(Arena &ar, int B) {
  Scales s;
  s.scale = static_cast<double *>(ar.take(size_t(B) * sizeof(double)));
  s.inv = static_cast<double *>(ar.take(size_t(B) * sizeof(double)));
  s.aux = static_cast<double *>(ar.take(size_t(B) * sizeof(double)));
  s.mscale = static_cast<double *>(ar.take(256));
  s.part = static_cast<double *>(ar.take(bytes_partials(B)));
  return s;
}

// Green's tensor of a homogeneous VTI reference on the offsets |dz| < nz, |dx| < nx (greens_vti.cu):
// FP64 values at slot (dz mod lz, dx mod lx) of W [nf][3][lz][lx] (and of Gspace when non-NULL).
int launch_green_vti(const dbi_grid *g, const dbi_medium &ref, const double *omega, int nf, double2 *W,
                     void *Gspace, int precision, cudaStream_t s);

int pow2_scales(const void *x, int precision, bool real, int B, size_t n, double *part, double *scale,
                double *inv, const double *extra, cudaStream_t s, const long long *offs = nullptr);

// Reference values (rho, C11, C13, C33, C55) of the homogeneous reference medium (Eq. 4, Eq. 39):
// the VTI stiffness when given, else the isotropic one.
inline bool reference_is_vti(const dbi_medium &r) { return r.c11 > 0.0; }
inline void reference_values(const dbi_medium &r, double out[5]) {
  if (reference_is_vti(r)) {
    out[0] = r.rho0; out[1] = r.c11; out[2] = r.c13; out[3] = r.c33; out[4] = r.c55;
    return;
  }
  const double a2 = r.alpha0 * r.alpha0, b2 = r.beta0 * r.beta0;
  out[0] = r.rho0;
  out[1] = r.rho0 * a2;
  out[2] = r.rho0 * (a2 - 2.0 * b2);
  out[3] = r.rho0 * a2;
  out[4] = r.rho0 * b2;
}

}  // namespace dbi
