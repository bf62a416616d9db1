// Internal interface of the LS operator pipeline (Eq. 6, 10, 12) shared by the library's TUs.
#pragma once

#include "common.cuh"

namespace dbi {

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
  double ref[5];        // subtracted from m per cell (the reference medium, or zeros)
  bool stencil;
  const void *in;       // device [B][2][nz][nx] complex
  const void *ident;    // device [B][2][nz][nx] complex or NULL
  void *out;            // device [B][2][nz][nx] complex
  void *T;              // device [B][2][nz][lx] complex scratch
  const void *Ghat;     // device [nf][3][lz][lx] complex
  const void *tw;       // device twiddle table of the precision
  const int *active;    // device [B] (0 = skip the problem) or NULL
};

int run_operator(const OpArgs &a, cudaStream_t s);

// Reference values (rho, C11, C13, C33, C55) of the isotropic medium (Eq. 4, Eq. 39).
inline void reference_values(const dbi_medium &r, double out[5]) {
  const double a2 = r.alpha0 * r.alpha0, b2 = r.beta0 * r.beta0;
  out[0] = r.rho0;
  out[1] = r.rho0 * a2;
  out[2] = r.rho0 * (a2 - 2.0 * b2);
  out[3] = r.rho0 * a2;
  out[4] = r.rho0 * b2;
}

}  // namespace dbi
