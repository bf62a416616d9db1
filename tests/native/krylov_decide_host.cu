// Host-side test of the BiCGSTAB end-of-iteration decision of the CUDA library (bicgstab_decide,
// compiled here for the CPU from the library's own header): every branch -- non-finite values,
// convergence, the iteration limit, the two breakdowns and their restart, and beta -- on crafted
// inner products, against std::complex arithmetic.
#include <cmath>
#include <complex>
#include <cstdio>
#include <limits>

#include "../../paper_2402_02116_gb300/csrc/krylov.cuh"

static int fails = 0;
#define EXPECT(c)                                                   \
  do {                                                              \
    if (!(c)) {                                                     \
      std::fprintf(stderr, "line %d: expected %s\n", __LINE__, #c); \
      ++fails;                                                      \
    }                                                               \
  } while (0)

static dbi::KState fresh() {
  dbi::KState k{};
  k.bnorm2 = 4.0;
  k.rho_re = 0.5; k.rho_im = -0.25;
  k.alpha_re = 0.7; k.alpha_im = 0.1;
  k.om_re = 0.9; k.om_im = -0.3;
  k.rhatnorm2 = 2.0;
  k.iters = 3;
  return k;
}

int main() {
  using dbi::bicgstab_decide;
  const double tol = 1e-6, nan = std::numeric_limits<double>::quiet_NaN();
  const double inf = std::numeric_limits<double>::infinity();
  {  // an ordinary step: beta = (rho_new / rho) (alpha / omega), rho := rho_new
    dbi::KState k = fresh();
    const double q[3] = {0.3, 0.2, 1.0};
    EXPECT(bicgstab_decide(k, q, tol, 100) == 1);
    const std::complex<double> beta = (std::complex<double>(0.3, 0.2) / std::complex<double>(0.5, -0.25)) *
                                      (std::complex<double>(0.7, 0.1) / std::complex<double>(0.9, -0.3));
    EXPECT(std::abs(std::complex<double>(k.beta_re, k.beta_im) - beta) < 1e-15 * std::abs(beta));
    EXPECT(k.rho_re == 0.3 && k.rho_im == 0.2 && k.code == DBI_NOT_CONVERGED && k.iters == 4 && !k.restart);
    EXPECT(k.rnorm2 == 1.0);
  }
  {  // converged on the residual, and on the half step
    dbi::KState k = fresh();
    const double q[3] = {0.0, 0.0, 4.0 * tol * tol};
    EXPECT(bicgstab_decide(k, q, tol, 100) == 0 && k.code == DBI_CONVERGED);
    dbi::KState h = fresh();
    h.half = 1;
    const double q2[3] = {0.3, 0.2, 1.0};
    EXPECT(bicgstab_decide(h, q2, tol, 100) == 0 && h.code == DBI_CONVERGED);
  }
  {  // the iteration limit
    dbi::KState k = fresh();
    const double q[3] = {0.3, 0.2, 1.0};
    EXPECT(bicgstab_decide(k, q, tol, 4) == 0 && k.code == DBI_NOT_CONVERGED && k.iters == 4);
  }
  {  // breakdown: omega = 0 restarts with rhat := r
    dbi::KState k = fresh();
    k.om_re = 0.0; k.om_im = 0.0;
    const double q[3] = {0.3, 0.2, 1.5};
    EXPECT(bicgstab_decide(k, q, tol, 100) == 1);
    EXPECT(k.restart == 1 && k.restarts == 1 && k.code == DBI_BREAKDOWN);
    EXPECT(k.rho_re == 1.5 && k.rho_im == 0.0 && k.rhatnorm2 == 1.5);
    EXPECT(k.alpha_re == 1.0 && k.om_re == 1.0 && k.beta_re == 0.0 && k.beta_im == 0.0);
  }
  {  // breakdown: <rhat, r> negligible against ||rhat|| ||r||; then an ordinary step clears restart
    dbi::KState k = fresh();
    const double q[3] = {1e-16, -1e-16, 1.0};
    EXPECT(bicgstab_decide(k, q, tol, 100) == 1 && k.restart == 1 && k.code == DBI_BREAKDOWN);
    const double q2[3] = {0.4, 0.0, 0.8};
    EXPECT(bicgstab_decide(k, q2, tol, 100) == 1 && k.restart == 0 && k.restarts == 1);
    EXPECT(k.code == DBI_NOT_CONVERGED);
  }
  {  // non-finite values stop the problem before any other test (even a met half step)
    const double cases[4][3] = {{nan, 0.0, 1.0}, {0.0, nan, 1.0}, {0.1, 0.1, nan}, {0.1, 0.1, inf}};
    for (const auto &q : cases) {
      dbi::KState k = fresh();
      k.half = 1;
      EXPECT(bicgstab_decide(k, q, tol, 100) == 0 && k.code == DBI_NONFINITE);
    }
    dbi::KState k = fresh();
    k.om_re = inf;
    const double q[3] = {0.3, 0.2, 1.0};
    EXPECT(bicgstab_decide(k, q, tol, 100) == 0 && k.code == DBI_NONFINITE);
    dbi::KState a = fresh();
    a.alpha_im = nan;
    EXPECT(bicgstab_decide(a, q, tol, 100) == 0 && a.code == DBI_NONFINITE);
  }
  if (fails) return 1;
  std::puts("decide ok");
  return 0;
}
