/* The library's C ABI used from plain C (no C++, no Python): the headers compile as C11 and the
 * host-side entry points answer as documented without a GPU. Prints one line per check; the exit
 * status is the number of failed checks. */
#include <stdio.h>
#include <string.h>

#include "dbi.h"
#include "dbi_group.h"

static int failed = 0;

static void check(int ok, const char *what) {
  printf("%s %s\n", ok ? "ok" : "FAIL", what);
  if (!ok) ++failed;
}

int main(void) {
  check(dbi_version() >= 100, "dbi_version");

  dbi_grid g = {32, 32, 64, 64, 10.0};
  const size_t apply64 = dbi_workspace_bytes(&g, 4, DBI_C64, DBI_OP_APPLY);
  const size_t apply128 = dbi_workspace_bytes(&g, 4, DBI_C128, DBI_OP_APPLY);
  check(apply64 >= (size_t)4 * 2 * 32 * 64 * 8, "workspace of an apply holds the spectra");
  check(apply128 > apply64, "complex128 needs more workspace");

  dbi_grid bad = {32, 32, 48, 64, 10.0};  /* 48 is not a supported FFT length */
  check(dbi_workspace_bytes(&bad, 4, DBI_C64, DBI_OP_APPLY) == 0, "unsupported FFT length gives 0");

  dbi_medium ref;
  memset(&ref, 0, sizeof ref);
  ref.rho0 = 2000.0;
  ref.alpha0 = 2000.0;
  ref.beta0 = 1155.0;
  const int rc = greens_tabulate(NULL, &ref, NULL, 1, DBI_C64, NULL, NULL, NULL, 0, NULL);
  check(rc == DBI_ERR_ARG, "NULL grid is an argument error");
  check(strstr(dbi_last_error(), "NULL") != NULL, "dbi_last_error names the NULL argument");

  dbi_grid3 g3 = {4, 3, 5, 16, 16, 16, 10.0};
  check(dbi_workspace_bytes_3d(&g3, 2, DBI_C64, DBI_OP_APPLY, 1) > 0, "3D workspace query");
  return failed;
}
