// Tuned run-time choices of the operator kernels.
#include <atomic>

#include "common.cuh"
#include "tune.cuh"

namespace dbi {

namespace {
std::atomic<int> g_plan[2][11];  // [precision][log2 L]
int log2_len(int L) {
  int k = 0;
  while ((1 << k) < L && k < 10) ++k;
  return k;
}
}  // namespace

int radix_plan(int precision, int L) {
  if ((precision != DBI_C64 && precision != DBI_C128) || !fft_len_ok(L)) return 0;
  return g_plan[precision][log2_len(L)].load(std::memory_order_relaxed);
}

void set_radix_plan(int precision, int L, int plan) {
  if ((precision != DBI_C64 && precision != DBI_C128) || !fft_len_ok(L)) return;
  g_plan[precision][log2_len(L)].store(plan ? 1 : 0, std::memory_order_relaxed);
}

}  // namespace dbi
