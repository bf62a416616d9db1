// Error reporting, argument validation, twiddle tables and workspace sizes.
#include <atomic>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "krylov.cuh"

namespace dbi {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

int cuda_fail(const char *what, cudaError_t e) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return DBI_ERR_CUDA;
}

static std::atomic<unsigned long long> g_launches{0};

unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
void add_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int check_launch(const char *what) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DBI_OK : cuda_fail(what, e);
}

// Stage profiler: event pairs recorded around every launch of the selected stage.
struct Profiler {
  std::mutex mu;
  int stage = PROF_NONE;
  std::vector<cudaEvent_t> ev;  // begin, end, begin, end, ...
  size_t used = 0;
};
static Profiler g_prof;

void prof_mark(int stage, bool after, cudaStream_t s) {
  if (g_prof.stage == PROF_NONE || g_prof.stage != stage) return;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  if (g_prof.used == g_prof.ev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    g_prof.ev.push_back(e);
  }
  // an end mark only pairs with a begin mark
  if (after != (g_prof.used % 2 == 1)) return;
  cudaEventRecord(g_prof.ev[g_prof.used++], s);
}

cudaError_t allow_dynamic_smem(const void *kernel, size_t bytes) {
  constexpr size_t kStaticReserve = 4096;  // static shared arrays of the reductions
  if (bytes + kStaticReserve <= 48 * 1024) return cudaSuccess;
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, size_t> raised;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t &have = raised[{kernel, dev}];
  if (have >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (e == cudaSuccess) have = bytes;
  return e;
}

static int check_grid_impl(const dbi_grid *g, bool allow768, bool mention768) {
  if (!g) { set_error("grid is NULL"); return DBI_ERR_ARG; }
  if (g->nz < 1 || g->nx < 1 || !(g->h > 0)) {
    set_error("grid needs nz, nx >= 1 and h > 0 (got %d, %d, %g)", g->nz, g->nx, g->h);
    return DBI_ERR_ARG;
  }
  auto ok = [&](int L) { return fft_len_ok(L) || (allow768 && L == 768); };
  if (!ok(g->lz) || !ok(g->lx)) {
    set_error("FFT grid %d x %d: each side must be a power of two in [16, 1024]%s", g->lz, g->lx,
              mention768 ? " (or 768 with complex64)" : "");
    return DBI_ERR_UNSUPPORTED;
  }
  if (g->lz < 2 * g->nz - 1 || g->lx < 2 * g->nx - 1) {
    set_error("FFT grid %d x %d too small for %d x %d cells (need >= 2n - 1)", g->lz, g->lx, g->nz, g->nx);
    return DBI_ERR_ARG;
  }
  return DBI_OK;
}

int check_grid(const dbi_grid *g) { return check_grid_impl(g, false, false); }
int check_grid(const dbi_grid *g, int precision) { return check_grid_impl(g, precision == DBI_C64, true); }

int check_batch(const dbi_batch *b) {
  if (!b) { set_error("batch is NULL"); return DBI_ERR_ARG; }
  if (b->B < 0 || b->nf < 1 || !b->omega || (b->B > 0 && !b->fidx)) {
    set_error("batch needs B >= 0, nf >= 1 and device omega / fidx arrays");
    return DBI_ERR_ARG;
  }
  return DBI_OK;
}

int check_precision(int precision) {
  if (precision != DBI_C64 && precision != DBI_C128) {
    set_error("precision must be DBI_C64 (0) or DBI_C128 (1), got %d", precision);
    return DBI_ERR_UNSUPPORTED;
  }
  return DBI_OK;
}

// W_3072^m = exp(-2 pi i m / 3072) for m < 3072, then W_1024^j for j = m - 3072 < 1024, evaluated
// in FP64 with sincospi and rounded to the precision (W_1024^j has the argument of W_3072^{3j}
// exactly, so the two tables agree bit for bit).
template <typename C>
__global__ void twiddle_kernel(C *tw) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= kTwiddleTotal) return;
  double s, c;
  if (m < kTwiddleN) sincospi(-2.0 * double(m) / double(kTwiddleN), &s, &c);
  else sincospi(-2.0 * double(m - kTw1024) / 1024.0, &s, &c);
  tw[m] = mk<C>(c, s);
}

int launch_twiddles(void *tw, int precision, cudaStream_t s) {
  const int threads = 256, blocks = (kTwiddleTotal + threads - 1) / threads;
  if (precision == DBI_C64) twiddle_kernel<float2><<<blocks, threads, 0, s>>>(static_cast<float2 *>(tw));
  else twiddle_kernel<double2><<<blocks, threads, 0, s>>>(static_cast<double2 *>(tw));
  return check_launch("twiddle_kernel");
}

static size_t csize(int precision) { return precision == DBI_C64 ? sizeof(float2) : sizeof(double2); }

size_t bytes_twiddles(int precision) { return align256(size_t(kTwiddleTotal) * csize(precision)); }

int spectral_chunk(const dbi_grid *g, int B, int precision) {
  // Default: the whole batch in one pass (measured faster on the 256-problem benchmark batch than
  // L2-sized chunks: the column pass is bound by shared memory, not by HBM, and small launches
  // lose to wave tails). DBI_SPECTRAL_CHUNK_MB bounds the spectral scratch per pass.
  static const size_t budget = [] {
    const char *e = getenv("DBI_SPECTRAL_CHUNK_MB");
    const long mb = e ? atol(e) : 0;
    return mb > 0 ? size_t(mb) << 20 : ~size_t(0);
  }();
  const size_t per = size_t(2) * g->nz * g->lx * csize(precision);
  size_t c = budget / per;
  if (c < 1) c = 1;
  if (c > size_t(B)) c = size_t(B);
  return int(c);
}

size_t bytes_spectral(const dbi_grid *g, int B, int precision) {
  const size_t chunk = size_t(spectral_chunk(g, B, precision));
  const size_t src = split_rows(g->lx, precision) ? chunk * 2 * g->nz * g->nx * csize(precision) : 0;
  return align256(chunk * 2 * g->nz * g->lx * csize(precision) + src);
}

size_t bytes_field(const dbi_grid *g, int B, int precision) {
  return align256(size_t(B) * 2 * g->nz * g->nx * csize(precision));
}

size_t bytes_partials(int B) {
  return align256(size_t(B) * kMaxParts * kRedSlots * sizeof(double));
}

size_t bytes_scales(int B) { return 3 * align256(size_t(B) * sizeof(double)) + 256 + bytes_partials(B); }

int imaging_chunks(int B) { return B < 16 ? (B > 0 ? B : 1) : 16; }

}  // namespace dbi

using namespace dbi;

namespace dbi {
int Arena::check(const char *who) const {
  if (!overflow) return DBI_OK;
  set_error("%s: the work buffer of %zu bytes is too small for the buffers carved from it", who, cap);
  return DBI_ERR_WORKSPACE;
}
}  // namespace dbi

extern "C" const char *dbi_last_error(void) { return g_err; }

extern "C" int dbi_version(void) { return 100; }

extern "C" unsigned long long dbi_kernel_launches(void) { return g_launches.load(); }

extern "C" int dbi_profile_begin(int stage) {
  clear_error();
  if (stage < PROF_NONE || stage > PROF_OPERATOR) {
    set_error("profile stage must be 0..4, got %d", stage);
    return DBI_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.stage = stage;
  g_prof.used = 0;
  return DBI_OK;
}

extern "C" int dbi_profile_end(double *total_ms, long long *launches) {
  clear_error();
  std::lock_guard<std::mutex> lk(g_prof.mu);
  double total = 0.0;
  const size_t pairs = g_prof.used / 2;
  for (size_t i = 0; i < pairs; ++i) {
    cudaError_t e = cudaEventSynchronize(g_prof.ev[2 * i + 1]);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, g_prof.ev[2 * i], g_prof.ev[2 * i + 1]);
    if (e != cudaSuccess) return cuda_fail("dbi_profile_end", e);
    total += ms;
  }
  if (total_ms) *total_ms = total;
  if (launches) *launches = (long long)pairs;
  g_prof.stage = PROF_NONE;
  g_prof.used = 0;
  return DBI_OK;
}

extern "C" size_t dbi_workspace_bytes(const dbi_grid *g, int B, int precision, int op) {
  if (check_grid(g, precision) != DBI_OK || check_precision(precision) != DBI_OK || B < 0) return 0;
  const size_t tw = bytes_twiddles(precision);
  const size_t spec = bytes_spectral(g, B, precision);
  const size_t fld = bytes_field(g, B, precision);
  const size_t solve = tw + spec + bytes_solver(g, B, precision);
  const size_t model = align256(size_t(5) * g->nz * g->nx * sizeof(double));
  switch (op) {
    case DBI_OP_GREENS:  // B counts frequencies here
      return bytes_twiddles(DBI_C128) +
             align256(size_t(B) * 3 * g->lz * g->lx * sizeof(double2));
    case DBI_OP_CONVOLVE:
    case DBI_OP_APPLY:
      return tw + spec + bytes_scales(B);
    case DBI_OP_SOLVE:
      return solve;
    case DBI_OP_FRECHET:
    case DBI_OP_ADJOINT:
      return solve + 2 * fld + model + bytes_scales(B) + imaging_chunks(B) * model;
    case DBI_OP_NORMAL_CG: {
      // receivers are cells: n_rec <= nz * nx
      const size_t data = align256(size_t(B) * g->nz * g->nx * 2 * csize(precision));
      return solve + 2 * fld + 6 * model + data + bytes_partials(1) + 256 + bytes_scales(B) +
             imaging_chunks(B) * model +
             align256(4097 * sizeof(double));
    }
    case DBI_OP_GREENS_K:  // B counts frequencies here
      return bytes_twiddles(DBI_C128) +
             align256(size_t(B) * 6 * g->lz * g->lx * sizeof(double2));
    case DBI_OP_APPLY_K:  // spectra of the five sources and of the two outputs
      return tw + bytes_spectral_k(g, B, precision) + bytes_scales(B);
    case DBI_OP_SOLVE_K:
      return tw + bytes_spectral_k(g, B, precision) + bytes_solver(g, B, precision);
    default:
      return 0;
  }
}
