// Shared types, complex arithmetic and error reporting of the DBI library.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/dbi.h"

namespace dbi {

// ---------------------------------------------------------------------------------------------
// complex helpers on float2 / double2 (interleaved re, im)
// ---------------------------------------------------------------------------------------------
template <typename R> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };
template <typename C> struct RealOf;
template <> struct RealOf<float2> { using type = float; };
template <> struct RealOf<double2> { using type = double; };

template <typename C> __host__ __device__ __forceinline__ C mk(typename RealOf<C>::type re,
                                                                 typename RealOf<C>::type im) {
  C c; c.x = re; c.y = im; return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return mk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __device__ __forceinline__ C cscale(C a, typename RealOf<C>::type s) {
  return mk<C>(a.x * s, a.y * s);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
template <typename C, bool INV> __device__ __forceinline__ C mul_mi(C a) {
  return INV ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x);
}
template <typename C> __device__ __forceinline__ C czero() { return mk<C>(0, 0); }

// ---------------------------------------------------------------------------------------------
// sizes and launch helpers
// ---------------------------------------------------------------------------------------------
constexpr int kTwiddleN = 3072;  // W_3072^m covers every FFT length that divides 3072
// The twiddle buffer holds W_3072^m (m < 3072) and after it W_1024^j (j < 1024) contiguously, so
// that the length-1024 kernels' per-point twiddles W_1024^{t + 64 m} are coalesced loads (from
// the first table they are 24 bytes apart: three times the sectors).
constexpr int kTw1024 = kTwiddleN;
constexpr int kTwiddleTotal = kTwiddleN + 1024;

inline size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

inline bool fft_len_ok(int L) {
  return L >= 16 && L <= 1024 && (L & (L - 1)) == 0;
}

// Complex64 operator stages with FFT length 1024 along x (rows) or z (columns) run as pairs of
// 512-point transforms (op_split.cuh), and with length 768 as triples of 256-point transforms
// (op_split3.cuh); split_kind gives the number of sub-transforms (0: the ordinary stages). Split
// rows also need a contrast-source scratch field per problem of a chunk, after the chunk's spectra.
constexpr int kSplitPair = 2, kSplitTriple = 3;
inline int split_kind(int L, int precision) {
  if (precision != DBI_C64) return 0;
  return L == 1024 ? kSplitPair : L == 768 ? kSplitTriple : 0;
}
inline bool split_rows(int lx, int precision) { return split_kind(lx, precision) != 0; }
inline bool split_cols(int lz, int precision) { return split_kind(lz, precision) != 0; }

#ifdef __CUDACC__
// Asynchronous global-to-shared copies: 16 bytes (L2 only), 8 bytes with a zero fill of the
// destination when `valid` is false (nothing is read then), and the wait for all of a thread's
// copies (a barrier after it makes them visible to the other threads of the CTA).
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src, bool valid) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
#endif

// Error reporting (per host thread).
void set_error(const char *fmt, ...);
void clear_error();
int cuda_fail(const char *what, cudaError_t e);
// Checks the last launch and counts it (every kernel launch is followed by exactly one call).
int check_launch(const char *what);
// The launch count, and n more launches made by replaying a captured graph.
unsigned long long launch_count();
void add_launches(unsigned long long n);

// Event timing of one operator stage on its launching stream (see dbi_profile_begin).
enum { PROF_NONE = 0, PROF_ROWS_FORWARD = 1, PROF_COLS = 2, PROF_ROWS_INVERSE = 3, PROF_OPERATOR = 4 };
void prof_mark(int stage, bool after, cudaStream_t s);

// Lets `kernel` take `bytes` of dynamic shared memory on the current device: above 48 KB minus a
// reserve for the kernel's own static shared arrays, the kernel's limit is raised (once per kernel,
// device and size).
cudaError_t allow_dynamic_smem(const void *kernel, size_t bytes);
template <typename K> inline cudaError_t allow_smem(K kernel, size_t bytes) {
  return allow_dynamic_smem(reinterpret_cast<const void *>(kernel), bytes);
}

// Validation shared by the entry points. check_grid(g) takes FFT sides that are powers of two in
// [16, 1024]; check_grid(g, precision), for the entry points whose stages also run length 768 (the
// operator and everything built on it, the Green's tables and incident fields), also takes 768
// with complex64.
int check_grid(const dbi_grid *g);
int check_grid(const dbi_grid *g, int precision);
int check_batch(const dbi_batch *b);
int check_precision(int precision);

// Twiddle table W_3072^m, m in [0, 3072), in the precision's complex type (written into `tw`).
int launch_twiddles(void *tw, int precision, cudaStream_t s);

// A bump allocator over the caller's work buffer. A carve that does not fit (or a missing buffer)
// returns nullptr and sets `overflow` for good; every entry point calls check() after its last
// carve and before its first launch, so no kernel is ever handed a pointer outside the buffer.
struct Arena {
  char *base;
  size_t cap;
  size_t used = 0;
  bool overflow = false;
  Arena(void *b, size_t c) : base(static_cast<char *>(b)), cap(c) {}
  void *take(size_t n) {
    const size_t off = used, a = align256(n);
    if (overflow || !base || a < n || off + a < off || off + a > cap) {
      overflow = true;
      used = cap;
      return nullptr;
    }
    used = off + a;
    return base + off;
  }
  // DBI_OK, or DBI_ERR_WORKSPACE with a message naming `who` after a carve past the buffer.
  int check(const char *who) const;
};

// Sizes of the buffers each operation carves out of the work buffer (see workspace.cu).
size_t bytes_twiddles(int precision);
size_t bytes_spectral(const dbi_grid *g, int B, int precision);
// Spectral scratch of the paper-literal form (Eq. 9): five source spectra and two output spectra.
inline size_t bytes_spectral_k(const dbi_grid *g, int B, int precision) {
  return align256(size_t(B) * 7 * g->lx * g->nz * (precision == DBI_C64 ? 8 : 16));
}
// Problems per operator pass: the three operator kernels run chunk by chunk over the batch; by
// default one chunk holds the whole batch (DBI_SPECTRAL_CHUNK_MB bounds the scratch per chunk).
int spectral_chunk(const dbi_grid *g, int B, int precision);
size_t bytes_field(const dbi_grid *g, int B, int precision);
size_t bytes_partials(int B);
// per-problem power-of-two scales (scale, inverse, model scale) and their partial sums
size_t bytes_scales(int B);
// problem chunks of the adjoint imaging (each accumulates its own FP64 partial image)
int imaging_chunks(int B);

// Geometry of the FP64 partial sums of the Krylov reductions.
constexpr int kRedBlocks = 64;    // blocks per problem in a reduction pass
constexpr int kRedThreads = 256;  // threads per reduction block
constexpr int kRedSlots = 4;      // doubles per block partial
constexpr int kMaxParts = 512;    // partials per problem at most (operator kernels: one per row block)

}  // namespace dbi
