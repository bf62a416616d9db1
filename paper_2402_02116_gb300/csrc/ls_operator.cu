// The batched LS operator A u = u - h^2 G * (w^2 drho u + div(dC : eps(u))) (Eq. 6, 10) and the
// plain Green's convolution, both evaluated by Eq. 12 on the zero-padded lz x lx grid, for a batch
// of problems on one grid: three kernels per batch (the tile bodies are in op_tiles.cuh), each
// with one CTA per (tile, problem):
//   k_rows_forward : contrast source and forward FFT along x of a few rows -> T[b][c][kx][z]
//   k_cols         : column FFTs, 2x2 Ghat multiply, inverse column FFTs, in place in T
//   k_rows_inverse : inverse FFT along x of a few rows, out = ident - result (or the result)
#include <algorithm>

#include "group.cuh"
#include "op_split.cuh"
#include "op_split3.cuh"
#include "op_tiles.cuh"
#include "operator.cuh"
#include "tune.cuh"

namespace dbi {

template <typename C> struct OpP {
  using Rl = typename RealOf<C>::type;
  int nz, nx, lz, lx, nf;
  Rl inv2h;
  const double *omega;
  const int *fidx;
  const Rl *m;
  Rl ref[5];
  const C *in;
  const C *ident;
  C *out;
  C *T;
  const C *Ghat;
  const C *tw;
  const int *active;
  const int *plist;  // slot -> problem (NULL: problem = s0 + slot)
  int s0;            // first slot of this launch
  int nb;            // slots in this launch
  const double *in_scale, *m_scale, *out_scale;
  const C *krhat;
  double *part_out;
  int part_count;
  C *S;  // [slots][2][nz][nx] contrast-source scratch of the split row stages (L = 1024, 768), or NULL
};

// Problem of this CTA's launch slot (blockIdx.y); the spectral scratch is indexed by the slot.
template <typename C> __device__ __forceinline__ int problem_of(const OpP<C> &p) {
  const int sl = p.s0 + int(blockIdx.y);
  return p.plist ? p.plist[sl] : sl;
}

// Tile accessor of problem b in launch slot `slot`: every value is read from the kernel's
// parameters where the tile body uses it (kernel parameters live in constant memory, so they cost
// no registers until then; a reference to the parameter would force generic loads through its
// address instead).
template <typename C> struct BatchTile {
  using Rl = typename RealOf<C>::type;
  OpP<C> p;  // a copy of the kernel parameter: its fields stay parameter reads (no address taken)
  int b, slot, f;
  __device__ __forceinline__ size_t fld() const { return size_t(b) * 2 * p.nz * p.nx; }
  __device__ __forceinline__ int nz() const { return p.nz; }
  __device__ __forceinline__ int nx() const { return p.nx; }
  __device__ __forceinline__ int lx() const { return p.lx; }
  __device__ __forceinline__ Rl inv2h() const { return p.inv2h; }
  __device__ __forceinline__ Rl ref(int i) const { return p.ref[i]; }
  __device__ __forceinline__ const Rl *m() const { return p.m; }
  __device__ __forceinline__ const C *in() const { return p.in + fld(); }
  __device__ __forceinline__ const C *ident() const { return p.ident ? p.ident + fld() : nullptr; }
  __device__ __forceinline__ C *out() const { return p.out + fld(); }
  __device__ __forceinline__ C *T() const { return p.T + size_t(slot) * 2 * p.lx * p.nz; }
  __device__ __forceinline__ const C *G() const { return p.Ghat + size_t(f) * 3 * p.lx * p.lz; }
  __device__ __forceinline__ const C *tw() const { return p.tw; }
  __device__ __forceinline__ const C *krhat() const { return p.krhat + fld(); }
  __device__ __forceinline__ C *S() const { return p.S + size_t(slot) * 2 * p.nz * p.nx; }
  __device__ __forceinline__ double *part() const { return p.part_out + size_t(b) * p.part_count * kRedSlots; }
  __device__ __forceinline__ Rl w2() const {
    const double om = p.omega[f];
    return Rl(om * om);
  }
  __device__ __forceinline__ Rl isc() const { return p.in_scale ? Rl(p.in_scale[b]) : Rl(1); }
  __device__ __forceinline__ Rl osc() const { return p.out_scale ? Rl(p.out_scale[b]) : Rl(1); }
  __device__ __forceinline__ Rl ms() const { return p.m_scale ? Rl(p.m_scale[0]) : Rl(1); }
};

template <typename C, int LX, bool STENCIL, int V>
__global__ void __launch_bounds__(kTileThreads, Cfg<C>::rowFwdMinBlocks(LX)) k_rows_forward(OpP<C> p) {
  const int b = problem_of(p), f = p.fidx[b];
  if ((p.active && !p.active[b]) || unsigned(f) >= unsigned(p.nf)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rows_forward_tile<C, LX, STENCIL, V>(BatchTile<C>{p, b, int(blockIdx.y), f}, blockIdx.x,
                                       reinterpret_cast<C *>(smem_raw));
}

template <typename C, int LZ, int V>
__global__ void __launch_bounds__(kTileThreads, Cfg<C>::colMinBlocks) k_cols(OpP<C> p) {
  const int b = problem_of(p), f = p.fidx[b];
  if ((p.active && !p.active[b]) || unsigned(f) >= unsigned(p.nf)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cols_tile<C, LZ, V>(BatchTile<C>{p, b, int(blockIdx.y), f}, blockIdx.x, reinterpret_cast<C *>(smem_raw));
}

template <typename C, int LX, int EPI, int V>
__global__ void __launch_bounds__(kTileThreads, Cfg<C>::rowInvMinBlocks) k_rows_inverse(OpP<C> p) {
  const int b = problem_of(p), f = p.fidx[b];
  if ((p.active && !p.active[b]) || unsigned(f) >= unsigned(p.nf)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rows_inverse_tile<C, LX, EPI, V>(BatchTile<C>{p, b, int(blockIdx.y), f}, blockIdx.x,
                                   reinterpret_cast<C *>(smem_raw));
}

// Stages of the L = 1024 complex64 operator as pairs of 512-point transforms (op_split.cuh).
__global__ void __launch_bounds__(kSrcThreads) k_source_split(OpP<float2> p) {
  const int b = problem_of(p), f = p.fidx[b];
  if ((p.active && !p.active[b]) || unsigned(f) >= unsigned(p.nf)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BatchTile<float2> a{p, b, int(blockIdx.y), f};
  source_rows(a, blockIdx.x, reinterpret_cast<float2 *>(smem_raw), a.S());
}

template <bool STENCIL>
__global__ void __launch_bounds__(kTileThreads, 2) k_rows_forward_split(OpP<float2> p) {
  const int b = problem_of(p), f = p.fidx[b];
  if ((p.active && !p.active[b]) || unsigned(f) >= unsigned(p.nf)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BatchTile<float2> a{p, b, int(blockIdx.y), f};
  float2 *smem = reinterpret_cast<float2 *>(smem_raw);
  if constexpr (STENCIL) rows_forward_tile_split(a, blockIdx.x, smem, a.S(), 1.0f);
  else rows_forward_tile_split(a, blockIdx.x, smem, a.in(), a.isc());
}

// Column kx = blockIdx.x of the four launch slots 4 blockIdx.y .. + 3 (64 threads each). The
// column's Green's tables of the first slot's frequency are staged in shared memory by
// asynchronous copies issued before the forward transforms, so their latency is hidden; slots of
// that frequency (consecutive slots share it, problems being frequency-major) read them there,
// others from global memory.
__global__ void __launch_bounds__(kTileThreads, 2) k_cols_split(OpP<float2> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *smem = reinterpret_cast<float2 *>(smem_raw);
  float4 *Gs = reinterpret_cast<float4 *>(smem + split_cols_lines_smem() / sizeof(float2));
  const int g = threadIdx.x / kSplitT, kx = blockIdx.x;
  const int sl0 = 4 * int(blockIdx.y), sl = sl0 + g;
  auto prob = [&](int slot) { return p.plist ? p.plist[p.s0 + slot] : p.s0 + slot; };
  auto freq = [&](int slot) {  // the slot's table, or -1 when it has no work
    if (slot >= p.nb) return -1;
    const int b = prob(slot), f = p.fidx[b];
    return ((p.active && !p.active[b]) || unsigned(f) >= unsigned(p.nf)) ? -1 : f;
  };
  const int f0 = freq(sl0), f = freq(sl);
  if (f0 >= 0) {  // Ghat(:, kx) of table f0: 3 x 1024 points, six 16-byte copies per thread
    const float2 *G = p.Ghat + size_t(f0) * 3 * p.lx * kSplitL + size_t(kx) * kSplitL;
    const size_t plane = size_t(p.lx) * kSplitL;
#pragma unroll
    for (int i = 0; i < 3 * kSplitL / 2 / kTileThreads; ++i) {
      const int e = threadIdx.x + i * kTileThreads, tb = e / (kSplitL / 2), k = e - tb * (kSplitL / 2);
      cp_async16(Gs + e, G + tb * plane + 2 * k);
    }
  }
  const int b = f >= 0 ? prob(sl) : 0;
  cols_column_split<true>(BatchTile<float2>{p, b, sl, f >= 0 ? f : 0}, kx, g, f >= 0, smem,
                          f == f0 ? Gs : nullptr);
}

template <int EPI>
__global__ void __launch_bounds__(kTileThreads, 2) k_rows_inverse_split(OpP<float2> p) {
  const int b = problem_of(p), f = p.fidx[b];
  if ((p.active && !p.active[b]) || unsigned(f) >= unsigned(p.nf)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rows_inverse_tile_split<EPI>(BatchTile<float2>{p, b, int(blockIdx.y), f}, blockIdx.x,
                               reinterpret_cast<float2 *>(smem_raw));
}

// Stages of the L = 768 complex64 operator as triples of 256-point transforms (op_split3.cuh);
// the contrast source comes from k_source_split.
template <bool STENCIL>
__global__ void __launch_bounds__(kS3Threads, 2) k_rows_forward_s3(OpP<float2> p) {
  const int b = problem_of(p), f = p.fidx[b];
  if ((p.active && !p.active[b]) || unsigned(f) >= unsigned(p.nf)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BatchTile<float2> a{p, b, int(blockIdx.y), f};
  float2 *smem = reinterpret_cast<float2 *>(smem_raw);
  if constexpr (STENCIL) rows_forward_tile_s3(a, blockIdx.x, smem, a.S(), 1.0f);
  else rows_forward_tile_s3(a, blockIdx.x, smem, a.in(), a.isc());
}

__global__ void __launch_bounds__(kS3Threads, 2) k_cols_s3(OpP<float2> p) {
  const int b = problem_of(p), f = p.fidx[b];
  if ((p.active && !p.active[b]) || unsigned(f) >= unsigned(p.nf)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cols_tile_s3(BatchTile<float2>{p, b, int(blockIdx.y), f}, blockIdx.x, reinterpret_cast<float2 *>(smem_raw));
}

template <int EPI>
__global__ void __launch_bounds__(kS3Threads, 2) k_rows_inverse_s3(OpP<float2> p) {
  const int b = problem_of(p), f = p.fidx[b];
  if ((p.active && !p.active[b]) || unsigned(f) >= unsigned(p.nf)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rows_inverse_tile_s3<EPI>(BatchTile<float2>{p, b, int(blockIdx.y), f}, blockIdx.x,
                            reinterpret_cast<float2 *>(smem_raw));
}

// Calls f.template operator()<V>() with the radix plan chosen for length L (plans differ only
// when L is not a power of 8).
template <int L, typename F> inline void with_plan(int precision, F &&f) {
  if constexpr (L == 64 || L == 512) f.template operator()<0>();
  else if (radix_plan(precision, L) == 1) f.template operator()<1>();
  else f.template operator()<0>();
}

// The three kernels for launch slots [s0, s0 + nb) (problems plist[slot], or the slots themselves),
// each slot using its own part of the spectral scratch.
template <typename C> static int run_chunk(const OpArgs &a, int s0, int nb, int cap, cudaStream_t s) {
  using Rl = typename RealOf<C>::type;
  OpP<C> p;
  p.nz = a.nz; p.nx = a.nx; p.lz = a.lz; p.lx = a.lx; p.nf = a.nf;
  p.inv2h = Rl(1.0 / (2.0 * a.h));
  p.omega = a.omega; p.fidx = a.fidx;
  p.m = static_cast<const Rl *>(a.m);
  for (int i = 0; i < 5; ++i) p.ref[i] = Rl(a.ref[i]);
  p.in = static_cast<const C *>(a.in);
  p.ident = static_cast<const C *>(a.ident);
  p.out = static_cast<C *>(a.out);
  p.T = static_cast<C *>(a.T);
  p.Ghat = static_cast<const C *>(a.Ghat);
  p.tw = static_cast<const C *>(a.tw);
  p.active = a.active;
  p.plist = a.plist;
  p.s0 = s0;
  p.nb = nb;
  p.in_scale = a.in_scale;
  p.m_scale = a.m_scale;
  p.out_scale = a.out_scale;
  p.part_count = operator_parts(a.nz, a.lx, a.precision);
  p.krhat = static_cast<const C *>(a.krhat);
  p.part_out = a.part_out;
  p.S = nullptr;
  int rc = DBI_OK;
  const bool stencil = a.stencil;
  const int kr = split_kind(a.lx, a.precision), kc = split_kind(a.lz, a.precision);
  const bool split_r = kr != 0, split_c = kc != 0;
  if (split_r) p.S = p.T + size_t(cap) * 2 * a.lx * a.nz;  // after the chunk's spectra
  prof_mark(PROF_ROWS_FORWARD, false, s);
  if constexpr (sizeof(C) == sizeof(float2)) {
    if (split_r) {
      OpP<float2> &q = reinterpret_cast<OpP<float2> &>(p);
      cudaError_t e = cudaSuccess;
      if (stencil) {
        const int chunks = (a.nz + kSrcRows - 1) / kSrcRows;
        e = allow_smem(k_source_split, source_smem());
        if (e == cudaSuccess) k_source_split<<<dim3(chunks, nb), kSrcThreads, source_smem(), s>>>(q);
        rc = e != cudaSuccess ? cuda_fail("k_source_split smem", e) : check_launch("k_source_split");
        if (rc) return rc;
      }
      if (kr == kSplitPair) {
        const dim3 grid((a.nz + kSplitRows - 1) / kSplitRows, nb);
        auto kern = stencil ? k_rows_forward_split<true> : k_rows_forward_split<false>;
        e = allow_smem(kern, split_rows_smem());
        if (e == cudaSuccess) kern<<<grid, kTileThreads, split_rows_smem(), s>>>(q);
        rc = e != cudaSuccess ? cuda_fail("k_rows_forward_split smem", e) : check_launch("k_rows_forward_split");
      } else {
        const dim3 grid((a.nz + kS3Units - 1) / kS3Units, nb);
        auto kern = stencil ? k_rows_forward_s3<true> : k_rows_forward_s3<false>;
        e = allow_smem(kern, s3_smem());
        if (e == cudaSuccess) kern<<<grid, kS3Threads, s3_smem(), s>>>(q);
        rc = e != cudaSuccess ? cuda_fail("k_rows_forward_s3 smem", e) : check_launch("k_rows_forward_s3");
      }
    }
  }
  if (!split_r) dispatch_len(a.lx, [&]<int LX>() {
    with_plan<LX>(a.precision, [&]<int V>() {
      using RC = RowCfg<C, LX>;
      const size_t bytes = rows_forward_smem<C, LX>(a.nx, stencil);
      dim3 grid((a.nz + RC::ROWS - 1) / RC::ROWS, nb);
      cudaError_t e;
      auto launch = [&](auto kernel) {
        e = allow_smem(kernel, bytes);
        if (e == cudaSuccess) kernel<<<grid, RC::NT, bytes, s>>>(p);
      };
      if (stencil) launch(k_rows_forward<C, LX, true, V>);
      else launch(k_rows_forward<C, LX, false, V>);
      rc = e != cudaSuccess ? cuda_fail("k_rows_forward smem", e) : check_launch("k_rows_forward");
    });
  });
  prof_mark(PROF_ROWS_FORWARD, true, s);
  if (rc) return rc;
  prof_mark(PROF_COLS, false, s);
  if constexpr (sizeof(C) == sizeof(float2)) {
    if (kc == kSplitPair) {
      OpP<float2> &q = reinterpret_cast<OpP<float2> &>(p);
      const dim3 grid(a.lx, (nb + 3) / 4);
      cudaError_t e = allow_smem(k_cols_split, split_cols_staged_smem());
      if (e == cudaSuccess) k_cols_split<<<grid, kTileThreads, split_cols_staged_smem(), s>>>(q);
      rc = e != cudaSuccess ? cuda_fail("k_cols_split smem", e) : check_launch("k_cols_split");
    } else if (kc == kSplitTriple) {
      OpP<float2> &q = reinterpret_cast<OpP<float2> &>(p);
      const dim3 grid((a.lx + kS3Units - 1) / kS3Units, nb);
      cudaError_t e = allow_smem(k_cols_s3, s3_smem());
      if (e == cudaSuccess) k_cols_s3<<<grid, kS3Threads, s3_smem(), s>>>(q);
      rc = e != cudaSuccess ? cuda_fail("k_cols_s3 smem", e) : check_launch("k_cols_s3");
    }
  }
  if (!split_c) dispatch_len(a.lz, [&]<int LZ>() {
    with_plan<LZ>(a.precision, [&]<int V>() {
      using CF = ColCfg<C, LZ>;
      const size_t bytes = cols_smem<C, LZ>();
      dim3 grid((a.lx + CF::CC - 1) / CF::CC, nb);
      cudaError_t e = allow_smem(k_cols<C, LZ, V>, bytes);
      if (e == cudaSuccess) k_cols<C, LZ, V><<<grid, CF::NT, bytes, s>>>(p);
      rc = e != cudaSuccess ? cuda_fail("k_cols smem", e) : check_launch("k_cols");
    });
  });
  prof_mark(PROF_COLS, true, s);
  if (rc) return rc;
  prof_mark(PROF_ROWS_INVERSE, false, s);
  if constexpr (sizeof(C) == sizeof(float2)) {
    if (kr == kSplitPair) {
      OpP<float2> &q = reinterpret_cast<OpP<float2> &>(p);
      const dim3 grid((a.nz + kSplitRows - 1) / kSplitRows, nb);
      auto kern = a.epi == 1 ? k_rows_inverse_split<1> : a.epi == 2 ? k_rows_inverse_split<2> : k_rows_inverse_split<0>;
      cudaError_t e = allow_smem(kern, split_rows_inverse_smem());
      if (e == cudaSuccess) kern<<<grid, kTileThreads, split_rows_inverse_smem(), s>>>(q);
      rc = e != cudaSuccess ? cuda_fail("k_rows_inverse_split smem", e) : check_launch("k_rows_inverse_split");
    } else if (kr == kSplitTriple) {
      OpP<float2> &q = reinterpret_cast<OpP<float2> &>(p);
      const dim3 grid((a.nz + kS3Units - 1) / kS3Units, nb);
      auto kern = a.epi == 1 ? k_rows_inverse_s3<1> : a.epi == 2 ? k_rows_inverse_s3<2> : k_rows_inverse_s3<0>;
      cudaError_t e = allow_smem(kern, s3_smem());
      if (e == cudaSuccess) kern<<<grid, kS3Threads, s3_smem(), s>>>(q);
      rc = e != cudaSuccess ? cuda_fail("k_rows_inverse_s3 smem", e) : check_launch("k_rows_inverse_s3");
    }
  }
  if (!split_r) dispatch_len(a.lx, [&]<int LX>() {
    with_plan<LX>(a.precision, [&]<int V>() {
      using RC = RowCfg<C, LX>;
      const size_t bytes = rows_inverse_smem<C, LX>();
      dim3 grid((a.nz + RC::ROWS - 1) / RC::ROWS, nb);
      cudaError_t e;
      auto launch = [&](auto kernel) {
        e = allow_smem(kernel, bytes);
        if (e == cudaSuccess) kernel<<<grid, RC::NT, bytes, s>>>(p);
      };
      if (a.epi == 1) launch(k_rows_inverse<C, LX, 1, V>);
      else if (a.epi == 2) launch(k_rows_inverse<C, LX, 2, V>);
      else launch(k_rows_inverse<C, LX, 0, V>);
      rc = e != cudaSuccess ? cuda_fail("k_rows_inverse smem", e) : check_launch("k_rows_inverse");
    });
  });
  prof_mark(PROF_ROWS_INVERSE, true, s);
  return rc;
}

template <typename C> static int run_typed(const OpArgs &a, cudaStream_t s) {
  const int nb = a.plist ? a.nb : a.B;
  if (nb <= 0) return DBI_OK;
  dbi_grid g{a.nz, a.nx, a.lz, a.lx, a.h};
  const int chunk = spectral_chunk(&g, a.B, a.precision);
  int rc = DBI_OK;
  prof_mark(PROF_OPERATOR, false, s);
  for (int s0 = 0; s0 < nb && rc == DBI_OK; s0 += chunk)
    rc = run_chunk<C>(a, s0, std::min(chunk, nb - s0), chunk, s);
  prof_mark(PROF_OPERATOR, true, s);
  return rc;
}

int operator_parts(int nz, int lx, int precision) {
  static_assert(kS3Units == kSplitRows, "split row tiles hold the same number of rows");
  if (split_rows(lx, precision)) return (nz + kSplitRows - 1) / kSplitRows;
  return operator_parts_k(nz, lx, precision);
}

int operator_parts_k(int nz, int lx, int precision) {
  int rows = 1;
  auto pick = [&](auto tag) {
    using C = decltype(tag);
    dispatch_len(lx, [&]<int LX>() { rows = RowCfg<C, LX>::ROWS; });
  };
  if (precision == DBI_C64) pick(float2{});
  else pick(double2{});
  return (nz + rows - 1) / rows;
}

int run_operator(const OpArgs &a, cudaStream_t s) {
  if (a.ny > 0) return run_operator_3d(a, s);
  if (a.group) return run_group_operator(a, s);
  if (a.Dhat) return run_form_k(a, s);
  return a.precision == DBI_C64 ? run_typed<float2>(a, s) : run_typed<double2>(a, s);
}

}  // namespace dbi

using namespace dbi;

// Common validation of the operator entry points.
static int check_op(const dbi_grid *g, const dbi_batch *batch, const void *Ghat, const void *in,
                    const void *out, int precision, void *work, size_t work_bytes, int op) {
  int rc;
  if ((rc = check_grid(g, precision)) || (rc = check_batch(batch)) || (rc = check_precision(precision))) return rc;
  if (batch->B > 0 && (!Ghat || !in || !out)) { set_error("NULL Ghat, input or output"); return DBI_ERR_ARG; }
  if (in == out && batch->B > 0) { set_error("input and output must be distinct buffers"); return DBI_ERR_ARG; }
  const size_t need = dbi_workspace_bytes(g, batch->B, precision, op);
  if (batch->B > 0 && (!work || work_bytes < need)) {
    set_error("work buffer of %zu bytes, need %zu", work_bytes, need);
    return DBI_ERR_WORKSPACE;
  }
  return DBI_OK;
}

extern "C" int green_convolve(const dbi_grid *g, const dbi_batch *batch, const void *Ghat,
                              const void *src, void *out, int precision, void *work,
                              size_t work_bytes, dbi_stream stream) {
  clear_error();
  int rc = check_op(g, batch, Ghat, src, out, precision, work, work_bytes, DBI_OP_CONVOLVE);
  if (rc || batch->B == 0) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Arena ar(work, work_bytes);
  void *tw = ar.take(bytes_twiddles(precision));
  void *T = ar.take(bytes_spectral(g, batch->B, precision));
  Scales sc = carve_scales(ar, batch->B);
  if ((rc = ar.check(__func__))) return rc;
  if ((rc = launch_twiddles(tw, precision, s))) return rc;
  if ((rc = pow2_scales(src, precision, false, batch->B, size_t(2) * g->nz * g->nx, sc.part, sc.scale, sc.inv,
                        nullptr, s)))
    return rc;
  OpArgs a{};
  a.precision = precision; a.nz = g->nz; a.nx = g->nx; a.lz = g->lz; a.lx = g->lx; a.h = g->h;
  a.B = batch->B; a.nf = batch->nf; a.omega = batch->omega; a.fidx = batch->fidx;
  a.stencil = false; a.in = src; a.ident = nullptr; a.out = out; a.T = T; a.Ghat = Ghat; a.tw = tw;
  a.in_scale = sc.scale; a.out_scale = sc.inv;
  return run_operator(a, s);
}

extern "C" int ls_apply(const dbi_model *model, const dbi_batch *batch, const void *Ghat,
                        const void *u, void *out, int precision, void *work, size_t work_bytes,
                        dbi_stream stream) {
  clear_error();
  if (!model) { set_error("model is NULL"); return DBI_ERR_ARG; }
  const dbi_grid *g = &model->grid;
  int rc = check_op(g, batch, Ghat, u, out, precision, work, work_bytes, DBI_OP_APPLY);
  if (rc || batch->B == 0) return rc;
  if (!model->m) { set_error("model->m is NULL"); return DBI_ERR_ARG; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Arena ar(work, work_bytes);
  void *tw = ar.take(bytes_twiddles(precision));
  void *T = ar.take(bytes_spectral(g, batch->B, precision));
  Scales sc = carve_scales(ar, batch->B);
  if ((rc = ar.check(__func__))) return rc;
  if ((rc = launch_twiddles(tw, precision, s))) return rc;
  if ((rc = pow2_scales(u, precision, false, batch->B, size_t(2) * g->nz * g->nx, sc.part, sc.scale, sc.inv,
                        nullptr, s)))
    return rc;
  OpArgs a{};
  a.precision = precision; a.nz = g->nz; a.nx = g->nx; a.lz = g->lz; a.lx = g->lx; a.h = g->h;
  a.B = batch->B; a.nf = batch->nf; a.omega = batch->omega; a.fidx = batch->fidx;
  a.m = model->m; reference_values(model->ref, a.ref);
  a.stencil = true; a.in = u; a.ident = u; a.out = out; a.T = T; a.Ghat = Ghat; a.tw = tw;
  a.in_scale = sc.scale; a.out_scale = sc.inv;
  return run_operator(a, s);
}
