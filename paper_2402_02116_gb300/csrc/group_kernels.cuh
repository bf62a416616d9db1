// Persistent kernels of the uneven-batch operator: each stage is one launch of `blocks` CTAs that
// walk the stage's tile space (tile = blockIdx.x, + gridDim.x, ...). A tile belongs to one slot of
// one member; the member is found by binary search over the members' first tiles, and the FFT
// length and radix plan of the member select the tile body (op_tiles.cuh) inside the kernel.
#pragma once

#include "group.cuh"
#include "op_split.cuh"
#include "op_split3.cuh"
#include "op_tiles.cuh"

namespace dbi {

template <typename C> struct GroupP {
  const GMember *desc;
  int nm, total;
  const C *in;
  const C *ident;
  C *out;
  C *T;
  C *S;  // contrast-source scratch of the split-row slots (element offsets GMember::S0)
  const C *tw;
  const int *active;
  const double *in_scale, *m_scale, *out_scale;
  const C *krhat;
  double *part_out;
  int parts;
  signed char plan[11];
};

// Last member whose first tile of `stage` is <= tile (members are in tile order).
__device__ __forceinline__ int find_member(const GMember *d, int nm, int stage, int tile) {
  int lo = 0, hi = nm - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (d[mid].tile0[stage] <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int ilog2(int L) { return 31 - __clz(L); }

// Tile arguments of slot q of member M (global slot b, table f).
template <typename C>
__device__ __forceinline__ TileArgs<C> group_args(const GroupP<C> &g, const GMember &M, int b, int q, int f) {
  using Rl = typename RealOf<C>::type;
  TileArgs<C> a;
  a.nz_ = M.nz; a.nx_ = M.nx; a.lz_ = M.lz; a.lx_ = M.lx;
  a.inv2h_ = Rl(M.inv2h);
  a.b_ = b; a.f_ = f;
  a.omega_ = M.omega;
  a.in_scale_ = g.in_scale; a.out_scale_ = g.out_scale; a.m_scale_ = g.m_scale;
  a.m_ = static_cast<const Rl *>(M.m);
#pragma unroll
  for (int i = 0; i < 5; ++i) a.ref_[i] = Rl(M.ref[i]);
  const size_t fld = size_t(M.field0) + size_t(q) * 2 * M.nz * M.nx;
  a.in_ = g.in + fld;
  a.ident_ = g.ident ? g.ident + fld : nullptr;
  a.out_ = g.out + fld;
  a.T_ = g.T + size_t(M.T0) + size_t(q) * 2 * M.lx * M.nz;
  a.G_ = static_cast<const C *>(M.Ghat) + size_t(f) * 3 * M.lx * M.lz;
  a.tw_ = g.tw;
  a.krhat_ = g.krhat ? g.krhat + fld : nullptr;
  a.part_ = g.part_out ? g.part_out + size_t(b) * g.parts * kRedSlots : nullptr;
  return a;
}

// The split kind of member M's `stage`: 0 (the ordinary kernels), kSplitPair (pairs of 512-point
// transforms) or kSplitTriple (triples of 256-point transforms).
__device__ __forceinline__ int split_stage(const GMember &M, int stage) {
  return stage == kStageCols ? M.split_cols : M.split_rows;
}

// Runs body(M, b, q, f, tt) for every tile of `stage` assigned to this CTA whose slot is active and
// whose member runs the stage on this kind of kernel (SPLIT: the member's split kind; the source
// stage has tiles of split-row members only and serves both kinds).
template <int STAGE, int SPLIT = 0, typename C, typename Body>
__device__ __forceinline__ void for_tiles(const GroupP<C> &g, Body &&body) {
  for (int tile = blockIdx.x; tile < g.total; tile += gridDim.x) {
    const int i = find_member(g.desc, g.nm, STAGE, tile);
    const GMember &M = g.desc[i];
    if (STAGE != kStageSource && split_stage(M, STAGE) != SPLIT) continue;  // uniform per CTA
    const int rel = tile - M.tile0[STAGE];
    const int q = rel / M.tiles[STAGE], tt = rel - q * M.tiles[STAGE];
    const int b = M.slot0 + q;
    const int f = M.fidx[q];
    if ((g.active && !g.active[b]) || unsigned(f) >= unsigned(M.nf)) continue;  // uniform per CTA
    __syncthreads();  // the previous tile's shared-memory reads are complete
    body(M, b, q, f, tt);
  }
}

// One call per (length, plan) body: each body keeps its own register allocation inside the
// persistent kernel (a tile is microseconds of work, so the call costs nothing measurable).
template <typename C, int LX, bool STENCIL, int V>
__device__ __noinline__ void call_rows_forward(const TileArgs<C> &a, int tt, C *smem) {
  rows_forward_tile<C, LX, STENCIL, V>(a, tt, smem);
}
template <typename C, int LZ, int V>
__device__ __noinline__ void call_cols(const TileArgs<C> &a, int tt, C *smem) {
  cols_tile<C, LZ, V>(a, tt, smem);
}
template <typename C, int LX, int EPI, int V>
__device__ __noinline__ void call_rows_inverse(const TileArgs<C> &a, int tt, C *smem) {
  rows_inverse_tile<C, LX, EPI, V>(a, tt, smem);
}

template <typename C> struct GroupCfg;
template <> struct GroupCfg<float2> { static constexpr int rowsMinBlocks = 3; };
template <> struct GroupCfg<double2> { static constexpr int rowsMinBlocks = 1; };

template <typename C, bool STENCIL>
__global__ void __launch_bounds__(kTileThreads, GroupCfg<C>::rowsMinBlocks) kg_rows_forward(GroupP<C> g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *smem = reinterpret_cast<C *>(smem_raw);
  for_tiles<kStageRowsForward>(g, [&](const GMember &M, int b, int q, int f, int tt) {
    const TileArgs<C> a = group_args(g, M, b, q, f);
    const int L = M.lx, v = g.plan[ilog2(L)];
    with_len(L, [&]<int LX>() {
      if constexpr (LX == 64 || LX == 512) call_rows_forward<C, LX, STENCIL, 0>(a, tt, smem);
      else if (v) call_rows_forward<C, LX, STENCIL, 1>(a, tt, smem);
      else call_rows_forward<C, LX, STENCIL, 0>(a, tt, smem);
    });
  });
}

template <typename C>
__global__ void __launch_bounds__(kTileThreads, Cfg<C>::colMinBlocks) kg_cols(GroupP<C> g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *smem = reinterpret_cast<C *>(smem_raw);
  for_tiles<kStageCols>(g, [&](const GMember &M, int b, int q, int f, int tt) {
    const TileArgs<C> a = group_args(g, M, b, q, f);
    const int L = M.lz, v = g.plan[ilog2(L)];
    with_len(L, [&]<int LZ>() {
      if constexpr (LZ == 64 || LZ == 512) call_cols<C, LZ, 0>(a, tt, smem);
      else if (v) call_cols<C, LZ, 1>(a, tt, smem);
      else call_cols<C, LZ, 0>(a, tt, smem);
    });
  });
}

template <typename C, int EPI>
__global__ void __launch_bounds__(kTileThreads, Cfg<C>::rowInvMinBlocks) kg_rows_inverse(GroupP<C> g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *smem = reinterpret_cast<C *>(smem_raw);
  for_tiles<kStageRowsInverse>(g, [&](const GMember &M, int b, int q, int f, int tt) {
    const TileArgs<C> a = group_args(g, M, b, q, f);
    const int L = M.lx, v = g.plan[ilog2(L)];
    with_len(L, [&]<int LX>() {
      if constexpr (LX == 64 || LX == 512) call_rows_inverse<C, LX, EPI, 0>(a, tt, smem);
      else if (v) call_rows_inverse<C, LX, EPI, 1>(a, tt, smem);
      else call_rows_inverse<C, LX, EPI, 0>(a, tt, smem);
    });
  });
}

// Split kernels of the members with FFT length 1024 or 768 (complex64 only, op_split.cuh,
// op_split3.cuh): the contrast source of both (512 threads, 32 rows per tile), the rows and columns
// as pairs of 512-point transforms or triples of 256-point transforms (4 rows or columns per tile).
// Templates on the element type so that only the complex64 unit instantiates them.
template <typename C> __device__ __forceinline__ C *group_S(const GroupP<C> &g, const GMember &M, int q) {
  return g.S + size_t(M.S0) + size_t(q) * 2 * M.nz * M.nx;
}

template <typename C> __global__ void __launch_bounds__(kSrcThreads) kg_source_split(GroupP<C> g) {
  static_assert(sizeof(C) == sizeof(float2), "complex64 only");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *smem = reinterpret_cast<C *>(smem_raw);
  for_tiles<kStageSource>(g, [&](const GMember &M, int b, int q, int f, int tt) {
    source_rows(group_args(g, M, b, q, f), tt, smem, group_S(g, M, q));
  });
}

template <typename C, bool STENCIL>
__global__ void __launch_bounds__(kTileThreads, 2) kg_rows_forward_split(GroupP<C> g) {
  static_assert(sizeof(C) == sizeof(float2), "complex64 only");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *smem = reinterpret_cast<C *>(smem_raw);
  for_tiles<kStageRowsForward, kSplitPair>(g, [&](const GMember &M, int b, int q, int f, int tt) {
    const TileArgs<C> a = group_args(g, M, b, q, f);
    if constexpr (STENCIL) rows_forward_tile_split(a, tt, smem, group_S(g, M, q), 1.0f);
    else rows_forward_tile_split(a, tt, smem, a.in(), a.isc());
  });
}

// (a call of its own: inlined into the tile loop the body spills; called, it keeps its registers)
template <typename C> __device__ __noinline__ void call_cols_split(const TileArgs<C> &a, int tt, C *smem) {
  cols_tile_split(a, tt, smem);
}

template <typename C> __global__ void __launch_bounds__(kTileThreads, 2) kg_cols_split(GroupP<C> g) {
  static_assert(sizeof(C) == sizeof(float2), "complex64 only");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *smem = reinterpret_cast<C *>(smem_raw);
  for_tiles<kStageCols, kSplitPair>(g, [&](const GMember &M, int b, int q, int f, int tt) {
    call_cols_split(group_args(g, M, b, q, f), tt, smem);
  });
}

template <typename C, int EPI>
__global__ void __launch_bounds__(kTileThreads, 2) kg_rows_inverse_split(GroupP<C> g) {
  static_assert(sizeof(C) == sizeof(float2), "complex64 only");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *smem = reinterpret_cast<C *>(smem_raw);
  for_tiles<kStageRowsInverse, kSplitPair>(g, [&](const GMember &M, int b, int q, int f, int tt) {
    rows_inverse_tile_split<EPI>(group_args(g, M, b, q, f), tt, smem);
  });
}

template <typename C, bool STENCIL>
__global__ void __launch_bounds__(kS3Threads, 2) kg_rows_forward_s3(GroupP<C> g) {
  static_assert(sizeof(C) == sizeof(float2), "complex64 only");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *smem = reinterpret_cast<C *>(smem_raw);
  for_tiles<kStageRowsForward, kSplitTriple>(g, [&](const GMember &M, int b, int q, int f, int tt) {
    const TileArgs<C> a = group_args(g, M, b, q, f);
    if constexpr (STENCIL) rows_forward_tile_s3(a, tt, smem, group_S(g, M, q), 1.0f);
    else rows_forward_tile_s3(a, tt, smem, a.in(), a.isc());
  });
}

template <typename C> __global__ void __launch_bounds__(kS3Threads, 2) kg_cols_s3(GroupP<C> g) {
  static_assert(sizeof(C) == sizeof(float2), "complex64 only");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *smem = reinterpret_cast<C *>(smem_raw);
  for_tiles<kStageCols, kSplitTriple>(g, [&](const GMember &M, int b, int q, int f, int tt) {
    cols_tile_s3(group_args(g, M, b, q, f), tt, smem);
  });
}

template <typename C, int EPI>
__global__ void __launch_bounds__(kS3Threads, 2) kg_rows_inverse_s3(GroupP<C> g) {
  static_assert(sizeof(C) == sizeof(float2), "complex64 only");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *smem = reinterpret_cast<C *>(smem_raw);
  for_tiles<kStageRowsInverse, kSplitTriple>(g, [&](const GMember &M, int b, int q, int f, int tt) {
    rows_inverse_tile_s3<EPI>(group_args(g, M, b, q, f), tt, smem);
  });
}

template <typename C> int group_split_occupancy_impl(int per_sm[7]) {
  cudaError_t e = cudaSuccess;
  auto occ = [&](auto kernel, int threads, size_t smem, int *n) {
    if (e != cudaSuccess) return;
    e = allow_smem(kernel, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, kernel, threads, smem);
  };
  occ(kg_source_split<C>, kSrcThreads, source_smem(), &per_sm[0]);
  int x = 0, y = 0;
  occ(kg_rows_forward_split<C, true>, kTileThreads, split_rows_smem(), &x);
  occ(kg_rows_forward_split<C, false>, kTileThreads, split_rows_smem(), &y);
  per_sm[1] = std::min(x, y);
  occ(kg_cols_split<C>, kTileThreads, split_cols_smem(), &per_sm[2]);
  per_sm[3] = 1 << 20;
  occ(kg_rows_inverse_split<C, 0>, kTileThreads, split_rows_inverse_smem(), &x);
  per_sm[3] = std::min(per_sm[3], x);
  occ(kg_rows_inverse_split<C, 1>, kTileThreads, split_rows_inverse_smem(), &x);
  per_sm[3] = std::min(per_sm[3], x);
  occ(kg_rows_inverse_split<C, 2>, kTileThreads, split_rows_inverse_smem(), &x);
  per_sm[3] = std::min(per_sm[3], x);
  occ(kg_rows_forward_s3<C, true>, kS3Threads, s3_smem(), &x);
  occ(kg_rows_forward_s3<C, false>, kS3Threads, s3_smem(), &y);
  per_sm[4] = std::min(x, y);
  occ(kg_cols_s3<C>, kS3Threads, s3_smem(), &per_sm[5]);
  per_sm[6] = 1 << 20;
  occ(kg_rows_inverse_s3<C, 0>, kS3Threads, s3_smem(), &x);
  per_sm[6] = std::min(per_sm[6], x);
  occ(kg_rows_inverse_s3<C, 1>, kS3Threads, s3_smem(), &x);
  per_sm[6] = std::min(per_sm[6], x);
  occ(kg_rows_inverse_s3<C, 2>, kS3Threads, s3_smem(), &x);
  per_sm[6] = std::min(per_sm[6], x);
  return e == cudaSuccess ? DBI_OK : cuda_fail("occupancy of the split group kernels", e);
}

template <typename C> int run_group_typed(const OpArgs &a, cudaStream_t s) {
  const GroupLaunch &gl = *a.group;
  GroupP<C> g;
  g.desc = gl.desc;
  g.nm = gl.nm;
  g.in = static_cast<const C *>(a.in);
  g.ident = static_cast<const C *>(a.ident);
  g.out = static_cast<C *>(a.out);
  g.T = static_cast<C *>(a.T);
  g.S = g.T + size_t(gl.T_elems);  // the split-row sources follow the spectra
  g.tw = static_cast<const C *>(a.tw);
  g.active = a.active;
  g.in_scale = a.in_scale;
  g.m_scale = a.m_scale;
  g.out_scale = a.out_scale;
  g.krhat = static_cast<const C *>(a.krhat);
  g.part_out = a.part_out;
  g.parts = gl.parts;
  for (int i = 0; i < 11; ++i) g.plan[i] = gl.plan[i];
  auto launch = [&](auto kernel, int stage, size_t smem, const char *what) -> int {
    g.total = gl.total[stage];
    if (g.total == 0) return DBI_OK;
    cudaError_t e = allow_smem(kernel, smem);
    if (e != cudaSuccess) return cuda_fail(what, e);
    const int blocks = std::max(1, std::min(gl.blocks[stage], g.total));
    kernel<<<blocks, kTileThreads, smem, s>>>(g);
    return check_launch(what);
  };
  // the split kernels of the length-1024 and length-768 members (complex64), each stage before the
  // others' kernel
  auto launch_split = [&](auto kernel, int stage, int blocks_max, int threads, size_t smem, const char *what) -> int {
    g.total = gl.total[stage];
    if (g.total == 0) return DBI_OK;
    cudaError_t e = allow_smem(kernel, smem);
    if (e != cudaSuccess) return cuda_fail(what, e);
    const int blocks = std::max(1, std::min(blocks_max, g.total));
    kernel<<<blocks, threads, smem, s>>>(g);
    return check_launch(what);
  };
  int rc = DBI_OK;
  if constexpr (sizeof(C) == sizeof(float2)) {
    if (a.stencil && (gl.split_rows || gl.s3_rows) &&
        (rc = launch_split(kg_source_split<C>, kStageSource, gl.split_blocks[0], kSrcThreads, source_smem(),
                           "kg_source_split")))
      return rc;
    if (gl.s3_rows) {
      if (a.stencil)
        rc = launch_split(kg_rows_forward_s3<C, true>, kStageRowsForward, gl.s3_blocks[0], kS3Threads, s3_smem(),
                          "kg_rows_forward_s3");
      else
        rc = launch_split(kg_rows_forward_s3<C, false>, kStageRowsForward, gl.s3_blocks[0], kS3Threads, s3_smem(),
                          "kg_rows_forward_s3");
      if (rc) return rc;
    }
    if (gl.split_rows) {
      if (a.stencil)
        rc = launch_split(kg_rows_forward_split<C, true>, kStageRowsForward, gl.split_blocks[1], kTileThreads,
                          split_rows_smem(),
                          "kg_rows_forward_split");
      else
        rc = launch_split(kg_rows_forward_split<C, false>, kStageRowsForward, gl.split_blocks[1], kTileThreads,
                          split_rows_smem(),
                          "kg_rows_forward_split");
      if (rc) return rc;
    }
  }
  if (a.stencil) rc = launch(kg_rows_forward<C, true>, kStageRowsForward, gl.smem[0], "kg_rows_forward");
  else rc = launch(kg_rows_forward<C, false>, kStageRowsForward, gl.smem[1], "kg_rows_forward");
  if (rc) return rc;
  if constexpr (sizeof(C) == sizeof(float2)) {
    if (gl.split_cols && (rc = launch_split(kg_cols_split<C>, kStageCols, gl.split_blocks[2], kTileThreads,
                                            split_cols_smem(), "kg_cols_split")))
      return rc;
    if (gl.s3_cols &&
        (rc = launch_split(kg_cols_s3<C>, kStageCols, gl.s3_blocks[1], kS3Threads, s3_smem(), "kg_cols_s3")))
      return rc;
  }
  if ((rc = launch(kg_cols<C>, kStageCols, gl.smem[2], "kg_cols"))) return rc;
  if constexpr (sizeof(C) == sizeof(float2)) {
    if (gl.split_rows) {
      if (a.epi == 1)
        rc = launch_split(kg_rows_inverse_split<C, 1>, kStageRowsInverse, gl.split_blocks[3], kTileThreads,
                          split_rows_inverse_smem(),
                          "kg_rows_inverse_split");
      else if (a.epi == 2)
        rc = launch_split(kg_rows_inverse_split<C, 2>, kStageRowsInverse, gl.split_blocks[3], kTileThreads,
                          split_rows_inverse_smem(),
                          "kg_rows_inverse_split");
      else
        rc = launch_split(kg_rows_inverse_split<C, 0>, kStageRowsInverse, gl.split_blocks[3], kTileThreads,
                          split_rows_inverse_smem(),
                          "kg_rows_inverse_split");
      if (rc) return rc;
    }
    if (gl.s3_rows) {
      if (a.epi == 1)
        rc = launch_split(kg_rows_inverse_s3<C, 1>, kStageRowsInverse, gl.s3_blocks[2], kS3Threads, s3_smem(),
                          "kg_rows_inverse_s3");
      else if (a.epi == 2)
        rc = launch_split(kg_rows_inverse_s3<C, 2>, kStageRowsInverse, gl.s3_blocks[2], kS3Threads, s3_smem(),
                          "kg_rows_inverse_s3");
      else
        rc = launch_split(kg_rows_inverse_s3<C, 0>, kStageRowsInverse, gl.s3_blocks[2], kS3Threads, s3_smem(),
                          "kg_rows_inverse_s3");
      if (rc) return rc;
    }
  }
  if (a.epi == 1) rc = launch(kg_rows_inverse<C, 1>, kStageRowsInverse, gl.smem[3], "kg_rows_inverse");
  else if (a.epi == 2) rc = launch(kg_rows_inverse<C, 2>, kStageRowsInverse, gl.smem[3], "kg_rows_inverse");
  else rc = launch(kg_rows_inverse<C, 0>, kStageRowsInverse, gl.smem[3], "kg_rows_inverse");
  return rc;
}

template <typename C> int group_occupancy(int stage, int epi, size_t smem, int *per_sm) {
  cudaError_t e = cudaSuccess;
  auto occ = [&](auto kernel) {
    e = allow_smem(kernel, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kernel, kTileThreads, smem);
  };
  if (stage == 0) occ(kg_rows_forward<C, true>);
  else if (stage == 1) occ(kg_rows_forward<C, false>);
  else if (stage == 2) occ(kg_cols<C>);
  else if (epi == 1) occ(kg_rows_inverse<C, 1>);
  else if (epi == 2) occ(kg_rows_inverse<C, 2>);
  else occ(kg_rows_inverse<C, 0>);
  return e == cudaSuccess ? DBI_OK : cuda_fail("cudaOccupancyMaxActiveBlocksPerMultiprocessor", e);
}

}  // namespace dbi
