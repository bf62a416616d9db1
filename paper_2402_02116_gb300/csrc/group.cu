// Uneven batches (dbi_group.h): plan, workspace, entry points and the autotuner.
//
// The plan orders the members by decreasing FFT length (lx, then lz) and lays the tiles of each
// operator stage out member by member, slot by slot; the persistent kernels (group_kernels.cuh)
// walk that tile space. Slots, fields and spectra keep the caller's member order.
#include <algorithm>
#include <chrono>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/dbi_group.h"
#include "group.cuh"
#include "krylov.cuh"
#include "op_split.cuh"
#include "op_split3.cuh"
#include "op_tiles.cuh"
#include "tune.cuh"

using namespace dbi;

struct dbi_group {
  int precision = DBI_C64;
  std::vector<dbi_group_member> mem;  // caller's order
  std::vector<GMember> desc;          // tile order
  std::vector<long long> offs;        // [B + 1] field offsets per slot
  int B = 0;
  long long field_elems = 0, T_elems = 0;
  GroupLaunch gl{};
  int ctas[3] = {0, 0, 0};     // persistent CTAs per SM per stage (0 = resident maximum)
  int max_ctas[3] = {0, 0, 0};
  int sms = 0;
  // bound workspace
  void *work = nullptr;
  int op = -1;
  GMember *d_desc = nullptr;
  long long *d_offs = nullptr;
  void *tw = nullptr, *T = nullptr;
  Scales sc{};
  SolverBufs sb{};
};

namespace dbi {

int run_group_operator(const OpArgs &a, cudaStream_t s) {
  return a.precision == DBI_C64 ? run_group_typed<float2>(a, s) : run_group_typed<double2>(a, s);
}

}  // namespace dbi

namespace {

int log2i(int L) {
  int k = 0;
  while ((1 << k) < L) ++k;
  return k;
}

size_t csize(int precision) { return precision == DBI_C64 ? sizeof(float2) : sizeof(double2); }

// Workspace layout shared by bind and the size query.
struct Layout {
  size_t desc, offs, tw, T, scales, solver, total;
};
Layout layout(const dbi_group *g, int op) {
  Layout l{};
  l.desc = align256(g->desc.size() * sizeof(GMember));
  l.offs = align256(g->offs.size() * sizeof(long long));
  l.tw = align256(bytes_twiddles(g->precision));
  l.T = align256(size_t(g->T_elems + g->gl.S_elems) * csize(g->precision));
  l.scales = align256(size_t(g->B) * sizeof(double)) * 3 + 256 + bytes_partials(g->B);
  l.solver = op == DBI_OP_SOLVE ? bytes_solver_fields(size_t(g->field_elems) * csize(g->precision), g->B) : 0;
  l.total = l.desc + l.offs + l.tw + l.T + l.scales + l.solver;
  return l;
}

template <typename C> void stage_smem(dbi_group *g) {
  size_t s[4] = {0, 0, 0, 0};
  for (const GMember &M : g->desc) {  // the members the non-split kernels run
    if (!M.split_rows)
      dispatch_len(M.lx, [&]<int LX>() {
        s[0] = std::max(s[0], rows_forward_smem<C, LX>(M.nx, true));
        s[1] = std::max(s[1], rows_forward_smem<C, LX>(M.nx, false));
        s[3] = std::max(s[3], rows_inverse_smem<C, LX>());
      });
    if (!M.split_cols) dispatch_len(M.lz, [&]<int LZ>() { s[2] = std::max(s[2], cols_smem<C, LZ>()); });
  }
  for (int i = 0; i < 4; ++i) g->gl.smem[i] = s[i];
}

int occupancy(const dbi_group *g, int stage, int epi, size_t smem, int *n) {
  return g->precision == DBI_C64 ? group_occupancy<float2>(stage, epi, smem, n)
                                 : group_occupancy<double2>(stage, epi, smem, n);
}

void set_blocks(dbi_group *g) {
  for (int st = 0; st < 3; ++st) {
    const int per = g->ctas[st] > 0 ? std::min(g->ctas[st], g->max_ctas[st]) : g->max_ctas[st];
    g->gl.blocks[st] = std::max(1, per) * std::max(1, g->sms);
  }
}

int check_group(const dbi_group *g, int need_op) {
  if (!g) { set_error("group plan is NULL"); return DBI_ERR_ARG; }
  if (!g->work || (need_op == DBI_OP_SOLVE && g->op != DBI_OP_SOLVE)) {
    set_error(need_op == DBI_OP_SOLVE ? "group plan needs a DBI_OP_SOLVE bind" : "group plan is not bound");
    return DBI_ERR_WORKSPACE;
  }
  return DBI_OK;
}

OpArgs group_op(const dbi_group *g) {
  OpArgs a{};
  a.precision = g->precision;
  a.B = g->B;
  a.group = &g->gl;
  a.offs = g->d_offs;
  a.T = g->T;
  a.tw = g->tw;
  a.stencil = true;
  return a;
}

int apply_impl(const dbi_group *g, const void *u, void *out, cudaStream_t s) {
  int rc;
  if ((rc = pow2_scales(u, g->precision, false, g->B, 0, g->sc.part, g->sc.scale, g->sc.inv, nullptr, s,
                        g->d_offs)))
    return rc;
  OpArgs a = group_op(g);
  a.in = u; a.ident = u; a.out = out;
  a.in_scale = g->sc.scale; a.out_scale = g->sc.inv;
  return run_operator(a, s);
}

}  // namespace

extern "C" int dbi_group_create(const dbi_group_member *members, int n, int precision, dbi_group **out) {
  clear_error();
  if (!out) { set_error("out is NULL"); return DBI_ERR_ARG; }
  *out = nullptr;
  int rc;
  if ((rc = check_precision(precision))) return rc;
  if (!members || n < 1) { set_error("need at least one member"); return DBI_ERR_ARG; }
  for (int k = 0; k < n; ++k) {
    const dbi_group_member &M = members[k];
    if ((rc = check_grid(&M.model.grid, precision))) return rc;
    if (M.B < 1 || M.nf < 1 || !M.model.m || !M.Ghat || !M.omega || !M.fidx) {
      set_error("member %d needs B >= 1, nf >= 1 and device m, Ghat, omega, fidx", k);
      return DBI_ERR_ARG;
    }
  }
  dbi_group *g = new (std::nothrow) dbi_group;
  if (!g) { set_error("out of host memory"); return DBI_ERR_ARG; }
  g->precision = precision;
  g->mem.assign(members, members + n);
  // slots and field / spectra offsets in the caller's order
  std::vector<int> slot0(n);
  std::vector<long long> f0(n), t0(n), s0(n);
  g->offs.assign(1, 0);
  long long S_elems = 0;
  for (int k = 0; k < n; ++k) {
    const dbi_grid &gr = members[k].model.grid;
    slot0[k] = g->B;
    f0[k] = g->field_elems;
    t0[k] = g->T_elems;
    s0[k] = S_elems;
    for (int q = 0; q < members[k].B; ++q) {
      g->field_elems += 2LL * gr.nz * gr.nx;
      g->offs.push_back(g->field_elems);
    }
    g->T_elems += 2LL * members[k].B * gr.lx * gr.nz;
    if (split_rows(gr.lx, precision)) S_elems += 2LL * members[k].B * gr.nz * gr.nx;
    g->B += members[k].B;
  }
  g->gl.T_elems = g->T_elems;
  g->gl.S_elems = S_elems;
  // tile order: decreasing lx, then lz, then the caller's order
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const dbi_grid &ga = members[a].model.grid, &gb = members[b].model.grid;
    return ga.lx != gb.lx ? ga.lx > gb.lx : ga.lz > gb.lz;
  });
  long long tot[4] = {0, 0, 0, 0};
  g->gl.parts = 1;
  for (int k : order) {
    const dbi_group_member &U = members[k];
    const dbi_grid &gr = U.model.grid;
    GMember M{};
    M.nz = gr.nz; M.nx = gr.nx; M.lz = gr.lz; M.lx = gr.lx;
    M.inv2h = 1.0 / (2.0 * gr.h);
    reference_values(U.model.ref, M.ref);
    M.m = U.model.m; M.Ghat = U.Ghat; M.omega = U.omega; M.fidx = U.fidx;
    M.nf = U.nf; M.B = U.B;
    M.slot0 = slot0[k]; M.field0 = f0[k]; M.T0 = t0[k]; M.S0 = s0[k];
    M.split_rows = split_kind(gr.lx, precision);
    M.split_cols = split_kind(gr.lz, precision);
    g->gl.split_rows |= M.split_rows == kSplitPair;
    g->gl.split_cols |= M.split_cols == kSplitPair;
    g->gl.s3_rows |= M.split_rows == kSplitTriple;
    g->gl.s3_cols |= M.split_cols == kSplitTriple;
    // rows / columns per tile (op_tiles.cuh; op_split.cuh and op_split3.cuh for the split stages,
    // both four rows or columns)
    static_assert(kS3Units == kSplitRows, "split tiles hold the same number of rows or columns");
    const int rows = M.split_rows ? kSplitRows : 2048 / gr.lx, cols = M.split_cols ? kSplitRows : 2048 / gr.lz;
    M.tiles[kStageRowsForward] = M.tiles[kStageRowsInverse] = (gr.nz + rows - 1) / rows;
    M.tiles[kStageCols] = (gr.lx + cols - 1) / cols;
    M.tiles[kStageSource] = M.split_rows ? (gr.nz + kSrcRows - 1) / kSrcRows : 0;
    for (int st = 0; st < 4; ++st) {
      M.tile0[st] = int(tot[st]);
      tot[st] += (long long)M.tiles[st] * U.B;
    }
    g->gl.parts = std::max(g->gl.parts, M.tiles[kStageRowsForward]);
    g->desc.push_back(M);
  }
  if (tot[0] > 0x7fffffffLL || tot[1] > 0x7fffffffLL || tot[3] > 0x7fffffffLL) {
    set_error("group too large: %lld tiles", std::max(tot[0], tot[1]));
    delete g;
    return DBI_ERR_ARG;
  }
  for (int st = 0; st < 4; ++st) g->gl.total[st] = int(tot[st]);
  g->gl.nm = n;
  g->gl.B = g->B;
  if (precision == DBI_C64) stage_smem<float2>(g);
  else stage_smem<double2>(g);
  *out = g;
  return DBI_OK;
}

extern "C" void dbi_group_destroy(dbi_group *g) { delete g; }

extern "C" int dbi_group_slots(const dbi_group *g) { return g ? g->B : 0; }

extern "C" long long dbi_group_field_elems(const dbi_group *g) { return g ? g->field_elems : 0; }

extern "C" int dbi_group_offsets(const dbi_group *g, long long *offs) {
  clear_error();
  if (!g || !offs) { set_error("NULL plan or offs"); return DBI_ERR_ARG; }
  std::copy(g->offs.begin(), g->offs.end(), offs);
  return DBI_OK;
}

extern "C" size_t dbi_group_workspace_bytes(const dbi_group *g, int op) {
  if (!g || (op != DBI_OP_APPLY && op != DBI_OP_SOLVE)) return 0;
  return layout(g, op).total;
}

extern "C" int dbi_group_bind(dbi_group *g, void *work, size_t work_bytes, int op, dbi_stream stream) {
  clear_error();
  if (!g) { set_error("group plan is NULL"); return DBI_ERR_ARG; }
  if (op != DBI_OP_APPLY && op != DBI_OP_SOLVE) { set_error("bind op must be APPLY or SOLVE"); return DBI_ERR_ARG; }
  const Layout l = layout(g, op);
  if (!work || work_bytes < l.total) {
    set_error("work buffer of %zu bytes, need %zu", work_bytes, l.total);
    return DBI_ERR_WORKSPACE;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Arena ar(work, work_bytes);
  // the carves take the sizes of the workspace query's layout, so the two cannot disagree
  g->d_desc = static_cast<GMember *>(ar.take(l.desc));
  g->d_offs = static_cast<long long *>(ar.take(l.offs));
  g->tw = ar.take(l.tw);
  g->T = ar.take(l.T);  // spectra, then the split-row sources
  g->sc = carve_scales(ar, g->B);
  if (op == DBI_OP_SOLVE) g->sb = carve_solver_fields(ar, size_t(g->field_elems) * csize(g->precision), g->B);
  if (const int crc = ar.check("dbi_group_bind")) return crc;
  cudaError_t e = cudaMemcpyAsync(g->d_desc, g->desc.data(), g->desc.size() * sizeof(GMember),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->d_offs, g->offs.data(), g->offs.size() * sizeof(long long), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail("uploading the group descriptors", e);
  int rc;
  if ((rc = launch_twiddles(g->tw, g->precision, s))) return rc;
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail("cudaGetDevice", e);
  if ((e = cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_fail("cudaDeviceGetAttribute", e);
  // resident CTAs per SM of each stage (rows inverse: the smallest over its epilogues)
  int occ[3] = {0, 0, 0}, n = 0;
  if ((rc = occupancy(g, 0, 0, std::max(g->gl.smem[0], g->gl.smem[1]), &n))) return rc;
  occ[0] = n;
  if ((rc = occupancy(g, 1, 0, std::max(g->gl.smem[0], g->gl.smem[1]), &n))) return rc;
  occ[0] = std::min(occ[0], n);
  if ((rc = occupancy(g, 2, 0, g->gl.smem[2], &n))) return rc;
  occ[1] = n;
  occ[2] = 1 << 20;
  for (int epi = 0; epi < 3; ++epi) {
    if ((rc = occupancy(g, 3, epi, g->gl.smem[3], &n))) return rc;
    occ[2] = std::min(occ[2], n);
  }
  for (int st = 0; st < 3; ++st) g->max_ctas[st] = std::max(1, occ[st]);
  if (g->gl.split_rows || g->gl.split_cols || g->gl.s3_rows || g->gl.s3_cols) {
    // the split kernels: the resident maximum per SM
    int sp[7] = {0, 0, 0, 0, 0, 0, 0};
    if ((rc = group_split_occupancy(sp))) return rc;
    for (int i = 0; i < 4; ++i) g->gl.split_blocks[i] = std::max(1, sp[i]) * std::max(1, g->sms);
    for (int i = 0; i < 3; ++i) g->gl.s3_blocks[i] = std::max(1, sp[4 + i]) * std::max(1, g->sms);
  }
  g->gl.desc = g->d_desc;
  set_blocks(g);
  g->work = work;
  g->op = op;
  return DBI_OK;
}

extern "C" int ls_apply_group(const dbi_group *g, const void *u, void *out, dbi_stream stream) {
  clear_error();
  int rc;
  if ((rc = check_group(g, DBI_OP_APPLY))) return rc;
  if (!u || !out || u == out) { set_error("u and out must be distinct non-NULL fields"); return DBI_ERR_ARG; }
  return apply_impl(g, u, out, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int ls_solve_group(const dbi_group *g, const void *rhs, void *u, const dbi_krylov_opts *opts,
                              const dbi_status *status, int flags, dbi_stream stream) {
  clear_error();
  int rc;
  if ((rc = check_group(g, DBI_OP_SOLVE))) return rc;
  if ((rc = check_krylov(opts))) return rc;
  if (!rhs || !u || rhs == u) { set_error("rhs and u must be distinct non-NULL fields"); return DBI_ERR_ARG; }
  OpArgs a = group_op(g);
  return run_bicgstab(a, g->sb, rhs, u, opts->zero_guess != 0, *opts, status, reinterpret_cast<cudaStream_t>(stream),
                      true, (flags & DBI_GROUP_GRAPH) != 0);
}

extern "C" int dbi_group_tune(dbi_group *g, const void *u, void *out, dbi_stream stream, dbi_group_tuning *report) {
  clear_error();
  int rc;
  if ((rc = check_group(g, DBI_OP_APPLY))) return rc;
  if (!u || !out || u == out) { set_error("u and out must be distinct non-NULL fields"); return DBI_ERR_ARG; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) return cuda_fail("tuner: a CUDA error was pending on entry", e);
  // Each candidate: one warm-up apply, then `reps` applies between two stream synchronisations,
  // timed by the host clock (every apply is milliseconds of GPU work, far above the clock's
  // resolution); an error names the candidate that met it.
  const char *what = "tuner: first timing";
  auto time_apply = [&](double *ms) -> int {
    constexpr int reps = 3;
    int r = apply_impl(g, u, out, s);
    if (r) return r;
    cudaError_t ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_fail(what, ce);
    const auto t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < reps && r == DBI_OK; ++i) r = apply_impl(g, u, out, s);
    if (r) return r;
    if ((ce = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(what, ce);
    const auto t1 = std::chrono::steady_clock::now();
    *ms = std::chrono::duration<double, std::milli>(t1 - t0).count() / reps;
    return DBI_OK;
  };
  dbi_group_tuning rep{};
  // FFT lengths present
  std::vector<int> lens;
  for (const GMember &M : g->desc) {
    lens.push_back(M.lx);
    lens.push_back(M.lz);
  }
  std::sort(lens.begin(), lens.end());
  lens.erase(std::unique(lens.begin(), lens.end()), lens.end());
  double best = 0.0;
  rc = time_apply(&best);
  // radix plan per length (coordinate descent: one length at a time, the others fixed)
  for (size_t i = 0; i < lens.size() && rc == DBI_OK && i < 8; ++i) {
    const int L = lens[i], k = log2i(L);
    rep.lengths[i] = L;
    if (L == 64 || L == 512 || L == 768) continue;  // one plan only
    double t[2];
    for (int v = 0; v < 2 && rc == DBI_OK; ++v) {
      g->gl.plan[k] = static_cast<signed char>(v);
      what = v ? "tuner: radix plan 1" : "tuner: radix plan 0";
      rc = time_apply(&t[v]);
    }
    if (rc) break;
    const int pick = t[1] < t[0] ? 1 : 0;
    g->gl.plan[k] = static_cast<signed char>(pick);
    rep.plan[i] = pick;
    rep.plan_ms[i][0] = t[0];
    rep.plan_ms[i][1] = t[1];
    best = t[pick];
  }
  // persistent grid of each stage
  for (int st = 0; st < 3 && rc == DBI_OK; ++st) {
    int pick = g->max_ctas[st];
    for (int c = 1; c <= g->max_ctas[st] && rc == DBI_OK; ++c) {
      g->ctas[st] = c;
      set_blocks(g);
      what = "tuner: persistent grid";
      double t;
      rc = time_apply(&t);
      if (rc == DBI_OK && t < best) {
        best = t;
        pick = c;
      }
    }
    g->ctas[st] = pick;
    set_blocks(g);
    rep.ctas_per_sm[st] = pick;
    rep.max_ctas[st] = g->max_ctas[st];
  }
  if (rc) return rc;
  what = "tuner: final timing";
  rc = time_apply(&rep.apply_ms);
  if (report) *report = rep;
  return rc;
}

extern "C" int dbi_set_radix_plan(int precision, int L, int plan) {
  clear_error();
  int rc;
  if ((rc = check_precision(precision))) return rc;
  if (!fft_len_ok(L) || (plan != 0 && plan != 1)) {
    set_error("radix plan needs L a power of two in [16, 1024] and plan 0 or 1");
    return DBI_ERR_ARG;
  }
  set_radix_plan(precision, L, plan);
  return DBI_OK;
}
