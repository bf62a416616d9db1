// Batched BiCGSTAB for the LS equation A u = u0 (Eq. 11), one independent system per
// (source, frequency) problem.
//
// Per iteration i (van der Vorst's BiCGSTAB, <a, b> = sum conj(a) b):
//   p = r + beta (p - omega v)                  k_update_p      (beta from the previous k_check)
//   v = A p, partials of <rhat, v>              operator (inner product in k_rows_inverse)
//   alpha = rho / <rhat, v>                     k_alpha         (one warp per problem)
//   s = r - alpha v                             k_update_s      (+ partials of ||s||^2)
//   t = A s, partials of <t, s>, <t, t>         operator (inner products in k_rows_inverse)
//   omega = <t,s>/<t,t>                         k_omega         (one warp per problem)
//   x += alpha p + omega s, r = s - omega t     k_update_xr     (+ partials of <rhat, r>, ||r||^2)
//   convergence, breakdown, beta = (rho_new / rho)(alpha / omega)  k_check
// Every scalar lives on the device in FP64. Each reduction is two-stage and deterministic: each
// thread sums its elements, the CTA sums its threads in a fixed tree, and every consumer sums the
// kRedBlocks CTA partials of its problem in the same fixed order. Converged problems drop out
// (their CTAs return at once); the host polls an active-problem counter every check_every
// iterations. A breakdown (rho or omega vanishing) restarts the problem from its iterate.
#include <cmath>

#include "group.cuh"
#include "krylov.cuh"
#include "reduce.cuh"
#include "vec.cuh"

namespace dbi {

// Largest |component| of every problem's array (real and imaginary parts of complex values):
// comparisons only, so nothing underflows whatever the scale of the values (a data residual of
// 1e-12 back-propagates to fields of 1e-21, whose squares would underflow FP32).
// The running maximum stays in the element's real type (FP32 comparisons for complex64 data);
// only the CTA's result is widened to FP64.
__device__ __forceinline__ float absmax(float v) { return fabsf(v); }
__device__ __forceinline__ double absmax(double v) { return fabs(v); }
__device__ __forceinline__ float absmax(float2 v) { return fmaxf(fabsf(v.x), fabsf(v.y)); }
__device__ __forceinline__ double absmax(double2 v) { return fmax(fabs(v.x), fabs(v.y)); }

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_absmax(Span sp, const T *x, double *part) {
  const int b = blockIdx.y;
  decltype(absmax(T{})) m = 0;
  DBI_PROBLEM_LOOP(sp) m = fmax(m, absmax(x[off + i]));
  block_max_store(double(m), part + (size_t(b) * kRedBlocks + blockIdx.x) * kRedSlots);
}

// Power-of-two scale per problem that brings max |rhs| into [1, 2); the solver iterates on the
// scaled system (exact in any precision) and unscales the solution at the end.
__global__ void k_scale(KState *st, const double *part) {
  const double m = gather_max(part + size_t(blockIdx.x) * kRedBlocks * kRedSlots, kRedBlocks);
  if (threadIdx.x == 0) st[blockIdx.x].scale = pow2_below(m);
}

// x *= scale (inverse = 0) or x /= scale (inverse = 1)
template <typename C>
__global__ void k_scale_x(Span sp, const KState *st, C *x, int inverse) {
  const int b = blockIdx.y;
  using R = typename RealOf<C>::type;
  const double sc = st[blockIdx.y].scale;
  const R f = R(inverse ? 1.0 / sc : sc);
  DBI_PROBLEM_LOOP(sp) x[off + i] = cscale(x[off + i], f);
}

template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_init(Span sp, const KState *st, const C *__restrict__ rhs,
                                                      C *__restrict__ v, C *__restrict__ r,
                                                      C *__restrict__ rhat, C *__restrict__ p,
                                                      C *__restrict__ x, int x_zero, double *part) {
  const int b = blockIdx.y;
  using A = typename Acc<C>::type;
  using R = typename RealOf<C>::type;
  const R sc = R(st[blockIdx.y].scale);
  A bb = 0, rr = 0;
  DBI_PROBLEM_LOOP(sp) {
    const C bi = cscale(rhs[off + i], sc);
    const C ax = x_zero ? czero<C>() : v[off + i];
    const C ri = csub(bi, ax);
    r[off + i] = ri;
    rhat[off + i] = ri;
    p[off + i] = czero<C>();
    v[off + i] = czero<C>();
    if (x_zero) x[off + i] = czero<C>();
    bb += bi.x * bi.x + bi.y * bi.y;
    rr += ri.x * ri.x + ri.y * ri.y;
  }
  A acc[2] = {bb, rr};
  block_sum_store<2>(acc, part + (size_t(b) * kRedBlocks + blockIdx.x) * kRedSlots);
}

__global__ void k_init_state(KState *st, int *active, int *counters, const double *part, double tol,
                             int max_iter) {
  const int b = blockIdx.x;
  double s[2];
  gather_n<2>(part + size_t(b) * kRedBlocks * kRedSlots, kRedBlocks, s);
  if (threadIdx.x == 0) {
    KState k{};
    k.scale = st[b].scale;
    k.bnorm2 = s[0];
    k.rnorm2 = s[1];
    k.rho_re = s[1]; k.rho_im = 0.0;  // rhat = r
    k.alpha_re = 1.0; k.om_re = 1.0;
    k.beta_re = 0.0; k.beta_im = 0.0;  // p = r on the first iteration (p = v = 0)
    k.rhatnorm2 = s[1];
    k.zero_rhs = s[0] == 0.0;
    const bool bad = !finite_value(s[0]) || !finite_value(s[1]);  // NaN or infinity in the right-hand side or x0
    const bool conv = !bad && (k.zero_rhs || s[1] <= tol * tol * s[0]);
    k.code = bad ? DBI_NONFINITE : conv ? DBI_CONVERGED : DBI_NOT_CONVERGED;
    st[b] = k;
    const int act = (!bad && !conv && max_iter > 0) ? 1 : 0;
    active[b] = act;
    atomicAdd(&counters[1], act);
  }
}

template <typename C>
__global__ void k_zero_flagged(Span sp, const KState *st, C *x) {
  const int b = blockIdx.y;
  if (!st[blockIdx.y].zero_rhs) return;
  DBI_PROBLEM_LOOP(sp) x[off + i] = czero<C>();
}

template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_update_p(Span sp, const int *plist, const KState *st,
                                                          const int *active, int *counters, int parity,
                                                          const C *__restrict__ r, C *__restrict__ rhat,
                                                          C *__restrict__ p, const C *__restrict__ v) {
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) counters[parity] = 0;
  const int b = problem_at(plist, blockIdx.y);
  if (!active[b]) return;
  const KState k = st[b];
  if (k.restart) {
    problem_loop_pairs<C>(sp, b, [&]<int N>(size_t o) {
      C ri[N];
      ldN(r + o, ri);
      stN(rhat + o, ri);
      stN(p + o, ri);
    });
    return;
  }
  const C be = from_z<C>(make_double2(k.beta_re, k.beta_im));
  const C om = from_z<C>(make_double2(k.om_re, k.om_im));
  problem_loop_pairs<C>(sp, b, [&]<int N>(size_t o) {
    C pi[N], vi[N], ri[N];
    ldN(p + o, pi);
    ldN(v + o, vi);
    ldN(r + o, ri);
#pragma unroll
    for (int n = 0; n < N; ++n) pi[n] = cadd(ri[n], cmul(be, csub(pi[n], cmul(om, vi[n]))));
    stN(p + o, pi);
  });
}

// alpha = rho / <rhat, A p> of every active problem, from the operator's fused partials, once
// per problem (one warp each) so that the s update starts streaming at once.
__global__ void k_alpha(const int *plist, KState *st, const int *active, int nparts, const double *partA) {
  const int b = problem_at(plist, blockIdx.x);
  if (!active[b]) return;
  double sg[2];
  gather_n<2>(partA + size_t(b) * nparts * kRedSlots, nparts, sg);
  if (threadIdx.x == 0) {
    const double2 sigma = make_double2(sg[0], sg[1]);
    const double2 alpha = (sigma.x == 0.0 && sigma.y == 0.0)
                              ? make_double2(0.0, 0.0)
                              : zdiv(make_double2(st[b].rho_re, st[b].rho_im), sigma);
    st[b].alpha_re = alpha.x;
    st[b].alpha_im = alpha.y;
  }
}

template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_update_s(Span sp, const int *plist, const KState *st,
                                                          const int *active, const C *__restrict__ r,
                                                          const C *__restrict__ v, C *__restrict__ s,
                                                          double *partS) {
  using A = typename Acc<C>::type;
  const int b = problem_at(plist, blockIdx.y);
  if (!active[b]) return;
  const C al = from_z<C>(make_double2(st[b].alpha_re, st[b].alpha_im));
  A ss = 0;
  problem_loop_pairs<C>(sp, b, [&]<int N>(size_t o) {
    C ri[N], vi[N];
    ldN(r + o, ri);
    ldN(v + o, vi);
#pragma unroll
    for (int n = 0; n < N; ++n) {
      ri[n] = csub(ri[n], cmul(al, vi[n]));
      ss += ri[n].x * ri[n].x + ri[n].y * ri[n].y;
    }
    stN(s + o, ri);
  });
  A acc[1] = {ss};
  block_sum_store<1>(acc, partS + (size_t(b) * kRedBlocks + blockIdx.x) * kRedSlots);
}

// omega = <t, s> / ||t||^2 (zero when the half step already met tol) of every active problem,
// once per problem (one warp each), from the second operator pass's partials and ||s||^2.
__global__ void k_omega(const int *plist, KState *st, const int *active, int nparts, const double *partB,
                        const double *partS, double tol) {
  const int b = problem_at(plist, blockIdx.x);
  if (!active[b]) return;
  double q[3], sn[1];
  gather_n<3>(partB + size_t(b) * nparts * kRedSlots, nparts, q);
  gather_n<1>(partS + size_t(b) * kRedBlocks * kRedSlots, kRedBlocks, sn);
  if (threadIdx.x == 0) {
    const int half = sn[0] <= tol * tol * st[b].bnorm2;
    const double2 om = (half || q[2] == 0.0) ? make_double2(0.0, 0.0)
                                             : make_double2(q[0] / q[2], q[1] / q[2]);
    st[b].om_re = om.x;
    st[b].om_im = om.y;
    st[b].half = half;
    st[b].snorm2 = sn[0];
  }
}

template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_update_xr(Span sp, const int *plist, const KState *st,
                                                           const int *active, const C *__restrict__ p,
                                                           const C *__restrict__ s, const C *__restrict__ t,
                                                           const C *__restrict__ rhat, C *__restrict__ x,
                                                           C *__restrict__ r, double *partC) {
  using A = typename Acc<C>::type;
  const int b = problem_at(plist, blockIdx.y);
  if (!active[b]) return;
  const KState k = st[b];
  const C al = from_z<C>(make_double2(k.alpha_re, k.alpha_im));
  const C o = from_z<C>(make_double2(k.om_re, k.om_im));
  A re = 0, im = 0, rr = 0;
  problem_loop_pairs<C>(sp, b, [&]<int N>(size_t e) {
    C si[N], xi[N], pi[N], ti[N], hi[N];
    ldN(s + e, si);
    ldN(x + e, xi);
    ldN(p + e, pi);
    ldN(t + e, ti);
    ldN(rhat + e, hi);
#pragma unroll
    for (int n = 0; n < N; ++n) {
      xi[n] = cadd(xi[n], cadd(cmul(al, pi[n]), cmul(o, si[n])));
      const C ri = csub(si[n], cmul(o, ti[n]));
      si[n] = ri;  // (reused as the new residual)
      re += hi[n].x * ri.x + hi[n].y * ri.y;
      im += hi[n].x * ri.y - hi[n].y * ri.x;
      rr += ri.x * ri.x + ri.y * ri.y;
    }
    stN(x + e, xi);
    stN(r + e, si);
  });
  A acc[3] = {re, im, rr};
  block_sum_store<3>(acc, partC + (size_t(b) * kRedBlocks + blockIdx.x) * kRedSlots);
}

// Convergence test, breakdown restart and beta for the next iteration (one CTA per problem;
// the decision itself is bicgstab_decide in krylov.cuh).
__global__ void k_check(const int *plist, KState *st, int *active, int *counters, int parity,
                        const double *partC, double tol, int max_iter) {
  const int b = problem_at(plist, blockIdx.x);
  if (!active[b]) return;
  double q[3];
  gather_n<3>(partC + size_t(b) * kRedBlocks * kRedSlots, kRedBlocks, q);
  if (threadIdx.x != 0) return;
  KState k = st[b];
  const int act = bicgstab_decide(k, q, tol, max_iter);
  st[b] = k;
  active[b] = act;
  atomicAdd(&counters[parity], act);
}

// plist = the active problems in ascending order, count = how many (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024) k_compact(int B, const int *active, int *plist, int *count) {
  __shared__ int warp_tot[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c0 = 0; c0 < B; c0 += blockDim.x) {
    const int i = c0 + threadIdx.x;
    const int a = (i < B && active[i]) ? 1 : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, a);
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += warp_tot[w];
    if (a) plist[base + before + __popc(bal & ((1u << lane) - 1u))] = i;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < int(blockDim.x >> 5); ++w) tot += warp_tot[w];
      base += tot;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base;
}

int compact_active(int B, const int *active, int *plist, int *count, cudaStream_t s) {
  k_compact<<<1, 1024, 0, s>>>(B, active, plist, count);
  return check_launch("k_compact");
}

__global__ void k_finalize(int B, const KState *st, int *iters, double *relres, int *code) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const KState k = st[b];
  if (iters) iters[b] = k.iters;
  if (relres) relres[b] = k.bnorm2 > 0 ? sqrt(k.rnorm2 / k.bnorm2) : 0.0;
  if (code) code[b] = k.code;
}

// ---------------------------------------------------------------------------------------------
// power-of-two normalisers
// ---------------------------------------------------------------------------------------------
__global__ void k_pow2(const double *part, double *scale, double *inv, const double *extra) {
  const double m = gather_max(part + size_t(blockIdx.x) * kRedBlocks * kRedSlots, kRedBlocks);
  if (threadIdx.x == 0) {
    const double sc = pow2_below(m);
    scale[blockIdx.x] = sc;
    if (inv) inv[blockIdx.x] = 1.0 / (sc * (extra ? extra[0] : 1.0));
  }
}

int pow2_scales(const void *x, int precision, bool real, int B, size_t n, double *part, double *scale,
                double *inv, const double *extra, cudaStream_t s, const long long *offs) {
  const dim3 grid(kRedBlocks, B);
  const Span sp{n, offs};
  if (precision == DBI_C64) {
    if (real) k_absmax<float><<<grid, kRedThreads, 0, s>>>(sp, static_cast<const float *>(x), part);
    else k_absmax<float2><<<grid, kRedThreads, 0, s>>>(sp, static_cast<const float2 *>(x), part);
  } else {
    if (real) k_absmax<double><<<grid, kRedThreads, 0, s>>>(sp, static_cast<const double *>(x), part);
    else k_absmax<double2><<<grid, kRedThreads, 0, s>>>(sp, static_cast<const double2 *>(x), part);
  }
  int rc;
  if ((rc = check_launch("k_absmax"))) return rc;
  k_pow2<<<B, 32, 0, s>>>(part, scale, inv, extra);
  return check_launch("k_pow2");
}

size_t bytes_solver_fields(size_t field_bytes, int B) {
  return 6 * align256(field_bytes) + align256(size_t(B) * sizeof(KState)) + 2 * align256(size_t(B) * sizeof(int)) +
         256 + 4 * bytes_partials(B);
}
size_t bytes_solver(const dbi_grid *g, int B, int precision) {
  return bytes_solver_fields(bytes_field(g, B, precision), B);
}

SolverBufs carve_solver_fields(Arena &ar, size_t f, int B) {
  SolverBufs sb{};
  sb.r = ar.take(f); sb.rhat = ar.take(f); sb.p = ar.take(f);
  sb.v = ar.take(f); sb.s = ar.take(f); sb.t = ar.take(f);
  sb.st = static_cast<KState *>(ar.take(size_t(B) * sizeof(KState)));
  sb.active = static_cast<int *>(ar.take(size_t(B) * sizeof(int)));
  sb.counters = static_cast<int *>(ar.take(256));
  sb.plist = static_cast<int *>(ar.take(size_t(B) * sizeof(int)));
  sb.partA = static_cast<double *>(ar.take(bytes_partials(B)));
  sb.partS = static_cast<double *>(ar.take(bytes_partials(B)));
  sb.partB = static_cast<double *>(ar.take(bytes_partials(B)));
  sb.partC = static_cast<double *>(ar.take(bytes_partials(B)));
  return sb;
}
SolverBufs carve_solver(Arena &ar, const dbi_grid *g, int B, int precision) {
  return carve_solver_fields(ar, bytes_field(g, B, precision), B);
}

static int read_counter(const int *dev, cudaStream_t s, int *host) {
  cudaError_t e = cudaMemcpyAsync(host, dev, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? DBI_OK : cuda_fail("reading the active-problem counter", e);
}

// Owns a capture stream, a captured graph and its executable instance.
struct GraphChunk {
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~GraphChunk() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
  }
};

template <typename C>
static int bicgstab_typed(OpArgs op, const SolverBufs &sb, const void *rhs_, void *x_, bool x_zero,
                          const dbi_krylov_opts &o, const dbi_status *status, cudaStream_t s, bool unscale,
                          bool use_graph) {
  const int B = op.B;
  if (B == 0) return DBI_OK;
  const bool group = op.group != nullptr;
  const Span sp{group ? 0 : size_t(2) * op.nz * op.nx, op.offs};
  const C *rhs = static_cast<const C *>(rhs_);
  C *x = static_cast<C *>(x_);
  C *r = static_cast<C *>(sb.r), *rhat = static_cast<C *>(sb.rhat), *p = static_cast<C *>(sb.p);
  C *v = static_cast<C *>(sb.v), *sv = static_cast<C *>(sb.s), *t = static_cast<C *>(sb.t);
  const dim3 grid(kRedBlocks, B);
  int rc;
  cudaError_t e = cudaMemsetAsync(sb.counters, 0, 3 * sizeof(int), s);
  if (e != cudaSuccess) return cuda_fail("cudaMemsetAsync(counters)", e);
  const int nparts = group    ? group_parts(op.group)
                     : op.Dhat ? operator_parts_k(op.nz, op.lx, op.precision)
                               : operator_parts(op.nz, op.lx, op.precision);
  op.stencil = true;
  op.active = nullptr;
  k_absmax<C><<<grid, kRedThreads, 0, s>>>(sp, rhs, sb.partA);
  if ((rc = check_launch("k_absmax"))) return rc;
  k_scale<<<B, 32, 0, s>>>(sb.st, sb.partA);
  if ((rc = check_launch("k_scale"))) return rc;
  if (!x_zero) {  // x0 into the scaled system, v = A x0
    k_scale_x<C><<<grid, kRedThreads, 0, s>>>(sp, sb.st, x, 0);
    if ((rc = check_launch("k_scale_x"))) return rc;
    op.in = x; op.ident = x; op.out = v;
    if ((rc = run_operator(op, s))) return rc;
  }
  k_init<C><<<grid, kRedThreads, 0, s>>>(sp, sb.st, rhs, v, r, rhat, p, x, x_zero ? 1 : 0, sb.partA);
  if ((rc = check_launch("k_init"))) return rc;
  k_init_state<<<B, 32, 0, s>>>(sb.st, sb.active, sb.counters, sb.partA, o.tol, o.max_iter);
  if ((rc = check_launch("k_init_state"))) return rc;
  if (!x_zero) {
    k_zero_flagged<C><<<grid, kRedThreads, 0, s>>>(sp, sb.st, x);
    if ((rc = check_launch("k_zero_flagged"))) return rc;
  }
  // Batches on one grid run their launches over the problems still active: at every host check
  // the active problems are compacted into sb.plist (ascending order) and the grids shrink to them.
  // Uneven batches keep every problem in the launches (finished ones return at once).
  int nact = B;   // problems still active (read back at host checks)
  int nrun = B;   // launch slots: the compacted active problems, or every problem of an uneven batch
  const int *plist = nullptr;
  auto compact = [&]() -> int {
    k_compact<<<1, 1024, 0, s>>>(B, sb.active, sb.plist, sb.counters + 2);
    int e2 = check_launch("k_compact");
    if (e2 == DBI_OK) e2 = read_counter(sb.counters + 2, s, &nact);
    plist = sb.plist;
    nrun = nact;
    return e2;
  };
  if (!group && o.check_every > 0 && (rc = compact())) return rc;
  op.active = sb.active;
  op.krhat = rhat;
  if (group) {  // members write only their own row tiles of the fused-reduction partials: zero the rest
    e = cudaMemsetAsync(sb.partA, 0, bytes_partials(B), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sb.partB, 0, bytes_partials(B), s);
    if (e != cudaSuccess) return cuda_fail("cudaMemsetAsync(partials)", e);
  }
  // One BiCGSTAB iteration of every active problem on stream `st`.
  auto iterate = [&](int it, cudaStream_t st) -> int {
    const int parity = it & 1;
    const dim3 g2(kRedBlocks, nrun);
    int rc2;
    op.plist = plist;
    op.nb = nrun;
    k_update_p<C><<<g2, kRedThreads, 0, st>>>(sp, plist, sb.st, sb.active, sb.counters, parity, r, rhat, p, v);
    if ((rc2 = check_launch("k_update_p"))) return rc2;
    op.epi = 1; op.in = p; op.ident = p; op.out = v; op.part_out = sb.partA;
    if ((rc2 = run_operator(op, st))) return rc2;
    k_alpha<<<nrun, 32, 0, st>>>(plist, sb.st, sb.active, nparts, sb.partA);
    if ((rc2 = check_launch("k_alpha"))) return rc2;
    k_update_s<C><<<g2, kRedThreads, 0, st>>>(sp, plist, sb.st, sb.active, r, v, sv, sb.partS);
    if ((rc2 = check_launch("k_update_s"))) return rc2;
    op.epi = 2; op.in = sv; op.ident = sv; op.out = t; op.part_out = sb.partB;
    if ((rc2 = run_operator(op, st))) return rc2;
    k_omega<<<nrun, 32, 0, st>>>(plist, sb.st, sb.active, nparts, sb.partB, sb.partS, o.tol);
    if ((rc2 = check_launch("k_omega"))) return rc2;
    k_update_xr<C><<<g2, kRedThreads, 0, st>>>(sp, plist, sb.st, sb.active, p, sv, t, rhat, x, r, sb.partC);
    if ((rc2 = check_launch("k_update_xr"))) return rc2;
    k_check<<<nrun, 32, 0, st>>>(plist, sb.st, sb.active, sb.counters, parity, sb.partC, o.tol, o.max_iter);
    return check_launch("k_check");
  };
  const int K = o.check_every;
  if (group && use_graph && K > 0) {
    // Capture K iterations once (on a capture stream of our own: the caller's stream may be the
    // legacy default stream, which cannot be captured) and replay the graph on the caller's
    // stream until every problem has stopped; the host reads the active count between replays.
    GraphChunk gc;
    if ((e = cudaStreamCreateWithFlags(&gc.cs, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail("cudaStreamCreateWithFlags", e);
    if ((e = cudaStreamBeginCapture(gc.cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_fail("cudaStreamBeginCapture", e);
    int crc = DBI_OK;
    const unsigned long long before = launch_count();
    for (int k = 0; k < K && crc == DBI_OK; ++k) crc = iterate(k, gc.cs);
    const unsigned long long captured = launch_count() - before;  // kernels per replay
    e = cudaStreamEndCapture(gc.cs, &gc.graph);
    if (crc) return crc;
    if (e != cudaSuccess) return cuda_fail("cudaStreamEndCapture", e);
    if ((e = cudaGraphInstantiate(&gc.exec, gc.graph, 0)) != cudaSuccess) return cuda_fail("cudaGraphInstantiate", e);
    add_launches(0 - captured);  // capturing launched nothing; every replay below launches them
    for (int it = 0; it < o.max_iter && nact > 0; it += K) {
      if ((e = cudaGraphLaunch(gc.exec, s)) != cudaSuccess) return cuda_fail("cudaGraphLaunch", e);
      add_launches(captured);
      if ((rc = read_counter(sb.counters + ((K - 1) & 1), s, &nact))) return rc;
    }
  } else {
    for (int it = 0; it < o.max_iter && nact > 0; ++it) {
      if ((rc = iterate(it, s))) return rc;
      if (K > 0 && ((it + 1) % K == 0)) {
        if (!group) rc = compact();
        else rc = read_counter(sb.counters + (it & 1), s, &nact);
        if (rc) return rc;
      }
    }
  }
  op.plist = nullptr;
  if (unscale) {
    k_scale_x<C><<<grid, kRedThreads, 0, s>>>(sp, sb.st, x, 1);
    if ((rc = check_launch("k_scale_x"))) return rc;
  }
  if (status) {
    k_finalize<<<(B + 127) / 128, 128, 0, s>>>(B, sb.st, status->iters, status->relres, status->code);
    if ((rc = check_launch("k_finalize"))) return rc;
  }
  return DBI_OK;
}

int run_bicgstab(OpArgs op, const SolverBufs &sb, const void *rhs, void *x, bool x_zero,
                 const dbi_krylov_opts &o, const dbi_status *status, cudaStream_t s, bool unscale,
                 bool use_graph) {
  return op.precision == DBI_C64 ? bicgstab_typed<float2>(op, sb, rhs, x, x_zero, o, status, s, unscale, use_graph)
                                 : bicgstab_typed<double2>(op, sb, rhs, x, x_zero, o, status, s, unscale, use_graph);
}

int check_krylov(const dbi_krylov_opts *o) {
  if (!o || !(o->tol >= 0) || o->max_iter < 0 || o->check_every < 0) {
    set_error("Krylov options need tol >= 0, max_iter >= 0, check_every >= 0");
    return DBI_ERR_ARG;
  }
  return DBI_OK;
}

}  // namespace dbi

using namespace dbi;

extern "C" int ls_solve(const dbi_model *model, const dbi_batch *batch, const void *Ghat,
                        const void *rhs, void *u, const dbi_krylov_opts *opts,
                        const dbi_status *status, int precision, void *work, size_t work_bytes,
                        dbi_stream stream) {
  clear_error();
  int rc;
  if (!model) { set_error("model is NULL"); return DBI_ERR_ARG; }
  const dbi_grid *g = &model->grid;
  if ((rc = check_grid(g, precision)) || (rc = check_batch(batch)) || (rc = check_precision(precision)) ||
      (rc = check_krylov(opts)))
    return rc;
  if (batch->B == 0) return DBI_OK;
  if (!model->m || !Ghat || !rhs || !u) { set_error("NULL model, Ghat, rhs or u"); return DBI_ERR_ARG; }
  if (rhs == u) { set_error("rhs and u must be distinct buffers"); return DBI_ERR_ARG; }
  const size_t need = dbi_workspace_bytes(g, batch->B, precision, DBI_OP_SOLVE);
  if (!work || work_bytes < need) {
    set_error("work buffer of %zu bytes, need %zu", work_bytes, need);
    return DBI_ERR_WORKSPACE;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Arena ar(work, work_bytes);
  void *tw = ar.take(bytes_twiddles(precision));
  void *T = ar.take(bytes_spectral(g, batch->B, precision));
  SolverBufs sb = carve_solver(ar, g, batch->B, precision);
  if ((rc = ar.check("ls_solve"))) return rc;
  if ((rc = launch_twiddles(tw, precision, s))) return rc;
  OpArgs a{};
  a.precision = precision; a.nz = g->nz; a.nx = g->nx; a.lz = g->lz; a.lx = g->lx; a.h = g->h;
  a.B = batch->B; a.nf = batch->nf; a.omega = batch->omega; a.fidx = batch->fidx;
  a.m = model->m; reference_values(model->ref, a.ref);
  a.T = T; a.Ghat = Ghat; a.tw = tw;
  return run_bicgstab(a, sb, rhs, u, opts->zero_guess != 0, *opts, status, s, true);
}
