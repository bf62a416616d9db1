// Batched restarted GMRES(m) for the LS equation A u = u0 (Eq. 11), the Krylov method of the
// paper's experiments; one independent system per (source, frequency) problem.
//
// A cycle (Saad and Schultz's GMRES, <a, b> = sum conj(a) b) from the iterate x:
//   v_0 = (b - A x) / beta, beta = ||b - A x||      operator + k_gm_residual, k_gm_begin, k_gm_scale_v
//   step j = 0 .. m-1 (every problem still active):
//     w = K v_j (A = I - K)                          operator without its identity term, into the
//                                                     slot of v_(j+1); then column j of H for A is
//                                                     e_j - <V, K v_j> and v_(j+1) = -w' / ||w'||
//     classical Gram-Schmidt                          k_gm_dots (h_i = <v_i, w>, ||w||^2), k_gm_hsum,
//                                                     k_gm_update (w -= sum h_i v_i, ||w||^2)
//     a second round where the first one removed     k_gm_need2, then the same three kernels
//       more than half of the norm (Kahan-Parlett: ||w'|| < 0.7 ||w||; "twice is enough").
//       Orthogonalising K v_j rather than A v_j = v_j - K v_j (the same Krylov space) keeps the
//       first round from cancelling the v_j component that dominates A v_j, so the second round
//       is rarely needed.
//     h_(j+1,j) = ||w||, plane rotations on the new Hessenberg column, the minimal residual
//       |g_(j+1)|, convergence and iteration limits   k_gm_close
//     v_(j+1) = -w' / h_(j+1,j)                      k_gm_scale_v
//   y from the triangular system R y = g, x += V y   k_gm_solve_y, k_gm_update_x
// The basis vectors are stored in the precision of the operator; the Hessenberg matrix, the
// rotations, every inner product and norm are FP64 and every reduction is two-stage and
// deterministic. The system is scaled by a power of two per problem (max |rhs| in [1, 2)) so that
// FP32 fields stay in range, and the solution is scaled back at the end. Problems that stop
// (converged or out of iterations) drop out of the launches at the next host check.
#include <cmath>

#include "krylov.cuh"
#include "reduce.cuh"
#include "vec.cuh"

namespace dbi {

constexpr int kDotGroup = 8;  // basis vectors per CTA of the inner-product pass
constexpr int kDotGroups = kGmresMaxRestart / kDotGroup;

struct GState {
  double bnorm2;  // ||scaled rhs||^2
  double res;     // minimal residual |g_(k+1)| of the current cycle (scaled system)
  double hn_inv;  // -1 / h_(j+1,j) of the last step (1 / beta at the start of a cycle)
  int iters;      // Arnoldi steps so far
  int code;
  int k;          // steps of the current cycle
  int kx;         // steps of the finished cycle to fold into x
  int incycle, zero_rhs;
  double wpre2;  // ||A v_j||^2 before the Gram-Schmidt rounds
  int need2;     // this step re-orthogonalises
  int pad;
};

constexpr int kDotSlots = 2 * kDotGroup + 2;  // per partial: 8 complex inner products, ||w||^2, pad

struct GmresBufs {
  void *V;         // [m + 1][B][n] basis vectors
  GState *st;      // [B]
  double2 *H;      // [B][m + 1][m] Hessenberg matrix, triangular after the rotations
  double2 *g;      // [B][m + 1] rotated right-hand side beta e_1
  double *cs;      // [B][m] rotation cosines
  double2 *sn;     // [B][m] rotation sines
  double2 *hc;     // [B][m + 1] coefficients of the current Gram-Schmidt round
  double2 *y;      // [B][m] cycle solution
  double *scale;   // [B] power-of-two scale of the system
  double *partD;   // [B][kDotGroups][kRedBlocks][kDotSlots] inner-product partials
  double *partN;   // [B][kRedBlocks][kRedSlots] norm partials
  int *active, *plist, *count;
};

// f: bytes of one field of the whole batch (B problems), 256-aligned.
size_t gmres_bytes_fields(size_t f, int B, int m) {
  const size_t small = align256(size_t(B) * sizeof(GState)) + align256(size_t(B) * (m + 1) * m * sizeof(double2)) +
                       2 * align256(size_t(B) * (m + 1) * sizeof(double2)) +
                       align256(size_t(B) * m * sizeof(double)) + 2 * align256(size_t(B) * m * sizeof(double2)) +
                       align256(size_t(B) * sizeof(double));
  const size_t parts = align256(size_t(B) * kDotGroups * kRedBlocks * kDotSlots * sizeof(double)) +
                       bytes_partials(B);
  return size_t(m + 1) * f + small + parts + 2 * align256(size_t(B) * sizeof(int)) + 256;
}

static GmresBufs carve_gmres(Arena &ar, size_t f, int B, int m) {
  GmresBufs gb{};
  gb.V = ar.take(size_t(m + 1) * f);
  gb.st = static_cast<GState *>(ar.take(size_t(B) * sizeof(GState)));
  gb.H = static_cast<double2 *>(ar.take(size_t(B) * (m + 1) * m * sizeof(double2)));
  gb.g = static_cast<double2 *>(ar.take(size_t(B) * (m + 1) * sizeof(double2)));
  gb.hc = static_cast<double2 *>(ar.take(size_t(B) * (m + 1) * sizeof(double2)));
  gb.cs = static_cast<double *>(ar.take(size_t(B) * m * sizeof(double)));
  gb.sn = static_cast<double2 *>(ar.take(size_t(B) * m * sizeof(double2)));
  gb.y = static_cast<double2 *>(ar.take(size_t(B) * m * sizeof(double2)));
  gb.scale = static_cast<double *>(ar.take(size_t(B) * sizeof(double)));
  gb.partD = static_cast<double *>(ar.take(size_t(B) * kDotGroups * kRedBlocks * kDotSlots * sizeof(double)));
  gb.partN = static_cast<double *>(ar.take(bytes_partials(B)));
  gb.active = static_cast<int *>(ar.take(size_t(B) * sizeof(int)));
  gb.plist = static_cast<int *>(ar.take(size_t(B) * sizeof(int)));
  gb.count = static_cast<int *>(ar.take(256));
  return gb;
}

// x *= scale (inverse = 0) or x /= scale (inverse = 1)
template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_gm_scale_x(Span sp, const double *scale, C *x, int inverse) {
  using R = typename RealOf<C>::type;
  const int b = blockIdx.y;
  const R f = R(inverse ? 1.0 / scale[b] : scale[b]);
  DBI_PROBLEM_LOOP(sp) x[off + i] = cscale(x[off + i], f);
}

// v0 = scale rhs - (A x if have_ax, held in v0) for the problems flagged in `live` (all when
// NULL); partials of ||scale rhs||^2 and ||v0||^2. A zero initial guess is written into x0z when
// it is non-NULL.
template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_gm_residual(Span sp, const int *live, const double *scale,
                                                             const C *__restrict__ rhs, C *__restrict__ v0,
                                                             int have_ax, C *__restrict__ x0z, double *part) {
  using A = typename Acc<C>::type;
  using R = typename RealOf<C>::type;
  const int b = blockIdx.y;
  if (live && !live[b]) return;
  const R sc = R(scale[b]);
  A bb = 0, rr = 0;
  DBI_PROBLEM_LOOP(sp) {
    const C bi = cscale(rhs[off + i], sc);
    const C ri = have_ax ? csub(bi, v0[off + i]) : bi;
    v0[off + i] = ri;
    if (x0z) x0z[off + i] = czero<C>();
    bb += bi.x * bi.x + bi.y * bi.y;
    rr += ri.x * ri.x + ri.y * ri.y;
  }
  A acc[2] = {bb, rr};
  block_sum_store<2>(acc, part + (size_t(b) * kRedBlocks + blockIdx.x) * kRedSlots);
}

// Start of a cycle (one CTA per problem): beta, the convergence test on the true residual, and
// g = beta e_1. On the first cycle every problem is initialised; later only active ones restart.
__global__ void k_gm_begin(GState *st, int *active, double2 *g, const double *part, double tol, int max_iter,
                           int first, int m) {
  const int b = blockIdx.x;
  if (!first && !active[b]) return;
  double s[2];
  gather_n<2>(part + size_t(b) * kRedBlocks * kRedSlots, kRedBlocks, s);
  if (threadIdx.x != 0) return;
  GState k = first ? GState{} : st[b];
  if (first) {
    k.bnorm2 = s[0];
    k.zero_rhs = s[0] == 0.0;
  }
  const double beta = sqrt(s[1]);
  k.res = beta;
  k.k = 0;
  int act = 0;
  if (!finite_value(k.bnorm2) || !finite_value(s[1])) {  // NaN or infinity in the data, the model or the iterate
    k.code = DBI_NONFINITE;
  } else if (k.zero_rhs || s[1] <= tol * tol * k.bnorm2) {
    k.code = DBI_CONVERGED;
  } else if (k.iters >= max_iter) {
    k.code = DBI_NOT_CONVERGED;
  } else {
    k.code = DBI_NOT_CONVERGED;
    k.incycle = 1;
    k.hn_inv = 1.0 / beta;
    double2 *gb = g + size_t(b) * (m + 1);
    gb[0] = make_double2(beta, 0.0);
    for (int i = 1; i <= m; ++i) gb[i] = make_double2(0.0, 0.0);
    act = 1;
  }
  st[b] = k;
  active[b] = act;
}

template <typename C>
__global__ void k_gm_zero_flagged(Span sp, const GState *st, C *x) {
  const int b = blockIdx.y;
  if (!st[b].zero_rhs) return;
  DBI_PROBLEM_LOOP(sp) x[off + i] = czero<C>();
}

// v *= hn_inv (the new basis vector normalised), active problems of the launch list.
template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_gm_scale_v(Span sp, const int *plist, const int *active,
                                                            const GState *st, C *v) {
  using R = typename RealOf<C>::type;
  const int b = problem_at(plist, blockIdx.y);
  if (!active[b]) return;
  const R f = R(st[b].hn_inv);
  DBI_PROBLEM_LOOP(sp) v[off + i] = cscale(v[off + i], f);
}

// Partials of h_i = <v_i, w> for the basis vectors i of group blockIdx.z (i <= j), w = v_(j+1),
// and (group 0 of the first pass) of ||w||^2. The second Gram-Schmidt pass (round = 1) runs only
// for the problems that re-orthogonalise.
template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_gm_dots(Span sp, const int *plist, const int *active,
                                                         const GState *st, const C *__restrict__ V,
                                                         size_t vstride, int j, int round, double *partD) {
  using A = typename Acc<C>::type;
  const int b = problem_at(plist, blockIdx.y);
  if (!active[b] || (round == 1 && !st[b].need2)) return;
  const int i0 = blockIdx.z * kDotGroup;
  const int nv = min(kDotGroup, j + 1 - i0);
  const bool norm = round == 0 && blockIdx.z == 0;
  const C *w = V + size_t(j + 1) * vstride;
  A re[kDotGroup], im[kDotGroup], ww = 0;
#pragma unroll
  for (int q = 0; q < kDotGroup; ++q) re[q] = im[q] = 0;
  const size_t off = sp.offset(b), cnt = sp.count(b);
  if (sizeof(C) == sizeof(float2) && ((off | cnt) & 1) == 0) {
    // complex64 in pairs: one 16-byte load per vector and pair (half the load instructions)
    const size_t np = cnt / 2, step = size_t(gridDim.x) * blockDim.x;
    const float4 *w4 = reinterpret_cast<const float4 *>(w + off);
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < np; i += step) {
      const float4 wi = w4[i];
      float4 v[kDotGroup];
#pragma unroll
      for (int q = 0; q < kDotGroup; ++q)
        v[q] = q < nv ? reinterpret_cast<const float4 *>(V + size_t(i0 + q) * vstride + off)[i]
                      : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int q = 0; q < kDotGroup; ++q) {  // conj(v) w of both points
        re[q] += v[q].x * wi.x + v[q].y * wi.y + v[q].z * wi.z + v[q].w * wi.w;
        im[q] += v[q].x * wi.y - v[q].y * wi.x + v[q].z * wi.w - v[q].w * wi.z;
      }
      if (norm) ww += wi.x * wi.x + wi.y * wi.y + wi.z * wi.z + wi.w * wi.w;
    }
  } else {
    DBI_PROBLEM_LOOP(sp) {
      const C wi = w[off + i];
      C v[kDotGroup];
#pragma unroll
      for (int q = 0; q < kDotGroup; ++q) v[q] = q < nv ? V[size_t(i0 + q) * vstride + off + i] : czero<C>();
#pragma unroll
      for (int q = 0; q < kDotGroup; ++q) {
        re[q] += v[q].x * wi.x + v[q].y * wi.y;  // conj(v) w
        im[q] += v[q].x * wi.y - v[q].y * wi.x;
      }
      if (norm) ww += wi.x * wi.x + wi.y * wi.y;
    }
  }
  A acc[kDotSlots];
#pragma unroll
  for (int q = 0; q < kDotGroup; ++q) {
    acc[2 * q] = re[q];
    acc[2 * q + 1] = im[q];
  }
  acc[2 * kDotGroup] = ww;
  acc[2 * kDotGroup + 1] = 0;
  block_sum_store<kDotSlots>(acc, partD + ((size_t(b) * kDotGroups + blockIdx.z) * kRedBlocks + blockIdx.x) * kDotSlots);
}

// h_i = <v_i, K v_j> (i <= j) from the partials, in a fixed order; hc[b][i] = h_i and column j
// of the Hessenberg matrix of A = I - K gets delta_ij - h_i (first pass) or -h_i more (second pass);
// the first pass also stores ||K v_j||^2. One CTA of 2 kGmresMaxRestart + 32 threads per problem.
__global__ void k_gm_hsum(const int *plist, const int *active, GState *st, const double *partD, double2 *hc,
                          double2 *H, int j, int round, int m) {
  const int b = problem_at(plist, blockIdx.x);
  if (!active[b] || (round == 1 && !st[b].need2)) return;
  const int t = threadIdx.x;
  if (t == 2 * kGmresMaxRestart) {
    if (round == 0) {
      const double *p = partD + size_t(b) * kDotGroups * kRedBlocks * kDotSlots + 2 * kDotGroup;
      double a = 0.0;
      for (int blk = 0; blk < kRedBlocks; ++blk) a += p[size_t(blk) * kDotSlots];
      st[b].wpre2 = a;
    }
    return;
  }
  const int i = t >> 1, comp = t & 1;
  if (i > j) return;
  const double *p = partD + (size_t(b) * kDotGroups + i / kDotGroup) * kRedBlocks * kDotSlots + 2 * (i % kDotGroup) +
                    comp;
  double a = 0.0;
  for (int blk = 0; blk < kRedBlocks; ++blk) a += p[size_t(blk) * kDotSlots];
  double *h = reinterpret_cast<double *>(hc + size_t(b) * (m + 1) + i) + comp;
  *h = a;
  double *Hij = reinterpret_cast<double *>(H + (size_t(b) * (m + 1) + i) * m + j) + comp;
  *Hij = round == 0 ? ((i == j && comp == 0) ? 1.0 : 0.0) - a : *Hij - a;
}

// w -= sum_(i <= j) h_i v_i, partials of ||w||^2. The basis vectors are read eight at a time so
// that their loads are in flight together.
template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_gm_update(Span sp, const int *plist, const int *active,
                                                           const GState *st, C *__restrict__ V, size_t vstride,
                                                           int j, int round, const double2 *hc, int m,
                                                           double *partN) {
  using A = typename Acc<C>::type;
  __shared__ C h[kGmresMaxRestart + kDotGroup];
  const int b = problem_at(plist, blockIdx.y);
  if (!active[b] || (round == 1 && !st[b].need2)) return;
  for (int i = threadIdx.x; i < kGmresMaxRestart + kDotGroup; i += blockDim.x)
    h[i] = i <= j ? from_z<C>(hc[size_t(b) * (m + 1) + i]) : czero<C>();
  __syncthreads();
  C *w = V + size_t(j + 1) * vstride;
  A ww = 0;
  const size_t off = sp.offset(b), cnt = sp.count(b);
  if (sizeof(C) == sizeof(float2) && ((off | cnt) & 1) == 0) {
    // complex64 in pairs: one 16-byte load per vector and pair
    const size_t np = cnt / 2, step = size_t(gridDim.x) * blockDim.x;
    float4 *w4 = reinterpret_cast<float4 *>(w + off);
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < np; i += step) {
      float4 wi = w4[i];
      for (int q0 = 0; q0 <= j; q0 += kDotGroup) {
        float4 v[kDotGroup];
#pragma unroll
        for (int u = 0; u < kDotGroup; ++u)
          v[u] = q0 + u <= j ? reinterpret_cast<const float4 *>(V + size_t(q0 + u) * vstride + off)[i]
                             : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < kDotGroup; ++u) {
          const float2 hu = reinterpret_cast<const float2 &>(h[q0 + u]);
          wi.x -= hu.x * v[u].x - hu.y * v[u].y;
          wi.y -= hu.x * v[u].y + hu.y * v[u].x;
          wi.z -= hu.x * v[u].z - hu.y * v[u].w;
          wi.w -= hu.x * v[u].w + hu.y * v[u].z;
        }
      }
      w4[i] = wi;
      ww += wi.x * wi.x + wi.y * wi.y + wi.z * wi.z + wi.w * wi.w;
    }
  } else {
    DBI_PROBLEM_LOOP(sp) {
      C wi = w[off + i];
      for (int q0 = 0; q0 <= j; q0 += kDotGroup) {
        C v[kDotGroup];
#pragma unroll
        for (int u = 0; u < kDotGroup; ++u)
          v[u] = q0 + u <= j ? V[size_t(q0 + u) * vstride + off + i] : czero<C>();
#pragma unroll
        for (int u = 0; u < kDotGroup; ++u) wi = csub(wi, cmul(h[q0 + u], v[u]));
      }
      w[off + i] = wi;
      ww += wi.x * wi.x + wi.y * wi.y;
    }
  }
  A acc[1] = {ww};
  block_sum_store<1>(acc, partN + (size_t(b) * kRedBlocks + blockIdx.x) * kRedSlots);
}

// After the first round: re-orthogonalise when ||w'||^2 < 0.49 ||w||^2 (one CTA per problem).
__global__ void k_gm_need2(const int *plist, const int *active, GState *st, const double *partN) {
  const int b = problem_at(plist, blockIdx.x);
  if (!active[b]) return;
  double s[1];
  gather_n<1>(partN + size_t(b) * kRedBlocks * kRedSlots, kRedBlocks, s);
  if (threadIdx.x == 0) st[b].need2 = s[0] < 0.49 * st[b].wpre2;
}

// End of step j (one CTA per problem): h_(j+1,j) = ||w||, the earlier rotations on column j, a
// new rotation that annihilates h_(j+1,j), the rotated right-hand side and its last entry, the
// minimal residual. Stops the problem when it is below tol ||b||, when the new basis vector
// vanishes (the solution lies in the space built so far), or at the iteration limit.
__global__ void k_gm_close(const int *plist, int *active, GState *st, double2 *H, double2 *g, double *cs,
                           double2 *sn, const double *partN, int j, int m, double tol, int max_iter) {
  const int b = problem_at(plist, blockIdx.x);
  if (!active[b]) return;
  double s[1];
  gather_n<1>(partN + size_t(b) * kRedBlocks * kRedSlots, kRedBlocks, s);
  if (threadIdx.x != 0) return;
  GState k = st[b];
  const double hn = sqrt(s[0]);
  double2 *Hb = H + size_t(b) * (m + 1) * m;
  double *cb = cs + size_t(b) * m;
  double2 *sb = sn + size_t(b) * m;
  double2 *gb = g + size_t(b) * (m + 1);
  for (int i = 0; i < j; ++i) {  // (h_i, h_(i+1)) <- (c h_i + s h_(i+1), -conj(s) h_i + c h_(i+1))
    const double2 a0 = Hb[size_t(i) * m + j], a1 = Hb[size_t(i + 1) * m + j];
    const double c = cb[i];
    const double2 sv = sb[i];
    Hb[size_t(i) * m + j] = make_double2(c * a0.x + sv.x * a1.x - sv.y * a1.y, c * a0.y + sv.x * a1.y + sv.y * a1.x);
    Hb[size_t(i + 1) * m + j] =
        make_double2(-(sv.x * a0.x + sv.y * a0.y) + c * a1.x, -(sv.x * a0.y - sv.y * a0.x) + c * a1.y);
  }
  // rotation of (a, hn), hn real >= 0: c = |a| / t, s = (a / |a|) hn / t, r = (a / |a|) t
  const double2 a = Hb[size_t(j) * m + j];
  const double aa = hypot(a.x, a.y), t = hypot(aa, hn);
  double c;
  double2 sv, r;
  if (hn == 0.0) {
    c = 1.0; sv = make_double2(0.0, 0.0); r = a;
  } else if (aa == 0.0) {
    c = 0.0; sv = make_double2(1.0, 0.0); r = make_double2(hn, 0.0);
  } else {
    const double2 ph = make_double2(a.x / aa, a.y / aa);
    c = aa / t; sv = make_double2(ph.x * hn / t, ph.y * hn / t); r = make_double2(ph.x * t, ph.y * t);
  }
  cb[j] = c;
  sb[j] = sv;
  Hb[size_t(j) * m + j] = r;
  const double2 gj = gb[j];
  gb[j + 1] = make_double2(-(sv.x * gj.x + sv.y * gj.y), -(sv.x * gj.y - sv.y * gj.x));  // -conj(s) g_j
  gb[j] = make_double2(c * gj.x, c * gj.y);
  k.res = hypot(gb[j + 1].x, gb[j + 1].y);
  k.iters += 1;
  k.k = j + 1;
  k.hn_inv = hn > 0.0 ? -1.0 / hn : 0.0;  // v_(j+1) = (A v_j - sum H_ij v_i) / hn = -w' / hn
  int act = 1;
  if (!finite_value(k.res) || !finite_value(hn)) {
    k.code = DBI_NONFINITE;
    act = 0;
  } else if (k.res <= tol * sqrt(k.bnorm2) || hn <= 1e-14 * t) {
    k.code = DBI_CONVERGED;
    act = 0;
  } else if (k.iters >= max_iter) {
    k.code = DBI_NOT_CONVERGED;
    act = 0;
  }
  st[b] = k;
  active[b] = act;
}

// End of a cycle: y from R y = g by back substitution for every problem that ran this cycle.
__global__ void k_gm_solve_y(int B, GState *st, const double2 *H, const double2 *g, double2 *y, int m) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  GState k = st[b];
  k.kx = k.incycle ? k.k : 0;
  k.incycle = 0;
  st[b] = k;
  const double2 *Hb = H + size_t(b) * (m + 1) * m;
  const double2 *gb = g + size_t(b) * (m + 1);
  double2 *yb = y + size_t(b) * m;
  for (int i = k.kx - 1; i >= 0; --i) {
    double2 acc = gb[i];
    for (int l = i + 1; l < k.kx; ++l) {
      const double2 p = zmul(Hb[size_t(i) * m + l], yb[l]);
      acc.x -= p.x;
      acc.y -= p.y;
    }
    yb[i] = zdiv(acc, Hb[size_t(i) * m + i]);
  }
}

// x += sum_(i < kx) y_i v_i
template <typename C>
__global__ void __launch_bounds__(kRedThreads) k_gm_update_x(Span sp, const GState *st, const C *__restrict__ V,
                                                             size_t vstride, const double2 *y, int m,
                                                             C *__restrict__ x) {
  __shared__ C c[kGmresMaxRestart + kDotGroup];
  const int b = blockIdx.y;
  const int kx = st[b].kx;
  if (kx == 0) return;
  for (int i = threadIdx.x; i < kGmresMaxRestart + kDotGroup; i += blockDim.x)
    c[i] = i < kx ? from_z<C>(y[size_t(b) * m + i]) : czero<C>();
  __syncthreads();
  DBI_PROBLEM_LOOP(sp) {
    C xi = x[off + i];
    for (int q0 = 0; q0 < kx; q0 += kDotGroup) {
      C v[kDotGroup];
#pragma unroll
      for (int u = 0; u < kDotGroup; ++u) v[u] = q0 + u < kx ? V[size_t(q0 + u) * vstride + off + i] : czero<C>();
#pragma unroll
      for (int u = 0; u < kDotGroup; ++u) xi = cadd(xi, cmul(c[q0 + u], v[u]));
    }
    x[off + i] = xi;
  }
}

__global__ void k_gm_finalize(int B, const GState *st, int *iters, double *relres, int *code) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const GState k = st[b];
  if (iters) iters[b] = k.iters;
  if (relres) relres[b] = k.bnorm2 > 0 ? k.res / sqrt(k.bnorm2) : 0.0;
  if (code) code[b] = k.code;
}

static int read_int(const int *dev, cudaStream_t s, int *host) {
  cudaError_t e = cudaMemcpyAsync(host, dev, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? DBI_OK : cuda_fail("reading the active-problem count", e);
}

template <typename C>
static int gmres_typed(OpArgs op, const GmresBufs &gb, int m, const void *rhs_, void *x_, bool x_zero,
                       const dbi_krylov_opts &o, const dbi_status *status, cudaStream_t s) {
  const int B = op.B;
  const size_t n = field_elems(op);
  const Span sp{n, nullptr};
  const size_t vstride = size_t(B) * n;
  const C *rhs = static_cast<const C *>(rhs_);
  C *x = static_cast<C *>(x_);
  C *V = static_cast<C *>(gb.V);
  auto Vj = [&](int j) { return V + size_t(j) * vstride; };
  const dim3 all(kRedBlocks, B);
  int rc;
  op.stencil = true;
  op.epi = 0;
  op.active = nullptr;
  op.plist = nullptr;
  op.nb = B;
  if ((rc = pow2_scales(rhs, op.precision, false, B, n, gb.partN, gb.scale, nullptr, nullptr, s))) return rc;
  if (!x_zero) {
    k_gm_scale_x<C><<<all, kRedThreads, 0, s>>>(sp, gb.scale, x, 0);
    if ((rc = check_launch("k_gm_scale_x"))) return rc;
  }
  int nact = B, nrun = B;
  const int *plist = nullptr;
  auto compact = [&]() -> int {
    int e2 = compact_active(B, gb.active, gb.plist, gb.count, s);
    if (e2 == DBI_OK) e2 = read_int(gb.count, s, &nact);
    plist = gb.plist;
    nrun = nact;
    return e2;
  };
  const int K = o.check_every;
  for (bool first = true;; first = false) {
    // residual of the problems that (re)start a cycle
    if (first && x_zero) {
      k_gm_residual<C><<<all, kRedThreads, 0, s>>>(sp, nullptr, gb.scale, rhs, Vj(0), 0, x, gb.partN);
    } else {
      op.plist = first ? nullptr : plist;
      op.nb = first ? B : nrun;
      op.active = first ? nullptr : gb.active;
      op.in = x; op.ident = x; op.out = Vj(0);
      if ((rc = run_operator(op, s))) return rc;
      k_gm_residual<C><<<all, kRedThreads, 0, s>>>(sp, first ? nullptr : gb.active, gb.scale, rhs, Vj(0), 1,
                                                   static_cast<C *>(nullptr), gb.partN);
    }
    if ((rc = check_launch("k_gm_residual"))) return rc;
    k_gm_begin<<<B, 32, 0, s>>>(gb.st, gb.active, gb.g, gb.partN, o.tol, o.max_iter, first ? 1 : 0, m);
    if ((rc = check_launch("k_gm_begin"))) return rc;
    if (first && !x_zero) {
      k_gm_zero_flagged<C><<<all, kRedThreads, 0, s>>>(sp, gb.st, x);
      if ((rc = check_launch("k_gm_zero_flagged"))) return rc;
    }
    if ((rc = compact())) return rc;
    if (nact == 0) break;
    k_gm_scale_v<C><<<dim3(kRedBlocks, nrun), kRedThreads, 0, s>>>(sp, plist, gb.active, gb.st, Vj(0));
    if ((rc = check_launch("k_gm_scale_v"))) return rc;
    for (int j = 0; j < m; ++j) {
      const dim3 g2(kRedBlocks, nrun);
      op.plist = plist; op.nb = nrun; op.active = gb.active;
      op.in = Vj(j); op.ident = nullptr; op.out = Vj(j + 1);  // K v_j
      if ((rc = run_operator(op, s))) return rc;
      for (int round = 0; round < 2; ++round) {
        if (round == 1) {
          k_gm_need2<<<nrun, 32, 0, s>>>(plist, gb.active, gb.st, gb.partN);
          if ((rc = check_launch("k_gm_need2"))) return rc;
        }
        const dim3 g3(kRedBlocks, nrun, (j + 1 + kDotGroup - 1) / kDotGroup);
        k_gm_dots<C><<<g3, kRedThreads, 0, s>>>(sp, plist, gb.active, gb.st, V, vstride, j, round, gb.partD);
        if ((rc = check_launch("k_gm_dots"))) return rc;
        k_gm_hsum<<<nrun, 2 * kGmresMaxRestart + 32, 0, s>>>(plist, gb.active, gb.st, gb.partD, gb.hc, gb.H, j,
                                                             round, m);
        if ((rc = check_launch("k_gm_hsum"))) return rc;
        k_gm_update<C><<<g2, kRedThreads, 0, s>>>(sp, plist, gb.active, gb.st, V, vstride, j, round, gb.hc, m,
                                                  gb.partN);
        if ((rc = check_launch("k_gm_update"))) return rc;
      }
      k_gm_close<<<nrun, 32, 0, s>>>(plist, gb.active, gb.st, gb.H, gb.g, gb.cs, gb.sn, gb.partN, j, m, o.tol,
                                     o.max_iter);
      if ((rc = check_launch("k_gm_close"))) return rc;
      if (j + 1 < m) {
        k_gm_scale_v<C><<<g2, kRedThreads, 0, s>>>(sp, plist, gb.active, gb.st, Vj(j + 1));
        if ((rc = check_launch("k_gm_scale_v"))) return rc;
      }
      if (j + 1 == m || (K > 0 && (j + 1) % K == 0)) {
        if ((rc = compact())) return rc;
        if (nact == 0) break;
      }
    }
    k_gm_solve_y<<<(B + 127) / 128, 128, 0, s>>>(B, gb.st, gb.H, gb.g, gb.y, m);
    if ((rc = check_launch("k_gm_solve_y"))) return rc;
    k_gm_update_x<C><<<all, kRedThreads, 0, s>>>(sp, gb.st, V, vstride, gb.y, m, x);
    if ((rc = check_launch("k_gm_update_x"))) return rc;
    if (nact == 0) break;
  }
  k_gm_scale_x<C><<<all, kRedThreads, 0, s>>>(sp, gb.scale, x, 1);
  if ((rc = check_launch("k_gm_scale_x"))) return rc;
  if (status) {
    k_gm_finalize<<<(B + 127) / 128, 128, 0, s>>>(B, gb.st, status->iters, status->relres, status->code);
    if ((rc = check_launch("k_gm_finalize"))) return rc;
  }
  return DBI_OK;
}

int run_gmres(const OpArgs &op, Arena &ar, size_t field_bytes, int m, const void *rhs, void *x, bool x_zero,
              const dbi_krylov_opts &o, const dbi_status *status, cudaStream_t s) {
  const GmresBufs gb = carve_gmres(ar, field_bytes, op.B, m);
  const int rc = ar.check("GMRES");
  if (rc) return rc;
  return op.precision == DBI_C64 ? gmres_typed<float2>(op, gb, m, rhs, x, x_zero, o, status, s)
                                 : gmres_typed<double2>(op, gb, m, rhs, x, x_zero, o, status, s);
}

}  // namespace dbi

using namespace dbi;

extern "C" size_t dbi_gmres_workspace_bytes(const dbi_grid *g, int B, int precision, int restart) {
  if (!g || check_grid(g, precision) || check_precision(precision) || B < 0 || restart < 1 || restart > kGmresMaxRestart)
    return 0;
  return bytes_twiddles(precision) + bytes_spectral(g, B, precision) +
         gmres_bytes_fields(bytes_field(g, B, precision), B, restart);
}

extern "C" int ls_solve_gmres(const dbi_model *model, const dbi_batch *batch, const void *Ghat, const void *rhs,
                              void *u, const dbi_krylov_opts *opts, int restart, const dbi_status *status,
                              int precision, void *work, size_t work_bytes, dbi_stream stream) {
  clear_error();
  int rc;
  if (!model) { set_error("model is NULL"); return DBI_ERR_ARG; }
  const dbi_grid *g = &model->grid;
  if ((rc = check_grid(g, precision)) || (rc = check_batch(batch)) || (rc = check_precision(precision)) ||
      (rc = check_krylov(opts)))
    return rc;
  if (restart < 1 || restart > kGmresMaxRestart) {
    set_error("restart length %d outside [1, %d]", restart, kGmresMaxRestart);
    return DBI_ERR_ARG;
  }
  if (batch->B == 0) return DBI_OK;
  if (!model->m || !Ghat || !rhs || !u) { set_error("NULL model, Ghat, rhs or u"); return DBI_ERR_ARG; }
  if (rhs == u) { set_error("rhs and u must be distinct buffers"); return DBI_ERR_ARG; }
  const size_t need = dbi_gmres_workspace_bytes(g, batch->B, precision, restart);
  if (!work || work_bytes < need) {
    set_error("work buffer of %zu bytes, need %zu", work_bytes, need);
    return DBI_ERR_WORKSPACE;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Arena ar(work, work_bytes);
  void *tw = ar.take(bytes_twiddles(precision));
  void *T = ar.take(bytes_spectral(g, batch->B, precision));
  if ((rc = ar.check("ls_solve_gmres"))) return rc;
  if ((rc = launch_twiddles(tw, precision, s))) return rc;
  OpArgs a{};
  a.precision = precision; a.nz = g->nz; a.nx = g->nx; a.lz = g->lz; a.lx = g->lx; a.h = g->h;
  a.B = batch->B; a.nf = batch->nf; a.omega = batch->omega; a.fidx = batch->fidx;
  a.m = model->m; reference_values(model->ref, a.ref);
  a.T = T; a.Ghat = Ghat; a.tw = tw;
  return run_gmres(a, ar, bytes_field(g, batch->B, precision), restart, rhs, u, opts->zero_guess != 0, *opts,
                   status, s);
}
