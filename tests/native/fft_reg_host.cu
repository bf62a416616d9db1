// Host run of the register-resident FFT plans (fft_reg.cuh), for the CPU test suite.
//
// The plans are __host__ __device__ code that a line's L/8 threads run together, meeting at a
// barrier between the shared-memory stores and loads of every exchange. Here each of those
// threads is a std::thread, the line's shared memory a host buffer and the barrier a
// std::barrier, so the exact code of the GPU kernels runs on the CPU: every length, both radix
// orders, forward (with and without the zero-half first pass) and inverse, complex64 and
// complex128. The line buffer carries guard slots on both sides that must stay untouched.
//
// Lines per thread group: 1, and 2, 3 and 4 (the kernels transform a column's components together,
// sharing the twiddle powers; at FFT length 1024 the column stage runs both parities of both
// components, four 512-point lines, through one exchange set), each line with its own input.
//
// Usage: fft_reg_host <out.bin>. For every line the file holds a header of six int32 values
// (precision bytes, L, V, INV, HIN, lines of the group) followed by the input and the output of
// that line as complex128 (the input as the plan saw it, after rounding to the precision).
#include <barrier>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <thread>
#include <vector>

#include "../../paper_2402_02116_gb300/csrc/fft_reg.cuh"

using namespace dbi;

namespace {

struct HostSync {
  std::barrier<> *bar;
  void operator()() const { bar->arrive_and_wait(); }
};

constexpr int kGuard = 64;

template <typename C> std::vector<C> twiddle_table() {
  std::vector<C> tw(kTwiddleN);
  for (int m = 0; m < kTwiddleN; ++m) {
    const double a = -2.0 * M_PI * double(m) / double(kTwiddleN);
    tw[m].x = decltype(tw[m].x)(std::cos(a));
    tw[m].y = decltype(tw[m].y)(std::sin(a));
  }
  return tw;
}

// Seeded input of one case (a 64-bit LCG; points >= L/2 zero when HIN).
template <typename C> std::vector<C> make_input(int L, bool hin, uint64_t seed) {
  std::vector<C> x(L);
  uint64_t s = seed * 6364136223846793005ULL + 1442695040888963407ULL;
  auto next = [&]() {
    s = s * 6364136223846793005ULL + 1442695040888963407ULL;
    return double((s >> 11) & ((1ULL << 53) - 1)) / double(1ULL << 53) * 2.0 - 1.0;
  };
  for (int i = 0; i < L; ++i) {
    const double re = next(), im = next();
    x[i].x = decltype(x[i].x)((hin && i >= L / 2) ? 0.0 : re);
    x[i].y = decltype(x[i].y)((hin && i >= L / 2) ? 0.0 : im);
  }
  return x;
}

template <typename C, int L, int V, bool INV, bool HIN, int NLT = 1>
bool run_case(FILE *f, const std::vector<C> &tw, uint64_t seed) {
  constexpr int T = L / 8, LP = RegFFT<C, L>::LP, SPAN = LP + 2 * kGuard;
  std::vector<std::vector<C>> in(NLT), out(NLT, std::vector<C>(L));
  for (int l = 0; l < NLT; ++l) in[l] = make_input<C>(L, HIN, seed * 8 + l);
  std::vector<C> buf(size_t(NLT) * SPAN);  // each line between its own guards
  const double sentinel = 1.0e30;
  for (auto &c : buf) { c.x = decltype(c.x)(sentinel); c.y = decltype(c.y)(-sentinel); }
  std::barrier<> bar(T);
  std::vector<std::thread> threads;
  threads.reserve(T);
  for (int t = 0; t < T; ++t) {
    threads.emplace_back([&, t] {
      const TwReg<C, L, V> tr(t, tw.data());
      C v[NLT][8];
      C *lines_[NLT];
      for (int l = 0; l < NLT; ++l) {
        lines_[l] = buf.data() + size_t(l) * SPAN + kGuard;
        for (int m = 0; m < 8; ++m) v[l][m] = in[l][t + m * T];
      }
      C *const(&lines)[NLT] = lines_;
      RegPlan<L, V>::template run<C, NLT, INV, HIN>(v, lines, t, tr, HostSync{&bar});
      for (int l = 0; l < NLT; ++l)
        for (int m = 0; m < 8; ++m) out[l][t + m * T] = v[l][m];
    });
  }
  for (auto &th : threads) th.join();
  for (int l = 0; l < NLT; ++l)
    for (int i = 0; i < kGuard; ++i) {
      const C a = buf[size_t(l) * SPAN + i], b = buf[size_t(l) * SPAN + kGuard + LP + i];
      if (a.x != decltype(a.x)(sentinel) || b.x != decltype(b.x)(sentinel)) {
        std::fprintf(stderr, "guard overwritten: L=%d V=%d INV=%d HIN=%d NLT=%d\n", L, V, int(INV), int(HIN), NLT);
        return false;
      }
    }
  for (int l = 0; l < NLT; ++l) {
    const int32_t hdr[6] = {int32_t(sizeof(C)), L, V, int32_t(INV), int32_t(HIN), NLT};
    std::fwrite(hdr, sizeof(hdr), 1, f);
    const std::vector<C> *both[2] = {&in[l], &out[l]};
    for (const std::vector<C> *vec : both)
      for (const C &c : *vec) {
        const double z[2] = {double(c.x), double(c.y)};
        std::fwrite(z, sizeof(z), 1, f);
      }
  }
  return true;
}

template <typename C, int L> bool run_length(FILE *f, const std::vector<C> &tw, uint64_t &seed) {
  bool ok = true;
  ok &= run_case<C, L, 0, false, false>(f, tw, ++seed);
  ok &= run_case<C, L, 0, false, true>(f, tw, ++seed);
  ok &= run_case<C, L, 0, true, false>(f, tw, ++seed);
  ok &= run_case<C, L, 1, false, false>(f, tw, ++seed);
  ok &= run_case<C, L, 1, false, true>(f, tw, ++seed);
  ok &= run_case<C, L, 1, true, false>(f, tw, ++seed);
  ok &= run_case<C, L, 0, false, true, 2>(f, tw, ++seed);
  ok &= run_case<C, L, 1, true, false, 2>(f, tw, ++seed);
  ok &= run_case<C, L, 0, false, true, 3>(f, tw, ++seed);
  ok &= run_case<C, L, 0, true, false, 3>(f, tw, ++seed);
  ok &= run_case<C, L, 0, false, false, 4>(f, tw, ++seed);
  ok &= run_case<C, L, 0, true, false, 4>(f, tw, ++seed);
  return ok;
}

template <typename C> bool run_all(FILE *f, uint64_t &seed) {
  const std::vector<C> tw = twiddle_table<C>();
  bool ok = true;
  ok &= run_length<C, 16>(f, tw, seed);
  ok &= run_length<C, 32>(f, tw, seed);
  ok &= run_length<C, 64>(f, tw, seed);
  ok &= run_length<C, 128>(f, tw, seed);
  ok &= run_length<C, 256>(f, tw, seed);
  ok &= run_length<C, 512>(f, tw, seed);
  ok &= run_length<C, 1024>(f, tw, seed);
  return ok;
}

}  // namespace

int main(int argc, char **argv) {
  if (argc != 2) {
    std::fprintf(stderr, "usage: %s <out.bin>\n", argv[0]);
    return 2;
  }
  FILE *f = std::fopen(argv[1], "wb");
  if (!f) return 2;
  uint64_t seed = 0;
  const bool ok = run_all<float2>(f, seed) && run_all<double2>(f, seed);
  std::fclose(f);
  return ok ? 0 : 1;
}
