// Run-time choices of the operator kernels, set by the autotuner (tune.cu) and read at launch.
#pragma once

namespace dbi {

// Radix plan (0 or 1, see fft_reg.cuh) of FFT length L in the given precision; 0 until tuned.
int radix_plan(int precision, int L);
void set_radix_plan(int precision, int L, int plan);

}  // namespace dbi
