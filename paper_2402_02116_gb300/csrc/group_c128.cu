// Persistent uneven-batch operator kernels instantiated for double2 (one translation unit per
// precision so that the two compile in parallel).
#include <algorithm>

#include "group_kernels.cuh"

namespace dbi {
template int run_group_typed<double2>(const OpArgs &a, cudaStream_t s);
template int group_occupancy<double2>(int stage, int epi, size_t smem, int *per_sm);
}  // namespace dbi
