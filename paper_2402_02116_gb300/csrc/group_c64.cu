// Persistent uneven-batch operator kernels instantiated for float2 (one translation unit per
// precision so that the two compile in parallel).
#include <algorithm>

#include "group_kernels.cuh"

namespace dbi {
template int run_group_typed<float2>(const OpArgs &a, cudaStream_t s);
template int group_occupancy<float2>(int stage, int epi, size_t smem, int *per_sm);
int group_split_occupancy(int per_sm[7]) { return group_split_occupancy_impl<float2>(per_sm); }
}  // namespace dbi
