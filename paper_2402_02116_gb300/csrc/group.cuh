// Internal description of an uneven batch (dbi_group.h): member descriptors on the device and
// the persistent launches of the three operator stages over the tiles of every member.
#pragma once

#include "operator.cuh"

namespace dbi {

enum { kStageRowsForward = 0, kStageCols = 1, kStageRowsInverse = 2 };

// One member, as the kernels see it (device array in tile order: members by decreasing lx, lz).
struct GMember {
  int nz, nx, lz, lx;
  double inv2h;
  double ref[5];
  const void *m;        // [5][nz][nx] real
  const void *Ghat;     // [nf][3][lx][lz] complex
  const double *omega;  // [nf]
  const int *fidx;      // [B] table of each of the member's slots
  int nf, B;
  int slot0;            // global index of the member's first slot
  long long field0;     // element offset of the first slot's field
  long long T0;         // element offset of the first slot's spectra
  int tile0[3];         // first tile of the member in each stage's tile space
  int tiles[3];         // tiles per slot in each stage
};

// Host-side launch description (lives in the plan; passed through OpArgs::group).
struct GroupLaunch {
  const GMember *desc;   // device [nm]
  int nm;
  int B;                 // slots
  int total[3];          // tiles per stage
  size_t smem[4];        // dynamic shared memory: rows forward with stencil, without, cols, rows inverse
  int blocks[3];         // persistent CTAs of each stage's launch
  int parts;             // fused-reduction partials per slot (largest row-tile count)
  signed char plan[11];  // radix plan per log2 of the FFT length
};

inline int group_parts(const GroupLaunch *g) { return g->parts; }

// Launches the three stages for the group in `a.group` (precision-specific, group_c64.cu /
// group_c128.cu).
template <typename C> int run_group_typed(const OpArgs &a, cudaStream_t s);
// Resident CTAs per SM of one stage's kernel with `smem` bytes (stage: 0 rows forward with
// stencil, 1 rows forward without, 2 cols, 3 rows inverse with epilogue epi).
template <typename C> int group_occupancy(int stage, int epi, size_t smem, int *per_sm);

int run_group_operator(const OpArgs &a, cudaStream_t s);

}  // namespace dbi
