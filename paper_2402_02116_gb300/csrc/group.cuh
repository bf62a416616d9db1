// Internal description of an uneven batch (dbi_group.h): member descriptors on the device and
// the persistent launches of the three operator stages over the tiles of every member.
#pragma once

#include "operator.cuh"

namespace dbi {

enum { kStageRowsForward = 0, kStageCols = 1, kStageRowsInverse = 2, kStageSource = 3 };

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
  long long S0;         // element offset of the first slot's contrast-source scratch (split rows)
  int split_rows;       // split_kind of the row stages: 2 (complex64, lx = 1024: pairs of 512-point
                        // transforms), 3 (complex64, lx = 768: triples of 256-point transforms), 0
  int split_cols;       // split_kind of the column stage (lz), likewise
  int tile0[4];         // first tile of the member in each stage's tile space (kStage*)
  int tiles[4];         // tiles per slot in each stage (the source stage: split-row members only)
};

// Host-side launch description (lives in the plan; passed through OpArgs::group).
struct GroupLaunch {
  const GMember *desc;   // device [nm]
  int nm;
  int B;                 // slots
  int total[4];          // tiles per stage
  size_t smem[4];        // dynamic shared memory: rows forward with stencil, without, cols, rows inverse
  int blocks[3];         // persistent CTAs of each stage's launch
  int parts;             // fused-reduction partials per slot (largest row-tile count)
  signed char plan[11];  // radix plan per log2 of the FFT length
  int split_rows, split_cols;  // some member runs row / column stages as pairs of 512-point transforms
  int s3_rows, s3_cols;        // some member runs row / column stages as triples of 256-point transforms
  int split_blocks[4];   // persistent CTAs of the split kernels: source, rows forward, cols, rows inverse
  int s3_blocks[3];      // persistent CTAs of the triple kernels: rows forward, cols, rows inverse
  long long T_elems;     // spectra of every slot (elements)
  long long S_elems;     // contrast-source scratch of the split-row slots, after the spectra
};

inline int group_parts(const GroupLaunch *g) { return g->parts; }

// Launches the three stages for the group in `a.group` (precision-specific, group_c64.cu /
// group_c128.cu).
template <typename C> int run_group_typed(const OpArgs &a, cudaStream_t s);
// Resident CTAs per SM of one stage's kernel with `smem` bytes (stage: 0 rows forward with
// stencil, 1 rows forward without, 2 cols, 3 rows inverse with epilogue epi).
template <typename C> int group_occupancy(int stage, int epi, size_t smem, int *per_sm);
// Resident CTAs per SM of the split kernels (complex64): [source, rows forward, cols, rows inverse]
// of the pair kernels, then [rows forward, cols, rows inverse] of the triple kernels.
int group_split_occupancy(int per_sm[7]);

int run_group_operator(const OpArgs &a, cudaStream_t s);

}  // namespace dbi
