/*
 * dbi_group.h -- uneven batches: many independent LS problems (Eq. 6, 10, 11) of different grid
 * sizes, models, frequencies and source counts, run together. Each operator stage is ONE
 * persistent launch over the tiles of every problem of every size (the FFT length of each tile
 * is dispatched inside the kernel), the Krylov iterations between host checks are captured once as
 * a CUDA graph and replayed, and an autotuner picks the radix order of every FFT length and the
 * persistent grid of every stage by timing them on the caller's data.
 *
 * The operator, its discretisation and the solver are those of dbi.h (same arithmetic per problem;
 * only the batching differs), and every convention of dbi.h holds. Terms:
 *   member    one problem of the batch: a grid, a model, a Green's table, a set of frequencies and
 *             B wavefields (its sources x frequencies);
 *   slot      one wavefield of one member; slots are numbered member by member in the order the
 *             members are given, and a member's B slots are contiguous;
 *   field     the concatenation of every slot's [2][nz][nx] complex array in slot order (element
 *             offsets per slot: dbi_group_offsets).
 */
#ifndef DBI_GROUP_H
#define DBI_GROUP_H

#include "dbi.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dbi_group_member {
  dbi_model model;     /* grid (nz, nx, lz, lx, h), reference medium, device model m */
  const void *Ghat;    /* device [nf][3][lx][lz] complex: greens_tabulate of this member's grid */
  const double *omega; /* device [nf] angular frequencies of the tables */
  int nf;              /* tables (frequencies) of this member */
  int B;               /* slots (wavefields) of this member, >= 1 */
  const int *fidx;     /* device [B] table index of each slot, in [0, nf) */
} dbi_group_member;

typedef struct dbi_group dbi_group; /* opaque plan */

enum dbi_group_flags { DBI_GROUP_GRAPH = 1 /* ls_solve_group: replay captured iterations */ };

/*
 * dbi_group_create -- validates n members (every grid as dbi.h requires; device pointers are
 *   copied, not dereferenced) and builds the plan on the host: slot and field offsets, the tile
 *   counts of each stage, and the tile order (members by decreasing FFT length). Allocates host
 *   memory only. *out is NULL on error. Release with dbi_group_destroy.
 */
int dbi_group_create(const dbi_group_member *members, int n, int precision, dbi_group **out);
void dbi_group_destroy(dbi_group *g);

/* Slots in all, and complex elements of one field array (all slots). */
int dbi_group_slots(const dbi_group *g);
long long dbi_group_field_elems(const dbi_group *g);
/* Host copy of the slot offsets: offs[n_slots + 1] (elements; slot b spans [offs[b], offs[b+1])). */
int dbi_group_offsets(const dbi_group *g, long long *offs);

/* Bytes of work for op = DBI_OP_APPLY (ls_apply_group, dbi_group_tune) or DBI_OP_SOLVE (also
 * ls_solve_group). */
size_t dbi_group_workspace_bytes(const dbi_group *g, int op);

/*
 * dbi_group_bind -- attaches `work` (work_bytes >= dbi_group_workspace_bytes(g, op)) to the plan
 *   and uploads the member descriptors, slot offsets and twiddles into it on `stream`. The plan
 *   uses this buffer until the next bind; the caller keeps it alive. Call it before any stream
 *   capture that contains ls_apply_group: after binding, ls_apply_group allocates nothing and
 *   never synchronises, so it can be captured.
 */
int dbi_group_bind(dbi_group *g, void *work, size_t work_bytes, int op, dbi_stream stream);

/*
 * ls_apply_group -- out = A u for every slot (Eq. 10 per member, as ls_apply). u, out: device
 *   fields (distinct). Three persistent launches (stencil + row FFTs, column FFTs with the
 *   Green's multiply, inverse row FFTs + epilogue), each over the tiles of every slot.
 */
int ls_apply_group(const dbi_group *g, const void *u, void *out, dbi_stream stream);

/*
 * ls_solve_group -- solves A u = rhs for every slot by BiCGSTAB exactly as ls_solve (FP64 scalars
 *   and reductions, power-of-two rhs scaling, breakdown restart). rhs, u: device fields; status
 *   arrays have one entry per slot. flags & DBI_GROUP_GRAPH (and opts->check_every > 0): the
 *   check_every iterations between host checks are captured once into a CUDA graph on a stream of
 *   the library's own and replayed on `stream`. Needs a DBI_OP_SOLVE bind. Synchronises `stream`
 *   at every host check.
 */
int ls_solve_group(const dbi_group *g, const void *rhs, void *u, const dbi_krylov_opts *opts,
                   const dbi_status *status, int flags, dbi_stream stream);

typedef struct dbi_group_tuning {
  int lengths[8];      /* FFT lengths present (0 = unused entry) */
  int plan[8];         /* radix plan chosen for lengths[i] (0: radix 8 first, 1: small radix first) */
  double plan_ms[8][2];/* apply time (ms) measured with each plan of lengths[i] (0 when one plan) */
  int ctas_per_sm[3];  /* persistent CTAs per SM chosen for each stage */
  int max_ctas[3];     /* resident CTAs per SM possible for each stage */
  double apply_ms;     /* apply time with the chosen settings */
} dbi_group_tuning;

/*
 * dbi_group_tune -- times ls_apply_group on u (writing scratch results into out) with each radix
 *   plan of every FFT length present and each persistent grid size of every stage (one to the
 *   resident maximum CTAs per SM), keeps the fastest, and reports the measurements (report may be
 *   NULL). Synchronises `stream`. The choices stay in the plan; results with another radix plan
 *   differ only by rounding.
 */
int dbi_group_tune(dbi_group *g, const void *u, void *out, dbi_stream stream, dbi_group_tuning *report);

/* Radix plan of FFT length L for the single-grid entry points of dbi.h (default 0). */
int dbi_set_radix_plan(int precision, int L, int plan);

#ifdef __cplusplus
}
#endif

#endif /* DBI_GROUP_H */
