/*
 * shiro.h -- C ABI of libshiro: the single-GPU hot path of SHIRO's sparsity-aware SpMM
 * (Zhuang et al., "SHIRO: Near-Optimal Communication Strategies for Distributed Sparse Matrix
 * Multiplication", ICS 2026), written for GB300 (sm_103a).
 *
 * The method computes C = A B (Sec. 2.1) for a CSR matrix A split into a grid of tiles A^(p,q)
 * (Tab. 1; Sec. 2.2 partitions A, B and C into row blocks and the block columns of A follow the
 * owners of B's row blocks).  For every tile it finds Cols(A^(p,q)), the distinct column indices
 * of the tile's nonzeros (Tab. 1, Eq. 2), gathers only those rows of B into a packed buffer
 * (Sec. 5.1, stage 3), remaps the tile's column indices into that buffer, and computes the local
 * product over the packed rows, summing the tiles of a row block into C (Sec. 2.2 stage 4 and
 * Sec. 5.1 stage 5).  On one GPU the P logical blocks are tiles of one matrix and the packed
 * buffer stands in for the rows that the paper's processes exchange.
 *
 * Conventions for every entry point:
 *   - All pointers named "device" are CUDA device pointers owned by the caller; the library never
 *     allocates device memory.  Plans live in a caller-provided workspace.
 *   - Dense matrices are row-major with a leading dimension (row stride) in elements.
 *   - "stream" is a cudaStream_t passed as void* (NULL = the legacy default stream).  Compute calls
 *     (pack, spmm, sddmm, backward) only enqueue work: they never synchronise, never allocate and
 *     can be captured in a CUDA graph.  Plan creation synchronises the stream.
 *   - Errors are returned as shiro_status; shiro_last_error() gives a message (thread-local).
 *     Nothing aborts or traps.  Device-side detection (e.g. a malformed CSR) sets a status word
 *     in the plan that plan creation or shiro_plan_check() reads back.
 *   - A plan may be used by one stream at a time: calls on the same plan must not overlap on the
 *     GPU (long rows use per-plan arrival counters, and the counter-form kernels a per-plan work
 *     counter that a memset node zeroes before each launch).
 */
#ifndef SHIRO_H
#define SHIRO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SHIRO_OK = 0,
  SHIRO_ERR_INVALID_ARG = 1,           /* a null pointer, a negative size, a bad combination */
  SHIRO_ERR_BAD_CSR = 2,               /* rowptr not monotone / wrong ends, column out of range,
                                          a nonzero outside its diagonal tile (DIAG_ONLY) */
  SHIRO_ERR_INSUFFICIENT_WORKSPACE = 3,/* workspace or scratch smaller than required */
  SHIRO_ERR_UNSUPPORTED = 4,           /* dtype combination or size beyond the limits below */
  SHIRO_ERR_CUDA = 5,                  /* a CUDA runtime call failed (message has the detail) */
  SHIRO_ERR_DEVICE_TIMEOUT = 6         /* a bounded device-side wait gave up */
} shiro_status;

typedef enum { SHIRO_F32 = 0, SHIRO_BF16 = 1, SHIRO_F64 = 2 } shiro_dtype;

/* Opaque plan handle (host memory; its device arrays live in the caller's workspace). */
typedef struct shiro_plan_s* shiro_plan_t;

/* A CSR matrix in device memory.  rowptr has M+1 entries with rowptr[0] = 0, non-decreasing,
 * rowptr[M] = nnz; col[e] in [0, K).  Column order inside a row is free (sums follow it) and
 * duplicates are summed.  val is F32 or F64 (the FP64 form exists for gradient checks). */
typedef struct {
  int64_t M, K, nnz;
  const int64_t* rowptr; /* device, M+1 */
  const int32_t* col;    /* device, nnz */
  const void* val;       /* device, nnz elements of vdt */
  shiro_dtype vdt;
} shiro_csr;

/* Plan flags. */
#define SHIRO_PLAN_LOCAL_DIAG 0x1u /* 1D reading (Sec. 2.2): diagonal tiles (p == q) are the
                                      "local computation" and read B in place; only off-diagonal
                                      tiles are packed.  Needs P_r == P_c. */
#define SHIRO_PLAN_DIAG_ONLY 0x2u  /* only tiles (p, p) exist (block-diagonal A, e.g. a batch of
                                      graphs); a nonzero outside them is SHIRO_ERR_BAD_CSR. */
#define SHIRO_PLAN_TRANSPOSE 0x4u  /* plan A^T (K x M) on the transposed grid: tile (q, p) of A^T
                                      is tile (p, q) of A, so its Cols are Rows(A^(p,q)) (Eq. 3).
                                      Used for dB = A^T dC. */

/* The tile grid.  Row block p covers rows [row_bounds[p], row_bounds[p+1]) and column block q
 * covers columns [col_bounds[q], col_bounds[q+1]).  NULL bounds mean uniform blocks starting at
 * p * ceil(M / P_r), clamped to M (the last block takes the remainder).  Tiles are numbered
 * t = p * P_c + q (t = p with DIAG_ONLY).  Limits: 1 <= P_r, P_c <= 65536, P_r * P_c <= 2^20. */
typedef struct {
  int32_t P_r, P_c;
  const int64_t* row_bounds; /* host, P_r + 1 ascending entries from 0 to M, or NULL */
  const int64_t* col_bounds; /* host, P_c + 1 ascending entries from 0 to K, or NULL */
  uint32_t flags;            /* SHIRO_PLAN_* */
} shiro_partition;

/* Work schedule of the SpMM/SDDMM kernels (zero fields take the defaults).  Rows with more than
 * long_row_nnz nonzeros are split into chunks of chunk_nnz (>= 32) nonzeros whose FP32 partial
 * sums are added in a fixed order (deterministic); shorter rows are grouped into work items of at
 * most group_nnz nonzeros and group_rows rows.  One warp runs one work item at a time.
 * group_nnz 0 (the default) is automatic: 256, or fewer when the matrix is small enough that
 * 256-nonzero groups would leave warp slots without an item (at most the short rows' nonzeros
 * over SMs x 40).  Rows are never split by a group, so results do not depend on group_nnz. */
typedef struct {
  int32_t long_row_nnz;
  int32_t chunk_nnz;
  int32_t group_nnz;
  int32_t group_rows;
  int32_t warps_per_cta; /* 1..8 */
  int32_t persistent;    /* 1: grid = SMs x resident CTAs; the warps of pipeline 6 take items
                            from a counter, those of the other pipelines stride over them */
  int32_t pipeline;      /* How the gathered B rows reach the accumulators (every pipeline sums
                            a row's nonzeros in the same order, except 3):
                            0: automatic -- 7 for BF16 rows of 512 bytes, 6 for the other
                               FP32/BF16 rows of 128 to 512 bytes (in its counter form except
                               for BF16 rows of 256 bytes; 5 in persistent mode), 4 for FP32/BF16
                               rows of 1-2 KB, else 5 (the fastest measured for each row size;
                               shiro_pack_spmm runs FP32 rows of 512 bytes as one fused launch);
                            1: staged through shared memory by per-lane asynchronous copies, two
                               stages per warp;
                            2: staged by one TMA bulk copy per row, two stages per warp (rows of
                               a multiple of 16 bytes, 16-byte aligned; else 1);
                            3: rows of 128 or 256 bytes (FP32 N = 32/64, BF16 N = 64/128) split
                               across 4 or 2 lane groups that take interleaved nonzeros of a row
                               (other rows as 0);
                            4: a per-warp ring of row slots refilled by per-lane asynchronous
                               copies stage_rows rows ahead (FP32/BF16 rows of 256 bytes to 2 KB;
                               else 5);
                            5: register gathers, 2-4 rows in flight per warp, 64 registers;
                            6: register gathers with a 48-register budget (FP32/BF16 rows of
                               128-512 bytes; else 5): 2-warp CTAs, 40 warps per SM, the next
                               batch's (index, value) pairs copied into shared memory
                               asynchronously; warps_per_cta does not apply; one item per warp,
                               or with persistent set, items taken from a counter in the plan;
                            7: FP32/BF16 rows of 512 bytes moved into shared memory by TMA gathers
                               of four packed rows (tile::gather4, one tensor map over the packed
                               buffer), eight gathers in flight per warp, items from a counter
                               (not LOCAL_DIAG plans, else as 5).
                            shiro_sddmm reads 5 and 6 too (see there). */
  int32_t stage_rows;    /* pipeline 1: rows per stage, 8, 16 or 32 (0 = the largest that keeps a
                            stage within 16 KB); pipeline 4: ring depth, 16 or 32 for 256-byte
                            rows (0 = 16), 8, 12 or 16 for 512-byte rows (0 = 8), 4 or 8 for
                            1-2 KB rows (0 = 4).  Accepted values: 0, 4, 8, 12, 16, 32; a ring
                            depth not compiled for the row size takes its default */
} shiro_opts;

/* Bytes of workspace shiro_plan_create needs for A and this partition (an upper bound that does
 * not depend on A's pattern, so it can be allocated before the plan exists).  A's pointers may be
 * NULL here: only M, K, nnz and vdt are read. */
shiro_status shiro_plan_workspace(const shiro_csr* A, const shiro_partition* part,
                                  const shiro_opts* opts, size_t* bytes);

/* Plan stage 1 of Sec. 5.1 (sparsity analysis) for every tile, once per pattern (the paper runs
 * it offline and reuses it across SpMM calls with the same pattern, Sec. 5.1 and Sec. 5.3.2):
 *   a1  tile split: the tile of every nonzero, nonzeros per tile;
 *   a2  Cols(A^(p,q)) in ascending column order and their exclusive scan over tiles (Eq. 2);
 *       Rows(A^(p,q)) counts (Eq. 3);
 *   a3  remap: every nonzero's row in the packed buffer;
 *   a4  per-tile volumes (see shiro_plan_volumes);
 * plus the work schedule.  The CSR is validated on the device first.  A's arrays must stay alive
 * and unchanged while the plan is used (except a TRANSPOSE plan, which keeps its own copy of A^T;
 * refresh its values with shiro_plan_update_values).  Synchronises `stream`.
 * On success *plan owns nothing but host memory; free it with shiro_plan_destroy. */
shiro_status shiro_plan_create(const shiro_csr* A, const shiro_partition* part,
                               const shiro_opts* opts, void* workspace, size_t workspace_bytes,
                               void* stream, shiro_plan_t* plan);

void shiro_plan_destroy(shiro_plan_t plan);

typedef struct {
  int64_t M, K, nnz;      /* of the planned matrix (A^T for a TRANSPOSE plan) */
  int32_t P_r, P_c;       /* grid of the planned matrix */
  int32_t n_tiles;
  uint32_t flags;
  shiro_dtype vdt;
  int64_t total_cols;     /* sum over tiles of |Cols(A^(p,q))| */
  int64_t packed_rows;    /* rows of the packed buffer (total_cols minus local diagonal tiles) */
  int64_t n_items;        /* work items of the schedule */
  int64_t n_long_rows;    /* rows split into chunks */
  int64_t n_chunks;       /* chunks of those rows (partial-sum slots) */
  size_t workspace_used;  /* bytes of the workspace in use */
  shiro_opts opts;        /* schedule in effect */
} shiro_plan_info;

shiro_status shiro_plan_query(shiro_plan_t plan, shiro_plan_info* info);

/* Per-tile statistics, host arrays: tile_nnz, tile_nrows (|Rows|), tile_ncols (|Cols|) have
 * n_tiles entries; tile_cols_ptr and pack_ptr have n_tiles + 1 (exclusive scans of |Cols| over all
 * tiles and over packed tiles).  Any pointer may be NULL. */
shiro_status shiro_plan_tile_stats(shiro_plan_t plan, int64_t* tile_nnz, int64_t* tile_nrows,
                                   int64_t* tile_ncols, int64_t* tile_cols_ptr, int64_t* pack_ptr);

/* Communication volumes in bytes for N columns (host arrays of n_tiles entries), B stored as
 * b_dt and partial C rows exchanged as c_dt (the accumulator type: F32 for F32 or BF16 B, F64 for
 * F64 B):
 *   v_block[t] = (width of column block q) * N * sz(b_dt)   (Eq. 1: the whole block B^(q));
 *   v_col[t]   = |Cols(A^(p,q))| * N * sz(b_dt)              (Eq. 2: the B rows the tile names);
 *   v_row[t]   = |Rows(A^(p,q))| * N * sz(c_dt)              (Eq. 3: one partial C row per row
 *                                                             of the tile holding a nonzero).
 * Diagonal tiles of a LOCAL_DIAG plan are local computation (Sec. 2.2) and report 0 in all three.
 * Any output pointer may be NULL. */
shiro_status shiro_plan_volumes(shiro_plan_t plan, int32_t N, shiro_dtype b_dt, shiro_dtype c_dt,
                                int64_t* v_block, int64_t* v_col, int64_t* v_row);

/* Joint row-column strategy (Sec. 5.2-5.3) for every tile: a minimum vertex cover of the bipartite
 * graph rows--columns whose edges are the tile's nonzeros (uniform costs, Sec. 5.4: the cover size
 * mu equals the maximum matching by Koenig's theorem; Hopcroft-Karp finds it and the cover is read
 * off the alternating reachability from unmatched rows).  Outputs (host arrays, any may be NULL):
 * tile_mu, tile_cover_rows, tile_cover_cols (n_tiles entries; mu = rows + columns of the cover,
 * V_joint = mu * N * sz, Eq. 9) and nnz_row_based (nnz bytes: 0 if the nonzero's column is in the
 * cover -- its B row is sent, Eq. 2 --, 1 if only its row is -- a partial C row is sent, Eq. 3).
 * Diagonal tiles of a LOCAL_DIAG plan communicate nothing and report 0.  Offline host work (tiles
 * in parallel threads); synchronises `stream`. */
shiro_status shiro_plan_joint(shiro_plan_t plan, int64_t* tile_mu, int64_t* tile_cover_rows,
                              int64_t* tile_cover_cols, uint8_t* nnz_row_based, void* stream);

/* Weighted joint strategy (Sec. 5.3.2-5.3.3): per tile, the minimum weighted vertex cover of the
 * row-column graph, with cost w_row[i] for sending the partial row c_i and w_col[j] for sending
 * row b_j (e.g. N * sizeof(C accumulator) and N * sizeof(B element) when B and the partial rows
 * differ in type).  Solved as the minimum s-t cut of the network source -> row (w_row) -> column
 * (unbounded, one arc per nonzero) -> sink (w_col) by Dinic's algorithm; the selection is read
 * off the vertices reachable from the source in the final residual network, which is the same for
 * every maximum flow, so the cover is unique (with all costs 1 it equals shiro_plan_joint's).
 * w_row (host, M entries, indexed by global row) or NULL for a uniform w_row_all; w_col (host, K
 * entries, indexed by global column) or NULL for w_col_all.  Costs must be >= 0 and each side's
 * total at most 2^60, else SHIRO_ERR_INVALID_ARG.  Outputs as shiro_plan_joint, with tile_cost
 * the cover's total cost (= the maximum flow).  Offline host work; synchronises `stream`. */
shiro_status shiro_plan_joint_weighted(shiro_plan_t plan, const int64_t* w_row,
                                       const int64_t* w_col, int64_t w_row_all, int64_t w_col_all,
                                       int64_t* tile_cost, int64_t* tile_cover_rows,
                                       int64_t* tile_cover_cols, uint8_t* nnz_row_based,
                                       void* stream);

/* Row-based strategy (Eq. 3) as a side assignment for shiro_joint_split: every nonzero of a
 * communicated tile is row-based (nnz_row_based = 1; 0 on the local diagonal tiles of a
 * LOCAL_DIAG plan), so the owners of B send one partial C row per row of Rows(A^(p,q)).
 * tile_rows (host, n_tiles) receives |Rows| of every communicated tile (0 for local ones).
 * Synchronises `stream`. */
shiro_status shiro_plan_row_based(shiro_plan_t plan, int64_t* tile_rows, uint8_t* nnz_row_based,
                                  void* stream);

/* Split of A by a joint cover (nnz_row_based from shiro_plan_joint, host, nnz bytes) into the
 * three CSR matrices whose SpMMs compute C = A B the joint way (Sec. 5.1 stages 3 and 5):
 *   A_col (M x K): the column-based nonzeros, to be planned on the same grid -- its tiles' Cols are
 *     the cover columns, so packing B for it sends exactly the cover's B rows (Eq. 2 part of Eq. 9);
 *   A_rs (split_rows x K): one row per (tile, cover row) pair, tiles in order, holding that row's
 *     row-based nonzeros of the tile; A_rs B is the packed buffer of partial C rows the owners of B
 *     would send (Eq. 3 part of Eq. 9); plan it 1 x 1 with LOCAL_DIAG so it reads B in place;
 *   A_agg (M x split_rows): 0/1 rows adding each partial row to its C row in tile order (stage 5);
 *     plan it 1 x 1 with LOCAL_DIAG and run its SpMM with SHIRO_SPMM_ACCUMULATE over the partials.
 * shiro_joint_split_sizes gives col_nnz, split_rows and split_nnz; shiro_joint_split fills caller
 * device buffers: col_* (M+1, col_nnz, col_nnz), rs_* (split_rows+1, split_nnz, split_nnz), agg_*
 * (M+1, split_rows, split_rows); values in the plan's vdt.  Host work; synchronises `stream`. */
shiro_status shiro_joint_split_sizes(shiro_plan_t plan, const uint8_t* nnz_row_based,
                                     int64_t* col_nnz, int64_t* split_rows, int64_t* split_nnz);
shiro_status shiro_joint_split(shiro_plan_t plan, const uint8_t* nnz_row_based,
                               int64_t* col_rowptr, int32_t* col_col, void* col_val,
                               int64_t* rs_rowptr, int32_t* rs_col, void* rs_val,
                               int64_t* agg_rowptr, int32_t* agg_col, void* agg_val, void* stream);

/* Copies the plan's index arrays into caller device buffers (any may be NULL):
 * cols_sorted (total_cols): Cols of every tile, ascending, concatenated in tile order;
 * pack_src (packed_rows): the B row gathered into each packed row;
 * colidx_local (nnz): position of every nonzero's column in its tile's Cols;
 * remap (nnz): packed row read by every nonzero, or -1 - col for a local diagonal tile.
 * Enqueued on `stream`; no synchronisation. */
shiro_status shiro_plan_export(shiro_plan_t plan, int32_t* cols_sorted, int32_t* pack_src,
                               int32_t* colidx_local, int32_t* remap, void* stream);

/* For a TRANSPOSE plan: copies A^T's CSR into caller device buffers (any may be NULL): rowptr
 * (K+1), col (nnz: the row of A of each entry, ascending within a row of A^T), perm (nnz: index
 * in A of each entry of A^T). */
shiro_status shiro_plan_export_transpose(shiro_plan_t plan, int64_t* rowptr, int32_t* col,
                                         int64_t* perm, void* stream);

/* For a TRANSPOSE plan: reloads A^T's values from A's value array `val` (device, nnz elements of
 * the plan's vdt) through the stored permutation.  Enqueued on `stream`. */
shiro_status shiro_plan_update_values(shiro_plan_t plan, const void* val, void* stream);

/* Reads and clears the plan's device status word (synchronises `stream`). */
shiro_status shiro_plan_check(shiro_plan_t plan, void* stream);

/* Rebuilds the work schedule with new options (the pattern analysis is kept).  Fails with
 * SHIRO_ERR_INSUFFICIENT_WORKSPACE if the new schedule does not fit.  Synchronises `stream`. */
shiro_status shiro_plan_reschedule(shiro_plan_t plan, const shiro_opts* opts, void* stream);

/* Pack (Sec. 5.1 stage 3): Bpack[r, :] = B[pack_src[r], :] for the packed_rows rows.
 * B: device, rows of the planned matrix's K, N columns, leading dimension ldb >= N.
 * Bpack: device, packed_rows x N with leading dimension ldp >= N.  dt is F32, BF16 or F64; the
 * copy is bit-exact. */
shiro_status shiro_pack(shiro_plan_t plan, const void* B, int64_t ldb, int32_t N, shiro_dtype dt,
                        void* Bpack, int64_t ldp, void* stream);

/* Scratch bytes shiro_spmm / shiro_spmm_backward need for N columns of dt with the plan's current
 * schedule (partial sums of split rows); 0 when no row is split. */
shiro_status shiro_spmm_scratch(shiro_plan_t plan, int32_t N, shiro_dtype dt, size_t* bytes);

#define SHIRO_SPMM_ACCUMULATE 0x1u /* C += A B instead of C = A B */

/* Local SpMM over the packed rows and aggregation over the tiles of each row block (Sec. 2.2
 * stages 3-4, Sec. 5.1 stage 5): C[i, :] = sum over the nonzeros e of row i of
 * val[e] * Bpack[remap[e], :] (or B[col[e], :] for local diagonal tiles), summed in the row's
 * stored order, i.e. ascending column blocks for column-sorted rows.
 * Types: values F32 with dt F32 or BF16 (C is F32, accumulation in FP32), or values F64 with dt
 * F64 (C is F64).  B may be NULL unless the plan has LOCAL_DIAG.  scratch: device, at least
 * shiro_spmm_scratch bytes (may be NULL when that is 0); its contents need no initialisation.
 * A plan holds the arrival counters of split rows and a work counter used by these calls, so
 * compute calls on one plan must not overlap on the GPU (serialise them on one stream). */
shiro_status shiro_spmm(shiro_plan_t plan, const void* Bpack, int64_t ldp, const void* B,
                        int64_t ldb, int32_t N, shiro_dtype dt, void* C, int64_t ldc,
                        uint32_t flags, void* scratch, size_t scratch_bytes, void* stream);

/* Pack + SpMM in one call (Sec. 5.1 stages 3 and 5 overlapped): the same results as shiro_pack
 * (Bpack[r] = B[pack_src[r]], bit-exact) followed by shiro_spmm(plan, Bpack, ldp, B, ldb, ...)
 * (C bit-identical: the same work items summed in the same order).  For FP32 rows of 512 bytes
 * (N = 128) with pipeline 0 or 6, and BF16 rows of 512 bytes (N = 256) with pipeline 6, not
 * persistent, and B, Bpack and C aligned to 16 bytes, it is one launch (BF16 rows of 512 bytes
 * with pipeline 0 take the pack and then the TMA gather4 ring, measured faster): the plan orders
 * the pack of row block p + 1
 * among the SpMM work of block p (after the pack of block 0), and a warp starts an item of block p
 * once every packed row of block p is written (a per-block count in the plan; the wait is bounded
 * and sets a device status bit that shiro_plan_check reports if it runs out).  Otherwise it
 * enqueues shiro_pack then shiro_spmm.  B: device K x N (ldb) of dt, read by the pack and, for
 * local diagonal tiles, by the SpMM; Bpack: device packed_rows x N (ldp), written; C, flags,
 * scratch: as shiro_spmm.  Calls on one plan must not overlap on the GPU. */
shiro_status shiro_pack_spmm(shiro_plan_t plan, const void* B, int64_t ldb, int32_t N,
                             shiro_dtype dt, void* Bpack, int64_t ldp, void* C, int64_t ldc,
                             uint32_t flags, void* scratch, size_t scratch_bytes, void* stream);

/* Allocation-free variant of shiro_spmm.  The paper has no counterpart: it exists for callers that
 * cannot allocate device memory for the split-row scratch -- code that runs while a stream is
 * being captured into a CUDA graph (cudaMalloc is not a capturable operation), plug-ins inside
 * runtimes that hand a kernel only its input and output buffers and own all device memory, and
 * serving paths that may not allocate after start-up.
 * Same arguments and results as shiro_spmm without scratch/scratch_bytes: the partial sums of
 * split rows go to one static device array of SHIRO_NOALLOC_SCRATCH_BYTES (16 MiB) inside the
 * library, which every GPU that loads the library holds until the process exits.  A plan whose
 * shiro_spmm_scratch(plan, N, dt) exceeds that size is rejected with
 * SHIRO_ERR_INSUFFICIENT_WORKSPACE (16 MiB holds up to 32,767 split-row chunks at N = 128 in
 * FP32: the size check keeps the 256-byte alignment margin of shiro_spmm_scratch).  The plan must
 * belong to the current device (SHIRO_ERR_INVALID_ARG otherwise).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture begins.  All calls on a device
 * share the one array, which keeps the last call's partial sums (nothing in it has to start at
 * zero): calls that overlap on the GPU -- on different streams, or with different plans -- race
 * and must be serialised by the caller. */
#define SHIRO_NOALLOC_SCRATCH_BYTES (16 << 20)
shiro_status shiro_spmm_noalloc(shiro_plan_t plan, const void* Bpack, int64_t ldp, const void* B,
                                int64_t ldb, int32_t N, shiro_dtype dt, void* C, int64_t ldc,
                                uint32_t flags, void* stream);

/* Gradient of C = A B with respect to A's stored values (a sampled dense-dense product on A's
 * pattern): dA[e] = sum_k dC[row(e), k] * Bpack[remap[e], k] (B[col[e], k] for local diagonal
 * tiles).  dC: device M x N of dt (F32/BF16 with F32 dA, or F64 with F64 dA).  The plan's
 * schedule options pick the kernel.  With pipeline 0 (the default), FP32 or BF16 rows of 128, 256
 * or 512 bytes whose rows start on 16-byte boundaries are taken by lane groups: eight lanes per
 * nonzero, four nonzeros per warp step, a three-level shuffle sum per nonzero (48 registers, 40
 * warps per SM, items taken from a counter in the plan).  Pipelines 3 and 6 (and pipeline 0 on
 * rows that are not 16-byte aligned) keep the earlier 48-register kernels: BF16 rows of 256 or
 * 512 bytes and FP32 rows of 256 bytes reduce through a shared-memory tile, FP32 rows of 512
 * bytes through a 4-wide shuffle butterfly (pipeline 6: the tile).  Other rows, pipeline 5 and
 * persistent mode use an 8-wide shuffle butterfly at 64 registers.  Each kernel sums in a fixed
 * order, so dA is deterministic for a given kernel. */
shiro_status shiro_sddmm(shiro_plan_t plan, const void* dC, int64_t lddc, const void* Bpack,
                         int64_t ldp, const void* B, int64_t ldb, int32_t N, shiro_dtype dt,
                         void* dA, void* stream);

/* Backward of C = A B: dB = A^T dC through the TRANSPOSE plan planT (pack dC by planT into
 * dCpack, then SpMM over it, as shiro_pack_spmm) and dA by shiro_sddmm on `plan`.  dB and dA may be NULL to skip
 * them; dCpack (planT's packed_rows x N, leading dimension lddp) is needed when dB is wanted.
 * scratch must hold shiro_spmm_scratch(planT, N, dt).
 * When both are wanted, B is given (device, K x N, rows aligned to 16 bytes for rows of 512 bytes,
 * to 8 for rows of 256), the rows are 256 or 512 bytes (F32 N = 64 / 128 or BF16 N = 128 / 256,
 * F32 values) and planT's schedule is pipeline 0 or 6, not
 * persistent, all of it is one launch over planT: a row j of A^T gathers the dC rows of column j's
 * nonzeros for dB, and each gathered row's dot product with B[j, :] is that nonzero's dA (one pass
 * of row gathers instead of two).  dCpack and dB are then bit-identical to the two calls; dA is
 * summed in another fixed order than shiro_sddmm (per lane, then a tree over the warp), within the
 * same error bound.  Otherwise the two calls are made.  Calls on plan or planT must not overlap on
 * the GPU. */
shiro_status shiro_spmm_backward(shiro_plan_t plan, shiro_plan_t planT, const void* dC,
                                 int64_t lddc, const void* Bpack, int64_t ldp, const void* B,
                                 int64_t ldb, int32_t N, shiro_dtype dt, void* dCpack,
                                 int64_t lddp, void* dB, int64_t lddb, void* dA, void* scratch,
                                 size_t scratch_bytes, void* stream);

/* Batched form: G independent graphs (CSR matrices, host array of G descriptors whose arrays are
 * on the device) become one block-diagonal matrix planned with DIAG_ONLY, one tile per graph, so
 * Cols of tile g are the non-empty columns of graph g.  B and C of the batch are the per-graph
 * operands stacked by rows in graph order (graph g's rows start at the sum of the earlier
 * graphs' row counts).  The plan holds its own copy of the graphs, so theirs may be freed
 * afterwards.  All graphs share one vdt.  Use shiro_pack / shiro_spmm / shiro_sddmm on the plan. */
shiro_status shiro_batch_workspace(int32_t G, const shiro_csr* graphs, const shiro_opts* opts,
                                   size_t* bytes);
shiro_status shiro_batch_plan_create(int32_t G, const shiro_csr* graphs, const shiro_opts* opts,
                                     void* workspace, size_t workspace_bytes, void* stream,
                                     shiro_plan_t* plan);

/* Autotuner: times shiro_spmm over a set of candidate schedules on the caller's operands (Bpack,
 * C and scratch as for shiro_spmm; C is overwritten) and leaves the fastest one in the plan
 * (*best receives it).  Candidates vary the row-group size (from the average row length), the
 * chunk size of long rows (only when some row is longer), the CTA size and the pipeline: register
 * gathers, plus lane groups for rows of 128 or 256 bytes, the per-lane copy ring for FP32/BF16
 * rows of 512 bytes to 2 KB and the 48-register gathers for FP32/BF16 rows of 128-512 bytes;
 * the persistent mode stays as set.  Candidates whose scratch
 * does not fit scratch_bytes are skipped.  Synchronises `stream`. */
shiro_status shiro_autotune(shiro_plan_t plan, const void* Bpack, int64_t ldp, const void* B,
                            int64_t ldb, int32_t N, shiro_dtype dt, void* C, int64_t ldc,
                            void* scratch, size_t scratch_bytes, int32_t reps, void* stream,
                            shiro_opts* best);

/* Makes `device` the calling host thread's current CUDA device for this library (the library
 * carries its own CUDA runtime, so a caller that switches devices must tell it).  Plans and
 * compute calls use the thread's current device; streams passed in must belong to it. */
shiro_status shiro_set_device(int32_t device);

/* Default schedule options: long_row_nnz 512, chunk_nnz 256, group_nnz 0 (automatic: 256 except
 * on small matrices), group_rows 32, warps_per_cta 1, persistent 0, pipeline 0, stage_rows 0. */
void shiro_default_opts(shiro_opts* opts);

/* Thread-local message of the last error. */
const char* shiro_last_error(void);

/* Library version: major * 10000 + minor * 100 + patch. */
int32_t shiro_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SHIRO_H */
