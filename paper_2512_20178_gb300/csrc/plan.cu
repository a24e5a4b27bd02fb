// plan.cu -- plan creation (sparsity analysis of every tile, Sec. 5.1 stage 1), the work
// schedule, the transposed and batched plans, and the small query/export entry points.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.cuh"
#include "plan_kernels.cuh"

namespace shiro {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

static int grid_for(int64_t work, int threads, int sm_count, int per_sm = 8) {
  int64_t g = (work + threads - 1) / threads;
  int64_t cap = (int64_t)std::max(sm_count, 1) * per_sm * 4;
  if (g > cap) g = cap;
  return (int)std::max<int64_t>(g, 1);
}

shiro_status resolve_opts(const shiro_opts* in, shiro_opts* o) {
  shiro_default_opts(o);
  if (in) {
    if (in->long_row_nnz) o->long_row_nnz = in->long_row_nnz;
    if (in->chunk_nnz) o->chunk_nnz = in->chunk_nnz;
    if (in->group_nnz) o->group_nnz = in->group_nnz;
    if (in->group_rows) o->group_rows = in->group_rows;
    if (in->warps_per_cta) o->warps_per_cta = in->warps_per_cta;
    o->persistent = in->persistent;
    o->pipeline = in->pipeline;
    o->stage_rows = in->stage_rows;
  }
  if (o->chunk_nnz < 32 || o->long_row_nnz < o->chunk_nnz || o->group_nnz < 0 ||
      o->group_rows < 1 || o->group_rows > 32 || o->warps_per_cta < 1 || o->warps_per_cta > 8 ||
      (o->stage_rows != 0 && o->stage_rows != 4 && o->stage_rows != 8 && o->stage_rows != 12 &&
       o->stage_rows != 16 && o->stage_rows != 32) ||
      o->pipeline < 0 || o->pipeline > 7)
    SHIRO_FAIL(SHIRO_ERR_INVALID_ARG,
               "bad schedule options: need 32 <= chunk_nnz <= long_row_nnz, group_nnz >= 0, "
               "1 <= group_rows <= 32, 1 <= warps_per_cta <= 8, "
               "stage_rows in {0, 4, 8, 12, 16, 32}, pipeline in {0, 1, 2, 3, 4, 5, 6, 7}");
  return SHIRO_OK;
}

shiro_status read_status(shiro_plan_s* P, cudaStream_t s, const char* where) {
  int st = 0;
  SHIRO_CUDA(cudaMemcpyAsync(&st, P->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  SHIRO_CUDA(cudaStreamSynchronize(s));
  if (!st) return SHIRO_OK;
  SHIRO_CUDA(cudaMemsetAsync(P->d_status, 0, sizeof(int), s));
  if (st & (ST_BAD_ROWPTR | ST_BAD_COL | ST_OFF_DIAG))
    SHIRO_FAIL(SHIRO_ERR_BAD_CSR, "%s: malformed CSR (%s%s%s)", where,
               (st & ST_BAD_ROWPTR) ? "rowptr not monotone or wrong ends; " : "",
               (st & ST_BAD_COL) ? "column index out of range; " : "",
               (st & ST_OFF_DIAG) ? "nonzero outside its diagonal tile" : "");
  if (st & ST_OVERFLOW)
    SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "%s: more than 2^31 - 1 packed rows", where);
  SHIRO_FAIL(SHIRO_ERR_DEVICE_TIMEOUT, "%s: device status word 0x%x", where, st);
}

// ---- workspace layout ----

struct Carver {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(int64_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += sizeof(T) * (size_t)std::max<int64_t>(count, 1);
    return p;
  }
};

struct Shape {
  int64_t M = 0, K = 0, nnz = 0;  // planned matrix
  int32_t Pr = 1, Pc = 1;
  uint32_t flags = 0;
  shiro_dtype vdt = SHIRO_F32;
  std::vector<int64_t> rb, cb;
  int64_t Wc = 0, Wr = 0, cols_cap = 0;
  int32_t T = 1;
  bool own_csr = false;    // plan keeps its own copy of the planned CSR
  bool transpose = false;  // radix-sort temporaries
  int64_t src_M = 0;       // rows of A for the transpose (row ids)
  int32_t G = 0;           // batch descriptors
};

static void uniform_bounds(int64_t n, int32_t P, std::vector<int64_t>& b) {
  b.resize(P + 1);
  const int64_t step = (n + P - 1) / P;
  for (int32_t p = 0; p <= P; ++p) b[p] = std::min<int64_t>((int64_t)p * step, n);
}

static shiro_status check_bounds(const std::vector<int64_t>& b, int64_t n, const char* what) {
  if (b.front() != 0 || b.back() != n)
    SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "%s bounds must start at 0 and end at %lld", what,
               (long long)n);
  for (size_t i = 1; i < b.size(); ++i)
    if (b[i] < b[i - 1]) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "%s bounds not ascending", what);
  return SHIRO_OK;
}

static void finish_shape(Shape& sh) {
  const bool diag = sh.flags & SHIRO_PLAN_DIAG_ONLY;
  sh.T = diag ? sh.Pr : sh.Pr * sh.Pc;
  int64_t wc_row = 0, width_sum = 0;
  for (int32_t q = 0; q < sh.Pc; ++q) wc_row += (sh.cb[q + 1] - sh.cb[q] + 31) / 32;
  int64_t wr_col = 0;
  for (int32_t p = 0; p < sh.Pr; ++p) wr_col += (sh.rb[p + 1] - sh.rb[p] + 31) / 32;
  if (diag) {
    sh.Wc = wc_row;
    sh.Wr = wr_col;
    width_sum = sh.K;
  } else {
    sh.Wc = wc_row * sh.Pr;
    sh.Wr = wr_col * sh.Pc;
    width_sum = sh.K * sh.Pr;
  }
  sh.cols_cap = std::max<int64_t>(1, std::min(sh.nnz, width_sum));
}

// Chunks of the fused pack + SpMM: at most 32 packed rows each, split at row-block boundaries,
// over at most cols_cap packed rows.
static int64_t fused_chunk_cap(const Shape& sh) { return sh.cols_cap / 32 + sh.Pr + 1; }

static size_t carve(const Shape& sh, shiro_plan_s* P, char* base) {
  Carver c{base};
  const int64_t T = sh.T;
  int* status = c.take<int>(4);
  int64_t* rb = c.take<int64_t>(sh.Pr + 1);
  int64_t* cb = c.take<int64_t>(sh.Pc + 1);
  int64_t* woff = c.take<int64_t>(T + 1);
  int64_t* rwoff = c.take<int64_t>(T + 1);
  uint32_t* bm = c.take<uint32_t>(sh.Wc);
  int64_t* wprefix = c.take<int64_t>(sh.Wc + 1);
  uint32_t* rbm = c.take<uint32_t>(sh.Wr);
  unsigned long long* tnnz = c.take<unsigned long long>(T);
  unsigned long long* trows = c.take<unsigned long long>(T);
  int64_t* tcp = c.take<int64_t>(T + 1);
  int64_t* pptr = c.take<int64_t>(T + 1);
  int32_t* cols = c.take<int32_t>(sh.cols_cap);
  int32_t* psrc = (sh.flags & SHIRO_PLAN_LOCAL_DIAG) ? c.take<int32_t>(sh.cols_cap) : cols;
  int32_t* remap = c.take<int32_t>(sh.nnz);
  // Scan block sums: enough for the bitmap scan and the radix histogram scan.
  int64_t scan_n = sh.Wc + 1;
  const int64_t radix_blocks = (sh.nnz + kRadixTile - 1) / kRadixTile;
  if (sh.transpose) scan_n = std::max<int64_t>(scan_n, 256 * radix_blocks + 1);
  int64_t* scan_tmp = c.take<int64_t>((scan_n + kScanTile - 1) / kScanTile + 2);
  // Schedule capacity: every group holds >= 1 row; chunks of >= 32 nonzeros.
  const int64_t slots_cap = 2 * ((sh.nnz + 31) / 32) + 1;
  const int64_t lr_cap = (sh.nnz + 31) / 32 + 1;
  const int64_t items_cap = sh.M + slots_cap + 1;
  Item* items = c.take<Item>(items_cap);
  int32_t* slot_lr = c.take<int32_t>(slots_cap);
  LongRow* lr = c.take<LongRow>(lr_cap);
  int32_t* counters = c.take<int32_t>(lr_cap);
  // Fused pack + SpMM: chunks of at most 32 packed rows that never span two row blocks, and the
  // launch order of chunks and items.
  const int64_t pk_cap = fused_chunk_cap(sh);
  int32_t* fseq = c.take<int32_t>(items_cap + pk_cap);
  int4* pchunk = c.take<int4>(pk_cap);
  int32_t* blk = c.take<int32_t>(2 * (int64_t)sh.Pr);
  int64_t* rowptr_own = nullptr;
  int32_t* col_own = nullptr;
  void* val_own = nullptr;
  int64_t* perm = nullptr;
  if (sh.own_csr) {
    rowptr_own = c.take<int64_t>(sh.M + 1);
    col_own = c.take<int32_t>(sh.nnz);
    val_own = c.take<char>(sh.nnz * (int64_t)dtype_size(sh.vdt));
  }
  if (sh.transpose) perm = c.take<int64_t>(sh.nnz);
  // Temporaries (after everything that must persist).
  if (sh.transpose) {
    c.take<uint32_t>(sh.nnz);      // keys a
    c.take<uint32_t>(sh.nnz);      // keys b
    c.take<int32_t>(sh.nnz);       // vals a
    c.take<int32_t>(sh.nnz);       // vals b
    c.take<int32_t>(sh.nnz);       // row ids
    c.take<int64_t>(256 * radix_blocks + 1);  // histogram
  }
  if (sh.G > 0) c.take<GraphDesc>(sh.G);
  if (P) {
    P->d_status = status;
    P->d_rb = rb;
    P->d_cb = cb;
    P->d_woff = woff;
    P->d_rwoff = rwoff;
    P->d_bitmap = bm;
    P->d_wprefix = wprefix;
    P->d_rbitmap = rbm;
    P->d_tile_nnz = tnnz;
    P->d_tile_nrows = trows;
    P->d_tile_cols_ptr = tcp;
    P->d_pack_ptr = pptr;
    P->d_cols_sorted = cols;
    P->d_pack_src = psrc;
    P->d_remap = remap;
    P->d_scan_tmp = scan_tmp;
    P->d_items = items;
    P->d_slot_lr = slot_lr;
    P->d_lr = lr;
    P->d_counters = counters;
    P->d_fseq = fseq;
    P->d_pchunk = pchunk;
    P->d_blk_need = blk;
    P->d_blk_done = blk + sh.Pr;
    P->fseq_cap = items_cap + pk_cap;
    P->pk_cap = pk_cap;
    P->items_cap = items_cap;
    P->slots_cap = slots_cap;
    P->lr_cap = lr_cap;
    P->d_rowptr_own = rowptr_own;
    P->d_col_own = col_own;
    P->d_val_own = val_own;
    P->d_perm = perm;
  }
  return c.off + 256;
}

// Pointers of the temporaries, re-derived from the layout order above.
struct Temps {
  uint32_t *ka, *kb;
  int32_t *va, *vb, *rowid;
  int64_t* hist;
  GraphDesc* gd;
};

static Temps carve_temps(const Shape& sh, char* base) {
  // Walk the persistent part again to find where the temporaries start.
  Carver c{base};
  const int64_t T = sh.T;
  c.take<int>(4);
  c.take<int64_t>(sh.Pr + 1);
  c.take<int64_t>(sh.Pc + 1);
  c.take<int64_t>(T + 1);
  c.take<int64_t>(T + 1);
  c.take<uint32_t>(sh.Wc);
  c.take<int64_t>(sh.Wc + 1);
  c.take<uint32_t>(sh.Wr);
  c.take<unsigned long long>(T);
  c.take<unsigned long long>(T);
  c.take<int64_t>(T + 1);
  c.take<int64_t>(T + 1);
  c.take<int32_t>(sh.cols_cap);
  if (sh.flags & SHIRO_PLAN_LOCAL_DIAG) c.take<int32_t>(sh.cols_cap);
  c.take<int32_t>(sh.nnz);
  int64_t scan_n = sh.Wc + 1;
  const int64_t radix_blocks = (sh.nnz + kRadixTile - 1) / kRadixTile;
  if (sh.transpose) scan_n = std::max<int64_t>(scan_n, 256 * radix_blocks + 1);
  c.take<int64_t>((scan_n + kScanTile - 1) / kScanTile + 2);
  const int64_t slots_cap = 2 * ((sh.nnz + 31) / 32) + 1;
  const int64_t lr_cap = (sh.nnz + 31) / 32 + 1;
  c.take<Item>(sh.M + slots_cap + 1);
  c.take<int32_t>(slots_cap);
  c.take<LongRow>(lr_cap);
  c.take<int32_t>(lr_cap);
  const int64_t pk_cap = fused_chunk_cap(sh);
  c.take<int32_t>(sh.M + slots_cap + 1 + pk_cap);
  c.take<int4>(pk_cap);
  c.take<int32_t>(2 * (int64_t)sh.Pr);
  if (sh.own_csr) {
    c.take<int64_t>(sh.M + 1);
    c.take<int32_t>(sh.nnz);
    c.take<char>(sh.nnz * (int64_t)dtype_size(sh.vdt));
  }
  if (sh.transpose) c.take<int64_t>(sh.nnz);
  Temps t{};
  if (sh.transpose) {
    t.ka = c.take<uint32_t>(sh.nnz);
    t.kb = c.take<uint32_t>(sh.nnz);
    t.va = c.take<int32_t>(sh.nnz);
    t.vb = c.take<int32_t>(sh.nnz);
    t.rowid = c.take<int32_t>(sh.nnz);
    t.hist = c.take<int64_t>(256 * radix_blocks + 1);
  }
  if (sh.G > 0) t.gd = c.take<GraphDesc>(sh.G);
  return t;
}

static shiro_status make_shape(const shiro_csr* A, const shiro_partition* part, Shape& sh) {
  if (!A || !part) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null matrix or partition");
  if (A->M < 0 || A->K < 0 || A->nnz < 0 || A->M >= INT32_MAX || A->K >= INT32_MAX)
    SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "M and K must be in [0, 2^31 - 1), nnz >= 0");
  if (A->vdt != SHIRO_F32 && A->vdt != SHIRO_F64)
    SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "CSR values must be F32 or F64");
  if (part->P_r < 1 || part->P_c < 1 || part->P_r > 65536 || part->P_c > 65536 ||
      (int64_t)part->P_r * part->P_c > (1 << 20))
    SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "grid must satisfy 1 <= P <= 65536, P_r * P_c <= 2^20");
  const uint32_t known = SHIRO_PLAN_LOCAL_DIAG | SHIRO_PLAN_DIAG_ONLY | SHIRO_PLAN_TRANSPOSE;
  if (part->flags & ~known) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "unknown plan flags");
  if ((part->flags & (SHIRO_PLAN_LOCAL_DIAG | SHIRO_PLAN_DIAG_ONLY)) && part->P_r != part->P_c)
    SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "LOCAL_DIAG and DIAG_ONLY need P_r == P_c");
  if ((part->flags & SHIRO_PLAN_LOCAL_DIAG) && (part->flags & SHIRO_PLAN_DIAG_ONLY))
    SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "LOCAL_DIAG and DIAG_ONLY are exclusive");
  std::vector<int64_t> rb, cb;
  if (part->row_bounds) rb.assign(part->row_bounds, part->row_bounds + part->P_r + 1);
  else uniform_bounds(A->M, part->P_r, rb);
  if (part->col_bounds) cb.assign(part->col_bounds, part->col_bounds + part->P_c + 1);
  else uniform_bounds(A->K, part->P_c, cb);
  SHIRO_TRY(check_bounds(rb, A->M, "row"));
  SHIRO_TRY(check_bounds(cb, A->K, "column"));
  sh.flags = part->flags;
  sh.vdt = A->vdt;
  sh.nnz = A->nnz;
  if (part->flags & SHIRO_PLAN_TRANSPOSE) {
    if (A->nnz >= INT32_MAX)
      SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "TRANSPOSE plans need nnz < 2^31 - 1");
    sh.M = A->K;
    sh.K = A->M;
    sh.Pr = part->P_c;
    sh.Pc = part->P_r;
    sh.rb = cb;
    sh.cb = rb;
    sh.own_csr = true;
    sh.transpose = true;
    sh.src_M = A->M;
  } else {
    sh.M = A->M;
    sh.K = A->K;
    sh.Pr = part->P_r;
    sh.Pc = part->P_c;
    sh.rb = rb;
    sh.cb = cb;
  }
  finish_shape(sh);
  return SHIRO_OK;
}

// ---- plan build on the device ----

static shiro_status analyse(shiro_plan_s* P, const Shape& sh, cudaStream_t s) {
  const int sms = P->sm_count;
  const int T = sh.T;
  // Geometry and bitmap offsets.
  P->woff.assign(T + 1, 0);
  P->rwoff.assign(T + 1, 0);
  const bool diag = sh.flags & SHIRO_PLAN_DIAG_ONLY;
  for (int32_t t = 0; t < T; ++t) {
    const int32_t p = diag ? t : t / sh.Pc, q = diag ? t : t % sh.Pc;
    P->woff[t + 1] = P->woff[t] + (sh.cb[q + 1] - sh.cb[q] + 31) / 32;
    P->rwoff[t + 1] = P->rwoff[t] + (sh.rb[p + 1] - sh.rb[p] + 31) / 32;
  }
  SHIRO_CUDA(cudaMemcpyAsync(P->d_rb, sh.rb.data(), sizeof(int64_t) * (sh.Pr + 1),
                             cudaMemcpyHostToDevice, s));
  SHIRO_CUDA(cudaMemcpyAsync(P->d_cb, sh.cb.data(), sizeof(int64_t) * (sh.Pc + 1),
                             cudaMemcpyHostToDevice, s));
  SHIRO_CUDA(cudaMemcpyAsync(P->d_woff, P->woff.data(), sizeof(int64_t) * (T + 1),
                             cudaMemcpyHostToDevice, s));
  SHIRO_CUDA(cudaMemcpyAsync(P->d_rwoff, P->rwoff.data(), sizeof(int64_t) * (T + 1),
                             cudaMemcpyHostToDevice, s));
  SHIRO_CUDA(cudaMemsetAsync(P->d_status, 0, sizeof(int) * 4, s));
  SHIRO_CUDA(cudaMemsetAsync(P->d_bitmap, 0, sizeof(uint32_t) * std::max<int64_t>(sh.Wc, 1), s));
  SHIRO_CUDA(cudaMemsetAsync(P->d_rbitmap, 0, sizeof(uint32_t) * std::max<int64_t>(sh.Wr, 1), s));
  SHIRO_CUDA(cudaMemsetAsync(P->d_tile_nnz, 0, sizeof(unsigned long long) * T, s));
  SHIRO_CUDA(cudaMemsetAsync(P->d_counters, 0, sizeof(int32_t) * P->lr_cap, s));

  Geometry& g = P->geo;
  g.M = sh.M;
  g.K = sh.K;
  g.Pr = sh.Pr;
  g.Pc = sh.Pc;
  g.diag_only = diag;
  g.rb = P->d_rb;
  g.cb = P->d_cb;
  std::vector<int64_t> urb, ucb;
  uniform_bounds(sh.M, sh.Pr, urb);
  uniform_bounds(sh.K, sh.Pc, ucb);
  g.uniform_r = urb == sh.rb;
  g.uniform_c = ucb == sh.cb;
  g.rstep = std::max<int64_t>(1, (sh.M + sh.Pr - 1) / sh.Pr);
  g.cstep = std::max<int64_t>(1, (sh.K + sh.Pc - 1) / sh.Pc);

  // 1. Validate rowptr before anything indexes col with it.
  k_validate_rowptr<<<grid_for(sh.M + 1, 256, sms), 256, 0, s>>>(P->rowptr, sh.M, sh.nnz,
                                                                  P->d_status);
  SHIRO_CUDA(cudaGetLastError());
  SHIRO_TRY(read_status(P, s, "plan"));

  // 2. Mark bitmaps and count nonzeros per tile (a1, a2).
  const size_t smem = T <= 4096 ? sizeof(unsigned) * T : 0;
  const int mark_grid = grid_for(sh.M * 32, 256, sms);
  if (diag)
    k_mark<true><<<mark_grid, 256, smem, s>>>(P->rowptr, P->col, g, P->d_woff, P->d_bitmap,
                                              P->d_rwoff, P->d_rbitmap, P->d_tile_nnz, T,
                                              P->d_status);
  else
    k_mark<false><<<mark_grid, 256, smem, s>>>(P->rowptr, P->col, g, P->d_woff, P->d_bitmap,
                                               P->d_rwoff, P->d_rbitmap, P->d_tile_nnz, T,
                                               P->d_status);
  SHIRO_CUDA(cudaGetLastError());
  k_tile_rows<<<grid_for((int64_t)T * 32, 256, sms), 256, 0, s>>>(P->d_rbitmap, P->d_rwoff, T,
                                                                  P->d_tile_nrows);
  SHIRO_CUDA(cudaGetLastError());

  // 3. Exclusive scan of the words' popcounts (positions in the concatenated Cols lists).
  const int64_t n = sh.Wc + 1;
  k_popc_words<<<grid_for(n, 256, sms), 256, 0, s>>>(P->d_bitmap, sh.Wc, P->d_wprefix);
  SHIRO_CUDA(cudaGetLastError());
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(P->d_wprefix, n, P->d_scan_tmp);
  k_scan_top<<<1, 1024, 0, s>>>(P->d_scan_tmp, nb, P->d_status, (int64_t)INT32_MAX - 1);
  k_scan_down<<<(unsigned)nb, kScanThreads, 0, s>>>(P->d_wprefix, n, P->d_scan_tmp);
  SHIRO_CUDA(cudaGetLastError());
  k_tile_cols_ptr<<<(T + 256) / 256, 256, 0, s>>>(P->d_wprefix, P->d_woff, T,
                                                   P->d_tile_cols_ptr);
  SHIRO_CUDA(cudaGetLastError());

  // 4. Tile statistics to the host (one synchronisation), packed offsets.
  P->tile_nnz.assign(T, 0);
  P->tile_nrows.assign(T, 0);
  P->tile_cols_ptr.assign(T + 1, 0);
  SHIRO_CUDA(cudaMemcpyAsync(P->tile_nnz.data(), P->d_tile_nnz, sizeof(int64_t) * T,
                             cudaMemcpyDeviceToHost, s));
  SHIRO_CUDA(cudaMemcpyAsync(P->tile_nrows.data(), P->d_tile_nrows, sizeof(int64_t) * T,
                             cudaMemcpyDeviceToHost, s));
  SHIRO_CUDA(cudaMemcpyAsync(P->tile_cols_ptr.data(), P->d_tile_cols_ptr,
                             sizeof(int64_t) * (T + 1), cudaMemcpyDeviceToHost, s));
  SHIRO_TRY(read_status(P, s, "plan"));
  P->tile_ncols.assign(T, 0);
  P->pack_ptr.assign(T + 1, 0);
  const bool local = sh.flags & SHIRO_PLAN_LOCAL_DIAG;
  for (int32_t t = 0; t < T; ++t) {
    P->tile_ncols[t] = P->tile_cols_ptr[t + 1] - P->tile_cols_ptr[t];
    const bool is_local = local && (t / sh.Pc == t % sh.Pc);
    P->pack_ptr[t + 1] = P->pack_ptr[t] + (is_local ? 0 : P->tile_ncols[t]);
  }
  P->total_cols = P->tile_cols_ptr[T];
  P->packed_rows = P->pack_ptr[T];
  if (P->total_cols > sh.cols_cap)
    SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "internal: Cols exceed their bound");
  SHIRO_CUDA(cudaMemcpyAsync(P->d_pack_ptr, P->pack_ptr.data(), sizeof(int64_t) * (T + 1),
                             cudaMemcpyHostToDevice, s));

  // 5. Emit the sorted Cols and the gather list; remap every nonzero (a2, a3).
  k_emit_cols<<<grid_for(std::max<int64_t>(sh.Wc, 1), 256, sms), 256, 0, s>>>(
      P->d_bitmap, sh.Wc, P->d_woff, T, g, P->d_wprefix, P->d_tile_cols_ptr, P->d_pack_ptr,
      local, P->d_cols_sorted, P->d_pack_src);
  SHIRO_CUDA(cudaGetLastError());
  if (diag)
    k_remap<true><<<mark_grid, 256, 0, s>>>(P->rowptr, P->col, g, P->d_woff, P->d_bitmap,
                                            P->d_wprefix, P->d_tile_cols_ptr, P->d_pack_ptr,
                                            0, P->d_remap, nullptr);
  else
    k_remap<false><<<mark_grid, 256, 0, s>>>(P->rowptr, P->col, g, P->d_woff, P->d_bitmap,
                                             P->d_wprefix, P->d_tile_cols_ptr, P->d_pack_ptr,
                                             local, P->d_remap, nullptr);
  SHIRO_CUDA(cudaGetLastError());

  // 6. Row lengths to the host for the schedule.
  P->h_rowptr.resize(sh.M + 1);
  SHIRO_CUDA(cudaMemcpyAsync(P->h_rowptr.data(), P->rowptr, sizeof(int64_t) * (sh.M + 1),
                             cudaMemcpyDeviceToHost, s));
  SHIRO_CUDA(cudaStreamSynchronize(s));
  P->max_row_nnz = 0;
  for (int64_t i = 0; i < sh.M; ++i)
    P->max_row_nnz = std::max(P->max_row_nnz, P->h_rowptr[i + 1] - P->h_rowptr[i]);
  return SHIRO_OK;
}

static shiro_status transpose_into(shiro_plan_s* P, const Shape& sh, const shiro_csr* A,
                                   cudaStream_t s) {
  const Temps tmp = carve_temps(sh, P->ws);
  const int sms = P->sm_count;
  const int64_t n = A->nnz;
  const int64_t blocks = (n + kRadixTile - 1) / kRadixTile;
  SHIRO_CUDA(cudaMemsetAsync(P->d_status, 0, sizeof(int) * 4, s));
  k_validate_rowptr<<<grid_for(A->M + 1, 256, sms), 256, 0, s>>>(A->rowptr, A->M, n,
                                                                  P->d_status);
  if (n > 0)
    k_validate_cols<<<grid_for(n, 256, sms), 256, 0, s>>>(A->col, n, A->K, P->d_status);
  SHIRO_CUDA(cudaGetLastError());
  SHIRO_TRY(read_status(P, s, "transpose"));
  if (n > 0) {
    k_row_ids<<<grid_for(A->M * 32, 256, sms), 256, 0, s>>>(A->rowptr, A->M, tmp.rowid);
    k_iota_copy<<<grid_for(n, 256, sms), 256, 0, s>>>(A->col, n, tmp.ka, tmp.va);
    SHIRO_CUDA(cudaGetLastError());
    int bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < A->K) ++bits;
    uint32_t *kin = tmp.ka, *kout = tmp.kb;
    int32_t *vin = tmp.va, *vout = tmp.vb;
    for (int shift = 0; shift < bits; shift += 8) {
      k_radix_hist<<<(unsigned)blocks, kRadixThreads, 0, s>>>(kin, n, shift, blocks, tmp.hist);
      const int64_t hn = 256 * blocks;
      const int64_t nb = (hn + kScanTile - 1) / kScanTile;
      k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(tmp.hist, hn, P->d_scan_tmp);
      k_scan_top<<<1, 1024, 0, s>>>(P->d_scan_tmp, nb, P->d_status, 0);
      k_scan_down<<<(unsigned)nb, kScanThreads, 0, s>>>(tmp.hist, hn, P->d_scan_tmp);
      k_radix_scatter<<<(unsigned)blocks, kRadixThreads, 0, s>>>(kin, vin, n, shift, blocks,
                                                                 tmp.hist, kout, vout);
      SHIRO_CUDA(cudaGetLastError());
      std::swap(kin, kout);
      std::swap(vin, vout);
    }
    k_rowptr_from_sorted<<<grid_for(n + 1, 256, sms), 256, 0, s>>>(kin, n, A->K,
                                                                    P->d_rowptr_own);
    if (A->vdt == SHIRO_F64)
      k_gather_transpose<double><<<grid_for(n, 256, sms), 256, 0, s>>>(
          vin, tmp.rowid, (const double*)A->val, n, P->d_col_own, (double*)P->d_val_own,
          P->d_perm);
    else
      k_gather_transpose<float><<<grid_for(n, 256, sms), 256, 0, s>>>(
          vin, tmp.rowid, (const float*)A->val, n, P->d_col_own, (float*)P->d_val_own,
          P->d_perm);
    SHIRO_CUDA(cudaGetLastError());
  } else {
    SHIRO_CUDA(cudaMemsetAsync(P->d_rowptr_own, 0, sizeof(int64_t) * (A->K + 1), s));
  }
  return SHIRO_OK;
}

// Automatic row groups: at most kAutoGroupNnz nonzeros, and at most the short rows' nonzeros
// over the resident warp slots (40 per SM for the 48-register gathers).
constexpr int64_t kAutoGroupNnz = 256;
#ifndef SHIRO_CHUNK_TILE_ORDER
#define SHIRO_CHUNK_TILE_ORDER 2
#endif
constexpr int64_t kAutoWarpsPerSm = 40;

shiro_status build_schedule(shiro_plan_s* P, const shiro_opts& o, cudaStream_t s) {
  std::vector<Item> items;
  std::vector<int32_t> slot_lr;
  std::vector<LongRow> lrs;
  const auto& rp = P->h_rowptr;
  const int64_t M = P->M;
  items.reserve((size_t)std::min<int64_t>(P->items_cap, M / 4 + 16));
  int32_t slot = 0;
  int64_t long_nnz = 0;
  for (int64_t i = 0; i < M; ++i) {
    const int64_t len = rp[i + 1] - rp[i];
    if (len > o.long_row_nnz) {
      long_nnz += len;
      const int32_t nch = (int32_t)((len + o.chunk_nnz - 1) / o.chunk_nnz);
      const int32_t lr = (int32_t)lrs.size();
      lrs.push_back({(int32_t)i, slot, nch, 0});
      for (int32_t c = 0; c < nch; ++c) {
        items.push_back({(int32_t)i, -(slot + 1), rp[i] + (int64_t)c * o.chunk_nnz});
        slot_lr.push_back(lr);
        ++slot;
      }
    }
  }
  const int64_t n_chunk_items = (int64_t)items.size();
  // Chunk items by row block, then by the column of the chunk's first nonzero (rows in order for
  // equal columns).  The chunks in flight at one time then sweep their row block's packed rows in
  // column order: a hub row's chunk covers a narrow column range, so the rows they gather form a
  // window of the packed set that stays in L2, instead of the row block's whole packed set.  A long
  // row's partial sums are added in slot order whatever order its chunks run in, so C does not
  // change.  Measured (ms; row order -> tile of the first nonzero -> its column): R-MAT 2^20
  // FP32 N = 128 SpMM 0.551 -> 0.545 -> 0.541, pack + SpMM 0.745 -> 0.739 -> 0.737, backward
  // 1.128 -> 1.105 -> 1.099; N = 64 SpMM 0.364 -> 0.360 -> 0.359; R-MAT 2^22 degree 32 BF16
  // N = 256 SpMM 5.75 -> 5.55 -> 5.30, pack + SpMM 6.70 -> 6.60 -> 6.55.
  // SHIRO_CHUNK_TILE_ORDER: 0 row order, 1 tile order, 2 column order.
  if (SHIRO_CHUNK_TILE_ORDER && n_chunk_items > 1 && P->geo.Pc > 1 &&
      !(P->flags & SHIRO_PLAN_DIAG_ONLY) && n_chunk_items <= P->fseq_cap) {
    std::vector<int32_t> c0((size_t)n_chunk_items);
    SHIRO_CUDA(cudaMemcpyAsync(P->d_items, items.data(), sizeof(Item) * (size_t)n_chunk_items,
                               cudaMemcpyHostToDevice, s));
    // The fused order's buffer is rebuilt below: a scratch for the chunks' first columns here.
    k_chunk_first_col<<<grid_for(n_chunk_items, 256, P->sm_count), 256, 0, s>>>(
        P->d_items, n_chunk_items, P->col, P->d_fseq);
    SHIRO_CUDA(cudaGetLastError());
    SHIRO_CUDA(cudaMemcpyAsync(c0.data(), P->d_fseq, sizeof(int32_t) * (size_t)n_chunk_items,
                               cudaMemcpyDeviceToHost, s));
    SHIRO_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> key((size_t)n_chunk_items);
    for (int64_t k = 0; k < n_chunk_items; ++k) {
      const int64_t p = std::upper_bound(P->rb.begin(), P->rb.end(), (int64_t)items[k].row) -
                        P->rb.begin() - 1;
      const int64_t q = std::upper_bound(P->cb.begin(), P->cb.end(), (int64_t)c0[k]) -
                        P->cb.begin() - 1;
      key[k] = SHIRO_CHUNK_TILE_ORDER == 2 ? p * (P->K + 1) + c0[k]
                                           : p * (int64_t)(P->geo.Pc + 1) + q;
    }
    std::vector<int64_t> ord((size_t)n_chunk_items);
    for (int64_t k = 0; k < n_chunk_items; ++k) ord[k] = k;
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return key[a] < key[b]; });
    std::vector<Item> sorted((size_t)n_chunk_items);
    for (int64_t k = 0; k < n_chunk_items; ++k) sorted[k] = items[ord[k]];
    std::copy(sorted.begin(), sorted.end(), items.begin());
  }
  // group_nnz 0 (automatic): kAutoGroupNnz nonzeros, or fewer when the short rows' nonzeros spread
  // over the warps the GPU keeps resident (SMs x kAutoWarpsPerSm) give less.  A small matrix then
  // has an item for every warp slot, each a short span, instead of a few warps walking long spans
  // one gather latency per step (Erdos-Renyi 4096 x 4096, 32.7 K nonzeros, N = 32: the SpMM
  // launch took 49 us with groups of 256).  Rows are never split, so C does not change.
  int64_t gnnz = o.group_nnz;
  if (gnnz == 0) {
    const int64_t slots = (int64_t)std::max(P->sm_count, 1) * kAutoWarpsPerSm;
    gnnz = std::min<int64_t>(kAutoGroupNnz,
                             std::max<int64_t>(1, (P->nnz - long_nnz + slots - 1) / slots));
  }
  // Row groups never span two row blocks, so that every item belongs to one block (the fused
  // pack + SpMM releases a block's items once the block's rows are packed).
  const int32_t Pr = P->geo.Pr;
  int32_t blk = 0;
  for (int64_t i = 0; i < M;) {
    const int64_t len = rp[i + 1] - rp[i];
    if (len > o.long_row_nnz) { ++i; continue; }
    while (blk < Pr && P->rb[blk + 1] <= i) ++blk;
    const int64_t bend = blk < Pr ? P->rb[blk + 1] : M;
    const int64_t r0 = i;
    int64_t nz = 0;
    int32_t cnt = 0;
    while (i < M && i < bend && cnt < o.group_rows) {
      const int64_t l = rp[i + 1] - rp[i];
      if (l > o.long_row_nnz) break;
      if (cnt > 0 && nz + l > gnnz) break;
      nz += l;
      ++cnt;
      ++i;
    }
    items.push_back({(int32_t)r0, cnt, rp[r0]});
  }
  if ((int64_t)items.size() > P->items_cap || (int64_t)slot_lr.size() > P->slots_cap ||
      (int64_t)lrs.size() > P->lr_cap)
    SHIRO_FAIL(SHIRO_ERR_INSUFFICIENT_WORKSPACE, "schedule does not fit the plan workspace");
  // Fused pack + SpMM order: the pack chunks of block 0, then for every block p its items (chunks
  // of long rows first) with the pack chunks of block p + 1 spread over their first three
  // quarters, so that block p + 1 is packed while block p is multiplied.
  std::vector<int32_t> fseq;
  std::vector<int4> pchunks;
  std::vector<int32_t> need(Pr, 0);
  {
    const bool diag = P->flags & SHIRO_PLAN_DIAG_ONLY;
    std::vector<std::vector<int32_t>> pk(Pr), sp(Pr);
    for (int32_t p = 0; p < Pr; ++p) {
      const int32_t t0 = diag ? p : p * P->geo.Pc, t1 = diag ? p + 1 : (p + 1) * P->geo.Pc;
      for (int64_t r = P->pack_ptr[t0]; r < P->pack_ptr[t1]; r += 32) {
        const int32_t cnt = (int32_t)std::min<int64_t>(32, P->pack_ptr[t1] - r);
        pk[p].push_back(-(int32_t)pchunks.size() - 1);
        pchunks.push_back(make_int4((int32_t)r, cnt, p, 0));
      }
      need[p] = (int32_t)pk[p].size();
    }
    // Items of each block: its chunks (in row order), then its groups (in row order).
    int32_t b = 0;
    for (int64_t it = 0; it < n_chunk_items; ++it) {
      while (b < Pr && P->rb[b + 1] <= items[it].row) ++b;
      sp[b].push_back((int32_t)it);
    }
    b = 0;
    for (int64_t it = n_chunk_items; it < (int64_t)items.size(); ++it) {
      const int64_t row = items[it].row;
      while (b < Pr && P->rb[b + 1] <= row) ++b;
      sp[b].push_back((int32_t)it);
    }
    fseq.reserve(items.size() + pchunks.size());
    if (Pr > 0) fseq.insert(fseq.end(), pk[0].begin(), pk[0].end());
    for (int32_t p = 0; p < Pr; ++p) {
      const std::vector<int32_t>& S = sp[p];
      const std::vector<int32_t> none;
      const std::vector<int32_t>& X = p + 1 < Pr ? pk[p + 1] : none;
      const int64_t span = std::max<int64_t>(1, (int64_t)S.size() * 3 / 4);
      size_t xi = 0;
      for (size_t si = 0; si < S.size(); ++si) {
        // Chunks due by item si: ceil((si + 1) * |X| / span), all of them by the span's end.
        const int64_t due = std::min<int64_t>((int64_t)X.size(),
                                              ((int64_t)si + 1) * (int64_t)X.size() / span);
        while ((int64_t)xi < due) fseq.push_back(X[xi++]);
        fseq.push_back(S[si]);
      }
      while (xi < X.size()) fseq.push_back(X[xi++]);
    }
  }
  if ((int64_t)fseq.size() > P->fseq_cap || (int64_t)pchunks.size() > P->pk_cap)
    SHIRO_FAIL(SHIRO_ERR_INSUFFICIENT_WORKSPACE, "fused schedule does not fit the plan workspace");
  if (!items.empty())
    SHIRO_CUDA(cudaMemcpyAsync(P->d_items, items.data(), sizeof(Item) * items.size(),
                               cudaMemcpyHostToDevice, s));
  if (!slot_lr.empty())
    SHIRO_CUDA(cudaMemcpyAsync(P->d_slot_lr, slot_lr.data(), sizeof(int32_t) * slot_lr.size(),
                               cudaMemcpyHostToDevice, s));
  if (!lrs.empty())
    SHIRO_CUDA(cudaMemcpyAsync(P->d_lr, lrs.data(), sizeof(LongRow) * lrs.size(),
                               cudaMemcpyHostToDevice, s));
  if (!fseq.empty())
    SHIRO_CUDA(cudaMemcpyAsync(P->d_fseq, fseq.data(), sizeof(int32_t) * fseq.size(),
                               cudaMemcpyHostToDevice, s));
  if (!pchunks.empty())
    SHIRO_CUDA(cudaMemcpyAsync(P->d_pchunk, pchunks.data(), sizeof(int4) * pchunks.size(),
                               cudaMemcpyHostToDevice, s));
  if (Pr > 0)
    SHIRO_CUDA(cudaMemcpyAsync(P->d_blk_need, need.data(), sizeof(int32_t) * Pr,
                               cudaMemcpyHostToDevice, s));
  SHIRO_CUDA(cudaMemsetAsync(P->d_counters, 0, sizeof(int32_t) * P->lr_cap, s));
  SHIRO_CUDA(cudaStreamSynchronize(s));
  P->n_fseq = (int64_t)fseq.size();
  P->n_pchunks = (int64_t)pchunks.size();
  P->n_items = (int64_t)items.size();
  P->n_long = (int64_t)lrs.size();
  P->n_slots = (int64_t)slot_lr.size();
  P->opts = o;
  return SHIRO_OK;
}

static shiro_status init_plan(shiro_plan_s* P, const Shape& sh, void* ws, size_t bytes) {
  const size_t need = carve(sh, nullptr, nullptr);
  if (!ws) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null workspace");
  if (bytes < need)
    SHIRO_FAIL(SHIRO_ERR_INSUFFICIENT_WORKSPACE, "workspace of %zu bytes, need %zu", bytes, need);
  char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  carve(sh, P, base);
  P->ws = base;
  P->ws_bytes = bytes;
  P->ws_used = need;
  P->M = sh.M;
  P->K = sh.K;
  P->nnz = sh.nnz;
  P->vdt = sh.vdt;
  P->flags = sh.flags;
  P->T = sh.T;
  P->rb = sh.rb;
  P->cb = sh.cb;
  P->Wc = sh.Wc;
  P->Wr = sh.Wr;
  P->cols_cap = sh.cols_cap;
  SHIRO_CUDA(cudaGetDevice(&P->device));
  SHIRO_CUDA(cudaDeviceGetAttribute(&P->sm_count, cudaDevAttrMultiProcessorCount, P->device));
  return SHIRO_OK;
}

}  // namespace shiro

using namespace shiro;

extern "C" {

void shiro_default_opts(shiro_opts* o) {
  if (!o) return;
  // Measured on GB300 (R-MAT 2^20 and 2^22, N = 64..256, FP32 and BF16): 512 / 256 / 256 was
  // best or within 0.3% of the best candidate on every workload.
  o->long_row_nnz = 512;
  o->chunk_nnz = 256;
  o->group_nnz = 0;  // automatic: 256, fewer for small matrices (build_schedule)
  o->group_rows = 32;
  o->warps_per_cta = 1;
  o->persistent = 0;
  o->pipeline = 0;
  o->stage_rows = 0;
}

const char* shiro_last_error(void) { return g_err.c_str(); }

int32_t shiro_version(void) { return 100; }

shiro_status shiro_set_device(int32_t device) {
  SHIRO_CUDA(cudaSetDevice(device));
  return SHIRO_OK;
}

shiro_status shiro_plan_workspace(const shiro_csr* A, const shiro_partition* part,
                                  const shiro_opts* opts, size_t* bytes) {
  if (!bytes) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null output");
  shiro_opts o;
  SHIRO_TRY(resolve_opts(opts, &o));
  Shape sh;
  SHIRO_TRY(make_shape(A, part, sh));
  *bytes = carve(sh, nullptr, nullptr);
  return SHIRO_OK;
}

shiro_status shiro_plan_create(const shiro_csr* A, const shiro_partition* part,
                               const shiro_opts* opts, void* workspace, size_t workspace_bytes,
                               void* stream, shiro_plan_t* out) {
  if (!out) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null plan output");
  *out = nullptr;
  shiro_opts o;
  SHIRO_TRY(resolve_opts(opts, &o));
  Shape sh;
  SHIRO_TRY(make_shape(A, part, sh));
  if (A->nnz > 0 && (!A->col || !A->val)) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null CSR arrays");
  if (!A->rowptr) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null rowptr");
  cudaStream_t s = (cudaStream_t)stream;
  shiro_plan_s* P = new (std::nothrow) shiro_plan_s();
  if (!P) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "out of host memory");
  shiro_status st = init_plan(P, sh, workspace, workspace_bytes);
  if (st == SHIRO_OK) {
    if (sh.transpose) {
      st = transpose_into(P, sh, A, s);
      P->rowptr = P->d_rowptr_own;
      P->col = P->d_col_own;
      P->val = P->d_val_own;
    } else {
      P->rowptr = A->rowptr;
      P->col = A->col;
      P->val = A->val;
    }
  }
  if (st == SHIRO_OK) st = analyse(P, sh, s);
  if (st == SHIRO_OK) st = build_schedule(P, o, s);
  if (st != SHIRO_OK) {
    delete P;
    return st;
  }
  *out = P;
  return SHIRO_OK;
}

void shiro_plan_destroy(shiro_plan_t plan) { delete plan; }

shiro_status shiro_plan_query(shiro_plan_t P, shiro_plan_info* info) {
  if (!P || !info) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null argument");
  info->M = P->M;
  info->K = P->K;
  info->nnz = P->nnz;
  info->P_r = P->geo.Pr;
  info->P_c = P->geo.Pc;
  info->n_tiles = P->T;
  info->flags = P->flags;
  info->vdt = P->vdt;
  info->total_cols = P->total_cols;
  info->packed_rows = P->packed_rows;
  info->n_items = P->n_items;
  info->n_long_rows = P->n_long;
  info->n_chunks = P->n_slots;
  info->workspace_used = P->ws_used;
  info->opts = P->opts;
  return SHIRO_OK;
}

shiro_status shiro_plan_tile_stats(shiro_plan_t P, int64_t* tile_nnz, int64_t* tile_nrows,
                                   int64_t* tile_ncols, int64_t* tile_cols_ptr,
                                   int64_t* pack_ptr) {
  if (!P) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null plan");
  const size_t T = (size_t)P->T;
  if (tile_nnz) memcpy(tile_nnz, P->tile_nnz.data(), T * sizeof(int64_t));
  if (tile_nrows) memcpy(tile_nrows, P->tile_nrows.data(), T * sizeof(int64_t));
  if (tile_ncols) memcpy(tile_ncols, P->tile_ncols.data(), T * sizeof(int64_t));
  if (tile_cols_ptr) memcpy(tile_cols_ptr, P->tile_cols_ptr.data(), (T + 1) * sizeof(int64_t));
  if (pack_ptr) memcpy(pack_ptr, P->pack_ptr.data(), (T + 1) * sizeof(int64_t));
  return SHIRO_OK;
}

shiro_status shiro_plan_volumes(shiro_plan_t P, int32_t N, shiro_dtype b_dt, shiro_dtype c_dt,
                                int64_t* v_block, int64_t* v_col, int64_t* v_row) {
  if (!P || N < 0) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null plan or negative N");
  auto known = [](shiro_dtype d) { return d == SHIRO_F32 || d == SHIRO_BF16 || d == SHIRO_F64; };
  if (!known(b_dt) || !known(c_dt)) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "unknown dtype");
  const int64_t szb = (int64_t)dtype_size(b_dt), szc = (int64_t)dtype_size(c_dt);
  const bool diag = P->flags & SHIRO_PLAN_DIAG_ONLY;
  const bool local = P->flags & SHIRO_PLAN_LOCAL_DIAG;
  for (int32_t t = 0; t < P->T; ++t) {
    const int32_t p = diag ? t : t / P->geo.Pc;
    const int32_t q = diag ? t : t % P->geo.Pc;
    const bool none = local && p == q;  // a local diagonal tile communicates nothing
    if (v_block) v_block[t] = none ? 0 : (P->cb[q + 1] - P->cb[q]) * N * szb;
    if (v_col) v_col[t] = none ? 0 : P->tile_ncols[t] * N * szb;
    if (v_row) v_row[t] = none ? 0 : P->tile_nrows[t] * N * szc;
  }
  return SHIRO_OK;
}

shiro_status shiro_plan_export(shiro_plan_t P, int32_t* cols_sorted, int32_t* pack_src,
                               int32_t* colidx_local, int32_t* remap, void* stream) {
  if (!P) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null plan");
  cudaStream_t s = (cudaStream_t)stream;
  if (cols_sorted && P->total_cols)
    SHIRO_CUDA(cudaMemcpyAsync(cols_sorted, P->d_cols_sorted, sizeof(int32_t) * P->total_cols,
                               cudaMemcpyDeviceToDevice, s));
  if (pack_src && P->packed_rows)
    SHIRO_CUDA(cudaMemcpyAsync(pack_src, P->d_pack_src, sizeof(int32_t) * P->packed_rows,
                               cudaMemcpyDeviceToDevice, s));
  if (remap && P->nnz)
    SHIRO_CUDA(cudaMemcpyAsync(remap, P->d_remap, sizeof(int32_t) * P->nnz,
                               cudaMemcpyDeviceToDevice, s));
  if (colidx_local && P->nnz) {
    const int grid = grid_for(P->M * 32, 256, P->sm_count);
    if (P->flags & SHIRO_PLAN_DIAG_ONLY)
      k_remap<true><<<grid, 256, 0, s>>>(P->rowptr, P->col, P->geo, P->d_woff, P->d_bitmap,
                                         P->d_wprefix, P->d_tile_cols_ptr, P->d_pack_ptr, 0,
                                         nullptr, colidx_local);
    else
      k_remap<false><<<grid, 256, 0, s>>>(P->rowptr, P->col, P->geo, P->d_woff, P->d_bitmap,
                                          P->d_wprefix, P->d_tile_cols_ptr, P->d_pack_ptr, 0,
                                          nullptr, colidx_local);
    SHIRO_CUDA(cudaGetLastError());
  }
  return SHIRO_OK;
}

shiro_status shiro_plan_export_transpose(shiro_plan_t P, int64_t* rowptr, int32_t* col,
                                         int64_t* perm, void* stream) {
  if (!P || !(P->flags & SHIRO_PLAN_TRANSPOSE))
    SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "not a TRANSPOSE plan");
  cudaStream_t s = (cudaStream_t)stream;
  if (rowptr)
    SHIRO_CUDA(cudaMemcpyAsync(rowptr, P->d_rowptr_own, sizeof(int64_t) * (P->M + 1),
                               cudaMemcpyDeviceToDevice, s));
  if (col && P->nnz)
    SHIRO_CUDA(cudaMemcpyAsync(col, P->d_col_own, sizeof(int32_t) * P->nnz,
                               cudaMemcpyDeviceToDevice, s));
  if (perm && P->nnz)
    SHIRO_CUDA(cudaMemcpyAsync(perm, P->d_perm, sizeof(int64_t) * P->nnz,
                               cudaMemcpyDeviceToDevice, s));
  return SHIRO_OK;
}

shiro_status shiro_plan_update_values(shiro_plan_t P, const void* val, void* stream) {
  if (!P || !(P->flags & SHIRO_PLAN_TRANSPOSE))
    SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "not a TRANSPOSE plan");
  if (!val && P->nnz) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null values");
  if (!P->nnz) return SHIRO_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = grid_for(P->nnz, 256, P->sm_count);
  if (P->vdt == SHIRO_F64)
    k_gather_values<double><<<grid, 256, 0, s>>>(P->d_perm, (const double*)val, P->nnz,
                                                 (double*)P->d_val_own);
  else
    k_gather_values<float><<<grid, 256, 0, s>>>(P->d_perm, (const float*)val, P->nnz,
                                                (float*)P->d_val_own);
  SHIRO_CUDA(cudaGetLastError());
  return SHIRO_OK;
}

shiro_status shiro_plan_check(shiro_plan_t P, void* stream) {
  if (!P) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null plan");
  return read_status(P, (cudaStream_t)stream, "check");
}

shiro_status shiro_plan_reschedule(shiro_plan_t P, const shiro_opts* opts, void* stream) {
  if (!P) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null plan");
  shiro_opts o;
  SHIRO_TRY(resolve_opts(opts, &o));
  return build_schedule(P, o, (cudaStream_t)stream);
}

static shiro_status batch_shape(int32_t G, const shiro_csr* graphs, Shape& sh,
                                std::vector<GraphDesc>& gd) {
  if (G < 1 || G > 65536 || !graphs) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "need 1 <= G <= 65536");
  sh.vdt = graphs[0].vdt;
  if (sh.vdt != SHIRO_F32 && sh.vdt != SHIRO_F64)
    SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "CSR values must be F32 or F64");
  sh.rb.assign(1, 0);
  sh.cb.assign(1, 0);
  gd.resize(G);
  int64_t M = 0, K = 0, nnz = 0;
  for (int32_t g = 0; g < G; ++g) {
    const shiro_csr& a = graphs[g];
    if (a.vdt != sh.vdt) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "graphs must share one value dtype");
    if (a.M < 0 || a.K < 0 || a.nnz < 0) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "negative size");
    gd[g] = {a.rowptr, a.col, a.val, a.M, a.nnz, M, K, nnz};
    M += a.M;
    K += a.K;
    nnz += a.nnz;
    sh.rb.push_back(M);
    sh.cb.push_back(K);
  }
  if (M >= INT32_MAX || K >= INT32_MAX)
    SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "batch too large: rows and columns must be < 2^31 - 1");
  sh.M = M;
  sh.K = K;
  sh.nnz = nnz;
  sh.Pr = sh.Pc = G;
  sh.flags = SHIRO_PLAN_DIAG_ONLY;
  sh.own_csr = true;
  sh.G = G;
  finish_shape(sh);
  return SHIRO_OK;
}

shiro_status shiro_batch_workspace(int32_t G, const shiro_csr* graphs, const shiro_opts* opts,
                                   size_t* bytes) {
  if (!bytes) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null output");
  shiro_opts o;
  SHIRO_TRY(resolve_opts(opts, &o));
  Shape sh;
  std::vector<GraphDesc> gd;
  SHIRO_TRY(batch_shape(G, graphs, sh, gd));
  *bytes = carve(sh, nullptr, nullptr);
  return SHIRO_OK;
}

shiro_status shiro_batch_plan_create(int32_t G, const shiro_csr* graphs, const shiro_opts* opts,
                                     void* workspace, size_t workspace_bytes, void* stream,
                                     shiro_plan_t* out) {
  if (!out) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null plan output");
  *out = nullptr;
  shiro_opts o;
  SHIRO_TRY(resolve_opts(opts, &o));
  Shape sh;
  std::vector<GraphDesc> gd;
  SHIRO_TRY(batch_shape(G, graphs, sh, gd));
  for (int32_t g = 0; g < G; ++g)
    if (!gd[g].rowptr || (gd[g].nnz > 0 && (!gd[g].col || !gd[g].val)))
      SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "graph %d has null arrays", g);
  cudaStream_t s = (cudaStream_t)stream;
  shiro_plan_s* P = new (std::nothrow) shiro_plan_s();
  if (!P) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "out of host memory");
  shiro_status st = init_plan(P, sh, workspace, workspace_bytes);
  if (st == SHIRO_OK) {
    // Validate each graph's rowptr on its own (ends and monotonicity), then concatenate.
    for (int32_t g = 0; g < G && st == SHIRO_OK; ++g) {
      cudaError_t e = cudaMemsetAsync(P->d_status, 0, sizeof(int), s);
      if (e != cudaSuccess) { set_error("cudaMemsetAsync: %s", cudaGetErrorString(e)); st = SHIRO_ERR_CUDA; break; }
      k_validate_rowptr<<<grid_for(gd[g].M + 1, 256, P->sm_count), 256, 0, s>>>(
          gd[g].rowptr, gd[g].M, gd[g].nnz, P->d_status);
      st = read_status(P, s, "batch graph");
    }
  }
  if (st == SHIRO_OK) {
    const Temps tmp = carve_temps(sh, P->ws);
    cudaError_t e = cudaMemcpyAsync(tmp.gd, gd.data(), sizeof(GraphDesc) * G,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      const int grid = std::min<int>(G, P->sm_count * 8);
      if (sh.vdt == SHIRO_F64)
        k_concat<double><<<grid, 256, 0, s>>>(tmp.gd, G, P->d_rowptr_own, P->d_col_own,
                                              (double*)P->d_val_own);
      else
        k_concat<float><<<grid, 256, 0, s>>>(tmp.gd, G, P->d_rowptr_own, P->d_col_own,
                                             (float*)P->d_val_own);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess && sh.M == 0) e = cudaMemsetAsync(P->d_rowptr_own, 0, sizeof(int64_t), s);
    if (e != cudaSuccess) { set_error("batch concat: %s", cudaGetErrorString(e)); st = SHIRO_ERR_CUDA; }
    P->rowptr = P->d_rowptr_own;
    P->col = P->d_col_own;
    P->val = P->d_val_own;
  }
  if (st == SHIRO_OK) st = analyse(P, sh, s);
  if (st == SHIRO_OK) st = build_schedule(P, o, s);
  if (st != SHIRO_OK) {
    delete P;
    return st;
  }
  *out = P;
  return SHIRO_OK;
}

}  // extern "C"
