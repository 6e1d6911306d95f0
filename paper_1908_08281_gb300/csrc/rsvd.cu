// rsvd.cu -- hgl_block_rsvd and the block preconditioner (Section 3, Algorithm 1 and
// Eq. 15).
//
// For every diagonal tessellation block b (contiguous vertex range) the dense block
// Theta_bb is assembled, and Algorithm 1 runs on it with l = k + p columns:
//   Y0 = Theta_bb Omega, S0 = QR(Y0);  q times: S~ = QR(Theta_bb S), S = QR(Theta_bb S~)
// (Theta_bb is symmetric, so the transposed products of Algorithm 1 are plain products),
// then T = S^T Theta_bb S (Rayleigh-Ritz, in place of the SVD of S^T X), T = V diag(ev) V^T,
// and Q_b = S V (top k).  Every QR is CholeskyQR2: G = Y^T Y, G = L L^T, Q = Y L^-T, twice.
// All blocks go through each step together: one grouped GEMM launch per product
// (tcgen05 tensor cores with BF16 operands, or FP64 CUDA cores for checking), one Gram,
// one Cholesky and one triangular-apply launch per orthonormalisation.
//
// The preconditioner applies z_b = r_b/(1+lam) + Q_b diag(g_b) Q_b^T r_b with
// g = ev / ((1+lam)(1+lam-ev)): the exact inverse of M_bb = (1+lam) I - Theta_bb on the
// span of Q_b, and 1/(1+lam) on its complement.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "rsvd_kernels.cuh"
#include "precond.cuh"
#include "solver.cuh"
#include "umma.cuh"

namespace hgl {
namespace {

constexpr int MAX_L = 96;

inline int64_t rup(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

hgl_status get_encoder(EncodeTiledFn* out) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
      return record_error(HGL_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  *out = fn;
  return HGL_OK;
}

}  // namespace

hgl_status encode_map_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t outer,
                         uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle sw) {
  EncodeTiledFn enc = nullptr;
  HGL_TRY(get_encoder(&enc));
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1u, 1u};
  // out-of-range elements of a box read as zero (OOB fill NONE fills zeros)
  CUresult r = enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return record_error(HGL_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return HGL_OK;
}

namespace {

// 2-D BF16 tensor map, 128-byte swizzle, box of 64 elements x box_rows rows.
hgl_status make_map(CUtensorMap* map, void* base, uint64_t inner, uint64_t outer, uint64_t row_bytes,
                    uint32_t box_rows) {
  return encode_map_2d(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, base, inner, outer, row_bytes, 64u, box_rows,
                       CU_TENSOR_MAP_SWIZZLE_128B);
}

#define HGL_LPAD_SWITCH(lp, ...)                              \
  switch (lp) {                                               \
    case 16: { constexpr int LP = 16; __VA_ARGS__; } break;   \
    case 32: { constexpr int LP = 32; __VA_ARGS__; } break;   \
    case 48: { constexpr int LP = 48; __VA_ARGS__; } break;   \
    case 64: { constexpr int LP = 64; __VA_ARGS__; } break;   \
    case 80: { constexpr int LP = 80; __VA_ARGS__; } break;   \
    default: { constexpr int LP = 96; __VA_ARGS__; } break;   \
  }

struct Work {
  // host metadata
  std::vector<int64_t> v0, arow, koff;
  std::vector<int32_t> rows, lb, kb, unit_block, unit_tile;
  int64_t rows_tot = 0, Ktot = 0, ldA = 0;
  // device pointers (inside g->rsvd)
  rsvd::Blocks B{};
  int32_t* d_unit_block = nullptr;
  int32_t* d_unit_tile = nullptr;
  void* A = nullptr;      // rows_tot x ldA (BF16 or FP64)
  void* St = nullptr;     // lpad x Ktot (BF16 or FP64)
  void* D = nullptr;      // rows_tot x lpad (FP32 or FP64)
  void* Qf = nullptr;     // rows_tot x lpad (FP32 or FP64)
  double* G = nullptr;    // nb x lpad x lpad
  double* Gpart = nullptr;  // nb x max_splits x lpad x lpad partial Grams
  int max_splits = 1;
  double* R = nullptr;    // nb x lpad x lpad
  double* ev = nullptr;   // nb x lpad
  int32_t* fail = nullptr;
  int* err = nullptr;
  bool sparse = false;    // Theta_bb S from the incidence lists (no dense blocks)
  // kept pattern of the dense blocks (plans with their own space): per storage row the
  // segments of in-block members, found once; builds clear and refill only those
  int64_t* seg_ptr = nullptr;
  rsvd::Segment* seg = nullptr;
  bool kept = false;
};

inline size_t a256(size_t b) { return (b + 255) & ~size_t(255); }

// Blocks given by their first global row v0s[b] and size sizes[b] (any ranges).
hgl_status plan_blocks(Buffer& space, const int64_t* v0s, const int64_t* sizes, int nb, int k, int l, int lpad,
                       int dtype, bool sparse, Work* w) {
  const bool bf16 = dtype == HGL_BF16;
  w->sparse = sparse;
  w->v0.resize(nb);
  w->arow.resize(nb);
  w->koff.resize(nb);
  w->rows.resize(nb);
  w->lb.resize(nb);
  w->kb.resize(nb);
  int64_t maxb = 0;
  for (int b = 0; b < nb; ++b) {
    const int64_t sz = sizes[b];
    w->v0[b] = v0s[b];
    w->rows[b] = (int32_t)sz;
    w->arow[b] = w->rows_tot;
    w->koff[b] = w->Ktot;
    w->rows_tot += rup(sz, 128);
    w->Ktot += rup(sz, 64);
    w->lb[b] = (int32_t)std::min<int64_t>(l, sz);
    w->kb[b] = (int32_t)std::min<int64_t>(k, sz);
    maxb = std::max(maxb, sz);
  }
  w->ldA = rup(maxb, 64);
  // units: 128-row tiles, blocks ordered by decreasing size (balances the persistent GEMM)
  std::vector<int> order(nb);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return w->rows[a] > w->rows[b]; });
  for (int b : order)
    for (int t = 0; t < (w->rows[b] + 127) / 128; ++t) {
      w->unit_block.push_back(b);
      w->unit_tile.push_back(t);
    }
  const size_t ea = bf16 ? 2 : 8, ed = bf16 ? 4 : 8;
  const size_t nu = w->unit_block.size();
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += a256(bytes);
    return o;
  };
  const size_t oA = take(sparse ? 0 : ea * (size_t)w->rows_tot * (size_t)w->ldA);
  const size_t oSt = take(ea * (size_t)lpad * (size_t)w->Ktot);
  const size_t oD = take(ed * (size_t)w->rows_tot * lpad);
  const size_t oQf = take(ed * (size_t)w->rows_tot * lpad);
  w->max_splits = (int)((maxb + rsvd::GRAM_SPLIT - 1) / rsvd::GRAM_SPLIT);
  const size_t oG = take(8 * (size_t)nb * lpad * lpad);
  const size_t oGp = take(8 * (size_t)nb * w->max_splits * lpad * lpad);
  const size_t oR = take(8 * (size_t)nb * lpad * lpad);
  const size_t oEv = take(8 * (size_t)nb * lpad);
  const size_t oMeta = take(8 * 3 * (size_t)nb + 4 * 3 * (size_t)nb + 4 * 2 * nu + 64);
  hgl_status st = HGL_OK;
  char* base = static_cast<char*>(buffer_get(space, off, &st));
  if (!base) return st;
  w->A = base + oA;
  w->St = base + oSt;
  w->D = base + oD;
  w->Qf = base + oQf;
  w->G = reinterpret_cast<double*>(base + oG);
  w->Gpart = reinterpret_cast<double*>(base + oGp);
  w->R = reinterpret_cast<double*>(base + oR);
  w->ev = reinterpret_cast<double*>(base + oEv);
  char* meta = base + oMeta;
  int64_t* d_v0 = reinterpret_cast<int64_t*>(meta);
  int64_t* d_arow = d_v0 + nb;
  int64_t* d_koff = d_arow + nb;
  int32_t* d_rows = reinterpret_cast<int32_t*>(d_koff + nb);
  int32_t* d_lb = d_rows + nb;
  int32_t* d_kb = d_lb + nb;
  w->d_unit_block = d_kb + nb;
  w->d_unit_tile = w->d_unit_block + nu;
  w->fail = w->d_unit_tile + nu;
  w->err = w->fail + 1;
  // one host staging buffer, one copy
  std::vector<char> hmeta(8 * 3 * (size_t)nb + 4 * 3 * (size_t)nb + 4 * 2 * nu + 8, 0);
  char* h = hmeta.data();
  memcpy(h, w->v0.data(), 8 * nb);
  memcpy(h + 8 * nb, w->arow.data(), 8 * nb);
  memcpy(h + 16 * nb, w->koff.data(), 8 * nb);
  memcpy(h + 24 * nb, w->rows.data(), 4 * nb);
  memcpy(h + 28 * nb, w->lb.data(), 4 * nb);
  memcpy(h + 32 * nb, w->kb.data(), 4 * nb);
  memcpy(h + 36 * nb, w->unit_block.data(), 4 * nu);
  memcpy(h + 36 * nb + 4 * nu, w->unit_tile.data(), 4 * nu);
  HGL_CHECK_CUDA(cudaMemcpy(meta, hmeta.data(), hmeta.size(), cudaMemcpyHostToDevice));
  rsvd::Blocks& B = w->B;
  B.nb = nb;
  B.l = l;
  B.lpad = lpad;
  B.k = k;
  B.ldA = w->ldA;
  B.Ktot = w->Ktot;
  B.v0 = d_v0;
  B.rows = d_rows;
  B.arow = d_arow;
  B.koff = d_koff;
  B.lb = d_lb;
  B.kb = d_kb;
  return HGL_OK;
}

// Contiguous tessellation blocks [bp[b], bp[b + 1]).
hgl_status plan(hgl_graph* g, Buffer& space, const int64_t* bp, int nb, int k, int l, int lpad, int dtype,
                bool sparse, Work* w) {
  (void)g;
  std::vector<int64_t> v0s(bp, bp + nb), sizes(nb);
  for (int b = 0; b < nb; ++b) sizes[b] = bp[b + 1] - bp[b];
  return plan_blocks(space, v0s.data(), sizes.data(), nb, k, l, lpad, dtype, sparse, w);
}

template <class F>
hgl_status set_smem(F* fn, size_t bytes) {
  HGL_CHECK_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void*>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)bytes));
  return HGL_OK;
}

// D = Theta_bb * S for all blocks: the grouped GEMM over the dense blocks (St holds
// S^T), or on the sparse route the product straight from the incidence lists (Qf
// holds S).
template <int LP>
hgl_status gemm(const hgl_graph* g, const Work& w, int dtype, int sms, cudaStream_t st) {
  if (w.sparse) {
    ProfScope prof(HGL_PROF_BLOCKSPMM, st);
    hgl::count_launch();
    rsvd::k_block_spmm<LP><<<sms * 8, 256, 0, st>>>(w.B, w.rows_tot, g->csr_ptr, g->csr_idx, g->csc_ptr, g->csc_idx,
                                                    g->s, g->t, static_cast<const float*>(w.Qf),
                                                    static_cast<float*>(w.D));
    HGL_CHECK_CUDA(cudaGetLastError());
    return HGL_OK;
  }
  const int nu = (int)w.unit_block.size();
  ProfScope prof(HGL_PROF_GEMM, st);
  if (dtype == HGL_BF16) {
    CUtensorMap ma, mb;
    HGL_TRY(make_map(&ma, w.A, (uint64_t)w.ldA, (uint64_t)w.rows_tot, (uint64_t)w.ldA * 2, 128));
    HGL_TRY(make_map(&mb, w.St, (uint64_t)w.Ktot, (uint64_t)LP, (uint64_t)w.Ktot * 2, LP));
    umma::GemmUnits U{w.d_unit_block, w.d_unit_tile, w.B.rows, w.B.arow, w.B.koff, nu};
    const size_t smem = umma::gemm_smem_bytes(LP);
    HGL_TRY(set_smem(umma::k_block_gemm<LP>, smem));
    const int grid = std::min(nu, sms);
    hgl::count_launch(); umma::k_block_gemm<LP><<<grid, umma::THREADS, smem, st>>>(ma, mb, U, static_cast<float*>(w.D), LP, w.err);
  } else {
    const int grid = std::min(nu, sms * 4);
    hgl::count_launch(); rsvd::k_block_gemm_f64<LP><<<grid, 256, 0, st>>>(w.B, w.d_unit_block, w.d_unit_tile, nu,
                                                      static_cast<const double*>(w.A),
                                                      static_cast<const double*>(w.St), static_cast<double*>(w.D));
  }
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

// G = X^T Y per block (partials over row ranges, then a fixed-order sum)
template <class T, int LP>
hgl_status gram(const Work& w, const T* X, const T* Y, cudaStream_t st) {
  const int nb = w.B.nb;
  hgl::count_launch(2);
  const bool sym = X == Y;
  if (sym)
    rsvd::k_gram_part<T, LP, true><<<nb * w.max_splits, 256, 0, st>>>(w.B, w.max_splits, X, Y, w.Gpart);
  else
    rsvd::k_gram_part<T, LP, false><<<nb * w.max_splits, 256, 0, st>>>(w.B, w.max_splits, X, Y, w.Gpart);
  rsvd::k_gram_reduce<LP><<<nb, 256, 0, st>>>(w.B, w.max_splits, w.Gpart, w.G, sym);
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

// Q = CholeskyQR2(D): G = D^T D, Rinv = chol^-T, Qf = D Rinv; again on Qf.  The final
// pass also refreshes the transposed basis St (when write_st).  passes = 1 stops after
// the first (shifted) factorisation: a basis of the same span whose orthonormality is
// off by about the shift over the smallest squared singular value -- enough between
// the products of the subspace iteration, whose last orthonormalisation takes both.
template <class T, class TB, int LP>
hgl_status cholqr2(const Work& w, int dtype, int sms, cudaStream_t st, bool write_st, int passes = 2) {
  const int nb = w.B.nb;
  const int nu = (int)w.unit_block.size();
  const size_t chol_smem = 2 * sizeof(double) * LP * (LP + 1);
  HGL_TRY(set_smem(rsvd::k_chol_inv<LP>, chol_smem));
  const size_t ap_smem = sizeof(T) * (LP * LP + 128 * (LP + 1));
  HGL_TRY(set_smem(rsvd::k_apply_rinv<T, TB, LP>, ap_smem));
  // first pass: a small shift keeps the factorisation defined; both passes drop
  // pivots at the working precision's noise level (rank-deficient blocks)
  const double shift = dtype == HGL_BF16 ? 1e-6 : 1e-14;
  const double drop = dtype == HGL_BF16 ? 1e-6 : 1e-13;
  const T* Y = static_cast<const T*>(w.D);
  T* Qf = static_cast<T*>(w.Qf);
  for (int pass = 0; pass < passes; ++pass) {
    HGL_TRY((gram<T, LP>(w, Y, Y, st)));
    hgl::count_launch(); rsvd::k_chol_inv<LP><<<nb, 256, chol_smem, st>>>(w.B, w.G, pass == 0 ? shift : 0.0, drop, w.R, w.fail);
    const bool last = pass == passes - 1;
    // in-place on the second pass is fine: each tile reads its rows before writing them
    hgl::count_launch(); rsvd::k_apply_rinv<T, TB, LP><<<std::min(nu, sms * 4), 256, ap_smem, st>>>(
        w.B, w.d_unit_block, w.d_unit_tile, nu, Y, w.R, Qf, (last && write_st) ? static_cast<TB*>(w.St) : nullptr);
    HGL_CHECK_CUDA(cudaGetLastError());
    Y = Qf;
  }
  return HGL_OK;
}

}  // namespace

// A block rSVD plan: the host metadata and device work space of one block layout
// (Work), and the preconditioner handle its builds write.  Creating it allocates and
// uploads; computing it only launches kernels, so a plan can be rebuilt inside a
// captured CUDA graph.
struct PrecondPlan {
  Work wk;
  hgl_precond* P = nullptr;
  Buffer own;            // the plan's own work space (graph plans); else g->rsvd
  Buffer pattern;        // kept pattern of the dense blocks (own-space BF16 plans)
  int dtype = HGL_BF16;
  int q = 0;
};

hgl_status precond_validate(const hgl_graph* g, const int64_t* bp, int32_t nb, int32_t k, int32_t p, int32_t q,
                            int gemm_dtype) {
  if (!bp || nb < 1) return record_error(HGL_ERR_INVALID_ARG, "block_ptr is NULL or nblocks < 1");
  if (k < 1 || p < 0 || q < 0 || k + p > MAX_L)
    return record_error(HGL_ERR_INVALID_ARG, "need k >= 1, p >= 0, q >= 0 and k + p <= %d", MAX_L);
  if (gemm_dtype != HGL_BF16 && gemm_dtype != HGL_FP64)
    return record_error(HGL_ERR_INVALID_ARG, "gemm_dtype must be HGL_BF16 or HGL_FP64");
  if (bp[0] != 0 || bp[nb] != g->n) return record_error(HGL_ERR_INVALID_ARG, "block_ptr must run from 0 to n");
  for (int b = 0; b < nb; ++b)
    if (bp[b + 1] <= bp[b]) return record_error(HGL_ERR_INVALID_ARG, "blocks must be non-empty and increasing");
  return HGL_OK;
}

// Route of the products Theta_bb S on the BF16 path: the graph's setting, or by fill
// (auto): the tcgen05 GEMM streams every dense block entry (2 bytes, 2 lpad flops),
// measured at ~3e12 entries/s with lpad = 80; the sparse route gathers one basis row
// (4 lpad bytes) per block entry after a binary search, measured at ~8e9 entries/s.
// Sparse when the blocks' entries are at most 1/512 of their dense size.  Synchronous.
static hgl_status block_route_sparse(hgl_graph* g, const int64_t* bp, int nb, cudaStream_t st, bool* sparse) {
  if (g->block_product != HGL_BLOCKS_AUTO) {
    *sparse = g->block_product == HGL_BLOCKS_SPARSE;
    return HGL_OK;
  }
  double dense = 0.0;
  for (int b = 0; b < nb; ++b) dense += (double)rup(bp[b + 1] - bp[b], 128) * (double)rup(bp[b + 1] - bp[b], 64);
  void* mem = nullptr;
  HGL_CHECK_CUDA(cudaMalloc(&mem, 8 * (size_t)(nb + 2)));
  int64_t* d_bp = static_cast<int64_t*>(mem);
  unsigned long long* d_cnt = reinterpret_cast<unsigned long long*>(d_bp + nb + 1);
  unsigned long long cnt = 0;
  cudaError_t e = cudaMemcpyAsync(d_bp, bp, 8 * (size_t)(nb + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, 8, st);
  if (e == cudaSuccess) {
    hgl::count_launch();
    rsvd::k_block_nnz<<<g->num_sms * 8, 256, 0, st>>>(g->n, nb, d_bp, g->csr_ptr, g->csr_idx, g->csc_ptr,
                                                      g->csc_idx, d_cnt);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, d_cnt, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(mem);
  if (e != cudaSuccess) return cuda_error(e, "block fill count", __FILE__, __LINE__);
  *sparse = 512.0 * (double)cnt <= dense;
  return HGL_OK;
}

// The dense blocks' pattern of an own-space plan: segment counts per storage row, their
// offsets (scanned on the host, once), the segments; then the block storage zeroed once.
// Synchronous.
static hgl_status keep_pattern(hgl_graph* g, PrecondPlan* pl, cudaStream_t st) {
  Work& wk = pl->wk;
  const int64_t rows = wk.rows_tot;
  void* tmp = nullptr;
  HGL_CHECK_CUDA(cudaMalloc(&tmp, sizeof(unsigned) * (size_t)rows));
  std::vector<unsigned> cnt(rows);
  hgl::count_launch();
  rsvd::k_segment_count<<<g->num_sms * 8, 256, 0, st>>>(wk.B, rows, g->csr_ptr, g->csr_idx, g->csc_ptr, g->csc_idx,
                                                        static_cast<unsigned*>(tmp));
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.data(), tmp, sizeof(unsigned) * (size_t)rows, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_error(e, "block pattern count", __FILE__, __LINE__);
  std::vector<int64_t> ptr(rows + 1, 0);
  for (int64_t r = 0; r < rows; ++r) ptr[r + 1] = ptr[r] + cnt[r];
  const size_t ptr_bytes = (sizeof(int64_t) * (size_t)(rows + 1) + 255) & ~size_t(255);
  hgl_status s = HGL_OK;
  char* base = static_cast<char*>(
      buffer_get(pl->pattern, ptr_bytes + sizeof(rsvd::Segment) * (size_t)std::max<int64_t>(ptr[rows], 1), &s));
  if (!base) return s;
  wk.seg_ptr = reinterpret_cast<int64_t*>(base);
  wk.seg = reinterpret_cast<rsvd::Segment*>(base + ptr_bytes);
  HGL_CHECK_CUDA(cudaMemcpyAsync(wk.seg_ptr, ptr.data(), sizeof(int64_t) * (size_t)(rows + 1), cudaMemcpyHostToDevice, st));
  hgl::count_launch();
  rsvd::k_segment_fill<<<g->num_sms * 8, 256, 0, st>>>(wk.B, rows, g->csr_ptr, g->csr_idx, g->csc_ptr, g->csc_idx,
                                                       wk.seg_ptr, wk.seg);
  HGL_CHECK_CUDA(cudaGetLastError());
  HGL_CHECK_CUDA(cudaMemsetAsync(wk.A, 0, sizeof(__nv_bfloat16) * (size_t)rows * (size_t)wk.ldA, st));
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  wk.kept = true;
  return HGL_OK;
}

void precond_plan_destroy(PrecondPlan* pl) {
  if (!pl) return;
  if (pl->P) hgl_precond_destroy(pl->P);
  buffer_free(pl->own);
  buffer_free(pl->pattern);
  delete pl;
}

// Plan, work space (own buffer if own_space, else the graph's shared one), handle.
// Synchronous (uploads the block metadata).
hgl_status precond_plan_create(const hgl_graph* gc, double lam, const int64_t* bp, int32_t nb, int32_t k, int32_t p,
                               int32_t q, int gemm_dtype, bool own_space, cudaStream_t st, PrecondPlan** out) {
  hgl_graph* g = const_cast<hgl_graph*>(gc);
  *out = nullptr;
  HGL_TRY(precond_validate(g, bp, nb, k, p, q, gemm_dtype));
  const int l = k + p;
  const int lpad = (int)rup(l, 16);
  PrecondPlan* pl = new (std::nothrow) PrecondPlan();
  if (!pl) return record_error(HGL_ERR_OOM, "host allocation failed");
  pl->dtype = gemm_dtype;
  pl->q = q;
  bool sparse = false;
  hgl_status s_ = gemm_dtype == HGL_BF16 ? block_route_sparse(g, bp, nb, st, &sparse) : HGL_OK;
  if (s_ != HGL_OK) {
    precond_plan_destroy(pl);
    return s_;
  }
  s_ = plan(g, own_space ? pl->own : g->rsvd, bp, nb, k, l, lpad, gemm_dtype, sparse, &pl->wk);
  if (s_ == HGL_OK && own_space && gemm_dtype == HGL_BF16 && !sparse) s_ = keep_pattern(g, pl, st);
  if (s_ != HGL_OK) {
    precond_plan_destroy(pl);
    return s_;
  }
  const Work& wk = pl->wk;
  const bool bf16 = gemm_dtype == HGL_BF16;
  // the handle: Q (n x k), gains, eigenvalues, block metadata and the apply's units
  hgl_precond* P = new (std::nothrow) hgl_precond();
  if (!P) {
    precond_plan_destroy(pl);
    return record_error(HGL_ERR_OOM, "host allocation failed");
  }
  pl->P = P;
  P->g = g;
  P->n = g->n;
  P->nb = nb;
  P->k = k;
  P->l = l;
  P->lpad = lpad;
  P->lam = lam;
  P->dtype = gemm_dtype;
  P->bptr.assign(bp, bp + nb + 1);
  P->kb = wk.kb;
  std::vector<int32_t> ub, ut;
  for (int b = 0; b < nb; ++b)
    for (int t = 0; t < (wk.rows[b] + 63) / 64; ++t) {  // 64-row units of the apply
      ub.push_back(b);
      ut.push_back(t);
    }
  P->nunits = (int)ub.size();
  std::vector<int32_t> sb, sr0, bs0, eb, et;
  for (int b = 0; b < nb; ++b) {
    bs0.push_back((int32_t)sb.size());
    for (int r0 = 0; r0 < wk.rows[b]; r0 += PC_SLAB) {
      sb.push_back(b);
      sr0.push_back(r0);
    }
    for (int t = 0; t < (wk.rows[b] + PC_TILE - 1) / PC_TILE; ++t) {
      eb.push_back(b);
      et.push_back(t);
    }
  }
  bs0.push_back((int32_t)sb.size());
  P->nslabs = (int)sb.size();
  P->nexp = (int)eb.size();
  const size_t eq = bf16 ? 4 : 8;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += a256(bytes);
    return o;
  };
  const size_t oQ = take(eq * (size_t)g->n * k);
  const size_t oGain = take(8 * (size_t)nb * k);
  const size_t oEv = take(8 * (size_t)nb * k);
  const size_t oV0 = take(8 * (size_t)(nb + 1));
  const size_t oRows = take(4 * (size_t)nb);
  const size_t oKb = take(4 * (size_t)nb);
  const size_t oUb = take(4 * ub.size());
  const size_t oUt = take(4 * ut.size());
  const size_t oSb = take(4 * sb.size());
  const size_t oSr = take(4 * sr0.size());
  const size_t oBs = take(4 * bs0.size());
  const size_t oEb = take(4 * eb.size());
  const size_t oEt = take(4 * et.size());
  // tensor-core apply: FP32 factors of rank <= 64, split into TF32 pairs
  P->tc = bf16 && k <= 64;
  P->kp = k <= 32 ? 32 : 64;
  P->n4 = rup(g->n, 4);
  const size_t tcq = P->tc ? 4 * (size_t)g->n * P->kp : 0;
  const size_t tcqt = P->tc ? 4 * (size_t)P->kp * P->n4 : 0;
  const size_t oQh = take(tcq), oQl = take(tcq), oQTh = take(tcqt), oQTl = take(tcqt);
  const size_t oG32 = take(P->tc ? 4 * (size_t)nb * k : 0);
  const size_t oOrd = take(4 * (size_t)nb);
  const size_t oErr = take(4);
  std::vector<int32_t> order(nb);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return wk.rows[a] > wk.rows[b]; });
  cudaError_t e = cudaMalloc(&P->dev, off);
  if (e != cudaSuccess) {
    P->dev = nullptr;
    precond_plan_destroy(pl);
    return cuda_error(e, "cudaMalloc(preconditioner)", __FILE__, __LINE__);
  }
  char* base = static_cast<char*>(P->dev);
  P->Q = base + oQ;
  P->gain = reinterpret_cast<double*>(base + oGain);
  P->ev = reinterpret_cast<double*>(base + oEv);
  P->d_v0 = reinterpret_cast<int64_t*>(base + oV0);
  P->d_rows = reinterpret_cast<int32_t*>(base + oRows);
  P->d_kb = reinterpret_cast<int32_t*>(base + oKb);
  P->unit_block = reinterpret_cast<int32_t*>(base + oUb);
  P->unit_tile = reinterpret_cast<int32_t*>(base + oUt);
  P->slab_block = reinterpret_cast<int32_t*>(base + oSb);
  P->slab_row0 = reinterpret_cast<int32_t*>(base + oSr);
  P->blk_slab0 = reinterpret_cast<int32_t*>(base + oBs);
  P->exp_block = reinterpret_cast<int32_t*>(base + oEb);
  P->exp_tile = reinterpret_cast<int32_t*>(base + oEt);
  if (P->tc) {
    P->Qh = reinterpret_cast<float*>(base + oQh);
    P->Ql = reinterpret_cast<float*>(base + oQl);
    P->QTh = reinterpret_cast<float*>(base + oQTh);
    P->QTl = reinterpret_cast<float*>(base + oQTl);
    P->gain32 = reinterpret_cast<float*>(base + oG32);
  }
  P->blk_order = reinterpret_cast<int32_t*>(base + oOrd);
  P->d_err = reinterpret_cast<int32_t*>(base + oErr);
  hgl_status fin = HGL_OK;
  auto chk = [&](cudaError_t ce) {
    if (ce != cudaSuccess && fin == HGL_OK) fin = cuda_error(ce, "preconditioner setup", __FILE__, __LINE__);
  };
  chk(cudaMemcpyAsync(P->d_v0, bp, 8 * (size_t)(nb + 1), cudaMemcpyHostToDevice, st));
  chk(cudaMemcpyAsync(P->d_rows, wk.rows.data(), 4 * (size_t)nb, cudaMemcpyHostToDevice, st));
  chk(cudaMemcpyAsync(P->d_kb, wk.kb.data(), 4 * (size_t)nb, cudaMemcpyHostToDevice, st));
  chk(cudaMemcpyAsync(P->unit_block, ub.data(), 4 * ub.size(), cudaMemcpyHostToDevice, st));
  chk(cudaMemcpyAsync(P->unit_tile, ut.data(), 4 * ut.size(), cudaMemcpyHostToDevice, st));
  chk(cudaMemcpyAsync(P->slab_block, sb.data(), 4 * sb.size(), cudaMemcpyHostToDevice, st));
  chk(cudaMemcpyAsync(P->slab_row0, sr0.data(), 4 * sr0.size(), cudaMemcpyHostToDevice, st));
  chk(cudaMemcpyAsync(P->blk_slab0, bs0.data(), 4 * bs0.size(), cudaMemcpyHostToDevice, st));
  chk(cudaMemcpyAsync(P->exp_block, eb.data(), 4 * eb.size(), cudaMemcpyHostToDevice, st));
  chk(cudaMemcpyAsync(P->exp_tile, et.data(), 4 * et.size(), cudaMemcpyHostToDevice, st));
  chk(cudaMemcpyAsync(P->blk_order, order.data(), 4 * (size_t)nb, cudaMemcpyHostToDevice, st));
  chk(cudaMemsetAsync(P->d_err, 0, 4, st));
  chk(cudaStreamSynchronize(st));  // the host vectors above go out of scope
  if (fin == HGL_OK && P->tc) fin = precond_tc_maps(P);
  if (fin != HGL_OK) {
    precond_plan_destroy(pl);
    return fin;
  }
  *out = pl;
  return HGL_OK;
}

// Launches only: Algorithm 1 on every block at the graph's current degrees, the
// Rayleigh-Ritz vectors and the gains, into the plan's handle.  The Omega seed is
// `seed`, or *seed_dev when seed_dev is given (read on the device).
hgl_status precond_plan_compute(const hgl_graph* gc, PrecondPlan* pl, uint64_t seed, const uint64_t* seed_dev,
                                cudaStream_t st) {
  hgl_graph* g = const_cast<hgl_graph*>(gc);
  Work& wk = pl->wk;
  hgl_precond* P = pl->P;
  const int gemm_dtype = pl->dtype;
  const int q = pl->q;
  const int nb = wk.B.nb;
  const int k = wk.B.k;
  const int lpad = wk.B.lpad;
  const int sms = g->num_sms;
  (void)k;
  ProfScope prof(HGL_PROF_RSVD, st);
  HGL_CHECK_CUDA(cudaMemsetAsync(wk.fail, 0, 8, st));
  const bool bf16 = gemm_dtype == HGL_BF16;

  // dense diagonal blocks and the Gaussian start basis (sparse route: the basis only,
  // in the row layout the sparse product reads)
  if (bf16 && wk.sparse) {
    HGL_LPAD_SWITCH(lpad, {
      hgl::count_launch();
      rsvd::k_omega_rows<LP><<<sms * 8, 256, 0, st>>>(wk.B, wk.rows_tot, seed, seed_dev, static_cast<float*>(wk.Qf));
    });
  } else if (bf16) {
    hgl::count_launch(2);
    if (wk.kept)
      rsvd::k_assemble_kept<__nv_bfloat16, float><<<sms * 8, 256, 0, st>>>(
          wk.B, wk.rows_tot, g->csr_ptr, g->csr_idx, g->csc_idx, wk.seg_ptr, wk.seg, g->s32, g->t32,
          static_cast<__nv_bfloat16*>(wk.A));
    else
      rsvd::k_assemble<__nv_bfloat16, float><<<sms * 8, 256, 0, st>>>(
          wk.B, wk.rows_tot, g->csr_ptr, g->csr_idx, g->csc_ptr, g->csc_idx, g->s32, g->t32,
          static_cast<__nv_bfloat16*>(wk.A));
    rsvd::k_omega<__nv_bfloat16><<<sms * 8, 256, 0, st>>>(wk.B, seed, seed_dev,
                                                         static_cast<__nv_bfloat16*>(wk.St));
  } else {
    hgl::count_launch(2);
    rsvd::k_assemble<double, double><<<sms * 8, 256, 0, st>>>(wk.B, wk.rows_tot, g->csr_ptr, g->csr_idx, g->csc_ptr,
                                                     g->csc_idx, g->s, g->t, static_cast<double*>(wk.A));
    rsvd::k_omega<double><<<sms * 8, 256, 0, st>>>(wk.B, seed, seed_dev, static_cast<double*>(wk.St));
  }
  HGL_CHECK_CUDA(cudaGetLastError());

  // Algorithm 1: 1 + 2q products each followed by an orthonormalisation, then W = Theta S
  const int nprod = 1 + 2 * q;
  hgl_status s_ = HGL_OK;
  HGL_LPAD_SWITCH(lpad, {
    for (int i = 0; i < nprod && s_ == HGL_OK; ++i) {
      s_ = gemm<LP>(g, wk, gemm_dtype, sms, st);
      // BF16 route: one CholeskyQR pass between products, two for the final basis (the
      // FP64 checking route keeps two throughout)
      if (s_ == HGL_OK)
        s_ = bf16 ? cholqr2<float, __nv_bfloat16, LP>(wk, gemm_dtype, sms, st, !wk.sparse, i + 1 < nprod ? 1 : 2)
                  : cholqr2<double, double, LP>(wk, gemm_dtype, sms, st, true);
    }
    if (s_ == HGL_OK) s_ = gemm<LP>(g, wk, gemm_dtype, sms, st);
    if (s_ == HGL_OK) {
      // T = S^T (Theta S), eigendecomposition, Ritz vectors
      s_ = bf16 ? gram<float, LP>(wk, static_cast<const float*>(wk.Qf), static_cast<const float*>(wk.D), st)
                : gram<double, LP>(wk, static_cast<const double*>(wk.Qf), static_cast<const double*>(wk.D), st);
      if (bf16) {
        // FP32 rotations: the BF16 products bound the accuracy of T well above FP32's
        const size_t jsm = 2 * sizeof(float) * LP * (LP + 1);
        if (s_ == HGL_OK) s_ = set_smem(rsvd::k_jacobi<float, LP>, jsm);
        if (s_ == HGL_OK) {
          hgl::count_launch();
          rsvd::k_jacobi<float, LP><<<nb, 256, jsm, st>>>(wk.B, wk.G, wk.R, wk.ev, 16, 1e-10);
        }
      } else {
        const size_t jsm = 2 * sizeof(double) * LP * (LP + 1);
        if (s_ == HGL_OK) s_ = set_smem(rsvd::k_jacobi<double, LP>, jsm);
        if (s_ == HGL_OK) {
          hgl::count_launch();
          rsvd::k_jacobi<double, LP><<<nb, 256, jsm, st>>>(wk.B, wk.G, wk.R, wk.ev, 40, 1e-30);
        }
      }
    }
  });
  HGL_TRY(s_);
  HGL_CHECK_CUDA(cudaGetLastError());

  const int nu = (int)wk.unit_block.size();
  HGL_LPAD_SWITCH(lpad, {
    if (bf16) {
      const size_t rs = sizeof(float) * (LP * LP + 128 * (LP + 1));
      s_ = set_smem(rsvd::k_ritz<float, LP>, rs);
      if (s_ == HGL_OK) {
        hgl::count_launch();
        rsvd::k_ritz<float, LP><<<std::min(nu, sms * 4), 256, rs, st>>>(
            wk.B, wk.d_unit_block, wk.d_unit_tile, nu, static_cast<const float*>(wk.Qf), wk.R,
            static_cast<float*>(P->Q));
      }
    } else {
      const size_t rs = sizeof(double) * (LP * LP + 128 * (LP + 1));
      s_ = set_smem(rsvd::k_ritz<double, LP>, rs);
      if (s_ == HGL_OK) {
        hgl::count_launch();
        rsvd::k_ritz<double, LP><<<std::min(nu, sms * 4), 256, rs, st>>>(
            wk.B, wk.d_unit_block, wk.d_unit_tile, nu, static_cast<const double*>(wk.Qf), wk.R,
            static_cast<double*>(P->Q));
      }
    }
  });
  HGL_TRY(s_);
  HGL_CHECK_CUDA(cudaGetLastError());
  HGL_TRY(precond_gains_launch(P, wk.ev, lpad, st));
  return P->tc ? precond_tc_prepare(P, st) : HGL_OK;
}

// The device status words of the last compute: HGL_ERR_TIMEOUT if the tensor-core
// GEMM gave up a wait.  Synchronises the stream.
hgl_status precond_plan_check(PrecondPlan* pl, cudaStream_t st) {
  int32_t flags[2] = {0, 0};
  HGL_CHECK_CUDA(cudaMemcpyAsync(flags, pl->wk.fail, 8, cudaMemcpyDeviceToHost, st));
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  if (flags[1] != 0) return record_error(HGL_ERR_TIMEOUT, "the tensor-core GEMM hit its wait limit");
  return precond_tc_status(pl->P, st);
}

const hgl_precond* precond_plan_handle(const PrecondPlan* pl) { return pl->P; }

hgl_status precond_build(const hgl_graph* gc, const double* w, double lam, const int64_t* bp, int32_t nb, int32_t k,
                         int32_t p, int32_t q, uint64_t seed, int gemm_dtype, cudaStream_t st, hgl_precond** out,
                         bool degrees_ready) {
  hgl_graph* g = const_cast<hgl_graph*>(gc);
  *out = nullptr;
  HGL_TRY(precond_validate(g, bp, nb, k, p, q, gemm_dtype));
  if (!degrees_ready) HGL_TRY(degrees_launch(g, w, st));
  PrecondPlan* pl = nullptr;
  HGL_TRY(precond_plan_create(g, lam, bp, nb, k, p, q, gemm_dtype, false, st, &pl));
  hgl_status s_ = precond_plan_compute(g, pl, seed, nullptr, st);
  if (s_ == HGL_OK) s_ = precond_plan_check(pl, st);
  if (s_ == HGL_OK) {
    *out = pl->P;
    pl->P = nullptr;
  }
  precond_plan_destroy(pl);
  return s_;
}
}  // namespace hgl

// D_b = Theta_bb S_b for every diagonal block, by the products of the BF16 builds (the
// tcgen05 grouped GEMM over dense BF16 blocks, or the sparse route, as the graph's
// block-product setting chooses).  Synchronous.
extern "C" hgl_status hgl_block_product(const hgl_graph* gc, const double* w, const int64_t* block_ptr,
                                        int32_t nblocks, int32_t l, const float* S, int64_t lds, float* D,
                                        int64_t ldd, void* stream) {
  using namespace hgl;
  hgl_graph* g = const_cast<hgl_graph*>(gc);
  if (!g || !w || !S || !D) return record_error(HGL_ERR_INVALID_ARG, "NULL argument");
  if (l < 1 || l > MAX_L) return record_error(HGL_ERR_INVALID_ARG, "l must be in [1, %d]", MAX_L);
  HGL_TRY(precond_validate(g, block_ptr, nblocks, l, 0, 0, HGL_BF16));
  if (lds < l || ldd < l) return record_error(HGL_ERR_INVALID_ARG, "leading dimensions must be >= l");
  cudaStream_t st = as_stream(stream);
  HGL_TRY(degrees_launch(g, w, st));
  bool sparse = false;
  HGL_TRY(block_route_sparse(g, block_ptr, nblocks, st, &sparse));
  const int lpad = (int)rup(l, 16);
  Work wk;
  HGL_TRY(plan(g, g->rsvd, block_ptr, nblocks, l, l, lpad, HGL_BF16, sparse, &wk));
  const int sms = g->num_sms;
  hgl_status s_ = HGL_OK;
  HGL_LPAD_SWITCH(lpad, {
    if (sparse) {
      hgl::count_launch();
      rsvd::k_rows_to_blockrows<LP><<<sms * 8, 256, 0, st>>>(wk.B, wk.rows_tot, S, lds, l, static_cast<float*>(wk.Qf));
    } else {
      hgl::count_launch(2);
      rsvd::k_assemble<__nv_bfloat16, float><<<sms * 8, 256, 0, st>>>(
          wk.B, wk.rows_tot, g->csr_ptr, g->csr_idx, g->csc_ptr, g->csc_idx, g->s32, g->t32,
          static_cast<__nv_bfloat16*>(wk.A));
      rsvd::k_rows_to_st<__nv_bfloat16><<<sms * 8, 256, 0, st>>>(wk.B, S, lds, l,
                                                                 static_cast<__nv_bfloat16*>(wk.St));
    }
    s_ = cudaGetLastError() == cudaSuccess ? HGL_OK : record_error(HGL_ERR_CUDA, "block product setup launch");
    if (s_ == HGL_OK) s_ = cudaMemsetAsync(wk.fail, 0, 8, st) == cudaSuccess ? HGL_OK
                                                                          : record_error(HGL_ERR_CUDA, "memset");
    if (s_ == HGL_OK) s_ = gemm<LP>(g, wk, HGL_BF16, sms, st);
    if (s_ == HGL_OK) {
      hgl::count_launch();
      rsvd::k_blockrows_to_rows<LP><<<sms * 8, 256, 0, st>>>(wk.B, g->n, static_cast<const float*>(wk.D), l, D, ldd);
      s_ = cudaGetLastError() == cudaSuccess ? HGL_OK : record_error(HGL_ERR_CUDA, "block product copy-out launch");
    }
  });
  HGL_TRY(s_);
  int32_t flags[2] = {0, 0};
  HGL_CHECK_CUDA(cudaMemcpyAsync(flags, wk.fail, 8, cudaMemcpyDeviceToHost, st));
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  if (flags[1] != 0) return record_error(HGL_ERR_TIMEOUT, "the tensor-core GEMM hit its wait limit");
  return HGL_OK;
}

namespace hgl {

// Algorithm 1 (Rayleigh-Ritz form, FP64 on CUDA cores) on nb dense matrices at once:
// the symmetric part of L_b (sizes[b] x sizes[b], row stride ldls[b], device pointer
// Ls[b]), the Gaussian test matrix drawn for the global rows v0s[b] .. (the same Philox
// stream as the block preconditioner), l = min(k + p, size) columns, q subspace
// iterations; every step one launch for all matrices.  Ritz vectors of matrix b go to
// rows v0s[b] - qrow0 .. of Qout (row-major, k columns; columns past min(k, size) are
// zero), its Ritz values, descending, to ev[b * k ..].  The row ranges must not overlap.
// Work space from `space`.  Asynchronous after the plan's metadata upload (which first
// lets earlier work on `st` finish: it rewrites metadata that work may read).
hgl_status dense_rsvd_batch_fp64(int nb, const double* const* Ls, const int64_t* ldls, const int64_t* v0s,
                                 const int64_t* sizes, int k, int p, int q, uint64_t seed, Buffer& space,
                                 double* Qout, int64_t qrow0, double* ev, cudaStream_t st) {
  if (nb < 1 || k < 1 || p < 0 || q < 0 || k + p > MAX_L)
    return record_error(HGL_ERR_INVALID_ARG, "dense rSVD: need nb >= 1, k >= 1, p, q >= 0, k + p <= %d", MAX_L);
  const int l = k + p;
  const int lpad = (int)rup(l, 16);
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  Work wk;
  HGL_TRY(plan_blocks(space, v0s, sizes, nb, k, l, lpad, HGL_FP64, false, &wk));
  int dev = 0, sms = 0;
  HGL_CHECK_CUDA(cudaGetDevice(&dev));
  HGL_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HGL_CHECK_CUDA(cudaMemsetAsync(wk.fail, 0, 8, st));
  double* A = static_cast<double*>(wk.A);
  for (int b = 0; b < nb; ++b) {
    const int64_t rows_b = rup(sizes[b], 128);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((rows_b * wk.ldA + 255) / 256, sms * 8));
    hgl::count_launch();
    rsvd::k_sym_load<<<grid, 256, 0, st>>>(sizes[b], rows_b, wk.ldA, Ls[b], ldls[b], A + wk.arow[b] * wk.ldA);
  }
  hgl::count_launch();
  rsvd::k_omega<double><<<sms * 8, 256, 0, st>>>(wk.B, seed, nullptr, static_cast<double*>(wk.St));
  HGL_CHECK_CUDA(cudaGetLastError());
  hgl_status s_ = HGL_OK;
  HGL_LPAD_SWITCH(lpad, {
    for (int i = 0; i < 1 + 2 * q && s_ == HGL_OK; ++i) {
      s_ = gemm<LP>(nullptr, wk, HGL_FP64, sms, st);
      if (s_ == HGL_OK) s_ = cholqr2<double, double, LP>(wk, HGL_FP64, sms, st, true);
    }
    if (s_ == HGL_OK) s_ = gemm<LP>(nullptr, wk, HGL_FP64, sms, st);
    if (s_ == HGL_OK)
      s_ = gram<double, LP>(wk, static_cast<const double*>(wk.Qf), static_cast<const double*>(wk.D), st);
    const size_t jsm = 2 * sizeof(double) * LP * (LP + 1);
    if (s_ == HGL_OK) s_ = set_smem(rsvd::k_jacobi<double, LP>, jsm);
    if (s_ == HGL_OK) {
      hgl::count_launch();
      rsvd::k_jacobi<double, LP><<<nb, 256, jsm, st>>>(wk.B, wk.G, wk.R, wk.ev, 40, 1e-30);
    }
    const size_t rs = sizeof(double) * (LP * LP + 128 * (LP + 1));
    if (s_ == HGL_OK) s_ = set_smem(rsvd::k_ritz<double, LP>, rs);
    if (s_ == HGL_OK) {
      // the Ritz kernel writes global row v0 + i of its output: offset the base so that
      // row v0 + i - qrow0 of Qout receives it
      hgl::count_launch();
      const int nu = (int)wk.unit_block.size();
      rsvd::k_ritz<double, LP><<<std::min(nu, sms * 4), 256, rs, st>>>(
          wk.B, wk.d_unit_block, wk.d_unit_tile, nu, static_cast<const double*>(wk.Qf), wk.R, Qout - qrow0 * k);
    }
    if (s_ == HGL_OK) {
      const cudaError_t ce = cudaMemcpy2DAsync(ev, sizeof(double) * k, wk.ev, sizeof(double) * LP, sizeof(double) * k,
                                               nb, cudaMemcpyDeviceToDevice, st);
      if (ce != cudaSuccess) s_ = cuda_error(ce, "Ritz values", __FILE__, __LINE__);
    }
  });
  HGL_TRY(s_);
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

}  // namespace hgl

// Route of the BF16 build's products, chosen by timing them on this graph: the dense
// route costs one assembly of the dense BF16 blocks plus 2q + 2 tcgen05 products, the
// sparse route 2q + 2 products from the incidence lists.  Each is timed (CUDA events)
// after a warm-up; the faster becomes the graph's block-product setting.  Synchronous.
extern "C" hgl_status hgl_tune_block_rsvd(hgl_graph* g, const double* w, const int64_t* block_ptr, int32_t nblocks,
                                          int32_t k, int32_t p, int32_t q, int32_t* route, double* ms_dense,
                                          double* ms_sparse, void* stream) {
  using namespace hgl;
  if (!g || !w) return record_error(HGL_ERR_INVALID_ARG, "graph or w is NULL");
  HGL_TRY(precond_validate(g, block_ptr, nblocks, k, p, q, HGL_BF16));
  cudaStream_t st = as_stream(stream);
  HGL_TRY(degrees_launch(g, w, st));
  const int l = k + p;
  const int lpad = (int)rup(l, 16);
  const int sms = g->num_sms;
  const int nprod = 2 * q + 2;
  double ms[2] = {0.0, 0.0};
  Buffer space;
  hgl_status s_ = HGL_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  HGL_CHECK_CUDA(cudaEventCreate(&e0));
  HGL_CHECK_CUDA(cudaEventCreate(&e1));
  for (int sparse = 0; sparse < 2 && s_ == HGL_OK; ++sparse) {
    Work wk;
    s_ = plan(g, space, block_ptr, nblocks, k, l, lpad, HGL_BF16, sparse != 0, &wk);
    if (s_ != HGL_OK) break;
    auto once = [&]() -> hgl_status {
      HGL_CHECK_CUDA(cudaMemsetAsync(wk.fail, 0, 8, st));
      HGL_LPAD_SWITCH(lpad, {
        if (sparse) {
          hgl::count_launch();
          rsvd::k_omega_rows<LP><<<sms * 8, 256, 0, st>>>(wk.B, wk.rows_tot, 1, nullptr, static_cast<float*>(wk.Qf));
        } else {
          hgl::count_launch(2);
          rsvd::k_assemble<__nv_bfloat16, float><<<sms * 8, 256, 0, st>>>(
              wk.B, wk.rows_tot, g->csr_ptr, g->csr_idx, g->csc_ptr, g->csc_idx, g->s32, g->t32,
              static_cast<__nv_bfloat16*>(wk.A));
          rsvd::k_omega<__nv_bfloat16><<<sms * 8, 256, 0, st>>>(wk.B, 1, nullptr, static_cast<__nv_bfloat16*>(wk.St));
        }
        HGL_CHECK_CUDA(cudaGetLastError());
        for (int i = 0; i < nprod; ++i) HGL_TRY(gemm<LP>(g, wk, HGL_BF16, sms, st));
      });
      return HGL_OK;
    };
    s_ = once();  // warm-up
    if (s_ != HGL_OK) break;
    HGL_CHECK_CUDA(cudaEventRecord(e0, st));
    s_ = once();
    if (s_ != HGL_OK) break;
    HGL_CHECK_CUDA(cudaEventRecord(e1, st));
    HGL_CHECK_CUDA(cudaEventSynchronize(e1));
    float t = 0.f;
    HGL_CHECK_CUDA(cudaEventElapsedTime(&t, e0, e1));
    ms[sparse] = t;
    int32_t flags[2] = {0, 0};
    HGL_CHECK_CUDA(cudaMemcpy(flags, wk.fail, 8, cudaMemcpyDeviceToHost));
    if (flags[1] != 0) s_ = record_error(HGL_ERR_TIMEOUT, "the tensor-core GEMM hit its wait limit");
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  buffer_free(space);
  HGL_TRY(s_);
  g->block_product = ms[1] < ms[0] ? HGL_BLOCKS_SPARSE : HGL_BLOCKS_DENSE;
  if (route) *route = g->block_product;
  if (ms_dense) *ms_dense = ms[0];
  if (ms_sparse) *ms_sparse = ms[1];
  return HGL_OK;
}
