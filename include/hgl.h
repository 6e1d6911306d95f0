/*
 * hgl.h -- C ABI of libhgl: adaptive hypergraph learning on NVIDIA GB300 (sm_103a).
 *
 * Method: Karantaidis, Sarridis and Kotropoulos, "Block randomized optimization for
 * adaptive hypergraph learning" (arXiv 1908.08281), Sections 2 and 3.
 *
 * Notation (the paper's Section 2 swaps the letters n and m):
 *   n vertices, m hyperedges, c right-hand-side (tag) columns, nnz incidences;
 *   H (n x m, 0/1) incidence; w (m) hyperedge weights; dv = H w; de = H^T 1;
 *   Theta = Dv^-1/2 H W De^-1 H^T Dv^-1/2                          (Eq. 1, the paper's A)
 *   Delta = I - Theta                                              (Zhou's Laplacian)
 *   ranking system  M F = lam Y,  M = (1 + lam) I - Theta          (Eqs. 3 and 6 times 1+lam)
 *   P(w) = tr(F^T Delta F) + mu ||w||^2,  1^T w = 1, w >= 0         (Eq. 4)
 * A vertex with dv = 0 gets Dv^-1/2 = 0 (pseudo-inverse), so its row and column of
 * Theta vanish.
 *
 * Conventions shared by every entry point
 *   - Panels (X, Y, F, Z, ...) are caller-owned DEVICE memory, row-major n x c with a
 *     leading dimension ld >= c (in elements); the base address must be 16-byte
 *     aligned and ld * element_size a multiple of 16 bytes, else HGL_ERR_INVALID_ARG.
 *     Columns c .. ld-1 are never written.
 *   - Vectors (w, grad, dv, ...) are caller-owned device arrays of FP64.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Calls are ordered on that stream.  Entry points that return statistics to the
 *     host synchronise the stream before returning; the others are asynchronous.
 *   - Opaque handles (hgl_graph, hgl_precond) are library-owned: create/destroy pairs.
 *     A handle holds device work buffers, so two calls on the same handle must not
 *     run concurrently (on different streams or host threads).
 *   - No exception crosses the ABI and nothing aborts.  A failed CUDA call returns
 *     HGL_ERR_CUDA (or HGL_ERR_OOM) and hgl_last_error() describes it.
 */
#ifndef HGL_H_
#define HGL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t hgl_status;

#define HGL_OK                    0
#define HGL_ERR_INVALID_ARG      -1  /* bad size, pointer, alignment or option            */
#define HGL_ERR_INDEX_RANGE      -2  /* a member vertex id outside [0, n)                  */
#define HGL_ERR_DUPLICATE_MEMBER -3  /* a vertex listed twice in one hyperedge (H is 0/1)   */
#define HGL_ERR_EMPTY_EDGE       -4  /* a hyperedge with no members (De^-1 undefined)       */
#define HGL_ERR_OOM              -5  /* device allocation failed                            */
#define HGL_ERR_CUDA             -6  /* a CUDA runtime call failed                          */
#define HGL_ERR_NOT_CONVERGED    -7  /* an iteration reached its limit before its tolerance */
#define HGL_ERR_TIMEOUT          -8  /* a device-side wait hit its spin limit               */
#define HGL_ERR_NONFINITE        -9  /* NaN or Inf met in a reduction                       */

/* Element type of a panel. */
typedef enum {
  HGL_FP64 = 0,
  HGL_FP32 = 1,
  HGL_BF16 = 2
} hgl_dtype;

/* Human-readable name of a status code (static string, never NULL). */
const char* hgl_status_string(hgl_status s);

/* Text of the last error met by the calling host thread ("" if none). */
const char* hgl_last_error(void);

/* Library version as 10000*major + 100*minor + patch. */
int32_t hgl_version(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (diagnostics; differences around a call count that call's launches). */
uint64_t hgl_launch_count(void);

/*
 * Kernel timing (diagnostics).  While enabled, the library records a CUDA event pair
 * on the launching stream around every launch of the kernel families below; the
 * totals are read back with hgl_profile_read, which synchronises the device.
 * hgl_profile_enable(1) clears the totals and starts recording; (0) stops.
 */
#define HGL_PROF_OPERATOR 0   /* operator apply: hyperedge + vertex gather passes      */
#define HGL_PROF_RESIDUAL 1   /* pair-arithmetic residual: its two gather passes        */
#define HGL_PROF_GEMM     2   /* block rSVD grouped GEMM (tcgen05 or FP64 CUDA cores)   */
#define HGL_PROF_GRADIENT 3   /* weight gradient: its two gather passes and final sum   */
#define HGL_PROF_PRECOND  4   /* block preconditioner apply (projection + expansion)    */
#define HGL_PROF_RSVD     5   /* whole block rSVD build (assembly, Omega, the GEMMs,    */
                              /* CholeskyQR2, Jacobi, Ritz vectors)                     */
#define HGL_PROF_VECTOR   6   /* CG vector updates and panel dot products/copies        */
#define HGL_PROF_PROJECT  7   /* simplex projection                                     */
#define HGL_PROF_OPRESID  8   /* residual from one operator pass with the residual      */
                              /* epilogue (FP32 estimate of the mixed solvers, FP64     */
                              /* residual of the FP64 solver)                           */
#define HGL_PROF_BLOCKSPMM 9  /* block rSVD products Theta_bb S on the sparse route    */
#define HGL_PROF_SCHUR_GEMM 10 /* dense products of the nested Schur-complement inverse */
#define HGL_PROF_FAMILIES 11
hgl_status hgl_profile_enable(int32_t on);
hgl_status hgl_profile_read(int32_t family, double* ms_total, int64_t* launches);

/*
 * hgl_selftest_wait_timeout -- failure detection without a GPU fault: runs the bounded
 * device wait that every tcgen05 kernel uses (an mbarrier poll that gives up after a
 * cycle limit, records the error in a device status word and returns) on a barrier
 * that nothing arrives on, with a limit of limit_cycles SM cycles (1 .. 8e9; the
 * kernels' own limit is 4e9, about 2 s).  Returns HGL_ERR_TIMEOUT, the status a kernel
 * reports when one of its waits runs out; the device stays usable.  Synchronises
 * `stream`.
 */
hgl_status hgl_selftest_wait_timeout(int64_t limit_cycles, void* stream);

/*
 * hgl_selftest_pair_split -- the conversions between an FP64 panel and the FP32 pair
 * (hi, lo) that the mixed-precision solver keeps its iterate in (refinement around an
 * FP32 CG whose residual is recomputed FP64-accurately), run on given values: for each
 * i, hi[i] = x[i] rounded to FP32 (nearest-even), lo[i] = x[i] - hi[i] rounded to FP32,
 * back[i] = (double)hi[i] + (double)lo[i] in FP64.  The solver computes these from the
 * IEEE-754 bit fields (no FP64 arithmetic in range) and this call exposes them for a test
 * against the plain FP64 definitions.  The paper has no counterpart: the refinement
 * around a low-precision CG is this library's way of reaching FP64 accuracy.
 *   x     device FP64[len];  hi, lo  device FP32[len];  back  device FP64[len]
 * Asynchronous on `stream`.  Errors: HGL_ERR_INVALID_ARG (NULL arrays, len < 0).
 */
hgl_status hgl_selftest_pair_split(const double* x, int64_t len, float* hi, float* lo, double* back, void* stream);

/* ------------------------------------------------------------------------- */
/* Incidence (Section 2: H(v,e) = 1 iff v in e; de(e) = sum_v H(v,e))         */
/* ------------------------------------------------------------------------- */

typedef struct hgl_graph hgl_graph;

/*
 * hgl_build_incidence -- build the device incidence structure from member lists.
 *   n, m       vertex and hyperedge counts (n >= 1, m >= 1, both < 2^31)
 *   edge_ptr   int64[m+1], host or device: hyperedge e owns members[edge_ptr[e] ..
 *              edge_ptr[e+1]); edge_ptr[0] = 0, non-decreasing, edge_ptr[m] = nnz
 *   members    int32[nnz], host or device, any order inside a hyperedge
 *   nnz        number of incidences (< 2^31)
 *   out        receives a new handle on success (NULL on failure)
 * Builds, bit-exactly and deterministically: the hyperedge-major layout (members of
 * each hyperedge in ascending order), the vertex-major layout (hyperedges of each
 * vertex in ascending order) and de.  Validation errors: HGL_ERR_INVALID_ARG
 * (pointer array), HGL_ERR_EMPTY_EDGE, HGL_ERR_INDEX_RANGE, HGL_ERR_DUPLICATE_MEMBER.
 * A vertex in no hyperedge is allowed.  Synchronises `stream`.
 */
hgl_status hgl_build_incidence(int64_t n, int64_t m, const int64_t* edge_ptr,
                               const int32_t* members, int64_t nnz, void* stream,
                               hgl_graph** out);

/* Release a graph handle and all of its device memory (NULL is a no-op). */
void hgl_graph_destroy(hgl_graph* g);

/* Sizes of a graph (any output pointer may be NULL). */
hgl_status hgl_graph_info(const hgl_graph* g, int64_t* n, int64_t* m, int64_t* nnz);

/*
 * hgl_graph_export -- copy the layouts into caller-owned DEVICE arrays (any may be
 * NULL): csc_ptr int64[m+1], csc_idx int32[nnz] (hyperedge -> sorted members),
 * csr_ptr int64[n+1], csr_idx int32[nnz] (vertex -> sorted hyperedges), de int32[m].
 * Asynchronous on `stream`.
 */
hgl_status hgl_graph_export(const hgl_graph* g, int64_t* csc_ptr, int32_t* csc_idx,
                            int64_t* csr_ptr, int32_t* csr_idx, int32_t* de, void* stream);

/*
 * hgl_degrees -- dv = H w, s = dv^-1/2 (0 where dv <= 0), t = w / de (Section 2,
 * the scalings of Eq. 1).  w: device FP64[m]; outputs device FP64 dv[n], s[n],
 * t[m] (any may be NULL).  Asynchronous.
 */
hgl_status hgl_degrees(const hgl_graph* g, const double* w, double* dv, double* s,
                       double* t, void* stream);

/* ------------------------------------------------------------------------- */
/* Operator (Eq. 1)                                                          */
/* ------------------------------------------------------------------------- */

/*
 * hgl_apply_theta -- Z = a X + b Theta(w) X, applied matrix-free from H (Eq. 1);
 * (a, b) = (1 + lam, -1) gives Z = M X.
 *   w        device FP64[m] (w >= 0 expected; dv <= 0 gives s = 0)
 *   X, Z     device panels n x c of type `dtype`, leading dimensions ldx, ldz; X and
 *            Z must not overlap.  FP64 panels accumulate in FP64; FP32 and BF16
 *            panels accumulate in FP32 (the intermediate m x c panel is FP32).
 * Uses a graph-owned scratch panel of m x min(c, chunk) accumulators, allocated on
 * first use.  Asynchronous.
 */
hgl_status hgl_apply_theta(const hgl_graph* g, const double* w, double a, double b,
                           const void* X, int64_t ldx, void* Z, int64_t ldz, int32_t c,
                           hgl_dtype dtype, void* stream);

/*
 * hgl_apply_theta_noalloc -- the same operator apply as hgl_apply_theta (same
 * arguments, same result up to the summation order of a narrower column chunk),
 * but the call allocates no device memory.  The paper has no counterpart: this entry
 * point serves callers that cannot let a library allocate during the call, such as
 * programs that route all device memory through their own pool or fixed budget, and
 * loops that cannot take the implicit synchronisation of cudaMalloc/cudaFree.
 * hgl_apply_theta allocates its m x chunk intermediate panel on first use; this
 * variant uses instead a 32 MiB array compiled into the library's device image
 * (every GPU that loads libhgl holds it until the process exits), narrowing the
 * column chunk to fit.  Limit: m <= 2,097,152 for FP64 and FP32 panels and
 * m <= 1,048,576 for BF16 panels, else HGL_ERR_INVALID_ARG (nothing launched).
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it; make that first
 * call before any stream capture.  The cached address belongs to the device's
 * context: after cudaDeviceReset the next call would use a stale address, so a
 * program that resets a device must not call this entry point on it again.  All
 * calls share the one array and it keeps the
 * last call's contents; it needs no clearing, since the hyperedge pass writes every
 * entry that the vertex pass then reads.  Calls that overlap on the GPU (on
 * different streams, or from different host threads) race on the array and give
 * wrong results: order them.  The graph handle's degree vectors are allocated when
 * the graph is built, so they are not allocated here either.  Asynchronous.
 */
hgl_status hgl_apply_theta_noalloc(const hgl_graph* g, const double* w, double a, double b,
                                   const void* X, int64_t ldx, void* Z, int64_t ldz,
                                   int32_t c, hgl_dtype dtype, void* stream);

/*
 * hgl_tune_operator -- choose, by timing on this graph, the column chunk that the
 * operator apply (Eq. 1) uses for c-column panels of `dtype`, and for FP32/BF16 also
 * the chunk of the FP64-accurate pair residual that the mixed-precision solvers use.
 * The paper has no counterpart: the chunk trades one long burst per gathered row
 * against re-reading the index arrays once per chunk, and the best width depends on
 * n, m, c, the panel type and the degree distribution.  The chunks are timed in the
 * variant the CG launches (for BF16 search directions: FP32 Z, with the column
 * partials of X.Z), and for the pair residual in both its full and compact forms.  At
 * the chosen chunk it also times the grid of the gather passes (the blocks resident at
 * once, one wave, or eight blocks per SM; eight only when more than 3% faster).  The
 * choices are stored in the graph and used by every later call with the same
 * (dtype, c); untuned graphs use 512-byte row chunks (64 FP64, 128 FP32 or 256 BF16
 * columns) and one-wave grids.  Results of later calls may differ from untuned ones in summation
 * order only (each column's sums are unchanged for the operator; the pair residual
 * is FP64-accurate either way).  Allocates and frees temporary panels (3 n x c plus,
 * for FP32/BF16, about 6 n x c floats).
 *   w               device FP64[m] weights (sets the graph's degree vectors)
 *   chunk_cols      optional host out: the chosen operator chunk in columns
 *   pair_chunk_cols optional host out: the chosen residual chunk (0 for FP64)
 *   grid_policy     optional host out: the chosen grid (0 = one wave of resident
 *                   blocks, 1 = eight blocks per SM)
 * Synchronises `stream`.
 */
hgl_status hgl_tune_operator(hgl_graph* g, const double* w, int32_t c, hgl_dtype dtype,
                             int32_t* chunk_cols, int32_t* pair_chunk_cols, int32_t* grid_policy,
                             void* stream);

/* ------------------------------------------------------------------------- */
/* Solve (Eq. 6 by conjugate gradient, Eqs. 16-20)                           */
/* ------------------------------------------------------------------------- */

typedef struct hgl_precond hgl_precond;

#define HGL_SOLVE_WARM_START 1   /* F holds the initial guess f_0 (else f_0 = 0) */

typedef struct {
  double  tol;         /* per-column target ||lam y_j - M f_j|| <= tol ||lam y_j||       */
  int32_t max_iter;    /* cap on CG iterations (all refinement sweeps together)          */
  int32_t dtype;       /* HGL_FP64: plain FP64 CG.  HGL_FP32: CG on FP32 panels with     */
                       /* FP32 arithmetic, inside FP64 iterative refinement (residual    */
                       /* recomputed FP64-accurately from F).  HGL_BF16: the same with   */
                       /* the search directions stored in BF16 (the operator's input;    */
                       /* its product, the residual and the iterate stay FP32)           */
  double  inner_tol;   /* mixed modes: floor of the relative reduction asked of each     */
                       /* inner solve; a sweep aims at max(inner_tol, 0.75 tol/relres)   */
                       /* (0 = 1e-5)                                                     */
  int32_t max_refine;  /* mixed modes: cap on refinement sweeps (0 = 8)                  */
  int32_t flags;       /* HGL_SOLVE_WARM_START                                           */
} hgl_solve_opts;

typedef struct {
  hgl_status status;     /* HGL_OK or HGL_ERR_NOT_CONVERGED / HGL_ERR_NONFINITE          */
  int32_t iters;         /* CG iterations done (max over columns, all sweeps together)   */
  int32_t refinements;   /* FP64 residual recomputations after the first (mixed modes)  */
  int32_t converged;     /* number of columns that met tol                               */
  double  relres_max;    /* max over columns of ||lam y_j - M f_j|| / ||lam y_j||,       */
                         /* recomputed from the returned F in FP64                        */
} hgl_solve_stats;

/*
 * hgl_cg_solve -- solve M F = lam Y for all c columns (independent CG per column).
 *   w          device FP64[m];  lam > 0
 *   Y          device FP64 panel n x c (ldy)
 *   F          device FP64 panel n x c (ldf): initial guess if HGL_SOLVE_WARM_START,
 *              solution on return
 *   precond    NULL, or a block preconditioner from hgl_block_rsvd built for this
 *              graph (then the recurrences are those of preconditioned CG)
 *   relres     optional device FP64[c]: per-column final relative residual
 *   iters      optional device int32[c]: per-column iteration count
 *   stats      optional host struct
 * A zero column of Y gives F_j = 0.  Returns HGL_ERR_NOT_CONVERGED if some column
 * missed tol within max_iter (F then holds the last iterate).  Synchronises `stream`.
 */
hgl_status hgl_cg_solve(const hgl_graph* g, const double* w, double lam, const double* Y,
                        int64_t ldy, double* F, int64_t ldf, int32_t c,
                        const hgl_precond* precond, const hgl_solve_opts* opts,
                        double* relres, int32_t* iters, hgl_solve_stats* stats,
                        void* stream);

/*
 * hgl_block_cg_solve -- M F = lam Y by block CG with a shared Krylov space (O'Leary 1980)
 * over groups of s columns (the last group may be narrower), FP64: per group
 *   R = lam Y - M F, P = orth(R); repeat Q = M P, a = (P^T Q)^+ P^T R, F += P a,
 *   R -= Q a, stop when every column has ||r_j|| <= tol ||lam y_j||,
 *   b = -(P^T Q)^+ Q^T R, P = orth(R + P b),
 * with orth = CholeskyQR2 on unit-normalised columns and dropped pivots (the
 * breakdown-free form of Ji and Li, 2017: converged or dependent directions leave the
 * search block).  A pivot of the unit-diagonal Gram below 1e-12 drops its direction,
 * i.e. singular values below 1e-6 of the column norms (the Gram squares them).  The
 * groups share every launch; with s = 1 this is CG.  A zero column of Y gives F_j = 0
 * (a warm start in that column is discarded) and reports relres_j = ||r_j|| = 0.
 *   Y, F      device FP64 n x c, leading dimensions ldy, ldf; F is read as f_0 with
 *             flags & HGL_SOLVE_WARM_START (else f_0 = 0) and holds the solution
 *   s         columns per group, 1 .. 32
 *   relres    optional device FP64[c]: the recomputed ||lam y_j - M f_j|| / ||lam y_j||
 *   iters     optional device int32[ceil(c/s)]: iterations per group
 * Allocates its work space (7 panels n x c and small per-group arrays) per call.
 * Returns HGL_ERR_NOT_CONVERGED or HGL_ERR_NONFINITE as hgl_cg_solve does.
 * Synchronises `stream`.
 */
hgl_status hgl_block_cg_solve(const hgl_graph* g, const double* w, double lam, const double* Y,
                              int64_t ldy, double* F, int64_t ldf, int32_t c, int32_t s, double tol,
                              int32_t max_iter, int32_t flags, double* relres, int32_t* iters,
                              void* stream);

/* ------------------------------------------------------------------------- */
/* Block randomized SVD (Section 3, Algorithm 1) as a block preconditioner   */
/* ------------------------------------------------------------------------- */

/*
 * hgl_block_rsvd -- tessellate the vertex range into contiguous diagonal blocks
 * [block_ptr[b], block_ptr[b+1]) (Section 3) and approximate each dense Theta_bb by
 * randomized subspace iteration (Algorithm 1) with l = k + p columns and q
 * iterations: Y0 = Theta_bb Omega, then q times two products each followed by an
 * orthonormalisation (CholeskyQR2), then the Rayleigh-Ritz factorisation
 * Theta_bb ~= Q_b diag(ev_b) Q_b^T (top k).  The handle then applies
 *   z_b = r_b / (1+lam) + Q_b diag(ev/((1+lam)(1+lam-ev))) Q_b^T r_b,
 * the inverse of M_bb = (1+lam) I - Theta_bb on the captured subspace (Eq. 15 with the
 * identity part of M kept).
 *   block_ptr  HOST int64[nblocks+1], 0 = block_ptr[0] < ... < block_ptr[nblocks] = n
 *   k, p, q    rank, oversampling, iterations (k >= 1, p >= 0, q >= 0)
 *   seed       seed of the Philox4x32-10 Gaussian test matrix Omega (see below)
 *   gemm_dtype HGL_BF16: products Theta_bb S with FP32 accumulation, by the route of
 *              hgl_set_block_product (dense BF16 blocks on the tcgen05 tensor cores,
 *              or FP32 straight from the incidence lists); HGL_FP64: dense FP64
 *              blocks, all products in FP64 on the CUDA cores (slow; for checking)
 * Omega[g, j] for global vertex row g and column j: x = Philox4x32-10(counter
 * (g, j>>1, 0x4F6D6567, 0), key (seed & 0xffffffff, seed >> 32)); u1, u2 in (0,1) from
 * (x0,x1) and (x2,x3) as ((hi>>5)*2^26 + (lo>>6) + 1/2) * 2^-53; Omega = sqrt(-2 ln u1)
 * times cos(2 pi u2) for even j, sin(2 pi u2) for odd j (Box-Muller).
 * Synchronises `stream`.
 */
hgl_status hgl_block_rsvd(const hgl_graph* g, const double* w, double lam,
                          const int64_t* block_ptr, int32_t nblocks, int32_t k, int32_t p,
                          int32_t q, uint64_t seed, hgl_dtype gemm_dtype, void* stream,
                          hgl_precond** out);

/*
 * hgl_set_block_product -- route of the BF16 path's products Theta_bb S for
 * preconditioners built on g afterwards (including the captured steps' own):
 *   HGL_BLOCKS_DENSE   assemble the diagonal blocks as dense BF16 matrices and multiply
 *                      them on the tcgen05 tensor cores (grouped GEMM): cost set by the
 *                      sum of the squared block sizes;
 *   HGL_BLOCKS_SPARSE  no dense blocks: each vertex row of Theta_bb S is summed from
 *                      its hyperedges' members inside its block (found by binary search
 *                      in the sorted member lists), FP32 basis and accumulation: cost
 *                      set by the blocks' entries;
 *   HGL_BLOCKS_AUTO    (default) sparse when the blocks' entries, counted once per
 *                      build setup, are at most 1/512 of their dense size (a sparse
 *                      entry costs a row gather, ~400x a dense entry on the GEMM).
 * Both compute the same products (up to the BF16 rounding of the dense route).
 */
#define HGL_BLOCKS_AUTO   0
#define HGL_BLOCKS_DENSE  1
#define HGL_BLOCKS_SPARSE 2
hgl_status hgl_set_block_product(hgl_graph* g, int32_t mode);

/*
 * hgl_tune_block_rsvd -- choose the route of the BF16 block rSVD's products Theta_bb S
 * (Section 3, Algorithm 1) for these blocks by timing both on this graph: the dense
 * route (assembly of the dense BF16 blocks + 2q + 2 tcgen05 products) against the
 * sparse route (2q + 2 products from the incidence lists), each after a warm-up, CUDA
 * events on `stream`.  The faster becomes the graph's hgl_set_block_product setting
 * (HGL_BLOCKS_DENSE or HGL_BLOCKS_SPARSE).  The paper has no counterpart: which route
 * is faster depends on how much of Theta the diagonal blocks hold.
 *   w            device FP64[m] (sets the degree vectors)
 *   block_ptr    host int64[nblocks + 1], 0 .. n;  k, p, q as for hgl_block_rsvd
 *   route        optional host out: the chosen setting
 *   ms_dense, ms_sparse  optional host out: the measured times of one build's products
 * Allocates and frees its work space.  Synchronises `stream`.
 */
hgl_status hgl_tune_block_rsvd(hgl_graph* g, const double* w, const int64_t* block_ptr, int32_t nblocks,
                               int32_t k, int32_t p, int32_t q, int32_t* route, double* ms_dense,
                               double* ms_sparse, void* stream);

/*
 * hgl_block_product -- D_b = Theta_bb S_b for every diagonal tessellation block b, the
 * product that each step of Algorithm 1 (Section 3) applies to the block's basis,
 * computed as the BF16 block rSVD computes it: the tcgen05 grouped GEMM over the dense
 * BF16 blocks (S rounded to BF16, FP32 accumulation in TMEM) or the sparse route from
 * the incidence lists (FP32), as hgl_set_block_product selects.
 *   w          device FP64[m] weights (sets the graph's degree vectors)
 *   block_ptr  host int64[nblocks + 1], 0 = b_0 < ... < b_nblocks = n
 *   l          columns of S and D, 1 .. 96
 *   S          device FP32, n x l row-major (lds >= l), block b's rows are S_b
 *   D          device FP32, n x l row-major (ldd >= l), out
 * Uses the graph's block work space.  Synchronises `stream`; HGL_ERR_TIMEOUT if the
 * tensor-core GEMM gave up a wait.
 */
hgl_status hgl_block_product(const hgl_graph* g, const double* w, const int64_t* block_ptr,
                             int32_t nblocks, int32_t l, const float* S, int64_t lds, float* D,
                             int64_t ldd, void* stream);

/*
 * hgl_schur_inverse -- the nested 2 x 2 Schur-complement inverse of Section 3
 * (Eqs. 12-14) for the principal submatrix of M = (1+lam) I - Theta(w) on the vertex
 * range [row0, row0 + nrows), as a dense matrix.  Split in halves 1 | 2:
 *   M^-1 = [[Z1^-1, -M11^-1 M12 Z2^-1], [-Z2^-1 M21 M11^-1, Z2^-1]],
 *   Z1 = (1+lam) I - (Theta11 + Theta12 M22^-1 Theta21), Z2 likewise;
 * M11^-1 and M22^-1 by the same scheme on the halves (nested tessellation) down to
 * blocks of at most 2 r_min rows; those blocks and the Schur complements Z1, Z2 are
 * inverted by Algorithm 1 (Rayleigh-Ritz form, FP64): with L the positive
 * semidefinite part, ((1+lam) I - L)^-1 ~= I/(1+lam) + Q diag(l/((1+lam)(1+lam-l))) Q^T
 * for the top min(k, size) Ritz pairs from min(k + p, size) columns and q subspace
 * iterations, the test matrix drawn as for hgl_block_rsvd on the submatrix's global
 * rows and `seed`.
 *   dtype      HGL_FP32: the dense products on the tcgen05 tensor cores (TF32 pairs,
 *              three products per pair, FP32 accumulation: about 2^-21 relative per
 *              product); HGL_FP64: on FP64 CUDA cores
 *   Minv       device FP64, nrows x nrows row-major (ldm >= nrows), out
 * Limits: nrows <= 65,536 (the call allocates about 7 nrows^2 doubles of work space),
 * k + p <= 96.  Synchronises `stream`; HGL_ERR_TIMEOUT if a tensor-core wait gave up.
 */
hgl_status hgl_schur_inverse(const hgl_graph* g, const double* w, double lam, int64_t row0,
                             int64_t nrows, int32_t r_min, int32_t k, int32_t p, int32_t q,
                             uint64_t seed, hgl_dtype dtype, double* Minv, int64_t ldm,
                             void* stream);

/* Release a preconditioner (NULL is a no-op). */
void hgl_precond_destroy(hgl_precond* P);

/*
 * hgl_step_precond -- the block-rSVD preconditioner (Section 3, Algorithm 1 on the
 * diagonal blocks, used as in Eq. 15) that the graph's captured adaptive step
 * (HGL_STEP_GRAPH, route HGL_ROUTE_BR) built in its last call, at that call's w before
 * the weight step.  The handle stays owned by the graph: read it (hgl_precond_export,
 * hgl_precond_apply) until the next hgl_adaptive_step call or hgl_graph_destroy, and do
 * not destroy it.  Errors: HGL_ERR_INVALID_ARG (no captured BR step on this graph).
 */
hgl_status hgl_step_precond(const hgl_graph* g, const hgl_precond** out);

/*
 * hgl_precond_export -- copy block b's factors to caller-owned DEVICE FP64 arrays:
 * Q row-major (block size) x k and ev[k] (descending).  kb receives the block's rank
 * (min(k, block size)).  Asynchronous.
 */
hgl_status hgl_precond_export(const hgl_precond* P, int32_t b, double* Q, double* ev,
                              int32_t* kb, void* stream);

/*
 * hgl_precond_apply -- Z = P^-1 R (formula above) for device panels of `dtype`
 * (FP64 or FP32), n x c.  Asynchronous.
 */
hgl_status hgl_precond_apply(const hgl_precond* P, const void* R, int64_t ldr, void* Z,
                             int64_t ldz, int32_t c, hgl_dtype dtype, void* stream);

/*
 * hgl_precond_tensor_cores -- choose how FP32 panels are applied when the factors are
 * FP32 (gemm_dtype BF16) and k <= 64: on = 1 (the default) runs the projection and the
 * expansion of Eq. 15 as TF32 tensor-core products with each operand split into two
 * TF32 numbers (three products per pair, ~2^-21 relative error per product, FP32
 * accumulation) and takes the PCG's r.z from the projection; on = 0 runs them on the
 * FP32 CUDA cores.  Other preconditioners and panel types ignore the switch.  *active
 * (optional, host) returns whether the tensor-core apply is available for P.
 * Applies to later calls on P.
 */
hgl_status hgl_precond_tensor_cores(hgl_precond* P, int32_t on, int32_t* active);

/* ------------------------------------------------------------------------- */
/* Weight update (Section 2, Eqs. 4 and 5)                                   */
/* ------------------------------------------------------------------------- */

#define HGL_GRAD_DV_FROZEN 1   /* differentiate only the explicit W De^-1 factor */

/*
 * hgl_weight_grad -- grad = -d tr(Z^T Theta(w) F) / dw + 2 mu w, at fixed F and Z.
 * With Z = NULL (Z = F) this is grad_w P(w) of Eq. 4.  The derivative includes the
 * dependence of dv on w (Section 2 defines dv through w):
 *   d/dw_e tr(Z^T Theta F) = <sF_e, sZ_e>/de_e
 *        - 1/2 sum_{v in e} (1/dv_v) (<G_v, UZ_v> + <R_v, UF_v>),
 *   G = Dv^-1/2 F, R = Dv^-1/2 Z, sF = H^T G, sZ = H^T R, UX = H diag(w/de) sX.
 *   F, Z       device panels n x c of `dtype` (FP64 or FP32), leading dimension ld
 *   grad       device FP64[m]
 * flags: HGL_GRAD_DV_FROZEN keeps only the first term.  Asynchronous.
 */
hgl_status hgl_weight_grad(const hgl_graph* g, const double* w, const void* F,
                           const void* Z, int64_t ld, int32_t c, hgl_dtype dtype,
                           double mu, int32_t flags, double* grad, void* stream);

/*
 * hgl_project_simplex -- w <- argmin_{u >= 0, 1^T u = 1} ||u - (w - eta grad)||,
 * the constrained steepest-descent step of Eq. 5 read as a Euclidean projection.
 * The threshold tau with sum_e max(v_e - tau, 0) = 1 is found by Michelot's
 * support-shrinking iteration, then w_e = max(v_e - tau, 0).
 *   w          device FP64[m], in/out;  grad device FP64[m] (NULL = zero)
 * Asynchronous.
 */
/*
 * hgl_active_set_step -- the steepest-descent step of Eq. 5 read literally: the
 * constraint 1^T w = 1 is always active and w_e = 0 is active for every weight already
 * at 0; their multipliers make the step vanish on the pinned weights and sum to zero
 * over the free ones, d_e = grad_e - mean over free of grad; w - eta d is clamped at 0
 * (weights that cross 0 join the pinned set) and rescaled to sum 1.  With no free
 * weight, or none left after clamping, w is unchanged.  w device FP64[m] in/out, grad
 * device FP64[m].  Fixed-order reductions (reproducible); allocates its work space
 * stream-ordered.  Asynchronous.
 */
hgl_status hgl_active_set_step(double* w, const double* grad, double eta, int64_t m, void* stream);

hgl_status hgl_project_simplex(double* w, const double* grad, double eta, int64_t m,
                               void* stream);

/*
 * hgl_adjoint_grad -- the part of dL/dw that flows through the ranking solve, for a
 * loss L(F(w), w) with F(w) the solution of M(w) F = lam Y (Eq. 6), by the adjoint
 * method.  Differentiating M F = lam Y gives dF = -M^-1 (dM) F with dM/dw_e =
 * -dTheta/dw_e (Eq. 1, dv(w) included), so for G = dL/dF
 *     grad_e = <G, dF/dw_e> = d/dw_e tr(Z^T Theta(w) F),   Z = M^-1 G,
 * computed by one batched CG solve of M Z = G (M is symmetric, so the "transposed"
 * system has the same operator) followed by the bilinear form of the Eq. 4 gradient.
 * The explicit dependence of L on w (e.g. the mu ||w||^2 term or the Delta in
 * tr(F^T Delta F), see hgl_weight_grad) is not included: add it.  The paper has no
 * counterpart; the forward solve's iterates are not needed (only F).
 *   w          device FP64[m];  lam > 0 (the lam of the forward solve)
 *   F          device FP64 panel n x c: the forward solution
 *   G          device FP64 panel n x c: dL/dF
 *   Z          device FP64 panel n x c, out: M^-1 G (must not alias F or G)
 *   ld         leading dimension shared by F, G and Z
 *   precond    NULL or a preconditioner from hgl_block_rsvd for (w, lam)
 *   opts       solve options for the adjoint CG (tol relative to ||G_j||, dtype:
 *              FP64 or a mixed mode, as in hgl_cg_solve)
 *   grad       device FP64[m], out
 *   stats      optional host out: statistics of the adjoint solve
 * Returns the adjoint solve's status (HGL_ERR_NOT_CONVERGED still writes Z and grad).
 * Synchronises `stream`.
 */
hgl_status hgl_adjoint_grad(hgl_graph* g, const double* w, double lam, const double* F,
                            const double* G, double* Z, int64_t ld, int32_t c,
                            const hgl_precond* precond, const hgl_solve_opts* opts,
                            double* grad, hgl_solve_stats* stats, void* stream);

/*
 * hgl_laplacian_quadratic -- tr(F^T Delta(w) F) with Delta = I - Theta(w) (Eq. 1), the
 * first term of the objective P(w) of Eq. 4 (and of the regularised loss), together
 * with Delta F, whose double is that term's gradient in F.  FP64 throughout: DF by
 * the operator apply with (a, b) = (1, -1), the trace as the deterministic sum over
 * all entries of F * DF (fixed-order partial sums).
 *   w          device FP64[m]
 *   F          device FP64 panel n x c (ldf)
 *   DF         device FP64 panel n x c (lddf), out: Delta F (must not alias F)
 *   value      host out: tr(F^T Delta F)
 * Synchronises `stream`.
 */
hgl_status hgl_laplacian_quadratic(hgl_graph* g, const double* w, const double* F, int64_t ldf,
                                   double* DF, int64_t lddf, int32_t c, double* value, void* stream);

/* ------------------------------------------------------------------------- */
/* Adaptive outer iteration (Section 2: F at fixed w, then w at fixed F)      */
/* ------------------------------------------------------------------------- */

#define HGL_ROUTE_CG 0   /* plain CG solve (CG-ITH-HWEG, Section 4)                     */
#define HGL_ROUTE_BR 1   /* CG preconditioned by the block rSVD (BR-ITH-HWEG)          */
#define HGL_ROUTE_BCG 2  /* block CG with a shared Krylov space over groups of k      */
                         /* columns (hgl_block_cg_solve), FP64, eager steps only       */

#define HGL_STEP_GRAPH      1 /* replay the step as one captured CUDA graph            */
#define HGL_STEP_ACTIVE_SET 2 /* weight step by hgl_active_set_step instead of the     */
                              /* Euclidean projection (hgl_project_simplex)            */

typedef struct {
  double  lam;           /* ranking regulariser (theta of Eq. 3), > 0                     */
  double  mu;            /* weight regulariser (kappa of Eq. 4), >= 0                     */
  double  eta;           /* step size of the projected gradient step                     */
  int32_t route;         /* HGL_ROUTE_CG, HGL_ROUTE_BR or HGL_ROUTE_BCG                  */
  int32_t flags;         /* HGL_STEP_GRAPH                                               */
  hgl_solve_opts solve;  /* inner solve options (warm start from F is always used)       */
  const int64_t* block_ptr; int32_t nblocks;   /* HGL_ROUTE_BR: host block boundaries     */
  int32_t k, p, q;       /* HGL_ROUTE_BR: rank, oversampling, iterations;                 */
                         /* HGL_ROUTE_BCG: k = columns per group (1 .. 32)                */
  uint64_t seed;         /* HGL_ROUTE_BR: Omega seed                                      */
} hgl_step_opts;

typedef struct {
  hgl_solve_stats solve;
  double objective;      /* P(w) = tr(F^T Delta F) + mu ||w||^2 at the solve's w and F    */
  double dw_norm;        /* ||w_new - w_old||_2                                           */
} hgl_step_stats;

/*
 * hgl_adaptive_step -- one outer iteration of the alternation:
 *   1. degrees from w;  [route BR: block rSVD preconditioner at this w]
 *   2. solve M(w) F = lam Y, warm-started from F;
 *   3. grad = grad_w P(w) at that F (hgl_weight_grad with Z = F);
 *   4. w <- projection of w - eta grad onto the simplex.
 *   g          graph;  w device FP64[m] in/out;  Y device FP64 panel (ldy);
 *   F          device FP64 panel (ldf), in: warm start, out: the solve of step 2
 * Synchronises `stream` (statistics).
 */
hgl_status hgl_adaptive_step(hgl_graph* g, double* w, const hgl_step_opts* opts,
                             const double* Y, int64_t ldy, double* F, int64_t ldf,
                             int32_t c, hgl_step_stats* stats, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HGL_H_ */
