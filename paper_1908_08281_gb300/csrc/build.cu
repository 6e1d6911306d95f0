// build.cu -- device construction of the incidence layouts (Section 2: H(v,e) = 1 iff
// v in e; de(e) = sum_v H(v,e)).
//
// Steps: validate the pointer array and compute de; range-check members and count
// the hyperedges of every vertex; sort the members of each hyperedge (segmented
// bitonic sort) and reject repeats; exclusive scan of the counts gives the vertex
// pointers; scatter hyperedge ids into vertex rows; sort every vertex row.  Every
// output is a pure function of the input, so the result is bit-exact and the same
// from run to run.
#include <algorithm>
#include <climits>
#include <new>
#include <vector>

#include "hgl_internal.cuh"

namespace hgl {
namespace {

constexpr unsigned BIT_INVALID = 1u, BIT_EMPTY = 2u, BIT_RANGE = 4u, BIT_DUP = 8u;
constexpr int SORT_SMEM_CAP = 12288;  // int32 elements sorted in shared memory (48 KB)

__global__ void k_check_ptr(const int64_t* __restrict__ ptr, int64_t m, int64_t nnz, int32_t* __restrict__ de,
                            unsigned* __restrict__ bits) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += stride) {
    int64_t a = ptr[e], b = ptr[e + 1];
    if (e == 0 && a != 0) atomicOr(bits, BIT_INVALID);
    if (e == m - 1 && b != nnz) atomicOr(bits, BIT_INVALID);
    if (b < a || a < 0 || b > nnz) {
      atomicOr(bits, BIT_INVALID);
      de[e] = 0;
    } else {
      if (b == a) atomicOr(bits, BIT_EMPTY);
      de[e] = (int32_t)(b - a);
    }
  }
}

__global__ void k_count_members(const int32_t* __restrict__ members, int64_t nnz, int64_t n,
                                 unsigned* __restrict__ cnt, unsigned* __restrict__ bits) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz; i += stride) {
    int32_t v = members[i];
    if (v < 0 || (int64_t)v >= n)
      atomicOr(bits, BIT_RANGE);
    else
      atomicAdd(cnt + v, 1u);
  }
}

// Split segments into short (2..32, one warp each) and long (> 32, one block each).
__global__ void k_classify(const int64_t* __restrict__ ptr, int64_t nseg, int32_t* __restrict__ short_list,
                           int32_t* __restrict__ long_list, unsigned* __restrict__ counts) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg; s += stride) {
    int64_t len = ptr[s + 1] - ptr[s];
    if (len <= 1) continue;
    if (len <= 32)
      short_list[atomicAdd(counts + 0, 1u)] = (int32_t)s;
    else
      long_list[atomicAdd(counts + 1, 1u)] = (int32_t)s;
  }
}

// Bitonic sort of up to 32 keys held one per lane (ascending; INT_MAX pads).
__device__ __forceinline__ int32_t warp_bitonic(int32_t x, int lane) {
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      int32_t y = __shfl_xor_sync(0xffffffffu, x, j);
      bool up = (lane & k) == 0;
      bool low = (lane & j) == 0;
      x = (low == up) ? min(x, y) : max(x, y);
    }
  }
  return x;
}

__global__ void k_sort_short(const int64_t* __restrict__ ptr, int32_t* __restrict__ data,
                             const int32_t* __restrict__ list, const unsigned* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t count = counts[0];
  for (int64_t i = warp; i < count; i += nwarps) {
    int32_t s = list[i];
    int64_t beg = ptr[s];
    int len = (int)(ptr[s + 1] - beg);
    int32_t x = lane < len ? data[beg + lane] : INT_MAX;
    x = warp_bitonic(x, lane);
    if (lane < len) data[beg + lane] = x;
  }
}

// Ascending bitonic sort of a[0..len) in place, by one thread block.  The first
// step of every stage compares mirrored positions, so all compare-exchanges move
// the smaller key to the lower index and positions >= len act as +infinity.
template <class Ptr>
__device__ void block_bitonic(Ptr a, int64_t len) {
  int64_t P = 1;
  while (P < len) P <<= 1;
  const int64_t half = P >> 1;
  for (int64_t k = 2; k <= P; k <<= 1) {
    const int64_t hk = k >> 1;
    for (int64_t p = threadIdx.x; p < half; p += blockDim.x) {
      int64_t start = (p / hk) * k, r = p % hk;
      int64_t i = start + r, j = start + k - 1 - r;
      if (j < len) {
        int32_t x = a[i], y = a[j];
        if (x > y) { a[i] = y; a[j] = x; }
      }
    }
    __syncthreads();
    for (int64_t d = k >> 2; d > 0; d >>= 1) {
      for (int64_t p = threadIdx.x; p < half; p += blockDim.x) {
        int64_t i = (p / d) * 2 * d + (p % d), j = i + d;
        if (j < len) {
          int32_t x = a[i], y = a[j];
          if (x > y) { a[i] = y; a[j] = x; }
        }
      }
      __syncthreads();
    }
  }
}

__global__ void k_sort_long(const int64_t* __restrict__ ptr, int32_t* __restrict__ data,
                            const int32_t* __restrict__ list, const unsigned* __restrict__ counts) {
  __shared__ int32_t sm[SORT_SMEM_CAP];
  const int64_t count = counts[1];
  for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
    int32_t s = list[i];
    int64_t beg = ptr[s];
    int64_t len = ptr[s + 1] - beg;
    if (len <= SORT_SMEM_CAP) {
      for (int64_t q = threadIdx.x; q < len; q += blockDim.x) sm[q] = data[beg + q];
      __syncthreads();
      block_bitonic(sm, len);
      for (int64_t q = threadIdx.x; q < len; q += blockDim.x) data[beg + q] = sm[q];
    } else {
      block_bitonic(data + beg, len);
    }
    __syncthreads();
  }
}

__global__ void k_check_dup(const int64_t* __restrict__ ptr, const int32_t* __restrict__ data, int64_t nseg,
                            unsigned* __restrict__ bits) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg; s += stride)
    for (int64_t i = ptr[s] + 1, end = ptr[s + 1]; i < end; ++i)
      if (data[i] == data[i - 1]) {
        atomicOr(bits, BIT_DUP);
        break;
      }
}

// ---- exclusive scan of unsigned counts into int64 pointers -------------------
constexpr int SCAN_THREADS = 256, SCAN_ITEMS = 8, SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ int64_t block_exclusive_scan(int64_t x, int64_t* total) {
  __shared__ int64_t warp_sums[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sums[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int64_t v = lane < SCAN_THREADS / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane < SCAN_THREADS / 32) warp_sums[lane] = v;
  }
  __syncthreads();
  int64_t warp_off = wid > 0 ? warp_sums[wid - 1] : 0;
  *total = warp_sums[SCAN_THREADS / 32 - 1];
  __syncthreads();
  return warp_off + incl - x;
}

__global__ void k_scan_tiles(const unsigned* __restrict__ in, int64_t n, int64_t* __restrict__ tile_sums) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t acc = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i)
    if (base + i < n) acc += in[base + i];
  int64_t total;
  block_exclusive_scan(acc, &total);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_tile_sums(int64_t* __restrict__ tile_sums, int64_t ntiles) {
  int64_t carry = 0;
  for (int64_t base = 0; base < ntiles; base += SCAN_THREADS) {
    int64_t i = base + threadIdx.x;
    int64_t x = i < ntiles ? tile_sums[i] : 0;
    int64_t total;
    int64_t ex = block_exclusive_scan(x, &total);
    if (i < ntiles) tile_sums[i] = carry + ex;
    carry += total;
  }
}

__global__ void k_scan_apply(const unsigned* __restrict__ in, int64_t n, const int64_t* __restrict__ tile_off,
                             int64_t* __restrict__ out) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t vals[SCAN_ITEMS];
  int64_t acc = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    vals[i] = base + i < n ? in[base + i] : 0;
    acc += vals[i];
  }
  int64_t total;
  int64_t ex = block_exclusive_scan(acc, &total) + tile_off[blockIdx.x];
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    if (base + i < n) out[base + i] = ex;
    ex += vals[i];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) out[n] = ex;
}

// One warp per hyperedge: append e to the row of every member (order fixed later).
__global__ void k_scatter_rows(const int64_t* __restrict__ csc_ptr, const int32_t* __restrict__ csc_idx, int64_t m,
                               const int64_t* __restrict__ csr_ptr, unsigned* __restrict__ cursor,
                               int32_t* __restrict__ csr_idx) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = warp; e < m; e += nwarps)
    for (int64_t i = csc_ptr[e] + lane, end = csc_ptr[e + 1]; i < end; i += 32) {
      int32_t v = csc_idx[i];
      unsigned pos = atomicAdd(cursor + v, 1u);
      csr_idx[csr_ptr[v] + pos] = (int32_t)e;
    }
}

hgl_status segmented_sort(const int64_t* ptr, int32_t* data, int64_t nseg, int32_t* list_a, int32_t* list_b,
                          unsigned* counts, int sms, cudaStream_t st) {
  HGL_CHECK_CUDA(cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned), st));
  hgl::count_launch(); k_classify<<<sms * 8, 256, 0, st>>>(ptr, nseg, list_a, list_b, counts);
  hgl::count_launch(); k_sort_short<<<sms * 8, 256, 0, st>>>(ptr, data, list_a, counts);
  hgl::count_launch(); k_sort_long<<<sms * 4, 256, 0, st>>>(ptr, data, list_b, counts);
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

hgl_status exclusive_scan(const unsigned* in, int64_t n, int64_t* out, int64_t* tile_sums, cudaStream_t st) {
  int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (ntiles == 0) ntiles = 1;
  hgl::count_launch(); k_scan_tiles<<<(unsigned)ntiles, SCAN_THREADS, 0, st>>>(in, n, tile_sums);
  hgl::count_launch(); k_scan_tile_sums<<<1, SCAN_THREADS, 0, st>>>(tile_sums, ntiles);
  hgl::count_launch(); k_scan_apply<<<(unsigned)ntiles, SCAN_THREADS, 0, st>>>(in, n, tile_sums, out);
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

hgl_status read_bits(const unsigned* dbits, cudaStream_t st, unsigned* hbits) {
  HGL_CHECK_CUDA(cudaMemcpyAsync(hbits, dbits, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  return HGL_OK;
}

hgl_status bits_status(unsigned b) {
  if (b & BIT_INVALID)
    return record_error(HGL_ERR_INVALID_ARG, "edge_ptr must start at 0, not decrease and end at nnz");
  if (b & BIT_EMPTY) return record_error(HGL_ERR_EMPTY_EDGE, "a hyperedge has no members");
  if (b & BIT_RANGE) return record_error(HGL_ERR_INDEX_RANGE, "a member id lies outside [0, n)");
  if (b & BIT_DUP) return record_error(HGL_ERR_DUPLICATE_MEMBER, "a vertex appears twice in one hyperedge");
  return HGL_OK;
}

// Split of the operator (see hgl_graph): per vertex, the number of its large hyperedges
// and of its entries over small ones (members other than itself).
__global__ void k_split_count(int64_t n, const int64_t* __restrict__ csr_ptr, const int32_t* __restrict__ csr_idx,
                              const int32_t* __restrict__ de, unsigned* __restrict__ lcnt,
                              unsigned* __restrict__ scnt) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    unsigned a = 0, b = 0;
    for (int64_t i = csr_ptr[v], end = csr_ptr[v + 1]; i < end; ++i) {
      const int d = de[csr_idx[i]];
      if (d > SMALL_EDGE) ++a; else b += (unsigned)(d - 1);
    }
    lcnt[v] = a;
    scnt[v] = b;
  }
}

__global__ void k_edge_slots(int64_t m_large, const int32_t* __restrict__ order, int32_t* __restrict__ slot) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m_large; q += (int64_t)gridDim.x * blockDim.x)
    slot[order[q]] = (int32_t)q;
}

// Per vertex, in its hyperedge order: the slots of the large hyperedges, and for each
// small hyperedge its other members (member order) with the hyperedge.
__global__ void k_split_fill(int64_t n, const int64_t* __restrict__ csr_ptr, const int32_t* __restrict__ csr_idx,
                             const int64_t* __restrict__ csc_ptr, const int32_t* __restrict__ csc_idx,
                             const int32_t* __restrict__ de, const int32_t* __restrict__ slot,
                             const int64_t* __restrict__ lptr, int32_t* __restrict__ lidx,
                             const int64_t* __restrict__ sptr, int32_t* __restrict__ sv, int32_t* __restrict__ se) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int64_t lp = lptr[v], sp = sptr[v];
    for (int64_t i = csr_ptr[v], end = csr_ptr[v + 1]; i < end; ++i) {
      const int32_t e = csr_idx[i];
      if (de[e] > SMALL_EDGE) {
        lidx[lp++] = slot[e];
      } else {
        for (int64_t j = csc_ptr[e]; j < csc_ptr[e + 1]; ++j) {
          const int32_t u = csc_idx[j];
          if (u != v) {
            sv[sp] = u;
            se[sp] = e;
            ++sp;
          }
        }
      }
    }
  }
}

// Hyperedges in decreasing size order (stable counting sort on the host; one-time).
// The gather passes give each hyperedge above HEAVY_ROW members a whole thread block
// and schedule the rest longest first, so no long row finishes last.
hgl_status order_edges(hgl_graph* g, cudaStream_t st) {
  const int64_t m = g->m;
  std::vector<int64_t> ptr(m + 1);
  HGL_CHECK_CUDA(cudaMemcpyAsync(ptr.data(), g->csc_ptr, sizeof(int64_t) * (m + 1), cudaMemcpyDeviceToHost, st));
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  int64_t maxs = 0;
  for (int64_t e = 0; e < m; ++e) maxs = std::max(maxs, ptr[e + 1] - ptr[e]);
  std::vector<int64_t> count(maxs + 2, 0);
  for (int64_t e = 0; e < m; ++e) count[maxs - (ptr[e + 1] - ptr[e])]++;
  int64_t acc = 0;
  for (auto& x : count) {
    const int64_t c = x;
    x = acc;
    acc += c;
  }
  std::vector<int32_t> order(m);
  g->nheavy = 0;
  g->m_large = 0;
  for (int64_t e = 0; e < m; ++e) {
    const int64_t sz = ptr[e + 1] - ptr[e];
    order[count[maxs - sz]++] = (int32_t)e;
    if (sz > HEAVY_ROW) g->nheavy++;
    if (sz > SMALL_EDGE) g->m_large++;
  }
  HGL_CHECK_CUDA(cudaMalloc(&g->edge_order, sizeof(int32_t) * m));
  HGL_CHECK_CUDA(cudaMemcpyAsync(g->edge_order, order.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  return HGL_OK;
}

struct TempMem {
  void* p = nullptr;
  ~TempMem() {
    if (p) cudaFree(p);
  }
};

hgl_status build(int64_t n, int64_t m, const int64_t* edge_ptr, const int32_t* members, int64_t nnz,
                 cudaStream_t st, hgl_graph* g) {
  g->n = n;
  g->m = m;
  g->nnz = nnz;
  HGL_CHECK_CUDA(cudaGetDevice(&g->device));
  g->num_sms = device_sm_count();
  const int sms = g->num_sms;
  HGL_CHECK_CUDA(cudaMalloc(&g->csc_ptr, sizeof(int64_t) * (m + 1)));
  HGL_CHECK_CUDA(cudaMalloc(&g->csc_idx, sizeof(int32_t) * (nnz > 0 ? nnz : 1)));
  HGL_CHECK_CUDA(cudaMalloc(&g->csr_ptr, sizeof(int64_t) * (n + 1)));
  HGL_CHECK_CUDA(cudaMalloc(&g->csr_idx, sizeof(int32_t) * (nnz > 0 ? nnz : 1)));
  HGL_CHECK_CUDA(cudaMalloc(&g->de, sizeof(int32_t) * m));
  HGL_CHECK_CUDA(cudaMalloc(&g->dv, sizeof(double) * n));
  HGL_CHECK_CUDA(cudaMalloc(&g->s, sizeof(double) * n));
  HGL_CHECK_CUDA(cudaMalloc(&g->t, sizeof(double) * m));
  HGL_CHECK_CUDA(cudaMalloc(&g->s32, sizeof(float) * n));
  HGL_CHECK_CUDA(cudaMalloc(&g->t32, sizeof(float) * m));

  // temporaries: bits | counts[2] | cnt[n] | cursor[n] | lists[max(n,m)] x2 | tile sums
  const int64_t nseg_max = n > m ? n : m;
  const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE + 1;
  size_t bytes = 64 + sizeof(unsigned) * (size_t)(2 * n) + sizeof(int32_t) * (size_t)(2 * nseg_max) +
                 sizeof(int64_t) * (size_t)ntiles + 64;
  TempMem tmp;
  HGL_CHECK_CUDA(cudaMalloc(&tmp.p, bytes));
  char* base = static_cast<char*>(tmp.p);
  unsigned* bits = reinterpret_cast<unsigned*>(base);
  unsigned* counts = bits + 4;
  unsigned* cnt = reinterpret_cast<unsigned*>(base + 64);
  unsigned* cursor = cnt + n;
  int32_t* list_a = reinterpret_cast<int32_t*>(cursor + n);
  int32_t* list_b = list_a + nseg_max;
  int64_t* tile_sums = reinterpret_cast<int64_t*>(
      (reinterpret_cast<uintptr_t>(list_b + nseg_max) + 15) & ~static_cast<uintptr_t>(15));
  HGL_CHECK_CUDA(cudaMemsetAsync(base, 0, 64 + sizeof(unsigned) * (size_t)(2 * n), st));

  HGL_CHECK_CUDA(cudaMemcpyAsync(g->csc_ptr, edge_ptr, sizeof(int64_t) * (m + 1), cudaMemcpyDefault, st));
  if (nnz > 0)
    HGL_CHECK_CUDA(cudaMemcpyAsync(g->csc_idx, members, sizeof(int32_t) * nnz, cudaMemcpyDefault, st));

  unsigned hbits = 0;
  hgl::count_launch(); k_check_ptr<<<sms * 4, 256, 0, st>>>(g->csc_ptr, m, nnz, g->de, bits);
  HGL_CHECK_CUDA(cudaGetLastError());
  HGL_TRY(read_bits(bits, st, &hbits));
  HGL_TRY(bits_status(hbits));

  hgl::count_launch(); k_count_members<<<sms * 8, 256, 0, st>>>(g->csc_idx, nnz, n, cnt, bits);
  HGL_CHECK_CUDA(cudaGetLastError());
  HGL_TRY(read_bits(bits, st, &hbits));
  HGL_TRY(bits_status(hbits));

  HGL_TRY(segmented_sort(g->csc_ptr, g->csc_idx, m, list_a, list_b, counts, sms, st));
  hgl::count_launch(); k_check_dup<<<sms * 8, 256, 0, st>>>(g->csc_ptr, g->csc_idx, m, bits);
  HGL_CHECK_CUDA(cudaGetLastError());
  HGL_TRY(read_bits(bits, st, &hbits));
  HGL_TRY(bits_status(hbits));

  HGL_TRY(exclusive_scan(cnt, n, g->csr_ptr, tile_sums, st));
  hgl::count_launch(); k_scatter_rows<<<sms * 8, 256, 0, st>>>(g->csc_ptr, g->csc_idx, m, g->csr_ptr, cursor, g->csr_idx);
  HGL_CHECK_CUDA(cudaGetLastError());
  HGL_TRY(segmented_sort(g->csr_ptr, g->csr_idx, n, list_a, list_b, counts, sms, st));
  HGL_TRY(order_edges(g, st));

  // the operator's split into large hyperedges (through the intermediate, by slot) and
  // small ones (vertex-to-vertex entries); cnt and cursor are free again, list_a holds
  // the slots
  HGL_CHECK_CUDA(cudaMalloc(&g->lcsr_ptr, sizeof(int64_t) * (n + 1)));
  HGL_CHECK_CUDA(cudaMalloc(&g->scsr_ptr, sizeof(int64_t) * (n + 1)));
  HGL_CHECK_CUDA(cudaMalloc(&g->sdiag, sizeof(double) * n));
  HGL_CHECK_CUDA(cudaMalloc(&g->sdiag32, sizeof(float) * n));
  hgl::count_launch(); k_split_count<<<sms * 8, 256, 0, st>>>(n, g->csr_ptr, g->csr_idx, g->de, cnt, cursor);
  HGL_CHECK_CUDA(cudaGetLastError());
  HGL_TRY(exclusive_scan(cnt, n, g->lcsr_ptr, tile_sums, st));
  HGL_TRY(exclusive_scan(cursor, n, g->scsr_ptr, tile_sums, st));
  int64_t nl = 0, ns = 0;
  HGL_CHECK_CUDA(cudaMemcpyAsync(&nl, g->lcsr_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  HGL_CHECK_CUDA(cudaMemcpyAsync(&ns, g->scsr_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  HGL_CHECK_CUDA(cudaMalloc(&g->lcsr_idx, sizeof(int32_t) * (size_t)(nl > 0 ? nl : 1)));
  HGL_CHECK_CUDA(cudaMalloc(&g->scsr_v, sizeof(int32_t) * (size_t)(ns > 0 ? ns : 1)));
  HGL_CHECK_CUDA(cudaMalloc(&g->scsr_e, sizeof(int32_t) * (size_t)(ns > 0 ? ns : 1)));
  HGL_CHECK_CUDA(cudaMalloc(&g->scoef, sizeof(double) * (size_t)(ns > 0 ? ns : 1)));
  HGL_CHECK_CUDA(cudaMalloc(&g->scoef32, sizeof(float) * (size_t)(ns > 0 ? ns : 1)));
  if (g->m_large > 0) {
    hgl::count_launch(); k_edge_slots<<<sms * 8, 256, 0, st>>>(g->m_large, g->edge_order, list_a);
    HGL_CHECK_CUDA(cudaGetLastError());
  }
  hgl::count_launch();
  k_split_fill<<<sms * 8, 256, 0, st>>>(n, g->csr_ptr, g->csr_idx, g->csc_ptr, g->csc_idx, g->de, list_a, g->lcsr_ptr,
                                        g->lcsr_idx, g->scsr_ptr, g->scsr_v, g->scsr_e);
  HGL_CHECK_CUDA(cudaGetLastError());
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  return HGL_OK;
}

}  // namespace
}  // namespace hgl

extern "C" hgl_status hgl_build_incidence(int64_t n, int64_t m, const int64_t* edge_ptr, const int32_t* members,
                                          int64_t nnz, void* stream, hgl_graph** out) {
  if (!out) return hgl::record_error(HGL_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || m < 1 || n >= INT32_MAX || m >= INT32_MAX || nnz < 0 || nnz >= INT32_MAX)
    return hgl::record_error(HGL_ERR_INVALID_ARG, "sizes must satisfy 1 <= n, m < 2^31 and 0 <= nnz < 2^31");
  if (!edge_ptr || (nnz > 0 && !members)) return hgl::record_error(HGL_ERR_INVALID_ARG, "NULL input array");
  hgl_graph* g = new (std::nothrow) hgl_graph();
  if (!g) return hgl::record_error(HGL_ERR_OOM, "host allocation failed");
  hgl_status s = hgl::build(n, m, edge_ptr, members, nnz, hgl::as_stream(stream), g);
  if (s != HGL_OK) {
    cudaStreamSynchronize(hgl::as_stream(stream));
    hgl_graph_destroy(g);
    return s;
  }
  *out = g;
  return HGL_OK;
}
