// Sparse-structure primitives used at set-up: scans, incidence lists, transpose and a
// deterministic sparse matrix product (Galerkin products of the AMG set-up).
#include <cstdarg>

#include "ch_internal.cuh"

namespace ch {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

const char* last_error() { return g_err.c_str(); }

// ---------------------------------------------------------------- exclusive scan (int64)
constexpr int SCAN_IT = 4;
constexpr int SCAN_TILE = TPB * SCAN_IT;

__global__ void k_scan_tile(int64_t* d, int64_t n, int64_t* tile_sum) {
  __shared__ int64_t warp_tot[TPB / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_IT;
  int64_t v[SCAN_IT];
  int64_t tsum = 0;
#pragma unroll
  for (int k = 0; k < SCAN_IT; ++k) {
    const int64_t i = base + k;
    v[k] = i < n ? d[i] : 0;
    tsum += v[k];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t x = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t t = lane < TPB / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < TPB / 32) warp_tot[lane] = t;
  }
  __syncthreads();
  int64_t excl = x - tsum + (w > 0 ? warp_tot[w - 1] : 0);
#pragma unroll
  for (int k = 0; k < SCAN_IT; ++k) {
    const int64_t i = base + k;
    if (i < n) d[i] = excl;
    excl += v[k];
  }
  if (threadIdx.x == TPB - 1) tile_sum[blockIdx.x] = excl;
}

__global__ void k_scan_add(int64_t* d, int64_t n, const int64_t* tile_off) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] += tile_off[i / SCAN_TILE];
}

static ch_status scan_rec(int64_t* d, int64_t n, cudaStream_t st, Alloc& tmp) {
  const int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  int64_t* ts = nullptr;
  CH_TRY(tmp.get(&ts, nt));
  k_scan_tile<<<(unsigned)nt, TPB, 0, st>>>(d, n, ts);
  CH_LAUNCHED();
  if (nt > 1) {
    CH_TRY(scan_rec(ts, nt, st, tmp));
    k_scan_add<<<blocks_for(n), TPB, 0, st>>>(d, n, ts);
    CH_LAUNCHED();
  }
  return CH_OK;
}

ch_status scan_i64(int64_t* d, int64_t n, int64_t* total, cudaStream_t st, Alloc& tmp) {
  if (n <= 0) {
    if (total) *total = 0;
    return CH_OK;
  }
  int64_t last = 0, lastx = 0;
  CH_CUDA(cudaMemcpyAsync(&last, d + n - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CH_TRY(scan_rec(d, n, st, tmp));
  CH_CUDA(cudaMemcpyAsync(&lastx, d + n - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CH_CUDA(cudaStreamSynchronize(st));
  if (total) *total = last + lastx;
  return CH_OK;
}

__global__ void k_i32_to_i64(const int* a, int64_t* b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
  if (i == n) b[i] = 0;
}
__global__ void k_i64_to_i32(const int64_t* a, int* b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (int)a[i];
}

ch_status scan_i32_to_rowptr(const int* counts, int* rowptr, int n, int64_t* total, cudaStream_t st,
                             Alloc& tmp) {
  int64_t* t = nullptr;
  CH_TRY(tmp.get(&t, (size_t)n + 1));
  k_i32_to_i64<<<blocks_for(n + 1), TPB, 0, st>>>(counts, t, n);
  CH_LAUNCHED();
  int64_t tot = 0;
  CH_TRY(scan_i64(t, n + 1, &tot, st, tmp));
  if (tot > 2147483647LL) {
    set_error("sparse structure with %lld entries exceeds int32 indexing", (long long)tot);
    return CH_ERR_INTERNAL;
  }
  k_i64_to_i32<<<blocks_for(n + 1), TPB, 0, st>>>(t, rowptr, n + 1);
  CH_LAUNCHED();
  if (total) *total = tot;
  return CH_OK;
}

// ---------------------------------------------------------------- incidence lists
__global__ void k_count_keys(const int* items, int64_t nent, int* cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nent) atomicAdd(&cnt[items[i]], 1);
}
__global__ void k_fill_keys(const int* items, int64_t nent, int k, const int* ptr, int* cur,
                            int* list) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nent) {
    const int key = items[i];
    const int slot = atomicAdd(&cur[key], 1);
    list[ptr[key] + slot] = (int)(i / k);
  }
}
// insertion sort of each list (lists are short: node -> incident simplices)
__global__ void k_sort_lists(const int* ptr, int* list, int nkeys) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nkeys) return;
  const int b = ptr[r], e = ptr[r + 1];
  for (int i = b + 1; i < e; ++i) {
    const int v = list[i];
    int j = i - 1;
    while (j >= b && list[j] > v) {
      list[j + 1] = list[j];
      --j;
    }
    list[j + 1] = v;
  }
}

ch_status build_incidence(const int* items, int nitems, int k, int nkeys, int** ptr, int** list,
                          cudaStream_t st, Alloc& mem) {
  const int64_t nent = (int64_t)nitems * k;
  Alloc tmp;
  int* cnt = nullptr;
  CH_TRY(tmp.get(&cnt, (size_t)nkeys));
  CH_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * nkeys, st));
  if (nent > 0) {
    k_count_keys<<<blocks_for(nent), TPB, 0, st>>>(items, nent, cnt);
    CH_LAUNCHED();
  }
  CH_TRY(mem.get(ptr, (size_t)nkeys + 1));
  int64_t tot = 0;
  CH_TRY(scan_i32_to_rowptr(cnt, *ptr, nkeys, &tot, st, tmp));
  CH_TRY(mem.get(list, (size_t)tot));
  CH_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * nkeys, st));
  if (nent > 0) {
    k_fill_keys<<<blocks_for(nent), TPB, 0, st>>>(items, nent, k, *ptr, cnt, *list);
    CH_LAUNCHED();
  }
  k_sort_lists<<<blocks_for(nkeys), TPB, 0, st>>>(*ptr, *list, nkeys);
  CH_LAUNCHED();
  CH_CUDA(cudaStreamSynchronize(st));  // tmp is released on return
  return CH_OK;
}

// ---------------------------------------------------------------- transpose
__global__ void k_col_count(const int* col, int64_t nnz, int* cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nnz) atomicAdd(&cnt[col[i]], 1);
}
__global__ void k_transpose_fill(Csr<double> A, const int* bptr, int* cur, int* bcol, double* bval) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= A.nrows) return;
  for (int p = A.rowptr[r]; p < A.rowptr[r + 1]; ++p) {
    const int c = A.col[p];
    const int q = bptr[c] + atomicAdd(&cur[c], 1);
    bcol[q] = r;
    bval[q] = A.val[p];
  }
}
__global__ void k_sort_rows(const int* ptr, int* col, double* val, int n) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int b = ptr[r], e = ptr[r + 1];
  for (int i = b + 1; i < e; ++i) {
    const int c = col[i];
    const double v = val[i];
    int j = i - 1;
    while (j >= b && col[j] > c) {
      col[j + 1] = col[j];
      val[j + 1] = val[j];
      --j;
    }
    col[j + 1] = c;
    val[j + 1] = v;
  }
}

ch_status transpose(const Csr<double>& A, Csr<double>* B, cudaStream_t st, Alloc& mem) {
  Alloc tmp;
  int* cnt = nullptr;
  CH_TRY(tmp.get(&cnt, (size_t)A.ncols));
  CH_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * A.ncols, st));
  if (A.nnz > 0) {
    k_col_count<<<blocks_for(A.nnz), TPB, 0, st>>>(A.col, A.nnz, cnt);
    CH_LAUNCHED();
  }
  B->nrows = A.ncols;
  B->ncols = A.nrows;
  CH_TRY(mem.get(&B->rowptr, (size_t)B->nrows + 1));
  int64_t tot = 0;
  CH_TRY(scan_i32_to_rowptr(cnt, B->rowptr, B->nrows, &tot, st, tmp));
  B->nnz = tot;
  CH_TRY(mem.get(&B->col, (size_t)tot));
  CH_TRY(mem.get(&B->val, (size_t)tot));
  CH_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * A.ncols, st));
  k_transpose_fill<<<blocks_for(A.nrows), TPB, 0, st>>>(A, B->rowptr, cnt, B->col, B->val);
  CH_LAUNCHED();
  k_sort_rows<<<blocks_for(B->nrows), TPB, 0, st>>>(B->rowptr, B->col, B->val, B->nrows);
  CH_LAUNCHED();
  CH_CUDA(cudaStreamSynchronize(st));
  return CH_OK;
}

// ---------------------------------------------------------------- C = A * B
// Row i of C is the k-way merge of the (sorted) rows B_k, k in row i of A, scaled by a_ik.
// One thread per row keeps a binary min-heap of (column, run) keys in a scratch array laid
// out like A's entries, so the merge has no size limit; ties pop in run order, which fixes
// the order of every floating-point sum (the product is bitwise reproducible).
__device__ __forceinline__ uint64_t mkey(int col, int run) {
  return ((uint64_t)(uint32_t)col << 32) | (uint32_t)run;
}

__device__ void heap_down(uint64_t* h, int n, int i) {
  for (;;) {
    int l = 2 * i + 1, m = i;
    if (l < n && h[l] < h[m]) m = l;
    if (l + 1 < n && h[l + 1] < h[m]) m = l + 1;
    if (m == i) return;
    const uint64_t t = h[i];
    h[i] = h[m];
    h[m] = t;
    i = m;
  }
}

template <bool FILL>
__global__ void k_spgemm_row(Csr<double> A, Csr<double> B, uint64_t* heap, int* cur, int* cnt,
                             const int* cptr, int* ccol, double* cval) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nrows) return;
  const int a0 = A.rowptr[i], a1 = A.rowptr[i + 1];
  uint64_t* h = heap + a0;
  int* cu = cur + a0;
  int n = 0;
  for (int r = 0; r < a1 - a0; ++r) {
    const int k = A.col[a0 + r];
    const int p = B.rowptr[k];
    cu[r] = p;
    if (p < B.rowptr[k + 1]) h[n++] = mkey(B.col[p], r);
  }
  for (int j = n / 2 - 1; j >= 0; --j) heap_down(h, n, j);
  int out = FILL ? cptr[i] : 0;
  int count = 0, last = -1;
  double acc = 0.0;
  while (n > 0) {
    const uint64_t top = h[0];
    const int c = (int)(top >> 32), r = (int)(top & 0xffffffffu);
    const int p = cu[r];
    if (c != last) {
      if (FILL && last >= 0) {
        ccol[out] = last;
        cval[out] = acc;
        ++out;
      }
      last = c;
      acc = 0.0;
      ++count;
    }
    if (FILL) acc = fma(A.val[a0 + r], B.val[p], acc);
    const int k = A.col[a0 + r];
    const int pn = p + 1;
    cu[r] = pn;
    if (pn < B.rowptr[k + 1]) {
      h[0] = mkey(B.col[pn], r);
    } else {
      h[0] = h[--n];
    }
    heap_down(h, n, 0);
  }
  if (FILL && last >= 0) {
    ccol[out] = last;
    cval[out] = acc;
  }
  if (!FILL) cnt[i] = count;
}

ch_status spgemm(const Csr<double>& A, const Csr<double>& B, Csr<double>* C, cudaStream_t st,
                 Alloc& mem) {
  if (A.ncols != B.nrows) {
    set_error("spgemm: inner sizes differ (%d vs %d)", A.ncols, B.nrows);
    return CH_ERR_INTERNAL;
  }
  Alloc tmp;
  uint64_t* heap = nullptr;
  int *cur = nullptr, *cnt = nullptr;
  CH_TRY(tmp.get(&heap, (size_t)A.nnz));
  CH_TRY(tmp.get(&cur, (size_t)A.nnz));
  CH_TRY(tmp.get(&cnt, (size_t)A.nrows));
  k_spgemm_row<false><<<blocks_for(A.nrows, 128), 128, 0, st>>>(A, B, heap, cur, cnt, nullptr,
                                                                 nullptr, nullptr);
  CH_LAUNCHED();
  C->nrows = A.nrows;
  C->ncols = B.ncols;
  CH_TRY(mem.get(&C->rowptr, (size_t)C->nrows + 1));
  int64_t tot = 0;
  CH_TRY(scan_i32_to_rowptr(cnt, C->rowptr, C->nrows, &tot, st, tmp));
  C->nnz = tot;
  CH_TRY(mem.get(&C->col, (size_t)tot));
  CH_TRY(mem.get(&C->val, (size_t)tot));
  k_spgemm_row<true><<<blocks_for(A.nrows, 128), 128, 0, st>>>(A, B, heap, cur, cnt, C->rowptr,
                                                                C->col, C->val);
  CH_LAUNCHED();
  CH_CUDA(cudaStreamSynchronize(st));
  return CH_OK;
}

}  // namespace ch
