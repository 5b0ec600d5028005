// Algebraic multigrid for the inner solves of Algorithm 1 (M~ ~ M and H = aK + sqrt(c)M).
//
// The paper uses Ruge-Stueben AMG from a CPU library (Section 4).  Here the hierarchy is
// built on the device by smoothed aggregation (Vanek, Mandel, Brezina 1996) with MIS(2)
// aggregates found by the parallel maximal-independent-set method of Bell, Dalton and
// Olson (2012):
//   strength  |a_ij| >= theta sqrt(a_ii a_jj), plus each row's strongest entry, symmetrised;
//   MIS(2)    random-priority independent set at graph distance 2, roots become aggregates;
//   P         (I - omega D^-1 A) T with T the aggregate indicator, omega = 4/(3 rho),
//             rho = min(Gershgorin bound, 1.05 x power-iteration estimate) of lambda_max(D^-1 A);
//   A_c       = P^T A P (deterministic sparse products), down to <= coarse_max rows, whose
//             dense inverse is formed on the device.
// Smoothing is Chebyshev on D^-1 A over [cheb_lower, 1] * 1.1 rho, with the same rho.  Every set-up sum has a fixed
// order, so the hierarchy is bitwise reproducible.  V-cycles run in FP64 or FP32 on two
// right-hand sides at once (the two species share M and H).
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <type_traits>

#include "ch_internal.cuh"

namespace ch {

template <typename T> struct V2T;
template <> struct V2T<double> { using t = double2; };
template <> struct V2T<float> { using t = float2; };

// Fine-level operator of a uniform mesh as diagonals: row i's neighbours sit at i + lat_off(d),
// the lattice directions a + b W + c WH (W, WH: the row's run's strides), ascending in d for any
// W, H >= 2, i.e. in CSR column order; val[d * n + i] is zero where row i has no such neighbour
// (the clamped column index is then read but multiplied by zero).
template <typename T>
struct Dia {
  int nd = 0;                      // 7 (2D) or 15 (3D); 0: not structured, use the CSR form
  int W = 0, WH = 0;               // strides of a single-run mesh
  const int* node_run = nullptr;   // several runs: run of each row ...
  const int2* run_wh = nullptr;    // ... and (W, WH) of each run
  T* val = nullptr;
};

// direction d of the 2D (7: uniform triangles) or 3D (15: Kuhn tetrahedra) lattice stencil
__host__ __device__ __forceinline__ int lat_off(int nd, int d, int W, int WH) {
  constexpr int a2[7] = {-1, 0, -1, 0, 1, 0, 1}, b2[7] = {-1, -1, 0, 0, 0, 1, 1};
  constexpr int a3[15] = {-1, 0, -1, 0, -1, 0, -1, 0, 1, 0, 1, 0, 1, 0, 1};
  constexpr int b3[15] = {-1, -1, 0, 0, -1, -1, 0, 0, 0, 1, 1, 0, 0, 1, 1};
  constexpr int c3[15] = {-1, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1};
  return nd == 7 ? a2[d] + b2[d] * W : a3[d] + b3[d] * W + c3[d] * WH;
}

template <typename T>
struct LevelT {
  Csr<T> A, P, R;
  Dia<T> dia;                          // level 0 of a structured mesh
  int tprA = 1, tprP = 1, tprR = 1;  // lanes per row of the SpMV-type kernels (autotuned)
  bool pdl = false;                  // launch the V-cycle kernels as programmatic dependents
  T* dinv = nullptr;
  typename V2T<T>::t *x = nullptr, *x2 = nullptr, *d = nullptr, *r = nullptr, *b = nullptr;
};

struct Hierarchy {
  int precision = 0;
  int nlev = 0;
  std::vector<Csr<double>> A, P, R;  // FP64 set-up results
  std::vector<double*> dinv;
  std::vector<double> rho;            // per level: min(Gershgorin bound, 1.05 x power estimate) of
                                      // lambda_max(D^-1 A); Chebyshev interval [lower, 1] x 1.1 rho
  std::vector<LevelT<double>> Ld;     // working copies (precision 0)
  std::vector<LevelT<float>> Lf;      // working copies (precision 1)
  int nc = 0;                         // coarsest size
  double* cinv = nullptr;             // nc x nc dense inverse (FP64)
  float* cinvf = nullptr;
  int cheb_degree = 2;
  int cheb_degree_coarse = 2;         // on the levels below the finest
  double cheb_lower = 0.3;
  int autotune = 1;
  bool pdl = true;
  Alloc mem;
};

// ---------------------------------------------------------------- set-up kernels
__global__ void k_diag_gersh(Csr<double> A, double* dinv, double* rowbound) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nrows) return;
  double d = 0.0, s = 0.0;
  for (int q = A.rowptr[i]; q < A.rowptr[i + 1]; ++q) {
    if (A.col[q] == i) d = A.val[q];
    s += fabs(A.val[q]);
  }
  dinv[i] = 1.0 / d;
  rowbound[i] = s / fabs(d);
}

__global__ void k_max_reduce(const double* v, int n, double* out) {
  __shared__ double sm[TPB];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, v[i]);
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}

__global__ void k_strength(Csr<double> A, const double* dinv, double theta, uint8_t* s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nrows) return;
  const double di = fabs(1.0 / dinv[i]);
  double mx = 0.0;
  for (int q = A.rowptr[i]; q < A.rowptr[i + 1]; ++q) {
    const int j = A.col[q];
    if (j == i) continue;
    mx = fmax(mx, fabs(A.val[q]) / sqrt(di * fabs(1.0 / dinv[j])));
  }
  for (int q = A.rowptr[i]; q < A.rowptr[i + 1]; ++q) {
    const int j = A.col[q];
    uint8_t st = 0;
    if (j != i) {
      const double nrm = fabs(A.val[q]) / sqrt(di * fabs(1.0 / dinv[j]));
      st = (nrm >= theta || (mx > 0.0 && nrm >= mx)) ? 1 : 0;
    }
    s[q] = st;
  }
}

__device__ __forceinline__ int find_in_row(const int* col, int b, int e, int c) {
  while (b < e) {
    const int m = (b + e) >> 1;
    if (col[m] < c) b = m + 1;
    else e = m;
  }
  return b;
}

// s2_ij = s_ij or s_ji (A has a symmetric pattern)
__global__ void k_strength_sym(Csr<double> A, const uint8_t* s, uint8_t* s2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nrows) return;
  for (int q = A.rowptr[i]; q < A.rowptr[i + 1]; ++q) {
    const int j = A.col[q];
    uint8_t v = s[q];
    if (!v && j != i) {
      const int p = find_in_row(A.col, A.rowptr[j], A.rowptr[j + 1], i);
      if (p < A.rowptr[j + 1] && A.col[p] == i) v = s[p];
    }
    s2[q] = v;
  }
}

__device__ __forceinline__ uint32_t hash32(uint32_t x) {  // integer hash (avalanche mixer)
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

// key = state (2 bits) | hash (32 bits) | index (30 bits); state 2 = in, 1 = undecided, 0 = out
__device__ __forceinline__ uint64_t mis_key(int state, int i) {
  return ((uint64_t)state << 62) | ((uint64_t)hash32((uint32_t)i) << 30) | (uint64_t)i;
}

__global__ void k_mis_keys(int n, const int8_t* state, uint64_t* key) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) key[i] = mis_key(state[i], i);
}

__global__ void k_strong_max(Csr<double> A, const uint8_t* s, const uint64_t* in, uint64_t* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nrows) return;
  uint64_t m = in[i];
  for (int q = A.rowptr[i]; q < A.rowptr[i + 1]; ++q)
    if (s[q]) {
      const uint64_t v = in[A.col[q]];
      m = v > m ? v : m;
    }
  out[i] = m;
}

__global__ void k_mis_update(int n, const uint64_t* key, const uint64_t* m2, int8_t* state,
                             int* undecided) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || state[i] != 1) return;
  if (m2[i] == key[i]) state[i] = 2;
  else if ((m2[i] >> 62) == 2) state[i] = 0;
  else atomicAdd(undecided, 1);
}

__global__ void k_roots(int n, const int8_t* state, int* isroot) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) isroot[i] = state[i] == 2 ? 1 : 0;
}

// pass 1: roots own aggregate id (scan of isroot); other nodes join the strongest-key
// neighbouring root.  pass >= 2: unassigned nodes join the aggregate of the max-key
// assigned neighbour (reading the previous pass only).
__global__ void k_agg_pass(Csr<double> A, const uint8_t* s, const int* isroot, const int* rootid,
                           const int* agg_in, int* agg_out, int first, int* unassigned) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nrows) return;
  if (first) {
    if (isroot[i]) {
      agg_out[i] = rootid[i];
      return;
    }
  } else if (agg_in[i] >= 0) {
    agg_out[i] = agg_in[i];
    return;
  }
  uint64_t best = 0;
  int bj = -1;
  for (int q = A.rowptr[i]; q < A.rowptr[i + 1]; ++q) {
    if (!s[q]) continue;
    const int j = A.col[q];
    const bool ok = first ? (isroot[j] != 0) : (agg_in[j] >= 0);
    if (!ok) continue;
    const uint64_t k = mis_key(0, j);
    if (bj < 0 || k > best) {
      best = k;
      bj = j;
    }
  }
  if (bj >= 0) agg_out[i] = first ? rootid[bj] : agg_in[bj];
  else {
    agg_out[i] = -1;
    atomicAdd(unassigned, 1);
  }
}

// P row i = sum_j (delta_ij - omega a_ij / a_ii) e_{agg(j)}: sort (agg, coef) pairs of row i
// by aggregate (stable insertion sort in a scratch laid out like A) and merge duplicates.
template <bool FILL>
__global__ void k_prolong(Csr<double> A, const double* dinv, const int* agg, double omega,
                          int* skey, double* sval, int* cnt, const int* pptr, int* pcol,
                          double* pval) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nrows) return;
  const int b = A.rowptr[i], e = A.rowptr[i + 1];
  for (int q = b; q < e; ++q) {
    const int j = A.col[q];
    const int k = agg[j];
    const double c = (j == i ? 1.0 : 0.0) - omega * A.val[q] * dinv[i];
    int t = q - 1;
    while (t >= b && skey[t] > k) {
      skey[t + 1] = skey[t];
      sval[t + 1] = sval[t];
      --t;
    }
    skey[t + 1] = k;
    sval[t + 1] = c;
  }
  int out = FILL ? pptr[i] : 0, n = 0;
  for (int q = b; q < e; ++q) {
    if (q == b || skey[q] != skey[q - 1]) {
      if (FILL) {
        pcol[out + n] = skey[q];
        pval[out + n] = sval[q];
      }
      ++n;
    } else if (FILL) {
      pval[out + n - 1] += sval[q];
    }
  }
  if (!FILL) cnt[i] = n;
}

__global__ void k_to_dense(Csr<double> A, double* D) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nrows) return;
  const int n = A.nrows;
  for (int j = 0; j < 2 * n; ++j) D[(size_t)i * 2 * n + j] = (j == n + i) ? 1.0 : 0.0;
  for (int q = A.rowptr[i]; q < A.rowptr[i + 1]; ++q) D[(size_t)i * 2 * n + A.col[q]] = A.val[q];
}

// Gauss-Jordan elimination of [A | I] in one thread block (A is SPD: no pivoting needed,
// a non-positive pivot is reported).  Leaves A^-1 in the right half.
__global__ void k_gauss_jordan(int n, double* D, double* inv, int* bad) {
  const int w = 2 * n;
  __shared__ double piv;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      piv = D[(size_t)k * w + k];
      if (!(piv > 0.0)) *bad = 1;
    }
    __syncthreads();
    const double ip = 1.0 / piv;
    for (int j = threadIdx.x; j < w; j += blockDim.x) D[(size_t)k * w + j] *= ip;
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * w; idx += blockDim.x) {
      const int i = idx / w, j = idx % w;
      if (i == k || j == k) continue;
      D[(size_t)i * w + j] -= D[(size_t)i * w + k] * D[(size_t)k * w + j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (i != k) D[(size_t)i * w + k] = 0.0;
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    inv[idx] = D[(size_t)i * w + n + j];
  }
}

// Grid-wide Gauss-Jordan for larger coarsest levels, two launches per pivot k: the first
// scales the pivot row of [A | I] and copies column k (so the update reads it race-free), the
// second eliminates column k from every other row.
__global__ void k_gj_pivot(int n, int k, double* D, double* colk, int* bad) {
  const int w = 2 * n;
  const double piv = D[(size_t)k * w + k];
  const double ip = 1.0 / piv;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0 && !(piv > 0.0)) *bad = 1;
  // column k of the other rows (the pivot row's own entry is not needed).  D[k][k] itself is
  // left as it is: every block reads it as the pivot, and no later step reads it again.
  if (t < n) colk[t] = t == k ? 0.0 : D[(size_t)t * w + k];
  for (int j = t; j < w; j += gridDim.x * blockDim.x) {
    if (j == k) continue;
    D[(size_t)k * w + j] *= ip;
  }
}

__global__ void k_gj_eliminate(int n, int k, double* D, const double* colk) {
  const int w = 2 * n;
  const int64_t total = (int64_t)n * w;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / w), j = (int)(idx % w);
    if (i == k) continue;
    D[idx] = j == k ? 0.0 : D[idx] - colk[i] * D[(size_t)k * w + j];
  }
}

__global__ void k_gj_extract(int n, const double* D, double* inv) {
  const int64_t total = (int64_t)n * n;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    inv[idx] = D[(size_t)i * 2 * n + n + j];
  }
}

__global__ void k_d2f(const double* a, float* b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
template <typename T>
__global__ void k_copy_cast(const double* a, T* b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (T)a[i];
}

// ---------------------------------------------------------------- spectral radius of D^-1 A
// Power iteration with the D-weighted Rayleigh quotient lambda = (x, A x) / (x, D x), which for
// symmetric A converges twice as fast as the norm ratio.  One launch computes y = D^-1 A x and
// the block partials of (x, A x), (x, D x) and (y, D y); a one-block launch sums them in block
// order and stores lambda and the D-norm scaling of y for the next iterate.
constexpr int POW_BLOCKS = 152 * 2;

__global__ void k_pow_init(int n, double* x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = 0.5 + (double)(hash32((uint32_t)i * 2654435761u + 12345u) >> 8) * 0x1.0p-24;
}

__global__ void k_pow_step(Csr<double> A, const double* __restrict__ dinv, const double* __restrict__ x,
                           double* __restrict__ y, double* partials) {
  __shared__ double sm[3][TPB];
  double p0 = 0.0, p1 = 0.0, p2 = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.nrows; i += gridDim.x * blockDim.x) {
    double ax = 0.0;
    for (int q = A.rowptr[i]; q < A.rowptr[i + 1]; ++q) ax = fma(A.val[q], x[A.col[q]], ax);
    const double di = dinv[i];
    p0 = fma(x[i], ax, p0);
    p1 = fma(x[i] * x[i], 1.0 / di, p1);
    p2 = fma(ax * ax, di, p2);
    y[i] = di * ax;
  }
  sm[0][threadIdx.x] = p0;
  sm[1][threadIdx.x] = p1;
  sm[2][threadIdx.x] = p2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int c = 0; c < 3; ++c) sm[c][threadIdx.x] += sm[c][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 3) partials[3 * blockIdx.x + threadIdx.x] = sm[threadIdx.x][0];
}

__global__ void k_pow_reduce(int nb, const double* partials, double* out /* lambda, scale */) {
  if (threadIdx.x != 0) return;
  double t0 = 0.0, t1 = 0.0, t2 = 0.0;
  for (int b = 0; b < nb; ++b) {
    t0 += partials[3 * b];
    t1 += partials[3 * b + 1];
    t2 += partials[3 * b + 2];
  }
  out[0] = t1 > 0.0 ? t0 / t1 : 0.0;
  out[1] = t2 > 0.0 ? 1.0 / sqrt(t2) : 0.0;
}

__global__ void k_pow_scale(int n, const double* y, const double* out, double* x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = y[i] * out[1];
}

// lambda_max(D^-1 A) estimate (20 iterations); the caller caps it by the Gershgorin bound
static ch_status power_estimate(const Csr<double>& A, const double* dinv, cudaStream_t st,
                                double* lambda) {
  const int n = A.nrows;
  Alloc tmp;
  double *x = nullptr, *y = nullptr, *part = nullptr, *out = nullptr;
  CH_TRY(tmp.get(&x, (size_t)n));
  CH_TRY(tmp.get(&y, (size_t)n));
  CH_TRY(tmp.get(&part, (size_t)3 * POW_BLOCKS));
  CH_TRY(tmp.get(&out, 2));
  const int nb = blocks_for(n) < POW_BLOCKS ? blocks_for(n) : POW_BLOCKS;
  k_pow_init<<<blocks_for(n), TPB, 0, st>>>(n, x);
  for (int it = 0; it < 20; ++it) {
    k_pow_step<<<nb, TPB, 0, st>>>(A, dinv, x, y, part);
    k_pow_reduce<<<1, 32, 0, st>>>(nb, part, out);
    k_pow_scale<<<blocks_for(n), TPB, 0, st>>>(n, y, out, x);
  }
  CH_LAUNCHED();
  double h_out[2] = {0.0, 0.0};
  CH_CUDA(cudaMemcpyAsync(h_out, out, sizeof(h_out), cudaMemcpyDeviceToHost, st));
  CH_CUDA(cudaStreamSynchronize(st));
  *lambda = h_out[0];
  return CH_OK;
}

// ---------------------------------------------------------------- set-up driver
static ch_status level_setup(Hierarchy* h, int l, const ch_params& p, cudaStream_t st,
                             bool* last) {
  const Csr<double>& A = h->A[l];
  const int n = A.nrows;
  double* dinv = nullptr;
  CH_TRY(h->mem.get(&dinv, (size_t)n));
  h->dinv.push_back(dinv);
  Alloc tmp;
  double *rb = nullptr, *rmax = nullptr;
  CH_TRY(tmp.get(&rb, (size_t)n));
  CH_TRY(tmp.get(&rmax, 1));
  k_diag_gersh<<<blocks_for(n), TPB, 0, st>>>(A, dinv, rb);
  k_max_reduce<<<1, TPB, 0, st>>>(rb, n, rmax);
  CH_LAUNCHED();
  double rho = 0.0;
  CH_CUDA(cudaMemcpyAsync(&rho, rmax, sizeof(double), cudaMemcpyDeviceToHost, st));
  CH_CUDA(cudaStreamSynchronize(st));
  if (!(rho > 0.0) || !std::isfinite(rho)) {
    set_error("AMG level %d: bad Gershgorin bound %g (zero or non-finite diagonal?)", l, rho);
    return CH_ERR_NONFINITE;
  }
  // Gershgorin overestimates lambda_max(D^-1 A) on coarse aggregation levels (by 30-150% on the
  // meshes here), which would misplace the Chebyshev interval: use a power-iteration estimate
  // with a 5% margin, never above the Gershgorin bound.
  double lam = 0.0;
  CH_TRY(power_estimate(A, dinv, st, &lam));
  if (lam > 0.0 && std::isfinite(lam)) rho = std::min(rho, 1.05 * lam);
  h->rho.push_back(rho);
  // coarse_max 0: 512 rows for FP64 V-cycles, 2048 for FP32 (where the dense inverse is half the
  // bytes); measured on 512 x 512, the dense solve beating the per-level launch chain up to there
  // (FP64: 512 and 1024 alike, 11.63 ms per step; FP32: 4.85-4.88 ms at 4096 rows, 4.75 at 2048;
  // the 64-run batch 30.9-31.1 ms either way, the 3D 128 x 128 x 32 box 14.8 ms either way)
  const int cmax = p.coarse_max > 0 ? p.coarse_max : (h->precision == 0 ? 512 : 2048);
  if (n <= cmax) {
    *last = true;
    return CH_OK;
  }
  // strength of connection
  uint8_t *s0 = nullptr, *s = nullptr;
  CH_TRY(tmp.get(&s0, (size_t)A.nnz));
  CH_TRY(tmp.get(&s, (size_t)A.nnz));
  k_strength<<<blocks_for(n), TPB, 0, st>>>(A, dinv, p.amg_theta, s0);
  k_strength_sym<<<blocks_for(n), TPB, 0, st>>>(A, s0, s);
  CH_LAUNCHED();
  // MIS(2)
  int8_t* state = nullptr;
  uint64_t *key = nullptr, *m1 = nullptr, *m2 = nullptr;
  int* und = nullptr;
  CH_TRY(tmp.get(&state, (size_t)n));
  CH_TRY(tmp.get(&key, (size_t)n));
  CH_TRY(tmp.get(&m1, (size_t)n));
  CH_TRY(tmp.get(&m2, (size_t)n));
  CH_TRY(tmp.get(&und, 1));
  CH_CUDA(cudaMemsetAsync(state, 1, (size_t)n, st));
  for (int round = 0;; ++round) {
    if (round > 200) {
      set_error("AMG level %d: MIS(2) did not finish", l);
      return CH_ERR_INTERNAL;
    }
    k_mis_keys<<<blocks_for(n), TPB, 0, st>>>(n, state, key);
    k_strong_max<<<blocks_for(n), TPB, 0, st>>>(A, s, key, m1);
    k_strong_max<<<blocks_for(n), TPB, 0, st>>>(A, s, m1, m2);
    CH_CUDA(cudaMemsetAsync(und, 0, sizeof(int), st));
    k_mis_update<<<blocks_for(n), TPB, 0, st>>>(n, key, m2, state, und);
    CH_LAUNCHED();
    int u = 0;
    CH_CUDA(cudaMemcpyAsync(&u, und, sizeof(int), cudaMemcpyDeviceToHost, st));
    CH_CUDA(cudaStreamSynchronize(st));
    if (u == 0) break;
  }
  // aggregates
  int *isroot = nullptr, *rootid = nullptr, *agg = nullptr, *agg2 = nullptr, *una = nullptr;
  CH_TRY(tmp.get(&isroot, (size_t)n));
  CH_TRY(tmp.get(&rootid, (size_t)n + 1));
  CH_TRY(tmp.get(&agg, (size_t)n));
  CH_TRY(tmp.get(&agg2, (size_t)n));
  CH_TRY(tmp.get(&una, 1));
  k_roots<<<blocks_for(n), TPB, 0, st>>>(n, state, isroot);
  CH_LAUNCHED();
  int64_t nc = 0;
  CH_TRY(scan_i32_to_rowptr(isroot, rootid, n, &nc, st, tmp));
  for (int pass = 0;; ++pass) {
    if (pass > 50) {
      set_error("AMG level %d: aggregation did not cover all nodes", l);
      return CH_ERR_INTERNAL;
    }
    CH_CUDA(cudaMemsetAsync(una, 0, sizeof(int), st));
    k_agg_pass<<<blocks_for(n), TPB, 0, st>>>(A, s, isroot, rootid, agg, agg2, pass == 0, una);
    CH_LAUNCHED();
    std::swap(agg, agg2);
    int u = 0;
    CH_CUDA(cudaMemcpyAsync(&u, una, sizeof(int), cudaMemcpyDeviceToHost, st));
    CH_CUDA(cudaStreamSynchronize(st));
    if (u == 0) break;
  }
  // smoothed prolongator
  Csr<double> P;
  P.nrows = n;
  P.ncols = (int)nc;
  int *skey = nullptr, *cnt = nullptr;
  double* sval = nullptr;
  CH_TRY(tmp.get(&skey, (size_t)A.nnz));
  CH_TRY(tmp.get(&sval, (size_t)A.nnz));
  CH_TRY(tmp.get(&cnt, (size_t)n));
  const double omega = (4.0 / 3.0) / rho;
  k_prolong<false><<<blocks_for(n), TPB, 0, st>>>(A, dinv, agg, omega, skey, sval, cnt, nullptr,
                                                   nullptr, nullptr);
  CH_LAUNCHED();
  CH_TRY(h->mem.get(&P.rowptr, (size_t)n + 1));
  int64_t pnnz = 0;
  CH_TRY(scan_i32_to_rowptr(cnt, P.rowptr, n, &pnnz, st, tmp));
  P.nnz = pnnz;
  CH_TRY(h->mem.get(&P.col, (size_t)pnnz));
  CH_TRY(h->mem.get(&P.val, (size_t)pnnz));
  k_prolong<true><<<blocks_for(n), TPB, 0, st>>>(A, dinv, agg, omega, skey, sval, cnt, P.rowptr,
                                                  P.col, P.val);
  CH_LAUNCHED();
  Csr<double> R, AP, Ac;
  CH_TRY(transpose(P, &R, st, h->mem));
  Alloc aptmp;
  CH_TRY(spgemm(A, P, &AP, st, aptmp));
  CH_TRY(spgemm(R, AP, &Ac, st, h->mem));
  h->P.push_back(P);
  h->R.push_back(R);
  h->A.push_back(Ac);
  CH_CUDA(cudaStreamSynchronize(st));
  return CH_OK;
}

template <typename T, typename V2>
static void launch_residual(int tpr, const Csr<T>& A, const V2* b, const V2* x, V2* r, cudaStream_t st,
                            const Dia<T>* dia = nullptr, bool pdl = false);
template <typename T, typename V2, bool ACC>
static void launch_spmv2(int tpr, const Csr<T>& A, const V2* x, V2* y, cudaStream_t st, bool pdl = false);

// ---------------------------------------------------------------- SpMV tile autotuner
// Lanes per row (1..32) for each matrix the V-cycle multiplies by: A (smoother steps and
// residuals), R (restriction), P (prolongation).  autotune = 0 takes the rule below; 1 times
// every candidate on the matrix itself (one warm-up, three timed launches) and keeps the rule's
// choice unless another is more than 5% faster.  Decisions are cached per process by matrix
// shape (kind, rows, columns, entries, value size), so rebuilding a hierarchy of the same shape
// reproduces its choices -- and its floating-point summation order -- exactly.  A process that
// wants its choices made on a busy GPU builds its first solver with autotune = 0 (nothing is
// cached then) and tunes afterwards.
static int tpr_rule(int64_t nnz, int rows) {
  const double avg = rows > 0 ? (double)nnz / rows : 1.0;
  int t = 1;
  while (t < 32 && 4.0 * t <= avg) t *= 2;
  return t;
}

static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int64_t, int>, int> g_tune_cache;

template <typename Launch>
static int tune_tpr(int kind, int rows, int cols, int64_t nnz, int tsize, int mode, Launch&& launch,
                    cudaStream_t st) {
  const int rule = tpr_rule(nnz, rows);
  if (mode == 0 || rows == 0) return rule;
  const auto key = std::make_tuple(kind, rows, cols, nnz, tsize);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) return it->second;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return rule;
  }
  // An idle GPU ramps its clocks over the first fraction of a second: warm up on the rule's width,
  // then time every width in two passes and keep each width's faster pass.
  for (int r = 0; r < 20; ++r) launch(rule);
  float t[6];
  for (int k = 0; k < 6; ++k) t[k] = 1e30f;
  for (int pass = 0; pass < 2; ++pass) {
    for (int k = 0, tpr = 1; k < 6; ++k, tpr *= 2) {
      launch(tpr);
      cudaEventRecord(e0, st);
      for (int r = 0; r < 3; ++r) launch(tpr);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 1e30f;
      cudaEventElapsedTime(&ms, e0, e1);
      t[k] = std::min(t[k], ms);
    }
  }
  float best = 1e30f, t_rule = 1e30f;
  int pick = rule;
  for (int k = 0, tpr = 1; k < 6; ++k, tpr *= 2) {
    if (tpr == rule) t_rule = t[k];
    if (t[k] < best) {
      best = t[k];
      pick = tpr;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  if (t_rule <= 1.05f * best) pick = rule;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = pick;
  return pick;
}

template <typename T>
static ch_status autotune_levels(Hierarchy* h, std::vector<LevelT<T>>& L, int mode, cudaStream_t st) {
  using V2 = typename V2T<T>::t;
  for (int l = 0; l < h->nlev; ++l) {
    const int n = L[l].A.nrows;
    V2* vecs[5] = {L[l].x, L[l].x2, L[l].d, L[l].r, L[l].b};
    for (int k = 0; k < 5; ++k) CH_CUDA(cudaMemsetAsync(vecs[k], 0, sizeof(V2) * n, st));
  }
  for (int l = 0; l < h->nlev; ++l) {
    LevelT<T>& W = L[l];
    W.tprA = W.dia.nd ? 1
                      : tune_tpr(0, W.A.nrows, W.A.ncols, W.A.nnz, sizeof(T), mode,
                                 [&](int t) { launch_residual<T, V2>(t, W.A, W.b, W.x, W.r, st); }, st);
    if (l + 1 < h->nlev) {
      LevelT<T>& C = L[l + 1];
      W.tprR = tune_tpr(1, W.R.nrows, W.R.ncols, W.R.nnz, sizeof(T), mode,
                        [&](int t) { launch_spmv2<T, V2, false>(t, W.R, W.r, C.b, st); }, st);
      W.tprP = tune_tpr(2, W.P.nrows, W.P.ncols, W.P.nnz, sizeof(T), mode,
                        [&](int t) { launch_spmv2<T, V2, true>(t, W.P, C.x, W.x, st); }, st);
    }
  }
  CH_LAUNCHED();
  CH_CUDA(cudaStreamSynchronize(st));
  return CH_OK;
}

__global__ void k_csr_to_dia(Csr<double> A, Dia<double> D) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nrows) return;
  int W = D.W, WH = D.WH;
  if (D.node_run) {
    const int2 w = D.run_wh[D.node_run[i]];
    W = w.x;
    WH = w.y;
  }
  for (int q = A.rowptr[i]; q < A.rowptr[i + 1]; ++q) {
    const int o = A.col[q] - i;
    for (int d = 0; d < D.nd; ++d)
      if (lat_off(D.nd, d, W, WH) == o) D.val[(size_t)d * A.nrows + i] = A.val[q];
  }
}

// The diagonal form of A when every stored entry of every row lies on the lattice stencil of its
// run (checked on the host from the pattern at set-up); else nd = 0 and the level stays CSR.
static ch_status dia_build(const Csr<double>& A, const FineLattice* lat, Alloc& mem, Dia<double>* out,
                           cudaStream_t st) {
  out->nd = 0;
  if (!lat || (lat->dim != 2 && lat->dim != 3)) return CH_OK;
  const int n = A.nrows, R = (int)lat->W.size();
  if (R < 1 || (int)lat->run_off.size() != R + 1 || lat->run_off[R] != n) return CH_OK;
  const int nd = lat->dim == 2 ? 7 : 15;
  std::vector<int> rp(n + 1), col((size_t)A.nnz);
  CH_CUDA(cudaMemcpyAsync(rp.data(), A.rowptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, st));
  CH_CUDA(cudaMemcpyAsync(col.data(), A.col, sizeof(int) * (size_t)A.nnz, cudaMemcpyDeviceToHost, st));
  CH_CUDA(cudaStreamSynchronize(st));
  for (int r = 0; r < R; ++r) {
    const int W = lat->W[r], WH = lat->WH[r];
    if (W < 2 || WH < 2 * W) return CH_OK;
    int offs[15];
    for (int d = 0; d < nd; ++d) offs[d] = lat_off(nd, d, W, WH);
    for (int i = lat->run_off[r]; i < lat->run_off[r + 1]; ++i)
      for (int q = rp[i]; q < rp[i + 1]; ++q) {
        const int o = col[q] - i;
        bool on = false;
        for (int d = 0; d < nd && !on; ++d) on = offs[d] == o;
        if (!on) return CH_OK;
      }
  }
  Dia<double> D;
  D.nd = nd;
  if (R == 1) {
    D.W = lat->W[0];
    D.WH = lat->WH[0];
  } else {
    std::vector<int2> wh(R);
    for (int r = 0; r < R; ++r) wh[r] = make_int2(lat->W[r], lat->WH[r]);
    int2* d_wh = nullptr;
    CH_TRY(mem.get(&d_wh, (size_t)R));
    CH_CUDA(cudaMemcpyAsync(d_wh, wh.data(), sizeof(int2) * R, cudaMemcpyHostToDevice, st));
    CH_CUDA(cudaStreamSynchronize(st));  // wh is a host temporary
    D.node_run = lat->node_run;
    D.run_wh = d_wh;
  }
  CH_TRY(mem.get(&D.val, (size_t)nd * n));
  CH_CUDA(cudaMemsetAsync(D.val, 0, sizeof(double) * (size_t)nd * n, st));
  k_csr_to_dia<<<blocks_for(n), TPB, 0, st>>>(A, D);
  CH_LAUNCHED();
  *out = D;
  return CH_OK;
}

template <typename T>
static ch_status make_working(Hierarchy* h, const FineLattice* lat, std::vector<LevelT<T>>& L, cudaStream_t st) {
  using V2 = typename V2T<T>::t;
  L.resize(h->nlev);
  for (int l = 0; l < h->nlev; ++l) {
    LevelT<T>& w = L[l];
    auto cast_csr = [&](const Csr<double>& src, Csr<T>& dst) -> ch_status {
      dst.nrows = src.nrows;
      dst.ncols = src.ncols;
      dst.nnz = src.nnz;
      dst.rowptr = src.rowptr;
      dst.col = src.col;
      if (std::is_same<T, double>::value) {
        dst.val = reinterpret_cast<T*>(src.val);
      } else {
        CH_TRY(h->mem.get(&dst.val, (size_t)src.nnz));
        k_copy_cast<T><<<blocks_for(src.nnz), TPB, 0, st>>>(src.val, dst.val, src.nnz);
        CH_LAUNCHED();
      }
      return CH_OK;
    };
    CH_TRY(cast_csr(h->A[l], w.A));
    if (l + 1 < h->nlev) {
      CH_TRY(cast_csr(h->P[l], w.P));
      CH_TRY(cast_csr(h->R[l], w.R));
    }
    const int n = h->A[l].nrows;
    if (std::is_same<T, double>::value) {
      w.dinv = reinterpret_cast<T*>(h->dinv[l]);
    } else {
      CH_TRY(h->mem.get(&w.dinv, (size_t)n));
      k_copy_cast<T><<<blocks_for(n), TPB, 0, st>>>(h->dinv[l], w.dinv, n);
      CH_LAUNCHED();
    }
    CH_TRY(h->mem.get(&w.x, (size_t)n));
    CH_TRY(h->mem.get(&w.x2, (size_t)n));
    CH_TRY(h->mem.get(&w.d, (size_t)n));
    CH_TRY(h->mem.get(&w.r, (size_t)n));
    CH_TRY(h->mem.get(&w.b, (size_t)n));
    w.pdl = h->pdl;
  }

  // the fine level of a uniform mesh in diagonal form
  Dia<double> d64;
  CH_TRY(dia_build(h->A[0], lat, h->mem, &d64, st));
  if (d64.nd) {
    Dia<T>& d = L[0].dia;
    d.nd = d64.nd;
    d.W = d64.W;
    d.WH = d64.WH;
    d.node_run = d64.node_run;
    d.run_wh = d64.run_wh;
    const size_t cnt = (size_t)d64.nd * h->A[0].nrows;
    if (std::is_same<T, double>::value) {
      d.val = reinterpret_cast<T*>(d64.val);
    } else {
      CH_TRY(h->mem.get(&d.val, cnt));
      k_copy_cast<T><<<blocks_for((int64_t)cnt), TPB, 0, st>>>(d64.val, d.val, (int64_t)cnt);
      CH_LAUNCHED();
    }
  }
  return autotune_levels<T>(h, L, h->autotune, st);
}

ch_status hierarchy_build(const Csr<double>& A0, const FineLattice* lat, const ch_params& p, int precision, cudaStream_t st,
                          Hierarchy** out) {
  *out = nullptr;
  Hierarchy* h = new Hierarchy();
  h->precision = precision;
  h->cheb_degree = p.cheb_degree;
  // cheb_degree_coarse 0: degree 2 below the finest level (at most cheb_degree).  Measured on
  // 512 x 512 with the finest degree 5: FP64 79.8 / 75.9 / 70.9 and mixed 173.3 / 170.5 / 164.1
  // steps/s for coarse degrees 2 / 3 / 4
  h->cheb_degree_coarse = p.cheb_degree_coarse > 0 ? p.cheb_degree_coarse : std::min(2, p.cheb_degree);
  h->autotune = p.autotune;
  h->pdl = p.pdl != 0;
  h->cheb_lower = p.cheb_lower;
  h->A.push_back(A0);
  ch_status s = CH_OK;
  for (int l = 0;; ++l) {
    if (l >= 25) {
      set_error("AMG: more than 25 levels");
      s = CH_ERR_INTERNAL;
      break;
    }
    bool last = false;
    s = level_setup(h, l, p, st, &last);
    if (s != CH_OK || last) break;
  }
  if (s == CH_OK) {
    h->nlev = (int)h->A.size();
    h->nc = h->A.back().nrows;
    if (h->nc > 4096) {
      set_error("AMG: coarsest level has %d rows (> 4096); coarsening stalled", h->nc);
      s = CH_ERR_INTERNAL;
    }
  }
  if (s == CH_OK) {
    Alloc tmp;
    double* D = nullptr;
    int* bad = nullptr;
    const int nc = h->nc;
    s = tmp.get(&D, (size_t)nc * 2 * nc);
    if (s == CH_OK) s = tmp.get(&bad, 1);
    if (s == CH_OK) s = h->mem.get(&h->cinv, (size_t)nc * nc);
    if (s == CH_OK) {
      cudaMemsetAsync(bad, 0, sizeof(int), st);
      k_to_dense<<<blocks_for(nc), TPB, 0, st>>>(h->A.back(), D);
      if (nc <= 256) {
        k_gauss_jordan<<<1, 1024, 0, st>>>(nc, D, h->cinv, bad);
      } else {
        double* colk = nullptr;
        if (tmp.get(&colk, (size_t)nc) != CH_OK) {
          s = CH_ERR_OOM;
        } else {
          const int gp = (2 * nc + TPB - 1) / TPB;
          for (int k = 0; k < nc; ++k) {
            k_gj_pivot<<<gp, TPB, 0, st>>>(nc, k, D, colk, bad);
            k_gj_eliminate<<<4 * 152, TPB, 0, st>>>(nc, k, D, colk);
          }
          k_gj_extract<<<4 * 152, TPB, 0, st>>>(nc, D, h->cinv);
        }
      }
      int hb = 0;
      cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        set_error("AMG: coarse inverse failed");
        s = CH_ERR_CUDA;
      } else if (hb) {
        set_error("AMG: coarsest operator not positive definite");
        s = CH_ERR_INTERNAL;
      }
    }
  }
  if (s == CH_OK) {
    if (precision == 0) {
      s = make_working<double>(h, lat, h->Ld, st);
    } else {
      s = make_working<float>(h, lat, h->Lf, st);
      if (s == CH_OK) s = h->mem.get(&h->cinvf, (size_t)h->nc * h->nc);
      if (s == CH_OK) {
        k_d2f<<<blocks_for((int64_t)h->nc * h->nc), TPB, 0, st>>>(h->cinv, h->cinvf,
                                                                  (int64_t)h->nc * h->nc);
      }
    }
    if (s == CH_OK && cudaStreamSynchronize(st) != cudaSuccess) {
      set_error("AMG: building working copies failed");
      s = CH_ERR_CUDA;
    }
  }
  if (s != CH_OK) {
    delete h;
    return s;
  }
  *out = h;
  return CH_OK;
}

void hierarchy_free(Hierarchy* h) { delete h; }
int hierarchy_levels(const Hierarchy* h) { return h ? h->nlev : 0; }
void hierarchy_level_tiles(const Hierarchy* h, int l, int* tA, int* tR, int* tP) {
  const int a = h->precision == 0 ? h->Ld[l].tprA : h->Lf[l].tprA;
  const int r = h->precision == 0 ? h->Ld[l].tprR : h->Lf[l].tprR;
  const int q = h->precision == 0 ? h->Ld[l].tprP : h->Lf[l].tprP;
  if (tA) *tA = a;
  if (tR) *tR = l + 1 < h->nlev ? r : 0;
  if (tP) *tP = l + 1 < h->nlev ? q : 0;
}

void hierarchy_level_size(const Hierarchy* h, int l, int64_t* rows, int64_t* nnz) {
  if (rows) *rows = h->A[l].nrows;
  if (nnz) *nnz = h->A[l].nnz;
}

// Level l as the V-cycle uses it: the FP64 set-up matrices A_l and P_l (device to device copies
// into caller buffers), the Chebyshev interval [cheb_lower, 1] x 1.1 rho_l of D^-1 A_l and the
// smoothing degree; the coarsest level has no P and no smoothing (dense inverse).
ch_status hierarchy_level_export(const Hierarchy* h, int l, int64_t* rows, int64_t* nnz, int64_t* nnz_P,
                                 double* lo, double* hi, int* degree, int* A_rowptr, int* A_col,
                                 double* A_val, int* P_rowptr, int* P_col, double* P_val, cudaStream_t st) {
  const Csr<double>& A = h->A[l];
  const bool coarsest = l + 1 == h->nlev;
  const int64_t np = coarsest ? 0 : h->P[l].nnz;
  if (rows) *rows = A.nrows;
  if (nnz) *nnz = A.nnz;
  if (nnz_P) *nnz_P = np;
  const double top = coarsest ? 0.0 : 1.1 * h->rho[l];
  if (hi) *hi = top;
  if (lo) *lo = h->cheb_lower * top;
  if (degree) *degree = coarsest ? 0 : (l == 0 ? h->cheb_degree : h->cheb_degree_coarse);
  const auto copy = [&](void* dst, const void* src, size_t bytes) -> ch_status {
    if (dst && bytes) CH_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st));
    return CH_OK;
  };
  CH_TRY(copy(A_rowptr, A.rowptr, sizeof(int) * ((size_t)A.nrows + 1)));
  CH_TRY(copy(A_col, A.col, sizeof(int) * (size_t)A.nnz));
  CH_TRY(copy(A_val, A.val, sizeof(double) * (size_t)A.nnz));
  if (!coarsest) {
    const Csr<double>& P = h->P[l];
    CH_TRY(copy(P_rowptr, P.rowptr, sizeof(int) * ((size_t)P.nrows + 1)));
    CH_TRY(copy(P_col, P.col, sizeof(int) * (size_t)P.nnz));
    CH_TRY(copy(P_val, P.val, sizeof(double) * (size_t)P.nnz));
  }
  return CH_OK;
}

// ---------------------------------------------------------------- V-cycle kernels (2 RHS)
// When a V-cycle kernel lets its successor be scheduled (programmatic dependent launch): right
// after its dependency wait in FP32, where the kernels are short and bound by latency, so the
// successor's blocks are resident when it finishes; not at all in FP64, where the kernels are
// bound by the FP64 pipe and successor blocks that arrive early crowd the SMs unevenly.  Measured
// on the 512 x 512 mesh, ms per time step: FP32 V-cycles 8.33 plain, 8.06 without the trigger,
// 7.96 with it; FP64 V-cycles 16.90 plain, 16.78 without, 17.70 with it (16.75 when only grids of
// at most 152 blocks trigger, 17.28 at most 608; that small-grid rule took FP64 32 x 32 steps from
// 2.26 to 2.21 ms but 128 x 128 steps from 2.95 to 3.03).
template <typename T>
__device__ __forceinline__ void pdl_trigger_t() {
  if (sizeof(T) == 4) pdl_trigger();
}

template <typename T, typename V2>
__device__ __forceinline__ V2 mk2(T a, T b) {
  V2 v;
  v.x = a;
  v.y = b;
  return v;
}

// x = D^-1 b / theta (first Chebyshev step from a zero guess); d = x
template <typename T, typename V2>
__global__ void k_cheb_first(int n, const T* dinv, const V2* b, T invtheta, V2* x, V2* d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const T di = i < n ? dinv[i] : T(0);  // set-up data: read before the dependency wait
  pdl_wait();
  pdl_trigger_t<T>();
  if (i >= n) return;
  const T s = invtheta * di;
  const V2 bi = b[i];
  const V2 v = mk2<T, V2>(s * bi.x, s * bi.y);
  x[i] = v;
  d[i] = v;
}

// Row sums of A x for both right-hand sides with TPR lanes per row: lane `sub` takes entries
// sub, sub+TPR, ... of the row and a butterfly of shuffles adds the lanes' partial sums, so the
// summation order is fixed for a given TPR.  Threads past the last row contribute zeros (no
// early return before the shuffles).  The sum adds onto the caller's (s0, s1), which lane 0 of a
// row may seed (with -b: the sum is then A x - b at no extra FP64 instruction).
//
// The row's structure and values are set-up data, so a kernel reads them before its programmatic
// dependency wait (row_prefetch: the lane's first CsrRow::PF entries, i.e. rowptr, then val and col)
// and only gathers x after it (row_acc): one dependent L2 round trip behind the wait instead of
// three (rowptr, col, x).  Entries past the prefetched ones are read after the wait, in the same
// order.
template <typename T, int TPR>
struct CsrRow {
  static constexpr int PF = TPR == 1 ? 8 : (TPR <= 4 ? 4 : 2);  // entries per lane read early
  int q = 0, e = 0;  // the lane's next entry after the prefetched ones; the row's end
  T a[PF];
  int c[PF];
};

template <typename T, int TPR>
__device__ __forceinline__ void row_prefetch(const Csr<T>& A, int row, int sub, CsrRow<T, TPR>& r) {
  constexpr int PF = CsrRow<T, TPR>::PF;
#pragma unroll
  for (int k = 0; k < PF; ++k) {
    r.a[k] = T(0);
    r.c[k] = -1;
  }
  if (row < A.nrows) {
    const int b = A.rowptr[row] + sub;
    r.e = A.rowptr[row + 1];
#pragma unroll
    for (int k = 0; k < PF; ++k) {
      const int q = b + k * TPR;
      if (q < r.e) {
        r.a[k] = A.val[q];
        r.c[k] = A.col[q];
      }
    }
    r.q = b + PF * TPR;
  }
}

template <typename T, typename V2, int TPR>
__device__ __forceinline__ void row_acc(const Csr<T>& A, const CsrRow<T, TPR>& r, const V2* __restrict__ x,
                                        T& s0, T& s1) {
  constexpr int PF = CsrRow<T, TPR>::PF;
  V2 xj[PF];
#pragma unroll
  for (int k = 0; k < PF; ++k)
    if (r.c[k] >= 0) xj[k] = x[r.c[k]];
#pragma unroll
  for (int k = 0; k < PF; ++k)
    if (r.c[k] >= 0) {
      s0 = fma(r.a[k], xj[k].x, s0);
      s1 = fma(r.a[k], xj[k].y, s1);
    }
  for (int q = r.q; q < r.e; q += TPR) {
    const T a = A.val[q];
    const V2 v = x[A.col[q]];
    s0 = fma(a, v.x, s0);
    s1 = fma(a, v.y, s1);
  }
#pragma unroll
  for (int o = TPR / 2; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
}

// r = b - A x;  d = alpha d + beta D^-1 r;  xo = x + d.  The row sum starts from -b, so it is
// -r, and nbeta = -beta turns it back: d = alpha d + (nbeta D^-1) (A x - b), three FP64
// instructions per right-hand side after the sum (multiply, fused multiply-add, add).
template <typename T, typename V2, int TPR>
__global__ void __launch_bounds__(TPB) k_cheb_step(Csr<T> A, const T* __restrict__ dinv,
                                                   const V2* __restrict__ b, const V2* __restrict__ x,
                                                   V2* __restrict__ d, V2* __restrict__ xo, T alpha,
                                                   T nbeta) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t / TPR, sub = t % TPR;
  CsrRow<T, TPR> row;
  row_prefetch<T, TPR>(A, i, sub, row);
  const T di = (sub == 0 && i < A.nrows) ? dinv[i] * nbeta : T(0);
  pdl_wait();
  pdl_trigger_t<T>();
  T s0 = 0, s1 = 0;
  if (sub == 0 && i < A.nrows) {
    const V2 bi = b[i];
    s0 = -bi.x;
    s1 = -bi.y;
  }
  row_acc<T, V2, TPR>(A, row, x, s0, s1);
  if (i >= A.nrows || sub != 0) return;
  const V2 xi = x[i];
  V2 dd;
  if (alpha != T(0)) {
    const V2 dold = d[i];
    dd = mk2<T, V2>(fma(alpha, dold.x, di * s0), fma(alpha, dold.y, di * s1));
  } else {
    dd = mk2<T, V2>(di * s0, di * s1);
  }
  d[i] = dd;
  xo[i] = mk2<T, V2>(xi.x + dd.x, xi.y + dd.y);
}

template <typename T, typename V2, int TPR>
__global__ void __launch_bounds__(TPB) k_residual(Csr<T> A, const V2* __restrict__ b,
                                                  const V2* __restrict__ x, V2* __restrict__ r) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t / TPR, sub = t % TPR;
  CsrRow<T, TPR> row;
  row_prefetch<T, TPR>(A, i, sub, row);
  pdl_wait();
  pdl_trigger_t<T>();
  T s0 = 0, s1 = 0;
  row_acc<T, V2, TPR>(A, row, x, s0, s1);
  if (i >= A.nrows || sub != 0) return;
  const V2 bi = b[i];
  r[i] = mk2<T, V2>(bi.x - s0, bi.y - s1);
}

// y = A x (ACC = false) or y += A x (ACC = true)
template <typename T, typename V2, int TPR, bool ACC>
__global__ void __launch_bounds__(TPB) k_spmv2(Csr<T> A, const V2* __restrict__ x, V2* __restrict__ y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t / TPR, sub = t % TPR;
  CsrRow<T, TPR> row;
  row_prefetch<T, TPR>(A, i, sub, row);
  pdl_wait();
  pdl_trigger_t<T>();
  T s0 = 0, s1 = 0;
  row_acc<T, V2, TPR>(A, row, x, s0, s1);
  if (i >= A.nrows || sub != 0) return;
  if (ACC) {
    const V2 yi = y[i];
    y[i] = mk2<T, V2>(yi.x + s0, yi.y + s1);
  } else {
    y[i] = mk2<T, V2>(s0, s1);
  }
}

// ---------------------------------------------------------------- structured (diagonal) fine level
// One row of the lattice form: its ND operator values and its run's strides (set-up data, so the
// kernels read them before their dependency wait).
template <typename T, int ND>
struct DiaRow {
  T a[ND];
  int W, WH;
};
template <typename T, int ND>
__device__ __forceinline__ DiaRow<T, ND> dia_row(const Dia<T>& D, int n, int i) {
  DiaRow<T, ND> r;
  r.W = D.W;
  r.WH = D.WH;
  if (D.node_run) {
    const int2 w = D.run_wh[D.node_run[i]];
    r.W = w.x;
    r.WH = w.y;
  }
#pragma unroll
  for (int d = 0; d < ND; ++d) r.a[d] = D.val[(size_t)d * n + i];
  return r;
}

// Row sum of the lattice form onto the caller's (s0, s1) (zero, or -b for a residual's negative).
template <typename T, typename V2, int ND>
__device__ __forceinline__ void dia_row_acc(const DiaRow<T, ND>& r, int n, int i, const V2* __restrict__ x,
                                            T& s0, T& s1) {
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    int j = i + lat_off(ND, d, r.W, r.WH);
    j = j < 0 ? 0 : (j >= n ? n - 1 : j);
    const V2 xj = x[j];
    s0 = fma(r.a[d], xj.x, s0);
    s1 = fma(r.a[d], xj.y, s1);
  }
}

// k_cheb_step on the lattice form (same arithmetic: the sum starts from -b, nbeta = -beta)
template <typename T, typename V2, int ND>
__global__ void __launch_bounds__(TPB) k_cheb_step_dia(Dia<T> D, int n, const T* __restrict__ dinv,
                                                       const V2* __restrict__ b, const V2* __restrict__ x,
                                                       V2* __restrict__ d, V2* __restrict__ xo, T alpha, T nbeta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  DiaRow<T, ND> row;
  T di = 0;
  if (i < n) {
    row = dia_row<T, ND>(D, n, i);
    di = dinv[i] * nbeta;
  }
  pdl_wait();
  pdl_trigger_t<T>();
  if (i >= n) return;
  const V2 bi = b[i];
  T s0 = -bi.x, s1 = -bi.y;
  dia_row_acc<T, V2, ND>(row, n, i, x, s0, s1);
  const V2 xi = x[i];
  V2 dd;
  if (alpha != T(0)) {
    const V2 dold = d[i];
    dd = mk2<T, V2>(fma(alpha, dold.x, di * s0), fma(alpha, dold.y, di * s1));
  } else {
    dd = mk2<T, V2>(di * s0, di * s1);
  }
  d[i] = dd;
  xo[i] = mk2<T, V2>(xi.x + dd.x, xi.y + dd.y);
}

template <typename T, typename V2, int ND>
__global__ void __launch_bounds__(TPB) k_residual_dia(Dia<T> D, int n, const V2* __restrict__ b,
                                                      const V2* __restrict__ x, V2* __restrict__ r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  DiaRow<T, ND> row;
  if (i < n) row = dia_row<T, ND>(D, n, i);
  pdl_wait();
  pdl_trigger_t<T>();
  if (i >= n) return;
  T s0 = 0, s1 = 0;
  dia_row_acc<T, V2, ND>(row, n, i, x, s0, s1);
  const V2 bi = b[i];
  r[i] = mk2<T, V2>(bi.x - s0, bi.y - s1);
}

template <typename T, typename V2, int ND>
__global__ void __launch_bounds__(TPB) k_spmv2_dia(Dia<T> D, int n, const V2* __restrict__ x, V2* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  DiaRow<T, ND> row;
  if (i < n) row = dia_row<T, ND>(D, n, i);
  pdl_wait();
  pdl_trigger_t<T>();
  if (i >= n) return;
  T s0 = 0, s1 = 0;
  dia_row_acc<T, V2, ND>(row, n, i, x, s0, s1);
  y[i] = mk2<T, V2>(s0, s1);
}

#define CH_DIA_DISPATCH(nd, KCALL)                    \
  switch (nd) {                                       \
    case 7: { constexpr int NDC = 7; KCALL; } break;  \
    default: { constexpr int NDC = 15; KCALL; } break; \
  }

// b_c = R r, fused with the coarse level's first Chebyshev step from a zero guess (pointwise:
// x_c = d_c = invtheta D_c^-1 b_c, the arithmetic of k_cheb_first): one launch instead of two.
template <typename T, typename V2, int TPR>
__global__ void __launch_bounds__(TPB) k_restrict_first(Csr<T> R, const V2* __restrict__ r, V2* __restrict__ bc,
                                                        const T* __restrict__ dinv_c, T invtheta,
                                                        V2* __restrict__ xc, V2* __restrict__ dc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t / TPR, sub = t % TPR;
  CsrRow<T, TPR> row;
  row_prefetch<T, TPR>(R, i, sub, row);
  const T s = (sub == 0 && i < R.nrows) ? invtheta * dinv_c[i] : T(0);
  pdl_wait();
  pdl_trigger_t<T>();
  T s0 = 0, s1 = 0;
  row_acc<T, V2, TPR>(R, row, r, s0, s1);
  if (i >= R.nrows || sub != 0) return;
  bc[i] = mk2<T, V2>(s0, s1);
  const V2 v = mk2<T, V2>(s * s0, s * s1);
  xc[i] = v;
  dc[i] = v;
}

#define CH_TPR_DISPATCH(tpr, KCALL)                      \
  switch (tpr) {                                         \
    case 1: { constexpr int TPRC = 1; KCALL; } break;    \
    case 2: { constexpr int TPRC = 2; KCALL; } break;    \
    case 4: { constexpr int TPRC = 4; KCALL; } break;    \
    case 8: { constexpr int TPRC = 8; KCALL; } break;    \
    case 16: { constexpr int TPRC = 16; KCALL; } break;  \
    default: { constexpr int TPRC = 32; KCALL; } break;  \
  }

// one Chebyshev step d = alpha d + beta D^-1 (b - A x), xo = x + d (the kernels take -beta)
template <typename T, typename V2>
static void launch_cheb_step(int tpr, const Csr<T>& A, const T* dinv, const V2* b, const V2* x, V2* d,
                             V2* xo, T alpha, T beta, cudaStream_t st, const Dia<T>* dia = nullptr,
                             bool pdl = false) {
  const T nbeta = -beta;
  if (dia && dia->nd) {
    const int g = blocks_for(A.nrows);
    CH_DIA_DISPATCH(dia->nd, (launch_k(pdl, k_cheb_step_dia<T, V2, NDC>, g, TPB, 0, st, *dia, A.nrows, dinv, b,
                                       x, d, xo, alpha, nbeta)));
    return;
  }
  const int g = blocks_for((int64_t)A.nrows * tpr);
  CH_TPR_DISPATCH(tpr, (launch_k(pdl, k_cheb_step<T, V2, TPRC>, g, TPB, 0, st, A, dinv, b, x, d, xo, alpha,
                                 nbeta)));
}
template <typename T, typename V2>
static void launch_residual(int tpr, const Csr<T>& A, const V2* b, const V2* x, V2* r, cudaStream_t st,
                            const Dia<T>* dia, bool pdl) {
  if (dia && dia->nd) {
    const int g = blocks_for(A.nrows);
    CH_DIA_DISPATCH(dia->nd, (launch_k(pdl, k_residual_dia<T, V2, NDC>, g, TPB, 0, st, *dia, A.nrows, b, x, r)));
    return;
  }
  const int g = blocks_for((int64_t)A.nrows * tpr);
  CH_TPR_DISPATCH(tpr, (launch_k(pdl, k_residual<T, V2, TPRC>, g, TPB, 0, st, A, b, x, r)));
}
// y = A x with the level's operator (the diagonal form where there is one)
template <typename T, typename V2>
static void launch_apply_level(const LevelT<T>& L, const V2* x, V2* y, cudaStream_t st) {
  if (L.dia.nd) {
    const int g = blocks_for(L.A.nrows);
    CH_DIA_DISPATCH(L.dia.nd, (launch_k(L.pdl, k_spmv2_dia<T, V2, NDC>, g, TPB, 0, st, L.dia, L.A.nrows, x, y)));
    return;
  }
  launch_spmv2<T, V2, false>(L.tprA, L.A, x, y, st, L.pdl);
}
template <typename T, typename V2, bool ACC>
static void launch_spmv2(int tpr, const Csr<T>& A, const V2* x, V2* y, cudaStream_t st, bool pdl) {
  const int g = blocks_for((int64_t)A.nrows * tpr);
  CH_TPR_DISPATCH(tpr, (launch_k(pdl, k_spmv2<T, V2, TPRC, ACC>, g, TPB, 0, st, A, x, y)));
}

// x = Ainv b, dense nc x nc.  WPR warps per row: lane l of the row's warp `sub` takes columns
// sub * 32 + l + k * 32 WPR, with its first U entries of Ainv read before the dependency wait and
// 8 loads in flight after it; the lanes' sums are added by a butterfly and the warps' in warp order.
template <typename T, typename V2, int WPR>
__global__ void __launch_bounds__(TPB) k_dense_solve(int n, const T* __restrict__ inv, const V2* __restrict__ b,
                                                     V2* __restrict__ x) {
  static_assert((TPB / 32) % WPR == 0, "a row's warps share a block");
  constexpr int U = 8;  // the lane's first entries, read before the dependency wait
  __shared__ T part[TPB / 32][2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int row = gw / WPR, sub = gw % WPR;
  const bool on = row < n;
  const int stride = 32 * WPR, j0 = sub * 32 + lane;
  const T* __restrict__ a = inv + (size_t)(on ? row : 0) * n;
  T pa[U];
#pragma unroll
  for (int k = 0; k < U; ++k) {
    const int j = j0 + k * stride;
    pa[k] = (on && j < n) ? a[j] : T(0);
  }
  pdl_wait();
  pdl_trigger_t<T>();
  T s0 = 0, s1 = 0;
  if (on) {
    V2 bj[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int j = j0 + k * stride;
      if (j < n) bj[k] = b[j];
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      if (j0 + k * stride < n) {
        s0 = fma(pa[k], bj[k].x, s0);
        s1 = fma(pa[k], bj[k].y, s1);
      }
    }
#pragma unroll 8
    for (int j = j0 + U * stride; j < n; j += stride) {
      const T aj = a[j];
      const V2 v = b[j];
      s0 = fma(aj, v.x, s0);
      s1 = fma(aj, v.y, s1);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if (WPR == 1) {
    if (on && lane == 0) x[row] = mk2<T, V2>(s0, s1);
    return;
  }
  if (lane == 0) {
    part[w][0] = s0;
    part[w][1] = s1;
  }
  __syncthreads();
  if (on && sub == 0 && lane == 0) {
    T t0 = s0, t1 = s1;
#pragma unroll
    for (int q = 1; q < WPR; ++q) {
      t0 += part[w + q][0];
      t1 += part[w + q][1];
    }
    x[row] = mk2<T, V2>(t0, t1);
  }
}

// x = Ainv b on the dense coarsest level, two warps per row.  Measured alone with the inverse
// flushed from L2 (us per solve, one / two / four warps per row): 3742 FP32 rows 26.2 / 22.5 / 24.8,
// 2048 FP32 rows 14.3 / 9.8 / 10.5, 512 FP64 rows 11.1 / 7.8 / 9.8.
template <typename T, typename V2>
static void launch_dense_solve(bool pdl, int n, const T* cinv, const V2* b, V2* x, cudaStream_t st) {
  launch_k(pdl, k_dense_solve<T, V2, 2>, blocks_for((int64_t)n * 64), TPB, 0, st, n, cinv, b, x);
}

// fine-level I/O: strided fp64 pairs <-> working precision pairs
template <typename T, typename V2>
__global__ void k_load2(int n, const double* src, int ld, V2* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_wait();
  pdl_trigger_t<T>();
  if (i >= n) return;
  const double2 v = *reinterpret_cast<const double2*>(src + (size_t)i * ld);
  dst[i] = mk2<T, V2>((T)v.x, (T)v.y);
}
// k_load2 fused with the finest level's first Chebyshev step from a zero guess (the arithmetic of
// k_cheb_first on the converted values): b = (T) src, x = d = invtheta D^-1 b.  One launch instead
// of two at the start of the first V-cycle of a solve.
template <typename T, typename V2>
__global__ void k_load2_first(int n, const double* src, int ld, const T* dinv, T invtheta, V2* b, V2* x, V2* d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const T di = i < n ? dinv[i] : T(0);  // set-up data: read before the dependency wait
  pdl_wait();
  pdl_trigger_t<T>();
  if (i >= n) return;
  const double2 v = *reinterpret_cast<const double2*>(src + (size_t)i * ld);
  const V2 bi = mk2<T, V2>((T)v.x, (T)v.y);
  b[i] = bi;
  const T s = invtheta * di;
  const V2 w = mk2<T, V2>(s * bi.x, s * bi.y);
  x[i] = w;
  d[i] = w;
}
template <typename T, typename V2>
__global__ void k_store2(int n, const V2* src, double* dst, int ld) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_wait();
  pdl_trigger_t<T>();
  if (i >= n) return;
  const V2 v = src[i];
  *reinterpret_cast<double2*>(dst + (size_t)i * ld) = make_double2((double)v.x, (double)v.y);
}

// ---------------------------------------------------------------- V-cycle driver
struct ChebCoef {
  double invtheta;
  double alpha[16], beta[16];
};

// Coefficients of `deg` Chebyshev semi-iteration steps for eigenvalues in [lo, hi]: the first
// step from zero is x = D^-1 b / theta, then d = alpha_s d + beta_s D^-1 (b - A x), x += d.
static ChebCoef cheb_coef_interval(double lo, double hi, int deg) {
  ChebCoef c{};
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  c.invtheta = 1.0 / theta;
  c.alpha[0] = 0.0;
  c.beta[0] = 1.0 / theta;
  double rho_prev = 1.0 / sigma;
  for (int s = 1; s < deg && s < 16; ++s) {
    const double r = 1.0 / (2.0 * sigma - rho_prev);
    c.alpha[s] = r * rho_prev;
    c.beta[s] = 2.0 * r / delta;
    rho_prev = r;
  }
  return c;
}

// the V-cycle smoother's interval: [lower, 1] x 1.1 rho
static ChebCoef cheb_coef(double rho, int deg, double lower) {
  const double hi = 1.1 * rho;
  return cheb_coef_interval(lower * hi, hi, deg);
}

// `deg` Chebyshev steps with coefficients c on level L (accounted as kernels kfirst / kstep).
// zero_guess: 0 continue from *xcur; 1 start from zero (the first step is pointwise); 2 start from
// zero with that first step already taken by the caller (fused into the restriction)
template <typename T_>
static ch_status smooth_coef(LevelT<T_>& L, const ChebCoef& c, int deg, int zero_guess, int kfirst, int kstep,
                             typename V2T<T_>::t** xcur, cudaStream_t st) {
  using V2 = typename V2T<T_>::t;
  const int n = L.A.nrows;
  V2* x = *xcur;
  V2* other = (x == L.x) ? L.x2 : L.x;
  int s0 = 0;
  const double T = sizeof(T_), nnz = (double)L.A.nnz;
  if (zero_guess == 1) {
    ProfScope ps(st, kfirst, sizeof(T_) == 4, 7.0 * T * n, 2.0 * n);
    launch_k(L.pdl, k_cheb_first<T_, V2>, blocks_for(n), TPB, 0, st, n, L.dinv, L.b, (T_)c.invtheta, x, L.d);
    s0 = 1;
  } else if (zero_guess == 2) {
    s0 = 1;
  }
  // operator bytes: CSR values + column indices + row pointers, or the diagonals' values
  const double opb = L.dia.nd ? T * L.dia.nd * (double)n : nnz * (4 + T) + 4.0 * (n + 1);
  for (int s = s0; s < deg; ++s) {
    ProfScope ps(st, kstep, sizeof(T_) == 4, opb + T * n * (c.alpha[s] != 0.0 ? 11 : 9), 2.0 * nnz + 4.0 * n);
    launch_cheb_step<T_, V2>(L.tprA, L.A, L.dinv, L.b, x, L.d, other, (T_)c.alpha[s], (T_)c.beta[s], st,
                             &L.dia, L.pdl);
    std::swap(x, other);
  }
  CH_LAUNCHED();
  *xcur = x;
  return CH_OK;
}

// the V-cycle's smoother on level l: its degree and interval
template <typename T_>
static ch_status smooth(Hierarchy* h, LevelT<T_>& L, int l, int zero_guess,
                        typename V2T<T_>::t** xcur, cudaStream_t st) {
  const int deg = l == 0 ? h->cheb_degree : h->cheb_degree_coarse;
  const ChebCoef c = cheb_coef(h->rho[l], deg, h->cheb_lower);
  return smooth_coef<T_>(L, c, deg, zero_guess, l == 0 ? K_CHEB_FIRST : K_CHEB_FIRST_C,
                         l == 0 ? K_CHEB_STEP : K_CHEB_STEP_C, xcur, st);
}

// M~^-1 by the Chebyshev semi-iteration (Section 3's alternative to AMG for the mass matrix):
// `steps` steps on D^-1 M from a zero guess over Wathen's bounds of its eigenvalues for P1
// simplices, [1/2, 2] (triangles) and [1/2, 5/2] (tetrahedra), on the finest level of M's
// hierarchy (its working-precision copy of M and D^-1).  b in L.b; result in *xres.
template <typename T_>
static ch_status semi_iteration(LevelT<T_>& L, int dim, int steps, typename V2T<T_>::t** xres, cudaStream_t st) {
  const ChebCoef c = cheb_coef_interval(0.5, dim == 2 ? 2.0 : 2.5, steps);
  *xres = L.x;
  return smooth_coef<T_>(L, c, steps, 1, K_CHEB_SEMI, K_CHEB_SEMI, xres, st);
}

// one V-cycle at level l on L[l].b; result in *xres (L[l].x or L[l].x2)
template <typename T>
static ch_status vcycle(Hierarchy* h, std::vector<LevelT<T>>& Ls, const T* cinv, int l,
                        int zero_guess, typename V2T<T>::t** xres, cudaStream_t st) {
  using V2 = typename V2T<T>::t;
  LevelT<T>& L = Ls[l];
  const int n = L.A.nrows;
  const double Tb = sizeof(T);
  if (l == h->nlev - 1) {
    ProfScope ps(st, K_COARSE, sizeof(T) == 4, Tb * n * (double)n + 4.0 * Tb * n, 2.0 * n * (double)n);
    launch_dense_solve<T, V2>(L.pdl, n, cinv, L.b, L.x, st);
    CH_LAUNCHED();
    *xres = L.x;
    return CH_OK;
  }
  V2* x = *xres;
  CH_TRY(smooth<T>(h, L, l, zero_guess, &x, st));
  LevelT<T>& C = Ls[l + 1];
  const int nc = C.A.nrows;
  {
    const double opb = L.dia.nd ? Tb * L.dia.nd * (double)n : L.A.nnz * (4 + Tb) + 4.0 * (n + 1);
    ProfScope ps(st, l == 0 ? K_VRESIDUAL : K_VRESIDUAL_C, sizeof(T) == 4, opb + 6.0 * Tb * n, 2.0 * L.A.nnz);
    launch_residual<T, V2>(L.tprA, L.A, L.b, x, L.r, st, &L.dia, L.pdl);
  }
  const bool fuse = l + 1 < h->nlev - 1;  // the coarse level smooths: fuse its first step
  {
    ProfScope ps(st, l == 0 ? K_RESTRICT : K_RESTRICT_C, sizeof(T) == 4,
                 L.R.nnz * (4 + Tb) + 4.0 * (nc + 1) + 2.0 * Tb * (n + nc) + (fuse ? 5.0 * Tb * nc : 0.0),
                 2.0 * L.R.nnz + (fuse ? 2.0 * nc : 0.0));
    if (fuse) {
      const int degc = h->cheb_degree_coarse;
      const ChebCoef cc = cheb_coef(h->rho[l + 1], degc, h->cheb_lower);
      const int g = blocks_for((int64_t)L.R.nrows * L.tprR);
      CH_TPR_DISPATCH(L.tprR, (launch_k(L.pdl, k_restrict_first<T, V2, TPRC>, g, TPB, 0, st, L.R, L.r, C.b,
                                        C.dinv, (T)cc.invtheta, C.x, C.d)));
    } else {
      launch_spmv2<T, V2, false>(L.tprR, L.R, L.r, C.b, st, L.pdl);
    }
  }
  CH_LAUNCHED();
  V2* xc = C.x;
  CH_TRY(vcycle<T>(h, Ls, cinv, l + 1, fuse ? 2 : 1, &xc, st));
  {
    ProfScope ps(st, l == 0 ? K_PROLONG : K_PROLONG_C, sizeof(T) == 4,
                 L.P.nnz * (4 + Tb) + 4.0 * (n + 1) + 2.0 * Tb * nc + 4.0 * Tb * n, 2.0 * L.P.nnz);
    launch_spmv2<T, V2, true>(L.tprP, L.P, xc, x, st, L.pdl);
  }
  CH_LAUNCHED();
  CH_TRY(smooth<T>(h, L, l, 0, &x, st));
  *xres = x;
  return CH_OK;
}

template <typename T>
static ch_status solve_t(Hierarchy* h, std::vector<LevelT<T>>& Ls, const T* cinv, const double* b,
                         int ldb, double* x, int ldx, int ncyc, cudaStream_t st) {
  using V2 = typename V2T<T>::t;
  LevelT<T>& L = Ls[0];
  const int n = L.A.nrows;
  launch_k(L.pdl, k_load2<T, V2>, blocks_for(n), TPB, 0, st, n, b, ldb, L.b);
  CH_LAUNCHED();
  V2* xr = L.x;
  for (int c = 0; c < ncyc; ++c) CH_TRY(vcycle<T>(h, Ls, cinv, 0, c == 0, &xr, st));
  launch_k(L.pdl, k_store2<T, V2>, blocks_for(n), TPB, 0, st, n, xr, x, ldx);
  CH_LAUNCHED();
  return CH_OK;
}

// `passes` passes of the finest level's Chebyshev smoother of degree `degree` (the V-cycle's
// interval), each continuing from the previous pass's x; x (N x 2, fp64) is read and overwritten
template <typename T>
static ch_status smooth_t(Hierarchy* h, std::vector<LevelT<T>>& Ls, const double* b, double* x, int degree,
                          int passes, cudaStream_t st) {
  using V2 = typename V2T<T>::t;
  LevelT<T>& L = Ls[0];
  const int n = L.A.nrows;
  const double io = n * (16.0 + 2.0 * sizeof(T));
  {
    ProfScope ps(st, K_VLOAD, sizeof(T) == 4, 2.0 * io, 0.0);
    launch_k(L.pdl, k_load2<T, V2>, blocks_for(n), TPB, 0, st, n, b, 2, L.b);
  }
  {
    ProfScope ps(st, K_VLOAD, sizeof(T) == 4, 0.0, 0.0);  // its bytes are counted with the first load
    launch_k(L.pdl, k_load2<T, V2>, blocks_for(n), TPB, 0, st, n, x, 2, L.x);
  }
  CH_LAUNCHED();
  const ChebCoef c = cheb_coef(h->rho[0], degree, h->cheb_lower);
  V2* xr = L.x;
  for (int k = 0; k < passes; ++k) CH_TRY(smooth_coef<T>(L, c, degree, 0, K_CHEB_FIRST, K_CHEB_STEP, &xr, st));
  {
    ProfScope ps(st, K_VSTORE, sizeof(T) == 4, io, 0.0);
    launch_k(L.pdl, k_store2<T, V2>, blocks_for(n), TPB, 0, st, n, xr, x, 2);
  }
  CH_LAUNCHED();
  return CH_OK;
}

ch_status hierarchy_smooth(Hierarchy* h, const double* b, double* x, int degree, int passes, cudaStream_t st) {
  if (h->precision == 0) return smooth_t<double>(h, h->Ld, b, x, degree, passes, st);
  return smooth_t<float>(h, h->Lf, b, x, degree, passes, st);
}

ch_status hierarchy_solve(Hierarchy* h, const double* b, int ldb, double* x, int ldx, int ncyc,
                          cudaStream_t st) {
  if (h->precision == 0) return solve_t<double>(h, h->Ld, h->cinv, b, ldb, x, ldx, ncyc, st);
  return solve_t<float>(h, h->Lf, h->cinvf, b, ldb, x, ldx, ncyc, st);
}

// ---------------------------------------------------------------- Algorithm 1
// w_1 = AMG(M) v_1;  w_2 = AMG(H) v_2;  w_2 = M w_2;  w_2 = AMG(H) w_2.
// v, w are N x 4 (phi_p, phi_n, mu_p, mu_n per node): block 1 at offset 0, block 2 at offset 2.
static int semi_steps(const ch_params& p) { return p.cheb_M_steps > 0 ? p.cheb_M_steps : 5; }

// The fine-level input of a solve: b = (T) v (strided FP64 pairs).  With AMG V-cycles on a
// hierarchy of more than one level the first V-cycle's first smoothing step (from zero) is done in
// the same launch (k_load2_first), and the V-cycle then starts at its second step (zero_guess 2).
// Returns the zero_guess for the first V-cycle.
template <typename T>
static int load_input(Hierarchy* h, LevelT<T>& L, bool amg, const double* v, int ld, cudaStream_t st) {
  using V2 = typename V2T<T>::t;
  const int n = L.A.nrows;
  if (amg && h->nlev > 1) {
    const ChebCoef c = cheb_coef(h->rho[0], h->cheb_degree, h->cheb_lower);
    ProfScope ps(st, K_VLOAD, sizeof(T) == 4, n * (16.0 + 7.0 * sizeof(T)), 2.0 * n);
    launch_k(L.pdl, k_load2_first<T, V2>, blocks_for(n), TPB, 0, st, n, v, ld, L.dinv, (T)c.invtheta, L.b, L.x,
             L.d);
    return 2;
  }
  ProfScope ps(st, K_VLOAD, sizeof(T) == 4, n * (16.0 + 2.0 * sizeof(T)), 0.0);
  launch_k(L.pdl, k_load2<T, V2>, blocks_for(n), TPB, 0, st, n, v, ld, L.b);
  return 1;
}

template <typename T>
static ch_status precond_t(ch_precond_s* pc, std::vector<LevelT<T>>& LM, std::vector<LevelT<T>>& LH,
                           const T* cinvM, const T* cinvH, const double* v, double* w,
                           cudaStream_t st) {
  using V2 = typename V2T<T>::t;
  const int n = LM[0].A.nrows;
  const ch_params& p = pc->sys->p;
  // Step 1 does not depend on steps 2-4: it runs on the preconditioner's side stream, forked
  // from and joined back into st (inside a stream capture this becomes two parallel graph
  // branches).  Both chains are mostly latency-bound coarse-level launches, so they overlap.
  // With per-launch event timing on, everything stays on st so that kernel times do not overlap.
  const bool fork = pc->side != nullptr && !prof_timing();
  cudaStream_t sm = st;
  if (fork) {
    CH_CUDA(cudaEventRecord(pc->ev_fork, st));
    CH_CUDA(cudaStreamWaitEvent(pc->side, pc->ev_fork, 0));
    sm = pc->side;
  }
  // step 1: M w_1 = v_1 (w_1 in columns 0-1 of w; steps 2-4 write columns 2-3)
  {
    LevelT<T>& L = LM[0];
    const int zg = load_input<T>(pc->hM, L, p.precond_M != 1, v, 4, sm);
    V2* xr = L.x;
    if (p.precond_M == 1) {
      CH_TRY(semi_iteration<T>(L, pc->sys->mesh->dim, semi_steps(p), &xr, sm));
    } else {
      for (int c = 0; c < p.vcycles_M; ++c) CH_TRY(vcycle<T>(pc->hM, LM, cinvM, 0, c == 0 ? zg : 0, &xr, sm));
    }
    {
      ProfScope ps(sm, K_VSTORE, sizeof(T) == 4, n * (16.0 + 2.0 * sizeof(T)), 0.0);
      launch_k(L.pdl, k_store2<T, V2>, blocks_for(n), TPB, 0, sm, n, xr, w, 4);
    }
    CH_LAUNCHED();
  }
  if (fork) CH_CUDA(cudaEventRecord(pc->ev_join, sm));
  // steps 2-4: H w_2 = v_2; w_2 = M w_2; H w_2 = w_2
  {
    LevelT<T>& L = LH[0];
    const int zg = load_input<T>(pc->hH, L, true, v + 2, 4, st);
    V2* xr = L.x;
    for (int c = 0; c < p.vcycles_H; ++c) CH_TRY(vcycle<T>(pc->hH, LH, cinvH, 0, c == 0 ? zg : 0, &xr, st));
    // b <- M x (M's fine level in working precision); the V-cycle reads only L.b afterwards
    {
      const double Tb = sizeof(T), nnz = (double)LM[0].A.nnz;
      const double opb = LM[0].dia.nd ? Tb * LM[0].dia.nd * (double)n : nnz * (4 + Tb) + 4.0 * (n + 1);
      ProfScope ps(st, K_SPMV_M, sizeof(T) == 4, opb + 4.0 * Tb * n, 2.0 * nnz);
      launch_apply_level<T, V2>(LM[0], xr, L.b, st);
    }
    CH_LAUNCHED();
    xr = L.x;  // the first solve's result now lives in L.b as M x; start afresh
    for (int c = 0; c < p.vcycles_H; ++c) CH_TRY(vcycle<T>(pc->hH, LH, cinvH, 0, c == 0, &xr, st));
    {
      ProfScope ps(st, K_VSTORE, sizeof(T) == 4, n * (16.0 + 2.0 * sizeof(T)), 0.0);
      launch_k(L.pdl, k_store2<T, V2>, blocks_for(n), TPB, 0, st, n, xr, w + 2, 4);
    }
    CH_LAUNCHED();
  }
  if (fork) CH_CUDA(cudaStreamWaitEvent(st, pc->ev_join, 0));
  return CH_OK;
}

ch_status precond_apply(ch_precond_s* pc, const double* v, double* w, cudaStream_t st) {
  if (pc->precision == 0)
    return precond_t<double>(pc, pc->hM->Ld, pc->hH->Ld, pc->hM->cinv, pc->hH->cinv, v, w, st);
  return precond_t<float>(pc, pc->hM->Lf, pc->hH->Lf, pc->hM->cinvf, pc->hH->cinvf, v, w, st);
}

// Algorithm 1's step 1 alone on two right-hand sides (N x 2): x = M~^-1 b
template <typename T>
static ch_status mass_solve_t(ch_precond_s* pc, std::vector<LevelT<T>>& LM, const T* cinvM, const double* b,
                              double* x, cudaStream_t st) {
  using V2 = typename V2T<T>::t;
  const ch_params& p = pc->sys->p;
  LevelT<T>& L = LM[0];
  const int n = L.A.nrows;
  k_load2<T, V2><<<blocks_for(n), TPB, 0, st>>>(n, b, 2, L.b);
  CH_LAUNCHED();
  V2* xr = L.x;
  if (p.precond_M == 1) {
    CH_TRY(semi_iteration<T>(L, pc->sys->mesh->dim, semi_steps(p), &xr, st));
  } else {
    for (int c = 0; c < p.vcycles_M; ++c) CH_TRY(vcycle<T>(pc->hM, LM, cinvM, 0, c == 0, &xr, st));
  }
  k_store2<T, V2><<<blocks_for(n), TPB, 0, st>>>(n, xr, x, 2);
  CH_LAUNCHED();
  return CH_OK;
}

ch_status mass_solve(ch_precond_s* pc, const double* b, double* x, cudaStream_t st) {
  if (pc->precision == 0) return mass_solve_t<double>(pc, pc->hM->Ld, pc->hM->cinv, b, x, st);
  return mass_solve_t<float>(pc, pc->hM->Lf, pc->hM->cinvf, b, x, st);
}

}  // namespace ch

// ---------------------------------------------------------------- allocation-free V-cycles
// ch_vcycle_noalloc runs the same V-cycles as ch_vcycle, but the per-level work vectors
// (x, x2, d, r, b for every level, two right-hand sides each) are carved out of one
// file-scope device array instead of the preconditioner's own buffers, so a call needs no
// device memory beyond the caller's b and x and the already-built hierarchy.  The array is
// reserved in every GPU that loads the library for the life of the process.
namespace ch {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(8) << 20;  // 8 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// The array's device address for the current device.  In host code the symbol names a host
// stand-in, so the address is looked up once per device (with that device current) and cached.
ch_status noalloc_scratch(void** out) {
  int dev = -1;
  CH_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    set_error("ch_vcycle_noalloc: device ordinal %d not supported (max %d)", dev, NOALLOC_MAX_DEVICES);
    return CH_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_error("ch_vcycle_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return CH_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return CH_OK;
}
}  // namespace

template <typename T>
static ch_status vcycle_static(Hierarchy* h, LevelT<T>* Ls, const T* cinv, int l, bool zero_guess,
                               typename V2T<T>::t** xres, cudaStream_t st) {
  using V2 = typename V2T<T>::t;
  LevelT<T>& L = Ls[l];
  const int n = L.A.nrows;
  if (l == h->nlev - 1) {
    launch_dense_solve<T, V2>(L.pdl, n, cinv, L.b, L.x, st);
    CH_LAUNCHED();
    *xres = L.x;
    return CH_OK;
  }
  const int deg = l == 0 ? h->cheb_degree : h->cheb_degree_coarse;
  const ChebCoef c = cheb_coef(h->rho[l], deg, h->cheb_lower);
  V2* x = *xres;
  auto smooth_static = [&](bool zg) {
    V2* other = (x == L.x) ? L.x2 : L.x;
    int s0 = 0;
    if (zg) {
      k_cheb_first<T, V2><<<blocks_for(n), TPB, 0, st>>>(n, L.dinv, L.b, (T)c.invtheta, x, L.d);
      s0 = 1;
    }
    for (int s = s0; s < deg; ++s) {
      launch_cheb_step<T, V2>(L.tprA, L.A, L.dinv, L.b, x, L.d, other, (T)c.alpha[s], (T)c.beta[s], st,
                              &L.dia);
      std::swap(x, other);
    }
  };
  smooth_static(zero_guess);
  LevelT<T>& C = Ls[l + 1];
  launch_residual<T, V2>(L.tprA, L.A, L.b, x, L.r, st, &L.dia);
  launch_spmv2<T, V2, false>(L.tprR, L.R, L.r, C.b, st);
  CH_LAUNCHED();
  V2* xc = C.x;
  CH_TRY(vcycle_static<T>(h, Ls, cinv, l + 1, true, &xc, st));
  launch_spmv2<T, V2, true>(L.tprP, L.P, xc, x, st);
  smooth_static(false);
  CH_LAUNCHED();
  *xres = x;
  return CH_OK;
}

template <typename T>
static ch_status solve_static(Hierarchy* h, const std::vector<LevelT<T>>& src, const T* cinv,
                              const double* b, double* x, int ncyc, cudaStream_t st) {
  using V2 = typename V2T<T>::t;
  constexpr int MAXLEV = 32;
  if (h->nlev > MAXLEV) {
    set_error("ch_vcycle_noalloc: hierarchy has %d levels (max %d)", h->nlev, MAXLEV);
    return CH_ERR_ARG;
  }
  // 5 vectors of n_l pairs per level, each rounded up to 256 bytes
  size_t need = 0;
  for (int l = 0; l < h->nlev; ++l) need += 5 * ((src[l].A.nrows * sizeof(V2) + 255) / 256 * 256);
  if (need > NOALLOC_SCRATCH_BYTES) {
    set_error("ch_vcycle_noalloc: hierarchy needs %zu bytes of work space, the static array holds %zu "
              "(use ch_vcycle for this size)", need, NOALLOC_SCRATCH_BYTES);
    return CH_ERR_ARG;
  }
  void* base = nullptr;
  CH_TRY(noalloc_scratch(&base));
  LevelT<T> Ls[MAXLEV];
  unsigned char* cur = static_cast<unsigned char*>(base);
  auto carve = [&](int n) {
    V2* p = reinterpret_cast<V2*>(cur);
    cur += (n * sizeof(V2) + 255) / 256 * 256;
    return p;
  };
  for (int l = 0; l < h->nlev; ++l) {
    Ls[l] = src[l];  // matrices, diagonal inverses: the hierarchy's own
    const int n = src[l].A.nrows;
    Ls[l].x = carve(n);
    Ls[l].x2 = carve(n);
    Ls[l].d = carve(n);
    Ls[l].r = carve(n);
    Ls[l].b = carve(n);
  }
  // Every work vector is written before it is read (zero initial guesses are applied by the
  // first Chebyshev step), so nothing in the array needs clearing between calls.
  const int n0 = Ls[0].A.nrows;
  k_load2<T, V2><<<blocks_for(n0), TPB, 0, st>>>(n0, b, 2, Ls[0].b);
  CH_LAUNCHED();
  V2* xr = Ls[0].x;
  for (int c = 0; c < ncyc; ++c) CH_TRY(vcycle_static<T>(h, Ls, cinv, 0, c == 0, &xr, st));
  k_store2<T, V2><<<blocks_for(n0), TPB, 0, st>>>(n0, xr, x, 2);
  CH_LAUNCHED();
  return CH_OK;
}

ch_status hierarchy_solve_noalloc(Hierarchy* h, const double* b, double* x, int ncyc, cudaStream_t st) {
  if (h->precision == 0) return solve_static<double>(h, h->Ld, h->cinv, b, x, ncyc, st);
  return solve_static<float>(h, h->Lf, h->cinvf, b, x, ncyc, st);
}

}  // namespace ch
