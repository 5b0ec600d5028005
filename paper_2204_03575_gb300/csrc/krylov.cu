// Flexible GMRES(m) in FP64 for the saddle-point systems of one time step (Eq. (14)),
// right-preconditioned by Algorithm 1, plus the time-step driver.
//
// The paper solves each system with preconditioned MINRES (Section 4).  MINRES needs a
// fixed symmetric positive definite preconditioner; one AMG V-cycle with Chebyshev
// smoothing (and its FP32 variant) is neither exactly fixed nor symmetric, so the outer
// method here is flexible GMRES (Saad 1993), which allows the preconditioner to vary.
//
// A state holds R independent runs (R = 1 for a plain mesh; a batched mesh is the disjoint
// union of R run meshes) and two species per run, i.e. 2R independent systems.  Every kernel
// processes the N x 4 node-major vectors (phi_p, phi_n, mu_p, mu_n) of all systems at once;
// the Krylov scalars -- Hessenberg matrix, Givens rotations, convergence flags -- are kept per
// (run, species).  Inner products and norms are segmented: the grid is split so that each
// thread block owns a contiguous node range of exactly one run, and the last block of a run to
// finish (a per-run ticket) sums that run's block partials in a fixed order.  There are no
// floating-point atomics, so runs are bitwise reproducible.  Orthogonalisation is classical
// Gram-Schmidt with one re-orthogonalisation (CGS2).  With CUDA graphs on, the convergence loop
// itself runs on the device (conditional graph nodes, see Ctl): a step is one graph launch.
#include <algorithm>
#include <cmath>

#include <cstdio>
#include <cstring>

#include "ch_internal.cuh"

namespace ch {

constexpr int MAXM = 64;
constexpr int MAXV = 2 * (MAXM + 1);  // reduced values per block (2 species x (j+1))

// Krylov scalars of one run (two species)
struct KrylovDev {
  double R[2][MAXM][MAXM];  // upper-triangular factor after Givens (column j in R[s][.][j])
  double cs[2][MAXM], sn[2][MAXM], g[2][MAXM + 1], y[2][MAXM];
  double h1[2][MAXM + 1], h2[2][MAXM + 1];
  double hinv[2], beta[2], bnorm[2], relres[2], tol[2], mass[2];
  int active[2];        // system still unsolved this step
  int cycle_active[2];  // system still iterating in the current restart cycle
  int k[2];             // Arnoldi steps taken in the current cycle
  int its[2];           // Arnoldi steps taken this step
  int nonfinite;
  unsigned int ticket;  // last-block counter of this run
  double relres_prev[2];  // initial-guess selection: residual of the previous step's state
  int warm[2];            // the caller's guess was taken for this species
  double w2[2];           // selective reorthogonalisation: ||w||^2 before the projection
  int reorth[2];          // ... this Arnoldi step needs the second Gram-Schmidt pass
  int reorth_count[2];    // Arnoldi steps of this time step that took the second pass
};

// Preconditioned MINRES scalars of one run, per species (the Lanczos process on P^-1 A in the
// P inner product and the Givens QR of its tridiagonal matrix).
struct MrDev {
  double gam[2];           // gamma_j: the norm that normalised the current Lanczos vector
  double c[2], cp[2];      // cosines c_j, c_{j-1}
  double s[2], sp[2];      // sines s_j, s_{j-1}
  double eta[2];           // |eta| estimates ||r||_{P^-1}
  double est[2];           // target for |eta| at which the true residual is checked
  double delta[2];         // delta_j = (A z_j) . z_j
  double a1[2], a2[2], a3[2], cn[2], etao[2];  // this iteration's update coefficients
  double scale[2];         // 1 / gamma_{j+1} (0 once the species stops)
  int upd[2];              // the species took this iteration
};

struct Flags {  // summary over all runs
  int cycle_active;  // systems still iterating in the cycle
  int active;        // systems not yet converged
  int nonfinite;
  int pad;
};

// Block decomposition: block b works on nodes [lo[b], hi[b]) of run run[b]; the blocks of run r
// are first[r] .. first[r+1]-1.
struct Seg {
  const int* run;
  const int* lo;
  const int* hi;
  const int* first;
  unsigned int* gticket;  // per block: the last-block counter of the reduction group it starts (else unused)
  int nblocks;            // blocks of the grid; group sums are rows nblocks + (group's first block) of partials
};

// ---------------------------------------------------------------- block reductions
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sm /* [TPB/32][NV] */) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sm[w * NV + k] = x;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int q = 0; q < TPB / 32; ++q) s += sm[q * NV + threadIdx.x];
    sm[threadIdx.x] = s;
  }
  __syncthreads();
}

// After a block has written its partials, returns true in the last block of its run to finish,
// which then reads the run's block partials (reduce_run, a fixed order).
__device__ __forceinline__ bool last_block_of_run(unsigned int* ticket, int nblocks) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int t = atomicAdd(ticket, 1u);
    am_last = (t == (unsigned)nblocks - 1u);
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

// out[v] = sum over k < count of rows[r0 + k stride][v] (rows of MAXV values), v < nv, by the TPB
// threads of one block.  Lanes take values and warps take rows: warp w adds the rows w, w + 8, ...,
// RP_ROWS of them loaded per round (independent loads, past L1: other blocks wrote them), and warp 0
// then adds the 8 warp sums in warp order, so the order is fixed and the sums reproducible.  Every
// FP64 add is a warp instruction over up to 32 values: a warp-wide FP64 instruction holds the SM's
// FP64 pipe equally long whatever its active lanes, so adds of absent rows are skipped.
constexpr int RP_ROWS = 4;  // rows loaded per warp and round: 32 per round (a run's group rows fit one)
__device__ void sum_rows(const double* rows, int r0, int count, int stride, int nv, double* out) {
  constexpr int NW = TPB / 32;
  __shared__ double wsum[NW][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int v0 = 0; v0 < nv; v0 += 32) {
    const int v = v0 + lane;
    const bool on = v < nv;
    double s = 0.0;
    for (int base = w; base < count; base += NW * RP_ROWS) {
      double t[RP_ROWS];
#pragma unroll
      for (int i = 0; i < RP_ROWS; ++i) {
        const int k = base + NW * i;
        t[i] = (on && k < count) ? __ldcg(rows + (size_t)(r0 + k * stride) * MAXV + v) : 0.0;
      }
#pragma unroll
      for (int i = 0; i < RP_ROWS; ++i) {
        if (base + NW * i >= count) break;
        s += t[i];
      }
    }
    wsum[w][lane] = s;
    __syncthreads();
    if (w == 0 && on) {
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < NW; ++q) t += wsum[q][lane];
      out[v] = t;
    }
    __syncthreads();
  }
}

// The run-wide sums of the nv values that each block of the run (blocks b0..b1-1) wrote to its row of
// `partials`: returns true in one block of the run, with out[0..nv) (shared) holding them.  The blocks
// form groups of RGS consecutive blocks of the run: the last block of a group to finish adds the
// group's rows into a group row (row nblocks + the group's first block), and the last of the group
// leaders adds the group rows (a run of at most RGS blocks: its last block adds the rows).  Each level
// adds at most 19 rows for a single run, one round of loads.  Measured (512 x 512, ms per step FP64 /
// mixed): two levels 11.62 / 4.82; one level for up to 32 values 11.75 / 4.98 (304 rows: ten rounds of
// loads); one level with 20 rows per warp in flight 11.69 / 4.90.  Per-block timer stamps at basis
// size 18: the last block's end to the dot sums ready 9.2 us with one level, 6.9 us with two.  The
// grouping and the orders are fixed: reproducible sums.
constexpr int RGS = 16;
__device__ bool reduce_run(const Seg& sg, double* partials, unsigned int* run_ticket, int b0, int b1, int nv,
                           double* out) {
  const int nbr = b1 - b0, ng = (nbr + RGS - 1) / RGS;
  if (ng == 1) {
    if (!last_block_of_run(run_ticket, nbr)) return false;
    sum_rows(partials, b0, nbr, 1, nv, out);
    return true;
  }
  const int gb0 = b0 + ((int)blockIdx.x - b0) / RGS * RGS, gb1 = min(gb0 + RGS, b1);
  if (!last_block_of_run(&sg.gticket[gb0], gb1 - gb0)) return false;
  double* grows = partials + (size_t)sg.nblocks * MAXV;
  sum_rows(partials, gb0, gb1 - gb0, 1, nv, grows + (size_t)gb0 * MAXV);
  if (threadIdx.x == 0) sg.gticket[gb0] = 0;
  if (!last_block_of_run(run_ticket, ng)) return false;
  sum_rows(grows, b0, ng, RGS, nv, out);
  return true;
}

// ---------------------------------------------------------------- residual / norms
// W = b - A x (all systems), then per run the last block computes ||b_s||, ||r_s||, relres and
// sets active / cycle flags, beta and g for a (re)start.  If init, also tol_s = rtol ||b_s||.
__global__ void k_residual4(Seg sg, const int* rowptr, const int* col, const double* valM,
                            const double* valK, double a, double c, const double4_32a* x,
                            const double4_32a* b, double4_32a* W, double* partials, KrylovDev* kds,
                            int init, double rtol) {
  __shared__ double sm[(TPB / 32) * 4];
  const int run = sg.run[blockIdx.x];
  double acc[4] = {0, 0, 0, 0};  // ||b_p||^2, ||b_n||^2, ||r_p||^2, ||r_n||^2
  // Two nodes per iteration (v and v + blockDim.x, the order of the plain loop) with their rows
  // walked in one loop, so that both rows' gathers are in flight together: the segmented grid has
  // 16 warps per SM to hide them.  Each row's sums keep their order.
  const int hi = sg.hi[blockIdx.x];
  for (int v = sg.lo[blockIdx.x] + threadIdx.x; v < hi; v += 2 * blockDim.x) {
    const int v2 = v + blockDim.x;
    const bool two = v2 < hi;
    const int q0 = rowptr[v], n0 = rowptr[v + 1] - q0;
    const int p0 = two ? rowptr[v2] : 0, n1 = two ? rowptr[v2 + 1] - p0 : 0;
    double u[8] = {0, 0, 0, 0, 0, 0, 0, 0}, t[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // M x, K x per node
    const int len = n0 > n1 ? n0 : n1;
    for (int e = 0; e < len; ++e) {
      if (e < n0) {
        const int q = q0 + e;
        const double m = valM[q], k = valK[q];
        const double4_32a z = x[col[q]];
        u[0] = fma(m, z.x, u[0]);
        u[1] = fma(m, z.y, u[1]);
        u[2] = fma(m, z.z, u[2]);
        u[3] = fma(m, z.w, u[3]);
        u[4] = fma(k, z.x, u[4]);
        u[5] = fma(k, z.y, u[5]);
        u[6] = fma(k, z.z, u[6]);
        u[7] = fma(k, z.w, u[7]);
      }
      if (e < n1) {
        const int q = p0 + e;
        const double m = valM[q], k = valK[q];
        const double4_32a z = x[col[q]];
        t[0] = fma(m, z.x, t[0]);
        t[1] = fma(m, z.y, t[1]);
        t[2] = fma(m, z.z, t[2]);
        t[3] = fma(m, z.w, t[3]);
        t[4] = fma(k, z.x, t[4]);
        t[5] = fma(k, z.y, t[5]);
        t[6] = fma(k, z.z, t[6]);
        t[7] = fma(k, z.w, t[7]);
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && !two) break;
      const int w = h == 0 ? v : v2;
      const double* s8 = h == 0 ? u : t;  // m1p, m1n, m2p, m2n, k1p, k1n, k2p, k2n
      const double4_32a bb = b[w];
      double4_32a r;
      r.x = bb.x - fma(a, s8[6], s8[0]);
      r.y = bb.y - fma(a, s8[7], s8[1]);
      r.z = bb.z - fma(a, s8[4], -c * s8[2]);
      r.w = bb.w - fma(a, s8[5], -c * s8[3]);
      W[w] = r;
      acc[0] += bb.x * bb.x + bb.z * bb.z;
      acc[1] += bb.y * bb.y + bb.w * bb.w;
      acc[2] += r.x * r.x + r.z * r.z;
      acc[3] += r.y * r.y + r.w * r.w;
    }
  }
  block_sum<4>(acc, sm);
  if (threadIdx.x < 4) partials[(size_t)blockIdx.x * MAXV + threadIdx.x] = sm[threadIdx.x];
  KrylovDev* kd = kds + run;
  const int b0 = sg.first[run], b1 = sg.first[run + 1];
  __shared__ double tot[4];
  if (!reduce_run(sg, partials, &kd->ticket, b0, b1, 4, tot)) return;
  if (threadIdx.x < 2) {
    const int s = threadIdx.x;
    const double bn = sqrt(tot[s]), rn = sqrt(tot[2 + s]);
    if (init) {
      kd->bnorm[s] = bn;
      kd->tol[s] = rtol * bn;
      kd->its[s] = 0;
      kd->reorth_count[s] = 0;
      kd->active[s] = 1;
      if (s == 0) kd->nonfinite = 0;
    }
    __syncwarp(0x3u);
    if (!isfinite(bn) || !isfinite(rn)) kd->nonfinite = 1;
    kd->relres[s] = bn > 0.0 ? rn / bn : 0.0;
    const int act = kd->active[s] && rn > kd->tol[s] && bn > 0.0;
    kd->active[s] = act;
    kd->cycle_active[s] = act;
    kd->k[s] = 0;
    kd->beta[s] = rn;
    kd->g[s][0] = rn;
    kd->hinv[s] = (act && rn > 0.0) ? 1.0 / rn : 0.0;
  }
  if (threadIdx.x == 0) kd->ticket = 0;
}

// dst = src * hinv[s] per system of the block's run (components x,z: polymer; y,w: NFA)
__global__ void k_scale4(Seg sg, const double4_32a* src, double4_32a* dst, const KrylovDev* kds) {
  const KrylovDev* kd = kds + sg.run[blockIdx.x];
  const double s0 = kd->hinv[0], s1 = kd->hinv[1];
  for (int v = sg.lo[blockIdx.x] + threadIdx.x; v < sg.hi[blockIdx.x]; v += blockDim.x) {
    const double4_32a a = src[v];
    dst[v] = make_double4_32a(a.x * s0, a.y * s1, a.z * s0, a.w * s1);
  }
}

// ---------------------------------------------------------------- Gram-Schmidt passes
// Classical Gram-Schmidt twice (CGS2, gs_reorth = 0):
// MODE 0: h1[s][k] = <V_k, W>_s                       k = 0..nv-1
// MODE 1: W -= sum_k h1[s][k] V_k;  h2[s][k] = <V_k, W>_s
// MODE 2: W -= sum_k h2[s][k] V_k;  ||W||_s^2, then the Hessenberg / Givens update (last block)
// Selective reorthogonalisation (gs_reorth = 1; Daniel, Gragg, Kaufman and Stewart 1976): MODE 0
// with with_norm also records ||W||_s^2, then
// MODE 3: W -= sum_k h1[s][k] V_k;  ||W||_s^2; a species whose norm kept at least half its square
//         (||W'|| >= ||W|| / sqrt(2): little cancellation) takes h2 = 0 and its column now; the others
//         are flagged for the second pass
// MODE 4: h2[s][k] = <V_k, W>_s for the flagged species (0 for the others)
// MODE 5: W -= sum_k h2[s][k] V_k;  ||W||_s^2, the column of the flagged species
// Blocks of a run with no flagged species leave MODE 4 and 5 at entry.
// <a, b>_s sums components (x, z) for species 0 and (y, w) for species 1 over the run's nodes.
constexpr int KC = 16;                // basis vectors per chunk: 2 KC = 32 values, one per lane
constexpr int ORTH_BLOCKS = 152 * 2;  // target grid of the segmented kernels (2 blocks per SM)
// threads per block of the Gram-Schmidt passes; measured (ms per step, 512 x 512 FP64 / mixed /
// 64-run batch): 256 threads 14.1 / 6.75 / 37.3, 128 threads 14.1 / 6.71 / 38.5, 64 threads
// 14.5 / 7.07 / 44.4 -- more nodes per thread halve the reduction's share but expose more latency
constexpr int ORTH_TPB = 256;
static_assert(ORTH_TPB == TPB, "sum_rows assumes TPB threads in the reducing block");

// Sum V per-lane values (V a power of two, 2..32) over the warp by recursive halving: at each of the
// log2 V steps a lane keeps half of its values and adds the partner's copy of that half; plain xor
// adds then finish each group of 32 / V lanes.  On return lane l holds the warp sum of value
// l / (32 / V): V - 1 + 5 - log2 V shuffle-adds instead of 5 per value (32 values: 31 instead of
// 160).  Every warp-wide FP64 add holds the SM's FP64 pipe for the same time, so V is the smallest
// power of two that holds the values in use.
template <int V>
__device__ __forceinline__ double warp_transpose_sum(double (&a)[32]) {
  static_assert(V >= 2 && V <= 32 && (V & (V - 1)) == 0, "V: a power of two in [2, 32]");
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int step = 0; (1 << step) < V; ++step) {
    const int o = 16 >> step, h = V >> (step + 1);  // partner offset, values kept
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const double send = up ? a[k] : a[k + h];
      const double keep = up ? a[k + h] : a[k];
      a[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  double r = a[0];
#pragma unroll
  for (int o = 16 / V; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  return r;
}

// Block sum of the first V per-thread values over NT threads: returns, in threads 0..V-1, the block
// total of value t (the warps' sums added in warp order).
template <int NT, int V>
__device__ __forceinline__ double block_sum_v(double (&a)[32], double* sm /* [NT/32][V] */) {
  constexpr int G = 32 / V;  // lanes that end up holding the same value
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const double r = warp_transpose_sum<V>(a);
  if ((lane & (G - 1)) == 0) sm[w * V + lane / G] = r;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < V)
    for (int q = 0; q < NT / 32; ++q) t += sm[q * V + threadIdx.x];
  __syncthreads();
  return t;
}

// block_sum_v for the first nvals (1..32) values, V rounded up to a power of two (uniform branch)
template <int NT>
__device__ __forceinline__ double block_sum_n(int nvals, double (&a)[32], double* sm) {
  if (nvals <= 2) return block_sum_v<NT, 2>(a, sm);
  if (nvals <= 4) return block_sum_v<NT, 4>(a, sm);
  if (nvals <= 8) return block_sum_v<NT, 8>(a, sm);
  if (nvals <= 16) return block_sum_v<NT, 16>(a, sm);
  return block_sum_v<NT, 32>(a, sm);
}

// W[v] -= sum_{k < nv} c[s][k] V_k[v] for one node (two partial sums, even / odd k, halve the
// FP64 dependency chains)
__device__ __forceinline__ void orth_update_node(const double4_32a* __restrict__ V, double4_32a* __restrict__ W,
                                                 size_t N, int nv, const double (*coef)[MAXM + 1], int v) {
  double ax = 0, ay = 0, az = 0, aw = 0, bx = 0, by = 0, bz = 0, bw = 0;
  int k = 0;
  for (; k + 1 < nv; k += 2) {
    const double4_32a q0 = V[(size_t)k * N + v];
    const double4_32a q1 = V[(size_t)(k + 1) * N + v];
    const double c00 = coef[0][k], c10 = coef[1][k], c01 = coef[0][k + 1], c11 = coef[1][k + 1];
    ax = fma(c00, q0.x, ax); az = fma(c00, q0.z, az); ay = fma(c10, q0.y, ay); aw = fma(c10, q0.w, aw);
    bx = fma(c01, q1.x, bx); bz = fma(c01, q1.z, bz); by = fma(c11, q1.y, by); bw = fma(c11, q1.w, bw);
  }
  if (k < nv) {
    const double4_32a q0 = V[(size_t)k * N + v];
    ax = fma(coef[0][k], q0.x, ax); az = fma(coef[0][k], q0.z, az);
    ay = fma(coef[1][k], q0.y, ay); aw = fma(coef[1][k], q0.w, aw);
  }
  double4_32a w = W[v];
  w.x -= ax + bx;
  w.y -= ay + by;
  w.z -= az + bz;
  w.w -= aw + bw;
  W[v] = w;
}

// Dots of W with the KW basis vectors k0 .. k0+KW-1 over this thread's nodes, into acc[2t] (species
// 0) and acc[2t+1] (species 1).  KW is exact, so no FP64 slot is spent on absent vectors.  With
// UPD the node is first updated with all nv vectors (the same vectors are then re-read from L1).
template <int KW, bool UPD>
__device__ __forceinline__ void orth_dots_chunk(const double4_32a* __restrict__ V, double4_32a* __restrict__ W,
                                                size_t N, int k0, int nv, const double (*coef)[MAXM + 1],
                                                int v0, int v1, double (&acc)[32]) {
  for (int v = v0; v < v1; v += blockDim.x) {
    if (UPD) orth_update_node(V, W, N, nv, coef, v);
    const double4_32a w = W[v];
#pragma unroll
    for (int t = 0; t < KW; ++t) {
      const double4_32a q = V[(size_t)(k0 + t) * N + v];
      acc[2 * t] = fma(q.x, w.x, fma(q.z, w.z, acc[2 * t]));
      acc[2 * t + 1] = fma(q.y, w.y, fma(q.w, w.w, acc[2 * t + 1]));
    }
  }
}

template <bool UPD>
__device__ __forceinline__ void orth_dots_dispatch(int kw, const double4_32a* __restrict__ V,
                                                   double4_32a* __restrict__ W, size_t N, int k0, int nv,
                                                   const double (*coef)[MAXM + 1], int v0, int v1,
                                                   double (&acc)[32]) {
#define CH_ORTH_CASE(n) \
  case n: orth_dots_chunk<n, UPD>(V, W, N, k0, nv, coef, v0, v1, acc); break;
  switch (kw) {
    CH_ORTH_CASE(1) CH_ORTH_CASE(2) CH_ORTH_CASE(3) CH_ORTH_CASE(4) CH_ORTH_CASE(5) CH_ORTH_CASE(6)
    CH_ORTH_CASE(7) CH_ORTH_CASE(8) CH_ORTH_CASE(9) CH_ORTH_CASE(10) CH_ORTH_CASE(11) CH_ORTH_CASE(12)
    CH_ORTH_CASE(13) CH_ORTH_CASE(14) CH_ORTH_CASE(15) default: orth_dots_chunk<16, UPD>(V, W, N, k0, nv, coef, v0, v1, acc);
  }
#undef CH_ORTH_CASE
}

// Column j's inputs for both species, staged in shared memory by the whole block in one round of
// parallel loads, so that the thread applying the rotations issues no dependent global load (each
// cost it about a microsecond): h_k = h1_k + h2_k (the two Gram-Schmidt passes' coefficients; h1
// alone with only_h1), the previous rotations (cs_k, sn_k), k < j, and the species' scalars.
struct ColumnStage {
  double h[2][MAXM + 1];
  double cs[2][MAXM];
  double sn[2][MAXM];
  double g[2], tol[2];          // g_j and the tolerance of each species
  int its[2], active[2], rcount[2];  // iterations, cycle_active, reorth_count
};
__device__ __forceinline__ void stage_columns(const KrylovDev* kd, int j, bool only_h1, ColumnStage* cst) {
  for (int t = threadIdx.x; t < 2 * (j + 1); t += blockDim.x) {
    const int sp = t / (j + 1), k = t - sp * (j + 1);
    cst->h[sp][k] = only_h1 ? kd->h1[sp][k] : kd->h1[sp][k] + kd->h2[sp][k];
    if (k < j) {
      cst->cs[sp][k] = kd->cs[sp][k];
      cst->sn[sp][k] = kd->sn[sp][k];
    }
  }
  if (threadIdx.x >= 32 && threadIdx.x < 34) {  // the species' scalars, in the same round of loads
    const int sp = threadIdx.x - 32;
    cst->g[sp] = kd->g[sp][j];
    cst->tol[sp] = kd->tol[sp];
    cst->its[sp] = kd->its[sp];
    cst->active[sp] = kd->cycle_active[sp];
    cst->rcount[sp] = kd->reorth_count[sp];
  }
  __syncthreads();
}

// Column j of the Arnoldi process for species sp once w is orthogonal to V_0..V_j with squared norm
// hsq, from the staged h and rotations: h_{j+1} = ||w||, the previous Givens rotations, a new one, the
// residual estimate |g_{j+1}| and the cycle's stopping tests.
__device__ __forceinline__ void arnoldi_column(KrylovDev* kd, int sp, int j, double hsq, ColumnStage* cst) {
  double* h = cst->h[sp];
  const double hn = sqrt(hsq);
  double cur = h[0];  // entry k after the rotations 0..k-1
  for (int k = 0; k < j; ++k) {  // previous rotations
    const double c = cst->cs[sp][k], s = cst->sn[sp][k], nxt = h[k + 1];
    h[k] = c * cur + s * nxt;
    cur = -s * cur + c * nxt;
  }
  const double den = hypot(cur, hn);
  double cs = 1.0, sn = 0.0;
  if (den > 0.0) {
    cs = cur / den;
    sn = hn / den;
  }
  kd->cs[sp][j] = cs;
  kd->sn[sp][j] = sn;
  h[j] = den;
  for (int k = 0; k <= j; ++k) kd->R[sp][k][j] = h[k];
  const double gj = cst->g[sp], gj1 = -sn * gj;
  kd->g[sp][j + 1] = gj1;
  kd->g[sp][j] = cs * gj;
  kd->k[sp] = j + 1;
  kd->its[sp] = cst->its[sp] + 1;
  if (!isfinite(hn) || !isfinite(den)) kd->nonfinite = 1;
  const bool breakdown = !(hn > 1e-300);
  kd->hinv[sp] = breakdown ? 0.0 : 1.0 / hn;
  if (fabs(gj1) <= cst->tol[sp] || breakdown || den == 0.0) kd->cycle_active[sp] = 0;
}

template <int MODE>
__global__ void __launch_bounds__(ORTH_TPB, 2) k_orth(Seg sg, int N, int nv, const double4_32a* __restrict__ V,
                                               double4_32a* __restrict__ W, double* partials,
                                               KrylovDev* kds, int with_norm = 0) {
  constexpr bool DOTS = MODE == 0 || MODE == 1 || MODE == 4;
  __shared__ double sm[(ORTH_TPB / 32) * 32];
  __shared__ double coef[2][MAXM + 1];
  const int run = sg.run[blockIdx.x];
  KrylovDev* kd = kds + run;
  if (MODE >= 4 && !(kd->reorth[0] | kd->reorth[1])) return;  // the run needs no second pass
  const int v0 = sg.lo[blockIdx.x] + threadIdx.x, v1 = sg.hi[blockIdx.x];
  if (MODE == 1 || MODE == 2 || MODE == 3 || MODE == 5) {
    const bool first = MODE == 1 || MODE == 3;
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
      coef[0][k] = first ? kd->h1[0][k] : kd->h2[0][k];
      coef[1][k] = first ? kd->h1[1][k] : kd->h2[1][k];
    }
    __syncthreads();
  }
  if (MODE == 2 || MODE == 3 || MODE == 5) {
    for (int v = v0; v < v1; v += blockDim.x) orth_update_node(V, W, (size_t)N, nv, coef, v);
  }
  const int b0 = sg.first[run], b1 = sg.first[run + 1];
  if (DOTS) {
    for (int k0 = 0; k0 < nv; k0 += KC) {
      double acc[32];
#pragma unroll
      for (int t = 0; t < 32; ++t) acc[t] = 0.0;
      const int kw = nv - k0 < KC ? nv - k0 : KC;
      // MODE 1: the update of each node is fused into the first chunk's dots
      if (MODE == 1 && k0 == 0)
        orth_dots_dispatch<true>(kw, V, W, (size_t)N, k0, nv, coef, v0, v1, acc);
      else
        orth_dots_dispatch<false>(kw, V, W, (size_t)N, k0, nv, coef, v0, v1, acc);
      const double tot = block_sum_n<ORTH_TPB>(2 * kw, acc, sm);
      if (threadIdx.x < 2 * kw) partials[(size_t)blockIdx.x * MAXV + 2 * k0 + threadIdx.x] = tot;
    }
    const bool norm = MODE == 0 && with_norm;
    if (norm) {  // ||W||_s^2 before the projection, into the slots after the dots
      double acc[32];
#pragma unroll
      for (int t = 0; t < 32; ++t) acc[t] = 0.0;
      for (int v = v0; v < v1; v += blockDim.x) {
        const double4_32a w = W[v];
        acc[0] = fma(w.x, w.x, fma(w.z, w.z, acc[0]));
        acc[1] = fma(w.y, w.y, fma(w.w, w.w, acc[1]));
      }
      const double bt = block_sum_v<ORTH_TPB, 2>(acc, sm);
      if (threadIdx.x < 2) partials[(size_t)blockIdx.x * MAXV + 2 * nv + threadIdx.x] = bt;
    }
    __shared__ double tot[MAXV];
    if (!reduce_run(sg, partials, &kd->ticket, b0, b1, 2 * nv + (norm ? 2 : 0), tot)) return;
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
      double* dst0 = MODE == 0 ? kd->h1[0] : kd->h2[0];
      double* dst1 = MODE == 0 ? kd->h1[1] : kd->h2[1];
      dst0[k] = MODE == 4 && !kd->reorth[0] ? 0.0 : tot[2 * k];
      dst1[k] = MODE == 4 && !kd->reorth[1] ? 0.0 : tot[2 * k + 1];
    }
    if (norm && threadIdx.x < 2) kd->w2[threadIdx.x] = tot[2 * nv + threadIdx.x];
    if (threadIdx.x == 0) kd->ticket = 0;
  } else {
    double acc[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) acc[t] = 0.0;
    for (int v = v0; v < v1; v += blockDim.x) {
      const double4_32a w = W[v];
      acc[0] = fma(w.x, w.x, fma(w.z, w.z, acc[0]));
      acc[1] = fma(w.y, w.y, fma(w.w, w.w, acc[1]));
    }
    const double bt = block_sum_v<ORTH_TPB, 2>(acc, sm);
    if (threadIdx.x < 2) partials[(size_t)blockIdx.x * MAXV + threadIdx.x] = bt;
    __shared__ double tot[2];
    if (!reduce_run(sg, partials, &kd->ticket, b0, b1, 2, tot)) return;
    __shared__ ColumnStage cst;
    stage_columns(kd, nv - 1, MODE == 3, &cst);
    if (threadIdx.x < 2) {
      const int sp = threadIdx.x;
      if (MODE == 2) {
        if (cst.active[sp]) {
          arnoldi_column(kd, sp, nv - 1, tot[sp], &cst);
          kd->reorth_count[sp] = cst.rcount[sp] + 1;
        } else {
          kd->hinv[sp] = 0.0;
        }
      } else if (MODE == 3) {
        kd->reorth[sp] = 0;
        if (kd->cycle_active[sp]) {
          if (tot[sp] >= 0.5 * kd->w2[sp]) {
            for (int k = 0; k < nv; ++k) kd->h2[sp][k] = 0.0;
            arnoldi_column(kd, sp, nv - 1, tot[sp], &cst);
          } else {
            kd->reorth[sp] = 1;
          }
        } else {
          kd->hinv[sp] = 0.0;
        }
      } else if (kd->reorth[sp]) {  // MODE 5
        arnoldi_column(kd, sp, nv - 1, tot[sp], &cst);
        kd->reorth_count[sp] += 1;
      }
    }
    if (MODE == 5) {
      __syncthreads();
      if (threadIdx.x < 2) kd->reorth[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) kd->ticket = 0;
  }
}

// y_s = R_s^-1 g_s (back substitution, k_s x k_s), one warp per (run, species): the warp stages the
// triangle and g in shared memory (one round of independent loads), then for i = k-1 .. 0 the lanes
// form the products R[i][q] y[q], q > i, a butterfly adds them and every lane takes
// y[i] = (g[i] - sum) / R[i][i].  One thread walking the triangle in global memory waited on a
// load at every entry it read after a store (47 us at k = 11 in a cold capture).
__global__ void __launch_bounds__(32) k_cycle_solve(int nruns, KrylovDev* kds) {
  __shared__ double Rs[MAXM][MAXM + 1];
  __shared__ double gs[MAXM], ys[MAXM];
  if ((int)blockIdx.x >= 2 * nruns) return;
  KrylovDev* kd = kds + blockIdx.x / 2;
  const int s = blockIdx.x % 2, lane = threadIdx.x;
  const int k = kd->k[s];
  for (int e = lane; e < k * k; e += 32) {
    const int i = e / k, q = e - i * k;
    Rs[i][q] = kd->R[s][i][q];
  }
  for (int i = lane; i < k; i += 32) gs[i] = kd->g[s][i];
  __syncwarp();
  for (int i = k - 1; i >= 0; --i) {
    double p = 0.0;
    for (int q = i + 1 + lane; q < k; q += 32) p = fma(Rs[i][q], ys[q], p);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    const double rii = Rs[i][i];
    const double yi = rii != 0.0 ? (gs[i] - p) / rii : 0.0;
    if (lane == 0) ys[i] = yi;
    __syncwarp();
  }
  for (int i = lane; i < MAXM; i += 32) kd->y[s][i] = i < k ? ys[i] : 0.0;
}

// x += sum_k y_s[k] Z_k with the coefficients of the block's run, k < kmax (read from kmax_dev
// when it is given: the device-side loop knows the cycle's length only on the device)
__global__ void k_update_x(Seg sg, int N, int kmax_arg, const int* kmax_dev, const double4_32a* __restrict__ Z,
                           double4_32a* x, const KrylovDev* kds) {
  __shared__ double ny[2][MAXM + 1];  // -y: x - sum(-y_k Z_k) is x + sum(y_k Z_k) exactly
  const int kmax = kmax_dev ? *kmax_dev : kmax_arg;
  const KrylovDev* kd = kds + sg.run[blockIdx.x];
  for (int k = threadIdx.x; k < kmax; k += blockDim.x) {
    ny[0][k] = -kd->y[0][k];
    ny[1][k] = -kd->y[1][k];
  }
  __syncthreads();
  // two partial sums (even / odd k) and the basis vectors loaded in pairs, as in the Gram-Schmidt
  // update: a single FMA chain per component left the loads of one vector at a time in flight
  for (int v = sg.lo[blockIdx.x] + threadIdx.x; v < sg.hi[blockIdx.x]; v += blockDim.x)
    orth_update_node(Z, x, (size_t)N, kmax, ny, v);
}

// summary flags over all runs (one block)
__global__ void k_flags(int nruns, const KrylovDev* kds, Flags* f) {
  __shared__ int c[3];
  if (threadIdx.x < 3) c[threadIdx.x] = 0;
  __syncthreads();
  for (int r = threadIdx.x; r < nruns; r += blockDim.x) {
    const KrylovDev* kd = kds + r;
    atomicAdd(&c[0], kd->cycle_active[0] + kd->cycle_active[1]);
    atomicAdd(&c[1], kd->active[0] + kd->active[1]);
    atomicAdd(&c[2], kd->nonfinite);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    f->cycle_active = c[0];
    f->active = c[1];
    f->nonfinite = c[2];
  }
}

// ---------------------------------------------------------------- device-side solve loop
// With CUDA graphs on, FGMRES runs without the host: the step's graph holds a while node whose
// body is a switch over m + 1 cases -- case j < m is Arnoldi step j (case 0 first forms V_0 from
// the residual), case m ends a restart cycle (Givens solve, x update, true residual) -- followed
// by k_ctl, which reduces the flags of every run, advances this state and picks the next case.
// The loop ends when every system has converged, at max_iter, or at a non-finite value; its
// passes are bounded (each Arnoldi pass raises `total`, a cycle end follows at most m of them).
struct Ctl {
  int sel;        // case of the next body pass
  int total;      // Arnoldi steps taken in this solve
  int restarts;   // restart cycles completed
  int passes;     // body passes
  int status;     // ch_status of the solve
  int where;      // non-finite value met in: 0 the initial residual, 1 an Arnoldi step, 2 a cycle's residual
  int active;     // systems not converged when the loop stopped
  int jcycle;     // Arnoldi steps of the current cycle (the x update's length)
  int sum_j;      // jcycle summed over the completed cycles (launch accounting)
  int count[MAXM + 1];  // body passes per case
};

// init = 1: after the initial residual (resets the state); 0: after a body pass.  One block.
__global__ void k_ctl(int nruns, const KrylovDev* kds, Ctl* c, int m, int max_iter, int init,
                      cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hs) {
  __shared__ int cnt[3];
  if (threadIdx.x < 3) cnt[threadIdx.x] = 0;
  if (init)
    for (int k = threadIdx.x; k <= m; k += blockDim.x) c->count[k] = 0;
  __syncthreads();
  int ca = 0, ac = 0, nf = 0;
  for (int r = threadIdx.x; r < nruns; r += blockDim.x) {
    const KrylovDev* kd = kds + r;
    ca += kd->cycle_active[0] + kd->cycle_active[1];
    ac += kd->active[0] + kd->active[1];
    nf += kd->nonfinite;
  }
  if (ca) atomicAdd(&cnt[0], ca);
  if (ac) atomicAdd(&cnt[1], ac);
  if (nf) atomicAdd(&cnt[2], nf);
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int cycle_active = cnt[0], active = cnt[1], nonfinite = cnt[2];
  int go = 1, sel = 0;
  if (init) {
    c->total = 0;
    c->restarts = 0;
    c->passes = 0;
    c->sum_j = 0;
    c->jcycle = 0;
    c->where = 0;
    c->status = CH_OK;
    if (nonfinite) {
      c->status = CH_ERR_NONFINITE;
      go = 0;
    } else if (active == 0) {
      go = 0;
    } else if (max_iter <= 0) {
      c->status = CH_ERR_NOT_CONVERGED;
      go = 0;
    }
  } else {
    const int cur = c->sel;
    c->count[cur] += 1;
    c->passes += 1;
    if (cur < m) {  // Arnoldi step cur was taken
      c->total += 1;
      if (nonfinite) {
        c->status = CH_ERR_NONFINITE;
        c->where = 1;
        go = 0;
      } else if (cycle_active == 0 || c->total >= max_iter || cur + 1 == m) {
        c->jcycle = cur + 1;
        sel = m;
      } else {
        sel = cur + 1;
      }
    } else {  // a restart cycle ended with its true residual
      c->restarts += 1;
      c->sum_j += c->jcycle;
      if (nonfinite) {
        c->status = CH_ERR_NONFINITE;
        c->where = 2;
        go = 0;
      } else if (active == 0) {
        go = 0;
      } else if (c->total >= max_iter) {
        c->status = CH_ERR_NOT_CONVERGED;
        go = 0;
      }
    }
    if (go && c->passes > 2 * max_iter + 2) {  // cannot happen by the rules above; a backstop
      c->status = CH_ERR_INTERNAL;
      go = 0;
    }
  }
  c->active = active;
  c->sel = sel;
  cudaGraphSetConditional(hs, (unsigned)sel);
  cudaGraphSetConditional(hw, (unsigned)go);
}

// MINRES's control kernel (same record): case 0 starts the recurrence, cases 1 and 3 take an
// iteration (3 after retargeting), case 2 checks the true residual.  As in `minres`: iterate while
// some system's estimate is above its target, then check; stop when every system has converged,
// at max_iter or at a non-finite value.  Passes are bounded: every pass but a start or a check
// raises `total`, and a check follows at least one other pass.
__global__ void k_ctl_mr(int nruns, const KrylovDev* kds, Ctl* c, int max_iter, int init,
                         cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hs) {
  __shared__ int cnt[3];
  if (threadIdx.x < 3) cnt[threadIdx.x] = 0;
  if (init)
    for (int k = threadIdx.x; k < 4; k += blockDim.x) c->count[k] = 0;
  __syncthreads();
  int ca = 0, ac = 0, nf = 0;
  for (int r = threadIdx.x; r < nruns; r += blockDim.x) {
    const KrylovDev* kd = kds + r;
    ca += kd->cycle_active[0] + kd->cycle_active[1];
    ac += kd->active[0] + kd->active[1];
    nf += kd->nonfinite;
  }
  if (ca) atomicAdd(&cnt[0], ca);
  if (ac) atomicAdd(&cnt[1], ac);
  if (nf) atomicAdd(&cnt[2], nf);
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int cycle_active = cnt[0], active = cnt[1], nonfinite = cnt[2];
  int go = 1, sel = 0;
  auto iterate_or_check = [&]() {
    if (cycle_active > 0) {
      if (c->total >= max_iter) {
        c->status = CH_ERR_NOT_CONVERGED;
        go = 0;
      } else {
        sel = 1;
      }
    } else {
      sel = 2;
    }
  };
  if (init) {
    c->total = 0;
    c->restarts = 0;
    c->passes = 0;
    c->sum_j = 0;
    c->jcycle = 0;
    c->where = 0;
    c->status = CH_OK;
    if (nonfinite) {
      c->status = CH_ERR_NONFINITE;
      go = 0;
    } else if (active == 0) {
      go = 0;
    }
  } else {
    const int cur = c->sel;
    c->count[cur] += 1;
    c->passes += 1;
    if (cur == 0) {
      iterate_or_check();
    } else if (cur == 2) {
      if (nonfinite) {
        c->status = CH_ERR_NONFINITE;
        c->where = 2;
        go = 0;
      } else if (active == 0) {
        go = 0;
      } else if (c->total >= max_iter) {
        c->status = CH_ERR_NOT_CONVERGED;
        go = 0;
      } else {
        c->restarts += 1;
        sel = 3;
      }
    } else {
      c->total += 1;
      if (nonfinite) {
        c->status = CH_ERR_NONFINITE;
        c->where = 1;
        go = 0;
      } else {
        iterate_or_check();
      }
    }
    if (go && c->passes > 2 * max_iter + 4) {  // cannot happen by the rules above; a backstop
      c->status = CH_ERR_INTERNAL;
      go = 0;
    }
  }
  c->active = active;
  c->sel = sel;
  cudaGraphSetConditional(hs, (unsigned)sel);
  cudaGraphSetConditional(hw, (unsigned)go);
}

// mass_s = sum_i (M 1)_i phi_s,i  (M symmetric: 1^T M phi), per run
__global__ void k_mass(Seg sg, const double* mlump, const double4_32a* x, double* partials,
                       KrylovDev* kds) {
  __shared__ double sm[(TPB / 32) * 2];
  const int run = sg.run[blockIdx.x];
  double acc[2] = {0.0, 0.0};
  for (int v = sg.lo[blockIdx.x] + threadIdx.x; v < sg.hi[blockIdx.x]; v += blockDim.x) {
    const double4_32a a = x[v];
    acc[0] = fma(mlump[v], a.x, acc[0]);
    acc[1] = fma(mlump[v], a.y, acc[1]);
  }
  block_sum<2>(acc, sm);
  if (threadIdx.x < 2) partials[(size_t)blockIdx.x * MAXV + threadIdx.x] = sm[threadIdx.x];
  KrylovDev* kd = kds + run;
  const int b0 = sg.first[run], b1 = sg.first[run + 1];
  __shared__ double tot[2];
  if (!reduce_run(sg, partials, &kd->ticket, b0, b1, 2, tot)) return;
  if (threadIdx.x < 2) kd->mass[threadIdx.x] = tot[threadIdx.x];
  if (threadIdx.x == 0) kd->ticket = 0;
}

__global__ void k_rowsum(int N, const int* rowptr, const double* val, double* out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N) return;
  double s = 0.0;
  for (int q = rowptr[v]; q < rowptr[v + 1]; ++q) s += val[q];
  out[v] = s;
}

// per-run statistics gathered for the host after a step
struct RunStats {
  int its[2];
  int reorth[2];
  double relres[2];
  double mass[2];
  int warm[2];
};

__global__ void k_run_stats(int nruns, const KrylovDev* kds, RunStats* out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nruns) return;
  const KrylovDev* kd = kds + r;
  for (int s = 0; s < 2; ++s) {
    out[r].its[s] = kd->its[s];
    out[r].reorth[s] = kd->reorth_count[s];
    out[r].relres[s] = kd->relres[s];
    out[r].mass[s] = kd->mass[s];
    out[r].warm[s] = kd->warm[s];
  }
}

__global__ void k_clear_warm(int nruns, KrylovDev* kds) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nruns) kds[r].warm[0] = kds[r].warm[1] = 0;
}

// initial-guess selection: remember the residual of the previous state, then take the guess
// per (run, species) where its residual is smaller
__global__ void k_save_relres(int nruns, KrylovDev* kds) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nruns) return;
  kds[r].relres_prev[0] = kds[r].relres[0];
  kds[r].relres_prev[1] = kds[r].relres[1];
}

__global__ void k_pick_guess(Seg sg, const double4_32a* __restrict__ guess, double4_32a* x, KrylovDev* kds) {
  KrylovDev* kd = kds + sg.run[blockIdx.x];
  const bool tp = kd->relres[0] < kd->relres_prev[0], tn = kd->relres[1] < kd->relres_prev[1];
  if (blockIdx.x == sg.first[sg.run[blockIdx.x]] && threadIdx.x == 0) {
    kd->warm[0] = tp;
    kd->warm[1] = tn;
  }
  for (int v = sg.lo[blockIdx.x] + threadIdx.x; v < sg.hi[blockIdx.x]; v += blockDim.x) {
    const double4_32a g = guess[v];
    double4_32a a = x[v];
    if (tp) {
      a.x = g.x;
      a.z = g.z;
    }
    if (tn) {
      a.y = g.y;
      a.w = g.w;
    }
    x[v] = a;
  }
}

}  // namespace ch

// ---------------------------------------------------------------- state
struct ch_state_s {
  const ch_system_s* sys = nullptr;
  ch_precond_s* pc = nullptr;
  int N = 0, m = 0, R = 1;
  double* x = nullptr;  // N x 4: the state (phi_p, phi_n, mu_p, mu_n)
  double* b = nullptr;  // N x 4
  double* W = nullptr;  // N x 4
  double* V = nullptr;  // (m+1) x N x 4
  double* Z = nullptr;  // m x N x 4
  double* mlump = nullptr;
  double* partials = nullptr;
  ch::KrylovDev* kd = nullptr;  // R runs
  ch::Seg seg{};
  int nblocks = 0;
  ch::Flags* dflags = nullptr;
  ch::Flags* hflags = nullptr;  // pinned
  ch::RunStats* dstats = nullptr;
  std::vector<ch::RunStats> hstats;
  int last_status = 0, last_restarts = 0;
  float last_ms = 0.f;
  bool set = false;
  bool use_graphs = true;
  int since_set = 0;                // steps taken since the state was last set
  int learn_k = 0;                  // consecutive learned steps (x_prev valid when >= 1, x_prev2 when >= 2)
  double* x_prev = nullptr;         // N x 4: the state before the last learned step
  double* x_prev2 = nullptr;        // N x 4: the state before that
  double* guess = nullptr;          // N x 4: the network's prediction
  cudaStream_t cap_stream = nullptr;            // private stream for graph capture
  cudaStream_t body_stream = nullptr;           // nested captures of the device loop's body
  ch::MrDev* mr = nullptr;                      // MINRES scalars, one per run
  // device-side FGMRES loop (graphs on, per-launch timing off): one graph per plain step, and
  // the solve alone for steps with a caller's guess; built on first use
  ch::Ctl* dctl = nullptr;
  ch::Ctl* hctl = nullptr;                      // pinned copy, written by the graphs
  ch::RunStats* hstats_pin = nullptr;           // pinned, written by the step graph
  cudaGraph_t step_g = nullptr, solve_g = nullptr;
  cudaGraphExec_t step_graph = nullptr, solve_graph = nullptr;
  ch::ProfTally tally_step, tally_solve, tally_ctl, tally_case[ch::MAXM + 1];
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  ch::Alloc mem;
  ~ch_state_s() {
    if (step_graph) cudaGraphExecDestroy(step_graph);
    if (solve_graph) cudaGraphExecDestroy(solve_graph);
    if (step_g) cudaGraphDestroy(step_g);
    if (solve_g) cudaGraphDestroy(solve_g);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (body_stream) cudaStreamDestroy(body_stream);
    if (hflags) cudaFreeHost(hflags);
    if (hctl) cudaFreeHost(hctl);
    if (hstats_pin) cudaFreeHost(hstats_pin);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
  }
};

namespace ch {

// Split every run into blocks of about the same node count (at least one block per run); a
// single mesh gets about ORTH_BLOCKS blocks.
static ch_status make_segments(ch_state_s* S, cudaStream_t st) {
  const std::vector<int>& off = S->sys->mesh->run_off;
  const int R = S->R;
  const int64_t N = S->N;
  // Nodes per block: every block owns nodes of one run, so each run's count rounds up.  Take the
  // smallest size at which the rounded total still fits ORTH_BLOCKS (one wave of the segmented
  // kernels at two blocks per SM; a few blocks more made a second, nearly empty wave that left the
  // SMs ~30 % idle on the 64-run batch), or one block per run when there are more runs than that.
  auto blocks_at = [&](int64_t npb) {
    int64_t nb = 0;
    for (int r = 0; r < R; ++r) nb += std::max<int64_t>(1, (off[r + 1] - off[r] + npb - 1) / npb);
    return nb;
  };
  int64_t npb = std::max<int64_t>(TPB, (N + ORTH_BLOCKS - 1) / ORTH_BLOCKS);
  if (blocks_at(npb) > ORTH_BLOCKS) {
    int64_t lo_n = npb, hi_n = std::max<int64_t>(npb, N);  // blocks_at(hi_n) == R
    while (lo_n < hi_n) {
      const int64_t mid = lo_n + (hi_n - lo_n) / 2;
      if (blocks_at(mid) <= ORTH_BLOCKS) hi_n = mid;
      else lo_n = mid + 1;
    }
    npb = lo_n;
  }
  std::vector<int> run, lo, hi, first(R + 1, 0);
  for (int r = 0; r < R; ++r) {
    const int64_t n = off[r + 1] - off[r];
    const int nb = (int)std::max<int64_t>(1, (n + npb - 1) / npb);
    const int64_t chunk = (n + nb - 1) / nb;
    first[r] = (int)run.size();
    for (int b = 0; b < nb; ++b) {
      run.push_back(r);
      lo.push_back((int)std::min<int64_t>(off[r] + b * chunk, off[r + 1]));
      hi.push_back((int)std::min<int64_t>(off[r] + (b + 1) * chunk, off[r + 1]));
    }
  }
  first[R] = (int)run.size();
  S->nblocks = (int)run.size();
  int *d_run = nullptr, *d_lo = nullptr, *d_hi = nullptr, *d_first = nullptr;
  CH_TRY(S->mem.get(&d_run, run.size()));
  CH_TRY(S->mem.get(&d_lo, lo.size()));
  CH_TRY(S->mem.get(&d_hi, hi.size()));
  CH_TRY(S->mem.get(&d_first, first.size()));
  CH_CUDA(cudaMemcpyAsync(d_run, run.data(), sizeof(int) * run.size(), cudaMemcpyHostToDevice, st));
  CH_CUDA(cudaMemcpyAsync(d_lo, lo.data(), sizeof(int) * lo.size(), cudaMemcpyHostToDevice, st));
  CH_CUDA(cudaMemcpyAsync(d_hi, hi.data(), sizeof(int) * hi.size(), cudaMemcpyHostToDevice, st));
  CH_CUDA(cudaMemcpyAsync(d_first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice, st));
  unsigned int* d_gticket = nullptr;
  CH_TRY(S->mem.get(&d_gticket, run.size()));
  CH_CUDA(cudaMemsetAsync(d_gticket, 0, sizeof(unsigned int) * run.size(), st));
  CH_CUDA(cudaStreamSynchronize(st));
  S->seg = Seg{d_run, d_lo, d_hi, d_first, d_gticket, S->nblocks};
  return CH_OK;
}

ch_status state_create(const ch_system_s* s, ch_precond_s* pc, cudaStream_t st, ch_state_s** out) {
  const int m = s->p.restart;
  if (m < 1 || m > MAXM) {
    set_error("restart must be in [1, %d]", MAXM);
    return CH_ERR_ARG;
  }
  if (s->p.krylov == 1 && m < 5) {
    set_error("MINRES keeps its 8 work vectors in the Krylov basis storage: restart must be >= 5");
    return CH_ERR_ARG;
  }
  ch_state_s* S = new ch_state_s();
  S->sys = s;
  S->pc = pc;
  S->N = s->N;
  S->m = m;
  S->R = (int)s->mesh->runs.size();
  S->hstats.resize(S->R);
  const size_t n4 = (size_t)s->N * 4;
  ch_status r = CH_OK;
  if (r == CH_OK) r = S->mem.get(&S->x, n4);
  if (r == CH_OK) r = S->mem.get(&S->b, n4);
  if (r == CH_OK) r = S->mem.get(&S->W, n4);
  if (r == CH_OK) r = S->mem.get(&S->V, n4 * (m + 1));
  if (r == CH_OK) r = S->mem.get(&S->Z, n4 * m);
  if (r == CH_OK) r = S->mem.get(&S->mlump, (size_t)s->N);
  if (r == CH_OK) r = S->mem.get(&S->kd, (size_t)S->R);
  if (r == CH_OK) r = S->mem.get(&S->mr, (size_t)S->R);
  if (r == CH_OK) r = S->mem.get(&S->dflags, 1);
  if (r == CH_OK) r = S->mem.get(&S->dstats, (size_t)S->R);
  if (r == CH_OK) r = S->mem.get(&S->dctl, 1);
  if (r == CH_OK) r = make_segments(S, st);
  if (r == CH_OK) r = S->mem.get(&S->partials, 2 * (size_t)S->nblocks * MAXV);  // block rows, group rows
  auto pinned = [&](void** ptr, size_t bytes) {
    if (r != CH_OK) return;
    if (cudaMallocHost(ptr, bytes) != cudaSuccess) {
      *ptr = nullptr;
      cudaGetLastError();
      set_error("pinned allocation of %zu bytes failed", bytes);
      r = CH_ERR_OOM;
    }
  };
  pinned(reinterpret_cast<void**>(&S->hflags), sizeof(Flags));
  pinned(reinterpret_cast<void**>(&S->hctl), sizeof(Ctl));
  pinned(reinterpret_cast<void**>(&S->hstats_pin), sizeof(RunStats) * S->R);
  S->use_graphs = s->p.graphs != 0;
  if (r == CH_OK && (cudaStreamCreateWithFlags(&S->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
                     cudaStreamCreateWithFlags(&S->body_stream, cudaStreamNonBlocking) != cudaSuccess)) {
    set_error("stream creation failed");
    r = CH_ERR_CUDA;
  }
  if (r == CH_OK && (cudaEventCreate(&S->ev0) != cudaSuccess || cudaEventCreate(&S->ev1) != cudaSuccess)) {
    set_error("event creation failed");
    r = CH_ERR_CUDA;
  }
  if (r == CH_OK) {
    cudaMemsetAsync(S->kd, 0, sizeof(KrylovDev) * S->R, st);
    cudaMemsetAsync(S->x, 0, n4 * sizeof(double), st);
    k_rowsum<<<blocks_for(s->N), TPB, 0, st>>>(s->N, s->rowptr, s->valM, S->mlump);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
      set_error("state initialisation failed");
      r = CH_ERR_CUDA;
    }
  }
  if (r != CH_OK) {
    delete S;
    return r;
  }
  *out = S;
  return CH_OK;
}

void state_destroy(ch_state_s* S) { delete S; }

static ch_status read_flags(ch_state_s* S, cudaStream_t st) {
  {
    ProfScope ps(st, K_FLAGS, 0, 0.0, 0.0);
    k_flags<<<1, 256, 0, st>>>(S->R, S->kd, S->dflags);
  }
  CH_LAUNCHED();
  CH_CUDA(cudaMemcpyAsync(S->hflags, S->dflags, sizeof(Flags), cudaMemcpyDeviceToHost, st));
  CH_CUDA(cudaStreamSynchronize(st));
  prof_drain();
  return CH_OK;
}

static double res4_bytes(const ch_system_s* s) { return 20.0 * s->nnz + 4.0 * (s->N + 1) + 96.0 * s->N; }

// One Arnoldi step j for all systems: Z_j = Prec(V_j) (Algorithm 1), W = A Z_j, CGS2 against
// V_0..V_j with the Givens update and V_{j+1} = W / h_{j+1,j}.  Everything is enqueued on `st`
// with no host synchronisation, so it can be captured.
static ch_status arnoldi_step(ch_state_s* S, int j, cudaStream_t st) {
  const ch_system_s* s = S->sys;
  const int N = S->N, nb = S->nblocks;
  double4_32a* W4 = reinterpret_cast<double4_32a*>(S->W);
  double4_32a* V4 = reinterpret_cast<double4_32a*>(S->V);
  double4_32a* Z4 = reinterpret_cast<double4_32a*>(S->Z);
  double4_32a* Vj = V4 + (size_t)j * N;
  double4_32a* Zj = Z4 + (size_t)j * N;
  CH_TRY(precond_apply(S->pc, reinterpret_cast<double*>(Vj), reinterpret_cast<double*>(Zj), st));
  CH_TRY(apply_A(s, reinterpret_cast<double*>(Zj), S->W, st));
  const double nv = j + 1, n32 = 32.0 * N;
  if (s->p.gs_reorth) {  // selective reorthogonalisation: the second pass only where it is needed
    {
      ProfScope ps(st, K_ORTH0, 0, (nv + 2) * n32, 4.0 * nv * N + 4.0 * N);
      k_orth<0><<<nb, ORTH_TPB, 0, st>>>(S->seg, N, j + 1, V4, W4, S->partials, S->kd, 1);
    }
    {
      ProfScope ps(st, K_ORTH2, 0, (nv + 2) * n32, 4.0 * nv * N + 4.0 * N);
      k_orth<3><<<nb, ORTH_TPB, 0, st>>>(S->seg, N, j + 1, V4, W4, S->partials, S->kd);
    }
    // the second pass's launches (its bytes count as if every run took it)
    {
      ProfScope ps(st, K_ORTH_RE, 0, (nv + 1) * n32, 4.0 * nv * N);
      k_orth<4><<<nb, ORTH_TPB, 0, st>>>(S->seg, N, j + 1, V4, W4, S->partials, S->kd);
    }
    {
      ProfScope ps(st, K_ORTH_RE, 0, (nv + 2) * n32, 4.0 * nv * N + 4.0 * N);
      k_orth<5><<<nb, ORTH_TPB, 0, st>>>(S->seg, N, j + 1, V4, W4, S->partials, S->kd);
    }
  } else {
    {
      ProfScope ps(st, K_ORTH0, 0, (nv + 1) * n32, 4.0 * nv * N);
      k_orth<0><<<nb, ORTH_TPB, 0, st>>>(S->seg, N, j + 1, V4, W4, S->partials, S->kd);
    }
    {
      ProfScope ps(st, K_ORTH1, 0, (nv + 2) * n32, 8.0 * nv * N);
      k_orth<1><<<nb, ORTH_TPB, 0, st>>>(S->seg, N, j + 1, V4, W4, S->partials, S->kd);
    }
    {
      ProfScope ps(st, K_ORTH2, 0, (nv + 2) * n32, 4.0 * nv * N + 4.0 * N);
      k_orth<2><<<nb, ORTH_TPB, 0, st>>>(S->seg, N, j + 1, V4, W4, S->partials, S->kd);
    }
  }
  {
    ProfScope ps(st, K_SCALE4, 0, 64.0 * N, 0.0);
    k_scale4<<<nb, TPB, 0, st>>>(S->seg, W4, V4 + (size_t)(j + 1) * N, S->kd);
  }
  CH_LAUNCHED();
  return CH_OK;
}

// Host-driven Arnoldi step (graphs off, or per-launch event timing on): the step's kernels, the
// summary flags, and a read of the flags.
static ch_status arnoldi_launch(ch_state_s* S, int j, cudaStream_t st) {
  CH_TRY(arnoldi_step(S, j, st));
  return read_flags(S, st);
}

static ch_status residual_launch(ch_state_s* S, int init, cudaStream_t st, const double* x = nullptr) {
  const ch_system_s* s = S->sys;
  ProfScope ps(st, K_RESIDUAL4, 0, res4_bytes(s), 8.0 * s->nnz + 12.0 * S->N);
  k_residual4<<<S->nblocks, TPB, 0, st>>>(S->seg, s->rowptr, s->col, s->valM, s->valK, s->a, s->c,
                                           reinterpret_cast<const double4_32a*>(x ? x : S->x),
                                           reinterpret_cast<const double4_32a*>(S->b),
                                           reinterpret_cast<double4_32a*>(S->W), S->partials, S->kd,
                                           init, s->p.rtol);
  CH_LAUNCHED();
  return CH_OK;
}

// Solve A x = b for all systems; x holds the initial guess on entry.
static ch_status fgmres(ch_state_s* S, cudaStream_t st, int* restarts) {
  const ch_params& p = S->sys->p;
  const int N = S->N, m = S->m, nb = S->nblocks;
  double4_32a* x4 = reinterpret_cast<double4_32a*>(S->x);
  double4_32a* W4 = reinterpret_cast<double4_32a*>(S->W);
  double4_32a* V4 = reinterpret_cast<double4_32a*>(S->V);
  double4_32a* Z4 = reinterpret_cast<double4_32a*>(S->Z);
  CH_TRY(residual_launch(S, 1, st));
  CH_TRY(read_flags(S, st));
  if (S->hflags->nonfinite) {
    set_error("non-finite right-hand side or initial residual");
    return CH_ERR_NONFINITE;
  }
  int total = 0;
  *restarts = 0;
  while (S->hflags->active > 0) {
    if (total >= p.max_iter) {
      set_error("FGMRES reached max_iter = %d with %d of %d systems unconverged", p.max_iter,
                S->hflags->active, 2 * S->R);
      return CH_ERR_NOT_CONVERGED;
    }
    {
      ProfScope ps(st, K_SCALE4, 0, 64.0 * N, 0.0);
      k_scale4<<<nb, TPB, 0, st>>>(S->seg, W4, V4, S->kd);  // V_0 = r / beta
    }
    CH_LAUNCHED();
    int j = 0;
    for (; j < m; ++j) {
      ++total;
      CH_TRY(arnoldi_launch(S, j, st));
      if (S->hflags->nonfinite) {
        set_error("non-finite value in the Arnoldi process");
        return CH_ERR_NONFINITE;
      }
      if (S->hflags->cycle_active == 0 || total >= p.max_iter) {
        ++j;
        break;
      }
    }
    if (j > m) j = m;
    {
      ProfScope ps(st, K_CYCLE_SOLVE, 0, 0.0, 0.0);
      k_cycle_solve<<<2 * S->R, 32, 0, st>>>(S->R, S->kd);
    }
    {
      ProfScope ps(st, K_UPDATE_X, 0, (j + 2) * 32.0 * N, 4.0 * j * N);
      k_update_x<<<nb, TPB, 0, st>>>(S->seg, N, j, nullptr, Z4, x4, S->kd);
    }
    CH_LAUNCHED();
    CH_TRY(residual_launch(S, 0, st));
    CH_TRY(read_flags(S, st));
    if (S->hflags->nonfinite) {
      set_error("non-finite residual");
      return CH_ERR_NONFINITE;
    }
    ++*restarts;
  }
  return CH_OK;
}

// ---------------------------------------------------------------- preconditioned MINRES
// The paper's Krylov method (Section 3): Lanczos vectors v_j (A-space) and z_j = P^-1 v_j, both
// normalised by gamma_j = sqrt(v_j . z_j); the tridiagonal matrix (delta_j on the diagonal,
// gamma_j off it) is reduced by Givens rotations, and x is updated by the direction w_{j+1}.
// MODE 0: gamma_1 from (v_1, z_1) and the start of the recurrence; 1: delta_j = (A z_j) . z_j;
// 2: gamma_{j+1} from (v_{j+1}, z_{j+1}) and the Givens step.  Dots per species: components
// (x, z) for species 0 and (y, w) for species 1, over the run's nodes, reduced in a fixed order.
template <int MODE>
__global__ void __launch_bounds__(TPB) k_mr_dot(Seg sg, const double4_32a* __restrict__ A_,
                                                const double4_32a* __restrict__ B_, double* partials,
                                                KrylovDev* kds, MrDev* mrs) {
  __shared__ double sm[(TPB / 32) * 2];
  const int run = sg.run[blockIdx.x];
  double acc[2] = {0.0, 0.0};
  for (int v = sg.lo[blockIdx.x] + threadIdx.x; v < sg.hi[blockIdx.x]; v += blockDim.x) {
    const double4_32a a = A_[v], b = B_[v];
    acc[0] = fma(a.x, b.x, fma(a.z, b.z, acc[0]));
    acc[1] = fma(a.y, b.y, fma(a.w, b.w, acc[1]));
  }
  block_sum<2>(acc, sm);
  if (threadIdx.x < 2) partials[(size_t)blockIdx.x * MAXV + threadIdx.x] = sm[threadIdx.x];
  KrylovDev* kd = kds + run;
  MrDev* mr = mrs + run;
  const int b0 = sg.first[run], b1 = sg.first[run + 1];
  __shared__ double tot[2];
  if (!reduce_run(sg, partials, &kd->ticket, b0, b1, 2, tot)) return;
  if (threadIdx.x < 2) {
    const int sp = threadIdx.x;
    const double d = tot[sp];
    if (!isfinite(d)) kd->nonfinite = 1;
    if (MODE == 0) {
      const bool go = kd->active[sp] && d > 0.0;
      const double g = go ? sqrt(d) : 0.0;
      mr->gam[sp] = g;
      mr->eta[sp] = g;
      mr->c[sp] = mr->cp[sp] = 1.0;
      mr->s[sp] = mr->sp[sp] = 0.0;
      // the preconditioned residual is to fall by the factor the true one must fall by
      mr->est[sp] = (go && kd->beta[sp] > 0.0) ? g * kd->tol[sp] / kd->beta[sp] : 0.0;
      mr->scale[sp] = go ? 1.0 / g : 0.0;
      kd->cycle_active[sp] = go;
    } else if (MODE == 1) {
      mr->delta[sp] = d;
    } else {
      mr->upd[sp] = kd->cycle_active[sp];
      if (kd->cycle_active[sp]) {
        const double gn = d > 0.0 ? sqrt(d) : 0.0;
        const double g = mr->gam[sp], dl = mr->delta[sp];
        const double a0 = mr->c[sp] * dl - mr->cp[sp] * mr->s[sp] * g;
        const double a1 = hypot(a0, gn);
        mr->a2[sp] = mr->s[sp] * dl + mr->cp[sp] * mr->c[sp] * g;
        mr->a3[sp] = mr->sp[sp] * g;
        mr->a1[sp] = a1;
        const double cn = a1 > 0.0 ? a0 / a1 : 1.0, sn = a1 > 0.0 ? gn / a1 : 0.0;
        mr->cn[sp] = cn;
        mr->etao[sp] = mr->eta[sp];
        mr->eta[sp] = -sn * mr->eta[sp];
        mr->cp[sp] = mr->c[sp];
        mr->c[sp] = cn;
        mr->sp[sp] = mr->s[sp];
        mr->s[sp] = sn;
        mr->gam[sp] = gn;
        const bool breakdown = !(gn > 1e-300) || !(a1 > 0.0);
        mr->scale[sp] = breakdown ? 0.0 : 1.0 / gn;
        if (!(a1 > 0.0)) mr->upd[sp] = 0;
        kd->its[sp] += 1;
        if (!isfinite(a1) || !isfinite(mr->eta[sp])) kd->nonfinite = 1;
        kd->cycle_active[sp] = !breakdown && fabs(mr->eta[sp]) > mr->est[sp];
      }
    }
  }
  if (threadIdx.x == 0) kd->ticket = 0;
}

// v *= 1 / gamma_1, z *= 1 / gamma_1 (start of the recurrence)
__global__ void k_mr_scale(Seg sg, double4_32a* v, double4_32a* z, const MrDev* mrs) {
  const MrDev* mr = mrs + sg.run[blockIdx.x];
  const double f0 = mr->scale[0], f1 = mr->scale[1];
  for (int i = sg.lo[blockIdx.x] + threadIdx.x; i < sg.hi[blockIdx.x]; i += blockDim.x) {
    double4_32a a = v[i], b = z[i];
    a.x *= f0; a.z *= f0; a.y *= f1; a.w *= f1;
    b.x *= f0; b.z *= f0; b.y *= f1; b.w *= f1;
    v[i] = a;
    z[i] = b;
  }
}

// v_{j+1} = A z_j - delta_j v_j - gamma_j v_{j-1} (zero for a species that has stopped)
__global__ void k_mr_lanczos(Seg sg, const double4_32a* __restrict__ q, const double4_32a* __restrict__ v,
                             const double4_32a* __restrict__ vp, double4_32a* __restrict__ vn,
                             const KrylovDev* kds, const MrDev* mrs) {
  const int run = sg.run[blockIdx.x];
  const KrylovDev* kd = kds + run;
  const MrDev* mr = mrs + run;
  const bool on0 = kd->cycle_active[0], on1 = kd->cycle_active[1];
  const double d0 = mr->delta[0], d1 = mr->delta[1], g0 = mr->gam[0], g1 = mr->gam[1];
  for (int i = sg.lo[blockIdx.x] + threadIdx.x; i < sg.hi[blockIdx.x]; i += blockDim.x) {
    const double4_32a a = q[i], b = v[i], c = vp[i];
    double4_32a o;
    o.x = on0 ? a.x - d0 * b.x - g0 * c.x : 0.0;
    o.z = on0 ? a.z - d0 * b.z - g0 * c.z : 0.0;
    o.y = on1 ? a.y - d1 * b.y - g1 * c.y : 0.0;
    o.w = on1 ? a.w - d1 * b.w - g1 * c.w : 0.0;
    vn[i] = o;
  }
}

// w_{j+1} = (z_j - a3 w_{j-1} - a2 w_j) / a1;  x += c_{j+1} eta_j w_{j+1};  then the roles move on:
// w_{j-1} <- w_j, w_j <- w_{j+1}, v_{j-1} <- v_j, v_j <- v_{j+1} / gamma_{j+1}, z_j <- z_{j+1} / gamma_{j+1}
__global__ void k_mr_update(Seg sg, double4_32a* __restrict__ x, double4_32a* __restrict__ w,
                            double4_32a* __restrict__ wp, double4_32a* __restrict__ z,
                            const double4_32a* __restrict__ zn, double4_32a* __restrict__ v,
                            double4_32a* __restrict__ vp, const double4_32a* __restrict__ vn,
                            const MrDev* mrs) {
  const MrDev* mr = mrs + sg.run[blockIdx.x];
  const bool u0 = mr->upd[0], u1 = mr->upd[1];
  const double i0 = u0 ? 1.0 / mr->a1[0] : 0.0, i1 = u1 ? 1.0 / mr->a1[1] : 0.0;
  const double a20 = mr->a2[0], a21 = mr->a2[1], a30 = mr->a3[0], a31 = mr->a3[1];
  const double f0 = mr->cn[0] * mr->etao[0], f1 = mr->cn[1] * mr->etao[1];
  const double s0 = mr->scale[0], s1 = mr->scale[1];
  for (int i = sg.lo[blockIdx.x] + threadIdx.x; i < sg.hi[blockIdx.x]; i += blockDim.x) {
    // a species that did not take this iteration keeps its vectors (it may resume after a
    // true-residual check)
    const double4_32a zz = z[i], ww = w[i], wwp = wp[i], vv = v[i], vnn = vn[i], znn = zn[i];
    double4_32a xx = x[i], wo = ww, wpo = wwp, vo = vv, vpo = vp[i], zo = zz;
    if (u0) {
      const double wx = (zz.x - a30 * wwp.x - a20 * ww.x) * i0;
      const double wz = (zz.z - a30 * wwp.z - a20 * ww.z) * i0;
      xx.x += f0 * wx;
      xx.z += f0 * wz;
      wpo.x = ww.x; wpo.z = ww.z;
      wo.x = wx; wo.z = wz;
      vpo.x = vv.x; vpo.z = vv.z;
      vo.x = vnn.x * s0; vo.z = vnn.z * s0;
      zo.x = znn.x * s0; zo.z = znn.z * s0;
    }
    if (u1) {
      const double wy = (zz.y - a31 * wwp.y - a21 * ww.y) * i1;
      const double ww_ = (zz.w - a31 * wwp.w - a21 * ww.w) * i1;
      xx.y += f1 * wy;
      xx.w += f1 * ww_;
      wpo.y = ww.y; wpo.w = ww.w;
      wo.y = wy; wo.w = ww_;
      vpo.y = vv.y; vpo.w = vv.w;
      vo.y = vnn.y * s1; vo.w = vnn.w * s1;
      zo.y = znn.y * s1; zo.w = znn.w * s1;
    }
    x[i] = xx;
    wp[i] = wpo;
    w[i] = wo;
    vp[i] = vpo;
    v[i] = vo;
    z[i] = zo;
  }
}

// after a true-residual check, species still unconverged aim their estimate lower: by the
// factor their true residual still has to fall (at least 2)
__global__ void k_mr_retarget(int nruns, const KrylovDev* kds, MrDev* mrs) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * nruns) return;
  const KrylovDev* kd = kds + t / 2;
  MrDev* mr = mrs + t / 2;
  const int sp = t % 2;
  if (!kd->active[sp]) return;
  const double rn = kd->relres[sp] * kd->bnorm[sp];
  const double f = rn > 0.0 ? fmin(0.5, 0.9 * kd->tol[sp] / rn) : 0.5;
  mr->est[sp] = fabs(mr->eta[sp]) * f;
}

// One MINRES iteration for all runs and species.  Work vectors (N x 4 each) live in the Krylov
// basis storage: V_0 v_j, V_1 v_{j-1}, V_2 v_{j+1}, V_3 w_j, V_4 w_{j-1}, V_5 A z_j; Z_0 z_j, Z_1 z_{j+1}.
static ch_status mr_iteration(ch_state_s* S, cudaStream_t st) {
  const int N = S->N, nb = S->nblocks;
  const size_t n4 = (size_t)N;
  double4_32a* V4 = reinterpret_cast<double4_32a*>(S->V);
  double4_32a* Z4 = reinterpret_cast<double4_32a*>(S->Z);
  double4_32a *v = V4, *vp = V4 + n4, *vn = V4 + 2 * n4, *w = V4 + 3 * n4, *wp = V4 + 4 * n4, *q = V4 + 5 * n4;
  double4_32a *z = Z4, *zn = Z4 + n4;
  CH_TRY(apply_A(S->sys, reinterpret_cast<const double*>(z), reinterpret_cast<double*>(q), st));
  {
    ProfScope ps(st, K_MR_DOT, 0, 64.0 * N, 4.0 * N);
    k_mr_dot<1><<<nb, TPB, 0, st>>>(S->seg, q, z, S->partials, S->kd, S->mr);
  }
  {
    ProfScope ps(st, K_MR_VEC, 0, 128.0 * N, 8.0 * N);
    k_mr_lanczos<<<nb, TPB, 0, st>>>(S->seg, q, v, vp, vn, S->kd, S->mr);
  }
  CH_LAUNCHED();
  CH_TRY(precond_apply(S->pc, reinterpret_cast<const double*>(vn), reinterpret_cast<double*>(zn), st));
  {
    ProfScope ps(st, K_MR_DOT, 0, 64.0 * N, 4.0 * N);
    k_mr_dot<2><<<nb, TPB, 0, st>>>(S->seg, vn, zn, S->partials, S->kd, S->mr);
  }
  {
    ProfScope ps(st, K_MR_VEC, 0, 10.0 * 32.0 * N, 12.0 * N);
    k_mr_update<<<nb, TPB, 0, st>>>(S->seg, reinterpret_cast<double4_32a*>(S->x), w, wp, z, zn, v, vp, vn, S->mr);
  }
  CH_LAUNCHED();
  return CH_OK;
}

static ch_status mr_iteration_flags(ch_state_s* S, cudaStream_t st) {
  CH_TRY(mr_iteration(S, st));
  {
    ProfScope ps(st, K_FLAGS, 0, 0.0, 0.0);
    k_flags<<<1, 256, 0, st>>>(S->R, S->kd, S->dflags);
  }
  CH_LAUNCHED();
  return CH_OK;
}

// The start of the recurrence: v_1 = r_0, z_1 = P^-1 v_1, v_0 = w_0 = w_{-1} = 0, gamma_1.
static ch_status mr_start(ch_state_s* S, cudaStream_t st) {
  const int N = S->N, nb = S->nblocks;
  const size_t n4 = (size_t)N;
  double4_32a* V4 = reinterpret_cast<double4_32a*>(S->V);
  double4_32a* Z4 = reinterpret_cast<double4_32a*>(S->Z);
  CH_CUDA(cudaMemcpyAsync(V4, S->W, sizeof(double4_32a) * n4, cudaMemcpyDeviceToDevice, st));
  CH_CUDA(cudaMemsetAsync(V4 + n4, 0, sizeof(double4_32a) * n4, st));
  CH_CUDA(cudaMemsetAsync(V4 + 3 * n4, 0, sizeof(double4_32a) * 2 * n4, st));
  CH_TRY(precond_apply(S->pc, reinterpret_cast<const double*>(V4), reinterpret_cast<double*>(Z4), st));
  {
    ProfScope ps(st, K_MR_DOT, 0, 64.0 * N, 4.0 * N);
    k_mr_dot<0><<<nb, TPB, 0, st>>>(S->seg, V4, Z4, S->partials, S->kd, S->mr);
  }
  {
    ProfScope ps(st, K_MR_VEC, 0, 128.0 * N, 4.0 * N);
    k_mr_scale<<<nb, TPB, 0, st>>>(S->seg, V4, Z4, S->mr);
  }
  CH_LAUNCHED();
  return CH_OK;
}

// Host-driven MINRES iteration (graphs off, or per-launch event timing on): the iteration, the
// summary flags, and a read of the flags.
static ch_status mr_launch(ch_state_s* S, cudaStream_t st) {
  CH_TRY(mr_iteration_flags(S, st));
  return read_flags(S, st);
}

// Preconditioned MINRES (the paper's Krylov method, Section 3) with Algorithm 1 as the fixed
// preconditioner; the stopping test is the true FP64 residual, checked whenever every system's
// MINRES estimate has reached its target (checks[0] counts the checks after the first).
static ch_status minres(ch_state_s* S, cudaStream_t st, int* checks) {
  const ch_params& p = S->sys->p;
  *checks = 0;
  CH_TRY(residual_launch(S, 1, st));
  CH_TRY(read_flags(S, st));
  if (S->hflags->nonfinite) {
    set_error("non-finite right-hand side or initial residual");
    return CH_ERR_NONFINITE;
  }
  if (S->hflags->active == 0) return CH_OK;
  CH_TRY(mr_start(S, st));
  CH_TRY(read_flags(S, st));
  int total = 0;
  for (;;) {
    while (S->hflags->cycle_active > 0) {
      if (total >= p.max_iter) {
        set_error("MINRES reached max_iter = %d with %d of %d systems unconverged", p.max_iter,
                  S->hflags->active, 2 * S->R);
        return CH_ERR_NOT_CONVERGED;
      }
      CH_TRY(mr_launch(S, st));
      ++total;
      if (S->hflags->nonfinite) {
        set_error("non-finite value in the MINRES recurrence");
        return CH_ERR_NONFINITE;
      }
    }
    CH_TRY(residual_launch(S, 0, st));
    CH_TRY(read_flags(S, st));
    if (S->hflags->nonfinite) {
      set_error("non-finite residual");
      return CH_ERR_NONFINITE;
    }
    if (S->hflags->active == 0) return CH_OK;
    if (total >= p.max_iter) {
      set_error("MINRES reached max_iter = %d with %d of %d systems unconverged", p.max_iter,
                S->hflags->active, 2 * S->R);
      return CH_ERR_NOT_CONVERGED;
    }
    k_mr_retarget<<<blocks_for(2 * S->R, 64), 64, 0, st>>>(S->R, S->kd, S->mr);
    CH_LAUNCHED();
    ++*checks;
  }
}

static ch_status krylov_solve(ch_state_s* S, cudaStream_t st, int* restarts) {
  return S->sys->p.krylov == 1 ? minres(S, st, restarts) : fgmres(S, st, restarts);
}

// ---------------------------------------------------------------- the Krylov loop on the device
// The loops of `fgmres` and `minres` as one CUDA graph (see Ctl): no host synchronisation inside
// a solve.
static bool device_loop(const ch_state_s* S) { return S->use_graphs && !prof_timing(); }

static bool is_minres(const ch_state_s* S) { return S->sys->p.krylov == 1; }

// MINRES's cases: 0 the start of the recurrence, 1 an iteration, 2 the true-residual check,
// 3 the retargeting of unconverged species followed by an iteration.
static ch_status mr_case(ch_state_s* S, int c, cudaStream_t st) {
  switch (c) {
    case 0:
      return mr_start(S, st);
    case 1:
      return mr_iteration(S, st);
    case 2:
      return residual_launch(S, 0, st);
    default:
      k_mr_retarget<<<blocks_for(2 * S->R, 64), 64, 0, st>>>(S->R, S->kd, S->mr);
      CH_LAUNCHED();
      return mr_iteration(S, st);
  }
}

// Case j < m of the loop body: Arnoldi step j (case 0 first forms V_0 = r / beta); case m: the
// end of a restart cycle (y = R^-1 g, x += Z y over the cycle's steps, the true residual).
static ch_status loop_case(ch_state_s* S, int j, cudaStream_t st) {
  const int N = S->N, nb = S->nblocks;
  double4_32a* W4 = reinterpret_cast<double4_32a*>(S->W);
  double4_32a* V4 = reinterpret_cast<double4_32a*>(S->V);
  if (j < S->m) {
    if (j == 0) {
      ProfScope ps(st, K_SCALE4, 0, 64.0 * N, 0.0);
      k_scale4<<<nb, TPB, 0, st>>>(S->seg, W4, V4, S->kd);
    }
    CH_LAUNCHED();
    return arnoldi_step(S, j, st);
  }
  {
    ProfScope ps(st, K_CYCLE_SOLVE, 0, 0.0, 0.0);
    k_cycle_solve<<<2 * S->R, 32, 0, st>>>(S->R, S->kd);
  }
  {
    // bytes of the x update beyond x itself (32 N per Krylov vector) are added per cycle from
    // the loop's record (Ctl::sum_j), the length being known on the device only
    ProfScope ps(st, K_UPDATE_X, 0, 2 * 32.0 * N, 0.0);
    k_update_x<<<nb, TPB, 0, st>>>(S->seg, N, S->m, &S->dctl->jcycle, reinterpret_cast<const double4_32a*>(S->Z),
                                    reinterpret_cast<double4_32a*>(S->x), S->kd);
  }
  CH_LAUNCHED();
  return residual_launch(S, 0, st);
}

// Capture `fill` into the graph `g` on the body stream, after the nodes deps[0..nd).
template <typename F>
static ch_status capture_into(ch_state_s* S, cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd, F fill) {
  cudaStream_t bs = S->body_stream;
  CH_CUDA(cudaStreamBeginCaptureToGraph(bs, g, deps, nullptr, nd, cudaStreamCaptureModeThreadLocal));
  const ch_status r = fill(bs);
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(bs, &out);
  CH_TRY(r);
  CH_CUDA(e);
  return CH_OK;
}

// Enqueue the whole solve on the capturing stream cs: the initial residual, k_ctl, and the while
// node with its body.  Launch accounting: the initial residual and k_ctl go to the tally that is
// current on entry, case j to tally_case[j], the body's k_ctl to tally_ctl.
static ch_status capture_solve(ch_state_s* S, cudaStream_t cs) {
  const int m = S->m, max_iter = S->sys->p.max_iter;
  const bool mr = is_minres(S);
  const int ncases = mr ? 4 : m + 1;
  auto ctl = [&](cudaStream_t st, int init, cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hs) {
    if (mr)
      k_ctl_mr<<<1, 256, 0, st>>>(S->R, S->kd, S->dctl, max_iter, init, hw, hs);
    else
      k_ctl<<<1, 256, 0, st>>>(S->R, S->kd, S->dctl, m, max_iter, init, hw, hs);
  };
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  CH_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, nullptr, nullptr, nullptr));
  cudaGraphConditionalHandle hw, hs;
  CH_CUDA(cudaGraphConditionalHandleCreate(&hw, g, 0, 0));
  CH_CUDA(cudaGraphConditionalHandleCreate(&hs, g, 0, 0));
  CH_TRY(residual_launch(S, 1, cs));
  {
    ProfScope ps(cs, K_FLAGS, 0, 0.0, 0.0);
    ctl(cs, 1, hw, hs);
  }
  CH_LAUNCHED();
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CH_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphNodeParams wp = {};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wn = nullptr;
  CH_CUDA(cudaGraphAddNode(&wn, g, deps, nullptr, nd, &wp));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  cudaGraphNodeParams sp = {};
  sp.type = cudaGraphNodeTypeConditional;
  sp.conditional.handle = hs;
  sp.conditional.type = cudaGraphCondTypeSwitch;
  sp.conditional.size = (unsigned)ncases;
  cudaGraphNode_t sn = nullptr;
  CH_CUDA(cudaGraphAddNode(&sn, body, nullptr, nullptr, 0, &sp));
  ProfTally* outer = prof_capture_swap(nullptr);
  ch_status r = CH_OK;
  for (int j = 0; j < ncases && r == CH_OK; ++j) {
    S->tally_case[j] = ProfTally();
    prof_capture_swap(&S->tally_case[j]);
    r = capture_into(S, sp.conditional.phGraph_out[j], nullptr, 0,
                     [&](cudaStream_t bs) { return mr ? mr_case(S, j, bs) : loop_case(S, j, bs); });
  }
  if (r == CH_OK) {
    S->tally_ctl = ProfTally();
    prof_capture_swap(&S->tally_ctl);
    r = capture_into(S, body, &sn, 1, [&](cudaStream_t bs) -> ch_status {
      ProfScope ps(bs, K_FLAGS, 0, 0.0, 0.0);
      ctl(bs, 0, hw, hs);
      CH_LAUNCHED();
      return CH_OK;
    });
  }
  prof_capture_swap(outer);
  CH_TRY(r);
  CH_CUDA(cudaStreamUpdateCaptureDependencies(cs, &wn, nullptr, 1, cudaStreamSetCaptureDependencies));
  return CH_OK;
}

// Build the graph of a whole plain step (whole = true: right-hand sides, solve, masses, run
// statistics, and the copies of the statistics and the loop record to pinned host memory) or of
// the solve alone (the loop record copied out).
static ch_status build_loop_graph(ch_state_s* S, bool whole, cudaGraph_t* gout, cudaGraphExec_t* xout,
                                  ProfTally* tally) {
  cudaGraph_t G = nullptr;
  CH_CUDA(cudaGraphCreate(&G, 0));
  cudaStream_t cs = S->cap_stream;
  cudaError_t e = cudaStreamBeginCaptureToGraph(cs, G, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(G);
    CH_CUDA(e);
  }
  *tally = ProfTally();
  ProfTally* prev = prof_capture_swap(tally);
  ch_status r = CH_OK;
  if (whole) {
    r = rhs_strided(S->sys, S->x, S->x + 1, 4, S->b, cs);
    if (r == CH_OK) {
      k_clear_warm<<<blocks_for(S->R, 64), 64, 0, cs>>>(S->R, S->kd);
      if (cudaGetLastError() != cudaSuccess) r = CH_ERR_CUDA;
    }
  }
  if (r == CH_OK) r = capture_solve(S, cs);
  if (r == CH_OK && whole) {
    {
      ProfScope ps(cs, K_MASS, 0, 40.0 * S->N, 2.0 * S->N);
      k_mass<<<S->nblocks, TPB, 0, cs>>>(S->seg, S->mlump, reinterpret_cast<const double4_32a*>(S->x),
                                          S->partials, S->kd);
    }
    k_run_stats<<<blocks_for(S->R, 64), 64, 0, cs>>>(S->R, S->kd, S->dstats);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(S->hstats_pin, S->dstats, sizeof(RunStats) * S->R, cudaMemcpyDeviceToHost, cs) !=
            cudaSuccess)
      r = CH_ERR_CUDA;
  }
  if (r == CH_OK && cudaMemcpyAsync(S->hctl, S->dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, cs) != cudaSuccess)
    r = CH_ERR_CUDA;
  prof_capture_swap(prev);
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(cs, &captured);
  if (r == CH_ERR_CUDA) set_error("capturing the device-side FGMRES loop failed: %s", cudaGetErrorString(cudaGetLastError()));
  if (r == CH_OK && e != cudaSuccess) {
    set_error("capturing the device-side FGMRES loop failed: %s", cudaGetErrorString(e));
    r = CH_ERR_CUDA;
  }
  if (r == CH_OK) {
    e = cudaGraphInstantiate(xout, G, 0);
    if (e != cudaSuccess) {
      set_error("instantiating the device-side FGMRES loop failed: %s", cudaGetErrorString(e));
      *xout = nullptr;
      r = CH_ERR_CUDA;
    }
  }
  if (r != CH_OK) {
    cudaGetLastError();
    cudaGraphDestroy(G);
    return r;
  }
  *gout = G;  // kept until the state goes (a graph with conditional nodes has one instantiation)
  return CH_OK;
}

// After the loop's graph has completed (stream synchronised): launch accounting of the passes
// taken and the solve's status from the loop record.
static ch_status finish_loop(ch_state_s* S, const ProfTally& pro, int* restarts) {
  const Ctl& c = *S->hctl;
  prof_add(pro);
  const bool mr = is_minres(S);
  for (int j = 0; j < (mr ? 4 : S->m + 1); ++j) prof_add_times(S->tally_case[j], c.count[j]);
  prof_add_times(S->tally_ctl, c.passes);
  prof_add_slot(K_UPDATE_X, 0, 0, 32.0 * S->N * c.sum_j, 4.0 * S->N * c.sum_j);
  *restarts = c.restarts;
  switch (c.status) {
    case CH_OK:
      return CH_OK;
    case CH_ERR_NONFINITE:
      set_error(c.where == 0   ? "non-finite right-hand side or initial residual"
                : c.where == 1 ? (mr ? "non-finite value in the MINRES recurrence"
                                     : "non-finite value in the Arnoldi process")
                               : "non-finite residual");
      return CH_ERR_NONFINITE;
    case CH_ERR_NOT_CONVERGED:
      set_error("%s reached max_iter = %d with %d of %d systems unconverged", mr ? "MINRES" : "FGMRES",
                S->sys->p.max_iter, c.active, 2 * S->R);
      return CH_ERR_NOT_CONVERGED;
    default:
      set_error("the device-side Krylov loop stopped at its pass limit (%d passes)", c.passes);
      return CH_ERR_INTERNAL;
  }
}


__global__ void k_set_state(int N, const double* pp, const double* pn, const double* mp,
                            const double* mn, double4_32a* x) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N) return;
  x[v] = make_double4_32a(pp[v], pn[v], mp ? mp[v] : 0.0, mn ? mn[v] : 0.0);
}

__global__ void k_get_state(int N, const double4_32a* x, double* pp, double* pn, double* ps, double* mp,
                            double* mn) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N) return;
  const double4_32a a = x[v];
  if (pp) pp[v] = a.x;
  if (pn) pn[v] = a.y;
  if (ps) ps[v] = 1.0 - a.x - a.y;  // Eq. (2)
  if (mp) mp[v] = a.z;
  if (mn) mn[v] = a.w;
}

// SplitMix64 (Steele, Lea, Flood 2014) on the counter seed_r ^ (field << 40) ^ local node index,
// seed_r = seed + r for run r
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__global__ void k_seeded(int N, const int* node_run, const int* run_off, const double* base_p,
                         const double* base_n, double noise, uint64_t seed, double4_32a* x) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N) return;
  const int r = node_run[v];
  const uint64_t sr = seed + (uint64_t)r, loc = (uint64_t)(v - run_off[r]);
  const double up = (double)(splitmix64(sr ^ (0ULL << 40) ^ loc) >> 11) * 0x1.0p-53;
  const double un = (double)(splitmix64(sr ^ (1ULL << 40) ^ loc) >> 11) * 0x1.0p-53;
  // base + noise (2u - 1) with every operation rounded on its own (no FMA contraction), as the
  // host generator computes it
  const double tp = __dmul_rn(noise, __dsub_rn(__dmul_rn(2.0, up), 1.0));
  const double tn = __dmul_rn(noise, __dsub_rn(__dmul_rn(2.0, un), 1.0));
  x[v] = make_double4_32a(__dadd_rn(base_p[r], tp), __dadd_rn(base_n[r], tn), 0.0, 0.0);
}

ch_status state_set(ch_state_s* S, const double* pp, const double* pn, const double* mp,
                    const double* mn, cudaStream_t st) {
  ProfScope prof_io(st, K_STATE_IO, 0, 72.0 * S->N, 0.0);
  k_set_state<<<blocks_for(S->N), TPB, 0, st>>>(S->N, pp, pn, mp, mn,
                                                 reinterpret_cast<double4_32a*>(S->x));
  CH_LAUNCHED();
  S->set = true;
  S->since_set = S->learn_k = 0;
  return CH_OK;
}

ch_status state_seeded_batch(ch_state_s* S, const double* base_p, const double* base_n, double noise,
                             uint64_t seed, cudaStream_t st) {
  const int R = S->R;
  double* d = nullptr;
  Alloc tmp;
  CH_TRY(tmp.get(&d, 2 * (size_t)R));
  CH_CUDA(cudaMemcpyAsync(d, base_p, sizeof(double) * R, cudaMemcpyHostToDevice, st));
  CH_CUDA(cudaMemcpyAsync(d + R, base_n, sizeof(double) * R, cudaMemcpyHostToDevice, st));
  {
    ProfScope prof_io(st, K_STATE_IO, 0, 72.0 * S->N, 0.0);
    k_seeded<<<blocks_for(S->N), TPB, 0, st>>>(S->N, S->sys->mesh->node_run, S->sys->mesh->run_off_d,
                                                d, d + R, noise, seed,
                                                reinterpret_cast<double4_32a*>(S->x));
  }
  CH_LAUNCHED();
  CH_CUDA(cudaStreamSynchronize(st));
  S->set = true;
  S->since_set = S->learn_k = 0;
  return CH_OK;
}

ch_status state_seeded(ch_state_s* S, double p0, double n0, double noise, uint64_t seed,
                       cudaStream_t st) {
  std::vector<double> bp(S->R, p0), bn(S->R, n0);
  return state_seeded_batch(S, bp.data(), bn.data(), noise, seed, st);
}

// ---------------------------------------------------------------- checkpoint / resume
// File: 8-byte magic "CHSTATE1", int64 N, int64 runs, then the N x 4 FP64 state (phi_p, phi_n,
// mu_p, mu_n per node, node-major), little-endian as the host writes it.
static const char kStateMagic[8] = {'C', 'H', 'S', 'T', 'A', 'T', 'E', '1'};

ch_status state_save(const ch_state_s* S, const char* path, cudaStream_t st) {
  if (!S->set) {
    set_error("state not initialised: nothing to save");
    return CH_ERR_STATE;
  }
  std::vector<double> h((size_t)S->N * 4);
  CH_CUDA(cudaMemcpyAsync(h.data(), S->x, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
  CH_CUDA(cudaStreamSynchronize(st));
  FILE* f = fopen(path, "wb");
  if (!f) {
    set_error("cannot open %s for writing", path);
    return CH_ERR_ARG;
  }
  const int64_t hdr[2] = {S->N, S->R};
  bool ok = fwrite(kStateMagic, 1, 8, f) == 8 && fwrite(hdr, sizeof(int64_t), 2, f) == 2 &&
            fwrite(h.data(), sizeof(double), h.size(), f) == h.size();
  ok = (fclose(f) == 0) && ok;
  if (!ok) {
    set_error("writing %s failed", path);
    return CH_ERR_ARG;
  }
  return CH_OK;
}

ch_status state_load(ch_state_s* S, const char* path, cudaStream_t st) {
  FILE* f = fopen(path, "rb");
  if (!f) {
    set_error("cannot open %s", path);
    return CH_ERR_ARG;
  }
  char magic[8] = {};
  int64_t hdr[2] = {0, 0};
  std::vector<double> h((size_t)S->N * 4);
  const bool head = fread(magic, 1, 8, f) == 8 && fread(hdr, sizeof(int64_t), 2, f) == 2;
  if (!head || memcmp(magic, kStateMagic, 8) != 0) {
    fclose(f);
    set_error("%s is not a state file", path);
    return CH_ERR_ARG;
  }
  if (hdr[0] != S->N || hdr[1] != S->R) {
    fclose(f);
    set_error("%s holds %lld nodes in %lld runs; this state has %d nodes in %d runs", path, (long long)hdr[0],
              (long long)hdr[1], S->N, S->R);
    return CH_ERR_ARG;
  }
  const bool body = fread(h.data(), sizeof(double), h.size(), f) == h.size();
  fclose(f);
  if (!body) {
    set_error("%s is truncated", path);
    return CH_ERR_ARG;
  }
  CH_CUDA(cudaMemcpyAsync(S->x, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, st));
  CH_CUDA(cudaStreamSynchronize(st));
  S->set = true;
  S->since_set = S->learn_k = 0;
  return CH_OK;
}

ch_status state_get(const ch_state_s* S, double* pp, double* pn, double* ps, double* mp, double* mn,
                    cudaStream_t st) {
  ProfScope prof_io(st, K_STATE_IO, 0, 72.0 * S->N, 0.0);
  k_get_state<<<blocks_for(S->N), TPB, 0, st>>>(S->N, reinterpret_cast<const double4_32a*>(S->x), pp,
                                                 pn, ps, mp, mn);
  CH_LAUNCHED();
  return CH_OK;
}

static void fill_stats(const ch_state_s* S, int run, ch_step_stats* o) {
  const RunStats& rs = S->hstats[run];
  o->iters[0] = rs.its[0];
  o->iters[1] = rs.its[1];
  o->restarts = S->last_restarts;
  o->status = S->last_status;
  o->relres[0] = rs.relres[0];
  o->relres[1] = rs.relres[1];
  o->mass[0] = rs.mass[0];
  o->mass[1] = rs.mass[1];
  o->ms = S->last_ms;
  o->warm[0] = rs.warm[0];
  o->warm[1] = rs.warm[1];
  o->reorth[0] = rs.reorth[0];
  o->reorth[1] = rs.reorth[1];
}

// The end of a step: the run statistics are in the host copy, the CUDA events recorded.
static ch_status step_done(ch_state_s* S, ch_status r, int restarts, ch_step_stats* stats) {
  cudaEventElapsedTime(&S->last_ms, S->ev0, S->ev1);
  S->last_status = r;
  S->last_restarts = restarts;
  S->since_set += 1;
  if (stats) fill_stats(S, 0, stats);
  return r;
}

// One step from the previous state; rec0: record the start event here (else the caller did).
static ch_status step_plain_core(ch_state_s* S, cudaStream_t st, ch_step_stats* stats, bool rec0) {
  if (rec0) CH_CUDA(cudaEventRecord(S->ev0, st));
  if (device_loop(S)) {  // the whole step is one graph launch and one synchronisation
    if (!S->step_graph) CH_TRY(build_loop_graph(S, true, &S->step_g, &S->step_graph, &S->tally_step));
    CH_CUDA(cudaGraphLaunch(S->step_graph, st));
    CH_CUDA(cudaEventRecord(S->ev1, st));
    CH_CUDA(cudaStreamSynchronize(st));
    std::memcpy(S->hstats.data(), S->hstats_pin, sizeof(RunStats) * S->R);
    int restarts = 0;
    const ch_status r = finish_loop(S, S->tally_step, &restarts);
    return step_done(S, r, restarts, stats);
  }
  // right-hand sides from phi^k (strided views of the state)
  CH_TRY(rhs_strided(S->sys, S->x, S->x + 1, 4, S->b, st));
  k_clear_warm<<<blocks_for(S->R, 64), 64, 0, st>>>(S->R, S->kd);
  int restarts = 0;
  ch_status r = krylov_solve(S, st, &restarts);
  {
    ProfScope ps(st, K_MASS, 0, 40.0 * S->N, 2.0 * S->N);
    k_mass<<<S->nblocks, TPB, 0, st>>>(S->seg, S->mlump, reinterpret_cast<const double4_32a*>(S->x),
                                        S->partials, S->kd);
  }
  k_run_stats<<<blocks_for(S->R, 64), 64, 0, st>>>(S->R, S->kd, S->dstats);
  CH_LAUNCHED();
  CH_CUDA(cudaEventRecord(S->ev1, st));
  CH_CUDA(cudaMemcpyAsync(S->hstats_pin, S->dstats, sizeof(RunStats) * S->R, cudaMemcpyDeviceToHost, st));
  CH_CUDA(cudaStreamSynchronize(st));
  std::memcpy(S->hstats.data(), S->hstats_pin, sizeof(RunStats) * S->R);
  return step_done(S, r, restarts, stats);
}

ch_status state_step(ch_state_s* S, cudaStream_t st, ch_step_stats* stats) {
  if (!S->set) {
    set_error("state not initialised (call ch_state_set or ch_state_init_seeded)");
    return CH_ERR_STATE;
  }
  S->learn_k = 0;
  return step_plain_core(S, st, stats, true);
}

// A step whose initial guess is, per (run, species), the caller's guess when its true residual
// ||b - A guess|| is smaller than that of the previous state, else the previous state.
static ch_status step_guess_core(ch_state_s* S, const double* guess, cudaStream_t st, ch_step_stats* stats,
                                 bool rec0) {
  if (rec0) CH_CUDA(cudaEventRecord(S->ev0, st));
  CH_TRY(rhs_strided(S->sys, S->x, S->x + 1, 4, S->b, st));
  CH_TRY(residual_launch(S, 1, st));  // previous state
  {
    ProfScope ps(st, K_GUESS, 0, 0.0, 0.0);
    k_save_relres<<<blocks_for(S->R, 64), 64, 0, st>>>(S->R, S->kd);
  }
  CH_TRY(residual_launch(S, 1, st, guess));
  {
    ProfScope ps(st, K_GUESS, 0, 96.0 * S->N, 0.0);
    k_pick_guess<<<S->nblocks, TPB, 0, st>>>(S->seg, reinterpret_cast<const double4_32a*>(guess),
                                              reinterpret_cast<double4_32a*>(S->x), S->kd);
  }
  CH_LAUNCHED();
  int restarts = 0;
  const bool dev = device_loop(S);
  ch_status r = CH_OK;
  if (dev) {  // the solve is one graph launch; its status is read after the synchronisation
    if (!S->solve_graph) CH_TRY(build_loop_graph(S, false, &S->solve_g, &S->solve_graph, &S->tally_solve));
    CH_CUDA(cudaGraphLaunch(S->solve_graph, st));
  } else {
    r = krylov_solve(S, st, &restarts);
  }
  {
    ProfScope ps(st, K_MASS, 0, 40.0 * S->N, 2.0 * S->N);
    k_mass<<<S->nblocks, TPB, 0, st>>>(S->seg, S->mlump, reinterpret_cast<const double4_32a*>(S->x),
                                        S->partials, S->kd);
  }
  k_run_stats<<<blocks_for(S->R, 64), 64, 0, st>>>(S->R, S->kd, S->dstats);
  CH_LAUNCHED();
  CH_CUDA(cudaEventRecord(S->ev1, st));
  CH_CUDA(cudaMemcpyAsync(S->hstats_pin, S->dstats, sizeof(RunStats) * S->R, cudaMemcpyDeviceToHost, st));
  CH_CUDA(cudaStreamSynchronize(st));
  std::memcpy(S->hstats.data(), S->hstats_pin, sizeof(RunStats) * S->R);
  if (dev) r = finish_loop(S, S->tally_solve, &restarts);
  return step_done(S, r, restarts, stats);
}

ch_status state_step_guess(ch_state_s* S, const double* guess, cudaStream_t st, ch_step_stats* stats) {
  if (!S->set) {
    set_error("state not initialised (call ch_state_set or ch_state_init_seeded)");
    return CH_ERR_STATE;
  }
  S->learn_k = 0;
  return step_guess_core(S, guess, st, stats, true);
}

// A step whose guess is the warm-start network's prediction from the state and its two
// predecessors (kept on the device across consecutive learned steps).  The network needs
// predecessors that are not the initial state (whose chemical potentials the first step sets up):
// until three steps have been taken since the state was set, and until two learned steps in a row
// have recorded the history, the step starts from the previous state.  ms in the statistics
// includes the prediction.
ch_status state_step_learned(ch_state_s* S, ch_ws_s* w, cudaStream_t st, ch_step_stats* stats) {
  if (!S->set) {
    set_error("state not initialised (call ch_state_set or ch_state_init_seeded)");
    return CH_ERR_STATE;
  }
  int H = 0, W = 0;
  ws_dims(w, &H, &W);
  const ch_params& mp = S->sys->mesh->p;
  if (S->R != 1 || mp.dim != 2 || W != mp.nx + 1 || H != mp.ny + 1) {
    set_error("the warm-start network's image is %d x %d; the state must be one 2D run of %d x %d nodes",
              H, W, H, W);
    return CH_ERR_ARG;
  }
  if (!S->x_prev) {
    CH_TRY(S->mem.get(&S->x_prev, (size_t)S->N * 4));
    CH_TRY(S->mem.get(&S->x_prev2, (size_t)S->N * 4));
    CH_TRY(S->mem.get(&S->guess, (size_t)S->N * 4));
  }
  const bool use_net = S->learn_k >= 2 && S->since_set >= 3;
  CH_CUDA(cudaEventRecord(S->ev0, st));
  if (use_net) CH_TRY(ws_predict(w, S->x, S->x_prev, S->x_prev2, S->guess, st));
  std::swap(S->x_prev, S->x_prev2);  // the history moves on: s_{k-1} becomes s_{k-2}, s_k becomes s_{k-1}
  {
    ProfScope ps(st, K_STATE_IO, 0, 64.0 * S->N, 0.0);
    CH_CUDA(cudaMemcpyAsync(S->x_prev, S->x, sizeof(double) * 4 * S->N, cudaMemcpyDeviceToDevice, st));
  }
  const ch_status r = use_net ? step_guess_core(S, S->guess, st, stats, false)
                              : step_plain_core(S, st, stats, false);
  S->learn_k += 1;
  if (r == CH_OK && use_net) return ws_check(w);  // the step synchronised: its prediction is done
  return r;
}



ch_status state_run_stats(const ch_state_s* S, int run, ch_step_stats* out) {
  if (run < 0 || run >= S->R) {
    set_error("run %d out of range [0, %d)", run, S->R);
    return CH_ERR_ARG;
  }
  fill_stats(S, run, out);
  return CH_OK;
}


}  // namespace ch
