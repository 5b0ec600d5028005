// Internal declarations shared by the CUDA translation units of libch.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ch.h"

namespace ch {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);

#define CH_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      ::ch::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return e_ == cudaErrorMemoryAllocation ? CH_ERR_OOM : CH_ERR_CUDA;                   \
    }                                                                                      \
  } while (0)

#define CH_LAUNCHED() CH_CUDA(cudaGetLastError())

#define CH_TRY(call)                \
  do {                              \
    ch_status s_ = (call);          \
    if (s_ != CH_OK) return s_;     \
  } while (0)

#define CH_ARG(cond, msg)                                        \
  do {                                                           \
    if (!(cond)) {                                               \
      ::ch::set_error("invalid argument: %s", msg);              \
      return CH_ERR_ARG;                                         \
    }                                                            \
  } while (0)

// ---------------------------------------------------------------- device memory owned by a handle
struct Alloc {
  std::vector<void*> ptrs;
  Alloc() = default;
  Alloc(const Alloc&) = delete;
  Alloc& operator=(const Alloc&) = delete;
  ~Alloc() { release(); }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
  template <typename T>
  ch_status get(T** out, size_t n) {
    *out = nullptr;
    if (n == 0) n = 1;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? CH_ERR_OOM : CH_ERR_CUDA;
    }
    ptrs.push_back(p);
    *out = static_cast<T*>(p);
    return CH_OK;
  }
  void forget(void* p) {  // free one allocation early
    for (size_t i = 0; i < ptrs.size(); ++i)
      if (ptrs[i] == p) {
        cudaFree(p);
        ptrs[i] = ptrs.back();
        ptrs.pop_back();
        return;
      }
  }
};

// ---------------------------------------------------------------- sparse matrices
template <typename T>
struct Csr {
  int nrows = 0, ncols = 0;
  int64_t nnz = 0;
  int* rowptr = nullptr;
  int* col = nullptr;
  T* val = nullptr;
};

constexpr int TPB = 256;  // threads per block of the plain node-parallel kernels
inline int blocks_for(int64_t n, int tpb = TPB) { return (int)((n + tpb - 1) / tpb); }
// fixed grid for deterministic grid-stride reductions: a multiple of the 152 SMs
constexpr int RED_BLOCKS_MAX = 152 * 4;
inline int red_blocks(int64_t n) {
  int b = blocks_for(n);
  return b < RED_BLOCKS_MAX ? (b < 1 ? 1 : b) : RED_BLOCKS_MAX;
}

// ---------------------------------------------------------------- programmatic dependent launch
// A kernel launched with `pdl` set may be scheduled while the kernel before it on the stream is
// still running (its blocks wait in pdl_wait() until that kernel has finished and its writes are
// visible).  The rules every such kernel keeps:
//   - before pdl_wait() it reads only data that no kernel of the current solve writes (operator
//     values, diagonals: set-up results) and writes no global memory;
//   - it calls pdl_trigger(), which lets its own successor be scheduled, only after pdl_wait(), so
//     that when the successor's blocks start every kernel but this one has finished.  Without the
//     call the successor is scheduled when this kernel's blocks have all exited (still before
//     the memory flush that pdl_wait() covers).
// Launched without the attribute (pdl = 0, per-launch timing with events between kernels) both
// instructions return at once and the kernel behaves as a plain launch.  No arithmetic changes.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

bool prof_timing();  // prof.cu: per-launch event timing on (launches then stay plain)
template <typename... KArgs, typename... Args>
inline void launch_k(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args&&... args) {
  if (!pdl || prof_timing()) {
    k<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
    return;
  }
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  (void)cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);  // errors reach cudaGetLastError
}

// ---------------------------------------------------------------- primitives (sparse.cu)
// exclusive scan of n int64 values in place; returns the total in *total (host)
ch_status scan_i64(int64_t* data, int64_t n, int64_t* total, cudaStream_t st, Alloc& tmp);
ch_status scan_i32_to_rowptr(const int* counts, int* rowptr, int n, int64_t* total,
                             cudaStream_t st, Alloc& tmp);
// incidence lists: for each of nitems items with k entries (ids in [0,nkeys)), build the
// key -> sorted item list (CSR)
ch_status build_incidence(const int* items, int nitems, int k, int nkeys, int** ptr, int** list,
                          cudaStream_t st, Alloc& mem);
// C = A * B (fp64, deterministic), allocated in mem
ch_status spgemm(const Csr<double>& A, const Csr<double>& B, Csr<double>* C, cudaStream_t st,
                 Alloc& mem);
// B = A^T (fp64), allocated in mem
ch_status transpose(const Csr<double>& A, Csr<double>* B, cudaStream_t st, Alloc& mem);

// ---------------------------------------------------------------- launch accounting (prof.cu)
enum KernelId {
  K_RHS, K_LOADS, K_APPLY_A, K_RESIDUAL4, K_ORTH0, K_ORTH1, K_ORTH2, K_SCALE4, K_UPDATE_X,
  K_CYCLE_SOLVE, K_FLAGS, K_MASS, K_CHEB_FIRST, K_CHEB_STEP, K_VRESIDUAL, K_RESTRICT, K_PROLONG,
  K_COARSE, K_VLOAD, K_VSTORE, K_SPMV_M, K_STATE_IO,
  // the same V-cycle kernels on levels below the finest (accounted separately)
  K_CHEB_FIRST_C, K_CHEB_STEP_C, K_VRESIDUAL_C, K_RESTRICT_C, K_PROLONG_C,
  K_WS_CONV, K_WS_IO, K_GUESS, K_ELEM_LOADS, K_MR_DOT, K_MR_VEC, K_CHEB_SEMI, K_MORPH, K_ORTH_RE, K_COUNT
};
// RAII around one kernel launch: counts it with its algorithmic bytes / FMAs and, when timing
// is on, records CUDA events around it on the launching stream.
class ProfScope {
 public:
  ProfScope(cudaStream_t st, int kid, int f32, double bytes, double fmas);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  cudaStream_t st_;
  int slot_;
  double bytes_, fmas_;
  cudaEvent_t e0_ = nullptr, e1_ = nullptr;
};
void prof_drain();
bool prof_timing();
// launch accounting of kernels recorded into a CUDA graph, replayed at each graph launch
struct ProfTally {
  int64_t launches[K_COUNT * 2] = {};
  double bytes[K_COUNT * 2] = {};
  double fmas[K_COUNT * 2] = {};
};
// the tally that ProfScopes record into while capturing (nullptr: none); returns the previous one
ProfTally* prof_capture_swap(ProfTally* t);
void prof_add(const ProfTally& t);
void prof_add_times(const ProfTally& t, int64_t times);
// add to one kernel's counters directly (work whose size only the device knew)
void prof_add_slot(int kid, int f32, int64_t launches, double bytes, double fmas);

}  // namespace ch

// ---------------------------------------------------------------- opaque handles
struct ch_mesh_s {
  ch_params p{};                 // parameters of run 0 (the only run of a plain mesh)
  std::vector<ch_params> runs;   // per-run parameters (box, cells)
  bool batch = false;            // built by ch_mesh_batch
  std::vector<int> run_off;      // host: first node of each run, run_off[R] = N
  int* run_off_d = nullptr;      // device copy
  int* node_run = nullptr;       // run of each node
  int dim = 2, N = 0, E = 0, Fb = 0, Ft = 0;
  double* coords = nullptr;   // N x dim
  int* elems = nullptr;       // E x (dim+1)
  int* bot = nullptr;         // Fb x dim
  int* top = nullptr;         // Ft x dim
  double* vol = nullptr;      // E element measures
  double* bvol = nullptr;     // Fb facet measures
  double* tvol = nullptr;     // Ft facet measures
  int *n2e_ptr = nullptr, *n2e = nullptr;  // node -> incident elements (sorted)
  int *n2b_ptr = nullptr, *n2b = nullptr;  // node -> incident bottom facets
  int *n2t_ptr = nullptr, *n2t = nullptr;  // node -> incident top facets
  ch::Alloc mem;
};

struct ch_system_s {
  const ch_mesh_s* mesh = nullptr;
  ch_params p{};
  int N = 0;
  int64_t nnz = 0;
  int* rowptr = nullptr;
  int* col = nullptr;
  double* valM = nullptr;
  double* valK = nullptr;
  double* valH = nullptr;
  int* diag = nullptr;  // position of the diagonal entry of each row
  double* eload = nullptr;  // E x (dim+1) x 2: per element and vertex, the f-load contributions
  double* bw = nullptr;     // pattern = 1: Fb x 2 species x (dim + dim^2) substrate weights, else null
  double a = 0, c = 0;  // A = [[M, aK], [aK, -cM]]
  ch::Alloc mem;
};

namespace ch {
struct Hierarchy;  // amg.cu
// The fine level's mesh structure, for the structured (diagonal) form of level 0: node i of run r
// has its neighbours at i + a + b W_r + c WH_r over the uniform mesh's lattice directions.
struct FineLattice {
  int dim = 0;                    // 2 or 3
  std::vector<int> run_off;       // host, runs + 1
  std::vector<int> W, WH;         // host, per run: nx + 1 and (nx + 1)(ny + 1)
  const int* node_run = nullptr;  // device, N (used when there are several runs)
};
ch_status hierarchy_build(const Csr<double>& A0, const FineLattice* lat, const ch_params& p, int precision,
                          cudaStream_t st, Hierarchy** out);
void hierarchy_free(Hierarchy* h);
int hierarchy_levels(const Hierarchy* h);
void hierarchy_level_size(const Hierarchy* h, int l, int64_t* rows, int64_t* nnz);
ch_status hierarchy_level_export(const Hierarchy* h, int l, int64_t* rows, int64_t* nnz, int64_t* nnz_P,
                                 double* lo, double* hi, int* degree, int* A_rowptr, int* A_col,
                                 double* A_val, int* P_rowptr, int* P_col, double* P_val, cudaStream_t st);
void hierarchy_level_tiles(const Hierarchy* h, int l, int* tA, int* tR, int* tP);
// x (N x 2, fp64, row stride ldx) ~ A^-1 b (N x 2, fp64, row stride ldb), ncyc V-cycles
ch_status hierarchy_solve(Hierarchy* h, const double* b, int ldb, double* x, int ldx, int ncyc,
                          cudaStream_t st);
// x (N x 2, fp64, read and overwritten) after `passes` passes of the finest level's Chebyshev smoother
ch_status hierarchy_smooth(Hierarchy* h, const double* b, double* x, int degree, int passes, cudaStream_t st);
// as hierarchy_solve (strides 2), work vectors in a static device array: no device allocation
ch_status hierarchy_solve_noalloc(Hierarchy* h, const double* b, double* x, int ncyc, cudaStream_t st);
// y (N x 2, fp64, stride ldy) = A0 x (N x 2, fp64, stride ldx) in the hierarchy's working precision

// assemble.cu
ch_status loads(const ch_system_s* s, const double* pp, const double* pn, double* Fp, double* Fn,
                double* gp, double* gn, cudaStream_t st);
// b (N x 4) from phi_p, phi_nfa read with element stride ld
ch_status rhs_strided(const ch_system_s* s, const double* pp, const double* pn, int ld, double* b,
                      cudaStream_t st);
ch_status mesh_build(ch_mesh_s* m, cudaStream_t st);
ch_status assemble_system(const ch_mesh_s* m, ch_system_s* s, cudaStream_t st);
ch_status apply_A(const ch_system_s* s, const double* x, double* y, cudaStream_t st);
}  // namespace ch

struct ch_precond_s {
  const ch_system_s* sys = nullptr;
  int precision = 0;
  ch::Hierarchy* hM = nullptr;
  ch::Hierarchy* hH = nullptr;
  double* t1 = nullptr;  // N x 2 temporaries for Algorithm 1
  double* t2 = nullptr;
  cudaStream_t side = nullptr;  // Algorithm 1's M-solve branch (non-blocking)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  ch::Alloc mem;
  ~ch_precond_s() {
    ch::hierarchy_free(hM);
    ch::hierarchy_free(hH);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (side) cudaStreamDestroy(side);
  }
};

struct ch_state_s;
namespace ch {
ch_status precond_apply(ch_precond_s* pc, const double* v, double* w, cudaStream_t st);
// Algorithm 1's step 1 on two right-hand sides (N x 2 fp64): x = M~^-1 b
ch_status mass_solve(ch_precond_s* pc, const double* b, double* x, cudaStream_t st);
// morphology.cu: Section 5's projection of a thresholded 2D morphology onto a finite-difference grid
ch_status morphology_project(const double* pp, const double* pn, int nx, int ny, double Lx, double Ly,
                             int use_thr, double thr, int gx, int gy, uint8_t* polymer, double* mu_e,
                             double* mu_h, cudaStream_t st);
const char* last_error();
ch_status state_create(const ch_system_s* s, ch_precond_s* pc, cudaStream_t st, ch_state_s** out);
void state_destroy(ch_state_s* S);
ch_status state_set(ch_state_s* S, const double* pp, const double* pn, const double* mp,
                    const double* mn, cudaStream_t st);
ch_status state_seeded(ch_state_s* S, double p0, double n0, double noise, uint64_t seed,
                       cudaStream_t st);
ch_status state_get(const ch_state_s* S, double* pp, double* pn, double* ps, double* mp, double* mn,
                    cudaStream_t st);
ch_status state_seeded_batch(ch_state_s* S, const double* base_p, const double* base_n, double noise,
                             uint64_t seed, cudaStream_t st);
ch_status state_run_stats(const ch_state_s* S, int run, ch_step_stats* out);
ch_status state_save(const ch_state_s* S, const char* path, cudaStream_t st);
ch_status state_load(ch_state_s* S, const char* path, cudaStream_t st);
ch_status state_step(ch_state_s* S, cudaStream_t st, ch_step_stats* stats);
}

// warmstart.cu
struct ch_ws_s;
namespace ch {
ch_status ws_create(int H, int W, int Bmax, ch_ws_s** out);
// convolution engine: 0 mma.sync, 1 tcgen05; ws_check reports a timed-out tcgen05 block (call
// after synchronising with the network's work)
ch_status ws_set_engine(ch_ws_s* w, int engine);
ch_status ws_withhold_mma(ch_ws_s* w, int on);
ch_status ws_check(const ch_ws_s* w);
void ws_destroy(ch_ws_s* w);
ch_status ws_set_params(ch_ws_s* w, const float* host, cudaStream_t st);
ch_status ws_get_params(const ch_ws_s* w, float* host, float* host_grads, cudaStream_t st);
ch_status ws_set_norm(ch_ws_s* w, const float* host20, cudaStream_t st);
ch_status ws_fit_norm(ch_ws_s* w, const void* x, int S, int fp32, double* host20, cudaStream_t st);
ch_status ws_predict(ch_ws_s* w, const double* state, const double* prev, const double* prev2, double* pred,
                     cudaStream_t st);
ch_status ws_train_step(ch_ws_s* w, const float* x, const float* q, const float* q2, const float* n, int B,
                        float lap, float lr, float* loss, cudaStream_t st);
ch_status ws_train_residual(ch_ws_s* w, const ch_system_s* sys, ch_precond_s* pc, const double* x,
                            const double* q, const double* q2, int B, float lr, float* loss, cudaStream_t st);
int ws_nparam();
void ws_dims(const ch_ws_s* w, int* H, int* W);
ch_status state_step_learned(ch_state_s* S, ch_ws_s* w, cudaStream_t st, ch_step_stats* stats);
ch_status state_step_guess(ch_state_s* S, const double* guess, cudaStream_t st, ch_step_stats* stats);
}  // namespace ch
