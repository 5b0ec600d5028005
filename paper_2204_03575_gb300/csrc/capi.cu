// extern "C" entry points declared in include/ch.h: argument checks, handle lifetime,
// and dispatch to the kernels of assemble.cu, amg.cu and krylov.cu.
#include <algorithm>
#include <cmath>
#include <new>

#include "ch_internal.cuh"

using ch::set_error;

namespace {
cudaStream_t S(void* stream) { return reinterpret_cast<cudaStream_t>(stream); }

ch_status check_params(const ch_params* p) {
  CH_ARG(p != nullptr, "params is NULL");
  CH_ARG(p->dim == 2 || p->dim == 3, "dim must be 2 or 3");
  CH_ARG(p->nx >= 1 && p->ny >= 1 && (p->dim == 2 || p->nz >= 1), "cell counts must be >= 1");
  CH_ARG(p->Lx > 0 && p->Ly > 0 && (p->dim == 2 || p->Lz > 0), "box extents must be > 0");
  const double nodes = (double)(p->nx + 1) * (p->ny + 1) * (p->dim == 3 ? (p->nz + 1) : 1);
  CH_ARG(nodes < 2.0e8, "mesh too large for int32 indexing");
  CH_ARG(p->tau > 0 && std::isfinite(p->tau), "tau must be > 0");
  CH_ARG(p->eps > 0 && std::isfinite(p->eps), "eps must be > 0");
  CH_ARG(p->mobility > 0 && std::isfinite(p->mobility), "mobility must be > 0");
  CH_ARG(p->bc_mode == 0 || p->bc_mode == 1, "bc_mode must be 0 or 1");
  CH_ARG(p->evap_sign == 1 || p->evap_sign == -1, "evap_sign must be +1 or -1");
  CH_ARG(p->potential >= 0 && p->potential <= 3, "potential must be 0, 1, 2 or 3");
  CH_ARG(p->precision == 0 || p->precision == 1, "precision must be 0 or 1");
  CH_ARG(p->rtol > 0 && p->rtol < 1, "rtol must be in (0, 1)");
  CH_ARG(p->restart >= 1 && p->restart <= 64, "restart must be in [1, 64]");
  CH_ARG(p->max_iter >= 1, "max_iter must be >= 1");
  CH_ARG(p->cheb_degree >= 0 && p->cheb_degree <= 16, "cheb_degree must be in [0, 16]");
  CH_ARG(p->coarse_max >= 0 && p->coarse_max <= 4096, "coarse_max must be in [0, 4096]");
  CH_ARG(p->amg_theta >= 0 && p->amg_theta < 1, "amg_theta must be in [0, 1)");
  CH_ARG(p->vcycles_M >= 1 && p->vcycles_H >= 1, "vcycles must be >= 1");
  CH_ARG(p->autotune == 0 || p->autotune == 1, "autotune must be 0 or 1");
  CH_ARG(p->cheb_lower > 0 && p->cheb_lower < 1, "cheb_lower must be in (0, 1)");
  CH_ARG(p->graphs == 0 || p->graphs == 1, "graphs must be 0 or 1");
  CH_ARG(p->cheb_degree_coarse >= 0 && p->cheb_degree_coarse <= 16, "cheb_degree_coarse must be in [0, 16]");
  CH_ARG(p->krylov == 0 || p->krylov == 1, "krylov must be 0 (FGMRES) or 1 (MINRES)");
  CH_ARG(p->cheb_degree_M >= 0 && p->cheb_degree_M <= 16, "cheb_degree_M must be in [0, 16]");
  CH_ARG(p->pattern == 0 || p->pattern == 1, "pattern must be 0 or 1");
  CH_ARG(p->precond_M == 0 || p->precond_M == 1, "precond_M must be 0 (AMG) or 1 (Chebyshev semi-iteration)");
  CH_ARG(p->cheb_M_steps >= 0 && p->cheb_M_steps <= 16, "cheb_M_steps must be in [0, 16]");
  CH_ARG(std::isfinite(p->chi_pn) && std::isfinite(p->chi_ps) && std::isfinite(p->chi_ns),
         "chi parameters must be finite");
  CH_ARG(p->N_p > 0 && p->N_nfa > 0 && p->N_s > 0 && std::isfinite(p->N_p) && std::isfinite(p->N_nfa) &&
             std::isfinite(p->N_s),
         "N_p, N_nfa, N_s must be > 0");
  CH_ARG(p->fh_delta > 0 && p->fh_delta < 1, "fh_delta must be in (0, 1)");
  CH_ARG(p->pdl == 0 || p->pdl == 1, "pdl must be 0 or 1");
  CH_ARG(p->gs_reorth == 0 || p->gs_reorth == 1, "gs_reorth must be 0 or 1");
  return CH_OK;
}
}  // namespace

extern "C" {

const char* ch_status_str(ch_status s) {
  switch (s) {
    case CH_OK: return "ok";
    case CH_ERR_ARG: return "invalid argument";
    case CH_ERR_CUDA: return "CUDA error";
    case CH_ERR_OOM: return "out of device memory";
    case CH_ERR_NOT_CONVERGED: return "not converged";
    case CH_ERR_BREAKDOWN: return "Krylov breakdown";
    case CH_ERR_NONFINITE: return "non-finite value";
    case CH_ERR_STATE: return "call out of order";
    case CH_ERR_INTERNAL: return "internal check failed";
  }
  return "unknown status";
}

const char* ch_last_error(void) { return ch::last_error(); }

void ch_params_default(ch_params* p) {
  if (!p) return;
  ch_params d{};
  d.dim = 2;
  d.nx = 32;
  d.ny = 32;
  d.nz = 0;
  d.Lx = 1.0;
  d.Ly = 1.0;
  d.Lz = 1.0;
  d.tau = 1e-4;
  d.eps = 1e-3;
  d.mobility = 1.0;
  d.bc_mode = 1;
  d.evap_sign = 1;
  d.potential = 0;
  d.precision = 0;
  d.k_evap = 5e-3;
  d.g_p = 0.01;
  d.g_nfa = 0.01;
  d.h_p = 0.0;
  d.h_nfa = 0.0;
  d.rtol = 1e-8;
  d.restart = 30;
  d.max_iter = 300;
  d.cheb_degree = 0;
  d.coarse_max = 0;
  d.amg_theta = 0.08;
  d.vcycles_M = 1;
  d.vcycles_H = 2;
  d.autotune = 1;
  d.cheb_lower = 0.3;
  d.graphs = 1;
  d.cheb_degree_coarse = 0;
  d.cheb_degree_M = 0;
  d.krylov = 0;
  d.pattern = 0;
  d.precond_M = 0;
  d.cheb_M_steps = 0;
  d.chi_pn = 1.0;
  d.chi_ps = 0.3;
  d.chi_ns = 0.3;
  d.N_p = 20.0;
  d.N_nfa = 20.0;
  d.N_s = 1.0;
  d.fh_delta = 1e-10;
  d.pdl = 1;
  d.gs_reorth = 0;
  *p = d;
}

// ---------------------------------------------------------------- mesh
ch_status ch_mesh(const ch_params* p, void* stream, ch_mesh_t** out) {
  CH_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  CH_TRY(check_params(p));
  ch_mesh_s* m = new (std::nothrow) ch_mesh_s();
  if (!m) return CH_ERR_OOM;
  m->p = *p;
  m->runs.assign(1, *p);
  ch_status r = ch::mesh_build(m, S(stream));
  if (r != CH_OK) {
    delete m;
    return r;
  }
  *out = m;
  return CH_OK;
}

ch_status ch_mesh_batch(int32_t nruns, const ch_params* runs, void* stream, ch_mesh_t** out) {
  CH_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  CH_ARG(nruns >= 1 && runs != nullptr, "need at least one run");
  for (int r = 0; r < nruns; ++r) {
    CH_TRY(check_params(&runs[r]));
    CH_ARG(runs[r].dim == runs[0].dim, "all runs of a batch must have the same dim");
  }
  ch_mesh_s* m = new (std::nothrow) ch_mesh_s();
  if (!m) return CH_ERR_OOM;
  m->p = runs[0];
  m->runs.assign(runs, runs + nruns);
  m->batch = true;
  ch_status r = ch::mesh_build(m, S(stream));
  if (r != CH_OK) {
    delete m;
    return r;
  }
  *out = m;
  return CH_OK;
}

ch_status ch_mesh_runs(const ch_mesh_t* m, int32_t* nruns, int32_t* run_offsets) {
  CH_ARG(m != nullptr, "mesh is NULL");
  if (nruns) *nruns = (int32_t)m->runs.size();
  if (run_offsets)
    for (size_t r = 0; r < m->run_off.size(); ++r) run_offsets[r] = m->run_off[r];
  return CH_OK;
}

ch_status ch_mesh_info(const ch_mesh_t* m, int64_t* n_nodes, int64_t* n_elems, int64_t* n_bottom,
                       int64_t* n_top) {
  CH_ARG(m != nullptr, "mesh is NULL");
  if (n_nodes) *n_nodes = m->N;
  if (n_elems) *n_elems = m->E;
  if (n_bottom) *n_bottom = m->Fb;
  if (n_top) *n_top = m->Ft;
  return CH_OK;
}

ch_status ch_mesh_copy(const ch_mesh_t* m, double* coords, int32_t* elems, int32_t* bottom,
                       int32_t* top, void* stream) {
  CH_ARG(m != nullptr, "mesh is NULL");
  const cudaStream_t st = S(stream);
  const int d = m->dim;
  if (coords)
    CH_CUDA(cudaMemcpyAsync(coords, m->coords, sizeof(double) * m->N * d, cudaMemcpyDeviceToDevice, st));
  if (elems)
    CH_CUDA(cudaMemcpyAsync(elems, m->elems, sizeof(int) * (size_t)m->E * (d + 1),
                            cudaMemcpyDeviceToDevice, st));
  if (bottom)
    CH_CUDA(cudaMemcpyAsync(bottom, m->bot, sizeof(int) * (size_t)m->Fb * d, cudaMemcpyDeviceToDevice, st));
  if (top)
    CH_CUDA(cudaMemcpyAsync(top, m->top, sizeof(int) * (size_t)m->Ft * d, cudaMemcpyDeviceToDevice, st));
  return CH_OK;
}

void ch_mesh_destroy(ch_mesh_t* m) { delete m; }

// ---------------------------------------------------------------- assembly
ch_status ch_assemble(const ch_mesh_t* m, const ch_params* p, void* stream, ch_system_t** out) {
  CH_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  CH_ARG(m != nullptr, "mesh is NULL");
  CH_TRY(check_params(p));
  CH_ARG(p->dim == m->p.dim, "params describe a mesh of another dimension");
  CH_ARG(m->batch || (p->nx == m->p.nx && p->ny == m->p.ny && (p->dim == 2 || p->nz == m->p.nz)),
         "params describe a different mesh");
  ch_system_s* s = new (std::nothrow) ch_system_s();
  if (!s) return CH_ERR_OOM;
  s->mesh = m;
  s->p = *p;
  s->a = p->tau * p->mobility;
  s->c = s->a / p->eps;
  ch_status r = ch::assemble_system(m, s, S(stream));
  if (r != CH_OK) {
    delete s;
    return r;
  }
  *out = s;
  return CH_OK;
}

ch_status ch_system_info(const ch_system_t* s, int64_t* n, int64_t* nnz) {
  CH_ARG(s != nullptr, "system is NULL");
  if (n) *n = s->N;
  if (nnz) *nnz = s->nnz;
  return CH_OK;
}

ch_status ch_system_copy(const ch_system_t* s, int32_t* rowptr, int32_t* col, double* valM,
                         double* valK, double* valH, void* stream) {
  CH_ARG(s != nullptr, "system is NULL");
  const cudaStream_t st = S(stream);
  if (rowptr)
    CH_CUDA(cudaMemcpyAsync(rowptr, s->rowptr, sizeof(int) * ((size_t)s->N + 1), cudaMemcpyDeviceToDevice, st));
  if (col) CH_CUDA(cudaMemcpyAsync(col, s->col, sizeof(int) * s->nnz, cudaMemcpyDeviceToDevice, st));
  if (valM) CH_CUDA(cudaMemcpyAsync(valM, s->valM, sizeof(double) * s->nnz, cudaMemcpyDeviceToDevice, st));
  if (valK) CH_CUDA(cudaMemcpyAsync(valK, s->valK, sizeof(double) * s->nnz, cudaMemcpyDeviceToDevice, st));
  if (valH) CH_CUDA(cudaMemcpyAsync(valH, s->valH, sizeof(double) * s->nnz, cudaMemcpyDeviceToDevice, st));
  return CH_OK;
}

void ch_system_destroy(ch_system_t* s) { delete s; }

ch_status ch_loads(const ch_system_t* s, const double* phi_p, const double* phi_nfa, double* F_p,
                   double* F_nfa, double* g_p, double* g_nfa, void* stream) {
  CH_ARG(s != nullptr && phi_p != nullptr && phi_nfa != nullptr, "NULL system or input");
  return ch::loads(s, phi_p, phi_nfa, F_p, F_nfa, g_p, g_nfa, S(stream));
}

ch_status ch_rhs(const ch_system_t* s, const double* phi_p, const double* phi_nfa, double* b,
                 void* stream) {
  CH_ARG(s != nullptr && phi_p != nullptr && phi_nfa != nullptr && b != nullptr, "NULL argument");
  CH_ARG((reinterpret_cast<uintptr_t>(b) & 31) == 0, "b must be 32-byte aligned");
  return ch::rhs_strided(s, phi_p, phi_nfa, 1, b, S(stream));
}

ch_status ch_apply_A(const ch_system_t* s, const double* x, double* y, void* stream) {
  CH_ARG(s != nullptr && x != nullptr && y != nullptr, "NULL argument");
  CH_ARG(x != y, "x and y must not alias");
  CH_ARG(((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 31) == 0,
         "x and y must be 32-byte aligned");
  return ch::apply_A(s, x, y, S(stream));
}

// ---------------------------------------------------------------- preconditioner
ch_status ch_precond_setup(const ch_system_t* s, void* stream, ch_precond_t** out) {
  CH_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  CH_ARG(s != nullptr, "system is NULL");
  ch_precond_s* pc = new (std::nothrow) ch_precond_s();
  if (!pc) return CH_ERR_OOM;
  pc->sys = s;
  pc->precision = s->p.precision;
  ch::Csr<double> M, H;
  M.nrows = M.ncols = H.nrows = H.ncols = s->N;
  M.nnz = H.nnz = s->nnz;
  M.rowptr = H.rowptr = s->rowptr;
  M.col = H.col = s->col;
  M.val = s->valM;
  H.val = s->valH;
  ch::FineLattice lat;
  lat.dim = s->mesh->dim;
  lat.run_off = s->mesh->run_off;
  for (const ch_params& rp : s->mesh->runs) {
    lat.W.push_back(rp.nx + 1);
    lat.WH.push_back((rp.nx + 1) * (rp.ny + 1));
  }
  lat.node_run = s->mesh->node_run;
  // The finest level's Chebyshev degree, cheb_degree 0: 5 in both precisions.  (FP64 512 x 512:
  // 79.8 / 76.0 steps/s at degree 5 / 6.  FP32 V-cycles: degree 6 gained 3 % on 512 x 512 steps
  // 4..63 but lost 3.6 % on the 3D box and 2-5 % on the 256 x 256 warm-start runs.)
  // M's hierarchy smooths with its own finest degree (0: min(3, that degree)); measured on
  // 512 x 512 with degree 5: M degree 5 / 3 / 2 gave 79.8 / 81.7 / 76.0 FP64 steps/s
  ch_params ph = s->p;
  if (ph.cheb_degree == 0) ph.cheb_degree = 5;
  ch_params pm = ph;
  pm.cheb_degree = ph.cheb_degree_M > 0 ? ph.cheb_degree_M : std::min(3, ph.cheb_degree);
  ch_status r = ch::hierarchy_build(M, &lat, pm, pc->precision, S(stream), &pc->hM);
  if (r == CH_OK) r = ch::hierarchy_build(H, &lat, ph, pc->precision, S(stream), &pc->hH);
  if (r == CH_OK && (cudaStreamCreateWithFlags(&pc->side, cudaStreamNonBlocking) != cudaSuccess ||
                     cudaEventCreateWithFlags(&pc->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                     cudaEventCreateWithFlags(&pc->ev_join, cudaEventDisableTiming) != cudaSuccess)) {
    cudaGetLastError();
    ch::set_error("preconditioner: creating its side stream or events failed");
    r = CH_ERR_CUDA;
  }
  if (r != CH_OK) {
    delete pc;
    return r;
  }
  *out = pc;
  return CH_OK;
}

ch_status ch_precond_info(const ch_precond_t* pc, int32_t which, int32_t level, int32_t* nlevels,
                          int64_t* rows, int64_t* nnz) {
  CH_ARG(pc != nullptr, "preconditioner is NULL");
  CH_ARG(which == 0 || which == 1, "which must be 0 (M) or 1 (H)");
  const ch::Hierarchy* h = which == 0 ? pc->hM : pc->hH;
  const int nl = ch::hierarchy_levels(h);
  if (nlevels) *nlevels = nl;
  if (rows || nnz) {
    CH_ARG(level >= 0 && level < nl, "level out of range");
    ch::hierarchy_level_size(h, level, rows, nnz);
  }
  return CH_OK;
}

ch_status ch_precond_level(const ch_precond_t* pc, int32_t which, int32_t level, int64_t* rows,
                           int64_t* nnz, int64_t* nnz_P, double* lo, double* hi, int32_t* degree,
                           int32_t* A_rowptr, int32_t* A_col, double* A_val, int32_t* P_rowptr,
                           int32_t* P_col, double* P_val, void* stream) {
  CH_ARG(pc != nullptr, "preconditioner is NULL");
  CH_ARG(which == 0 || which == 1, "which must be 0 (M) or 1 (H)");
  const ch::Hierarchy* h = which == 0 ? pc->hM : pc->hH;
  CH_ARG(level >= 0 && level < ch::hierarchy_levels(h), "level out of range");
  return ch::hierarchy_level_export(h, level, rows, nnz, nnz_P, lo, hi, degree, A_rowptr, A_col, A_val,
                                    P_rowptr, P_col, P_val, S(stream));
}

ch_status ch_precond_tiles(const ch_precond_t* pc, int32_t which, int32_t level, int32_t* tpr_A,
                           int32_t* tpr_R, int32_t* tpr_P) {
  CH_ARG(pc != nullptr, "preconditioner is NULL");
  CH_ARG(which == 0 || which == 1, "which must be 0 (M) or 1 (H)");
  const ch::Hierarchy* h = which == 0 ? pc->hM : pc->hH;
  CH_ARG(level >= 0 && level < ch::hierarchy_levels(h), "level out of range");
  int a = 0, r = 0, q = 0;
  ch::hierarchy_level_tiles(h, level, &a, &r, &q);
  if (tpr_A) *tpr_A = a;
  if (tpr_R) *tpr_R = r;
  if (tpr_P) *tpr_P = q;
  return CH_OK;
}

ch_status ch_precond_apply(ch_precond_t* pc, const double* v, double* w, void* stream) {
  CH_ARG(pc != nullptr && v != nullptr && w != nullptr, "NULL argument");
  CH_ARG(v != w, "v and w must not alias");
  CH_ARG(((reinterpret_cast<uintptr_t>(v) | reinterpret_cast<uintptr_t>(w)) & 31) == 0,
         "v and w must be 32-byte aligned");
  return ch::precond_apply(pc, v, w, S(stream));
}

ch_status ch_vcycle(ch_precond_t* pc, int32_t which, int32_t vcycles, const double* b, double* x,
                    void* stream) {
  CH_ARG(pc != nullptr && b != nullptr && x != nullptr, "NULL argument");
  CH_ARG(which == 0 || which == 1, "which must be 0 (M) or 1 (H)");
  CH_ARG(vcycles >= 1, "vcycles must be >= 1");
  CH_ARG(b != x, "b and x must not alias");
  CH_ARG(((reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(x)) & 15) == 0,
         "b and x must be 16-byte aligned");
  return ch::hierarchy_solve(which == 0 ? pc->hM : pc->hH, b, 2, x, 2, vcycles, S(stream));
}

ch_status ch_smooth(ch_precond_t* pc, int32_t which, int32_t degree, int32_t passes, const double* b, double* x,
                    void* stream) {
  CH_ARG(pc != nullptr && b != nullptr && x != nullptr, "NULL argument");
  CH_ARG(which == 0 || which == 1, "which must be 0 (M) or 1 (H)");
  CH_ARG(degree >= 1 && degree <= 16, "degree must be in [1, 16]");
  CH_ARG(passes >= 1, "passes must be >= 1");
  CH_ARG(b != x, "b and x must not alias");
  CH_ARG(((reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(x)) & 15) == 0,
         "b and x must be 16-byte aligned");
  ch::Hierarchy* h = which == 0 ? pc->hM : pc->hH;
  CH_ARG(ch::hierarchy_levels(h) >= 2, "the hierarchy has one level (solved directly: it has no smoother)");
  return ch::hierarchy_smooth(h, b, x, degree, passes, S(stream));
}

ch_status ch_mass_solve(ch_precond_t* pc, const double* b, double* x, void* stream) {
  CH_ARG(pc != nullptr && b != nullptr && x != nullptr, "NULL argument");
  CH_ARG(b != x, "b and x must not alias");
  CH_ARG(((reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(x)) & 15) == 0,
         "b and x must be 16-byte aligned");
  return ch::mass_solve(pc, b, x, S(stream));
}

void ch_precond_destroy(ch_precond_t* pc) { delete pc; }

// ---------------------------------------------------------------- morphology projection
ch_status ch_morphology_project(const double* phi_p, const double* phi_nfa, int32_t nx, int32_t ny, double Lx,
                                double Ly, int32_t use_threshold, double threshold, int32_t gx, int32_t gy,
                                uint8_t* polymer, double* mu_e, double* mu_h, void* stream) {
  CH_ARG(phi_p != nullptr && (use_threshold || phi_nfa != nullptr), "NULL field");
  CH_ARG(use_threshold == 0 || use_threshold == 1, "use_threshold must be 0 or 1");
  CH_ARG(nx >= 1 && ny >= 1 && gx >= 1 && gy >= 1, "mesh and grid sizes must be >= 1");
  CH_ARG((double)(nx + 1) * (ny + 1) < 2.0e9 && (double)gx * gy < 2.0e9, "image or grid too large");
  CH_ARG(Lx > 0 && Ly > 0 && std::isfinite(Lx) && std::isfinite(Ly), "box extents must be > 0");
  CH_ARG(!use_threshold || std::isfinite(threshold), "threshold must be finite");
  return ch::morphology_project(phi_p, phi_nfa, nx, ny, Lx, Ly, use_threshold, threshold, gx, gy, polymer, mu_e,
                                mu_h, S(stream));
}

ch_status ch_vcycle_noalloc(ch_precond_t* pc, int32_t which, int32_t vcycles, const double* b,
                            double* x, void* stream) {
  CH_ARG(pc != nullptr && b != nullptr && x != nullptr, "NULL argument");
  CH_ARG(which == 0 || which == 1, "which must be 0 (M) or 1 (H)");
  CH_ARG(vcycles >= 1, "vcycles must be >= 1");
  CH_ARG(b != x, "b and x must not alias");
  CH_ARG(((reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(x)) & 15) == 0,
         "b and x must be 16-byte aligned");
  return ch::hierarchy_solve_noalloc(which == 0 ? pc->hM : pc->hH, b, x, vcycles, S(stream));
}

// ---------------------------------------------------------------- state and stepping
ch_status ch_state_create(const ch_system_t* s, ch_precond_t* pc, void* stream, ch_state_t** out) {
  CH_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  CH_ARG(s != nullptr && pc != nullptr, "NULL system or preconditioner");
  CH_ARG(pc->sys == s, "preconditioner was built for another system");
  return ch::state_create(s, pc, S(stream), out);
}

ch_status ch_state_set(ch_state_t* st, const double* phi_p, const double* phi_nfa,
                       const double* mu_p, const double* mu_nfa, void* stream) {
  CH_ARG(st != nullptr && phi_p != nullptr && phi_nfa != nullptr, "NULL argument");
  return ch::state_set(st, phi_p, phi_nfa, mu_p, mu_nfa, S(stream));
}

ch_status ch_state_init_seeded(ch_state_t* st, double phi_p0, double phi_nfa0, double noise,
                               uint64_t seed, void* stream) {
  CH_ARG(st != nullptr, "state is NULL");
  return ch::state_seeded(st, phi_p0, phi_nfa0, noise, seed, S(stream));
}

ch_status ch_state_init_seeded_batch(ch_state_t* st, const double* phi_p0, const double* phi_nfa0,
                                     double noise, uint64_t seed, void* stream) {
  CH_ARG(st != nullptr && phi_p0 != nullptr && phi_nfa0 != nullptr, "NULL argument");
  return ch::state_seeded_batch(st, phi_p0, phi_nfa0, noise, seed, S(stream));
}

ch_status ch_state_run_stats(const ch_state_t* st, int32_t run, ch_step_stats* out) {
  CH_ARG(st != nullptr && out != nullptr, "NULL argument");
  return ch::state_run_stats(st, run, out);
}

ch_status ch_state_get(const ch_state_t* st, double* phi_p, double* phi_nfa, double* phi_s,
                       double* mu_p, double* mu_nfa, void* stream) {
  CH_ARG(st != nullptr, "state is NULL");
  return ch::state_get(st, phi_p, phi_nfa, phi_s, mu_p, mu_nfa, S(stream));
}

ch_status ch_state_save(const ch_state_t* st, const char* path, void* stream) {
  CH_ARG(st != nullptr && path != nullptr, "NULL argument");
  return ch::state_save(st, path, S(stream));
}

ch_status ch_state_load(ch_state_t* st, const char* path, void* stream) {
  CH_ARG(st != nullptr && path != nullptr, "NULL argument");
  return ch::state_load(st, path, S(stream));
}

ch_status ch_step(ch_state_t* st, void* stream, ch_step_stats* stats) {
  CH_ARG(st != nullptr, "state is NULL");
  return ch::state_step(st, S(stream), stats);
}

ch_status ch_run(ch_state_t* st, int32_t nsteps, void* stream, ch_step_stats* per_step) {
  CH_ARG(st != nullptr, "state is NULL");
  CH_ARG(nsteps >= 0, "nsteps must be >= 0");
  for (int k = 0; k < nsteps; ++k) CH_TRY(ch::state_step(st, S(stream), per_step ? per_step + k : nullptr));
  return CH_OK;
}

void ch_state_destroy(ch_state_t* st) { ch::state_destroy(st); }

ch_status ch_step_guess(ch_state_t* st, const double* guess, void* stream, ch_step_stats* stats) {
  CH_ARG(st != nullptr && guess != nullptr, "NULL argument");
  CH_ARG((reinterpret_cast<uintptr_t>(guess) & 31) == 0, "guess must be 32-byte aligned");
  return ch::state_step_guess(st, guess, S(stream), stats);
}

ch_status ch_step_learned(ch_state_t* state, ch_ws_t* w, void* stream, ch_step_stats* stats) {
  CH_ARG(state != nullptr && w != nullptr, "NULL argument");
  return ch::state_step_learned(state, w, S(stream), stats);
}

// ---------------------------------------------------------------- learned warm start
int32_t ch_ws_nparams(void) { return ch::ws_nparam(); }

ch_status ch_ws_create(int32_t H, int32_t W, int32_t max_batch, ch_ws_t** out) {
  CH_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  CH_ARG(H >= 1 && W >= 1 && (double)H * W < 1.0e8, "image size out of range");
  CH_ARG(max_batch >= 1 && max_batch <= 256, "max_batch must be in [1, 256]");
  return ch::ws_create(H, W, max_batch, out);
}

void ch_ws_destroy(ch_ws_t* w) { ch::ws_destroy(w); }

ch_status ch_ws_inject_mma_timeout(ch_ws_t* w, int32_t on) {
  CH_ARG(w != nullptr, "NULL argument");
  CH_ARG(on == 0 || on == 1, "on must be 0 or 1");
  return ch::ws_withhold_mma(w, on);
}

ch_status ch_ws_set_engine(ch_ws_t* w, int32_t engine) {
  CH_ARG(w != nullptr, "NULL argument");
  CH_ARG(engine == 0 || engine == 1, "engine must be 0 (mma.sync) or 1 (tcgen05)");
  return ch::ws_set_engine(w, engine);
}

ch_status ch_ws_set_params(ch_ws_t* w, const float* params, void* stream) {
  CH_ARG(w != nullptr && params != nullptr, "NULL argument");
  return ch::ws_set_params(w, params, S(stream));
}

ch_status ch_ws_get_params(const ch_ws_t* w, float* params, float* grads, void* stream) {
  CH_ARG(w != nullptr, "NULL argument");
  return ch::ws_get_params(w, params, grads, S(stream));
}

ch_status ch_ws_set_norm(ch_ws_t* w, const float* norm20, void* stream) {
  CH_ARG(w != nullptr && norm20 != nullptr, "NULL argument");
  return ch::ws_set_norm(w, norm20, S(stream));
}

ch_status ch_ws_fit_norm(ch_ws_t* w, const void* x, int32_t nsamples, int32_t fp32, double* norm20, void* stream) {
  CH_ARG(w != nullptr && x != nullptr && norm20 != nullptr, "NULL argument");
  CH_ARG(nsamples >= 1, "nsamples must be >= 1");
  CH_ARG(fp32 == 0 || fp32 == 1, "fp32 must be 0 or 1");
  return ch::ws_fit_norm(w, x, nsamples, fp32, norm20, S(stream));
}

ch_status ch_ws_predict(ch_ws_t* w, const double* state, const double* prev, const double* prev2, double* pred,
                        void* stream) {
  CH_ARG(w != nullptr && state != nullptr && prev != nullptr && prev2 != nullptr && pred != nullptr,
         "NULL argument");
  CH_ARG(state != pred && prev != pred && prev2 != pred, "pred must not alias the inputs");
  return ch::ws_predict(w, state, prev, prev2, pred, S(stream));
}

ch_status ch_ws_train_step(ch_ws_t* w, const float* x, const float* q, const float* q2, const float* n, int32_t B,
                           float lap, float lr, float* loss, void* stream) {
  CH_ARG(w != nullptr && x != nullptr && q != nullptr && q2 != nullptr && n != nullptr, "NULL argument");
  return ch::ws_train_step(w, x, q, q2, n, B, lap, lr, loss, S(stream));
}

ch_status ch_ws_train_residual(ch_ws_t* w, const ch_system_t* sys, ch_precond_t* pc, const double* x,
                               const double* q, const double* q2, int32_t B, float lr, float* loss, void* stream) {
  CH_ARG(w != nullptr && sys != nullptr && x != nullptr && q != nullptr && q2 != nullptr, "NULL argument");
  return ch::ws_train_residual(w, sys, pc, x, q, q2, B, lr, loss, S(stream));
}

}  // extern "C"
