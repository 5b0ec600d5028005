// Per-kernel launch counters and (optional) CUDA-event timing.
//
// Every launch site on the solve path opens a ProfScope naming its kernel, the working
// precision and the algorithmic bytes and FMAs of that launch.  Launch counts are always
// kept; when timing is enabled (ch_profile_enable(1)), a pair of CUDA events is recorded
// on the launching stream around the launch and the elapsed time is accumulated once the
// events have completed.
#include <deque>
#include <mutex>

#include "ch_internal.cuh"

namespace ch {

static const char* const kNames[K_COUNT] = {
    "rhs",          "loads",         "apply_A",     "residual4",  "orth_dots",  "orth_update_dots",
    "orth_update_norm", "scale4",    "update_x",    "cycle_solve", "flags",     "mass",
    "cheb_first",   "cheb_step",     "vresidual",   "restrict",    "prolong",   "coarse_solve",
    "vload",        "vstore",        "spmv_M",      "state_io",    "cheb_first_coarse",
    "cheb_step_coarse", "vresidual_coarse", "restrict_coarse", "prolong_coarse", "ws_conv",
    "ws_io",        "guess_select",  "elem_loads",   "minres_dot",   "minres_update", "cheb_semi", "ray_parity",
    "orth_reorth"};

struct Acc {
  int64_t launches = 0;
  double ms = 0.0, bytes = 0.0, fmas = 0.0;
};

struct Pending {
  cudaEvent_t e0, e1;
  int slot;
  double bytes, fmas;
};

static thread_local ProfTally* t_capture = nullptr;  // set while a graph is being captured

static struct {
  std::mutex mu;
  bool timing = false;
  Acc acc[K_COUNT * 2];
  std::deque<Pending> pending;
  std::vector<cudaEvent_t> pool;
} g;

static cudaEvent_t get_event() {
  if (!g.pool.empty()) {
    cudaEvent_t e = g.pool.back();
    g.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

static void drain_locked(bool wait) {
  while (!g.pending.empty()) {
    Pending& p = g.pending.front();
    if (wait) cudaEventSynchronize(p.e1);
    else if (cudaEventQuery(p.e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.e0, p.e1);
    g.acc[p.slot].ms += ms;
    g.pool.push_back(p.e0);
    g.pool.push_back(p.e1);
    g.pending.pop_front();
  }
  cudaGetLastError();  // a not-ready query is not an error for the caller
}

ProfScope::ProfScope(cudaStream_t st, int kid, int f32, double bytes, double fmas)
    : st_(st), slot_(kid * 2 + (f32 ? 1 : 0)), bytes_(bytes), fmas_(fmas) {
  if (t_capture) {  // counted each time the captured graph is launched
    t_capture->launches[slot_] += 1;
    t_capture->bytes[slot_] += bytes;
    t_capture->fmas[slot_] += fmas;
    return;
  }
  std::lock_guard<std::mutex> lk(g.mu);
  Acc& a = g.acc[slot_];
  a.launches += 1;
  a.bytes += bytes;
  a.fmas += fmas;
  if (g.timing) {
    e0_ = get_event();
    e1_ = get_event();
    cudaEventRecord(e0_, st_);
  }
}

ProfScope::~ProfScope() {
  if (!e0_) return;
  std::lock_guard<std::mutex> lk(g.mu);
  cudaEventRecord(e1_, st_);
  g.pending.push_back({e0_, e1_, slot_, bytes_, fmas_});
  if (g.pending.size() > 2048) drain_locked(true);
}

bool prof_timing() {
  std::lock_guard<std::mutex> lk(g.mu);
  return g.timing;
}

ProfTally* prof_capture_swap(ProfTally* t) {
  ProfTally* prev = t_capture;
  t_capture = t;
  return prev;
}

void prof_add_times(const ProfTally& t, int64_t times) {
  if (times <= 0) return;
  std::lock_guard<std::mutex> lk(g.mu);
  for (int s = 0; s < K_COUNT * 2; ++s) {
    if (!t.launches[s]) continue;
    g.acc[s].launches += t.launches[s] * times;
    g.acc[s].bytes += t.bytes[s] * (double)times;
    g.acc[s].fmas += t.fmas[s] * (double)times;
  }
}

void prof_add(const ProfTally& t) { prof_add_times(t, 1); }

void prof_add_slot(int kid, int f32, int64_t launches, double bytes, double fmas) {
  std::lock_guard<std::mutex> lk(g.mu);
  Acc& a = g.acc[kid * 2 + (f32 ? 1 : 0)];
  a.launches += launches;
  a.bytes += bytes;
  a.fmas += fmas;
}

void prof_drain() {
  std::lock_guard<std::mutex> lk(g.mu);
  drain_locked(false);
}

}  // namespace ch

extern "C" {

ch_status ch_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(ch::g.mu);
  ch::drain_locked(true);
  ch::g.timing = on != 0;
  return CH_OK;
}

ch_status ch_profile_read(ch_prof_entry* out, int32_t cap, int32_t* n, int32_t reset) {
  CH_ARG(n != nullptr, "n is NULL");
  std::lock_guard<std::mutex> lk(ch::g.mu);
  ch::drain_locked(true);
  int k = 0;
  for (int s = 0; s < ch::K_COUNT * 2; ++s) {
    const ch::Acc& a = ch::g.acc[s];
    if (a.launches == 0) continue;
    if (out && k < cap) {
      ch_prof_entry& e = out[k];
      snprintf(e.name, sizeof(e.name), "%s_%s", ch::kNames[s / 2], (s & 1) ? "f32" : "f64");
      e.launches = a.launches;
      e.ms = a.ms;
      e.bytes = a.bytes;
      e.fmas = a.fmas;
    }
    ++k;
  }
  *n = k;
  if (reset)
    for (auto& a : ch::g.acc) a = ch::Acc();
  return CH_OK;
}

}  // extern "C"
