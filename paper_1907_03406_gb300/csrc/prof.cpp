// Launch accounting (see prof.h).
#include "prof.h"

#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

namespace sgf {

namespace {
struct Acc {
  long long launches = 0;
  double ms = 0, flops = 0, bytes = 0;
};
struct Pending {
  cudaEvent_t a, b;
  int kind;
  double flops, bytes;
  std::string note;
};
struct State {
  std::mutex mu;
  Acc acc[P_NKINDS];
  int timing = 0;
  double next_flops = 0, next_bytes = 0;
  double next_flops_seen = 0, next_bytes_seen = 0;   // work of the launch being opened
  std::string next_note;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
};
thread_local bool t_capturing = false;
State& st() {
  static State s;
  return s;
}
cudaEvent_t get_event(State& S) {
  if (!S.pool.empty()) {
    cudaEvent_t e = S.pool.back();
    S.pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}
// SGF_PROF_LOG=1: every timed launch is also printed to stderr (kind, its
// algorithmic flops and bytes, device time), in launch order
const bool g_log = std::getenv("SGF_PROF_LOG") != nullptr;
void drain(State& S) {
  for (auto& p : S.pending) {
    cudaEventSynchronize(p.b);
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) S.acc[p.kind].ms += ms;
    if (g_log)
      std::fprintf(stderr, "[sgf launch] %-10s flops %.4e bytes %.4e ms %.5f GB/s %.1f %s\n", prof_name(p.kind),
                   p.flops, p.bytes, ms, ms > 0 ? p.bytes / (ms * 1e-3) / 1e9 : 0.0, p.note.c_str());
    S.pool.push_back(p.a);
    S.pool.push_back(p.b);
  }
  S.pending.clear();
}
}  // namespace

bool prof_logging() { return g_log; }

void prof_note(const char* note) {
  State& S = st();
  std::lock_guard<std::mutex> g(S.mu);
  S.next_note = note ? note : "";
}

void prof_work(double flops, double bytes) {
  State& S = st();
  std::lock_guard<std::mutex> g(S.mu);
  S.next_flops += flops;
  S.next_bytes += bytes;
}

ProfScope::ProfScope(int kind, cudaStream_t s) : kind_(kind), s_(s), slot_(-1) {
  State& S = st();
  std::lock_guard<std::mutex> g(S.mu);
  std::string note;
  note.swap(S.next_note);
  if (t_capturing) {
    S.next_flops = S.next_bytes = 0;
    return;
  }
  Acc& a = S.acc[kind];
  a.launches++;
  a.flops += S.next_flops;
  a.bytes += S.next_bytes;
  S.next_flops_seen = S.next_flops;
  S.next_bytes_seen = S.next_bytes;
  S.next_flops = S.next_bytes = 0;
  const bool timed = S.timing == 1 || (S.timing == 2 && (kind == P_GEMM || kind == P_DIAG || kind == P_QR || kind == P_APPLY));
  if (timed) {
    Pending p;
    p.a = get_event(S);
    p.b = get_event(S);
    p.kind = kind;
    p.flops = S.next_flops_seen;
    p.bytes = S.next_bytes_seen;
    p.note = std::move(note);
    cudaEventRecord(p.a, s);
    S.pending.push_back(p);
    slot_ = (int)S.pending.size() - 1;
  }
}

ProfScope::~ProfScope() {
  if (slot_ < 0) return;
  State& S = st();
  std::lock_guard<std::mutex> g(S.mu);
  if (slot_ < (int)S.pending.size()) cudaEventRecord(S.pending[slot_].b, s_);
}

void prof_count(int kind, double flops, double bytes) {
  State& S = st();
  std::lock_guard<std::mutex> g(S.mu);
  S.acc[kind].launches++;
  S.acc[kind].flops += flops;
  S.acc[kind].bytes += bytes;
}

void prof_capture(bool on) { t_capturing = on; }

void prof_reset(int timing) {
  State& S = st();
  std::lock_guard<std::mutex> g(S.mu);
  drain(S);
  for (auto& a : S.acc) a = Acc();
  S.timing = timing;
  S.next_flops = S.next_bytes = 0;
}

int prof_read(int kind, long long* launches, double* ms, double* flops, double* bytes) {
  if (kind < 0 || kind >= P_NKINDS) return -1;
  State& S = st();
  std::lock_guard<std::mutex> g(S.mu);
  drain(S);
  const Acc& a = S.acc[kind];
  if (launches) *launches = a.launches;
  if (ms) *ms = a.ms;
  if (flops) *flops = a.flops;
  if (bytes) *bytes = a.bytes;
  return 0;
}

const char* prof_name(int kind) {
  static const char* n[P_NKINDS] = {"k_gemm",   "k_diag",     "k_copy", "k_qrcp", "k_gemv_n", "k_gemv_t",
                                    "k_veccopy", "k_assemble", "k_spmv", "k_dot",  "k_vector", "apply"};
  return (kind >= 0 && kind < P_NKINDS) ? n[kind] : "?";
}

}  // namespace sgf
