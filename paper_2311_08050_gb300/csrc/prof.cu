// Launch counting and a light per-kernel profiler (test hooks of include/inla_testing.h).
// While enabled, a CUDA event is recorded on the evaluation stream before every kernel the
// library launches; the time between consecutive events is attributed to the kernel that was
// launched at the first of them (one stream: kernels run in launch order).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>
#include "internal.h"

namespace inla {

namespace {
struct ProfEvent {
  cudaEvent_t ev;
  const char* kernel;
  const char* phase;  // the phase mark in force when the kernel was launched ("" before any)
};
struct Prof {
  bool on = false;
  cudaStream_t st = nullptr;
  const char* phase = "";
  std::vector<ProfEvent> ev;
  std::vector<std::pair<cudaEvent_t, const char*>> phases;  // phase boundaries of a batch
};
Prof g_prof;
}  // namespace

void prof_set_stream(cudaStream_t st) { g_prof.st = st; }
bool prof_active() { return g_prof.on; }

int count_launch(const char* name) {
  ++g_kernel_launches;
  if (g_prof.on) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) == cudaSuccess) {
      cudaEventRecord(e, g_prof.st);
      g_prof.ev.push_back({e, name, g_prof.phase});
    }
  }
  return 0;
}

void prof_phase(const char* name) {
  if (!g_prof.on) return;
  g_prof.phase = name;
  cudaEvent_t e;
  if (cudaEventCreate(&e) == cudaSuccess) {
    cudaEventRecord(e, g_prof.st);
    g_prof.phases.push_back({e, name});
  }
}

}  // namespace inla

using namespace inla;

// Writes "name count total_ms\n" lines, in order of first appearance, for the phases of the
// batches run while the profiler was on (a phase lasts until the next phase mark or the read).
extern "C" int inla_test_phase_read(char* buf, int len) {
  if (!buf || len <= 0) return INLA_E_BADARG;
  buf[0] = 0;
  if (g_prof.phases.empty()) return 0;
  cudaEvent_t last;
  if (cudaEventCreate(&last) != cudaSuccess) return INLA_E_CUDA;
  cudaEventRecord(last, g_prof.st);
  cudaEventSynchronize(last);
  std::vector<std::string> order;
  std::map<std::string, std::pair<long, double>> acc;
  for (size_t i = 0; i < g_prof.phases.size(); ++i) {
    cudaEvent_t next = i + 1 < g_prof.phases.size() ? g_prof.phases[i + 1].first : last;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g_prof.phases[i].first, next);
    const std::string nm = g_prof.phases[i].second;
    if (!acc.count(nm)) order.push_back(nm);
    auto& a = acc[nm];
    a.first += 1;
    a.second += ms;
  }
  for (auto& p : g_prof.phases) cudaEventDestroy(p.first);
  cudaEventDestroy(last);
  g_prof.phases.clear();
  int off = 0;
  for (auto& nm : order) {
    const int w = snprintf(buf + off, len - off, "%s %ld %.4f\n", nm.c_str(), acc[nm].first, acc[nm].second);
    if (w < 0 || w >= len - off) break;
    off += w;
  }
  return off;
}


extern "C" void inla_test_profile_enable(int on) {
  g_prof.on = on != 0;
  g_prof.phase = "";
}

// Writes "name launches total_ms\n" lines (largest total first) into buf; returns the
// number of bytes written (0 if nothing was recorded), or a negative status.
// by_phase: key "phase/kernel" instead of "kernel"
static int profile_read(char* buf, int len, bool by_phase) {
  if (!buf || len <= 0) return INLA_E_BADARG;
  buf[0] = 0;
  if (g_prof.ev.empty()) return 0;
  cudaEvent_t last;
  if (cudaEventCreate(&last) != cudaSuccess) return INLA_E_CUDA;
  cudaEventRecord(last, g_prof.st);
  cudaEventSynchronize(last);
  std::map<std::string, std::pair<long, double>> acc;
  for (size_t i = 0; i < g_prof.ev.size(); ++i) {
    cudaEvent_t next = i + 1 < g_prof.ev.size() ? g_prof.ev[i + 1].ev : last;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g_prof.ev[i].ev, next);
    const std::string key = by_phase ? std::string(g_prof.ev[i].phase) + "/" + g_prof.ev[i].kernel
                                     : std::string(g_prof.ev[i].kernel);
    auto& a = acc[key];
    a.first += 1;
    a.second += ms;
  }
  for (auto& p : g_prof.ev) cudaEventDestroy(p.ev);
  cudaEventDestroy(last);
  g_prof.ev.clear();
  std::vector<std::pair<std::string, std::pair<long, double>>> v(acc.begin(), acc.end());
  std::sort(v.begin(), v.end(), [](const auto& a, const auto& b) { return a.second.second > b.second.second; });
  int off = 0;
  for (auto& e : v) {
    const int w = snprintf(buf + off, len - off, "%s %ld %.4f\n", e.first.c_str(), e.second.first, e.second.second);
    if (w < 0 || w >= len - off) break;
    off += w;
  }
  return off;
}

extern "C" int inla_test_profile_read(char* buf, int len) { return profile_read(buf, len, false); }
extern "C" int inla_test_profile_read_by_phase(char* buf, int len) { return profile_read(buf, len, true); }
