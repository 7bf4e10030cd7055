// Per-category launch accounting (see profiler.h).
#include "profiler.h"

namespace irk {

thread_local Profiler* g_prof = nullptr;

Profiler::~Profiler() {
  for (auto e : ev) cudaEventDestroy(e);
}

void Profiler::reset(unsigned new_mask) {
  mask = new_mask;
  for (auto& l : launches) l = 0;
  used = 0;
  ev_cat.clear();
}

void Profiler::start(int cat, cudaEvent_t* stop_out) {
  launches[cat] += 1;
  *stop_out = nullptr;
  if (!(mask & (1u << cat))) return;
  if (2 * (used + 1) > ev.size()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      ev.push_back(e);
    }
  }
  cudaEvent_t a = ev[2 * used], b = ev[2 * used + 1];
  ev_cat.push_back(cat);
  ++used;
  cudaEventRecord(a, st);
  *stop_out = b;
}

void Profiler::read(int cat, double* ms, long long* n_launches, long long* n_timed) {
  double total = 0.0;
  long long timed = 0;
  for (size_t i = 0; i < used; ++i) {
    if (ev_cat[i] != cat) continue;
    float t = 0.f;
    cudaEventSynchronize(ev[2 * i + 1]);
    if (cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]) == cudaSuccess) {
      total += t;
      ++timed;
    }
  }
  if (ms) *ms = total;
  if (n_launches) *n_launches = launches[cat];
  if (n_timed) *n_timed = timed;
}

}  // namespace irk
