// Registry of the autotuned operator launch shapes (host side of tune_op).
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"

namespace irk {

namespace {
std::mutex g_tune_mu;
std::vector<std::string> g_tune_lines;
}  // namespace

void tune_record(const char* kernel, int k, int epi, int N, int nstage, int cxs, int zc, int cluster, double us,
                 double us_model, int model_cxs, int model_zc, int model_cluster) {
  static const char* epis[] = {"store", "dual", "resid", "cheb"};
  char line[256];
  std::snprintf(line, sizeof(line),
                "%s k=%d %s N=%d stages=%d: cxs=%d zc=%d cluster=%d %.2f us (model cxs=%d zc=%d cluster=%d %.2f us)",
                kernel, k, (epi >= 0 && epi < 4) ? epis[epi] : "?", N, nstage, cxs, zc, cluster, us, model_cxs,
                model_zc, model_cluster, us_model);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_lines.emplace_back(line);
}

int tune_report(char* buf, int len) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  std::string all;
  for (const auto& l : g_tune_lines) {
    all += l;
    all += '\n';
  }
  if (buf && len > 0) {
    const size_t n = std::min((size_t)(len - 1), all.size());
    std::memcpy(buf, all.data(), n);
    buf[n] = '\0';
  }
  return (int)all.size();
}

}  // namespace irk
