// Registry of the autotuned operator launch shapes (host side of tune_op).
#include <atomic>
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

// Forced launch shape and the shape of the last 3D launch, per element size (index 0: 4-byte FP32
// multigrid kernels, 1: 8-byte FP64-accurate kernels).  Packed as cxs | zc << 8 | cluster << 24 |
// nch << 32 so that one atomic word holds a consistent shape; 0 = none.
namespace {
std::atomic<long long> g_force[2] = {{0}, {0}};
std::atomic<long long> g_last[2] = {{0}, {0}};
int slot(int elem) { return elem == 4 ? 0 : 1; }
long long pack(int cxs, int zc, int cluster, int nch) {
  return (long long)cxs | ((long long)zc << 8) | ((long long)cluster << 24) | ((long long)nch << 32);
}
void unpack(long long v, int* out4) {
  out4[0] = (int)(v & 0xff);
  out4[1] = (int)((v >> 8) & 0xffff);
  out4[2] = (int)((v >> 24) & 0xff);
  out4[3] = (int)((v >> 32) & 0xffff);
}
}  // namespace

void op_shape_force(int elem, int cxs, int zc, int cluster) {
  g_force[slot(elem)].store(cxs > 0 ? pack(cxs, zc, cluster, 0) : 0);
}

bool op_shape_forced(int elem, int* cxs, int* zc, int* cluster) {
  const long long v = g_force[slot(elem)].load();
  if (!v) return false;
  int s[4];
  unpack(v, s);
  *cxs = s[0];
  *zc = s[1];
  *cluster = s[2];
  return true;
}

void op_shape_record(int elem, int cxs, int zc, int cluster, int nch) {
  g_last[slot(elem)].store(pack(cxs, zc, cluster, nch));
}

bool op_shape_last(int elem, int* out4) {
  const long long v = g_last[slot(elem)].load();
  if (!v) return false;
  unpack(v, out4);
  return true;
}

}  // namespace irk
