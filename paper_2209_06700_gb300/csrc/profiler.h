// Per-category launch accounting of libirk: every kernel launch is counted, and
// launches of the categories selected by irk_profile's mask are bracketed by CUDA
// events on the handle's stream (device time, read back by irk_profile_read).
#pragma once
#include <cuda_runtime.h>

#include <vector>

namespace irk {

enum ProfCat {
  PROF_APPLY64 = 0,   // FP64-accurate stage operator kernel of Eq. (irk:A) (M and K of every stage)
  PROF_MG_OP = 1,     // multigrid level-operator kernels on the coarser levels
  PROF_MG_POINT = 2,  // first Chebyshev step from zero (pointwise)
  PROF_TRANSFER = 3,  // restriction / prolongation passes
  PROF_COARSE = 4,    // dense coarse solve
  PROF_COMBINE = 5,   // stage combinations (A^{-1}, S~, S~^{-1}, T, casts)
  PROF_KRYLOV = 6,    // FGMRES vector kernels (dots, axpys, norms, scaling)
  PROF_RHS = 7,       // K y_n, stage right-hand side and solution update
  PROF_MG_OP_FINE = 8,  // multigrid level-operator kernels on the finest level
  PROF_NCAT = 9
};

struct Profiler {
  cudaStream_t st = nullptr;
  unsigned mask = 0;
  long long launches[PROF_NCAT] = {};
  std::vector<cudaEvent_t> ev;  // pairs (start, stop)
  std::vector<int> ev_cat;
  size_t used = 0;              // pairs in use
  ~Profiler();
  void reset(unsigned new_mask);
  void start(int cat, cudaEvent_t* stop_out);
  void read(int cat, double* ms, long long* n_launches, long long* n_timed);
};

extern thread_local Profiler* g_prof;

class ProfScope {
 public:
  explicit ProfScope(int cat) : stop_(nullptr) {
    if (g_prof) g_prof->start(cat, &stop_);
  }
  ~ProfScope() {
    if (stop_) cudaEventRecord(stop_, g_prof->st);
  }
 private:
  cudaEvent_t stop_;
};

class ProfBind {
 public:
  explicit ProfBind(Profiler* p) : prev_(g_prof) { g_prof = p; }
  ~ProfBind() { g_prof = prev_; }
 private:
  Profiler* prev_;
};

}  // namespace irk

#define IRK_LAUNCH(cat, ...)            \
  do {                                  \
    ::irk::ProfScope ps_(cat);          \
    IRK_CUDA(__VA_ARGS__);              \
  } while (0)
