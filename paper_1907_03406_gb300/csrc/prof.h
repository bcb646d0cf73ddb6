// Launch accounting for the benchmark: per kernel kind, the number of
// launches, the algorithmic flops / bytes the host attached to them and, when
// timing is on, their device time from CUDA events recorded on the launching
// stream around each launch.
#pragma once

#include <cuda_runtime.h>

namespace sgf {

enum ProfKind {
  P_GEMM = 0, P_DIAG, P_COPY, P_QR, P_GEMV_N, P_GEMV_T, P_VECCOPY, P_ASSEMBLE, P_SPMV, P_DOT,
  P_VEC,
  P_APPLY,   // one replay of an apply program's graph (its kernels are counted under their own kinds)
  P_NKINDS
};

// work of the next launch (set by the code that built its tasks)
void prof_work(double flops, double bytes);
// a description of the next launch, printed beside it in the launch log
// (SGF_PROF_LOG); copied
void prof_note(const char* note);
// whether the launch log is on
bool prof_logging();

class ProfScope {
 public:
  ProfScope(int kind, cudaStream_t s);
  ~ProfScope();

 private:
  int kind_;
  cudaStream_t s_;
  int slot_;
};

// one launch of a replayed graph node: counted, not timed
void prof_count(int kind, double flops, double bytes);
// while a stream capture records launches, they are neither counted nor timed
void prof_capture(bool on);

// timing: 0 none, 1 every launch, 2 the factor contractions (GEMM, fronts, QR)
// and the apply graph replays
void prof_reset(int timing);
int prof_read(int kind, long long* launches, double* ms, double* flops, double* bytes);
const char* prof_name(int kind);

}  // namespace sgf
