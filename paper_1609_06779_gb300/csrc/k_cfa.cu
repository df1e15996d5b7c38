// CFA kernels: launcher dispatching to the per-precision translation units.
#include "fd_launch.h"

namespace fdk {

cudaError_t launch_cfa_f64(const KArgs &a, int team, cudaStream_t s);
cudaError_t launch_cfa_f32(const KArgs &a, int team, cudaStream_t s);
cudaError_t launch_cfa_mixed(const KArgs &a, int team, cudaStream_t s);
cudaError_t launch_cfa_w_f64(const KArgs &a, int team, cudaStream_t s);
cudaError_t launch_cfa_w_f32(const KArgs &a, int team, cudaStream_t s);
cudaError_t launch_cfa_cr_f64(const KArgs &a, int team, cudaStream_t s);
cudaError_t launch_cfa_cr_f32(const KArgs &a, int team, cudaStream_t s);
cudaError_t launch_cfa_cr_mixed(const KArgs &a, int team, cudaStream_t s);
cudaError_t launch_cfa2_f64(const KArgs &a, int team, cudaStream_t s);
cudaError_t launch_cfa2_f32(const KArgs &a, int team, cudaStream_t s);
cudaError_t launch_cfa2_mixed(const KArgs &a, int team, cudaStream_t s);
cudaError_t launch_cfa_cr2_f64(const KArgs &a, int team, cudaStream_t s);
cudaError_t launch_cfa_cr2_f32(const KArgs &a, int team, cudaStream_t s);
cudaError_t launch_cfa_cr2_mixed(const KArgs &a, int team, cudaStream_t s);

cudaError_t launch_cfa(const KArgs &a, int prec, int team, cudaStream_t s) {
  if (a.mode == MODE_FD2) {
    switch (prec) {
      case 0: return launch_cfa2_f64(a, team, s);
      case 1: return launch_cfa2_f32(a, team, s);
      case 2: return launch_cfa2_mixed(a, team, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (prec) {
    case 0: return launch_cfa_f64(a, team, s);
    case 1: return launch_cfa_f32(a, team, s);
    case 2: return launch_cfa_mixed(a, team, s);
    default: return cudaErrorInvalidValue;
  }
}

// CFA with a general projection (a.wmode, a.wq): FP64 and FP32
cudaError_t launch_cfa_w(const KArgs &a, int prec, int team, cudaStream_t s) {
  switch (prec) {
    case 0: return launch_cfa_w_f64(a, team, s);
    case 1: return launch_cfa_w_f32(a, team, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_cfa_cr(const KArgs &a, int prec, int team, cudaStream_t s) {
  if (a.mode == MODE_FD2) {
    switch (prec) {
      case 0: return launch_cfa_cr2_f64(a, team, s);
      case 1: return launch_cfa_cr2_f32(a, team, s);
      case 2: return launch_cfa_cr2_mixed(a, team, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (prec) {
    case 0: return launch_cfa_cr_f64(a, team, s);
    case 1: return launch_cfa_cr_f32(a, team, s);
    case 2: return launch_cfa_cr_mixed(a, team, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_cfa_multi_f64(const KArgs &a, const ClassTable &ct, cudaStream_t s);
cudaError_t launch_cfa_multi_f32(const KArgs &a, const ClassTable &ct, cudaStream_t s);
cudaError_t launch_cfa_multi_mixed(const KArgs &a, const ClassTable &ct, cudaStream_t s);
cudaError_t launch_cfa_cr_multi_f64(const KArgs &a, const ClassTable &ct, cudaStream_t s);
cudaError_t launch_cfa_cr_multi_f32(const KArgs &a, const ClassTable &ct, cudaStream_t s);
cudaError_t launch_cfa_cr_multi_mixed(const KArgs &a, const ClassTable &ct, cudaStream_t s);

cudaError_t launch_cfa_hy_f64(const KArgs &a, int team, cudaStream_t s);
cudaError_t launch_cfa_hy_f32(const KArgs &a, int team, cudaStream_t s);
cudaError_t launch_cfa_hy_mixed(const KArgs &a, int team, cudaStream_t s);
cudaError_t launch_cfa_hy_multi_f64(const KArgs &a, const ClassTable &ct, cudaStream_t s);
cudaError_t launch_cfa_hy_multi_f32(const KArgs &a, const ClassTable &ct, cudaStream_t s);
cudaError_t launch_cfa_hy_multi_mixed(const KArgs &a, const ClassTable &ct, cudaStream_t s);

cudaError_t launch_cfa_hy(const KArgs &a, int prec, int team, cudaStream_t s) {
  switch (prec) {
    case 0: return launch_cfa_hy_f64(a, team, s);
    case 1: return launch_cfa_hy_f32(a, team, s);
    case 2: return launch_cfa_hy_mixed(a, team, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_cfa_hy_multi(const KArgs &a, int prec, const ClassTable &ct, cudaStream_t s) {
  switch (prec) {
    case 0: return launch_cfa_hy_multi_f64(a, ct, s);
    case 1: return launch_cfa_hy_multi_f32(a, ct, s);
    case 2: return launch_cfa_hy_multi_mixed(a, ct, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_cfa_multi(const KArgs &a, int prec, const ClassTable &ct, cudaStream_t s) {
  switch (prec) {
    case 0: return launch_cfa_multi_f64(a, ct, s);
    case 1: return launch_cfa_multi_f32(a, ct, s);
    case 2: return launch_cfa_multi_mixed(a, ct, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_cfa_cr_multi(const KArgs &a, int prec, const ClassTable &ct, cudaStream_t s) {
  switch (prec) {
    case 0: return launch_cfa_cr_multi_f64(a, ct, s);
    case 1: return launch_cfa_cr_multi_f32(a, ct, s);
    case 2: return launch_cfa_cr_multi_mixed(a, ct, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fdk
