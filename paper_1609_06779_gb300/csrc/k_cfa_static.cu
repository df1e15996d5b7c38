// k_cfa_static.cu -- fd_solve_cfa_static: the CFA solve with no allocation at
// all. Its scratch is a file-scope device array, so a caller that must not call
// cudaMalloc at solve time can still run CFA on chains it created earlier.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "fd_internal.h"
#include "fd_launch.h"
#include "fd_layout.h"

namespace {

// 32 MiB per device, all of it CFA workspace. At FP64 the workspace needs
// 32 x 8 + 196 x 8 = 1 824 bytes per link (about 18 000 links); mixed
// 32 x 4 + 196 x 8 = 1 696 (about 19 000); FP32 32 x 4 + 196 x 4 = 912 (about
// 36 000). Problem p is chain p, so no problem map is needed (the kernels read a
// null map as the identity).
constexpr size_t kScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char *g_base[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Once per device, with that device current: the device address of g_scratch
// (in host code its name is only a stand-in for the device array). Nothing is
// copied to the device, so there is nothing to wait for.
fd_status setup(int dev, unsigned char **base) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_base[dev]) {
    *base = g_base[dev];
    return FD_OK;
  }
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char msg[256];
    snprintf(msg, sizeof msg, "fd_solve_cfa_static: cudaGetSymbolAddress: %s",
             cudaGetErrorString(e));
    return fdk_fail(FD_ERR_CUDA, msg);
  }
  g_base[dev] = static_cast<unsigned char *>(p);
  *base = g_base[dev];
  return FD_OK;
}

}  // namespace

extern "C" fd_status fd_solve_cfa_static(fd_chain_t chain, const void *q, const void *qdot,
                                         const void *tau, void *qddot, fd_prec prec,
                                         int32_t team, int32_t *status, void *stream) {
  if (!chain) return fdk_fail(FD_ERR_INVALID_ARG, "fd_solve_cfa_static: NULL chain");
  if (chain->d_parent)
    return fdk_fail(FD_ERR_UNSUPPORTED, "fd_solve_cfa_static: serial chains only (not trees)");
  if (prec != FD_FP64 && prec != FD_FP32 && prec != FD_MIXED)
    return fdk_fail(FD_ERR_INVALID_ARG, "fd_solve_cfa_static: bad precision");
  if (team < 0 || (team > 0 && !fdk_valid_team(team)))
    return fdk_fail(FD_ERR_INVALID_ARG,
                    "fd_solve_cfa_static: team is not 0 or a power of two <= 256");
  if (chain->n_chains == 0 || chain->n_links == 0) return FD_OK;
  if (!q || !qdot || !tau || !qddot)
    return fdk_fail(FD_ERR_INVALID_ARG, "fd_solve_cfa_static: NULL state array");
  const size_t ts = prec == FD_FP64 ? 8 : 4, as = prec == FD_FP32 ? 4 : 8;
  const size_t L = static_cast<size_t>(chain->n_links);
  const size_t t_bytes = align256(L * fdk::NT * ts);
  const size_t need = t_bytes + align256(L * fdk::NA_CFA * as);
  if (need > kScratchBytes) {
    char msg[320];
    snprintf(msg, sizeof msg,
             "fd_solve_cfa_static: %d chains / %lld links need %zu bytes of scratch; the "
             "static scratch holds %zu bytes (use fd_solve_batch with a workspace for "
             "larger sets)",
             chain->n_chains, static_cast<long long>(chain->n_links), need, kScratchBytes);
    return fdk_fail(FD_ERR_INVALID_ARG, msg);
  }
  if (chain->device >= kMaxDevices)
    return fdk_fail(FD_ERR_INVALID_ARG, "fd_solve_cfa_static: device index too large");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(chain->device);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fdk_fail(FD_ERR_CUDA, "fd_solve_cfa_static: cudaSetDevice");
  }
  unsigned char *base = nullptr;
  fd_status st = setup(chain->device, &base);
  if (st != FD_OK) {
    cudaSetDevice(prev);
    return st;
  }
  // team 0: the same default as fd_solve_batch with an untuned batch plan
  const int t = team > 0 ? team : fdk_default_team(FD_CFA, chain->n_chains, chain->max_links);
  fdk::KArgs a{};
  a.model = prec == FD_FP64 ? chain->d_model64 : chain->d_model32;
  a.model64 = chain->d_model64;
  a.model_off = chain->d_off;
  a.prob_chain = nullptr;  // problem p is chain p
  a.state_off = chain->d_off;
  a.sq_off = chain->d_off;
  a.order = nullptr;
  a.n_problems = chain->n_chains;
  a.team = t;
  a.q = q;
  a.qd = qdot;
  a.in3 = tau;
  a.out = qddot;
  a.ws_t = base;
  a.ws_a = base + t_bytes;
  a.status = status;
  for (int k = 0; k < 3; ++k) a.grav[k] = chain->grav[k];
  const int prec_k = prec == FD_FP64 ? 0 : (prec == FD_FP32 ? 1 : 2);
  e = fdk::launch_cfa(a, prec_k, t, static_cast<cudaStream_t>(stream));
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char msg[256];
    snprintf(msg, sizeof msg, "fd_solve_cfa_static: launch: %s", cudaGetErrorString(e));
    return fdk_fail(FD_ERR_CUDA, msg);
  }
  return FD_OK;
}
