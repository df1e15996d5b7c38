// fd_abi.cu -- the C ABI declared in include/fd_gb300.h: model packing (chain
// sets in canonical link frames), batch plans, argument validation and kernel
// dispatch. Host code only; the arithmetic of the method runs in the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/fd_gb300.h"
#include "fd_internal.h"
#include "fd_launch.h"
#include "fd_layout.h"

namespace {

thread_local std::string g_err;

fd_status fail(fd_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

fd_status cuda_fail(cudaError_t e, const char *what) {
  cudaGetLastError();  // the status carries the error; do not leave it for the caller's runtime
  return fail(e == cudaErrorMemoryAllocation ? FD_ERR_OOM : FD_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

// packed symmetric 6x6 index (upper triangle row by row), as in the kernels
constexpr int s6(int i, int j) {
  return i <= j ? i * 6 - (i * (i - 1)) / 2 + (j - i) : j * 6 - (j * (j - 1)) / 2 + (i - j);
}

// Cholesky of a dense 6x6 (row-major); false if not positive definite.
bool chol6(const double *A, double *L) {
  std::memset(L, 0, 36 * sizeof(double));
  for (int j = 0; j < 6; ++j) {
    double d = A[6 * j + j];
    for (int k = 0; k < j; ++k) d -= L[6 * j + k] * L[6 * j + k];
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    L[6 * j + j] = std::sqrt(d);
    for (int i = j + 1; i < 6; ++i) {
      double s = A[6 * i + j];
      for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
      L[6 * i + j] = s / L[6 * j + j];
    }
  }
  return true;
}

void inv_from_chol6(const double *L, double *Ai) {
  for (int c = 0; c < 6; ++c) {
    double x[6] = {0, 0, 0, 0, 0, 0};
    x[c] = 1.0;
    for (int i = 0; i < 6; ++i) {
      double s = x[i];
      for (int k = 0; k < i; ++k) s -= L[6 * i + k] * x[k];
      x[i] = s / L[6 * i + i];
    }
    for (int i = 5; i >= 0; --i) {
      double s = x[i];
      for (int k = i + 1; k < 6; ++k) s -= L[6 * k + i] * x[k];
      x[i] = s / L[6 * i + i];
    }
    for (int i = 0; i < 6; ++i) Ai[6 * i + c] = x[i];
  }
}

// Q with first column a (unit): a right-handed frame whose x axis is the joint axis.
void axis_frame(const double *a, double *Q) {
  int m = 0;
  if (std::fabs(a[1]) < std::fabs(a[m])) m = 1;
  if (std::fabs(a[2]) < std::fabs(a[m])) m = 2;
  double e[3] = {0, 0, 0};
  e[m] = 1.0;
  const double d = e[0] * a[0] + e[1] * a[1] + e[2] * a[2];
  double b[3] = {e[0] - d * a[0], e[1] - d * a[1], e[2] - d * a[2]};
  const double nb = std::sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
  for (double &v : b) v /= nb;
  const double c[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2],
                       a[0] * b[1] - a[1] * b[0]};
  for (int r = 0; r < 3; ++r) {
    Q[3 * r + 0] = a[r];
    Q[3 * r + 1] = b[r];
    Q[3 * r + 2] = c[r];
  }
}

void m3_mul(const double *A, const double *B, double *C) {
  double T[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      T[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
  std::memcpy(C, T, sizeof T);
}

void m3_tmul(const double *A, const double *B, double *C) {  // A^T B
  double T[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      T[3 * i + j] = A[i] * B[j] + A[3 + i] * B[3 + j] + A[6 + i] * B[6 + j];
  std::memcpy(C, T, sizeof T);
}

int pow2_floor(long long v) {
  int p = 1;
  while (2LL * p <= v) p *= 2;
  return p;
}

}  // namespace

// Re-expresses one chain (links first .. first+n-1 of the packed user arrays) in
// canonical link frames (x axis = joint axis) and writes its model records to
// rec[0 .. n*REC). Clears *rigid if an inertia is not of the rigid-body form.
fd_status fdk_pack_chain(int64_t first, int64_t n, const double *joint_axes,
                         const double *link_frames, const double *spatial_inertias, double *rec,
                         bool *rigid, const int32_t *parents) {
  // the canonical rotation of every link of this chain: a child's home
  // transform is re-expressed between its parent's canonical frame and its own
  std::vector<double> Qs(static_cast<size_t>(std::max<int64_t>(n, 1)) * 9);
  for (int64_t i = first; i < first + n; ++i) {
    const int64_t par = parents ? parents[i] : i - first - 1;
    double Qprev[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (par >= 0) std::memcpy(Qprev, Qs.data() + 9 * par, sizeof Qprev);
    const double *ax = joint_axes + 3 * i;
    const double *fr = link_frames + 12 * i;
    const double *J = spatial_inertias + 36 * i;
    const double na = std::sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
    if (!(na > 1e-12) || !std::isfinite(na))
      return fail(FD_ERR_INVALID_ARG, "fd_create_chain: link %lld has a zero joint axis",
                  static_cast<long long>(i));
    const double a[3] = {ax[0] / na, ax[1] / na, ax[2] / na};
    double RtR[9];
    m3_tmul(fr, fr, RtR);
    for (int r = 0; r < 9; ++r)
      if (!(std::fabs(RtR[r] - (r % 4 == 0 ? 1.0 : 0.0)) < 1e-9))
        return fail(FD_ERR_INVALID_ARG, "fd_create_chain: link %lld frame is not a rotation",
                    static_cast<long long>(i));
    const double det = fr[0] * (fr[4] * fr[8] - fr[5] * fr[7]) -
                       fr[1] * (fr[3] * fr[8] - fr[5] * fr[6]) +
                       fr[2] * (fr[3] * fr[7] - fr[4] * fr[6]);
    if (!(det > 0.0))
      return fail(FD_ERR_INVALID_ARG, "fd_create_chain: link %lld frame has det <= 0",
                  static_cast<long long>(i));
    double scale = 0.0;
    for (int r = 0; r < 36; ++r) scale = std::max(scale, std::fabs(J[r]));
    for (int r = 0; r < 6; ++r)
      for (int c = r + 1; c < 6; ++c)
        if (!(std::fabs(J[6 * r + c] - J[6 * c + r]) <= 1e-9 * scale))
          return fail(FD_ERR_INVALID_ARG, "fd_create_chain: link %lld inertia not symmetric",
                      static_cast<long long>(i));
    double Q[9];
    axis_frame(a, Q);
    // R0' = Qprev^T R0 Q, p0' = Qprev^T p0
    double t[9], R0c[9], p0c[3];
    m3_mul(fr, Q, t);
    m3_tmul(Qprev, t, R0c);
    for (int r = 0; r < 3; ++r)
      p0c[r] = Qprev[r] * fr[9] + Qprev[3 + r] * fr[10] + Qprev[6 + r] * fr[11];
    // J' = diag(Q, Q)^T J diag(Q, Q)
    double B[36] = {0};
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) B[6 * r + c] = B[6 * (r + 3) + c + 3] = Q[3 * r + c];
    double JB[36], Jc[36];
    for (int r = 0; r < 6; ++r)
      for (int c = 0; c < 6; ++c) {
        double s = 0;
        for (int k2 = 0; k2 < 6; ++k2) s += 0.5 * (J[6 * r + k2] + J[6 * k2 + r]) * B[6 * k2 + c];
        JB[6 * r + c] = s;
      }
    for (int r = 0; r < 6; ++r)
      for (int c = 0; c < 6; ++c) {
        double s = 0;
        for (int k2 = 0; k2 < 6; ++k2) s += B[6 * k2 + r] * JB[6 * k2 + c];
        Jc[6 * r + c] = s;
      }
    {  // rigid-body form: lower-right block m 1, off-diagonal block m c^ (skew)
      const double m = Jc[6 * 3 + 3];
      for (int r = 0; r < 3 && *rigid; ++r)
        for (int cc = 0; cc < 3; ++cc) {
          if (std::fabs(Jc[6 * (3 + r) + 3 + cc] - (r == cc ? m : 0.0)) > 1e-9 * scale)
            *rigid = false;
          if (std::fabs(Jc[6 * r + 3 + cc] + Jc[6 * cc + 3 + r]) > 1e-9 * scale) *rigid = false;
        }
      if (!(m > 0.0)) *rigid = false;
    }
    double Lc[36], Ji[36];
    if (!chol6(Jc, Lc))
      return fail(FD_ERR_INVALID_ARG,
                  "fd_create_chain: link %lld inertia is not positive definite",
                  static_cast<long long>(i));
    inv_from_chol6(Lc, Ji);
    double *rc = rec + static_cast<size_t>(i - first) * fdk::REC;
    std::memcpy(rc + fdk::REC_R0, R0c, 9 * sizeof(double));
    std::memcpy(rc + fdk::REC_P0, p0c, 3 * sizeof(double));
    for (int r = 0; r < 6; ++r)
      for (int c = r; c < 6; ++c) {
        rc[fdk::REC_J + s6(r, c)] = Jc[6 * r + c];
        rc[fdk::REC_JI + s6(r, c)] = 0.5 * (Ji[6 * r + c] + Ji[6 * c + r]);
      }
    std::memcpy(Qs.data() + 9 * (i - first), Q, 9 * sizeof(double));
  }
  return FD_OK;
}

// Records an error message for fd_last_error from the library's other
// translation units.
fd_status fdk_fail(fd_status st, const char *msg) { return fail(st, "%s", msg); }

int fdk_default_team(int32_t algo, int64_t n_problems, int32_t max_links) {
  // the ABI scan: segments of about four links (its lanes do about five times the
  // serial work, so longer segments pay only when the GPU is full)
  if (algo == FD_ABIA_SCAN) {
    int t = 8;
    while (t < 256 && 4 * t < max_links) t *= 2;
    return t;
  }
  // ABIA: one thread per problem once a warp per FP64 unit (152 SMs x 4) is
  // busy with 32 problems each; below that, spread each step over a team of 8
  if (algo == FD_ABIA) return n_problems > 152 * 4 * 8 ? 1 : 8;
  // about four resident warps' worth of lanes per FP64 unit of the GPU
  // (152 SMs x 2048 threads), but no more lanes than links and at most 256
  const long long want = 152LL * 2048;
  long long per = n_problems > 0 ? want / n_problems : 1;
  int p = pow2_floor(std::max<long long>(per, 1));
  int cap = 1;
  while (cap < max_links && cap < 256) cap *= 2;
  return std::min(p, cap);
}

bool fdk_valid_team(int t) {
  return t == 1 || t == 2 || t == 4 || t == 8 || t == 16 || t == 32 || t == 64 || t == 128 ||
         t == 256;
}

extern "C" {

const char *fd_last_error(void) { return g_err.c_str(); }

int32_t fd_abi_version(void) { return FD_ABI_VERSION; }

// fd_create_chain, and fd_create_tree with parents (validated by the caller)
static fd_status create_set(int32_t n_chains, const int64_t *link_offsets,
                            const int32_t *parents, const double *joint_axes,
                            const double *link_frames, const double *spatial_inertias,
                            const double gravity[3], int32_t device, fd_chain_t *out) {
  if (!out) return fail(FD_ERR_INVALID_ARG, "fd_create_chain: out is NULL");
  *out = nullptr;
  if (n_chains < 0) return fail(FD_ERR_INVALID_ARG, "fd_create_chain: n_chains < 0");
  if (!link_offsets || !gravity)
    return fail(FD_ERR_INVALID_ARG, "fd_create_chain: link_offsets or gravity is NULL");
  if (link_offsets[0] != 0)
    return fail(FD_ERR_INVALID_ARG, "fd_create_chain: link_offsets[0] must be 0");
  int32_t max_links = 0;
  for (int32_t k = 0; k < n_chains; ++k) {
    const int64_t len = link_offsets[k + 1] - link_offsets[k];
    if (len < 0 || len > (1 << 20))
      return fail(FD_ERR_INVALID_ARG, "fd_create_chain: chain %d has %lld links", k,
                  static_cast<long long>(len));
    max_links = std::max<int32_t>(max_links, static_cast<int32_t>(len));
  }
  const int64_t L = link_offsets[n_chains];
  if (L > 0 && (!joint_axes || !link_frames || !spatial_inertias))
    return fail(FD_ERR_INVALID_ARG, "fd_create_chain: model array is NULL");
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(gravity[k])) return fail(FD_ERR_INVALID_ARG, "fd_create_chain: gravity");

  // Canonical link frames (joint axis = x axis of the child frame), model records.
  // Chains are independent: pack them on several host threads.
  bool rigid = true;
  std::vector<double> rec64(static_cast<size_t>(std::max<int64_t>(L, 1)) * fdk::REC, 0.0);
  {
    const int hw = static_cast<int>(std::max(1u, std::thread::hardware_concurrency()));
    const int nt = static_cast<int>(std::min<int64_t>(std::min(hw, 32), std::max<int64_t>(L / 65536, 1)));
    std::vector<fd_status> sts(nt, FD_OK);
    std::vector<std::string> msgs(nt);
    std::vector<char> rig(nt, 1);
    std::atomic<int32_t> next{0};
    auto work = [&](int t) {
      bool rg = true;
      for (;;) {
        const int32_t k0 = next.fetch_add(256);
        if (k0 >= n_chains || sts[t] != FD_OK) break;
        for (int32_t k = k0; k < std::min(n_chains, k0 + 256); ++k) {
          const fd_status st = fdk_pack_chain(
              link_offsets[k], link_offsets[k + 1] - link_offsets[k], joint_axes, link_frames,
              spatial_inertias, rec64.data() + static_cast<size_t>(link_offsets[k]) * fdk::REC, &rg,
              parents);
          if (st != FD_OK) {
            sts[t] = st;
            msgs[t] = g_err;
            break;
          }
        }
      }
      rig[t] = rg;
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto &th : pool) th.join();
    for (int t = 0; t < nt; ++t) {
      if (sts[t] != FD_OK) {
        g_err = msgs[t];
        return sts[t];
      }
      rigid = rigid && rig[t];
    }
  }
  std::vector<float> rec32(rec64.size());
  for (size_t k = 0; k < rec64.size(); ++k) rec32[k] = static_cast<float>(rec64[k]);

  int n_dev = 0;
  cudaError_t e = cudaGetDeviceCount(&n_dev);
  if (e != cudaSuccess || n_dev == 0)
    return fail(FD_ERR_CUDA, "fd_create_chain: no CUDA device (%s)", cudaGetErrorString(e));
  if (device < 0 || device >= n_dev)
    return fail(FD_ERR_INVALID_ARG, "fd_create_chain: device %d of %d", device, n_dev);
  int prev = 0;
  cudaGetDevice(&prev);
  if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");

  auto *c = new fd_chain_s();
  c->device = device;
  c->n_chains = n_chains;
  c->n_links = L;
  c->max_links = max_links;
  c->rigid = rigid;
  std::memcpy(c->grav, gravity, sizeof c->grav);
  c->h_off.assign(link_offsets, link_offsets + n_chains + 1);
  const size_t b64 = rec64.size() * sizeof(double), b32 = rec32.size() * sizeof(float);
  const size_t boff = (n_chains + 1) * sizeof(int64_t);
  if ((e = cudaMalloc(&c->d_model64, b64)) != cudaSuccess ||
      (e = cudaMalloc(&c->d_model32, b32)) != cudaSuccess ||
      (e = cudaMalloc(reinterpret_cast<void **>(&c->d_off), boff)) != cudaSuccess ||
      (e = cudaMemcpy(c->d_model64, rec64.data(), b64, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(c->d_model32, rec32.data(), b32, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(c->d_off, link_offsets, boff, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (parents && L > 0 &&
       ((e = cudaMalloc(reinterpret_cast<void **>(&c->d_parent), L * sizeof(int32_t))) !=
            cudaSuccess ||
        (e = cudaMemcpy(c->d_parent, parents, L * sizeof(int32_t), cudaMemcpyHostToDevice)) !=
            cudaSuccess))) {
    cudaFree(c->d_model64);
    cudaFree(c->d_model32);
    cudaFree(c->d_off);
    cudaFree(c->d_parent);
    delete c;
    cudaSetDevice(prev);
    return cuda_fail(e, "fd_create_chain: device copy");
  }
  if (parents && L == 0) {  // an empty tree set: keep it marked as trees
    if ((e = cudaMalloc(reinterpret_cast<void **>(&c->d_parent), sizeof(int32_t))) != cudaSuccess) {
      cudaFree(c->d_model64);
      cudaFree(c->d_model32);
      cudaFree(c->d_off);
      delete c;
      cudaSetDevice(prev);
      return cuda_fail(e, "fd_create_tree: device allocation");
    }
  }
  if (parents) {
    c->h_axes.assign(joint_axes, joint_axes + 3 * L);
    c->h_parent.assign(parents, parents + L);
  }
  cudaSetDevice(prev);
  *out = c;
  return FD_OK;
}

fd_status fd_create_chain(int32_t n_chains, const int64_t *link_offsets, const double *joint_axes,
                          const double *link_frames, const double *spatial_inertias,
                          const double gravity[3], int32_t device, fd_chain_t *out) {
  return create_set(n_chains, link_offsets, nullptr, joint_axes, link_frames, spatial_inertias,
                    gravity, device, out);
}

fd_status fd_create_tree(int32_t n_trees, const int64_t *link_offsets, const int32_t *parents,
                         const double *joint_axes, const double *link_frames,
                         const double *spatial_inertias, const double gravity[3], int32_t device,
                         fd_chain_t *out) {
  if (!out) return fail(FD_ERR_INVALID_ARG, "fd_create_tree: out is NULL");
  *out = nullptr;
  if (n_trees < 0 || !link_offsets)
    return fail(FD_ERR_INVALID_ARG, "fd_create_tree: n_trees < 0 or link_offsets is NULL");
  if (link_offsets[0] != 0)
    return fail(FD_ERR_INVALID_ARG, "fd_create_tree: link_offsets[0] must be 0");
  for (int32_t k = 0; k < n_trees; ++k) {
    const int64_t a = link_offsets[k], z = link_offsets[k + 1];
    if (z < a) return fail(FD_ERR_INVALID_ARG, "fd_create_tree: tree %d has %lld links", k,
                           static_cast<long long>(z - a));
    if (z > a && !parents) return fail(FD_ERR_INVALID_ARG, "fd_create_tree: parents is NULL");
    for (int64_t i = a; i < z; ++i)
      if (parents[i] < -1 || parents[i] >= i - a)
        return fail(FD_ERR_INVALID_ARG,
                    "fd_create_tree: link %lld of tree %d has parent %d (need -1 <= parent < "
                    "its own index in the tree)", static_cast<long long>(i - a), k, parents[i]);
  }
  static const int32_t none = 0;
  return create_set(n_trees, link_offsets, parents ? parents : &none, joint_axes, link_frames,
                    spatial_inertias, gravity, device, out);
}

fd_status fd_destroy_chain(fd_chain_t c) {
  if (!c) return fail(FD_ERR_INVALID_ARG, "fd_destroy_chain: NULL");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(c->device);
  cudaFree(c->d_model64);
  cudaFree(c->d_model32);
  cudaFree(c->d_off);
  cudaFree(c->d_parent);
  cudaFree(c->d_loop_off);
  cudaFree(c->d_loop_ab);
  cudaFree(c->d_loop_T);
  cudaSetDevice(prev);
  cudaGetLastError();  // leave no error state behind for other users of the runtime
  delete c;
  return FD_OK;
}

fd_status fd_tree_add_loops(fd_chain_t c, int32_t n_loops, const int32_t *loop_tree,
                            const int32_t *link_a, const int32_t *link_b, const double *frame_a,
                            const double *frame_b) {
  const char *who = "fd_tree_add_loops";
  if (!c) return fail(FD_ERR_INVALID_ARG, "%s: NULL chain set", who);
  if (!c->d_parent) return fail(FD_ERR_INVALID_ARG, "%s: not a set of kinematic trees", who);
  if (c->n_loops > 0) return fail(FD_ERR_INVALID_ARG, "%s: the set already has its loops", who);
  if (n_loops < 0 || (n_loops > 0 && (!loop_tree || !link_a || !link_b || !frame_a || !frame_b)))
    return fail(FD_ERR_INVALID_ARG, "%s: bad count or NULL array", who);
  if (n_loops == 0) return FD_OK;
  // loops grouped by tree (stable), frames to canonical link coordinates
  std::vector<int32_t> cnt(static_cast<size_t>(c->n_chains) + 1, 0);
  for (int32_t k = 0; k < n_loops; ++k) {
    const int32_t t = loop_tree[k];
    if (t < 0 || t >= c->n_chains) return fail(FD_ERR_INVALID_ARG, "%s: loop %d: tree %d", who, k, t);
    const int64_t n = c->h_off[t + 1] - c->h_off[t];
    if (link_b[k] < 0 || link_b[k] >= n || link_a[k] < -1 || link_a[k] >= n || link_a[k] == link_b[k])
      return fail(FD_ERR_INVALID_ARG, "%s: loop %d: links %d, %d of a %lld-link tree", who, k,
                  link_a[k], link_b[k], static_cast<long long>(n));
    for (int h = 0; h < 2; ++h) {
      const double *fr = (h ? frame_b : frame_a) + 12 * k;
      double RtR[9];
      m3_tmul(fr, fr, RtR);
      for (int r = 0; r < 9; ++r)
        if (!(std::fabs(RtR[r] - (r % 4 == 0 ? 1.0 : 0.0)) < 1e-9))
          return fail(FD_ERR_INVALID_ARG, "%s: loop %d: a joint frame is not a rotation", who, k);
    }
    if (++cnt[t + 1] > fdk::MAX_LOOPS_PER_TREE)
      return fail(FD_ERR_INVALID_ARG, "%s: tree %d has more than %d loops", who, t,
                  fdk::MAX_LOOPS_PER_TREE);
  }
  for (int32_t t = 0; t < c->n_chains; ++t) cnt[t + 1] += cnt[t];
  std::vector<int32_t> ab(2 * static_cast<size_t>(n_loops));
  std::vector<double> Tc(24 * static_cast<size_t>(n_loops));
  std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
  for (int32_t k = 0; k < n_loops; ++k) {
    const int32_t t = loop_tree[k], at = fill[t]++;
    ab[2 * at] = link_a[k];
    ab[2 * at + 1] = link_b[k];
    for (int h = 0; h < 2; ++h) {
      const int32_t link = h ? link_b[k] : link_a[k];
      const double *fr = (h ? frame_b : frame_a) + 12 * k;
      double *dst = Tc.data() + 24 * at + 12 * h;
      if (link < 0) {  // the base keeps its frame
        std::memcpy(dst, fr, 12 * sizeof(double));
        continue;
      }
      const double *ax = c->h_axes.data() + 3 * (c->h_off[t] + link);
      const double na = std::sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
      const double a3[3] = {ax[0] / na, ax[1] / na, ax[2] / na};
      double Q[9];
      axis_frame(a3, Q);  // user link coordinates = Q canonical ones
      m3_tmul(Q, fr, dst);  // R_c = Q^T R
      for (int r = 0; r < 3; ++r)
        dst[9 + r] = Q[r] * fr[9] + Q[3 + r] * fr[10] + Q[6 + r] * fr[11];  // p_c = Q^T p
    }
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  if ((e = cudaMalloc(reinterpret_cast<void **>(&c->d_loop_off), cnt.size() * sizeof(int32_t))) != cudaSuccess ||
      (e = cudaMalloc(reinterpret_cast<void **>(&c->d_loop_ab), ab.size() * sizeof(int32_t))) != cudaSuccess ||
      (e = cudaMalloc(reinterpret_cast<void **>(&c->d_loop_T), Tc.size() * sizeof(double))) != cudaSuccess ||
      (e = cudaMemcpy(c->d_loop_off, cnt.data(), cnt.size() * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(c->d_loop_ab, ab.data(), ab.size() * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(c->d_loop_T, Tc.data(), Tc.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) {
    cudaFree(c->d_loop_off);
    cudaFree(c->d_loop_ab);
    cudaFree(c->d_loop_T);
    c->d_loop_off = c->d_loop_ab = nullptr;
    c->d_loop_T = nullptr;
    cudaSetDevice(prev);
    return cuda_fail(e, who);
  }
  c->n_loops = n_loops;
  cudaSetDevice(prev);
  return FD_OK;
}

fd_status fd_chain_info(fd_chain_t c, int32_t *n_chains, int64_t *n_links, int32_t *max_links) {
  if (!c) return fail(FD_ERR_INVALID_ARG, "fd_chain_info: NULL chain");
  if (n_chains) *n_chains = c->n_chains;
  if (n_links) *n_links = c->n_links;
  if (max_links) *max_links = c->max_links;
  return FD_OK;
}

fd_status fd_batch_create(fd_chain_t c, int32_t n_problems, const int32_t *chain_index,
                          fd_batch_t *out) {
  if (!out) return fail(FD_ERR_INVALID_ARG, "fd_batch_create: out is NULL");
  *out = nullptr;
  if (!c) return fail(FD_ERR_INVALID_ARG, "fd_batch_create: NULL chain");
  if (n_problems < 0) return fail(FD_ERR_INVALID_ARG, "fd_batch_create: n_problems < 0");
  if (!chain_index && n_problems != c->n_chains)
    return fail(FD_ERR_INVALID_ARG,
                "fd_batch_create: without chain_index n_problems (%d) must equal the number "
                "of chains (%d)", n_problems, c->n_chains);
  std::vector<int32_t> pc(static_cast<size_t>(n_problems));
  std::vector<int64_t> so(static_cast<size_t>(n_problems) + 1, 0), sq(so.size(), 0);
  std::vector<int32_t> len(pc.size());
  int32_t max_links = 0;
  for (int32_t p = 0; p < n_problems; ++p) {
    const int32_t k = chain_index ? chain_index[p] : p;
    if (k < 0 || k >= c->n_chains)
      return fail(FD_ERR_INVALID_ARG, "fd_batch_create: chain_index[%d] = %d out of range", p, k);
    pc[p] = k;
    const int64_t n = c->h_off[k + 1] - c->h_off[k];
    len[p] = static_cast<int32_t>(n);
    max_links = std::max<int32_t>(max_links, static_cast<int32_t>(n));
    so[p + 1] = so[p] + n;
    sq[p + 1] = sq[p] + n * n;
  }
  // longest problems first (a ragged batch then finishes together)
  std::vector<int32_t> order(pc.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t x, int32_t y) { return len[x] > len[y]; });

  // length classes over the processing order (ceil(log2 n) decreases along it)
  std::vector<fd_batch_s::LenClass> classes;
  for (int32_t t = 0; t < n_problems; ++t) {
    const int32_t n = len[order[t]];
    int key = 0;
    while ((1 << key) < n) ++key;
    if (classes.empty() || classes.back().key != key)
      classes.push_back({key, t, 0, n, n});
    auto &cl = classes.back();
    ++cl.count;
    cl.min_len = std::min(cl.min_len, n);
    cl.max_len = std::max(cl.max_len, n);
  }

  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  auto *b = new fd_batch_s();
  b->classes = classes;
  b->ctuned.assign(classes.size() * FD_N_ALGOS * 3, 0);
  b->chain = c;
  b->device = c->device;
  b->n_problems = n_problems;
  b->n_state_links = so.back();
  b->sum_sq = sq.back();
  b->max_links = max_links;
  const size_t np = std::max<size_t>(pc.size(), 1);
  if ((e = cudaMalloc(reinterpret_cast<void **>(&b->d_prob_chain), np * sizeof(int32_t))) != cudaSuccess ||
      (e = cudaMalloc(reinterpret_cast<void **>(&b->d_order), np * sizeof(int32_t))) != cudaSuccess ||
      (e = cudaMalloc(reinterpret_cast<void **>(&b->d_state_off), so.size() * sizeof(int64_t))) != cudaSuccess ||
      (e = cudaMalloc(reinterpret_cast<void **>(&b->d_sq_off), sq.size() * sizeof(int64_t))) != cudaSuccess ||
      (n_problems > 0 &&
       ((e = cudaMemcpy(b->d_prob_chain, pc.data(), pc.size() * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_order, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess)) ||
      (e = cudaMemcpy(b->d_state_off, so.data(), so.size() * sizeof(int64_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->d_sq_off, sq.data(), sq.size() * sizeof(int64_t), cudaMemcpyHostToDevice)) != cudaSuccess) {
    cudaFree(b->d_prob_chain);
    cudaFree(b->d_order);
    cudaFree(b->d_state_off);
    cudaFree(b->d_sq_off);
    delete b;
    cudaSetDevice(prev);
    return cuda_fail(e, "fd_batch_create: device copy");
  }
  cudaSetDevice(prev);
  *out = b;
  return FD_OK;
}

fd_status fd_batch_destroy(fd_batch_t b) {
  if (!b) return fail(FD_ERR_INVALID_ARG, "fd_batch_destroy: NULL");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  cudaFree(b->d_prob_chain);
  cudaFree(b->d_order);
  cudaFree(b->d_state_off);
  cudaFree(b->d_sq_off);
  cudaSetDevice(prev);
  cudaGetLastError();  // leave no error state behind for other users of the runtime
  delete b;
  return FD_OK;
}

fd_status fd_batch_info(fd_batch_t b, int32_t *n_problems, int64_t *n_state_links,
                        int32_t *max_links) {
  if (!b) return fail(FD_ERR_INVALID_ARG, "fd_batch_info: NULL batch");
  if (n_problems) *n_problems = b->n_problems;
  if (n_state_links) *n_state_links = b->n_state_links;
  if (max_links) *max_links = b->max_links;
  return FD_OK;
}

}  // extern "C"

namespace {

int resolve_team(const fd_batch_s *b, int32_t algo, fd_prec prec, int32_t team) {
  if (team > 0) return team;
  const int tuned = (algo >= 0 && algo < FD_N_ALGOS && prec >= 0 && prec < 3) ? b->tuned[algo][prec] : 0;
  if (tuned > 0) return tuned;
  return fdk_default_team(algo, b->n_problems, b->max_links);
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct WsPlan {
  size_t t_bytes, a_bytes;
};

WsPlan ws_plan(const fd_batch_s *b, int32_t algo, fd_prec prec, int /*team: no layout depends on it*/) {
  const size_t ts = prec == FD_FP64 ? 8 : 4;
  const size_t as = prec == FD_FP32 ? 4 : 8;
  const size_t L = static_cast<size_t>(b->n_state_links);
  WsPlan w{align256(L * fdk::NT * ts), 0};
  if (b->chain->d_parent) {  // kinematic trees
    if (algo == FD_ABIA) w.a_bytes = align256(L * fdk::NA_TREE * as);
    if (algo == FD_JSIIA)
      w.a_bytes = align256((L * fdk::NA_TREE + static_cast<size_t>(b->sum_sq) +
                            (b->chain->n_loops > 0 ? L * fdk::NA_LOOP_LINK : 0)) * as);
    return w;
  }
  if (algo == FD_CFA || algo == FD_CFA_CR || algo == FD_CFA_HYBRID)
    w.a_bytes = L * fdk::NA_CFA * as;
  if (algo == FD_JSIIA)
    w.a_bytes = (L * fdk::NA_JSIIA + static_cast<size_t>(b->sum_sq) * fdk::NSQ_JSIIA) * as;
  if (algo == FD_ABIA || algo == FD_ABIA_SCAN) w.a_bytes = L * fdk::NA_ABIA * as;
  w.a_bytes = align256(w.a_bytes);
  return w;
}

bool valid_team(int t) { return fdk_valid_team(t); }

// team 0 on a batch of several length classes: one launch split by class
// (at most fdk::MAX_CLASSES classes fit a launch's table; chains of up to 2^20
// links give 21)
bool use_classes(const fd_batch_s *b, int32_t team) {
  return team == 0 && b->classes.size() > 1 && b->classes.size() <= fdk::MAX_CLASSES;
}
bool use_classes(const fd_batch_s *b, int32_t algo, int32_t team) {
  return algo != FD_ABIA_SCAN && use_classes(b, team);
}

int class_team(const fd_batch_s *b, size_t c, int32_t algo, fd_prec prec) {
  if (algo >= 0) {
    const int tuned = b->ctuned[(c * FD_N_ALGOS + static_cast<size_t>(algo)) * 3 + prec];
    if (tuned > 0) return tuned;
  }
  const auto &cl = b->classes[c];
  return std::min(fdk_default_team(algo, cl.count, cl.max_len), 128);
}

// The adjoint's reverse sweep: component lanes (team 8..32) up to 64 links, else
// the forward solve's team (ABIA's serial team 1 would scan nothing: CFA's).
int sweep_team(const fd_batch_s *b, size_t c, int32_t algo, fd_prec prec) {
  const int t = class_team(b, c, algo, prec);
  if (b->classes[c].max_len <= 64) return std::min(std::max(t, 8), 32);
  return algo == FD_ABIA ? class_team(b, c, FD_CFA, prec) : t;
}

// The grid split of a class launch: every class (only < 0) or class `only` alone.
fdk::ClassTable class_table(const fd_batch_s *b, const std::vector<int> &teams, int only = -1) {
  fdk::ClassTable ct{};
  int nb = 0, k = 0;
  for (size_t c = 0; c < b->classes.size(); ++c) {
    if (only >= 0 && static_cast<int>(c) != only) continue;
    const auto &cl = b->classes[c];
    ct.blk[k] = nb;
    ct.first[k] = cl.first;
    ct.team[k] = teams[c];
    nb += static_cast<int>((static_cast<int64_t>(cl.count) * teams[c] + fdk::BLOCK - 1) /
                           fdk::BLOCK);
    ++k;
    ct.first[k] = cl.first + cl.count;
  }
  ct.n = k;
  ct.blk[k] = nb;
  return ct;
}

cudaError_t launch_classes(const fdk::KArgs &a, int32_t algo, int prec_k,
                           const fdk::ClassTable &ct, cudaStream_t s) {
  if (algo == -1) return fdk::launch_id_multi(a, prec_k, ct, s);
  if (algo == FD_CFA) return fdk::launch_cfa_multi(a, prec_k, ct, s);
  if (algo == FD_CFA_CR) return fdk::launch_cfa_cr_multi(a, prec_k, ct, s);
  if (algo == FD_CFA_HYBRID) return fdk::launch_cfa_hy_multi(a, prec_k, ct, s);
  if (algo == FD_JSIIA) return fdk::launch_jsiia_multi(a, prec_k, ct, s);
  return fdk::launch_abia_multi(a, prec_k, ct, s);
}

}  // namespace

extern "C" {

size_t fd_workspace_size(fd_batch_t b, int32_t algo, fd_prec prec, int32_t team) {
  if (!b) return 0;
  const int t = resolve_team(b, algo, prec, team);
  const WsPlan w = ws_plan(b, algo, prec, t);
  return w.t_bytes + w.a_bytes;
}

// only_class >= 0: launch that length class alone with `team` (the autotuner);
// wmode != 0: CFA with a general projection (fdk::WPROJ_*, Q_i in wq)
static fd_status launch_common(fd_batch_t b, const void *q, const void *qd, const void *in3,
                               void *out, int32_t algo, fd_prec prec, int32_t team, void *ws,
                               size_t ws_bytes, int32_t *status, void *stream, const char *who,
                               int only_class = -1, int wmode = 0, const double *wq = nullptr) {
  if (!b) return fail(FD_ERR_INVALID_ARG, "%s: NULL batch", who);
  if (prec != FD_FP64 && prec != FD_FP32 && prec != FD_MIXED)
    return fail(FD_ERR_INVALID_ARG, "%s: bad precision %d", who, static_cast<int>(prec));
  if (algo != -1 && algo != FD_ABIA && algo != FD_JSIIA && algo != FD_CFA && algo != FD_CFA_CR &&
      algo != FD_CFA_HYBRID && algo != FD_ABIA_SCAN)
    return fail(FD_ERR_INVALID_ARG, "%s: bad algorithm %d", who, algo);
  if (team < 0 || (team > 0 && !valid_team(team)))
    return fail(FD_ERR_INVALID_ARG, "%s: team %d is not 0 or a power of two <= 256", who, team);
  if (algo == FD_ABIA && team > 0 && !fdk::abia_team_ok(team))
    return fail(FD_ERR_UNSUPPORTED, "%s: ABIA runs teams of 1, 8, 16 or 32 lanes, not %d", who,
                team);
  if (algo == FD_ABIA_SCAN && (prec != FD_FP64 || (team > 0 && !fdk::abia_scan_team_ok(team))))
    return fail(FD_ERR_UNSUPPORTED, "%s: the ABI scan runs in FP64 on teams of 8 .. 256 lanes",
                who);
  const bool tree = b->chain->d_parent != nullptr;
  if (tree) {
    if ((algo != FD_ABIA && algo != FD_JSIIA && algo != -1) || wmode != 0)
      return fail(FD_ERR_UNSUPPORTED,
                  "%s: kinematic trees run ABIA, JSIIA and inverse dynamics (CFA's system is "
                  "block tri-diagonal only on a serial chain)", who);
    if (prec == FD_MIXED)
      return fail(FD_ERR_UNSUPPORTED, "%s: kinematic trees run in FP64 or FP32", who);
    if (team > 1 || only_class >= 0)
      return fail(FD_ERR_UNSUPPORTED, "%s: kinematic trees run one thread per tree (team 1)",
                  who);
    if (b->chain->n_loops > 0 && (algo != FD_JSIIA || prec != FD_FP64))
      return fail(FD_ERR_UNSUPPORTED,
                  "%s: trees closed by loops run JSIIA in FP64 (its factor of M solves the "
                  "constrained system)", who);
  }
  if (b->n_problems == 0 || b->n_state_links == 0) return FD_OK;
  if (!q || !qd || !in3 || !out) return fail(FD_ERR_INVALID_ARG, "%s: NULL state array", who);
  const int t = tree ? 1 : resolve_team(b, algo, prec, team);
  const WsPlan w = ws_plan(b, algo, prec, t);
  if (!ws || ws_bytes < w.t_bytes + w.a_bytes)
    return fail(FD_ERR_INVALID_ARG, "%s: workspace of %zu bytes, %zu needed", who, ws_bytes,
                w.t_bytes + w.a_bytes);
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0)
    return fail(FD_ERR_INVALID_ARG, "%s: workspace not 256-byte aligned", who);
  const int prec_k = prec == FD_FP64 ? 0 : (prec == FD_FP32 || algo == -1 ? 1 : 2);
  fdk::KArgs a{};
  a.model = prec == FD_FP64 ? b->chain->d_model64 : b->chain->d_model32;
  a.model64 = b->chain->d_model64;
  a.model_off = b->chain->d_off;
  a.prob_chain = b->d_prob_chain;
  a.state_off = b->d_state_off;
  a.sq_off = b->d_sq_off;
  a.order = b->d_order;
  a.n_problems = b->n_problems;
  a.team = t;
  a.q = q;
  a.qd = qd;
  a.in3 = in3;
  a.out = out;
  a.ws_t = ws;
  a.ws_a = static_cast<char *>(ws) + w.t_bytes;
  a.status = status;
  a.wq = wq;
  a.wmode = wmode;
  a.parent = b->chain->d_parent;
  std::memcpy(a.grav, b->chain->grav, sizeof a.grav);
  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(b->chain->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  auto s = static_cast<cudaStream_t>(stream);
  if (tree) {
    e = fdk::launch_tree(a, algo == FD_ABIA ? 0 : (algo == FD_JSIIA ? 1 : -1), prec_k, s);
    if (e == cudaSuccess && b->chain->n_loops > 0) {
      a.loop_off = b->chain->d_loop_off;
      a.loop_ab = b->chain->d_loop_ab;
      a.loop_T = b->chain->d_loop_T;
      a.loop_ws = static_cast<int64_t>(b->n_state_links) * fdk::NA_TREE + b->sum_sq;
      e = fdk::launch_tree_loops(a, s);
    }
  } else if (wmode != 0) {
    e = fdk::launch_cfa_w(a, prec_k, t, s);
  } else if (only_class >= 0 || use_classes(b, algo, team)) {
    std::vector<int> teams(b->classes.size());
    for (size_t c = 0; c < teams.size(); ++c)
      teams[c] = (only_class >= 0 && static_cast<int>(c) == only_class && team > 0)
                     ? team
                     : class_team(b, c, algo, prec);
    e = launch_classes(a, algo, prec_k, class_table(b, teams, only_class), s);
  } else if (algo == -1) e = fdk::launch_id(a, prec_k, t, s);
  else if (algo == FD_CFA) e = fdk::launch_cfa(a, prec_k, t, s);
  else if (algo == FD_CFA_CR) e = fdk::launch_cfa_cr(a, prec_k, t, s);
  else if (algo == FD_CFA_HYBRID) e = fdk::launch_cfa_hy(a, prec_k, t, s);
  else if (algo == FD_JSIIA) e = fdk::launch_jsiia(a, prec_k, t, s);
  else if (algo == FD_ABIA_SCAN) e = fdk::launch_abia_scan(a, prec_k, t, s);
  else e = fdk::launch_abia(a, prec_k, t, s);
  cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(e, who);
  return FD_OK;
}

fd_status fd_solve_batch(fd_batch_t b, const void *q, const void *qdot, const void *tau,
                         void *qddot, fd_algo algo, fd_prec prec, int32_t team, void *workspace,
                         size_t workspace_bytes, int32_t *status, void *stream) {
  return launch_common(b, q, qdot, tau, qddot, static_cast<int32_t>(algo), prec, team, workspace,
                       workspace_bytes, status, stream, "fd_solve_batch");
}

fd_status fd_inverse_dynamics(fd_batch_t b, const void *q, const void *qdot, const void *qddot,
                              void *tau, fd_prec prec, int32_t team, void *workspace,
                              size_t workspace_bytes, void *stream) {
  return launch_common(b, q, qdot, qddot, tau, -1, prec == FD_MIXED ? FD_FP32 : prec, team,
                       workspace, workspace_bytes, nullptr, stream, "fd_inverse_dynamics");
}

fd_status fd_projection_to_canonical(int64_t n_links, const double *joint_axes, const double *W,
                                     double *Q) {
  const char *who = "fd_projection_to_canonical";
  if (n_links < 0) return fail(FD_ERR_INVALID_ARG, "%s: n_links %lld", who, static_cast<long long>(n_links));
  if (n_links > 0 && (!joint_axes || !W || !Q))
    return fail(FD_ERR_INVALID_ARG, "%s: NULL array", who);
  for (int64_t i = 0; i < n_links; ++i) {
    const double *ax = joint_axes + 3 * i;
    const double na = std::sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
    if (!(na > 1e-12) || !std::isfinite(na))
      return fail(FD_ERR_INVALID_ARG, "%s: link %lld has a zero joint axis", who,
                  static_cast<long long>(i));
    const double a[3] = {ax[0] / na, ax[1] / na, ax[2] / na};
    double F[9];
    axis_frame(a, F);  // link coordinates of the canonical axes (columns)
    // a wrench in canonical coordinates: (F^T n; F^T f)
    const double *Wi = W + 30 * i;
    double Wc[30], scale = 0.0;
    for (int k = 0; k < 30; ++k) scale = std::max(scale, std::fabs(Wi[k]));
    for (int h = 0; h < 2; ++h)
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 5; ++c)
          Wc[5 * (3 * h + r) + c] = F[r] * Wi[5 * (3 * h) + c] + F[3 + r] * Wi[5 * (3 * h + 1) + c] +
                                    F[6 + r] * Wi[5 * (3 * h + 2) + c];
    if (!(scale > 0.0) || !std::isfinite(scale))
      return fail(FD_ERR_INVALID_ARG, "%s: link %lld: W is zero or not finite", who,
                  static_cast<long long>(i));
    for (int c = 0; c < 5; ++c)  // row 0 of Wc is S_i^T W_i
      if (!(std::fabs(Wc[c]) <= 1e-9 * scale))
        return fail(FD_ERR_INVALID_ARG, "%s: link %lld: W^T S = %.3e, not 0", who,
                    static_cast<long long>(i), Wc[c]);
    double *Qi = Q + 25 * i;
    for (int k = 0; k < 25; ++k) Qi[k] = Wc[5 + k];
    // |det Q_i| against the product of its column norms, by Gaussian elimination
    // with partial pivoting on a copy
    double M[25], cn = 1.0, det = 1.0;
    std::memcpy(M, Qi, sizeof M);
    for (int c = 0; c < 5; ++c) {
      double s2 = 0.0;
      for (int r = 0; r < 5; ++r) s2 += M[5 * r + c] * M[5 * r + c];
      cn *= std::sqrt(s2);
    }
    for (int c = 0; c < 5 && det != 0.0; ++c) {
      int piv = c;
      for (int r = c + 1; r < 5; ++r)
        if (std::fabs(M[5 * r + c]) > std::fabs(M[5 * piv + c])) piv = r;
      if (M[5 * piv + c] == 0.0) {
        det = 0.0;
        break;
      }
      if (piv != c) {
        for (int k = 0; k < 5; ++k) std::swap(M[5 * c + k], M[5 * piv + k]);
        det = -det;
      }
      det *= M[5 * c + c];
      for (int r = c + 1; r < 5; ++r) {
        const double f = M[5 * r + c] / M[5 * c + c];
        for (int k = c; k < 5; ++k) M[5 * r + k] -= f * M[5 * c + k];
      }
    }
    if (!(std::fabs(det) > 1e-12 * cn))
      return fail(FD_ERR_INVALID_ARG, "%s: link %lld: W has rank below 5", who,
                  static_cast<long long>(i));
  }
  return FD_OK;
}

fd_status fd_solve_cfa_projected(fd_batch_t b, const void *q, const void *qdot, const void *tau,
                                 void *qddot, fd_prec prec, int32_t team, fd_projection proj,
                                 const double *Q, void *workspace, size_t workspace_bytes,
                                 int32_t *status, void *stream) {
  const char *who = "fd_solve_cfa_projected";
  if (!b) return fail(FD_ERR_INVALID_ARG, "%s: NULL batch", who);
  if (b->chain->d_parent)
    return fail(FD_ERR_UNSUPPORTED, "%s: serial chains only (not kinematic trees)", who);
  if (proj != FD_PROJ_CANONICAL && proj != FD_PROJ_GIVEN && proj != FD_PROJ_BLOCK_JACOBI)
    return fail(FD_ERR_INVALID_ARG, "%s: bad projection %d", who, static_cast<int>(proj));
  if (prec == FD_MIXED)
    return fail(FD_ERR_UNSUPPORTED, "%s: FP64 and FP32 only", who);
  if (prec != FD_FP64 && prec != FD_FP32)
    return fail(FD_ERR_INVALID_ARG, "%s: bad precision %d", who, static_cast<int>(prec));
  if (proj == FD_PROJ_GIVEN && !Q && b->n_problems > 0 && b->n_state_links > 0)
    return fail(FD_ERR_INVALID_ARG, "%s: FD_PROJ_GIVEN needs Q", who);
  if (team < 0 || (team > 0 && !valid_team(team)))
    return fail(FD_ERR_INVALID_ARG, "%s: team %d is not 0 or a power of two <= 256", who, team);
  // one team for the whole batch (no split by length class)
  const int t = resolve_team(b, FD_CFA, prec, team);
  const int wmode = proj == FD_PROJ_GIVEN ? fdk::WPROJ_GIVEN
                    : proj == FD_PROJ_BLOCK_JACOBI ? fdk::WPROJ_BLOCK_JACOBI : 0;
  return launch_common(b, q, qdot, tau, qddot, FD_CFA, prec, t, workspace, workspace_bytes,
                       status, stream, who, -1, wmode, Q);
}

}  // extern "C"

extern "C" {

size_t fd_adjoint_workspace_size(fd_batch_t b, fd_algo algo, fd_prec prec, int32_t team) {
  if (!b) return 0;
  const int t = resolve_team(b, algo, prec, team);
  const WsPlan w = ws_plan(b, algo, prec, t);
  const size_t ts = prec == FD_FP64 ? 8 : 4;
  const size_t L = static_cast<size_t>(b->n_state_links);
  return align256(L * ts) + std::max(w.t_bytes + w.a_bytes, align256(L * fdk::NT_ADJ * ts));
}

fd_status fd_solve_adjoint(fd_batch_t b, const void *q, const void *qdot, const void *tau,
                           const void *qddot, const void *qddot_bar, void *q_bar,
                           void *qdot_bar, void *tau_bar, void *mass_bar, fd_algo algo,
                           fd_prec prec, int32_t team, void *workspace, size_t workspace_bytes,
                           int32_t *status, void *stream) {
  const char *who = "fd_solve_adjoint";
  if (!b) return fail(FD_ERR_INVALID_ARG, "%s: NULL batch", who);
  if (b->chain->d_parent)
    return fail(FD_ERR_UNSUPPORTED, "%s: serial chains only (not kinematic trees)", who);
  if (algo != FD_ABIA && algo != FD_JSIIA && algo != FD_CFA && algo != FD_CFA_CR &&
      algo != FD_CFA_HYBRID && algo != FD_ABIA_SCAN)
    return fail(FD_ERR_INVALID_ARG, "%s: bad algorithm %d", who, static_cast<int>(algo));
  if (prec != FD_FP64 && prec != FD_FP32 && prec != FD_MIXED)
    return fail(FD_ERR_INVALID_ARG, "%s: bad precision %d", who, static_cast<int>(prec));
  if (team < 0 || (team > 0 && !valid_team(team)))
    return fail(FD_ERR_INVALID_ARG, "%s: team %d is not 0 or a power of two <= 256", who, team);
  if (algo == FD_ABIA && team > 0 && !fdk::abia_team_ok(team))
    return fail(FD_ERR_UNSUPPORTED, "%s: ABIA runs teams of 1, 8, 16 or 32 lanes, not %d", who,
                team);
  if (algo == FD_ABIA_SCAN && (prec != FD_FP64 || (team > 0 && !fdk::abia_scan_team_ok(team))))
    return fail(FD_ERR_UNSUPPORTED, "%s: the ABI scan runs in FP64 on teams of 8 .. 256 lanes",
                who);
  if (mass_bar && !b->chain->rigid)
    return fail(FD_ERR_UNSUPPORTED,
                "%s: mass gradients need rigid-body inertias (J = [[I - m c^c^, m c^], "
                "[-m c^, m 1]])", who);
  if (b->n_problems == 0 || b->n_state_links == 0) return FD_OK;
  if (!q || !qdot || !tau || !qddot_bar || !q_bar || !qdot_bar || !tau_bar)
    return fail(FD_ERR_INVALID_ARG, "%s: NULL array", who);
  const size_t need = fd_adjoint_workspace_size(b, algo, prec, team);
  if (!workspace || workspace_bytes < need)
    return fail(FD_ERR_INVALID_ARG, "%s: workspace of %zu bytes, %zu needed", who,
                workspace_bytes, need);
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
    return fail(FD_ERR_INVALID_ARG, "%s: workspace not 256-byte aligned", who);
  const int t = resolve_team(b, algo, prec, team);
  const WsPlan w = ws_plan(b, algo, prec, t);
  const size_t ts = prec == FD_FP64 ? 8 : 4;
  const size_t L = static_cast<size_t>(b->n_state_links);
  char *qdd_scratch = static_cast<char *>(workspace);
  char *region = qdd_scratch + align256(L * ts);
  const int prec_k = prec == FD_FP64 ? 0 : (prec == FD_FP32 ? 1 : 2);

  fdk::KArgs a{};
  a.model = prec == FD_FP64 ? b->chain->d_model64 : b->chain->d_model32;
  a.model64 = b->chain->d_model64;
  a.model_off = b->chain->d_off;
  a.prob_chain = b->d_prob_chain;
  a.state_off = b->d_state_off;
  a.sq_off = b->d_sq_off;
  a.order = b->d_order;
  a.n_problems = b->n_problems;
  a.team = t;
  a.q = q;
  a.qd = qdot;
  a.status = status;
  std::memcpy(a.grav, b->chain->grav, sizeof a.grav);
  a.ws_t = region;
  a.ws_a = region + w.t_bytes;

  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(b->chain->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  auto s = static_cast<cudaStream_t>(stream);
  const bool split = use_classes(b, algo, team);
  std::vector<int> fd_teams(b->classes.size()), sw_teams(b->classes.size());
  for (size_t c = 0; split && c < fd_teams.size(); ++c) {
    fd_teams[c] = class_team(b, c, algo, prec);
    sw_teams[c] = sweep_team(b, c, algo, prec);
  }
  auto run_fd = [&](fdk::KArgs &k) {
    if (split) return launch_classes(k, algo, prec_k, class_table(b, fd_teams), s);
    if (algo == FD_CFA) return fdk::launch_cfa(k, prec_k, t, s);
    if (algo == FD_CFA_CR) return fdk::launch_cfa_cr(k, prec_k, t, s);
    if (algo == FD_CFA_HYBRID) return fdk::launch_cfa_hy(k, prec_k, t, s);
    if (algo == FD_JSIIA) return fdk::launch_jsiia(k, prec_k, t, s);
    if (algo == FD_ABIA_SCAN) return fdk::launch_abia_scan(k, prec_k, t, s);
    return fdk::launch_abia(k, prec_k, t, s);
  };
  // 1-2. lambda = M^{-1} qdd_bar with the algorithm's own factorisation: tau_bar;
  // without a given qdd, FD and this solve share one elimination (MODE_FD2)
  const void *qdd = qddot;
  if (!qdd) {
    a.mode = fdk::MODE_FD2;
    a.in3 = tau;
    a.out = qdd_scratch;
    a.in4 = qddot_bar;
    a.out4 = tau_bar;
    e = run_fd(a);
    qdd = qdd_scratch;
  } else {
    a.mode = fdk::MODE_LINEAR;
    a.in3 = qddot_bar;
    a.out = tau_bar;
    e = run_fd(a);
  }
  // 3. q_bar, qdot_bar, mass_bar = -(d ID / d x)^T lambda
  if (e == cudaSuccess) {
    fdk::KArgs r = a;
    r.mode = fdk::MODE_ID;
    r.in3 = qdd;
    r.lam = tau_bar;
    r.out = q_bar;
    r.out2 = qdot_bar;
    r.out3 = mass_bar;
    r.ws_t = region;
    r.status = nullptr;
    // the reverse sweep: component lanes (team 8) for chains of up to 64 links,
    // else the algorithm's team (ABIA's serial team 1 would scan nothing)
    const int tr = b->max_links <= 64 ? std::max(t, 8) > 32 ? 32 : std::max(t, 8)
                   : ((algo == FD_ABIA || algo == FD_ABIA_SCAN) ? resolve_team(b, FD_CFA, prec, 0)
                                                                : t);
    r.team = tr;
    e = split ? fdk::launch_adjoint_rnea_multi(r, prec == FD_FP64 ? 0 : 1,
                                               class_table(b, sw_teams), s)
              : fdk::launch_adjoint_rnea(r, prec == FD_FP64 ? 0 : 1, tr, s);
  }
  cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(e, who);
  return FD_OK;
}

}  // extern "C"

namespace {

// ------------------------------------------------------------ autotune cache
//
// Process-wide: the fastest team per (GPU, algorithm, precision, length class,
// problem-count class), filled by fd_autotune and persisted as JSON by
// fd_autotune_cache_save / _load, so a later process skips the timing.
// mix: 0 for a class timed alone (or a one-class batch); for a class's team
// refined inside its batch's whole launch, a hash of the batch's classes and
// their problem-count classes (the choice depends on the company it keeps)
struct TuneKey {
  std::string gpu;
  int algo, prec, len_class, count_class;
  uint32_t mix;
  bool operator<(const TuneKey &o) const {
    return std::tie(gpu, algo, prec, len_class, count_class, mix) <
           std::tie(o.gpu, o.algo, o.prec, o.len_class, o.count_class, o.mix);
  }
};
struct TuneVal {
  int team;
  float ms;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

int ceil_log2(int64_t v) {
  int k = 0;
  while ((int64_t(1) << k) < v) ++k;
  return k;
}

std::string gpu_name(int dev) {
  cudaDeviceProp pr{};
  if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  char buf[320];
  snprintf(buf, sizeof buf, "%s (%d SMs)", pr.name, pr.multiProcessorCount);
  return buf;
}

// Times `cand` teams on one length class (cls >= 0) or the whole batch (cls < 0):
// one warm-up and two timed solves each; returns the fastest (0 if none fits).
fd_status time_teams(fd_batch_t b, fd_algo algo, fd_prec prec, const void *q, const void *qdot,
                     const void *tau, void *qddot, void *workspace, size_t workspace_bytes,
                     cudaStream_t s, const std::vector<int> &cand, int cls, int *best,
                     float *best_ms, const char *who) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  *best = 0;
  *best_ms = 0.f;
  fd_status st = FD_OK;
  for (int t : cand) {
    const WsPlan w = ws_plan(b, algo, prec, t);
    if (w.t_bytes + w.a_bytes > workspace_bytes) continue;
    st = launch_common(b, q, qdot, tau, qddot, algo, prec, t, workspace, workspace_bytes,
                       nullptr, s, who, cls);
    if (st != FD_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 2 && st == FD_OK; ++r)
      st = launch_common(b, q, qdot, tau, qddot, algo, prec, t, workspace, workspace_bytes,
                         nullptr, s, who, cls);
    cudaEventRecord(e1, s);
    const cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      st = cuda_fail(e, who);
      break;
    }
    if (st != FD_OK) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= 2;
    if (*best == 0 || ms < *best_ms) {
      *best = t;
      *best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

std::vector<int> team_candidates(fd_algo algo, int max_len, int cap_team) {
  std::vector<int> cand;
  if (algo == FD_ABIA) {
    // ABIA's lane teams spread each step's 6x6 update over 6 or 12 lanes, which
    // pays even for chains shorter than the team
    for (int t : {1, 8, 16, 32}) cand.push_back(t);
  } else if (algo == FD_ABIA_SCAN) {
    int cap = 8;
    while (cap < max_len && cap < cap_team) cap *= 2;
    for (int t = 8; t <= cap; t *= 2) cand.push_back(t);
  } else {
    int cap = 1;
    while (cap < max_len && cap < cap_team) cap *= 2;
    for (int t = 1; t <= cap; t *= 2) cand.push_back(t);
  }
  return cand;
}

}  // namespace

extern "C" fd_status fd_autotune(fd_batch_t b, fd_algo algo, fd_prec prec, const void *q,
                                 const void *qdot, const void *tau, void *qddot,
                                 void *workspace, size_t workspace_bytes, void *stream,
                                 int32_t *best_team) {
  const char *who = "fd_autotune";
  if (!b) return fail(FD_ERR_INVALID_ARG, "%s: NULL batch", who);
  if (algo != FD_ABIA && algo != FD_JSIIA && algo != FD_CFA && algo != FD_CFA_CR &&
      algo != FD_CFA_HYBRID && algo != FD_ABIA_SCAN)
    return fail(FD_ERR_INVALID_ARG, "%s: bad algorithm", who);
  if (algo == FD_ABIA_SCAN && prec != FD_FP64)
    return fail(FD_ERR_UNSUPPORTED, "%s: the ABI scan runs in FP64", who);
  if (prec != FD_FP64 && prec != FD_FP32 && prec != FD_MIXED)
    return fail(FD_ERR_INVALID_ARG, "%s: bad precision", who);
  if (b->chain->d_parent && algo != FD_ABIA && algo != FD_JSIIA)
    return fail(FD_ERR_UNSUPPORTED, "%s: kinematic trees run ABIA and JSIIA", who);
  if (b->chain->d_parent && prec == FD_MIXED)
    return fail(FD_ERR_UNSUPPORTED, "%s: kinematic trees run in FP64 or FP32", who);
  if (b->n_problems == 0 || b->n_state_links == 0 || b->chain->d_parent) {
    if (best_team) *best_team = 1;  // one thread per tree: nothing to choose
    return FD_OK;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(b->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  const std::string gpu = gpu_name(b->device);
  auto s = static_cast<cudaStream_t>(stream);
  fd_status st = FD_OK;
  const bool split = algo != FD_ABIA_SCAN && use_classes(b, 0);
  // one length class (or the whole batch): its team from the cache, else timed
  auto tune = [&](int cls, int max_len, int64_t count, int len_class, int cap_team,
                  int *out) -> fd_status {
    const TuneKey key{gpu, static_cast<int>(algo), static_cast<int>(prec), len_class,
                      ceil_log2(count), 0u};
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) {
        *out = it->second.team;
        return FD_OK;
      }
    }
    int best = 0;
    float ms = 0.f;
    const fd_status r = time_teams(b, algo, prec, q, qdot, tau, qddot, workspace, workspace_bytes,
                                   s, team_candidates(algo, max_len, cap_team), cls, &best, &ms,
                                   who);
    if (r != FD_OK) return r;
    if (best == 0) return fail(FD_ERR_INVALID_ARG, "%s: workspace too small for any team", who);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = TuneVal{best, ms};
    *out = best;
    return FD_OK;
  };
  if (split) {
    // per length class, each timed alone in the class launch (teams up to 128)
    for (size_t c = 0; c < b->classes.size() && st == FD_OK; ++c) {
      const auto &cl = b->classes[c];
      int best = 0;
      st = tune(static_cast<int>(c), cl.max_len, cl.count, cl.key, 128, &best);
      if (st == FD_OK) b->ctuned[(c * FD_N_ALGOS + static_cast<size_t>(algo)) * 3 + prec] = best;
    }
    // then refine inside the whole launch: a class's best team alone is not its
    // best among the others (the longest class sets the launch's tail), so each
    // class in turn, longest first, tries its other teams with the rest fixed
    uint32_t mix = 2166136261u;  // FNV-1a over the classes' keys and count classes
    for (const auto &cl : b->classes)
      for (int v : {cl.key, ceil_log2(cl.count)}) mix = (mix ^ static_cast<uint32_t>(v)) * 16777619u;
    mix |= 1u;
    const size_t nc = b->classes.size();
    auto slot = [&](size_t c) -> int & {
      return b->ctuned[(c * FD_N_ALGOS + static_cast<size_t>(algo)) * 3 + prec];
    };
    bool cached = true;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      for (size_t c = 0; c < nc && cached; ++c) {
        const auto &cl = b->classes[c];
        auto it = g_tune.find(TuneKey{gpu, static_cast<int>(algo), static_cast<int>(prec), cl.key,
                                      ceil_log2(cl.count), mix});
        if (it == g_tune.end()) cached = false;
      }
      if (cached)
        for (size_t c = 0; c < nc; ++c) {
          const auto &cl = b->classes[c];
          slot(c) = g_tune[TuneKey{gpu, static_cast<int>(algo), static_cast<int>(prec), cl.key,
                                   ceil_log2(cl.count), mix}].team;
        }
    }
    if (st == FD_OK && !cached) {
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      auto whole = [&](float *ms) -> fd_status {
        fd_status r = launch_common(b, q, qdot, tau, qddot, algo, prec, 0, workspace,
                                    workspace_bytes, nullptr, s, who);
        if (r != FD_OK) return r;
        cudaEventRecord(e0, s);
        for (int k = 0; k < 2 && r == FD_OK; ++k)
          r = launch_common(b, q, qdot, tau, qddot, algo, prec, 0, workspace, workspace_bytes,
                            nullptr, s, who);
        cudaEventRecord(e1, s);
        const cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) return cuda_fail(e, who);
        cudaEventElapsedTime(ms, e0, e1);
        *ms /= 2;
        return r;
      };
      float best_ms = 0.f;
      st = whole(&best_ms);
      for (size_t c = 0; c < nc && st == FD_OK; ++c) {
        const int keep = slot(c);
        int best_t = keep;
        for (int t : team_candidates(algo, b->classes[c].max_len, 128)) {
          if (t == keep) continue;
          slot(c) = t;
          float ms = 0.f;
          st = whole(&ms);
          if (st != FD_OK) break;
          if (ms < 0.99f * best_ms) {
            best_ms = ms;
            best_t = t;
          }
        }
        slot(c) = best_t;
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (st == FD_OK) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (size_t c = 0; c < nc; ++c) {
          const auto &cl = b->classes[c];
          g_tune[TuneKey{gpu, static_cast<int>(algo), static_cast<int>(prec), cl.key,
                         ceil_log2(cl.count), mix}] = TuneVal{slot(c), best_ms};
        }
      }
    }
    if (st == FD_OK && best_team) *best_team = 0;
  } else {
    int best = 0;
    st = tune(-1, b->max_links, b->n_problems, ceil_log2(std::max(b->max_links, 1)), 256, &best);
    if (st == FD_OK) {
      b->tuned[algo][prec] = best;
      if (best_team) *best_team = best;
    }
  }
  cudaSetDevice(prev);
  return st;
}

extern "C" fd_status fd_batch_classes(fd_batch_t b, int32_t algo, fd_prec prec, int32_t max,
                                      int32_t *n_classes, int32_t *min_len, int32_t *max_len,
                                      int32_t *count, int32_t *team) {
  if (!b || !n_classes) return fail(FD_ERR_INVALID_ARG, "fd_batch_classes: NULL argument");
  if (algo < -1 || algo >= FD_N_ALGOS || prec < FD_FP64 || prec > FD_MIXED)
    return fail(FD_ERR_INVALID_ARG, "fd_batch_classes: bad algorithm or precision");
  *n_classes = static_cast<int32_t>(b->classes.size());
  const bool split = use_classes(b, 0);
  for (size_t c = 0; c < b->classes.size() && static_cast<int32_t>(c) < max; ++c) {
    const auto &cl = b->classes[c];
    if (min_len) min_len[c] = cl.min_len;
    if (max_len) max_len[c] = cl.max_len;
    if (count) count[c] = cl.count;
    if (team)
      team[c] = (split && algo != FD_ABIA_SCAN) ? class_team(b, c, algo, prec)
                                                 : resolve_team(b, algo, prec, 0);
  }
  return FD_OK;
}

extern "C" fd_status fd_autotune_cache_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  return FD_OK;
}

extern "C" fd_status fd_autotune_cache_save(const char *path) {
  if (!path) return fail(FD_ERR_INVALID_ARG, "fd_autotune_cache_save: NULL path");
  std::string js = "{\"format\": \"fd_gb300 autotune cache 1\", \"entries\": [";
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    bool first = true;
    for (const auto &kv : g_tune) {
      std::string g;
      for (char ch : kv.first.gpu)
        if (ch != '"' && ch != '\\') g += ch;
      char buf[512];
      snprintf(buf, sizeof buf,
               "%s\n  {\"gpu\": \"%s\", \"algo\": %d, \"prec\": %d, \"len_class\": %d, "
               "\"count_class\": %d, \"mix\": %u, \"team\": %d, \"ms\": %.6g}",
               first ? "" : ",", g.c_str(), kv.first.algo, kv.first.prec, kv.first.len_class,
               kv.first.count_class, kv.first.mix, kv.second.team,
               static_cast<double>(kv.second.ms));
      js += buf;
      first = false;
    }
  }
  js += "\n]}\n";
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = std::fopen(tmp.c_str(), "w");
  if (!f) return fail(FD_ERR_INVALID_ARG, "fd_autotune_cache_save: cannot write %s", tmp.c_str());
  const bool ok = std::fwrite(js.data(), 1, js.size(), f) == js.size();
  std::fclose(f);
  if (!ok || std::rename(tmp.c_str(), path) != 0)
    return fail(FD_ERR_INVALID_ARG, "fd_autotune_cache_save: cannot write %s", path);
  return FD_OK;
}

extern "C" fd_status fd_autotune_cache_load(const char *path, int32_t *n_loaded) {
  if (n_loaded) *n_loaded = 0;
  if (!path) return fail(FD_ERR_INVALID_ARG, "fd_autotune_cache_load: NULL path");
  FILE *f = std::fopen(path, "r");
  if (!f) return FD_OK;  // no cache yet
  std::string js;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) js.append(buf, got);
  std::fclose(f);
  if (js.find("fd_gb300 autotune cache 1") == std::string::npos)
    return fail(FD_ERR_INVALID_ARG, "fd_autotune_cache_load: %s is not an autotune cache", path);
  // entries are flat objects of string and integer fields
  auto field = [](const std::string &obj, const char *name, std::string *sval, long *ival) {
    const std::string pat = std::string("\"") + name + "\"";
    size_t p = obj.find(pat);
    if (p == std::string::npos) return false;
    p = obj.find(':', p + pat.size());
    if (p == std::string::npos) return false;
    ++p;
    while (p < obj.size() && obj[p] == ' ') ++p;
    if (sval) {
      if (p >= obj.size() || obj[p] != '"') return false;
      const size_t q = obj.find('"', p + 1);
      if (q == std::string::npos) return false;
      *sval = obj.substr(p + 1, q - p - 1);
      return true;
    }
    char *end = nullptr;
    *ival = std::strtol(obj.c_str() + p, &end, 10);
    return end != obj.c_str() + p;
  };
  size_t pos = js.find('[');
  int n = 0;
  std::map<TuneKey, TuneVal> add;
  while (pos != std::string::npos) {
    const size_t a = js.find('{', pos);
    if (a == std::string::npos) break;
    const size_t z = js.find('}', a);
    if (z == std::string::npos)
      return fail(FD_ERR_INVALID_ARG, "fd_autotune_cache_load: %s is truncated", path);
    const std::string obj = js.substr(a, z - a + 1);
    std::string gpu;
    long algo = 0, prec = 0, lc = 0, cc = 0, team = 0;
    if (!field(obj, "gpu", &gpu, nullptr) || !field(obj, "algo", nullptr, &algo) ||
        !field(obj, "prec", nullptr, &prec) || !field(obj, "len_class", nullptr, &lc) ||
        !field(obj, "count_class", nullptr, &cc) || !field(obj, "team", nullptr, &team) ||
        algo < 0 || algo >= FD_N_ALGOS || prec < 0 || prec > FD_MIXED || !fdk_valid_team(team) ||
        (algo == FD_ABIA && !fdk::abia_team_ok(static_cast<int>(team))))
      return fail(FD_ERR_INVALID_ARG, "fd_autotune_cache_load: bad entry in %s", path);
    long mixv = 0;
    if (obj.find("\"mix\"") != std::string::npos && !field(obj, "mix", nullptr, &mixv))
      return fail(FD_ERR_INVALID_ARG, "fd_autotune_cache_load: bad entry in %s", path);
    add[TuneKey{gpu, int(algo), int(prec), int(lc), int(cc), static_cast<uint32_t>(mixv)}] =
        TuneVal{int(team), 0.f};
    ++n;
    pos = z + 1;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto &kv : add) g_tune[kv.first] = kv.second;
  if (n_loaded) *n_loaded = n;
  return FD_OK;
}
