// fd_serve.cu -- the serving runtime: continuous batching of forward-dynamics
// requests on one GPU.
//
// Models are registered once and stay resident (canonical records in a model
// region). A request names a model and carries its state: an FD+gradient query
// (qdd = FD(q, qd, tau) and the adjoint for a given cotangent) or a rollout
// (steps of semi-implicit Euler, qd += dt qdd, q += dt qd, with a given torque per
// step). A worker thread runs ticks: admit queued requests while the memory
// budget allows (one batched upload), run one forward-dynamics launch per
// algorithm over every active request, the adjoint over the new FD+gradient
// requests and an integration step over the rollouts, then gather the finished
// requests' results (one batched download) and release their memory.
#include <cuda_runtime.h>
#include <time.h>

#include <algorithm>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fd_internal.h"
#include "fd_launch.h"
#include "fd_layout.h"

namespace {

double now_s() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return static_cast<double>(ts.tv_sec) + 1e-9 * static_cast<double>(ts.tv_nsec);
}

// First-fit allocator of ranges of [0, cap).
class RangeAlloc {
 public:
  void reset(int64_t cap) {
    free_.clear();
    if (cap > 0) free_[0] = cap;
    used_ = 0;
  }
  int64_t alloc(int64_t n) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        const int64_t s = it->first, len = it->second;
        free_.erase(it);
        if (len > n) free_[s + n] = len - n;
        used_ += n;
        return s;
      }
    }
    return -1;
  }
  void release(int64_t s, int64_t n) {
    if (n <= 0) return;
    used_ -= n;
    auto nx = free_.lower_bound(s);
    if (nx != free_.begin()) {
      auto pv = std::prev(nx);
      if (pv->first + pv->second == s) {
        s = pv->first;
        n += pv->second;
        free_.erase(pv);
      }
    }
    if (nx != free_.end() && s + n == nx->first) {
      n += nx->second;
      free_.erase(nx);
    }
    free_[s] = n;
  }
  int64_t used() const { return used_; }

 private:
  std::map<int64_t, int64_t> free_;
  int64_t used_ = 0;
};

struct Model {
  int n = 0;
  int64_t rec = -1;  // first record in the model region
  int refs = 0;
  bool removing = false;
};

struct Req {
  uint64_t ticket = 0;
  int kind = 0, algo = 0, model = 0, n = 0, steps = 1, step = 0;
  int adv = 0;  // rollout steps this tick
  int64_t mrec = 0;  // first record of the model (stable while the request holds it)
  double dt = 0.0;
  std::vector<double> q, qd, tau, w;  // tau: n (FD+grad) or steps x n (rollout)
  int64_t slot = -1, hist = -1;
  double t_submit = 0.0, t_done = 0.0;
  int state = 0;  // 0 queued, 1 active, 2 done
  int32_t status = 0;
  std::vector<double> out;  // FD+grad: qdd, q_bar, qd_bar, tau_bar; rollout: q, qd, qdd
};

// per admitted request, for the scatter kernel
struct UpDesc {
  int64_t stage;  // offset in the upload staging buffer (doubles)
  int64_t slot;   // first link slot
  int64_t hist;   // first torque-history entry (rollouts), or -1
  int32_t n, kind, steps, pad;
  double dt;
};

// per finished request, for the gather kernel
struct OutDesc {
  int64_t slot, out;  // link slot, offset in the download staging buffer (doubles)
  int32_t n, kind, prob, pad;
};

struct Arena {
  double *model;                                    // model records [cap_rec][REC]
  double *q, *qd, *tau, *qdd, *w, *qbar, *qdbar, *tbar;  // [cap] per link slot
  // workspaces per link slot, one region per kernel kind: the kinds index them
  // with different strides and run concurrently on the side streams
  double *ws_t;                                     // [cap][NT]      FD kernels
  double *ws_r;                                     // [cap][NT_ADJ]  reverse sweep
  double *ws_c;                                     // [cap][NA_CFA]  CFA rows
  double *ws_b;                                     // [cap][NA_ABIA] ABIA
  double *hist;                                     // rollout torques
  int64_t *r_hist;                                  // per slot: history start
  int32_t *r_step, *r_steps;                        // per slot: step, total steps
  double *r_dt;                                     // per slot: dt
};

// Teams depend on a request's algorithm and chain length only, so its arithmetic
// does not depend on the mix. They are chosen for latency, since a tick lasts as
// long as its longest chains' solves: CFA takes about one lane per two links
// beyond 32 (8, 32, 64, 128: a 256-link chain's FD in 0.46 ms on 128 lanes
// against 0.82 ms on 64, measured in batches of 48), ABIA 16 up to 64 links and
// 32 beyond (its twelve-lane step: 64 links 0.31 against 0.42 ms on 8 lanes, 256
// links 0.84 against 0.95 ms on 16), the reverse sweep about one lane per four
// links (8..64).
enum TeamKind { kTeamCFA, kTeamReverse, kTeamABIA };
int team_for(TeamKind k, int n) {
  if (k == kTeamABIA) return n <= 64 ? 16 : 32;
  if (k == kTeamCFA) return n <= 32 ? 8 : (n <= 64 ? 32 : (n <= 128 ? 64 : 128));
  return n <= 32 ? 8 : (n <= 64 ? 16 : (n <= 128 ? 32 : 64));
}
// ABIA rollouts of chains over 64 links run the ABI recursion as a scan
// (FD_ABIA_SCAN) on 64 lanes (one to four links per lane up to 256 links), so a
// step's depth is a few links plus log2 64 instead of the whole chain. About 150
// such rollouts are in flight at 20 000 requests/s, so the class is not purely
// latency-bound: 64 lanes measured a little faster than the serial recursion on
// twelve lanes (tick 0.97 -> 0.96 ms), 128 lanes slower (1.21 ms: the scan's
// fivefold work). One team for the whole class keeps a request's arithmetic
// independent of the mix.
constexpr int kScanAbove = 64;
constexpr int kScanTeam = 64;

// Rollouts by length class, by algorithm and chain length only. A tick lasts
// about as long as its longest chains' serial recursions (an ABIA step costs a
// few microseconds per link on its critical lane), so the rollouts of a shorter
// class take several steps in that time, about 160 link-steps per tick for ABIA:
// each step is the same FD launch and Euler step as alone, on the class's own
// side stream. The per-size baseline takes one step per tick.
int roll_class(int algo, int n) {
  if (algo == FD_ABIA) return n <= 20 ? 0 : (n <= 40 ? 1 : (n <= 64 ? 2 : 3));
  return n <= 32 ? 0 : (n <= 64 ? 1 : (n <= 128 ? 2 : 3));
}
int substeps(int algo, int n) {
  static const int kAbia[4] = {8, 4, 2, 1}, kCfa[4] = {4, 2, 1, 1};
  return (algo == FD_ABIA ? kAbia : kCfa)[roll_class(algo, n)];
}
// side stream of a request, by algorithm and chain length only (its FD, adjoint
// solve and reverse sweep launches all go there, in order): CFA length classes
// on streams 0..3, ABIA up to 64 links on 4, longer ABIA on 5
int aux_of(bool abia, int n) {
  if (abia) return n <= 64 ? 4 : 5;
  return n <= 32 ? 0 : (n <= 64 ? 1 : (n <= 128 ? 2 : 3));
}
// side stream of a rollout's steps: ABIA rollouts of up to 20 and 40 links on
// streams 6 and 7, the others on their FD stream (behind its FD+gradient work)
int roll_aux(int algo, int n) {
  if (algo == FD_ABIA && n <= 40) return n <= 20 ? 6 : 7;
  return aux_of(algo == FD_ABIA, n);
}

__global__ void scatter_kernel(const double *stage, const UpDesc *d, int nd, Arena A) {
  const int k = blockIdx.x;
  if (k >= nd) return;
  const UpDesc u = d[k];
  const double *src = stage + u.stage;
  const int n = u.n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    A.q[u.slot + i] = src[i];
    A.qd[u.slot + i] = src[n + i];
    A.tau[u.slot + i] = src[2 * n + i];
    A.w[u.slot + i] = src[3 * n + i];
  }
  if (u.hist >= 0) {
    const int64_t m = static_cast<int64_t>(u.steps - 1) * n;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) A.hist[u.hist + i] = src[4 * n + i];
  }
  if (threadIdx.x == 0) {
    A.r_hist[u.slot] = u.hist;
    A.r_step[u.slot] = 0;
    A.r_steps[u.slot] = u.steps;
    A.r_dt[u.slot] = u.dt;
  }
}

// one semi-implicit Euler step per rollout: qd += dt qdd, q += dt qd, then the
// next step's torque from the request's history; one warp per rollout, lanes
// over its links
__global__ void rollout_step_kernel(const int32_t *prob_chain, const int64_t *model_off,
                                    const int64_t *state_off, int np, Arena A) {
  const int p = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (p >= np) return;
  const int c = prob_chain[p];
  const int n = static_cast<int>(model_off[c + 1] - model_off[c]);
  const int64_t s = state_off[p];
  const double dt = A.r_dt[s];
  const int step = A.r_step[s] + 1;
  const bool more = step < A.r_steps[s];
  const int64_t h = A.r_hist[s] + static_cast<int64_t>(step - 1) * n;
  for (int i = lane; i < n; i += 32) {
    const double v = A.qd[s + i] + dt * A.qdd[s + i];
    A.qd[s + i] = v;
    A.q[s + i] += dt * v;
    if (more) A.tau[s + i] = A.hist[h + i];
  }
  __syncwarp();
  if (lane == 0) A.r_step[s] = step;
}

__global__ void gather_kernel(const OutDesc *d, int nd, Arena A, const int32_t *status,
                              double *out) {
  const int k = blockIdx.x;
  if (k >= nd) return;
  const OutDesc o = d[k];
  double *dst = out + o.out;
  if (threadIdx.x == 0) dst[0] = static_cast<double>(status[o.prob]);
  dst += 1;
  const int n = o.n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (o.kind == FD_REQ_FD_GRAD) {
      dst[i] = A.qdd[o.slot + i];
      dst[n + i] = A.qbar[o.slot + i];
      dst[2 * n + i] = A.qdbar[o.slot + i];
      dst[3 * n + i] = A.tbar[o.slot + i];
    } else {
      dst[i] = A.q[o.slot + i];
      dst[n + i] = A.qd[o.slot + i];
      dst[2 * n + i] = A.qdd[o.slot + i];
    }
  }
}

template <class V>
void grow_pinned(V **p, size_t *cap, size_t need) {
  if (need <= *cap) return;
  size_t c = std::max<size_t>(need, *cap * 2 + 1024);
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  if (cudaHostAlloc(reinterpret_cast<void **>(p), c * sizeof(V), cudaHostAllocDefault) !=
      cudaSuccess) {
    *p = nullptr;
    *cap = 0;
    return;
  }
  *cap = c;
}

}  // namespace

struct fd_server_s {
  int device = 0;
  int flags = 0;
  double grav[3] = {0, 0, 0};
  size_t budget = 0;
  int64_t cap = 0, cap_rec = 0, cap_hist = 0, cap_stage = 0, cap_out = 0;
  char *mem = nullptr;
  Arena A{};
  // device tables (capacity cap problems)
  int32_t *d_prob = nullptr, *d_status = nullptr;
  int64_t *d_moff = nullptr, *d_soff = nullptr;
  double *d_stage = nullptr, *d_out = nullptr;
  UpDesc *d_up = nullptr;
  OutDesc *d_outd = nullptr;
  // pinned host mirrors
  int32_t *h_prob = nullptr;
  int64_t *h_moff = nullptr, *h_soff = nullptr;
  double *h_stage = nullptr, *h_out = nullptr;
  UpDesc *h_up = nullptr;
  OutDesc *h_outd = nullptr;
  size_t c_prob = 0, c_moff = 0, c_soff = 0, c_stage = 0, c_out = 0, c_up = 0, c_outd = 0;
  cudaStream_t stream = nullptr;
  // side streams of a tick, one per length class (four CFA, two ABIA, and two
  // more for short ABIA rollouts); a request's launches (FD with its adjoint's
  // linear solve in the same elimination, the reverse sweep, or a rollout's
  // steps) stay on one of them, in order, and the classes run concurrently
  static constexpr int kAux = 8;
  cudaStream_t aux[kAux] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kAux] = {};

  RangeAlloc slots, recs, hist;
  std::unordered_map<int, Model> models;
  int next_model = 1;
  std::deque<Req *> queued;
  std::vector<Req *> active;
  std::unordered_map<uint64_t, Req *> reqs;
  uint64_t next_ticket = 1;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  fd_status fatal = FD_OK;
  // statistics
  uint64_t ticks = 0, launches = 0, completed = 0;
  double link_solves = 0.0, busy_s = 0.0;
};

namespace {

fd_status sfail(fd_status st, const char *msg) { return fdk_fail(st, msg); }

// Problem tables for active requests [lo, hi) (of `list`), appended at `base`.
void fill_tables(fd_server_s *S, const std::vector<Req *> &list, int base) {
  for (size_t k = 0; k < list.size(); ++k) {
    const Req *r = list[k];
    const int p = base + static_cast<int>(k);
    S->h_prob[p] = 2 * p;
    S->h_moff[2 * p] = r->mrec;
    S->h_moff[2 * p + 1] = r->mrec + r->n;
    S->h_soff[p] = r->slot;
  }
}

fdk::KArgs base_args(fd_server_s *S) {
  fdk::KArgs a{};
  a.model = S->A.model;
  a.model64 = S->A.model;
  a.model_off = S->d_moff;
  a.prob_chain = S->d_prob;
  a.state_off = S->d_soff;
  a.sq_off = S->d_soff;
  a.order = nullptr;
  a.ws_t = S->A.ws_t;
  a.ws_a = S->A.ws_c;
  std::memcpy(a.grav, S->grav, sizeof a.grav);
  return a;
}

// Launch kernel `fn(first, count, team)` over the problems [p0, p0 + np), sorted
// by length within their group: once per team class (a handful of launches) or,
// in the per-size mode, once per distinct chain length.
template <class F>
cudaError_t over(fd_server_s *S, const std::vector<Req *> &all, int p0, int np, TeamKind k,
                 F fn) {
  if (np <= 0) return cudaSuccess;
  const bool per_size = (S->flags & FD_SERVE_PER_SIZE) != 0;
  int s = p0;
  while (s < p0 + np) {
    const int t = team_for(k, all[s]->n);
    int e = s + 1;
    while (e < p0 + np &&
           (per_size ? all[e]->n == all[s]->n : team_for(k, all[e]->n) == t))
      ++e;
    ++S->launches;
    cudaError_t err = fn(s, e - s, t);
    if (err != cudaSuccess) return err;
    s = e;
  }
  return cudaSuccess;
}

fd_status tick(fd_server_s *S, std::unique_lock<std::mutex> &lk) {
  // 1. admission: queued requests, in order, while memory allows
  std::vector<Req *> admitted;
  int64_t stage_need = 0;
  while (!S->queued.empty()) {
    Req *r = S->queued.front();
    const int64_t hn = r->kind == FD_REQ_ROLLOUT ? static_cast<int64_t>(r->steps - 1) * r->n : 0;
    const int64_t need = 4 * r->n + hn;
    if (stage_need + need > S->cap_stage) break;
    const int64_t slot = S->slots.alloc(r->n);
    if (slot < 0) break;
    int64_t h = -1;
    if (hn > 0) {
      h = S->hist.alloc(hn);
      if (h < 0) {
        S->slots.release(slot, r->n);
        break;
      }
    }
    r->slot = slot;
    r->hist = h;
    r->state = 1;
    S->queued.pop_front();
    admitted.push_back(r);
    stage_need += need;
  }
  for (Req *r : admitted) S->active.push_back(r);
  if (S->active.empty()) return FD_OK;
  // work on a snapshot; submissions may continue meanwhile
  std::vector<Req *> act = S->active;
  lk.unlock();
  auto pinned_ok = [&] {
    return S->h_prob && S->h_moff && S->h_soff && (admitted.empty() || (S->h_stage && S->h_up));
  };
  const double t0 = now_s();
  cudaError_t e = cudaSuccess;

  // upload admitted requests' states (one copy) and scatter them to their slots
  if (!admitted.empty()) {
    grow_pinned(&S->h_stage, &S->c_stage, static_cast<size_t>(stage_need));
    grow_pinned(&S->h_up, &S->c_up, admitted.size());
    int64_t off = 0;
    for (size_t k = 0; k < admitted.size() && S->h_stage && S->h_up; ++k) {
      Req *r = admitted[k];
      const int n = r->n;
      double *dst = S->h_stage + off;
      std::memcpy(dst, r->q.data(), n * sizeof(double));
      std::memcpy(dst + n, r->qd.data(), n * sizeof(double));
      std::memcpy(dst + 2 * n, r->tau.data(), n * sizeof(double));
      if (r->kind == FD_REQ_FD_GRAD) std::memcpy(dst + 3 * n, r->w.data(), n * sizeof(double));
      else std::memset(dst + 3 * n, 0, n * sizeof(double));
      int64_t len = 4 * n;
      if (r->hist >= 0) {
        const int64_t hn = static_cast<int64_t>(r->steps - 1) * n;
        std::memcpy(dst + 4 * n, r->tau.data() + n, hn * sizeof(double));
        len += hn;
      }
      S->h_up[k] = UpDesc{off, r->slot, r->hist, n, r->kind, r->steps, 0, r->dt};
      off += len;
    }
    e = cudaMemcpyAsync(S->d_stage, S->h_stage, off * sizeof(double), cudaMemcpyHostToDevice,
                        S->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(S->d_up, S->h_up, admitted.size() * sizeof(UpDesc),
                          cudaMemcpyHostToDevice, S->stream);
    if (e == cudaSuccess) {
      scatter_kernel<<<static_cast<unsigned>(admitted.size()), 128, 0, S->stream>>>(
          S->d_stage, S->d_up, static_cast<int>(admitted.size()), S->A);
      ++S->launches;
      e = cudaGetLastError();
    }
  }

  // 2. problem order: [CFA FD+grad | CFA rollout | ABIA FD+grad | ABIA rollout],
  // each sorted by length (the per-size mode launches one kernel per length)
  // (rollouts: within a team class, by the steps they take this tick, so that the
  // k-th step of the tick covers a prefix of the class)
  const bool per_size = (S->flags & FD_SERVE_PER_SIZE) != 0;
  std::vector<Req *> groups[4];
  for (Req *r : act) {
    const bool first = r->step == 0;
    const int g = (r->algo == FD_CFA ? 0 : 2) + (r->kind == FD_REQ_ROLLOUT ? 1 : 0);
    if (r->kind == FD_REQ_FD_GRAD && !first) continue;  // finished last tick
    r->adv = r->kind == FD_REQ_ROLLOUT
                 ? std::min(per_size ? 1 : substeps(r->algo, r->n), r->steps - r->step)
                 : 1;
    groups[g].push_back(r);
  }
  std::vector<Req *> all;
  int gstart[5] = {0, 0, 0, 0, 0};
  for (int g = 0; g < 4; ++g) {
    const int algo = g < 2 ? FD_CFA : FD_ABIA;
    std::stable_sort(groups[g].begin(), groups[g].end(), [&](const Req *x, const Req *y) {
      if (per_size || (g & 1) == 0) return x->n > y->n;
      const int cx = roll_class(algo, x->n), cy = roll_class(algo, y->n);
      if (cx != cy) return cx > cy;
      if (x->adv != y->adv) return x->adv > y->adv;
      return x->n > y->n;
    });
    gstart[g] = static_cast<int>(all.size());
    all.insert(all.end(), groups[g].begin(), groups[g].end());
  }
  gstart[4] = static_cast<int>(all.size());
  const int np = gstart[4];
  grow_pinned(&S->h_prob, &S->c_prob, np + 1);
  grow_pinned(&S->h_moff, &S->c_moff, 2 * np + 2);
  grow_pinned(&S->h_soff, &S->c_soff, np + 1);
  if (!pinned_ok()) e = cudaErrorMemoryAllocation;
  if (e == cudaSuccess) fill_tables(S, all, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S->d_prob, S->h_prob, np * sizeof(int32_t), cudaMemcpyHostToDevice,
                        S->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S->d_moff, S->h_moff, 2 * np * sizeof(int64_t), cudaMemcpyHostToDevice,
                        S->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S->d_soff, S->h_soff, np * sizeof(int64_t), cudaMemcpyHostToDevice,
                        S->stream);

  // 3. forward dynamics of every active request, on the side streams
  if (e == cudaSuccess) e = cudaEventRecord(S->ev_fork, S->stream);
  for (int k = 0; k < fd_server_s::kAux && e == cudaSuccess; ++k)
    e = cudaStreamWaitEvent(S->aux[k], S->ev_fork, 0);
  auto fd_range = [&](int algo, int mode, int s, int c, int t, cudaStream_t st,
                      bool scan = false) {
    fdk::KArgs a = base_args(S);
    a.prob_chain = S->d_prob + s;
    a.state_off = S->d_soff + s;
    a.n_problems = c;
    a.q = S->A.q;
    a.qd = S->A.qd;
    a.in3 = S->A.tau;
    a.out = S->A.qdd;
    a.in4 = S->A.w;     // MODE_FD2: lambda = M^-1 w beside qdd
    a.out4 = S->A.tbar;
    a.mode = mode;
    a.status = S->d_status + s;
    a.team = t;
    a.ws_a = algo == FD_CFA ? S->A.ws_c : S->A.ws_b;
    if (algo == FD_CFA) return fdk::launch_cfa(a, 0, t, st);
    if (scan) return fdk::launch_abia_scan(a, 0, t, st);
    return fdk::launch_abia(a, 0, t, st);
  };
  auto fd_launch = [&](int algo, int mode, int p0, int cnt) {
    const TeamKind k = algo == FD_CFA ? kTeamCFA : kTeamABIA;
    return over(S, all, p0, cnt, k, [&](int s, int c, int t) {
      return fd_range(algo, mode, s, c, t, S->aux[aux_of(algo != FD_CFA, all[s]->n)]);
    });
  };
  // rollouts: per team class, step j of the tick (FD, then one semi-implicit Euler
  // step) over the class's requests that take more than j steps, a prefix of it;
  // all on the class's side stream, in order
  auto roll_launch = [&](int algo, int p0, int cnt) -> cudaError_t {
    const TeamKind k = algo == FD_CFA ? kTeamCFA : kTeamABIA;
    int s = p0;
    while (s < p0 + cnt) {
      const int rc = roll_class(algo, all[s]->n);
      int e2 = s + 1;
      while (e2 < p0 + cnt &&
             (per_size ? all[e2]->n == all[s]->n : roll_class(algo, all[e2]->n) == rc))
        ++e2;
      const bool scan = algo == FD_ABIA && all[s]->n > kScanAbove;
      const int c = e2 - s, t = scan ? kScanTeam : team_for(k, all[s]->n);
      cudaStream_t st = S->aux[roll_aux(algo, all[s]->n)];
      for (int j = 0; j < all[s]->adv; ++j) {
        int cj = 0;
        while (cj < c && all[s + cj]->adv > j) ++cj;
        S->launches += 2;
        cudaError_t err = fd_range(algo, fdk::MODE_FD, s, cj, t, st, scan);
        if (err != cudaSuccess) return err;
        rollout_step_kernel<<<(cj + 3) / 4, 128, 0, st>>>(S->d_prob + s, S->d_moff,
                                                          S->d_soff + s, cj, S->A);
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
      }
      s = e2;
    }
    return cudaSuccess;
  };
  // FD+gradient requests: qdd and lambda = M^-1 w in one elimination (MODE_FD2)
  if (e == cudaSuccess) e = fd_launch(FD_CFA, fdk::MODE_FD2, gstart[0], gstart[1] - gstart[0]);
  if (e == cudaSuccess) e = fd_launch(FD_ABIA, fdk::MODE_FD2, gstart[2], gstart[3] - gstart[2]);
  auto reverse = [&](int p0, int cnt, bool abia) {
    return over(S, all, p0, cnt, kTeamReverse, [&](int s, int c, int t) {
      fdk::KArgs a = base_args(S);
      a.prob_chain = S->d_prob + s;
      a.state_off = S->d_soff + s;
      a.n_problems = c;
      a.team = t;
      a.q = S->A.q;
      a.qd = S->A.qd;
      a.in3 = S->A.qdd;
      a.lam = S->A.tbar;
      a.out = S->A.qbar;
      a.out2 = S->A.qdbar;
      a.out3 = nullptr;
      a.ws_t = S->A.ws_r;
      return fdk::launch_adjoint_rnea(a, 0, t, S->aux[aux_of(abia, all[s]->n)]);
    });
  };
  if (e == cudaSuccess) e = reverse(gstart[0], gstart[1] - gstart[0], false);
  if (e == cudaSuccess) e = reverse(gstart[2], gstart[3] - gstart[2], true);
  // rollouts: their steps of this tick, queued behind the FD+gradient work of the
  // same side stream
  if (e == cudaSuccess) e = roll_launch(FD_CFA, gstart[1], gstart[2] - gstart[1]);
  if (e == cudaSuccess) e = roll_launch(FD_ABIA, gstart[3], gstart[4] - gstart[3]);
  for (int k = 0; k < fd_server_s::kAux && e == cudaSuccess; ++k) {
    e = cudaEventRecord(S->ev_join[k], S->aux[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(S->stream, S->ev_join[k], 0);
  }

  // 4. which requests finish this tick (rollouts advanced on their side streams)
  std::vector<Req *> done;
  for (int g = 0; g < 4; ++g)
    for (int p = gstart[g]; p < gstart[g + 1]; ++p) {
      Req *r = all[p];
      if (r->kind == FD_REQ_FD_GRAD || r->step + r->adv >= r->steps) done.push_back(r);
    }

  // 5. gather the finished requests' results into one download
  int64_t out_len = 0;
  if (!done.empty()) {
    grow_pinned(&S->h_outd, &S->c_outd, done.size());
    std::unordered_map<const Req *, int> pos;
    for (int p = 0; p < np; ++p) pos[all[p]] = p;
    for (size_t k = 0; k < done.size(); ++k) {
      Req *r = done[k];
      S->h_outd[k] = OutDesc{r->slot, out_len, r->n, r->kind, pos[r], 0};
      out_len += 1 + (r->kind == FD_REQ_FD_GRAD ? 4 : 3) * static_cast<int64_t>(r->n);
    }
    if (out_len > S->cap_out) e = cudaErrorMemoryAllocation;
    grow_pinned(&S->h_out, &S->c_out, static_cast<size_t>(out_len));
    if (!S->h_out || !S->h_outd) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(S->d_outd, S->h_outd, done.size() * sizeof(OutDesc),
                          cudaMemcpyHostToDevice, S->stream);
    if (e == cudaSuccess) {
      gather_kernel<<<static_cast<unsigned>(done.size()), 128, 0, S->stream>>>(
          S->d_outd, static_cast<int>(done.size()), S->A, S->d_status, S->d_out);
      ++S->launches;
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(S->h_out, S->d_out, out_len * sizeof(double), cudaMemcpyDeviceToHost,
                          S->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
  const double t1 = now_s();

  lk.lock();
  if (e != cudaSuccess) {
    cudaGetLastError();
    S->fatal = FD_ERR_CUDA;
    return fdk_fail(FD_ERR_CUDA, cudaGetErrorString(e));
  }
  S->ticks += 1;
  S->busy_s += t1 - t0;
  for (Req *r : all) {
    S->link_solves += static_cast<double>(r->n) * r->adv;
    if (r->kind == FD_REQ_ROLLOUT) r->step += r->adv;
  }
  for (size_t k = 0; k < done.size(); ++k) {
    Req *r = done[k];
    const double *src = S->h_out + S->h_outd[k].out;
    r->status = static_cast<int32_t>(src[0]);
    r->out.assign(src + 1, src + 1 + (r->kind == FD_REQ_FD_GRAD ? 4 : 3) * r->n);
    if (r->kind == FD_REQ_FD_GRAD) r->step = 1;
    r->t_done = t1;
    r->state = 2;
    S->slots.release(r->slot, r->n);
    if (r->hist >= 0) S->hist.release(r->hist, static_cast<int64_t>(r->steps - 1) * r->n);
    S->models[r->model].refs -= 1;
    S->completed += 1;
  }
  S->active.erase(std::remove_if(S->active.begin(), S->active.end(),
                                 [](const Req *r) { return r->state == 2; }),
                  S->active.end());
  S->cv_done.notify_all();
  return FD_OK;
}

void worker_main(fd_server_s *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    if (S->active.empty() && S->queued.empty()) {
      S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    const size_t before = S->active.size();
    if (tick(S, lk) != FD_OK) {
      S->cv_done.notify_all();
      break;
    }
    if (S->active.empty() && !S->queued.empty() && before == 0) {
      // nothing admitted: the head request waits for memory held elsewhere
      S->cv_work.wait_for(lk, std::chrono::milliseconds(1));
    }
  }
}

size_t per_link_bytes() {
  return 8 * sizeof(double) +
         (fdk::NT + fdk::NA_CFA + fdk::NA_ABIA + fdk::NT_ADJ) * sizeof(double) +
         sizeof(int64_t) + 2 * sizeof(int32_t) + sizeof(double) +
         2 * sizeof(int32_t) + 3 * sizeof(int64_t);
}

// streams and events of a server (null handles are skipped)
void destroy_streams(fd_server_s *S) {
  for (int k = 0; k < fd_server_s::kAux; ++k) {
    if (S->aux[k]) cudaStreamSynchronize(S->aux[k]);
    if (S->aux[k]) cudaStreamDestroy(S->aux[k]);
    if (S->ev_join[k]) cudaEventDestroy(S->ev_join[k]);
  }

  if (S->ev_fork) cudaEventDestroy(S->ev_fork);
  if (S->stream) cudaStreamDestroy(S->stream);
}

}  // namespace

extern "C" {

double fd_serve_clock(void) { return now_s(); }

fd_status fd_serve_create(int32_t device, size_t mem_budget_bytes, const double gravity[3],
                          int32_t flags, fd_server_t *out) {
  if (!out) return sfail(FD_ERR_INVALID_ARG, "fd_serve_create: out is NULL");
  *out = nullptr;
  if (!gravity) return sfail(FD_ERR_INVALID_ARG, "fd_serve_create: gravity is NULL");
  if (mem_budget_bytes < (size_t(16) << 20))
    return sfail(FD_ERR_INVALID_ARG, "fd_serve_create: budget below 16 MiB");
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || n_dev == 0) {
    cudaGetLastError();
    return sfail(FD_ERR_CUDA, "fd_serve_create: no CUDA device");
  }
  if (device < 0 || device >= n_dev) return sfail(FD_ERR_INVALID_ARG, "fd_serve_create: device");
  auto *S = new fd_server_s();
  S->device = device;
  S->flags = flags;
  S->budget = mem_budget_bytes;
  std::memcpy(S->grav, gravity, sizeof S->grav);
  // budget split: 10% models, 15% rollout torques, 5% staging, the rest link slots
  const size_t b = mem_budget_bytes;
  S->cap_rec = static_cast<int64_t>(b / 10 / (fdk::REC * sizeof(double)));
  S->cap_hist = static_cast<int64_t>(b * 15 / 100 / sizeof(double));
  S->cap_stage = static_cast<int64_t>(b * 25 / 1000 / sizeof(double));
  S->cap_out = S->cap_stage;
  const size_t rest = b - size_t(S->cap_rec) * fdk::REC * 8 - size_t(S->cap_hist) * 8 -
                      size_t(S->cap_stage + S->cap_out) * 8 - (size_t(1) << 20);
  S->cap = static_cast<int64_t>(rest / (per_link_bytes() + sizeof(UpDesc) + sizeof(OutDesc)));
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&S->mem), mem_budget_bytes);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
  for (int k = 0; k < fd_server_s::kAux && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&S->aux[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_join[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_fork, cudaEventDisableTiming);

  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (S->mem) cudaFree(S->mem);
    destroy_streams(S);
    delete S;
    return sfail(e == cudaErrorMemoryAllocation ? FD_ERR_OOM : FD_ERR_CUDA,
                 "fd_serve_create: device allocation of the budget failed");
  }
  char *p = S->mem;
  auto take = [&](size_t bytes) {
    char *r = p;
    p += (bytes + 255) & ~size_t(255);
    return r;
  };
  const int64_t C = S->cap;
  S->A.model = reinterpret_cast<double *>(take(size_t(S->cap_rec) * fdk::REC * 8));
  S->A.hist = reinterpret_cast<double *>(take(size_t(S->cap_hist) * 8));
  S->d_stage = reinterpret_cast<double *>(take(size_t(S->cap_stage) * 8));
  S->d_out = reinterpret_cast<double *>(take(size_t(S->cap_out) * 8));
  double **arrs[] = {&S->A.q, &S->A.qd, &S->A.tau, &S->A.qdd, &S->A.w, &S->A.qbar, &S->A.qdbar,
                     &S->A.tbar};
  for (double **a : arrs) *a = reinterpret_cast<double *>(take(size_t(C) * 8));
  S->A.ws_t = reinterpret_cast<double *>(take(size_t(C) * fdk::NT * 8));
  S->A.ws_r = reinterpret_cast<double *>(take(size_t(C) * fdk::NT_ADJ * 8));
  S->A.ws_c = reinterpret_cast<double *>(take(size_t(C) * fdk::NA_CFA * 8));
  S->A.ws_b = reinterpret_cast<double *>(take(size_t(C) * fdk::NA_ABIA * 8));

  S->A.r_hist = reinterpret_cast<int64_t *>(take(size_t(C) * 8));
  S->A.r_step = reinterpret_cast<int32_t *>(take(size_t(C) * 4));
  S->A.r_steps = reinterpret_cast<int32_t *>(take(size_t(C) * 4));
  S->A.r_dt = reinterpret_cast<double *>(take(size_t(C) * 8));
  S->d_prob = reinterpret_cast<int32_t *>(take(size_t(C) * 4));
  S->d_status = reinterpret_cast<int32_t *>(take(size_t(C) * 4));
  S->d_moff = reinterpret_cast<int64_t *>(take(size_t(C) * 16));
  S->d_soff = reinterpret_cast<int64_t *>(take(size_t(C) * 8));
  S->d_up = reinterpret_cast<UpDesc *>(take(size_t(C) * sizeof(UpDesc)));
  S->d_outd = reinterpret_cast<OutDesc *>(take(size_t(C) * sizeof(OutDesc)));
  if (p > S->mem + mem_budget_bytes) {
    cudaFree(S->mem);
    destroy_streams(S);
    delete S;
    return sfail(FD_ERR_INVALID_ARG, "fd_serve_create: budget too small for its tables");
  }
  S->slots.reset(C);
  S->recs.reset(S->cap_rec);
  S->hist.reset(S->cap_hist);
  S->worker = std::thread(worker_main, S);
  *out = S;
  return FD_OK;
}

fd_status fd_serve_destroy(fd_server_t S) {
  if (!S) return sfail(FD_ERR_INVALID_ARG, "fd_serve_destroy: NULL");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(S->device);
  cudaStreamSynchronize(S->stream);
  destroy_streams(S);
  cudaFree(S->mem);
  cudaFreeHost(S->h_prob);
  cudaFreeHost(S->h_moff);
  cudaFreeHost(S->h_soff);
  cudaFreeHost(S->h_stage);
  cudaFreeHost(S->h_out);
  cudaFreeHost(S->h_up);
  cudaFreeHost(S->h_outd);
  cudaSetDevice(prev);
  cudaGetLastError();
  for (auto &kv : S->reqs) delete kv.second;
  delete S;
  return FD_OK;
}

fd_status fd_serve_add_model(fd_server_t S, int32_t n_links, const double *joint_axes,
                             const double *link_frames, const double *spatial_inertias,
                             int32_t *model_id) {
  if (!S || !model_id) return sfail(FD_ERR_INVALID_ARG, "fd_serve_add_model: NULL argument");
  if (n_links < 1 || n_links > 4096 || !joint_axes || !link_frames || !spatial_inertias)
    return sfail(FD_ERR_INVALID_ARG, "fd_serve_add_model: need 1..4096 links and model arrays");
  std::vector<double> rec(static_cast<size_t>(n_links) * fdk::REC, 0.0);
  bool rigid = true;
  fd_status st = fdk_pack_chain(0, n_links, joint_axes, link_frames, spatial_inertias,
                                rec.data(), &rigid);
  if (st != FD_OK) return st;
  std::lock_guard<std::mutex> lk(S->mu);
  const int64_t at = S->recs.alloc(n_links);
  if (at < 0) return sfail(FD_ERR_OOM, "fd_serve_add_model: model region of the budget is full");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(S->device);
  cudaError_t e = cudaMemcpy(S->A.model + at * fdk::REC, rec.data(), rec.size() * sizeof(double),
                             cudaMemcpyHostToDevice);
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    S->recs.release(at, n_links);
    return sfail(FD_ERR_CUDA, "fd_serve_add_model: copy to the device failed");
  }
  const int id = S->next_model++;
  Model m;
  m.n = n_links;
  m.rec = at;
  S->models[id] = m;
  *model_id = id;
  return FD_OK;
}

fd_status fd_serve_remove_model(fd_server_t S, int32_t model_id) {
  if (!S) return sfail(FD_ERR_INVALID_ARG, "fd_serve_remove_model: NULL server");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->models.find(model_id);
  if (it == S->models.end()) return sfail(FD_ERR_INVALID_ARG, "fd_serve_remove_model: unknown id");
  if (it->second.refs > 0) return sfail(FD_ERR_BUSY, "fd_serve_remove_model: model in use");
  S->recs.release(it->second.rec, it->second.n);
  S->models.erase(it);
  return FD_OK;
}

fd_status fd_serve_submit(fd_server_t S, const fd_request *rq, uint64_t *ticket) {
  if (!S || !rq || !ticket) return sfail(FD_ERR_INVALID_ARG, "fd_serve_submit: NULL argument");
  if (rq->kind != FD_REQ_FD_GRAD && rq->kind != FD_REQ_ROLLOUT)
    return sfail(FD_ERR_INVALID_ARG, "fd_serve_submit: bad request kind");
  if (rq->algo != FD_ABIA && rq->algo != FD_CFA)
    return sfail(FD_ERR_UNSUPPORTED, "fd_serve_submit: serving runs FD_ABIA or FD_CFA");
  if (!rq->q || !rq->qdot || !rq->tau || (rq->kind == FD_REQ_FD_GRAD && !rq->qddot_bar))
    return sfail(FD_ERR_INVALID_ARG, "fd_serve_submit: NULL state array");
  if (rq->kind == FD_REQ_ROLLOUT && (rq->steps < 1 || !(rq->dt > 0.0)))
    return sfail(FD_ERR_INVALID_ARG, "fd_serve_submit: rollout needs steps >= 1 and dt > 0");
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->fatal != FD_OK) return sfail(S->fatal, "fd_serve_submit: the server stopped on an error");
  auto it = S->models.find(rq->model_id);
  if (it == S->models.end()) return sfail(FD_ERR_INVALID_ARG, "fd_serve_submit: unknown model id");
  const int n = it->second.n;
  const int steps = rq->kind == FD_REQ_ROLLOUT ? rq->steps : 1;
  if (n > S->cap || int64_t(steps - 1) * n > S->cap_hist || 4LL * n + int64_t(steps - 1) * n > S->cap_stage)
    return sfail(FD_ERR_INVALID_ARG, "fd_serve_submit: request larger than the budget allows");
  if (S->queued.size() >= 1000000)
    return sfail(FD_ERR_BUSY, "fd_serve_submit: queue full, retry later");
  auto *r = new Req();
  r->ticket = S->next_ticket++;
  r->kind = rq->kind;
  r->algo = rq->algo;
  r->model = rq->model_id;
  r->n = n;
  r->mrec = it->second.rec;
  r->steps = steps;
  r->dt = rq->dt;
  r->q.assign(rq->q, rq->q + n);
  r->qd.assign(rq->qdot, rq->qdot + n);
  r->tau.assign(rq->tau, rq->tau + static_cast<size_t>(steps) * n);
  if (rq->kind == FD_REQ_FD_GRAD) r->w.assign(rq->qddot_bar, rq->qddot_bar + n);
  r->t_submit = now_s();
  it->second.refs += 1;
  S->reqs[r->ticket] = r;
  S->queued.push_back(r);
  *ticket = r->ticket;
  lk.unlock();
  S->cv_work.notify_one();
  return FD_OK;
}

static void copy_result(const Req *r, fd_result *out) {
  out->status = r->status;
  out->n_links = r->n;
  out->steps_done = r->step;
  out->submit_time = r->t_submit;
  out->done_time = r->t_done;
  const int n = r->n;
  auto put = [&](double *dst, int k) {
    if (dst) std::memcpy(dst, r->out.data() + static_cast<size_t>(k) * n, n * sizeof(double));
  };
  if (r->kind == FD_REQ_FD_GRAD) {
    put(out->qddot, 0);
    put(out->q_bar, 1);
    put(out->qdot_bar, 2);
    put(out->tau_bar, 3);
  } else {
    put(out->q, 0);
    put(out->qdot, 1);
    put(out->qddot, 2);
  }
}

fd_status fd_serve_wait(fd_server_t S, uint64_t ticket, int32_t timeout_ms, fd_result *out) {
  if (!S || !out) return sfail(FD_ERR_INVALID_ARG, "fd_serve_wait: NULL argument");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return sfail(FD_ERR_INVALID_ARG, "fd_serve_wait: unknown ticket");
  Req *r = it->second;
  if (r->state != 2 && timeout_ms > 0)
    S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                        [&] { return r->state == 2 || S->fatal != FD_OK; });
  if (r->state != 2) {
    if (S->fatal != FD_OK) return sfail(S->fatal, "fd_serve_wait: the server stopped on an error");
    return timeout_ms > 0 ? sfail(FD_ERR_TIMEOUT, "fd_serve_wait: not done within the timeout")
                          : FD_ERR_BUSY;
  }
  copy_result(r, out);
  S->reqs.erase(it);
  delete r;
  return FD_OK;
}

fd_status fd_serve_poll(fd_server_t S, uint64_t ticket, fd_result *out) {
  return fd_serve_wait(S, ticket, 0, out);
}

fd_status fd_serve_drain(fd_server_t S, int32_t max, uint64_t *tickets, double *submit_times,
                         double *done_times, int32_t *statuses, int32_t *count) {
  if (!S || !count || max < 0 || (max > 0 && (!tickets || !done_times)))
    return sfail(FD_ERR_INVALID_ARG, "fd_serve_drain: bad argument");
  std::lock_guard<std::mutex> lk(S->mu);
  int32_t k = 0;
  for (auto it = S->reqs.begin(); it != S->reqs.end() && k < max;) {
    Req *r = it->second;
    if (r->state != 2) {
      ++it;
      continue;
    }
    tickets[k] = r->ticket;
    if (submit_times) submit_times[k] = r->t_submit;
    done_times[k] = r->t_done;
    if (statuses) statuses[k] = r->status;
    ++k;
    delete r;
    it = S->reqs.erase(it);
  }
  *count = k;
  return S->fatal;
}

fd_status fd_serve_stats(fd_server_t S, fd_serve_stats_t *out) {
  if (!S || !out) return sfail(FD_ERR_INVALID_ARG, "fd_serve_stats: NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  out->ticks = S->ticks;
  out->launches = S->launches;
  out->completed = S->completed;
  out->queued = S->queued.size();
  out->active = S->active.size();
  out->link_slots_used = S->slots.used();
  out->link_slots = S->cap;
  out->link_solves = S->link_solves;
  out->busy_seconds = S->busy_s;
  return FD_OK;
}

}  // extern "C"
