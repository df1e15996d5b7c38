// fd_kernels.cuh -- the forward-dynamics kernels (ABIA, JSIIA, CFA) and the
// inverse-dynamics kernel, generic in the arithmetic type T, the accumulation
// type TA (OEE, articulated inertia, JSIIA Cholesky) and the team size P.
//
// One team of P lanes solves one problem (chain + state). Link i of an n-link
// chain belongs to lane floor(i / S), S = ceil(n / P): each lane runs the
// recursions serially over its segment and the lanes combine their segments'
// operators by a Kogge-Stone scan (Section II-B); P = 1 is the serial recursion.
#pragma once

#include "fd_device.cuh"

namespace fdk {

template <class T>
struct Prob {
  int p;          // problem index
  int n;          // links
  int a, b;       // this lane's segment [a, b)
  const T *rec;   // model records of the chain
  int64_t m0;     // the chain's first record in the arena
  const T *q, *qd, *in3;
  T *out;
  T *wt;          // T workspace of the problem [n][NT]
};

template <class T, int P>
__device__ __forceinline__ bool load_problem(const KArgs &A, const Range &rg, const Team<P> &tm,
                                             Prob<T> &pb, int nt_stride) {
  const long long team =
      rg.t0 + (static_cast<long long>(blockIdx.x - rg.blk0) * blockDim.x + threadIdx.x) / P;
  if (team >= rg.t1) return false;
  const int p = A.order ? A.order[team] : static_cast<int>(team);
  const int c = A.prob_chain ? A.prob_chain[p] : p;  // no map: problem p is chain p
  const int64_t m0 = A.model_off[c];
  const int n = static_cast<int>(A.model_off[c + 1] - m0);
  const int64_t s0 = A.state_off[p];
  const int S = (n + P - 1) / P;
  pb.p = p;
  pb.n = n;
  pb.a = min(tm.r * S, n);
  pb.b = min(pb.a + S, n);
  pb.rec = static_cast<const T *>(A.model) + m0 * REC;
  pb.m0 = m0;
  pb.q = static_cast<const T *>(A.q) + s0;
  pb.qd = static_cast<const T *>(A.qd) + s0;
  pb.in3 = static_cast<const T *>(A.in3) + s0;
  pb.out = static_cast<T *>(A.out) + s0;
  pb.wt = static_cast<T *>(A.ws_t) + s0 * nt_stride;
  return true;
}

// -------------------------------------------------------- inverse dynamics

// Chains up to this many links run inverse dynamics on component lanes
// (id_lanes) when the team has 8..32 lanes; longer ones take the segmented scans.
// The scans cost about three compositions per level of log2 P levels per lane;
// the component lanes about nineteen FP64 instructions per link per lane.
// Measured on GB300 (teams 8, 16, 32): the component lanes are faster up to 32
// links (by 7-50%), even at 64, slower from 128 on.
template <int P>
__host__ __device__ constexpr int lanes_id_max_links() {
  return (P >= 8 && P <= 32) ? 64 : 0;
}

// Eq. 2a-2c with the six components of every twist, acceleration and force on
// lanes 0..5 of the team (lanes 6.. shadow lane 5 and store nothing): the
// recursions run serially over the links, one transport per lane per link,
//   (Ad_{g^-1} x)_k   = (R^T w)_k                        (k < 3)
//                     = (R^T v)_k + (w' x R^T p)_k,  w' = R^T w,
//   (Ad_{g^-1}^T y)_k = (R n)_k + (p x R f)_k          (k < 3)
//                     = (R f)_k,
// the cross-product terms taking the other lanes' rotated components by
// shuffle. Joint transforms and f_i = J_i Vd_i - ad_{V_i}^T J_i V_i, which do
// not recur, run one link per lane. Same outputs as the scans (W_G, W_TD; V_i in
// W_V, f_i in W_F), visible to the whole team on return.
template <class T, int P>
__device__ __forceinline__ void id_lanes(const Team<P> &tm, const Prob<T> &pb, const double *grav,
                                         int mode) {
  static_assert(P >= 8 && P <= 32, "component lanes need a team of 8..32 lanes");
  const int n = pb.n;
  const bool mode_fd = mode == MODE_FD || mode == MODE_FD2 || mode == MODE_RES;
  const T *qdd_in = mode == MODE_ID ? pb.in3 : (mode == MODE_RES ? pb.out : nullptr);
  const int r = tm.r < 6 ? tm.r : 5;
  const bool top = r < 3;
  const int k = top ? r : r - 3;
  const int ka = k == 2 ? 0 : k + 1, kb = k == 0 ? 2 : k - 1;  // k+1, k+2 mod 3
  const bool store = tm.r < 6;

  // joint transforms and R^T p, one link per lane
  for (int i = tm.r; i < n; i += P) {
    T *w = pb.wt + static_cast<int64_t>(i) * NT;
    SE3<T> g;
    joint_transform(pb.rec + static_cast<int64_t>(i) * REC, pb.q[i], g);
    st_se3(w + W_G, g);
    if (mode == MODE_LINEAR) {
      w[W_TD] = pb.in3[i];
    } else {
#pragma unroll
      for (int j = 0; j < 3; ++j)
        w[W_PT + j] = g.R[j] * g.p[0] + g.R[3 + j] * g.p[1] + g.R[6 + j] * g.p[2];
    }
  }
  tm.sync();
  if (mode == MODE_LINEAR) return;

  // twist V_i (Eq. 2a) and acceleration Vd_i (Eq. 2b), forward; Vd_i parks in W_F
  T V[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  T Ac[6] = {T(0), T(0), T(0), T(-grav[0]), T(-grav[1]), T(-grav[2])};
  for (int i = 0; i < n; ++i) {
    T *w = pb.wt + static_cast<int64_t>(i) * NT;
    // every lane runs the same FP64 instructions: operands are picked by selects
    // and the cross-product coefficients are zero on the angular lanes
    const T c0 = w[W_G + k], c1 = w[W_G + 3 + k], c2 = w[W_G + 6 + k];
    const T pa = top ? T(0) : w[W_PT + ka], pbk = top ? T(0) : w[W_PT + kb];
    const T qdi = pb.qd[i];
    const T e0 = (r == 0) ? qdi : T(0);
    // twist
    T t = c0 * (top ? V[0] : V[3]) + c1 * (top ? V[1] : V[4]) + c2 * (top ? V[2] : V[5]);
    T oa = __shfl_sync(tm.mask, t, ka, P), ob = __shfl_sync(tm.mask, t, kb, P);
    T y = ((t + e0) + oa * pbk) - ob * pa;
#pragma unroll
    for (int j = 0; j < 6; ++j) V[j] = __shfl_sync(tm.mask, y, j, P);
    if (store) w[W_V + r] = y;
    // acceleration: + ad_{V_i} e_1 qd_i = (0, w_z, -w_y; 0, v_z, -v_y) qd_i (+ e_1 qdd_i)
    const T cv = neg_if(r == 1 ? V[2] : (r == 2 ? V[1] : (r == 4 ? V[5] : (r == 5 ? V[4] : T(0)))),
                        r == 2 || r == 5);
    const T a0 = (r == 0 && qdd_in) ? qdd_in[i] : T(0);
    t = c0 * (top ? Ac[0] : Ac[3]) + c1 * (top ? Ac[1] : Ac[4]) + c2 * (top ? Ac[2] : Ac[5]);
    oa = __shfl_sync(tm.mask, t, ka, P);
    ob = __shfl_sync(tm.mask, t, kb, P);
    y = (((t + a0) + oa * pbk) - ob * pa) + cv * qdi;
#pragma unroll
    for (int j = 0; j < 6; ++j) Ac[j] = __shfl_sync(tm.mask, y, j, P);
    if (store) w[W_F + r] = y;
  }
  tm.sync();

  // f_i = J_i Vd_i - ad_{V_i}^T J_i V_i, one link per lane
  for (int i = tm.r; i < n; i += P) {
    T *w = pb.wt + static_cast<int64_t>(i) * NT;
    const T *rec = pb.rec + static_cast<int64_t>(i) * REC;
    T Vi[6], Ai[6], JV[6], f[6];
    ldv<T, 6>(w + W_V, Vi);
    ldv<T, 6>(w + W_F, Ai);
    sym6_apply(rec + REC_J, Vi, JV);
    sym6_apply(rec + REC_J, Ai, f);
    adT_sub(Vi, JV, f);
    stv<T, 6>(w + W_F, f);
  }
  tm.sync();

  // force F_i = Ad_{g_{i+1}^{-1}}^T F_{i+1} + f_i (Eq. 2c), backward; tau_i = F_i[0] (2d)
  T F[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  for (int i = n - 1; i >= 0; --i) {
    T *w = pb.wt + static_cast<int64_t>(i) * NT;
    const T fi = w[W_F + r];
    T y = fi;
    if (i + 1 < n) {
      const T *wn = w + NT;
      const T c0 = wn[W_G + 3 * k], c1 = wn[W_G + 3 * k + 1], c2 = wn[W_G + 3 * k + 2];
      // the cross product only on the angular lanes (coefficients zero on the others)
      const T pa = top ? wn[W_G + 9 + ka] : T(0), pbk = top ? wn[W_G + 9 + kb] : T(0);
      const T t = c0 * (top ? F[0] : F[3]) + c1 * (top ? F[1] : F[4]) + c2 * (top ? F[2] : F[5]);
      const T fa = __shfl_sync(tm.mask, t, 3 + ka, P), fb = __shfl_sync(tm.mask, t, 3 + kb, P);
      y = ((t + pa * fb) - pbk * fa) + fi;
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) F[j] = __shfl_sync(tm.mask, y, j, P);
    if (tm.r == 0) w[W_TD] = mode_fd ? pb.in3[i] - y : y;
  }
  tm.sync();
}


// Eq. 2a-2c for a team of two: the angular half of every twist, acceleration and
// force on lane 0, the linear half on lane 1, one half-transport per lane per link
// (nine rotation products, and the cross-product term with the other half taken
// by shuffle), against a whole transport per link on each lane for the scans at
// this team size. Joint transforms and f_i, which do not recur, run one link per
// lane. Same outputs as the scans (W_G, W_TD; V_i in W_V, f_i in W_F), visible to
// both lanes on return.
template <class T, int P>
__device__ __forceinline__ void id_pair(const Team<P> &tm, const Prob<T> &pb, const double *grav,
                                        int mode) {
  static_assert(P == 2, "the component pair is a team of two lanes");
  const int n = pb.n;
  const bool mode_fd = mode == MODE_FD || mode == MODE_FD2 || mode == MODE_RES;
  const T *qdd_in = mode == MODE_ID ? pb.in3 : (mode == MODE_RES ? pb.out : nullptr);
  const bool h = tm.r != 0;  // false: components 0..2, true: 3..5
  auto xch = [&](T v) { return __shfl_xor_sync(tm.mask, v, 1); };

  // joint transforms and R^T p, one link per lane
  for (int i = tm.r; i < n; i += P) {
    T *w = pb.wt + static_cast<int64_t>(i) * NT;
    SE3<T> g;
    joint_transform(pb.rec + static_cast<int64_t>(i) * REC, pb.q[i], g);
    st_se3(w + W_G, g);
    if (mode == MODE_LINEAR) {
      w[W_TD] = pb.in3[i];
    } else {
#pragma unroll
      for (int j = 0; j < 3; ++j)
        w[W_PT + j] = g.R[j] * g.p[0] + g.R[3 + j] * g.p[1] + g.R[6 + j] * g.p[2];
    }
  }
  tm.sync();
  if (mode == MODE_LINEAR) return;

  // twist V_i (Eq. 2a) and acceleration Vd_i (Eq. 2b), forward; Vd_i parks in W_F.
  // (Ad_{g^-1} x) = (R^T w; R^T v + R^T w x R^T p): this lane's half of R^T x, and on
  // the linear lane the cross product with the angular lane's half.
  T x[3] = {T(0), T(0), T(0)};                                   // this lane's half of V
  T ax[3] = {h ? T(-grav[0]) : T(0), h ? T(-grav[1]) : T(0), h ? T(-grav[2]) : T(0)};
  for (int i = 0; i < n; ++i) {
    T *w = pb.wt + static_cast<int64_t>(i) * NT;
    T R[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = w[W_G + k];
    const T pt0 = h ? w[W_PT] : T(0), pt1 = h ? w[W_PT + 1] : T(0), pt2 = h ? w[W_PT + 2] : T(0);
    const T qdi = pb.qd[i];
    // twist
    T t[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = R[k] * x[0] + R[3 + k] * x[1] + R[6 + k] * x[2];
    T o[3];  // the angular lane's R^T w on the linear lane
#pragma unroll
    for (int k = 0; k < 3; ++k) o[k] = xch(t[k]);
    x[0] = ((h ? t[0] : t[0] + qdi) + o[1] * pt2) - o[2] * pt1;
    x[1] = (t[1] + o[2] * pt0) - o[0] * pt2;
    x[2] = (t[2] + o[0] * pt1) - o[1] * pt0;
    // the whole V_i for the acceleration's ad_{V_i} e_1 qd_i = (0, w_z, -w_y; 0, v_z, -v_y) qd_i
    const T v1 = x[1], v2 = x[2];
    if (tm.r < 2) {
#pragma unroll
      for (int k = 0; k < 3; ++k) w[W_V + (h ? 3 : 0) + k] = x[k];
    }
    // acceleration
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = R[k] * ax[0] + R[3 + k] * ax[1] + R[6 + k] * ax[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) o[k] = xch(t[k]);
    const T a0 = (!h && qdd_in) ? qdd_in[i] : T(0);
    ax[0] = ((t[0] + a0) + o[1] * pt2) - o[2] * pt1;
    ax[1] = ((t[1] + o[2] * pt0) - o[0] * pt2) + v2 * qdi;
    ax[2] = ((t[2] + o[0] * pt1) - o[1] * pt0) - v1 * qdi;
    if (tm.r < 2) {
#pragma unroll
      for (int k = 0; k < 3; ++k) w[W_F + (h ? 3 : 0) + k] = ax[k];
    }
  }
  tm.sync();

  // f_i = J_i Vd_i - ad_{V_i}^T J_i V_i, one link per lane
  for (int i = tm.r; i < n; i += P) {
    T *w = pb.wt + static_cast<int64_t>(i) * NT;
    const T *rec = pb.rec + static_cast<int64_t>(i) * REC;
    T Vi[6], Ai[6], JV[6], f[6];
    ldv<T, 6>(w + W_V, Vi);
    ldv<T, 6>(w + W_F, Ai);
    sym6_apply(rec + REC_J, Vi, JV);
    sym6_apply(rec + REC_J, Ai, f);
    adT_sub(Vi, JV, f);
    stv<T, 6>(w + W_F, f);
  }
  tm.sync();

  // force F_i = Ad_{g_{i+1}^{-1}}^T F_{i+1} + f_i (Eq. 2c), backward; tau_i = F_i[0] (2d).
  // (Ad_{g^-1}^T y) = (R n + p x R f; R f): this lane's half of R y, and on the
  // angular lane the cross product with the linear lane's half.
  T y[3] = {T(0), T(0), T(0)};
  for (int i = n - 1; i >= 0; --i) {
    T *w = pb.wt + static_cast<int64_t>(i) * NT;
    T f[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) f[k] = w[W_F + (h ? 3 : 0) + k];
    if (i + 1 < n) {
      const T *wn = w + NT;
      T R[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) R[k] = wn[W_G + k];
      const T p0 = h ? T(0) : wn[W_G + 9], p1 = h ? T(0) : wn[W_G + 10], p2 = h ? T(0) : wn[W_G + 11];
      T t[3], o[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) t[k] = R[3 * k] * y[0] + R[3 * k + 1] * y[1] + R[3 * k + 2] * y[2];
#pragma unroll
      for (int k = 0; k < 3; ++k) o[k] = xch(t[k]);  // R f on the angular lane
      y[0] = (((t[0] + p1 * o[2]) - p2 * o[1])) + f[0];
      y[1] = (((t[1] + p2 * o[0]) - p0 * o[2])) + f[1];
      y[2] = (((t[2] + p0 * o[1]) - p1 * o[0])) + f[2];
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) y[k] = f[k];
    }
    if (tm.r == 0) w[W_TD] = mode_fd ? pb.in3[i] - y[0] : y[0];
  }
  tm.sync();
}

// Eq. 2a-2d for one problem: the twist and acceleration recursions (forward,
// block lower bi-diagonal) and the force recursion (backward, block upper
// bi-diagonal), each as a segmented scan over SE(3)-affine operators.
//   MODE_FD, MODE_FD2: qdd = 0 and gravity; writes tau_delta_i = tau_i - tau_bias_i
//   MODE_ID:           qdd = in3;           writes tau_i
//   MODE_RES:          qdd = out;           writes the residual tau_i - ID_i(q, qd, out)
// Leaves g_i, V_i, f_i in the workspace.
template <class T, int P>
__device__ __forceinline__ void id_team(const Team<P> &tm, const Prob<T> &pb, const double *grav,
                                        int mode, bool skip_force = false) {
  if constexpr (P >= 8 && P <= 32) {
    if (pb.n <= lanes_id_max_links<P>()) {
      id_lanes<T, P>(tm, pb, grav, mode);
      return;
    }
  }
  if constexpr (P == 2) {
    id_pair<T, P>(tm, pb, grav, mode);
    return;
  }
  const int a = pb.a, b = pb.b;
  const bool mode_fd = mode == MODE_FD || mode == MODE_FD2 || mode == MODE_RES;
  const T *qdd_in = mode == MODE_ID ? pb.in3 : (mode == MODE_RES ? pb.out : nullptr);
  SegOp<T> op;
  se3_identity(op.h);
  if constexpr (P == 1) {
    // one thread: the joint transform, Eq. 2a and Eq. 2b and f_i in one forward
    // sweep, the twist and acceleration recursions interleaved (two independent
    // dependency chains) and g_i, V_i used from registers
    T V[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    T Vd[6] = {T(0), T(0), T(0), T(-grav[0]), T(-grav[1]), T(-grav[2])};
    for (int i = 0; i < pb.n; ++i) {
      T *w = pb.wt + static_cast<int64_t>(i) * NT;
      const T *rec = pb.rec + static_cast<int64_t>(i) * REC;
      SE3<T> g;
      joint_transform(rec, pb.q[i], g);
      st_se3(w + W_G, g);
      if (mode == MODE_LINEAR) {
        w[W_TD] = pb.in3[i];
        continue;
      }
      const T qdi = pb.qd[i];
      adinv(g, V, V);
      V[0] += qdi;
      adinv(g, Vd, Vd);
      // ad_V e_1 = (0, w_z, -w_y; 0, v_z, -v_y)
      Vd[1] += V[2] * qdi;
      Vd[2] -= V[1] * qdi;
      Vd[4] += V[5] * qdi;
      Vd[5] -= V[4] * qdi;
      if (qdd_in) Vd[0] += qdd_in[i];
      stv<T, 6>(w + W_V, V);
      T JV[6], f[6];
      sym6_apply(rec + REC_J, V, JV);
      sym6_apply(rec + REC_J, Vd, f);
      adT_sub(V, JV, f);  // J Vd - ad_V^T J V
      stv<T, 6>(w + W_F, f);
    }
    if (mode == MODE_LINEAR) return;
  } else {
    // joint transforms and this segment's product h = g_a ... g_{b-1}
    for (int i = a; i < b; ++i) {
      SE3<T> g;
      joint_transform(pb.rec + static_cast<int64_t>(i) * REC, pb.q[i], g);
      st_se3(pb.wt + static_cast<int64_t>(i) * NT + W_G, g);
      if (P > 1) se3_mul(op.h, g, op.h);
      if (mode == MODE_LINEAR) pb.wt[static_cast<int64_t>(i) * NT + W_TD] = pb.in3[i];
    }
    if (mode == MODE_LINEAR) return;
    const T zero6[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    T x[6];

    // ---- twist: V_i = Ad_{g_i^{-1}} V_{i-1} + e_1 qd_i, V_{-1} = 0 (Eq. 2a)
    if (P > 1) {
      for (int k = 0; k < 6; ++k) x[k] = T(0);
      for (int i = a; i < b; ++i) {
        SE3<T> g;
        ld_se3(pb.wt + static_cast<int64_t>(i) * NT + W_G, g);
        adinv(g, x, x);
        x[0] += pb.qd[i];
      }
      for (int k = 0; k < 6; ++k) op.psi[k] = x[k];
      team_scan_fwd(tm, op, zero6, x);
    } else {
      for (int k = 0; k < 6; ++k) x[k] = T(0);
    }
    for (int i = a; i < b; ++i) {
      T *w = pb.wt + static_cast<int64_t>(i) * NT;
      SE3<T> g;
      ld_se3(w + W_G, g);
      adinv(g, x, x);
      x[0] += pb.qd[i];
      stv<T, 6>(w + W_V, x);
    }

    // ---- acceleration: Vd_i = Ad_{g_i^{-1}} Vd_{i-1} + e_1 qdd_i + ad_{V_i} e_1 qd_i,
    //      Vd_{-1} = (0; -g) (Eq. 2b, gravity as base acceleration)
    const T base[6] = {T(0), T(0), T(0), T(-grav[0]), T(-grav[1]), T(-grav[2])};
    auto accel_step = [&](int i, T *xx) {
      const T *w = pb.wt + static_cast<int64_t>(i) * NT;
      SE3<T> g;
      ld_se3(w + W_G, g);
      adinv(g, xx, xx);
      const T *V = w + W_V;
      const T qdi = pb.qd[i];
      // ad_V e_1 = (0, w_z, -w_y; 0, v_z, -v_y)
      xx[1] += V[2] * qdi;
      xx[2] -= V[1] * qdi;
      xx[4] += V[5] * qdi;
      xx[5] -= V[4] * qdi;
      if (qdd_in) xx[0] += qdd_in[i];
    };
    if (P > 1) {
      for (int k = 0; k < 6; ++k) x[k] = T(0);
      for (int i = a; i < b; ++i) accel_step(i, x);
      for (int k = 0; k < 6; ++k) op.psi[k] = x[k];
      team_scan_fwd(tm, op, base, x);
    } else {
      for (int k = 0; k < 6; ++k) x[k] = base[k];
    }
    for (int i = a; i < b; ++i) {
      accel_step(i, x);
      T *w = pb.wt + static_cast<int64_t>(i) * NT;
      const T *rec = pb.rec + static_cast<int64_t>(i) * REC;
      T V[6], JV[6], JA[6];
      ldv<T, 6>(w + W_V, V);
      sym6_apply(rec + REC_J, V, JV);
      sym6_apply(rec + REC_J, x, JA);
      adT_sub(V, JV, JA);  // J Vd - ad_V^T J V
      stv<T, 6>(w + W_F, JA);
    }
  }

  // ---- force: F_i = Ad_{g_{i+1}^{-1}}^T F_{i+1} + f_i, F_n = 0 (Eq. 2c), tau = S^T F (2d);
  // skip_force (serial schedule only) leaves f_i in W_F for the caller's own backward loop
  if (P == 1 && skip_force) return;
  T y[6];
  if (P > 1) {
    for (int k = 0; k < 6; ++k) y[k] = T(0);
    for (int i = b - 1; i >= a; --i) {
      const T *w = pb.wt + static_cast<int64_t>(i) * NT;
      SE3<T> g;
      ld_se3(w + W_G, g);
      for (int k = 0; k < 6; ++k) y[k] += w[W_F + k];
      adinvT(g, y, y);
    }
    for (int k = 0; k < 6; ++k) op.psi[k] = y[k];
    team_scan_bwd(tm, op, y);
  } else {
    for (int k = 0; k < 6; ++k) y[k] = T(0);
  }
  for (int i = b - 1; i >= a; --i) {
    T *w = pb.wt + static_cast<int64_t>(i) * NT;
    SE3<T> g;
    ld_se3(w + W_G, g);
    for (int k = 0; k < 6; ++k) y[k] += w[W_F + k];
    w[W_TD] = mode_fd ? pb.in3[i] - y[0] : y[0];
    adinvT(g, y, y);
  }
}

template <class T, int P>
__device__ __forceinline__ void id_body(const KArgs &A, const Range &rg) {
  Team<P> tm;
  Prob<T> pb;
  if (!load_problem<T, P>(A, rg, tm, pb, NT)) return;
  id_team<T, P>(tm, pb, A.grav, MODE_ID);
  for (int i = pb.a; i < pb.b; ++i) pb.out[i] = pb.wt[static_cast<int64_t>(i) * NT + W_TD];
}

template <class T, int P>
__global__ void __launch_bounds__(block_for<P>()) id_kernel(KArgs A) {
  id_body<T, P>(A, Range{0, 0, A.n_problems});
}

// -------------------------------------------------------------------- CFA

// Row i of a chain's CFA workspace: NA_CFA entries of TA, stored field-major
// over the chain's n rows (entry k of row i at base[k n + i]), so that the lanes
// of a team, working on neighbouring rows, touch neighbouring addresses.
template <class E>
struct RowP {
  E *p;
  int s;
  __device__ __forceinline__ E &operator[](int k) const { return p[static_cast<int64_t>(k) * s]; }
  __device__ __forceinline__ RowP operator+(int k) const {
    return RowP{p + static_cast<int64_t>(k) * s, s};
  }
};
template <class E>
__device__ __forceinline__ RowP<E> rowp(E *wa, int n, int i) {
  return RowP<E>{wa + i, n};
}

// (X K X^T)[1..5][1..5] + Kd[1..5][1..5] into packed lower 5x5, X = Ad_{g^{-1}},
// K, Kd packed symmetric 6x6 (T_ii of Algorithm 1's CalcA, W_i^T T_ii W_i).
// acc + (a0 b0 + a1 b1 + a2 b2): one chain of fused multiply-adds from acc when the
// products are in the accumulation type, else the sum in T added in TA
template <class T, class TA>
__device__ __forceinline__ TA add_dot3(TA acc, T a0, T b0, T a1, T b1, T a2, T b2) {
  if constexpr (std::is_same<T, TA>::value)
    return ((acc + a0 * b0) + a1 * b1) + a2 * b2;
  else
    return acc + TA(a0 * b0 + a1 * b1 + a2 * b2);
}

template <class T, class TA, class Out>
__device__ __forceinline__ void calc_dblock(const SE3<T> *g, const T *Kprev, const T *Kself,
                                            Out D) {
  TA acc[15];
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c) acc[l5(r, c)] = TA(Kself[s6(r + 1, c + 1)]);
  if (g) {
    // X K X^T with X = Ad_{g^{-1}} = [[R^T, 0], [-R^T p^, R^T]] and K = [[A, B],
    // [B^T, C]] in 3x3 blocks: with Bt = B + A p^ (rows: a_r x p) and
    // Cs = C - p^ B + Bt^T p^ ((Cs)_rc = C_rc - (p x b_c)_r + (bt_r x p)_c for the
    // columns b_c of B and bt_r of Bt),
    //   X K X^T = [[R^T A R, R^T Bt R], [R^T Bt^T R, R^T Cs R]];
    // only rows and columns 1..5 are needed (W^T x = x[1..5]).
    const T *R = g->R, *p = g->p;
    T A[3][3], B[3][3], C[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        A[r][c] = Kprev[s6(r, c)];
        B[r][c] = Kprev[s6(r, 3 + c)];
        C[r][c] = Kprev[s6(3 + r, 3 + c)];
      }
    T Bt[3][3], Cs[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      Bt[r][0] = (B[r][0] + A[r][1] * p[2]) - A[r][2] * p[1];
      Bt[r][1] = (B[r][1] + A[r][2] * p[0]) - A[r][0] * p[2];
      Bt[r][2] = (B[r][2] + A[r][0] * p[1]) - A[r][1] * p[0];
    }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c <= r; ++c) {
        const int r1 = (r + 1) % 3, r2 = (r + 2) % 3, c1 = (c + 1) % 3, c2 = (c + 2) % 3;
        T t = C[r][c];
        t = (t - p[r1] * B[r2][c]) + p[r2] * B[r1][c];   // - (p x b_c)_r
        t = (t + Bt[c1][r] * p[c2]) - Bt[c2][r] * p[c1];  // + (bt_r x p)_c
        Cs[r][c] = t;
        Cs[c][r] = t;
      }
    // top-left rows / columns 1..2: (R^T A R)_ab = R_{:,a} . (A R_{:,b})
    T AR[3][2];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int b = 0; b < 2; ++b)
        AR[k][b] = A[k][0] * R[1 + b] + A[k][1] * R[4 + b] + A[k][2] * R[7 + b];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b <= a; ++b)
        acc[l5(a, b)] = add_dot3<T, TA>(acc[l5(a, b)], R[1 + a], AR[0][b], R[4 + a], AR[1][b],
                                        R[7 + a], AR[2][b]);
    // off-diagonal rows 1..2 of R^T Bt R, as rows 3..5 x columns 1..2 of D
    T RB[2][3];  // (R^T Bt)_{a,:} for a = 1, 2
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        RB[a][c] = R[1 + a] * Bt[0][c] + R[4 + a] * Bt[1][c] + R[7 + a] * Bt[2][c];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        acc[l5(2 + b, a)] = add_dot3<T, TA>(acc[l5(2 + b, a)], RB[a][0], R[b], RB[a][1],
                                            R[3 + b], RB[a][2], R[6 + b]);
    // bottom-right R^T Cs R
    T RC[3][3];  // R^T Cs
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        RC[a][c] = R[a] * Cs[0][c] + R[3 + a] * Cs[1][c] + R[6 + a] * Cs[2][c];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b <= a; ++b)
        acc[l5(2 + a, 2 + b)] = add_dot3<T, TA>(acc[l5(2 + a, 2 + b)], RC[a][0], R[b], RC[a][1],
                                                R[3 + b], RC[a][2], R[6 + b]);
  }
#pragma unroll
  for (int k = 0; k < 15; ++k) D[k] = acc[k];
}

// U_i = W_i^T T_{i,i+1} W_{i+1} = -(J_i^{-1} Ad_{g_{i+1}^{-1}}^T)[1..5][1..5].
// Column j of Ad_{g^{-1}}^T = [[R, p^ R], [0, R]] is (R_{:,j}; 0) for j < 3 and
// (p x R_{:,j-3}; R_{:,j-3}) for j >= 3; rows 1..5 of J^{-1} times it.
template <class T, class TA, class Out>
__device__ __forceinline__ void calc_ublock(const SE3<T> &gn, const T *Ki, Out U) {
  const T *R = gn.R, *p = gn.p;
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const T k0 = Ki[s6(r + 1, 0)], k1 = Ki[s6(r + 1, 1)], k2 = Ki[s6(r + 1, 2)];
#pragma unroll
    for (int j = 1; j < 3; ++j)
      U[5 * r + j - 1] = TA(-k0 * R[j] - k1 * R[3 + j] - k2 * R[6 + j]);
    // columns 3..5: k_top . (p x x) + k_bot . x = (k_top x p + k_bot) . x, x = R_{:,m}
    const T a0 = (Ki[s6(r + 1, 3)] + k1 * p[2]) - k2 * p[1];
    const T a1 = (Ki[s6(r + 1, 4)] + k2 * p[0]) - k0 * p[2];
    const T a2 = (Ki[s6(r + 1, 5)] + k0 * p[1]) - k1 * p[0];
#pragma unroll
    for (int m = 0; m < 3; ++m)
      U[5 * r + 2 + m] = TA(-a0 * R[m] - a1 * R[3 + m] - a2 * R[6 + m]);
  }
}

// Per row and level, once: the Cholesky factor L of D, G = L^{-1} U and
// g = L^{-1} R. Both neighbours of the row reuse them (SolvSys of Algorithm 2
// with D = L L^T): E U_{i+d} = Z G_{i+d}, E R_{i+d} = Z g_{i+d} with
// Z = U_i L_{i+d}^{-T}, and K U_{i-d} = G^T G, K R_{i-d} = G^T g of row i-d.
// has_next: U_m couples row m to a row below it (else no G is formed).
template <class TA>
__device__ __forceinline__ bool oee_factor_at(int m, bool has_next, int n, TA *wa, int srcD,
                                              int srcU, int srcR, int srcR2 = -1) {
  const RowP<TA> row = rowp(wa, n, m);
  TA Dm[15], L[15], inv[5];
#pragma unroll
  for (int k = 0; k < 15; ++k) Dm[k] = row[srcD + k];
  const bool ok = chol5(Dm, L, inv);
#pragma unroll
  for (int k = 0; k < 15; ++k) row[A_L + k] = L[k];
#pragma unroll
  for (int k = 0; k < 5; ++k) row[A_LI + k] = inv[k];
  TA r[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) r[k] = row[srcR + k];
  fwd5(L, inv, r);
#pragma unroll
  for (int k = 0; k < 5; ++k) row[A_GR + k] = r[k];
  if (srcR2 >= 0) {  // the second right-hand side: g2 = L^{-1} R2
#pragma unroll
    for (int k = 0; k < 5; ++k) r[k] = row[srcR2 + k];
    fwd5(L, inv, r);
#pragma unroll
    for (int k = 0; k < 5; ++k) row[A_GR2 + k] = r[k];
  }
  if (has_next) {  // U_m couples row m to the next row; zero beyond
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      TA col[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) col[k] = row[srcU + 5 * k + c];
      fwd5(L, inv, col);
#pragma unroll
      for (int k = 0; k < 5; ++k) row[A_G + 5 * k + c] = col[k];
    }
  }
  return ok;
}

template <class TA>
__device__ __forceinline__ bool oee_factor(int m, int d, int n, TA *wa, int srcD, int srcU,
                                           int srcR, int srcR2 = -1) {
  return oee_factor_at<TA>(m, m + d < n, n, wa, srcD, srcU, srcR, srcR2);
}

// One OEE update of row i at distance d (Section IV, update rule and Algorithm 2,
// right-hand sides all at level j-1):
//   D_i -= E_i U_i^T + K_i U_{i-d},  R_i -= E_i R_{i+d} + K_i R_{i-d},
//   U_i = -E_i U_{i+d},  E_i = U_i D_{i+d}^{-1},  K_i = U_{i-d}^T D_{i-d}^{-1}.
// The rows it reads are given explicitly: inext / iprev are the rows row i is
// coupled to below and above (-1: none), has_nn whether inext has a row below it.
template <class TA>
__device__ __forceinline__ void oee_row_at(int i, int inext, bool has_nn, int iprev, int n,
                                           const TA *wa, int srcD, int srcU, int srcR, TA *Dn,
                                           TA *Un, TA *Rn, int srcR2 = -1, TA *Rn2 = nullptr) {
  const RowP<const TA> row = rowp(wa, n, i);
  const bool two = srcR2 >= 0;
#pragma unroll
  for (int k = 0; k < 15; ++k) Dn[k] = row[srcD + k];
#pragma unroll
  for (int k = 0; k < 5; ++k) Rn[k] = row[srcR + k];
  if (two) {
#pragma unroll
    for (int k = 0; k < 5; ++k) Rn2[k] = row[srcR2 + k];
  }
#pragma unroll
  for (int k = 0; k < 25; ++k) Un[k] = TA(0);
  if (inext >= 0) {
    const RowP<const TA> nb = rowp(wa, n, inext);
    TA L[15], inv[5];
#pragma unroll
    for (int k = 0; k < 15; ++k) L[k] = nb[A_L + k];
#pragma unroll
    for (int k = 0; k < 5; ++k) inv[k] = nb[A_LI + k];
    TA Z[5][5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
#pragma unroll
      for (int c = 0; c < 5; ++c) Z[k][c] = row[srcU + 5 * k + c];
      fwd5(L, inv, Z[k]);  // z_k^T = L^{-1} u_k^T  (Z = U_i L^{-T})
    }
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
      for (int c = 0; c <= r; ++c)
#pragma unroll
        for (int k = 0; k < 5; ++k) Dn[l5(r, c)] -= Z[r][k] * Z[c][k];  // E_i U_i^T = Z Z^T
    TA gr[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) gr[k] = nb[A_GR + k];
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
      for (int k = 0; k < 5; ++k) Rn[r] -= Z[r][k] * gr[k];  // E_i R_{i+d} = Z g_{i+d}
    if (two) {
#pragma unroll
      for (int k = 0; k < 5; ++k) gr[k] = nb[A_GR2 + k];
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int k = 0; k < 5; ++k) Rn2[r] -= Z[r][k] * gr[k];
    }
    if (has_nn) {
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          TA s = TA(0);
#pragma unroll
          for (int k = 0; k < 5; ++k) s -= Z[r][k] * nb[A_G + 5 * k + c];
          Un[5 * r + c] = s;  // U_i <- -E_i U_{i+d} = -Z G_{i+d}
        }
    }
  }
  if (iprev >= 0) {
    const RowP<const TA> pr = rowp(wa, n, iprev);
    TA G[5][5];
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
      for (int c = 0; c < 5; ++c) G[k][c] = pr[A_G + 5 * k + c];
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
      for (int c = 0; c <= r; ++c)
#pragma unroll
        for (int k = 0; k < 5; ++k) Dn[l5(r, c)] -= G[k][r] * G[k][c];  // K_i U_{i-d} = G^T G
    TA gr[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) gr[k] = pr[A_GR + k];
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
      for (int k = 0; k < 5; ++k) Rn[r] -= G[k][r] * gr[k];  // K_i R_{i-d} = G^T g
    if (two) {
#pragma unroll
      for (int k = 0; k < 5; ++k) gr[k] = pr[A_GR2 + k];
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int k = 0; k < 5; ++k) Rn2[r] -= G[k][r] * gr[k];
    }
  }
}

template <class TA>
__device__ __forceinline__ void oee_row(int i, int d, int n, const TA *wa, int srcD, int srcU,
                                        int srcR, TA *Dn, TA *Un, TA *Rn, int srcR2 = -1,
                                        TA *Rn2 = nullptr) {
  oee_row_at<TA>(i, i + d < n ? i + d : -1, i + 2 * d < n, i - d >= 0 ? i - d : -1, n, wa, srcD,
                 srcU, srcR, Dn, Un, Rn, srcR2, Rn2);
}

// Block cyclic reduction of the symmetric block tri-diagonal system (the
// work-efficient alternative to OEE): at level j (distance d = 2^{j-1}) the
// active rows are i with (i + 1) % d == 0; those with (i + 1) / d odd are
// eliminated: they factor themselves (L, G = L^{-1} U, g = L^{-1} R, as in OEE)
// and keep their lower coupling; the others are updated in place with the OEE
// row formulas. About n row updates in total instead of n ceil(log2 n). Back
// substitution then solves the rows level by level from the last one down:
// x_i = D_i^{-1} (R_i - U_{i-d}^T x_{i-d} - U_i x_{i+d}).
//
// cr_solve_map runs it on a system of N rows stored at rows row(0) < ... <
// row(N-1) of a chain's n-row workspace: row(r)'s U0 couples it to row(r+1)
// (the hybrid schedule's reduced system); cr_solve is the identity map.
template <class TA, int P, class Map>
__device__ __forceinline__ bool cr_solve_map(const Team<P> &tm, TA *wa, int n, int N,
                                             const Map &row_of, bool two) {
  bool bad = false;
  int levels = 0;
  while ((1 << levels) < N) ++levels;
  // the active rows of level j are i = (t + 1) d - 1, t = 0, 1, ...: lanes take t
  // round robin (t even: eliminated, t odd: kept)
  for (int j = 1; j <= levels; ++j) {
    const int d = 1 << (j - 1);
    for (int t = 2 * tm.r; (t + 1) * d - 1 < N; t += 2 * P) {  // eliminated rows
      const int m = (t + 1) * d - 1;
      const int rm = row_of(m);
      bad |= !oee_factor_at<TA>(rm, m + d < N, n, wa, A_D0, A_U0, A_R0, two ? A_R20 : -1);
      if (m - d >= 0) {  // keep the lower coupling for the back substitution
        const RowP<TA> lo = rowp(wa, n, row_of(m - d)) + A_U0;
        const RowP<TA> row = rowp(wa, n, rm);
#pragma unroll
        for (int k = 0; k < 25; ++k) row[A_LO + k] = lo[k];
      }
    }
    tm.sync();
    for (int t = 2 * tm.r + 1; (t + 1) * d - 1 < N; t += 2 * P) {  // kept rows: update in place
      const int i = (t + 1) * d - 1;
      const int ri = row_of(i);
      TA Dn[15], Un[25], Rn[5], Rn2[5];
      oee_row_at<TA>(ri, i + d < N ? row_of(i + d) : -1, i + 2 * d < N,
                     i - d >= 0 ? row_of(i - d) : -1, n, wa, A_D0, A_U0, A_R0, Dn, Un, Rn,
                     two ? A_R20 : -1, Rn2);
      const RowP<TA> row = rowp(wa, n, ri);
#pragma unroll
      for (int k = 0; k < 15; ++k) row[A_D0 + k] = Dn[k];
#pragma unroll
      for (int k = 0; k < 25; ++k) row[A_U0 + k] = Un[k];
#pragma unroll
      for (int k = 0; k < 5; ++k) row[A_R0 + k] = Rn[k];
      if (two) {
#pragma unroll
        for (int k = 0; k < 5; ++k) row[A_R20 + k] = Rn2[k];
      }
    }
    tm.sync();
  }
  // rows never eliminated (N a power of two: row N - 1) are decoupled by now;
  // a row is eliminated at level 1 + (trailing zeros of i + 1)
  for (int i = tm.r; i < N; i += P) {
    const int je = __ffs(i + 1);
    if (je <= levels) continue;
    const RowP<TA> row = rowp(wa, n, row_of(i));
    TA Dm[15], L[15], inv[5], r[5];
#pragma unroll
    for (int k = 0; k < 15; ++k) Dm[k] = row[A_D0 + k];
#pragma unroll
    for (int k = 0; k < 5; ++k) r[k] = row[A_R0 + k];
    bad |= !chol5(Dm, L, inv);
    fwd5(L, inv, r);
    bwd5(L, inv, r);
#pragma unroll
    for (int k = 0; k < 5; ++k) row[A_FC + k] = r[k];
    if (two) {
#pragma unroll
      for (int k = 0; k < 5; ++k) r[k] = row[A_R20 + k];
      fwd5(L, inv, r);
      bwd5(L, inv, r);
#pragma unroll
      for (int k = 0; k < 5; ++k) row[A_FC2 + k] = r[k];
    }
  }
  tm.sync();
  for (int j = levels; j >= 1; --j) {
    const int d = 1 << (j - 1);
    for (int t = 2 * tm.r; (t + 1) * d - 1 < N; t += 2 * P) {
      const int i = (t + 1) * d - 1;
      const RowP<TA> row = rowp(wa, n, row_of(i));
      TA L[15], inv[5];
#pragma unroll
      for (int k = 0; k < 15; ++k) L[k] = row[A_L + k];
#pragma unroll
      for (int k = 0; k < 5; ++k) inv[k] = row[A_LI + k];
      for (int h = 0; h < (two ? 2 : 1); ++h) {
        const int fR = h ? A_R20 : A_R0, fX = h ? A_FC2 : A_FC;
        TA r[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) r[k] = row[fR + k];
        if (i + d < N) {  // - U_i x_{i+d}
          const RowP<TA> xn = rowp(wa, n, row_of(i + d)) + fX;
#pragma unroll
          for (int rr = 0; rr < 5; ++rr)
#pragma unroll
            for (int k = 0; k < 5; ++k) r[rr] -= row[A_U0 + 5 * rr + k] * xn[k];
        }
        if (i - d >= 0) {  // - U_{i-d}^T x_{i-d}
          const RowP<TA> xp = rowp(wa, n, row_of(i - d)) + fX;
#pragma unroll
          for (int rr = 0; rr < 5; ++rr)
#pragma unroll
            for (int k = 0; k < 5; ++k) r[rr] -= row[A_LO + 5 * k + rr] * xp[k];
        }
        fwd5(L, inv, r);
        bwd5(L, inv, r);
#pragma unroll
        for (int k = 0; k < 5; ++k) row[fX + k] = r[k];
      }
    }
    tm.sync();
  }
  return bad;
}

struct IdentityRows {
  __device__ __forceinline__ int operator()(int r) const { return r; }
};

template <class TA, int P>
__device__ __forceinline__ bool cr_solve(const Team<P> &tm, TA *wa, int n, bool two) {
  return cr_solve_map<TA, P>(tm, wa, n, n, IdentityRows{}, two);
}

// The hybrid partition / cyclic-reduction schedule of the block tri-diagonal
// system (a work-efficient relative of OEE; Section IV discusses reductions of
// this system). The n rows are cut into m = min(P, n / 2) contiguous segments,
// one per lane; segment l = [s_l, e_l) keeps its first and last rows and its
// lane eliminates the interior rows s_l + 1 .. e_l - 2 top down by block
// Gaussian elimination: row k, coupled to the segment's first row a by F and to
// row k + 1 by U_k, is factored (D_k = L L^T) and folded into both, D_a -= G1^T
// G1, R_a -= G1^T g, D_{k+1} -= G2^T G2, R_{k+1} -= G2^T g, and the coupling of a
// moves on to k + 1, F <- -G1^T G2 (G1 = L^{-1} F^T, G2 = L^{-1} U_k, g = L^{-1}
// R_k): Schur complements of the SPD matrix, so every pivot stays SPD. The
// kept rows form a block tri-diagonal system of 2m rows (a_l -- e_l - 1 coupled
// by the final F, e_l - 1 -- a_{l+1} by the original U) that block cyclic
// reduction solves across the lanes; each lane then back-substitutes its
// interior bottom up, L^T x_k = g - G1 x_a - G2 x_{k+1}. Interior rows keep L,
// 1 / diag L, g, G1 and G2 in their own fields (A_L, A_LI, A_GR, A_LO, A_G).
template <class TA, int P>
__device__ __forceinline__ bool hybrid_solve(const Team<P> &tm, TA *wa, int n, bool two) {
  bool bad = false;
  if (n <= 2) return cr_solve<TA, P>(tm, wa, n, two);
  const int m = min(P, n / 2);
  auto seg_start = [&](int l) { return static_cast<int>((static_cast<int64_t>(l) * n) / m); };
  if (tm.r < m) {
    const int a = seg_start(tm.r), e = seg_start(tm.r + 1);
    const RowP<TA> ra = rowp(wa, n, a);
    TA F[25];  // the coupling block (a, k) of the current frontier row k
#pragma unroll
    for (int k = 0; k < 25; ++k) F[k] = ra[A_U0 + k];
    for (int k = a + 1; k <= e - 2; ++k) {
      const RowP<TA> rk = rowp(wa, n, k);
      TA Dm[15], L[15], inv[5];
#pragma unroll
      for (int q = 0; q < 15; ++q) Dm[q] = rk[A_D0 + q];
      bad |= !chol5(Dm, L, inv);
#pragma unroll
      for (int q = 0; q < 15; ++q) rk[A_L + q] = L[q];
#pragma unroll
      for (int q = 0; q < 5; ++q) rk[A_LI + q] = inv[q];
      // G1 = L^{-1} F^T (column c of F^T is row c of F), G2 = L^{-1} U_k
      TA G1[5][5], G2[5][5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        TA col[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) col[q] = F[5 * c + q];
        fwd5(L, inv, col);
#pragma unroll
        for (int q = 0; q < 5; ++q) G1[q][c] = col[q];
#pragma unroll
        for (int q = 0; q < 5; ++q) col[q] = rk[A_U0 + 5 * q + c];
        fwd5(L, inv, col);
#pragma unroll
        for (int q = 0; q < 5; ++q) G2[q][c] = col[q];
      }
#pragma unroll
      for (int q = 0; q < 5; ++q)
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          rk[A_LO + 5 * q + c] = G1[q][c];
          rk[A_G + 5 * q + c] = G2[q][c];
        }
      const RowP<TA> rn = rowp(wa, n, k + 1);
      for (int h = 0; h < (two ? 2 : 1); ++h) {
        const int fR = h ? A_R20 : A_R0, fG = h ? A_GR2 : A_GR;
        TA g[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) g[q] = rk[fR + q];
        fwd5(L, inv, g);
#pragma unroll
        for (int q = 0; q < 5; ++q) rk[fG + q] = g[q];
#pragma unroll
        for (int r = 0; r < 5; ++r) {
          TA sa = ra[fR + r], sn = rn[fR + r];
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            sa -= G1[q][r] * g[q];
            sn -= G2[q][r] * g[q];
          }
          ra[fR + r] = sa;
          rn[fR + r] = sn;
        }
      }
      // D_a -= G1^T G1, D_{k+1} -= G2^T G2 (lower triangles), F <- -G1^T G2
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int c = 0; c <= r; ++c) {
          TA sa = ra[A_D0 + l5(r, c)], sn = rn[A_D0 + l5(r, c)];
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            sa -= G1[q][r] * G1[q][c];
            sn -= G2[q][r] * G2[q][c];
          }
          ra[A_D0 + l5(r, c)] = sa;
          rn[A_D0 + l5(r, c)] = sn;
        }
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          TA t = TA(0);
#pragma unroll
          for (int q = 0; q < 5; ++q) t -= G1[q][r] * G2[q][c];
          F[5 * r + c] = t;
        }
    }
    // the segment's first row now couples to its last row by F
#pragma unroll
    for (int k = 0; k < 25; ++k) ra[A_U0 + k] = F[k];
  }
  tm.sync();
  // the reduced system: reduced row 2l is s_l, 2l + 1 is e_l - 1
  auto row_of = [&](int r) { return (r & 1) ? seg_start((r >> 1) + 1) - 1 : seg_start(r >> 1); };
  bad |= cr_solve_map<TA, P>(tm, wa, n, 2 * m, row_of, two);
  if (tm.r < m) {
    const int a = seg_start(tm.r), e = seg_start(tm.r + 1);
    const RowP<TA> ra = rowp(wa, n, a);
    for (int h = 0; h < (two ? 2 : 1); ++h) {
      const int fX = h ? A_FC2 : A_FC, fG = h ? A_GR2 : A_GR;
      TA xa[5], xn[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        xa[q] = ra[fX + q];
        xn[q] = rowp(wa, n, e - 1)[fX + q];
      }
      for (int k = e - 2; k >= a + 1; --k) {
        const RowP<TA> rk = rowp(wa, n, k);
        TA L[15], inv[5], x[5];
#pragma unroll
        for (int q = 0; q < 15; ++q) L[q] = rk[A_L + q];
#pragma unroll
        for (int q = 0; q < 5; ++q) inv[q] = rk[A_LI + q];
#pragma unroll
        for (int r = 0; r < 5; ++r) {
          TA t = rk[fG + r];
#pragma unroll
          for (int q = 0; q < 5; ++q) t -= rk[A_LO + 5 * r + q] * xa[q] + rk[A_G + 5 * r + q] * xn[q];
          x[r] = t;
        }
        bwd5(L, inv, x);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          rk[fX + q] = x[q];
          xn[q] = x[q];
        }
      }
    }
  }
  tm.sync();
  return bad;
}

// Algorithm 1 for one problem; BTD selects SolvBTDSys: 0 = odd-even
// elimination (Algorithm 2), 1 = block cyclic reduction, 2 = the hybrid
// partition / cyclic-reduction schedule. In MODE_FD2 a second
// right-hand side (tau_delta := in4) rides along: the blocks D, U and their
// elimination are shared, only R, F_c and CalcAcc are done twice.
// WP: a general projection W_i = Wc_i Q_i (A.wmode; odd-even elimination, one
// right-hand side).
template <class T, class TA, int P, int BTD, bool TWO, bool WP = false>
__device__ __forceinline__ void cfa_body(const KArgs &A, const Range &rg) {
  static_assert(!WP || (BTD == 0 && !TWO), "a general projection runs with OEE, one right-hand side");
  Team<P> tm;
  Prob<T> pb;
  if (!load_problem<T, P>(A, rg, tm, pb, NT)) return;
  const int n = pb.n;
  TA *wa = static_cast<TA *>(A.ws_a) + A.state_off[pb.p] * NA_CFA;
  bool bad = false;
  constexpr bool two = TWO;  // A.mode == MODE_FD2
  const T *td2 = two ? static_cast<const T *>(A.in4) + A.state_off[pb.p] : nullptr;
  T *out2 = two ? static_cast<T *>(A.out4) + A.state_off[pb.p] : nullptr;

  // Single precision only: refinement. Algorithm 2 finishes every row with a
  // full Schur complement of A, which in FP32 cancels down to about cond(A)
  // eps32 relative accuracy; a second pass solves M d = tau - ID(q, qd, qdd)
  // with the same algorithm (a Newton step on the inverse dynamics, Eq. 2, whose
  // residual is exact to the inverse dynamics' own rounding) and adds d. Each
  // step shrinks the error by about the solve's own relative accuracy, so a
  // problem whose first correction exceeds 1% of its solution (its first solve
  // was that far off) takes a third pass.
  constexpr bool refine = std::is_same<T, float>::value && std::is_same<TA, float>::value && !TWO;
  const int passes = (refine && A.mode == MODE_FD) ? 3 : 1;
  T corr = T(0), qmax = T(0);  // this lane's largest correction and |qdd| of the last pass
  for (int pass = 0; pass < passes; ++pass) {
  if (pass == 2) {
    T qm = qmax;
    if constexpr (P > 1 && P <= 32) {  // the team's largest |qdd| (lanes of larger teams use their own)
#pragma unroll
      for (int o = 1; o < P; o *= 2) qm = fmax(qm, __shfl_xor_sync(tm.mask, qm, o, P));
    }
    if (!tm.any(corr > T(1e-2) * qm)) break;
  }
  corr = T(0);
  qmax = T(0);
  // bias torque and tau_delta (Algorithm 1: CalcInvDyn, CalcDiffTorques); on the
  // refinement pass the residual tau - ID(q, qd, qdd) of the first pass's qdd
  id_team<T, P>(tm, pb, A.grav, pass ? MODE_RES : A.mode);
  tm.sync();

  // CalcA, R = -B tau_delta and CalcAcc run in the accumulation type TA on the
  // model record of that type. Under mixed precision (float T, double TA) that is
  // the FP64 record: the blocks of A, B and C are then formed in FP64 from one set
  // of joint transforms, so M^{-1} = C - B^T A^{-1} B holds to FP64 rounding and
  // only the FP32 inverse dynamics (tau_delta) and joint transforms perturb the
  // problem. The products z = J^{-1} (...) live in the T workspace when T = TA and
  // in the row's G slot (free before the elimination and after it) otherwise.
  constexpr bool same = std::is_same<T, TA>::value;
  const TA *recA;
  if constexpr (same) recA = pb.rec;
  else recA = static_cast<const TA *>(A.model64) + pb.m0 * REC;
  auto zst = [&](int i) -> RowP<TA> {
    if constexpr (same) return RowP<TA>{pb.wt + static_cast<int64_t>(i) * NT + W_Z, 1};
    else return rowp(wa, n, i) + A_G;
  };

  // CalcA: D_i, U_i; R = -B tau_delta applied as -W^T (I-Gamma) J^{-1} (I-Gamma)^T S tau_delta.
  // From here on lanes take rows round robin (neighbouring rows on neighbouring lanes).
  for (int i = tm.r; i < n; i += P) {
    const T *w = pb.wt + static_cast<int64_t>(i) * NT;
    const TA *rec = recA + static_cast<int64_t>(i) * REC;
    const RowP<TA> row = rowp(wa, n, i);
    SE3<TA> g;
    ld_se3(w + W_G, g);
    calc_dblock<TA, TA>(i > 0 ? &g : nullptr, i > 0 ? rec - REC + REC_JI : nullptr,
                        rec + REC_JI, row + A_D0);
    TA yv[6] = {TA(w[W_TD]), TA(0), TA(0), TA(0), TA(0), TA(0)};
    TA y2[3] = {two ? TA(td2[i]) : TA(0), TA(0), TA(0)};
    if (i + 1 < n) {
      SE3<TA> gn;
      ld_se3(w + NT + W_G, gn);
      calc_ublock<TA, TA>(gn, rec + REC_JI, row + A_U0);
      const TA tn = TA(w[NT + W_TD]);
      // Ad_{g_{i+1}^{-1}}^T (e_1 t) = (t R e_1; 0)
      yv[0] -= gn.R[0] * tn;
      yv[1] -= gn.R[3] * tn;
      yv[2] -= gn.R[6] * tn;
      if (two) {
        const TA t2 = TA(td2[i + 1]);
        y2[0] -= gn.R[0] * t2;
        y2[1] -= gn.R[3] * t2;
        y2[2] -= gn.R[6] * t2;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 25; ++k) row[A_U0 + k] = TA(0);
    }
    // z = J^{-1} y with y = (y_0, y_1, y_2, 0, 0, 0): columns 0..2 only
    const TA *Ki = rec + REC_JI;
    const RowP<TA> zs = zst(i);
#pragma unroll
    for (int k = 0; k < 6; ++k)
      zs[k] = Ki[s6(k, 0)] * yv[0] + Ki[s6(k, 1)] * yv[1] + Ki[s6(k, 2)] * yv[2];
    if (two) {
#pragma unroll
      for (int k = 0; k < 6; ++k)
        row[A_Z2 + k] = Ki[s6(k, 0)] * y2[0] + Ki[s6(k, 1)] * y2[1] + Ki[s6(k, 2)] * y2[2];
    }
  }
  tm.sync();
  for (int i = tm.r; i < n; i += P) {
    // R_i = -(z_i - Ad_{g_i^{-1}} z_{i-1}), components 1..5
    const T *w = pb.wt + static_cast<int64_t>(i) * NT;
    TA z[6], t[6] = {TA(0), TA(0), TA(0), TA(0), TA(0), TA(0)};
    const RowP<TA> zs = zst(i);
#pragma unroll
    for (int k = 0; k < 6; ++k) z[k] = zs[k];
    SE3<TA> g;
    if (i > 0) {
      ld_se3(w + W_G, g);
      const RowP<TA> zq = zst(i - 1);
      TA zp[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) zp[k] = zq[k];
      adinv(g, zp, t);
    }
    const RowP<TA> row = rowp(wa, n, i);
#pragma unroll
    for (int k = 0; k < 5; ++k) row[A_R0 + k] = t[k + 1] - z[k + 1];
    if (two) {
      TA z2[6], t2[6] = {TA(0), TA(0), TA(0), TA(0), TA(0), TA(0)};
#pragma unroll
      for (int k = 0; k < 6; ++k) z2[k] = row[A_Z2 + k];
      if (i > 0) {
        const RowP<TA> rp = rowp(wa, n, i - 1);
        TA zp[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) zp[k] = rp[A_Z2 + k];
        adinv(g, zp, t2);
      }
#pragma unroll
      for (int k = 0; k < 5; ++k) row[A_R20 + k] = t2[k + 1] - z2[k + 1];
    }
  }
  tm.sync();

  // A general projection (the paper's closing question: other choices of W in
  // Eq. cfa-eq1). Any W_i with W_i^T S_i = 0 and full rank is Wc_i Q_i with Q_i
  // invertible, Wc_i the canonical complement e_2 .. e_6 the blocks above use. With
  // Q = diag(Q_i) the system of Eq. cfa-eq2 becomes A' = Q^T A Q, R' = Q^T R and
  // its solution F_c' = Q^{-1} F_c, so qdd is unchanged and only the
  // elimination's numbers differ: D_i' = Q_i^T D_i Q_i, U_i' = Q_i^T U_i Q_{i+1},
  // R_i' = Q_i^T R_i, and F_c,i = Q_i F_c,i' after the solve. Block Jacobi takes
  // Q_i = L_i^{-T} with D_i = L_i L_i^T: every D_i' is the identity and the rest
  // are triangular solves, U_i' = L_i^{-1} U_i L_{i+1}^{-T}, R_i' = L_i^{-1} R_i,
  // F_c,i = L_i^{-T} F_c,i'. The row's A_Q slot holds Q_i, or L_i and 1 / L_jj.
  if constexpr (WP) {
    const bool bj = A.wmode == WPROJ_BLOCK_JACOBI;
    for (int i = tm.r; i < n; i += P) {
      const RowP<TA> row = rowp(wa, n, i);
      if (bj) {
        TA Dm[15], L[15], inv[5];
#pragma unroll
        for (int k = 0; k < 15; ++k) Dm[k] = row[A_D0 + k];
        bad |= !chol5(Dm, L, inv);
#pragma unroll
        for (int k = 0; k < 15; ++k) row[A_Q + k] = L[k];
#pragma unroll
        for (int k = 0; k < 5; ++k) row[A_Q + 15 + k] = inv[k];
      } else {
        const double *src = A.wq + (pb.m0 + i) * 25;
#pragma unroll
        for (int k = 0; k < 25; ++k) row[A_Q + k] = TA(src[k]);
      }
    }
    tm.sync();
    for (int i = tm.r; i < n; i += P) {
      const RowP<TA> row = rowp(wa, n, i);
      TA X[25];
      if (bj) {
        TA L[15], inv[5];
#pragma unroll
        for (int k = 0; k < 15; ++k) L[k] = row[A_Q + k];
#pragma unroll
        for (int k = 0; k < 5; ++k) inv[k] = row[A_Q + 15 + k];
#pragma unroll
        for (int r = 0; r < 5; ++r)
#pragma unroll
          for (int c = 0; c <= r; ++c) row[A_D0 + l5(r, c)] = r == c ? TA(1) : TA(0);
        if (i + 1 < n) {
#pragma unroll
          for (int c = 0; c < 5; ++c) {  // X = L_i^{-1} U_i, column by column
            TA col[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) col[k] = row[A_U0 + 5 * k + c];
            fwd5(L, inv, col);
#pragma unroll
            for (int k = 0; k < 5; ++k) X[5 * k + c] = col[k];
          }
          const RowP<TA> nx = rowp(wa, n, i + 1) + A_Q;
#pragma unroll
          for (int k = 0; k < 15; ++k) L[k] = nx[k];
#pragma unroll
          for (int k = 0; k < 5; ++k) inv[k] = nx[15 + k];
#pragma unroll
          for (int r = 0; r < 5; ++r) {  // row r of X L_{i+1}^{-T} = L_{i+1}^{-1} X_r^T
            fwd5(L, inv, X + 5 * r);
#pragma unroll
            for (int c = 0; c < 5; ++c) row[A_U0 + 5 * r + c] = X[5 * r + c];
          }
#pragma unroll
          for (int k = 0; k < 15; ++k) L[k] = row[A_Q + k];
#pragma unroll
          for (int k = 0; k < 5; ++k) inv[k] = row[A_Q + 15 + k];
        }
        TA rr[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) rr[k] = row[A_R0 + k];
        fwd5(L, inv, rr);
#pragma unroll
        for (int k = 0; k < 5; ++k) row[A_R0 + k] = rr[k];
      } else {
        TA Qm[25];
#pragma unroll
        for (int k = 0; k < 25; ++k) Qm[k] = row[A_Q + k];
        // X = D Q, D' = Q^T X (lower triangle)
#pragma unroll
        for (int r = 0; r < 5; ++r)
#pragma unroll
          for (int c = 0; c < 5; ++c) {
            TA t = TA(0);
#pragma unroll
            for (int k = 0; k < 5; ++k)
              t += row[A_D0 + (r >= k ? l5(r, k) : l5(k, r))] * Qm[5 * k + c];
            X[5 * r + c] = t;
          }
#pragma unroll
        for (int r = 0; r < 5; ++r)
#pragma unroll
          for (int c = 0; c <= r; ++c) {
            TA t = TA(0);
#pragma unroll
            for (int k = 0; k < 5; ++k) t += Qm[5 * k + r] * X[5 * k + c];
            row[A_D0 + l5(r, c)] = t;
          }
        if (i + 1 < n) {  // X = U Q_{i+1}, U' = Q_i^T X
          const RowP<TA> qn = rowp(wa, n, i + 1) + A_Q;
#pragma unroll
          for (int r = 0; r < 5; ++r)
#pragma unroll
            for (int c = 0; c < 5; ++c) {
              TA t = TA(0);
#pragma unroll
              for (int k = 0; k < 5; ++k) t += row[A_U0 + 5 * r + k] * qn[5 * k + c];
              X[5 * r + c] = t;
            }
#pragma unroll
          for (int r = 0; r < 5; ++r)
#pragma unroll
            for (int c = 0; c < 5; ++c) {
              TA t = TA(0);
#pragma unroll
              for (int k = 0; k < 5; ++k) t += Qm[5 * k + r] * X[5 * k + c];
              row[A_U0 + 5 * r + c] = t;
            }
        }
        TA rr[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) rr[k] = row[A_R0 + k];
#pragma unroll
        for (int r = 0; r < 5; ++r) {
          TA t = TA(0);
#pragma unroll
          for (int k = 0; k < 5; ++k) t += Qm[5 * k + r] * rr[k];
          row[A_R0 + r] = t;
        }
      }
    }
    tm.sync();
  }

  if constexpr (BTD == 1) {
    // SolvBTDSys by block cyclic reduction
    bad |= cr_solve<TA, P>(tm, wa, n, two);
  } else if constexpr (BTD == 2) {
    // SolvBTDSys by the hybrid partition / cyclic-reduction schedule
    bad |= hybrid_solve<TA, P>(tm, wa, n, two);
  } else {
  // SolvBTDSys: odd-even elimination, ceil(log2 n) levels (Algorithm 2)
  int levels = 0;
  while ((1 << levels) < n) ++levels;
  int src = 0;
  for (int j = 1; j <= levels; ++j) {
    const int d = 1 << (j - 1);
    const int sD = src ? A_D1 : A_D0, sU = src ? A_U1 : A_U0, sR = src ? A_R1 : A_R0;
    const int tD = src ? A_D0 : A_D1, tU = src ? A_U0 : A_U1, tR = src ? A_R0 : A_R1;
    const int sR2 = two ? (src ? A_R21 : A_R20) : -1, tR2 = src ? A_R20 : A_R21;
    for (int m = tm.r; m < n; m += P) bad |= !oee_factor<TA>(m, d, n, wa, sD, sU, sR, sR2);
    tm.sync();
    for (int i = tm.r; i < n; i += P) {
      TA Dn[15], Un[25], Rn[5], Rn2[5];
      oee_row<TA>(i, d, n, wa, sD, sU, sR, Dn, Un, Rn, sR2, Rn2);
      const RowP<TA> row = rowp(wa, n, i);
      for (int k = 0; k < 15; ++k) row[tD + k] = Dn[k];
      for (int k = 0; k < 25; ++k) row[tU + k] = Un[k];
      for (int k = 0; k < 5; ++k) row[tR + k] = Rn[k];
      if (two) {
        for (int k = 0; k < 5; ++k) row[tR2 + k] = Rn2[k];
      }
    }
    tm.sync();
    src ^= 1;
  }
  // F_c,i = D_i^{-1} R_i
  for (int i = tm.r; i < n; i += P) {
    const RowP<TA> row = rowp(wa, n, i);
    TA Dm[15], L[15], inv[5], r[5];
    for (int k = 0; k < 15; ++k) Dm[k] = row[(src ? A_D1 : A_D0) + k];
    for (int k = 0; k < 5; ++k) r[k] = row[(src ? A_R1 : A_R0) + k];
    bad |= !chol5(Dm, L, inv);
    fwd5(L, inv, r);
    bwd5(L, inv, r);
    for (int k = 0; k < 5; ++k) row[A_FC + k] = r[k];
    if (two) {
      for (int k = 0; k < 5; ++k) r[k] = row[(src ? A_R21 : A_R20) + k];
      fwd5(L, inv, r);
      bwd5(L, inv, r);
      for (int k = 0; k < 5; ++k) row[A_FC2 + k] = r[k];
    }
  }
  tm.sync();
  }
  if constexpr (WP) {  // F_c,i = Q_i F_c,i'
    for (int i = tm.r; i < n; i += P) {
      const RowP<TA> row = rowp(wa, n, i);
      TA y[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) y[k] = row[A_FC + k];
      if (A.wmode == WPROJ_BLOCK_JACOBI) {
        TA L[15], inv[5];
#pragma unroll
        for (int k = 0; k < 15; ++k) L[k] = row[A_Q + k];
#pragma unroll
        for (int k = 0; k < 5; ++k) inv[k] = row[A_Q + 15 + k];
        bwd5(L, inv, y);
#pragma unroll
        for (int k = 0; k < 5; ++k) row[A_FC + k] = y[k];
      } else {
#pragma unroll
        for (int r = 0; r < 5; ++r) {
          TA t = TA(0);
#pragma unroll
          for (int k = 0; k < 5; ++k) t += row[A_Q + 5 * r + k] * y[k];
          row[A_FC + r] = t;
        }
      }
    }
    tm.sync();
  }

  // CalcAcc: qdd = C tau_delta + B^T F_c = S^T (I-Gamma) J^{-1} (I-Gamma)^T F,
  // F_i = S tau_delta_i + W F_c,i (Eq. force-decomposition-global), in TA
  for (int i = tm.r; i < n; i += P) {
    const T *w = pb.wt + static_cast<int64_t>(i) * NT;
    const TA *rec = recA + static_cast<int64_t>(i) * REC;
    const RowP<TA> row = rowp(wa, n, i);
    TA yv[6] = {TA(w[W_TD]), row[A_FC], row[A_FC + 1], row[A_FC + 2], row[A_FC + 3],
                row[A_FC + 4]};
    SE3<TA> gn;
    if (i + 1 < n) {
      ld_se3(w + NT + W_G, gn);
      const RowP<TA> rn = rowp(wa, n, i + 1);
      TA Fn[6] = {TA(w[NT + W_TD]), rn[A_FC], rn[A_FC + 1], rn[A_FC + 2], rn[A_FC + 3],
                  rn[A_FC + 4]};
      TA t[6];
      adinvT(gn, Fn, t);
      for (int k = 0; k < 6; ++k) yv[k] -= t[k];
    }
    TA z[6];
    sym6_apply(rec + REC_JI, yv, z);
    const RowP<TA> zs = zst(i);
#pragma unroll
    for (int k = 0; k < 6; ++k) zs[k] = z[k];
    if (two) {
      TA y[6] = {TA(td2[i]), row[A_FC2], row[A_FC2 + 1], row[A_FC2 + 2], row[A_FC2 + 3],
                 row[A_FC2 + 4]};
      if (i + 1 < n) {
        const RowP<TA> rn = rowp(wa, n, i + 1);
        TA Fn[6] = {TA(td2[i + 1]), rn[A_FC2], rn[A_FC2 + 1], rn[A_FC2 + 2], rn[A_FC2 + 3],
                    rn[A_FC2 + 4]};
        TA t[6];
        adinvT(gn, Fn, t);
        for (int k = 0; k < 6; ++k) y[k] -= t[k];
      }
      sym6_apply(rec + REC_JI, y, z);
#pragma unroll
      for (int k = 0; k < 6; ++k) row[A_Z2 + k] = z[k];
    }
  }
  tm.sync();
  for (int i = tm.r; i < n; i += P) {
    const T *w = pb.wt + static_cast<int64_t>(i) * NT;
    const RowP<TA> zs = zst(i);
    TA qdd = zs[0];
    if (i > 0) {
      // (Ad_{g_i^{-1}} z_{i-1})_0 = (R^T omega)_0
      const RowP<TA> zp = zst(i - 1);
      qdd -= TA(w[W_G + 0]) * zp[0] + TA(w[W_G + 3]) * zp[1] + TA(w[W_G + 6]) * zp[2];
    }
    const T q2 = pass ? T(TA(pb.out[i]) + qdd) : T(qdd);
    pb.out[i] = q2;
    if (!finite_t(q2)) bad = true;
    if (passes > 1) {
      qmax = fmax(qmax, fabs(q2));
      if (pass) corr = fmax(corr, T(fabs(qdd)));
    }
    if (two) {
      const RowP<TA> row = rowp(wa, n, i);
      TA x = row[A_Z2];
      if (i > 0) {
        const RowP<TA> rp = rowp(wa, n, i - 1);
        x -= TA(w[W_G + 0]) * rp[A_Z2] + TA(w[W_G + 3]) * rp[A_Z2 + 1] + TA(w[W_G + 6]) * rp[A_Z2 + 2];
      }
      out2[i] = T(x);
      if (!finite_t(T(x))) bad = true;
    }
  }
  if (passes > 1) tm.sync();  // the refinement pass reads this pass's qdd
  }  // passes
  const bool any_bad = tm.any(bad);
  if (tm.r == 0) set_status(A.status, pb.p, any_bad ? 2 : 0);
}

template <class T, class TA, int P>
__global__ void __launch_bounds__(block_for<P>(), P <= 128 ? 3 : 1) cfa_kernel(KArgs A) {
  cfa_body<T, TA, P, 0, false>(A, Range{0, 0, A.n_problems});
}

template <class T, class TA, int P>
__global__ void __launch_bounds__(block_for<P>(), P <= 128 ? 3 : 1) cfa_w_kernel(KArgs A) {
  cfa_body<T, TA, P, 0, false, true>(A, Range{0, 0, A.n_problems});
}

template <class T, class TA, int P>
__global__ void __launch_bounds__(block_for<P>(), P <= 128 ? 3 : 1) cfa_cr_kernel(KArgs A) {
  cfa_body<T, TA, P, 1, false>(A, Range{0, 0, A.n_problems});
}

// MODE_FD2: forward dynamics and the adjoint's linear solve in one elimination
template <class T, class TA, int P>
__global__ void __launch_bounds__(block_for<P>(), P <= 128 ? 3 : 1) cfa2_kernel(KArgs A) {
  cfa_body<T, TA, P, 0, true>(A, Range{0, 0, A.n_problems});
}

template <class T, class TA, int P>
__global__ void __launch_bounds__(block_for<P>(), P <= 128 ? 3 : 1) cfa_cr2_kernel(KArgs A) {
  cfa_body<T, TA, P, 1, true>(A, Range{0, 0, A.n_problems});
}

// the hybrid partition / cyclic-reduction schedule (one or two right-hand sides)
template <class T, class TA, bool TWO, int P>
__global__ void __launch_bounds__(block_for<P>(), P <= 128 ? 3 : 1) cfa_hy_kernel(KArgs A) {
  cfa_body<T, TA, P, 2, TWO>(A, Range{0, 0, A.n_problems});
}

// ------------------------------------------------------------------ JSIIA

// Rows of one lane blocked together in the entries of M and in the Cholesky's
// trailing updates (a shared operand loaded once serves them all), for teams of
// up to four lanes, whose lanes hold many rows. Measured: 65 536 x 32 at team 2,
// one row 4.17 ms, two 3.86-3.90, four 3.95 (register pressure); 256 x 256 at
// team 128 two rows took 4.35 to 5.00 ms, so larger teams keep one.
template <int P>
__host__ __device__ constexpr int jsiia_rows_blocked() {
  return P <= 4 ? 2 : 1;
}

// Ad_{g^{-1}}^T P Ad_{g^{-1}} of a packed symmetric 6x6 P, added to Out.
// With X^T = [[I, p^], [0, I]] diag(R, R) (X^T (n; f) = (R n + p x R f; R f)) and
// P = [[A, B], [B^T, C]] in 3x3 blocks: rotate the blocks, A' = R A R^T,
// B' = R B R^T, C' = R C R^T, then
//   X^T P X = [[A' + B' p^T + p^ B''^T, B''], [B''^T, C']],  B'' = B' + p^ C',
// where (B' p^T)_rc = (p x b'_r)_c and (p^ B''^T)_rc = (p x b''_c)_r for the rows
// b'_r, b''_c: about 200 fused operations instead of twelve 6-vector transports.
//
// ZERO0: row and column 0 of P are zero and never read (the articulated inertia
// Pa = P - P S D^{-1} S^T P has Pa S = 0 with S = e_1), which drops the first
// column of A from R A, the first row of B from R B and the first column of R A
// from A' (36 fewer operations).
template <class TA, bool ZERO0 = false>
__device__ __forceinline__ void congruence_add(const SE3<TA> &g, const TA *P6, TA *Out) {
  const TA *R = g.R, *p = g.p;
  TA RA[3][3], RB[3][3], RC[3][3];  // R A, R B, R C
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if constexpr (ZERO0) {
        RA[r][c] = c == 0 ? TA(0) : R[3 * r + 1] * P6[s6(1, c)] + R[3 * r + 2] * P6[s6(2, c)];
        RB[r][c] = R[3 * r + 1] * P6[s6(1, 3 + c)] + R[3 * r + 2] * P6[s6(2, 3 + c)];
      } else {
        RA[r][c] = R[3 * r] * P6[s6(0, c)] + R[3 * r + 1] * P6[s6(1, c)] + R[3 * r + 2] * P6[s6(2, c)];
        RB[r][c] = R[3 * r] * P6[s6(0, 3 + c)] + R[3 * r + 1] * P6[s6(1, 3 + c)] +
                   R[3 * r + 2] * P6[s6(2, 3 + c)];
      }
      RC[r][c] = R[3 * r] * P6[s6(3, 3 + c)] + R[3 * r + 1] * P6[s6(4, 3 + c)] +
                 R[3 * r + 2] * P6[s6(5, 3 + c)];
    }
  TA Bp[3][3], Cp[3][3];  // B' = (R B) R^T, C' = (R C) R^T
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Bp[r][c] = RB[r][0] * R[3 * c] + RB[r][1] * R[3 * c + 1] + RB[r][2] * R[3 * c + 2];
      if (c >= r)
        Cp[r][c] = RC[r][0] * R[3 * c] + RC[r][1] * R[3 * c + 1] + RC[r][2] * R[3 * c + 2];
    }
#pragma unroll
  for (int r = 1; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < r; ++c) Cp[r][c] = Cp[c][r];
  // B'' = B' + p^ C': (p^ C')_rc = (p x C'_{:,c})_r
  TA Bq[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Bq[0][c] = (Bp[0][c] + p[1] * Cp[2][c]) - p[2] * Cp[1][c];
    Bq[1][c] = (Bp[1][c] + p[2] * Cp[0][c]) - p[0] * Cp[2][c];
    Bq[2][c] = (Bp[2][c] + p[0] * Cp[1][c]) - p[1] * Cp[0][c];
  }
  // top left: A' + (p x b'_r)_c + (p x b''_c)_r, upper triangle
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = r; c < 3; ++c) {
      const int c1 = (c + 1) % 3, c2 = (c + 2) % 3, r1 = (r + 1) % 3, r2 = (r + 2) % 3;
      // one chain of fused multiply-adds from Out's entry (no separate additions)
      TA t = Out[s6(r, c)];
      if constexpr (!ZERO0) t = t + RA[r][0] * R[3 * c];
      t = (t + RA[r][1] * R[3 * c + 1]) + RA[r][2] * R[3 * c + 2];
      t = (t + p[c1] * Bp[r][c2]) - p[c2] * Bp[r][c1];
      t = (t + p[r1] * Bq[c][r2]) - p[r2] * Bq[c][r1];
      Out[s6(r, c)] = t;
    }
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) Out[s6(r, 3 + c)] += Bq[r][c];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = r; c < 3; ++c) Out[s6(3 + r, 3 + c)] += Cp[r][c];
}


// The same congruence X^T P X + J on a pair of lanes (h = lane & 1), both holding
// the whole P: lane 0 rotates A and rows 0, 1 of B, lane 1 rotates C and rows 2, 1
// of B; they swap halves with shuffles, each forms its rows of B'' and three
// entries of the top-left block and of C' + J_C, and they swap those. Both lanes
// end with the whole result in Out: about 117 operations on each lane instead of
// 201 on one. J is the link's packed inertia (added at the end, since B'' and the
// top-left block use the bare rotated blocks). Lanes pick their operands with
// selects, never by a lane-dependent register index.
template <class TA, class T, int P>
__device__ __forceinline__ void congruence_pair(const Team<P> &tm, const SE3<TA> &g,
                                                const TA *P6, const T *J, TA *Out) {
  const bool h = (tm.r & 1) != 0;
  const TA *R = g.R, *p = g.p;
  auto xch = [&](TA v) { return __shfl_xor_sync(tm.mask, v, 1); };
  // S' = R S R^T of this lane's symmetric block (A or C), upper triangle
  TA S[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) S[k][c] = h ? P6[s6(3 + k, 3 + c)] : P6[s6(k, c)];
  TA RS[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      RS[r][c] = R[3 * r] * S[0][c] + R[3 * r + 1] * S[1][c] + R[3 * r + 2] * S[2][c];
  TA Sp[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = r; c < 3; ++c)
      Sp[r][c] = RS[r][0] * R[3 * c] + RS[r][1] * R[3 * c + 1] + RS[r][2] * R[3 * c + 2];
  // rows a = (h ? 2 : 0) and 1 of B' = R B R^T
  TA Ra[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) Ra[k] = h ? R[6 + k] : R[k];
  TA RBa[3], RBb[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    RBa[c] = Ra[0] * P6[s6(0, 3 + c)] + Ra[1] * P6[s6(1, 3 + c)] + Ra[2] * P6[s6(2, 3 + c)];
    RBb[c] = R[3] * P6[s6(0, 3 + c)] + R[4] * P6[s6(1, 3 + c)] + R[5] * P6[s6(2, 3 + c)];
  }
  TA Bpa[3], Bp1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Bpa[c] = RBa[0] * R[3 * c] + RBa[1] * R[3 * c + 1] + RBa[2] * R[3 * c + 2];
    Bp1[c] = RBb[0] * R[3 * c] + RBb[1] * R[3 * c + 1] + RBb[2] * R[3 * c + 2];
  }
  // swap: A', C' and B' whole on both lanes
  TA Ap[3][3], Cp[3][3], Bp[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = r; c < 3; ++c) {
      const TA o = xch(Sp[r][c]);
      Ap[r][c] = h ? o : Sp[r][c];
      Cp[r][c] = h ? Sp[r][c] : o;
      Ap[c][r] = Ap[r][c];
      Cp[c][r] = Cp[r][c];
    }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const TA o = xch(Bpa[c]);
    Bp[0][c] = h ? o : Bpa[c];
    Bp[1][c] = Bp1[c];
    Bp[2][c] = h ? Bpa[c] : o;
  }
  // rows a and 1 of B'' = B' + p^ C', (p^ C')_rc = p_{r+1} C'_{r+2,c} - p_{r+2} C'_{r+1,c}
  const TA pu = h ? p[0] : p[1], pv = h ? p[1] : p[2];
  TA Bqa[3], Bq1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const TA xa = h ? Cp[1][c] : Cp[2][c], xb = h ? Cp[0][c] : Cp[1][c];
    Bqa[c] = (Bpa[c] + pu * xa) - pv * xb;
    Bq1[c] = (Bp1[c] + p[2] * Cp[0][c]) - p[0] * Cp[2][c];
  }
  TA Bq[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const TA o = xch(Bqa[c]);
    Bq[0][c] = h ? o : Bqa[c];
    Bq[1][c] = Bq1[c];
    Bq[2][c] = h ? Bqa[c] : o;
  }
  // this lane's entries of the upper triangles of the top-left block and of C:
  // lane 0 (0,0) (0,1) (0,2), lane 1 (1,1) (1,2) (2,2);
  // top left (r, c) = A'_rc + (p x b'_r)_c + (p x b''_c)_r + J_rc
  TA tl[3], cn[3], bn[3], b1[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int ra = 0, ca = e, rb = e == 2 ? 2 : 1, cb = e == 0 ? 1 : 2;
    const TA a_rc = h ? Ap[rb][cb] : Ap[ra][ca];
    // (p x b'_r)_c = p_{c+1} B'_{r,c+2} - p_{c+2} B'_{r,c+1}
    const TA q1 = h ? p[(cb + 1) % 3] : p[(ca + 1) % 3], q2 = h ? p[(cb + 2) % 3] : p[(ca + 2) % 3];
    const TA y2 = h ? Bp[rb][(cb + 2) % 3] : Bp[ra][(ca + 2) % 3];
    const TA y1 = h ? Bp[rb][(cb + 1) % 3] : Bp[ra][(ca + 1) % 3];
    // (p x b''_c)_r = p_{r+1} B''_{c,r+2} - p_{r+2} B''_{c,r+1}
    const TA s1 = h ? p[(rb + 1) % 3] : p[(ra + 1) % 3], s2 = h ? p[(rb + 2) % 3] : p[(ra + 2) % 3];
    const TA z2 = h ? Bq[cb][(rb + 2) % 3] : Bq[ca][(ra + 2) % 3];
    const TA z1 = h ? Bq[cb][(rb + 1) % 3] : Bq[ca][(ra + 1) % 3];
    const int r = h ? rb : ra, c = h ? cb : ca;
    TA t = a_rc + TA(J[s6(r, c)]);
    t = (t + q1 * y2) - q2 * y1;
    t = (t + s1 * z2) - s2 * z1;
    tl[e] = t;
    cn[e] = (h ? Cp[rb][cb] : Cp[ra][ca]) + TA(J[s6(3 + r, 3 + c)]);
  }
  const int a = h ? 2 : 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    bn[c] = Bqa[c] + TA(J[s6(a, 3 + c)]);
    b1[c] = Bq1[c] + TA(J[s6(1, 3 + c)]);
  }
  // swap the entries and assemble the whole result on both lanes
  TA to[3], co[3], bo[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    to[e] = xch(tl[e]);
    co[e] = xch(cn[e]);
    bo[e] = xch(bn[e]);
  }
  Out[s6(0, 0)] = h ? to[0] : tl[0];
  Out[s6(0, 1)] = h ? to[1] : tl[1];
  Out[s6(0, 2)] = h ? to[2] : tl[2];
  Out[s6(1, 1)] = h ? tl[0] : to[0];
  Out[s6(1, 2)] = h ? tl[1] : to[1];
  Out[s6(2, 2)] = h ? tl[2] : to[2];
  Out[s6(3, 3)] = h ? co[0] : cn[0];
  Out[s6(3, 4)] = h ? co[1] : cn[1];
  Out[s6(3, 5)] = h ? co[2] : cn[2];
  Out[s6(4, 4)] = h ? cn[0] : co[0];
  Out[s6(4, 5)] = h ? cn[1] : co[1];
  Out[s6(5, 5)] = h ? cn[2] : co[2];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Out[s6(0, 3 + c)] = h ? bo[c] : bn[c];
    Out[s6(1, 3 + c)] = b1[c];
    Out[s6(2, 3 + c)] = h ? bn[c] : bo[c];
  }
}

// JSIIA (Section II-C): M by the unit-acceleration inverse dynamics of every
// column, its Cholesky factor, two triangular solves.
//
// Column k's inverse dynamics (qdd = e_k, qdot = 0, no gravity) has the
// accelerations x_i = X_{i<-k} e_1 (i >= k) and the force recursion
// F_i = X_{i+1}^T F_{i+1} + J_i x_i. Every column's force recursion composes the
// same operators, and composing them once gives the composite inertias
// I^c_{i-1} = J_{i-1} + X_i^T I^c_i X_i with F_i = I^c_i x_i, so
//   M[i][k] = e_1^T F_i = (X_{k+1}^T ... X_i^T h_i)[0],  h_i = I^c_i e_1:
// one SE(3) transport per entry of the lower triangle. The composite recursion
// runs on six lanes (row r of I^c on lane r, the congruence as two transports
// per lane through a shared-memory transpose) for teams of 8 and more, on a pair
// of lanes for teams of 2 and 4, on one lane alone.
template <class T, class TA, int P>
__device__ __forceinline__ void jsiia_body(const KArgs &A, const Range &rg) {
  constexpr int NXB = P >= 8 ? block_for<P>() / P : 1;
  __shared__ TA xbuf[NXB][2][36];
  Team<P> tm;
  Prob<T> pb;
  if (!load_problem<T, P>(A, rg, tm, pb, NT)) return;
  const int n = pb.n, a = pb.a, b = pb.b;
  const int64_t s0 = A.state_off[pb.p];
  TA *vec = static_cast<TA *>(A.ws_a) + s0 * NA_JSIIA + A.sq_off[pb.p] * NSQ_JSIIA;
  TA *H = vec + n;                                   // h_i = I^c_i e_1, [n][6]
  TA *vec2 = vec + 7 * static_cast<int64_t>(n);      // MODE_FD2: second right-hand side
  TA *Sb = vec + 8 * static_cast<int64_t>(n);        // teams of 1..4: s_i, [n][6]
  TA *const vec1 = vec;
  const bool two = A.mode == MODE_FD2;
  TA *M = vec + static_cast<int64_t>(n) * NA_JSIIA;  // n x n, column-major, lower triangle
  // entry (i, l) of M (and of L) at M[l n + i]: the lanes, on neighbouring rows,
  // touch neighbouring addresses
  auto Mat = [&](int i, int l) -> TA & { return M[static_cast<int64_t>(l) * n + i]; };
  bool bad = false;

  id_team<T, P>(tm, pb, A.grav, A.mode);
  for (int i = a; i < b; ++i) vec[i] = TA(pb.wt[static_cast<int64_t>(i) * NT + W_TD]);
  if (two) {
    const T *in4 = static_cast<const T *>(A.in4) + s0;
    for (int i = a; i < b; ++i) vec2[i] = TA(in4[i]);
  }

  // composite inertias, backward over the links; h_i = column 0 of I^c_i
  auto load_g = [&](int i, SE3<TA> &ga) {
    SE3<T> g;
    ld_se3(pb.wt + static_cast<int64_t>(i) * NT + W_G, g);
#pragma unroll
    for (int c = 0; c < 9; ++c) ga.R[c] = TA(g.R[c]);
#pragma unroll
    for (int c = 0; c < 3; ++c) ga.p[c] = TA(g.p[c]);
  };
  if constexpr (P >= 8) {
    tm.sync();  // the g_i of every link
    if (P <= 32 || tm.r < 32) {  // warp 0 of the team
      const unsigned wmask = P <= 32 ? tm.mask : 0xffffffffu;
      const int r = tm.r < 6 ? tm.r : 5;  // lanes 6.. shadow row 5 and write nothing
      TA(*xb)[36] = xbuf[(threadIdx.x % block_for<P>()) / P];
      TA prow[6];
      if (n > 0) {
        const T *J = pb.rec + static_cast<int64_t>(n - 1) * REC + REC_J;
#pragma unroll
        for (int c = 0; c < 6; ++c) prow[c] = TA(J[s6(r, c)]);
      }
      for (int i = n - 1; i >= 0; --i) {
        if (tm.r < 6) H[static_cast<int64_t>(i) * 6 + r] = prow[0];
        if (i == 0) break;
        SE3<TA> ga;
        load_g(i, ga);
        TA Jr[6], ncol[6], nrow[6], orow[6];
        const T *J = pb.rec + static_cast<int64_t>(i - 1) * REC + REC_J;
#pragma unroll
        for (int c = 0; c < 6; ++c) Jr[c] = TA(J[s6(r, c)]);
        adinvT(ga, prow, ncol);  // column r of N = X^T I^c
        TA *x = xb[i & 1];
        if (tm.r < 6) {
#pragma unroll
          for (int c = 0; c < 6; ++c) x[c * 6 + r] = ncol[c];
        }
        __syncwarp(wmask);
#pragma unroll
        for (int c = 0; c < 6; ++c) nrow[c] = x[r * 6 + c];
        adinvT(ga, nrow, orow);  // row r of N X = X^T I^c X
#pragma unroll
        for (int c = 0; c < 6; ++c) prow[c] = Jr[c] + orow[c];
      }
    }
  } else if constexpr (P >= 2) {
    // teams of 2 and 4: the congruence on a pair of lanes (lanes 2, 3 of a team of
    // 4 repeat lanes 0, 1 and write nothing)
    tm.sync();
    TA Pm[21];
    if (n > 0) {
      const T *J = pb.rec + static_cast<int64_t>(n - 1) * REC + REC_J;
#pragma unroll
      for (int k = 0; k < 21; ++k) Pm[k] = TA(J[k]);
    }
    // FP64: the forward kinematics g_0j of the base-frame entries below runs in the
    // same loop, link j = n-1-i beside the congruence of link i (two independent
    // dependency chains); the lane that owns link j parks g_0j in the link's
    // twist and force slots, which the inverse dynamics no longer needs
    constexpr bool fk = std::is_same<T, double>::value;
    SE3<TA> g0f;
    se3_identity(g0f);
    for (int i = n - 1; i >= 0; --i) {
      if constexpr (fk) {
        const int j = n - 1 - i;
        SE3<TA> gj, t;
        load_g(j, gj);
        se3_mul(g0f, gj, t);
        g0f = t;
        if ((j & (P - 1)) == tm.r) st_se3(pb.wt + static_cast<int64_t>(j) * NT + W_V, g0f);
      }
      if (tm.r == 0) {
#pragma unroll
        for (int c = 0; c < 6; ++c) H[static_cast<int64_t>(i) * 6 + c] = Pm[s6(0, c)];
      }
      if (i == 0) break;
      SE3<TA> ga;
      load_g(i, ga);
      TA Pn[21];
      congruence_pair<TA, T, P>(tm, ga, Pm, pb.rec + static_cast<int64_t>(i - 1) * REC + REC_J, Pn);
#pragma unroll
      for (int k = 0; k < 21; ++k) Pm[k] = Pn[k];
    }
  } else {
    if (tm.r == 0) {
      TA Pm[21];
      if (n > 0) {
        const T *J = pb.rec + static_cast<int64_t>(n - 1) * REC + REC_J;
        for (int k = 0; k < 21; ++k) Pm[k] = TA(J[k]);
      }
      for (int i = n - 1; i >= 0; --i) {
        for (int c = 0; c < 6; ++c) H[static_cast<int64_t>(i) * 6 + c] = Pm[s6(0, c)];
        if (i == 0) break;
        SE3<TA> ga;
        load_g(i, ga);
        TA Pn[21];
        const T *J = pb.rec + static_cast<int64_t>(i - 1) * REC + REC_J;
        for (int k = 0; k < 21; ++k) Pn[k] = TA(J[k]);
        congruence_add(ga, Pm, Pn);
        for (int k = 0; k < 21; ++k) Pm[k] = Pn[k];
      }
    }
  }
  tm.sync();

  // lower triangle, row by row: row i costs i transports (or dot products), so
  // lanes take rows in snake order (round t: t P + r, then t P + P - 1 - r) to
  // balance the work
  if constexpr (P <= 4 && std::is_same<T, double>::value) {
    // Teams of up to four lanes pair vectors in the base frame instead: with
    // s_k = Ad_{g_0k} e_1 (joint k's axis as a base-frame twist) and
    // F_i = Ad_{g_0i^{-1}}^T h_i (the composite force h_i in base coordinates),
    // M[i][k] = s_k . F_i, the same power pairing as in frame k: one 6-term dot
    // product per entry instead of one SE(3) transport. The forward kinematics
    // g_0i = g_0,i-1 g_{i-1,i} runs on every lane (here for P = 1; for teams of
    // 2 and 4 inside the composite-inertia loop above, each lane keeping the
    // g_0i of its own links i = r mod P); lane r forms s_i and F_i for its links
    // (F_i over h_i). The base-frame terms grow with the distance from the base
    // and cancel in the pairing, which costs digits in proportion: FP64 only
    // (with joint transforms rounded to FP32, the mixed mode's entries would
    // lose about two digits).
    SE3<TA> g0;
    se3_identity(g0);
    for (int i = (P == 1 ? 0 : tm.r); i < n; i += (P == 1 ? 1 : P)) {
      if constexpr (P == 1) {
        SE3<TA> gi, t;
        load_g(i, gi);
        se3_mul(g0, gi, t);
        g0 = t;
      } else {
        ld_se3(pb.wt + static_cast<int64_t>(i) * NT + W_V, g0);
      }
      {
        const TA ax = g0.R[0], ay = g0.R[3], az = g0.R[6];  // R_0i e_1
        TA *sv = Sb + static_cast<int64_t>(i) * 6;
        sv[0] = ax;
        sv[1] = ay;
        sv[2] = az;
        sv[3] = g0.p[1] * az - g0.p[2] * ay;  // p_0i x R_0i e_1
        sv[4] = g0.p[2] * ax - g0.p[0] * az;
        sv[5] = g0.p[0] * ay - g0.p[1] * ax;
        TA *hv = H + static_cast<int64_t>(i) * 6;
        TA h[6], f[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) h[c] = hv[c];
        Mat(i, i) = h[0];
        adinvT(g0, h, f);
#pragma unroll
        for (int c = 0; c < 6; ++c) hv[c] = f[c];
      }
    }
    tm.sync();
    // rows RB rounds at a time (in snake order, increasing): each s_k loaded once
    // serves every row below k
    constexpr int RB = jsiia_rows_blocked<P>();
    for (int t = 0; t * P < n; t += RB) {
      int iq[RB];
      TA f[RB][6];
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        const int tt = t + q;
        iq[q] = tt * P + ((tt & 1) ? (P - 1 - tm.r) : tm.r);
#pragma unroll
        for (int c = 0; c < 6; ++c) f[q][c] = iq[q] < n ? H[static_cast<int64_t>(iq[q]) * 6 + c] : TA(0);
      }
      const int last = min(iq[RB - 1], n);
      for (int k = 0; k < last; ++k) {
        const TA *sv = Sb + static_cast<int64_t>(k) * 6;
        const TA s0 = sv[0], s1 = sv[1], s2 = sv[2], s3 = sv[3], s4 = sv[4], s5 = sv[5];
#pragma unroll
        for (int q = 0; q < RB; ++q)
          if (k < iq[q] && iq[q] < n)
            Mat(iq[q], k) = (((((s0 * f[q][0] + s1 * f[q][1]) + s2 * f[q][2]) + s3 * f[q][3]) +
                              s4 * f[q][4]) + s5 * f[q][5]);
      }
    }
  } else {
    for (int t = 0; t * P < n; ++t) {
      const int i = t * P + ((t & 1) ? (P - 1 - tm.r) : tm.r);
      if (i >= n) continue;
      TA z[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) z[c] = H[static_cast<int64_t>(i) * 6 + c];
      Mat(i, i) = z[0];
      for (int j = i; j >= 1; --j) {
        SE3<TA> ga;
        load_g(j, ga);
        adinvT(ga, z, z);
        Mat(i, j - 1) = z[0];
      }
    }
  }
  tm.sync();

  // Cholesky M = L L^T by blocks of eight columns (right-looking, rows shared by
  // the team): every lane factors the 8x8 diagonal block, each lane forms the
  // panel of its rows below it, then applies the rank-8 update to its rows of
  // the trailing matrix (eight fused operations per load and store of M). Then
  // the two triangular solves, also by blocks of eight (the "inversion" of
  // Section II-C read as a factorisation). 1 / L_jj is kept in h_j[0]. Measured
  // against blocks of two and four: 65 536 x 32 at team 2 5.6 / 6.8 / 5.9 ms,
  // 256 x 256 at team 128 4.3 / 7.3 / 5.2 ms.
  constexpr int NB = 8;
  for (int j0 = 0; j0 < n; j0 += NB) {
    const int jb = min(NB, n - j0);
    TA Ld[NB][NB], rinv[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u)
#pragma unroll
      for (int v = 0; v < NB; ++v) Ld[u][v] = (u < jb && v <= u) ? Mat(j0 + u, j0 + v) : TA(0);
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      rinv[u] = TA(0);
      if (u < jb) {
        TA d = Ld[u][u];
#pragma unroll
        for (int w = 0; w < u; ++w) d -= Ld[u][w] * Ld[u][w];
        bad |= !pos_t(d);
        const TA r = rsqrt_t(d);  // inf or NaN for a non-positive pivot, flagged by bad
        Ld[u][u] = r;  // L_jj itself is never read: the panel and the solves take 1 / L_jj
        rinv[u] = r;
#pragma unroll
        for (int v = u + 1; v < NB; ++v) {
          TA x = Ld[v][u];
#pragma unroll
          for (int w = 0; w < u; ++w) x -= Ld[v][w] * Ld[u][w];
          Ld[v][u] = x * r;
        }
      }
    }
    // panel: L(i, j0+u) = (M(i, j0+u) - sum_{w<u} L(i, j0+w) L(j0+u, j0+w)) / L(j0+u, j0+u)
    for (int i = j0 + jb + tm.r; i < n; i += P) {  // below the block, jb == NB
      TA li[NB];
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        TA x = Mat(i, j0 + u);
#pragma unroll
        for (int w = 0; w < u; ++w) x -= li[w] * Ld[u][w];
        li[u] = x * rinv[u];
      }
#pragma unroll
      for (int u = 0; u < NB; ++u) Mat(i, j0 + u) = li[u];
    }
    tm.sync();
    if (tm.r == 0) {  // every lane has read the diagonal block by now
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        if (u < jb) {
#pragma unroll
          for (int v = 0; v <= u; ++v) Mat(j0 + u, j0 + v) = Ld[u][v];
          H[static_cast<int64_t>(j0 + u) * 6] = rinv[u];
        }
      }
    }
    // rank-NB update of the trailing rows: M(i, l) -= sum_u L(i, j0+u) L(l, j0+u),
    // RB of a lane's rows (i, i + P, ...) at a time: each row l of the panel,
    // loaded once, serves all of them (rows below l only)
    constexpr int RB = jsiia_rows_blocked<P>();
    for (int i = j0 + jb + tm.r; i < n; i += RB * P) {
      TA li[RB][NB];
#pragma unroll
      for (int q = 0; q < RB; ++q)
#pragma unroll
        for (int u = 0; u < NB; ++u) li[q][u] = (i + q * P < n) ? Mat(i + q * P, j0 + u) : TA(0);
      const int last = min(i + (RB - 1) * P, n - 1);
      for (int l = j0 + jb; l <= last; ++l) {
        TA pl[NB];
#pragma unroll
        for (int u = 0; u < NB; ++u) pl[u] = Mat(l, j0 + u);
#pragma unroll
        for (int q = 0; q < RB; ++q) {
          const int iq = i + q * P;
          if (iq < n && l <= iq) {
            TA x = Mat(iq, l);
#pragma unroll
            for (int u = 0; u < NB; ++u) x -= li[q][u] * pl[u];
            Mat(iq, l) = x;
          }
        }
      }
    }
    tm.sync();
  }
  for (int h = 0; h < (two ? 2 : 1); ++h) {
    TA *vec = h ? vec2 : vec1;
    for (int j0 = 0; j0 < n; j0 += NB) {  // L y = b
      const int jb = min(NB, n - j0);
      TA y[NB];
  #pragma unroll
      for (int u = 0; u < NB; ++u) {
        y[u] = TA(0);
        if (u < jb) {
          TA x = vec[j0 + u];
  #pragma unroll
          for (int w = 0; w < u; ++w) x -= Mat(j0 + u, j0 + w) * y[w];
          y[u] = x * H[static_cast<int64_t>(j0 + u) * 6];
        }
      }
      for (int i = j0 + jb + tm.r; i < n; i += P) {
        TA x = vec[i];
  #pragma unroll
        for (int u = 0; u < NB; ++u) x -= Mat(i, j0 + u) * y[u];
        vec[i] = x;
      }
      tm.sync();
      if (tm.r == 0) {  // after every lane has read this block's right-hand side
  #pragma unroll
        for (int u = 0; u < NB; ++u)
          if (u < jb) vec[j0 + u] = y[u];
      }
    }
    tm.sync();
    for (int j0 = ((n - 1) / NB) * NB; j0 >= 0; j0 -= NB) {  // L^T x = y
      const int jb = min(NB, n - j0);
      TA x[NB];
  #pragma unroll
      for (int u = NB - 1; u >= 0; --u) {
        x[u] = TA(0);
        if (u < jb) {
          TA t = vec[j0 + u];
  #pragma unroll
          for (int w = u + 1; w < NB; ++w)
            if (w < jb) t -= Mat(j0 + w, j0 + u) * x[w];
          x[u] = t * H[static_cast<int64_t>(j0 + u) * 6];
        }
      }
      for (int i = tm.r; i < j0; i += P) {
        TA t = vec[i];
  #pragma unroll
        for (int u = 0; u < NB; ++u)
          if (u < jb) t -= Mat(j0 + u, i) * x[u];
        vec[i] = t;
      }
      tm.sync();
      if (tm.r == 0) {
  #pragma unroll
        for (int u = 0; u < NB; ++u)
          if (u < jb) vec[j0 + u] = x[u];
      }
    }
    tm.sync();
  }
  for (int i = a; i < b; ++i) {
    const T v = T(vec[i]);
    pb.out[i] = v;
    if (!finite_t(v)) bad = true;
  }
  if (two) {
    T *out4 = static_cast<T *>(A.out4) + s0;
    for (int i = a; i < b; ++i) {
      const T v = T(vec2[i]);
      out4[i] = v;
      if (!finite_t(v)) bad = true;
    }
  }
  const bool any_bad = tm.any(bad);
  if (tm.r == 0) set_status(A.status, pb.p, any_bad ? 2 : 0);
}

template <class T, class TA, int P>
__global__ void __launch_bounds__(block_for<P>(), P <= 128 ? 4 : 1) jsiia_kernel(KArgs A) {
  jsiia_body<T, TA, P>(A, Range{0, 0, A.n_problems});
}

// ------------------------------------------------------------------- ABIA


// ABIA (Section II-C): tau_delta by inverse dynamics, the articulated-body
// inertia recursion P_{i-1} = J_{i-1} + X_i^T (P_i - P_i S D_i^{-1} S^T P_i) X_i
// (serial in i, Section III), the bias-force recursion (backward) and the
// acceleration recursion (forward) of M^{-1} = [I - S^T Y Pi]^T (S^T J^ S)^{-1}
// [I - S^T Y Pi]. One thread per problem. TWO (MODE_FD2): a second right-hand
// side in4 shares the articulated inertias; its bias force and acceleration pass
// give M^{-1} in4 in out4.
template <class T, class TA, bool TWO>
__device__ __forceinline__ void abia_body(const KArgs &A, const Range &rg) {
  Team<1> tm;
  Prob<T> pb;
  if (!load_problem<T, 1>(A, rg, tm, pb, NT)) return;
  const int n = pb.n;
  TA *wa = static_cast<TA *>(A.ws_a) + A.state_off[pb.p] * NA_ABIA;
  bool bad = false;
  // inverse dynamics up to f_i; its force pass runs inside the backward loop below,
  // beside the articulated-inertia step of the same link (two independent
  // recursions sharing g_i)
  const bool linear = A.mode == MODE_LINEAR;
  id_team<T, 1>(tm, pb, A.grav, A.mode, true);
  const T *td2 = TWO ? static_cast<const T *>(A.in4) + A.state_off[pb.p] : nullptr;
  T *out2 = TWO ? static_cast<T *>(A.out4) + A.state_off[pb.p] : nullptr;
  TA pbias2[6] = {TA(0), TA(0), TA(0), TA(0), TA(0), TA(0)};

  TA Pm[21], pbias[6];
  T Fy[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};  // force recursion F_{i+1} transported
  if (n > 0) {
    const T *J = pb.rec + static_cast<int64_t>(n - 1) * REC + REC_J;
    for (int k = 0; k < 21; ++k) Pm[k] = TA(J[k]);
  }
  for (int k = 0; k < 6; ++k) pbias[k] = TA(0);
  for (int i = n - 1; i >= 0; --i) {
    T *w = pb.wt + static_cast<int64_t>(i) * NT;
    SE3<T> g;
    ld_se3(w + W_G, g);
    // tau_delta_i: the force pass F_i = X_{i+1}^T F_{i+1} + f_i, tau_i = F_i[0]
    T tdi;
    if (linear) {
      tdi = w[W_TD];
    } else {
      for (int k = 0; k < 6; ++k) Fy[k] += w[W_F + k];
      tdi = pb.in3[i] - Fy[0];
      adinvT(g, Fy, Fy);
    }
    TA *ra = wa + static_cast<int64_t>(i) * NA_ABIA;
    TA h[6];
    for (int k = 0; k < 6; ++k) h[k] = Pm[s6(0, k)];
    const TA D = h[0];
    const TA u = TA(tdi) - pbias[0];
    bad |= !pos_t(D);
    const TA Dinv = rcp_t(D);
    for (int k = 0; k < 6; ++k) ra[A_H + k] = h[k];
    ra[A_DD] = Dinv;
    ra[A_UU] = u * Dinv;
    TA u2 = TA(0);
    if constexpr (TWO) {
      u2 = TA(td2[i]) - pbias2[0];
      ra[A_UU2] = u2 * Dinv;
    }
    if (i == 0) break;
    // Pa = P - h h^T / D (row and column 0 vanish: Pa e_1 = 0), pa = p + h u / D
    TA Pa[21], pa[6], hs[6];
    for (int k = 0; k < 6; ++k) hs[k] = h[k] * Dinv;
    for (int r = 1; r < 6; ++r)
      for (int c = r; c < 6; ++c) Pa[s6(r, c)] = Pm[s6(r, c)] - h[r] * hs[c];
    for (int k = 0; k < 6; ++k) pa[k] = pbias[k] + hs[k] * u;
    TA pa2[6];
    if constexpr (TWO) {
      for (int k = 0; k < 6; ++k) pa2[k] = pbias2[k] + hs[k] * u2;
    }
    SE3<TA> ga;
    for (int c = 0; c < 9; ++c) ga.R[c] = TA(g.R[c]);
    for (int c = 0; c < 3; ++c) ga.p[c] = TA(g.p[c]);
    const T *J = pb.rec + static_cast<int64_t>(i - 1) * REC + REC_J;
    for (int k = 0; k < 21; ++k) Pm[k] = TA(J[k]);
    congruence_add<TA, true>(ga, Pa, Pm);
    adinvT(ga, pa, pbias);
    if constexpr (TWO) adinvT(ga, pa2, pbias2);
  }
  // forward: a' = X_i a_{i-1}, qdd_i = (u_i - h_i . a') / D_i, a_i = a' + e_1 qdd_i
  TA acc[6] = {TA(0), TA(0), TA(0), TA(0), TA(0), TA(0)};
  TA acc2[6] = {TA(0), TA(0), TA(0), TA(0), TA(0), TA(0)};
  for (int i = 0; i < n; ++i) {
    const TA *ra = wa + static_cast<int64_t>(i) * NA_ABIA;
    SE3<T> g;
    ld_se3(pb.wt + static_cast<int64_t>(i) * NT + W_G, g);
    SE3<TA> ga;
    for (int c = 0; c < 9; ++c) ga.R[c] = TA(g.R[c]);
    for (int c = 0; c < 3; ++c) ga.p[c] = TA(g.p[c]);
    adinv(ga, acc, acc);
    TA s = TA(0);
    for (int k = 0; k < 6; ++k) s += ra[A_H + k] * acc[k];
    const TA qdd = ra[A_UU] - s * ra[A_DD];
    acc[0] += qdd;
    const T v = T(qdd);
    pb.out[i] = v;
    if (!finite_t(v)) bad = true;
    if constexpr (TWO) {
      adinv(ga, acc2, acc2);
      TA s2 = TA(0);
      for (int k = 0; k < 6; ++k) s2 += ra[A_H + k] * acc2[k];
      const TA x = ra[A_UU2] - s2 * ra[A_DD];
      acc2[0] += x;
      out2[i] = T(x);
      if (!finite_t(T(x))) bad = true;
    }
  }
  set_status(A.status, pb.p, bad ? 2 : 0);
}

template <class T, class TA, bool TWO>
__global__ void __launch_bounds__(128, TWO ? 3 : 4) abia_kernel(KArgs A) {
  abia_body<T, TA, TWO>(A, Range{0, 0, A.n_problems});
}


// ABIA with a team of P (8..32) lanes per problem. Inverse dynamics runs on
// the team (component lanes or segmented scans). The articulated-inertia
// recursion stays serial in i, but each step's rank-1 update and congruence
// P_{i-1} = J_{i-1} + X_i^T Pa_i X_i (X_i = Ad_{g_i^{-1}}) is spread over six
// lanes, lane r carrying row r of the symmetric P: lane r forms column r of
// N = X_i^T Pa_i, the team transposes N through shared memory, and lane r then
// forms row r of N X_i = X_i^T N^T. The bias force and the acceleration pass
// carry one component per lane, as in the component-lane inverse dynamics.
// Each step's operands are loaded one step ahead (the loop is latency-bound).
template <class T, class TA, int P, bool TWO>
__device__ __forceinline__ void abia_team_body(const KArgs &A, const Range &rg) {
  static_assert(P >= 8 && P <= 32, "six rows of P need a team of 8..32 lanes");
  __shared__ TA xbuf[128 / P][2][36];
  Team<P> tm;
  Prob<T> pb;
  if (!load_problem<T, P>(A, rg, tm, pb, NT)) return;
  const int n = pb.n;
  const int r = tm.r < 6 ? tm.r : 5;  // lanes 6.. shadow row 5 and write nothing
  const bool top = r < 3;
  const int k = top ? r : r - 3;
  const int ka = k == 2 ? 0 : k + 1, kb = k == 0 ? 2 : k - 1;  // k+1, k+2 mod 3
  TA(*xb)[36] = xbuf[(threadIdx.x & 127) / P];
  TA *wa = static_cast<TA *>(A.ws_a) + A.state_off[pb.p] * NA_ABIA;
  bool bad = false;
  id_team<T, P>(tm, pb, A.grav, A.mode);
  tm.sync();
  // TWO (MODE_FD2): a second right-hand side in4 rides along (its own bias force
  // and acceleration pass); M^{-1} in4 goes to out4
  const T *td2 = TWO ? static_cast<const T *>(A.in4) + A.state_off[pb.p] : nullptr;
  T *out2 = TWO ? static_cast<T *>(A.out4) + A.state_off[pb.p] : nullptr;

  if constexpr (P < 16) {
    // operands of step i: tau_delta_i, g_i, row r of J_{i-1}
    TA nt_td = TA(0), nt_td2 = TA(0), nt_J[6] = {TA(0), TA(0), TA(0), TA(0), TA(0), TA(0)};
    // g_i, and this lane's row k of R with p_{k+1}, p_{k+2} (zero on the linear
    // lanes, which take no cross product in X^T), read by lane-dependent offsets
    // from memory rather than by lane-dependent register indices
    SE3<T> nt_g;
    se3_identity(nt_g);
    TA nt_rk[3] = {TA(0), TA(0), TA(0)}, nt_pka = TA(0), nt_pkb = TA(0);
    auto fetch = [&](int i) {
      const T *w = pb.wt + static_cast<int64_t>(i) * NT;
      nt_td = TA(w[W_TD]);
      if (TWO) nt_td2 = TA(td2[i]);
      if (i > 0) {
        ld_se3(w + W_G, nt_g);
  #pragma unroll
        for (int c = 0; c < 3; ++c) nt_rk[c] = TA(w[W_G + 3 * k + c]);
        nt_pka = top ? TA(w[W_G + 9 + ka]) : TA(0);
        nt_pkb = top ? TA(w[W_G + 9 + kb]) : TA(0);
        const T *J = pb.rec + static_cast<int64_t>(i - 1) * REC + REC_J;
  #pragma unroll
        for (int c = 0; c < 6; ++c) nt_J[c] = TA(J[s6(r, c)]);
      }
    };
    TA prow[6], pbr = TA(0), pbr2 = TA(0);  // row r of P_i; component r of the bias forces
    if (n > 0) {
      const T *J = pb.rec + static_cast<int64_t>(n - 1) * REC + REC_J;
  #pragma unroll
      for (int c = 0; c < 6; ++c) prow[c] = TA(J[s6(r, c)]);
      fetch(n - 1);
    }
    for (int i = n - 1; i >= 0; --i) {
      const TA td = nt_td, tdb = nt_td2;
      const TA rk0 = nt_rk[0], rk1 = nt_rk[1], rk2 = nt_rk[2], pka = nt_pka, pkb = nt_pkb;
      SE3<TA> ga;
      TA Jr[6];
  #pragma unroll
      for (int c = 0; c < 9; ++c) ga.R[c] = TA(nt_g.R[c]);
  #pragma unroll
      for (int c = 0; c < 3; ++c) ga.p[c] = TA(nt_g.p[c]);
  #pragma unroll
      for (int c = 0; c < 6; ++c) Jr[c] = nt_J[c];
      if (i > 0) fetch(i - 1);
      TA *ra = wa + static_cast<int64_t>(i) * NA_ABIA;
      TA h[6];
  #pragma unroll
      for (int c = 0; c < 6; ++c) h[c] = __shfl_sync(tm.mask, prow[c], 0, P);
      const TA p0 = __shfl_sync(tm.mask, pbr, 0, P);
      const TA D = h[0];
      bad |= !pos_t(D);
      const TA Dinv = rcp_t(D);
      const TA uD = (td - p0) * Dinv;  // u_i / D_i
      TA uD2 = TA(0);
      if constexpr (TWO) uD2 = (tdb - __shfl_sync(tm.mask, pbr2, 0, P)) * Dinv;
      if (tm.r < 6) ra[A_H + tm.r] = prow[0];
      if (tm.r == 0) {
        ra[A_DD] = Dinv;
        ra[A_UU] = uD;
        if (TWO) ra[A_UU2] = uD2;
      }
      if (i == 0) break;
      // row r of Pa = P - h h^T / D; component r of pa = p + h u / D
      const TA tr = prow[0] * Dinv;
      TA par[6];
  #pragma unroll
      for (int c = 0; c < 6; ++c) par[c] = prow[c] - tr * h[c];
      const TA par_b = pbr + prow[0] * uD;
      TA ncol[6], nrow[6], orow[6];
      adinvT(ga, par, ncol);  // column r of N = X^T Pa
      TA *x = xb[i & 1];
      if (tm.r < 6) {
  #pragma unroll
        for (int c = 0; c < 6; ++c) x[c * 6 + r] = ncol[c];
      }
      // bias p_{i-1} = X^T pa, component r (the other lanes' components by shuffle)
      TA pa[6];
  #pragma unroll
      for (int c = 0; c < 6; ++c) pa[c] = __shfl_sync(tm.mask, par_b, c, P);
      const TA tb = rk0 * (top ? pa[0] : pa[3]) + rk1 * (top ? pa[1] : pa[4]) +
                    rk2 * (top ? pa[2] : pa[5]);
      const TA fa = __shfl_sync(tm.mask, tb, 3 + ka, P), fb = __shfl_sync(tm.mask, tb, 3 + kb, P);
      pbr = (tb + pka * fb) - pkb * fa;
      if constexpr (TWO) {
        const TA pb2 = pbr2 + prow[0] * uD2;
#pragma unroll
        for (int c = 0; c < 6; ++c) pa[c] = __shfl_sync(tm.mask, pb2, c, P);
        const TA t2 = rk0 * (top ? pa[0] : pa[3]) + rk1 * (top ? pa[1] : pa[4]) +
                      rk2 * (top ? pa[2] : pa[5]);
        const TA fa2 = __shfl_sync(tm.mask, t2, 3 + ka, P), fb2 = __shfl_sync(tm.mask, t2, 3 + kb, P);
        pbr2 = (t2 + pka * fb2) - pkb * fa2;
      }
      tm.sync();
  #pragma unroll
      for (int c = 0; c < 6; ++c) nrow[c] = x[r * 6 + c];
      adinvT(ga, nrow, orow);  // row r of N X = X^T Pa X
  #pragma unroll
      for (int c = 0; c < 6; ++c) prow[c] = Jr[c] + orow[c];
    }
  } else {
    // Twelve lanes carry P in half columns: lane L < 12 holds rows 3h..3h+2 of
    // column c = L / 2 (h = L % 2), so each transport X^T v splits between a lane
    // pair (the bottom half R f; the top half R n + p x R f with R f from the
    // partner): about 15 FP64 operations per lane instead of 24. Lanes 12 and 13
    // carry the bias force p as a seventh column: the same instructions form
    // pa = p + h u / D and X^T pa. Lanes 14.. shadow lane 13 and write nothing.
    const int L = tm.r < (TWO ? 16 : 14) ? tm.r : (TWO ? 15 : 13);
    const int cc = L >> 1, hh = L & 1, q0 = 3 * hh;
    const bool colP = cc < 6;
    const int cr = colP ? cc : 5;  // the column whose N row a bias lane reads (unused)
    auto xt_pair = [&](const SE3<TA> &g, const TA *x3, TA *o3) {
      TA v[3], w[3];
#pragma unroll
      for (int k = 0; k < 3; ++k)
        v[k] = g.R[3 * k] * x3[0] + g.R[3 * k + 1] * x3[1] + g.R[3 * k + 2] * x3[2];
#pragma unroll
      for (int k = 0; k < 3; ++k) w[k] = __shfl_xor_sync(tm.mask, v[k], 1, P);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int k1 = k == 2 ? 0 : k + 1, k2 = k == 0 ? 2 : k - 1;
        const TA t = (v[k] + g.p[k1] * w[k2]) - g.p[k2] * w[k1];  // R n + p x R f
        o3[k] = hh == 0 ? t : v[k];
      }
    };
    TA nt_td = TA(0), nt_td2 = TA(0), nt_J[3] = {TA(0), TA(0), TA(0)};
    SE3<T> nt_g;
    se3_identity(nt_g);
    auto fetch = [&](int i) {
      const T *w = pb.wt + static_cast<int64_t>(i) * NT;
      nt_td = TA(w[W_TD]);
      if (TWO) nt_td2 = TA(td2[i]);
      if (i > 0) {
        ld_se3(w + W_G, nt_g);
        const T *J = pb.rec + static_cast<int64_t>(i - 1) * REC + REC_J;
#pragma unroll
        for (int k = 0; k < 3; ++k) nt_J[k] = colP ? TA(J[s6(q0 + k, cr)]) : TA(0);
      }
    };
    TA pc[3] = {TA(0), TA(0), TA(0)};  // rows q0.. of column cc of P_i (bias lanes: p_i)
    if (n > 0) {
      const T *J = pb.rec + static_cast<int64_t>(n - 1) * REC + REC_J;
#pragma unroll
      for (int k = 0; k < 3; ++k) pc[k] = colP ? TA(J[s6(q0 + k, cr)]) : TA(0);
      fetch(n - 1);
    }
    for (int i = n - 1; i >= 0; --i) {
      const TA td = nt_td, tdb = nt_td2;
      SE3<TA> ga;
      TA Jr[3];
#pragma unroll
      for (int c = 0; c < 9; ++c) ga.R[c] = TA(nt_g.R[c]);
#pragma unroll
      for (int c = 0; c < 3; ++c) ga.p[c] = TA(nt_g.p[c]);
#pragma unroll
      for (int k = 0; k < 3; ++k) Jr[k] = nt_J[k];
      if (i > 0) fetch(i - 1);
      TA *ra = wa + static_cast<int64_t>(i) * NA_ABIA;
      // h = column 0 of P (lanes 0, 1); D = P_00; h_cc = P_{0,cc}; p_0 on lane 12
      const TA D = __shfl_sync(tm.mask, pc[0], 0, P);
      const TA p0 = __shfl_sync(tm.mask, pc[0], 12, P);
      const TA hc = __shfl_sync(tm.mask, pc[0], 2 * cr, P);
      TA hr[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) hr[k] = __shfl_sync(tm.mask, pc[k], hh, P);
      bad |= !pos_t(D);
      const TA Dinv = rcp_t(D);
      const TA uD = (td - p0) * Dinv;  // u_i / D_i
      TA uD2 = TA(0);  // the second right-hand side's bias force rides on lanes 14, 15
      if constexpr (TWO) uD2 = (tdb - __shfl_sync(tm.mask, pc[0], 14, P)) * Dinv;
      if (tm.r < 2) {
#pragma unroll
        for (int k = 0; k < 3; ++k) ra[A_H + q0 + k] = pc[k];
      }
      if (tm.r == 0) {
        ra[A_DD] = Dinv;
        ra[A_UU] = uD;
        if (TWO) ra[A_UU2] = uD2;
      }
      if (i == 0) break;
      // Pa = P - h h^T / D (column cc); pa = p + h u / D (bias lanes)
      const TA t = colP ? hc * Dinv : (cc == 6 ? -uD : -uD2);
      TA pa[3], o[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) pa[k] = pc[k] - t * hr[k];
      xt_pair(ga, pa, o);  // column cc of N = X^T Pa; bias lanes: p_{i-1} = X^T pa
      TA *x = xb[i & 1];
      if (tm.r < 12) {
#pragma unroll
        for (int k = 0; k < 3; ++k) x[(q0 + k) * 6 + cc] = o[k];
      }
      if (!colP) {
#pragma unroll
        for (int k = 0; k < 3; ++k) pc[k] = o[k];
      }
      tm.sync();
      TA nr[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) nr[k] = x[cr * 6 + q0 + k];  // row cc of N, half hh
      xt_pair(ga, nr, o);  // column cc of X^T N^T = X^T Pa X
      if (colP) {
#pragma unroll
        for (int k = 0; k < 3; ++k) pc[k] = Jr[k] + o[k];
      }
    }
  }
  tm.sync();

  // forward: a' = X_i a_{i-1}, qdd_i = u_i / D_i - (h_i . a') / D_i, a_i = a' + e_1 qdd_i;
  // lane r forms component r of a' (as in the component-lane inverse dynamics)
  TA nx_h[6], nx_dd = TA(0), nx_ud = TA(0), nx_ud2 = TA(0), nx_c[3], nx_p[3];
  auto fetch_f = [&](int i) {
    const TA *ra = wa + static_cast<int64_t>(i) * NA_ABIA;
    const T *w = pb.wt + static_cast<int64_t>(i) * NT;
#pragma unroll
    for (int c = 0; c < 6; ++c) nx_h[c] = ra[A_H + c];
    nx_dd = ra[A_DD];
    nx_ud = ra[A_UU];
    if (TWO) nx_ud2 = ra[A_UU2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      nx_c[c] = TA(w[W_G + 3 * c + k]);  // column k of R
      nx_p[c] = TA(w[W_G + 9 + c]);
    }
  };
  if (n > 0) fetch_f(0);
  TA acc[6] = {TA(0), TA(0), TA(0), TA(0), TA(0), TA(0)};
  TA acc2[6] = {TA(0), TA(0), TA(0), TA(0), TA(0), TA(0)};
  for (int i = 0; i < n; ++i) {
    TA hh[6], cc[3], pp[3];
#pragma unroll
    for (int c = 0; c < 6; ++c) hh[c] = nx_h[c];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cc[c] = nx_c[c];
      pp[c] = nx_p[c];
    }
    const TA dd = nx_dd, ud = nx_ud, ud2 = nx_ud2;
    if (i + 1 < n) fetch_f(i + 1);
    // (Ad_{g^-1} a)_k = R^T w (k < 3), R^T (v + w x p) (k >= 3)
    TA xv[3];
    if (top) {
      xv[0] = acc[0];
      xv[1] = acc[1];
      xv[2] = acc[2];
    } else {
      xv[0] = acc[3] + acc[1] * pp[2] - acc[2] * pp[1];
      xv[1] = acc[4] + acc[2] * pp[0] - acc[0] * pp[2];
      xv[2] = acc[5] + acc[0] * pp[1] - acc[1] * pp[0];
    }
    const TA y = cc[0] * xv[0] + cc[1] * xv[1] + cc[2] * xv[2];
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] = __shfl_sync(tm.mask, y, c, P);
    TA sh = TA(0);
#pragma unroll
    for (int c = 0; c < 6; ++c) sh += hh[c] * acc[c];
    const TA qdd = ud - sh * dd;
    acc[0] += qdd;
    const T v = T(qdd);
    if ((i & (P - 1)) == tm.r) pb.out[i] = v;
    if (!finite_t(v)) bad = true;
    if constexpr (TWO) {
      if (top) {
        xv[0] = acc2[0];
        xv[1] = acc2[1];
        xv[2] = acc2[2];
      } else {
        xv[0] = acc2[3] + acc2[1] * pp[2] - acc2[2] * pp[1];
        xv[1] = acc2[4] + acc2[2] * pp[0] - acc2[0] * pp[2];
        xv[2] = acc2[5] + acc2[0] * pp[1] - acc2[1] * pp[0];
      }
      const TA y2 = cc[0] * xv[0] + cc[1] * xv[1] + cc[2] * xv[2];
#pragma unroll
      for (int c = 0; c < 6; ++c) acc2[c] = __shfl_sync(tm.mask, y2, c, P);
      TA s2 = TA(0);
#pragma unroll
      for (int c = 0; c < 6; ++c) s2 += hh[c] * acc2[c];
      const TA x2 = ud2 - s2 * dd;
      acc2[0] += x2;
      if ((i & (P - 1)) == tm.r) out2[i] = T(x2);
      if (!finite_t(T(x2))) bad = true;
    }
  }
  if (tm.r == 0) set_status(A.status, pb.p, bad ? 2 : 0);
}

template <class T, class TA, int P, bool TWO>
__global__ void __launch_bounds__(128) abia_team_kernel(KArgs A) {
  abia_team_body<T, TA, P, TWO>(A, Range{0, 0, A.n_problems});
}

// ---------------------------------------------------------- length classes
//
// One launch over a batch whose problems fall into length classes: the grid is
// split into the classes' block ranges (ClassTable), and each block runs the
// body of its class's team size. The kernels instantiate every team size up to
// one 128-thread block, so a class of short chains can run one thread per chain
// while a class of long chains runs a warp or a block per chain in the same
// launch.

__device__ __forceinline__ int class_of_block(const ClassTable &ct) {
  int c = 0;
  while (c + 1 < ct.n && static_cast<int>(blockIdx.x) >= ct.blk[c + 1]) ++c;
  return c;
}

#define FDK_CLASS_TEAMS(CALL)                                                          \
  switch (ct.team[c]) {                                                                \
    CALL(1) CALL(2) CALL(4) CALL(8) CALL(16) CALL(32) CALL(64) CALL(128) default: break; \
  }

template <class T>
__global__ void __launch_bounds__(128) id_multi_kernel(KArgs A, ClassTable ct) {
  const int c = class_of_block(ct);
  const Range rg{ct.blk[c], ct.first[c], ct.first[c + 1]};
#define FDK_C(PP) \
  case PP: id_body<T, PP>(A, rg); break;
  FDK_CLASS_TEAMS(FDK_C)
#undef FDK_C
}

template <class T, class TA, int BTD, bool TWO>
__global__ void __launch_bounds__(128, 3) cfa_multi_kernel(KArgs A, ClassTable ct) {
  const int c = class_of_block(ct);
  const Range rg{ct.blk[c], ct.first[c], ct.first[c + 1]};
#define FDK_C(PP) \
  case PP: cfa_body<T, TA, PP, BTD, TWO>(A, rg); break;
  FDK_CLASS_TEAMS(FDK_C)
#undef FDK_C
}

template <class T, class TA>
__global__ void __launch_bounds__(128, 4) jsiia_multi_kernel(KArgs A, ClassTable ct) {
  const int c = class_of_block(ct);
  const Range rg{ct.blk[c], ct.first[c], ct.first[c + 1]};
#define FDK_C(PP) \
  case PP: jsiia_body<T, TA, PP>(A, rg); break;
  FDK_CLASS_TEAMS(FDK_C)
#undef FDK_C
}

// ABIA: team 1 (one thread per chain) or the six-row lane teams of 8, 16, 32
template <class T, class TA, bool TWO>
__global__ void __launch_bounds__(128, TWO ? 3 : 4) abia_multi_kernel(KArgs A, ClassTable ct) {
  const int c = class_of_block(ct);
  const Range rg{ct.blk[c], ct.first[c], ct.first[c + 1]};
  switch (ct.team[c]) {
    case 1: abia_body<T, TA, TWO>(A, rg); break;
    case 8: abia_team_body<T, TA, 8, TWO>(A, rg); break;
    case 16: abia_team_body<T, TA, 16, TWO>(A, rg); break;
    case 32: abia_team_body<T, TA, 32, TWO>(A, rg); break;
    default: break;
  }
}

}  // namespace fdk
