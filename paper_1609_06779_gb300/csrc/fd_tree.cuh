// Branched robots (kinematic trees): inverse dynamics, ABIA and JSIIA over a
// parent array, one thread per tree. The paper treats serial chains only
// (its building blocks are block bi- and tri-diagonal systems, Sections II-IV);
// on a tree the same recursions run over each link's parent instead of link
// i-1: the twist and acceleration recursions read the parent's values (Eq. 2a,
// 2b), and the force, articulated-inertia and composite-inertia recursions add
// each link's transported contribution into its parent's (Eq. 2c, Section II-C).
// Links are numbered so that a parent precedes its children, so one ascending
// and one descending sweep over the links visit every parent before (after) its
// children. CFA's A stops being block tri-diagonal on a tree, so OEE has no
// tree form here. Trees closed by revolute loop joints take JSIIA and then the
// constrained correction of tree_loop_kernel (below).
#pragma once

#include "fd_kernels.cuh"

namespace fdk {

// T workspace of a tree link (NT entries): g (12), V (6), F (6: f_i, then the
// subtree's force as children add into it), tau_delta (1), Vd (6).
constexpr int TW_G = 0;
constexpr int TW_V = 12;
constexpr int TW_F = 18;
constexpr int TW_TD = 24;
constexpr int TW_A = 25;
static_assert(TW_A + 6 <= NT, "tree link record");

// TA workspace of a tree link: P (21: the articulated inertia for ABIA, the
// composite inertia for JSIIA, children adding into it), the bias force (6),
// h = P S (6), 1 / D (1), u / D (1), the acceleration (6); JSIIA keeps its
// right-hand side in the 1 / D slot and M after the per-link records.
constexpr int TA_P = 0;
constexpr int TA_PB = 21;
constexpr int TA_H = 27;
constexpr int TA_DD = 33;
constexpr int TA_UU = 34;
constexpr int TA_AC = 35;
static_assert(TA_AC + 6 <= NA_TREE, "tree link record");

template <class T>
__device__ __forceinline__ T tree_force_step(const Prob<T> &pb, const int32_t *par, int i,
                                             const SE3<T> &g, bool fdm);

// Eq. 2a-2b forward over the parent array, f_i = J_i Vd_i - ad_{V_i}^T J_i V_i,
// then Eq. 2c-2d backward: F_i = f_i + sum over children c of Ad_{g_c^-1}^T F_c,
// tau_i = F_i[0]. Writes tau_delta (MODE_FD: tau - tau_bias; MODE_ID: tau) to
// TW_TD. With init_P, TA_P of every link starts as J_i and TA_PB as zero.
// Without force, the backward pass is left to the caller (tree_force_step inside
// its own backward loop).
template <class T, class TA>
__device__ __forceinline__ void tree_id(const KArgs &A, const Prob<T> &pb, const int32_t *par,
                                        TA *wa, int mode, bool init_P, bool force = true) {
  const int n = pb.n;
  const T *qdd_in = mode == MODE_ID ? pb.in3 : nullptr;
  for (int i = 0; i < n; ++i) {
    T *w = pb.wt + static_cast<int64_t>(i) * NT;
    const T *rec = pb.rec + static_cast<int64_t>(i) * REC;
    SE3<T> g;
    joint_transform(rec, pb.q[i], g);
    st_se3(w + TW_G, g);
    const int l = par[i];
    T V[6], Vd[6];
    if (l >= 0) {
      const T *wl = pb.wt + static_cast<int64_t>(l) * NT;
      ldv<T, 6>(wl + TW_V, V);
      ldv<T, 6>(wl + TW_A, Vd);
    } else {
#pragma unroll
      for (int k = 0; k < 6; ++k) V[k] = T(0);
      Vd[0] = Vd[1] = Vd[2] = T(0);  // the base's acceleration (0; -g): gravity
      Vd[3] = T(-A.grav[0]);
      Vd[4] = T(-A.grav[1]);
      Vd[5] = T(-A.grav[2]);
    }
    const T qdi = pb.qd[i];
    adinv(g, V, V);
    V[0] += qdi;
    adinv(g, Vd, Vd);
    // ad_V e_1 qd = (0, w_z, -w_y; 0, v_z, -v_y) qd
    Vd[1] += V[2] * qdi;
    Vd[2] -= V[1] * qdi;
    Vd[4] += V[5] * qdi;
    Vd[5] -= V[4] * qdi;
    if (qdd_in) Vd[0] += qdd_in[i];
    stv<T, 6>(w + TW_V, V);
    stv<T, 6>(w + TW_A, Vd);
    T JV[6], f[6];
    sym6_apply(rec + REC_J, V, JV);
    sym6_apply(rec + REC_J, Vd, f);
    adT_sub(V, JV, f);
    stv<T, 6>(w + TW_F, f);
    if (init_P) {
      TA *ra = wa + static_cast<int64_t>(i) * NA_TREE;
#pragma unroll
      for (int k = 0; k < 21; ++k) ra[TA_P + k] = TA(rec[REC_J + k]);
#pragma unroll
      for (int k = 0; k < 6; ++k) ra[TA_PB + k] = TA(0);
    }
  }
  if (!force) return;
  const bool fdm = mode != MODE_ID;
  for (int i = n - 1; i >= 0; --i) {
    SE3<T> g;
    ld_se3(pb.wt + static_cast<int64_t>(i) * NT + TW_G, g);
    pb.wt[static_cast<int64_t>(i) * NT + TW_TD] = tree_force_step(pb, par, i, g, fdm);
  }
}

// One step of Eq. 2c-2d over the parent array: link i's force F_i (its f_i plus
// what its children added), tau_delta_i (or tau_i), and Ad_{g_i^-1}^T F_i added
// into the parent's. Children have larger indices, so a descending sweep sees
// every F_i complete.
template <class T>
__device__ __forceinline__ T tree_force_step(const Prob<T> &pb, const int32_t *par, int i,
                                             const SE3<T> &g, bool fdm) {
  const T *w = pb.wt + static_cast<int64_t>(i) * NT;
  T F[6];
  ldv<T, 6>(w + TW_F, F);
  const int l = par[i];
  if (l >= 0) {
    T t[6];
    adinvT(g, F, t);
    T *wl = pb.wt + static_cast<int64_t>(l) * NT;
#pragma unroll
    for (int k = 0; k < 6; ++k) wl[TW_F + k] += t[k];
  }
  return fdm ? pb.in3[i] - F[0] : F[0];
}

// ABIA on a tree (Section II-C over a parent array): backward, link i's
// articulated inertia P_i (J_i plus its children's X^T Pa X) gives h = P_i S,
// D = S^T h, u = tau_delta_i - S^T p_i, and adds X_i^T Pa_i X_i, X_i^T pa_i into
// its parent's; forward, a_i = X_i a_parent, qdd_i = (u - h . a_i) / D,
// a_i += S qdd_i.
template <class T, class TA>
__device__ __forceinline__ void tree_abia_body(const KArgs &A, const Range &rg) {
  Team<1> tm;
  Prob<T> pb;
  if (!load_problem<T, 1>(A, rg, tm, pb, NT)) return;
  const int n = pb.n;
  const int32_t *par = A.parent + pb.m0;
  TA *wa = static_cast<TA *>(A.ws_a) + A.state_off[pb.p] * NA_TREE;
  bool bad = false;
  // the force pass runs inside the articulated-inertia sweep (both descend over
  // the links and share g_i)
  tree_id<T, TA>(A, pb, par, wa, A.mode, true, false);
  for (int i = n - 1; i >= 0; --i) {
    SE3<T> g;
    ld_se3(pb.wt + static_cast<int64_t>(i) * NT + TW_G, g);
    const T tdi = tree_force_step(pb, par, i, g, true);
    TA *ra = wa + static_cast<int64_t>(i) * NA_TREE;
    TA Pm[21], pbias[6], h[6];
#pragma unroll
    for (int k = 0; k < 21; ++k) Pm[k] = ra[TA_P + k];
#pragma unroll
    for (int k = 0; k < 6; ++k) pbias[k] = ra[TA_PB + k];
#pragma unroll
    for (int k = 0; k < 6; ++k) h[k] = Pm[s6(0, k)];
    const TA D = h[0];
    const TA u = TA(tdi) - pbias[0];
    bad |= !pos_t(D);
    const TA Dinv = rcp_t(D);
#pragma unroll
    for (int k = 0; k < 6; ++k) ra[TA_H + k] = h[k];
    ra[TA_DD] = Dinv;
    ra[TA_UU] = u * Dinv;
    const int l = par[i];
    if (l < 0) continue;
    // Pa = P - h h^T / D (row and column 0 vanish), pa = p + h u / D
    TA Pa[21], pa[6], hs[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) hs[k] = h[k] * Dinv;
#pragma unroll
    for (int r = 1; r < 6; ++r)
#pragma unroll
      for (int c = r; c < 6; ++c) Pa[s6(r, c)] = Pm[s6(r, c)] - h[r] * hs[c];
#pragma unroll
    for (int k = 0; k < 6; ++k) pa[k] = pbias[k] + hs[k] * u;
    SE3<TA> ga;
#pragma unroll
    for (int k = 0; k < 9; ++k) ga.R[k] = TA(g.R[k]);
#pragma unroll
    for (int k = 0; k < 3; ++k) ga.p[k] = TA(g.p[k]);
    TA *rl = wa + static_cast<int64_t>(l) * NA_TREE;
    TA Pl[21], t[6];
#pragma unroll
    for (int k = 0; k < 21; ++k) Pl[k] = rl[TA_P + k];
    congruence_add<TA, true>(ga, Pa, Pl);
#pragma unroll
    for (int k = 0; k < 21; ++k) rl[TA_P + k] = Pl[k];
    adinvT(ga, pa, t);
#pragma unroll
    for (int k = 0; k < 6; ++k) rl[TA_PB + k] += t[k];
  }
  for (int i = 0; i < n; ++i) {
    TA *ra = wa + static_cast<int64_t>(i) * NA_TREE;
    SE3<TA> ga;
    ld_se3(pb.wt + static_cast<int64_t>(i) * NT + TW_G, ga);
    TA acc[6] = {TA(0), TA(0), TA(0), TA(0), TA(0), TA(0)};
    const int l = par[i];
    if (l >= 0) {
      const TA *al = wa + static_cast<int64_t>(l) * NA_TREE + TA_AC;
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[k] = al[k];
      adinv(ga, acc, acc);
    }
    TA s = TA(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) s += ra[TA_H + k] * acc[k];
    const TA qdd = ra[TA_UU] - s * ra[TA_DD];
    acc[0] += qdd;
#pragma unroll
    for (int k = 0; k < 6; ++k) ra[TA_AC + k] = acc[k];
    const T v = T(qdd);
    pb.out[i] = v;
    if (!finite_t(v)) bad = true;
  }
  set_status(A.status, pb.p, bad ? 2 : 0);
}

// JSIIA on a tree (Section II-C over a parent array): composite inertias
// I^c_i = J_i + sum over children c of X_c^T I^c_c X_c (backward), then
// M[i][j] = S_j^T X_{j'}^T ... X_i^T I^c_i S_i for every ancestor j of i (the
// composite force of i's subtree carried up the path to j; zero off the paths),
// M = L^T L without fill-in and two triangular solves along the same paths.
template <class T, class TA>
__device__ __forceinline__ void tree_jsiia_body(const KArgs &A, const Range &rg) {
  Team<1> tm;
  Prob<T> pb;
  if (!load_problem<T, 1>(A, rg, tm, pb, NT)) return;
  const int n = pb.n;
  const int32_t *par = A.parent + pb.m0;
  const int64_t s0 = A.state_off[pb.p];
  TA *wa = static_cast<TA *>(A.ws_a) + s0 * NA_TREE + A.sq_off[pb.p];
  TA *M = wa + static_cast<int64_t>(n) * NA_TREE;  // n x n, column-major, lower triangle
  auto Mat = [&](int i, int j) -> TA & { return M[static_cast<int64_t>(j) * n + i]; };
  bool bad = false;
  tree_id<T, TA>(A, pb, par, wa, A.mode, true, false);
  for (int i = n - 1; i >= 0; --i) {
    SE3<T> g;
    ld_se3(pb.wt + static_cast<int64_t>(i) * NT + TW_G, g);
    const T tdi = tree_force_step(pb, par, i, g, true);
    TA *ra = wa + static_cast<int64_t>(i) * NA_TREE;
    TA Pm[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) Pm[k] = ra[TA_P + k];
#pragma unroll
    for (int k = 0; k < 6; ++k) ra[TA_H + k] = Pm[s6(0, k)];
    ra[TA_DD] = TA(tdi);  // the right-hand side
    const int l = par[i];
    if (l < 0) continue;
    SE3<TA> ga;
#pragma unroll
    for (int k = 0; k < 9; ++k) ga.R[k] = TA(g.R[k]);
#pragma unroll
    for (int k = 0; k < 3; ++k) ga.p[k] = TA(g.p[k]);
    TA *rl = wa + static_cast<int64_t>(l) * NA_TREE;
    TA Pl[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) Pl[k] = rl[TA_P + k];
    congruence_add<TA>(ga, Pm, Pl);
#pragma unroll
    for (int k = 0; k < 21; ++k) rl[TA_P + k] = Pl[k];
  }
  // entries on the paths to the base only: the factorisation below reads no other
  for (int i = 0; i < n; ++i) {
    TA F[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) F[k] = wa[static_cast<int64_t>(i) * NA_TREE + TA_H + k];
    Mat(i, i) = F[0];
    for (int j = i; par[j] >= 0;) {
      SE3<TA> ga;
      ld_se3(pb.wt + static_cast<int64_t>(j) * NT + TW_G, ga);
      adinvT(ga, F, F);
      j = par[j];
      Mat(i, j) = F[0];
    }
  }
  // M = L^T L factored from the leaves (row k of L has entries only at k's
  // ancestors, as M does: no fill-in; on a serial chain it is the Cholesky
  // factor of M with the links in reverse order). 1 / L_kk is kept in the h slot.
  for (int k = n - 1; k >= 0; --k) {
    const TA d = Mat(k, k);
    bad |= !pos_t(d);
    const TA r = rsqrt_t(d);
    wa[static_cast<int64_t>(k) * NA_TREE + TA_H] = r;  // L_kk itself is never read
    for (int i = par[k]; i >= 0; i = par[i]) Mat(k, i) *= r;
    for (int i = par[k]; i >= 0; i = par[i]) {
      const TA lki = Mat(k, i);
      for (int j = i; j >= 0; j = par[j]) Mat(i, j) -= lki * Mat(k, j);
    }
  }
  // L^T y = b from the leaves, then L x = y from the base, in the right-hand
  // side slot
  auto rhs = [&](int i) -> TA & { return wa[static_cast<int64_t>(i) * NA_TREE + TA_DD]; };
  for (int i = n - 1; i >= 0; --i) {
    const TA y = rhs(i) * wa[static_cast<int64_t>(i) * NA_TREE + TA_H];
    rhs(i) = y;
    for (int j = par[i]; j >= 0; j = par[j]) rhs(j) -= Mat(i, j) * y;
  }
  for (int i = 0; i < n; ++i) {
    TA x = rhs(i);
    for (int j = par[i]; j >= 0; j = par[j]) x -= Mat(i, j) * rhs(j);
    x *= wa[static_cast<int64_t>(i) * NA_TREE + TA_H];
    rhs(i) = x;
    const T v = T(x);
    pb.out[i] = v;
    if (!finite_t(v)) bad = true;
  }
  set_status(A.status, pb.p, bad ? 2 : 0);
}

// Closed loops: revolute loop joints between a frame F_a on link a (or the
// base) and a frame F_b on link b, turning about their x axes. The relative
// twist V_rel = V_Fb - Ad_{g_ba} V_Fa (F_b's body twist relative to F_a,
// g_ba = g_0Fb^-1 g_0Fa) may only turn about x, so its components 1..5 vanish:
// G qd = 0 with the rows G = (Ad_{g_0Fb^-1} sum over the path of b minus the path
// of a of s_j e_j^T)[1..5], s_j joint j's axis as a world twist, and at the
// acceleration level G qdd + gamma = 0 with
//   gamma = (Vd_Fb - Ad_{g_ba} Vd_Fa + ad_{V_Fb} Ad_{g_ba} V_Fa)[1..5]
// at qdd = 0 (the base's gravity enters both frames and cancels). JSIIA's
// factor M = L^T L and its free solution x0 = M^-1 (tau - bias) then give the
// constrained accelerations qdd = x0 - Y lam, Y = M^-1 G^T,
// (G Y) lam = G x0 + gamma (M qdd + G^T lam = tau - bias). Runs after the tree
// JSIIA kernel on its workspace: g_i, V_i, Vd_i of the inverse dynamics, L and
// 1 / L_kk, x0 in the output.
constexpr int MAX_LOOPS = MAX_LOOPS_PER_TREE;
constexpr int NA_LOOP = 12 + 2 * 5 * MAX_LOOPS;  // per link: g_0i, G's rows, Y's rows
static_assert(NA_LOOP == NA_LOOP_LINK, "loop workspace per link");
constexpr int LW_G0 = 0, LW_G = 12, LW_Y = 12 + 5 * MAX_LOOPS;

template <class T>
__device__ __forceinline__ void ad_fwd(const SE3<T> &g, const T *x, T *y) {  // Ad_g x
  T o[6];
#pragma unroll
  for (int i = 0; i < 3; ++i) o[i] = g.R[3 * i] * x[0] + g.R[3 * i + 1] * x[1] + g.R[3 * i + 2] * x[2];
#pragma unroll
  for (int i = 0; i < 3; ++i) o[3 + i] = g.R[3 * i] * x[3] + g.R[3 * i + 1] * x[4] + g.R[3 * i + 2] * x[5];
  T c[3];
  cross3(g.p, o, c);
#pragma unroll
  for (int i = 0; i < 3; ++i) y[i] = o[i];
#pragma unroll
  for (int i = 0; i < 3; ++i) y[3 + i] = o[3 + i] + c[i];
}

__device__ __forceinline__ void tree_loop_body(const KArgs &A, const Range &rg) {
  using T = double;
  Team<1> tm;
  Prob<T> pb;
  if (!load_problem<T, 1>(A, rg, tm, pb, NT)) return;
  const int n = pb.n;
  const int c = A.prob_chain ? A.prob_chain[pb.p] : pb.p;
  const int l0 = A.loop_off[c], nl = A.loop_off[c + 1] - l0;
  if (nl == 0 || n == 0) return;
  const int m = 5 * nl;
  const int32_t *par = A.parent + pb.m0;
  const int64_t s0 = A.state_off[pb.p];
  T *wj = static_cast<T *>(A.ws_a) + s0 * NA_TREE + A.sq_off[pb.p];
  const T *M = wj + static_cast<int64_t>(n) * NA_TREE;
  auto Lm = [&](int i, int j) -> T { return M[static_cast<int64_t>(j) * n + i]; };
  auto rinv = [&](int k) -> T { return wj[static_cast<int64_t>(k) * NA_TREE + TA_H]; };
  T *wl = static_cast<T *>(A.ws_a) + A.loop_ws + s0 * NA_LOOP;
  auto lw = [&](int i) -> T * { return wl + static_cast<int64_t>(i) * NA_LOOP; };
  bool bad = false;
  // world poses
  for (int i = 0; i < n; ++i) {
    SE3<T> g, g0;
    ld_se3(pb.wt + static_cast<int64_t>(i) * NT + TW_G, g);
    if (par[i] >= 0) {
      ld_se3(lw(par[i]) + LW_G0, g0);
      se3_mul(g0, g, g0);
    } else {
      g0 = g;
    }
    st_se3(lw(i) + LW_G0, g0);
#pragma unroll 1
    for (int r = 0; r < m; ++r) lw(i)[LW_G + r] = T(0);
  }
  // G's rows and gamma, loop by loop
  T gam[5 * MAX_LOOPS];
  for (int k = 0; k < nl; ++k) {
    const int a = A.loop_ab[2 * (l0 + k)], b = A.loop_ab[2 * (l0 + k) + 1];
    const double *Tk = A.loop_T + 24 * static_cast<int64_t>(l0 + k);
    SE3<T> Ta, Tb, gFa, gFb, gb;
    ld_se3(Tk, Ta);
    ld_se3(Tk + 12, Tb);
    ld_se3(lw(b) + LW_G0, gb);
    se3_mul(gb, Tb, gFb);
    if (a >= 0) {
      SE3<T> ga;
      ld_se3(lw(a) + LW_G0, ga);
      se3_mul(ga, Ta, gFa);
    } else {
      gFa = Ta;
    }
    for (int side = 0; side < 2; ++side) {
      const T sg = side ? T(-1) : T(1);
      for (int j = side ? a : b; j >= 0; j = par[j]) {
        SE3<T> g0;
        ld_se3(lw(j) + LW_G0, g0);
        // s_j = Ad_{g_0j} e_1 = (R e_1; p x R e_1)
        T sj[6] = {g0.R[0], g0.R[3], g0.R[6], T(0), T(0), T(0)};
        sj[3] = g0.p[1] * sj[2] - g0.p[2] * sj[1];
        sj[4] = g0.p[2] * sj[0] - g0.p[0] * sj[2];
        sj[5] = g0.p[0] * sj[1] - g0.p[1] * sj[0];
        T col[6];
        adinv(gFb, sj, col);
#pragma unroll
        for (int r = 0; r < 5; ++r) lw(j)[LW_G + 5 * k + r] += sg * col[r + 1];
      }
    }
    // gamma: the frames' twists and accelerations from the links' (qdd = 0)
    T Vb[6], Ab[6], VFb[6], AFb[6], VFa[6], AFa[6];
    ldv<T, 6>(pb.wt + static_cast<int64_t>(b) * NT + TW_V, Vb);
    ldv<T, 6>(pb.wt + static_cast<int64_t>(b) * NT + TW_A, Ab);
    adinv(Tb, Vb, VFb);
    adinv(Tb, Ab, AFb);
    if (a >= 0) {
      T Va[6], Aa[6];
      ldv<T, 6>(pb.wt + static_cast<int64_t>(a) * NT + TW_V, Va);
      ldv<T, 6>(pb.wt + static_cast<int64_t>(a) * NT + TW_A, Aa);
      adinv(Ta, Va, VFa);
      adinv(Ta, Aa, AFa);
    } else {
      const T base[6] = {T(0), T(0), T(0), T(-A.grav[0]), T(-A.grav[1]), T(-A.grav[2])};
#pragma unroll
      for (int r = 0; r < 6; ++r) VFa[r] = T(0);
      adinv(Ta, base, AFa);
    }
    T t[6], u[6], w[6];
    ad_fwd(gFa, AFa, t);   // Ad_{g_ba} = Ad_{g_0Fb^-1} Ad_{g_0Fa}
    adinv(gFb, t, u);
    ad_fwd(gFa, VFa, t);
    adinv(gFb, t, w);
    ad_apply(VFb, w, t);
#pragma unroll
    for (int r = 0; r < 5; ++r) gam[5 * k + r] = AFb[r + 1] - u[r + 1] + t[r + 1];
  }
  // Y = M^-1 G^T, row by row of G: L^T y = g from the leaves, L x = y from the base
  for (int r = 0; r < m; ++r) {
    for (int i = 0; i < n; ++i) lw(i)[LW_Y + r] = lw(i)[LW_G + r];
    for (int i = n - 1; i >= 0; --i) {
      const T y = lw(i)[LW_Y + r] * rinv(i);
      lw(i)[LW_Y + r] = y;
      for (int j = par[i]; j >= 0; j = par[j]) lw(j)[LW_Y + r] -= Lm(i, j) * y;
    }
    for (int i = 0; i < n; ++i) {
      T x = lw(i)[LW_Y + r];
      for (int j = par[i]; j >= 0; j = par[j]) x -= Lm(i, j) * lw(j)[LW_Y + r];
      lw(i)[LW_Y + r] = x * rinv(i);
    }
  }
  // K = G Y (m x m, symmetric positive definite when the loops are independent),
  // rhs = G x0 + gamma, K lam = rhs by Cholesky (packed lower, local memory)
  T K[5 * MAX_LOOPS * (5 * MAX_LOOPS + 1) / 2], lam[5 * MAX_LOOPS];
  for (int r = 0; r < m; ++r) {
    T rhs = gam[r];
    for (int i = 0; i < n; ++i) rhs += lw(i)[LW_G + r] * pb.out[i];
    lam[r] = rhs;
    for (int c2 = 0; c2 <= r; ++c2) {
      T kk = T(0);
      for (int i = 0; i < n; ++i) kk += lw(i)[LW_G + r] * lw(i)[LW_Y + c2];
      K[r * (r + 1) / 2 + c2] = kk;
    }
  }
  for (int j = 0; j < m; ++j) {
    T d = K[j * (j + 1) / 2 + j];
    for (int k = 0; k < j; ++k) d -= K[j * (j + 1) / 2 + k] * K[j * (j + 1) / 2 + k];
    bad |= !pos_t(d);
    const T rr = rsqrt_t(d);
    K[j * (j + 1) / 2 + j] = rr;  // 1 / L_jj
    for (int i = j + 1; i < m; ++i) {
      T x = K[i * (i + 1) / 2 + j];
      for (int k = 0; k < j; ++k) x -= K[i * (i + 1) / 2 + k] * K[j * (j + 1) / 2 + k];
      K[i * (i + 1) / 2 + j] = x * rr;
    }
  }
  for (int i = 0; i < m; ++i) {
    T x = lam[i];
    for (int k = 0; k < i; ++k) x -= K[i * (i + 1) / 2 + k] * lam[k];
    lam[i] = x * K[i * (i + 1) / 2 + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    T x = lam[i];
    for (int k = i + 1; k < m; ++k) x -= K[k * (k + 1) / 2 + i] * lam[k];
    lam[i] = x * K[i * (i + 1) / 2 + i];
  }
  // qdd = x0 - Y lam
  for (int i = 0; i < n; ++i) {
    T x = pb.out[i];
    for (int r = 0; r < m; ++r) x -= lw(i)[LW_Y + r] * lam[r];
    pb.out[i] = x;
    if (!finite_t(x)) bad = true;
  }
  if (bad) set_status(A.status, pb.p, 2);
}

__global__ void __launch_bounds__(128, 4) tree_loop_kernel(KArgs A) {
  tree_loop_body(A, Range{0, 0, A.n_problems});
}

// Inverse dynamics alone (MODE_ID): tau = ID(q, qd, qdd) on a tree.
template <class T>
__device__ __forceinline__ void tree_id_body(const KArgs &A, const Range &rg) {
  Team<1> tm;
  Prob<T> pb;
  if (!load_problem<T, 1>(A, rg, tm, pb, NT)) return;
  tree_id<T, T>(A, pb, A.parent + pb.m0, static_cast<T *>(nullptr), MODE_ID, false);
  for (int i = 0; i < pb.n; ++i) pb.out[i] = pb.wt[static_cast<int64_t>(i) * NT + TW_TD];
}

template <class T, class TA>
__global__ void __launch_bounds__(128, 4) tree_abia_kernel(KArgs A) {
  tree_abia_body<T, TA>(A, Range{0, 0, A.n_problems});
}

template <class T, class TA>
__global__ void __launch_bounds__(128, 4) tree_jsiia_kernel(KArgs A) {
  tree_jsiia_body<T, TA>(A, Range{0, 0, A.n_problems});
}

template <class T>
__global__ void __launch_bounds__(128, 4) tree_id_kernel(KArgs A) {
  tree_id_body<T>(A, Range{0, 0, A.n_problems});
}

}  // namespace fdk
