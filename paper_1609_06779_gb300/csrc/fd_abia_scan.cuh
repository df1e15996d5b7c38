// fd_abia_scan.cuh -- ABIA with the articulated-inertia recursion as a parallel
// scan (not in the paper: Section III notes that the ABI recursion, a rational
// recurrence, cannot be sped up beyond a constant factor by parallel
// processors; this is the associative form of this particular recurrence).
//
// In canonical frames (S_i = e_1, W = [e_2 .. e_6]) write the articulated
// inertia's constraint-space compliance C_i = W^T P_i^{-1} W (5x5). By the
// Woodbury identity the recursion P_i = J_i + X_{i+1}^T Pa_{i+1} X_{i+1}, with
// Pa = W C^{-1} W^T, becomes
//   C_i = K_i - H_i^T (C_{i+1} + G_i)^{-1} H_i,
//   K_i = W^T J_i^{-1} W,  H_i = (X_{i+1} J_i^{-1})[1..5][1..5] = -U_i^T,
//   G_i = (X_{i+1} J_i^{-1} X_{i+1}^T)[1..5][1..5]            (X = Ad_{g^{-1}}),
// and C_{n-1} = K_{n-1}: the same blocks as CFA's matrix A (D_i = K_i + G_{i-1},
// U_i = -H_i^T): ABIA factors A from the tip. Maps of this form compose in the
// same form -- f1 o f2 (f2 first) = (K1 - A^T A, B^T A, G2 - B^T B) with
// Z = K2 + G1 = L L^T, A = L^{-1} H1, B = L^{-1} H2^T -- by eliminating the
// shared block of an SPD block matrix: a Schur complement, stable where the
// 10x10 transfer matrices of the same maps lose their accuracy within a few
// links. So the recursion is a scan: each lane composes the maps of its
// segment, the team scans the segment maps (Kogge-Stone through shared memory),
// and each lane applies its maps from the value entering its segment. The bias
// force and acceleration recursions are affine (6x6 matrix + vector) and are
// scanned the same way. Every lane does about five times the serial arithmetic;
// the depth falls from n to n / P + log2 P steps.
#pragma once

#include "fd_kernels.cuh"

namespace fdk {

// per-lane shared-memory slot of the team scans (one Riccati map or one affine
// 6x6 map and a flag)
constexpr int SCAN_SLOT = 56;

// A Riccati map C -> K - H^T (C + G)^{-1} H: K, G packed symmetric (l5), H
// row-major 5x5; id: the identity map (no links); H == 0: a constant map.
struct RicMap {
  double K[15], H[25], G[15];
  bool id;
};

__device__ __forceinline__ void ric_store(double *s, const RicMap &m) {
#pragma unroll
  for (int k = 0; k < 15; ++k) s[k] = m.K[k];
#pragma unroll
  for (int k = 0; k < 25; ++k) s[15 + k] = m.H[k];
#pragma unroll
  for (int k = 0; k < 15; ++k) s[40 + k] = m.G[k];
  s[55] = m.id ? 1.0 : 0.0;
}

__device__ __forceinline__ void ric_load(const double *s, RicMap &m) {
#pragma unroll
  for (int k = 0; k < 15; ++k) m.K[k] = s[k];
#pragma unroll
  for (int k = 0; k < 25; ++k) m.H[k] = s[15 + k];
#pragma unroll
  for (int k = 0; k < 15; ++k) m.G[k] = s[40 + k];
  m.id = s[55] != 0.0;
}

// m1 <- m1 o m2 (m2 applied first); false if Z = K2 + G1 is not positive definite
__device__ __forceinline__ bool ric_compose(RicMap &m1, const RicMap &m2) {
  if (m2.id) return true;
  if (m1.id) {
    m1 = m2;
    return true;
  }
  double Z[15], L[15], inv[5];
#pragma unroll
  for (int k = 0; k < 15; ++k) Z[k] = m2.K[k] + m1.G[k];
  const bool ok = chol5(Z, L, inv);
  double A[5][5], B[5][5];  // A = L^{-1} H1, B = L^{-1} H2^T
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    double a[5], b[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      a[q] = m1.H[5 * q + c];
      b[q] = m2.H[5 * c + q];
    }
    fwd5(L, inv, a);
    fwd5(L, inv, b);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      A[q][c] = a[q];
      B[q][c] = b[q];
    }
  }
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c) {
      double k = m1.K[l5(r, c)], g = m2.G[l5(r, c)];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        k -= A[q][r] * A[q][c];
        g -= B[q][r] * B[q][c];
      }
      m1.K[l5(r, c)] = k;
      m1.G[l5(r, c)] = g;
    }
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      double h = 0.0;
#pragma unroll
      for (int q = 0; q < 5; ++q) h += B[q][r] * A[q][c];
      m1.H[5 * r + c] = h;
    }
  return ok;
}

// C <- m(C); false if C + G is not positive definite
__device__ __forceinline__ bool ric_apply(const RicMap &m, double *C) {
  if (m.id) return true;
  double Z[15], L[15], inv[5];
#pragma unroll
  for (int k = 0; k < 15; ++k) Z[k] = C[k] + m.G[k];
  const bool ok = chol5(Z, L, inv);
  double A[5][5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    double a[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) a[q] = m.H[5 * q + c];
    fwd5(L, inv, a);
#pragma unroll
    for (int q = 0; q < 5; ++q) A[q][c] = a[q];
  }
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c) {
      double k = m.K[l5(r, c)];
#pragma unroll
      for (int q = 0; q < 5; ++q) k -= A[q][r] * A[q][c];
      C[l5(r, c)] = k;
    }
  return ok;
}

// The map of link i: C_{i+1} -> C_i (the tip link's is constant, K_{n-1}).
__device__ __forceinline__ void ric_link(const Prob<double> &pb, int i, RicMap &m) {
  const double *Ki = pb.rec + static_cast<int64_t>(i) * REC + REC_JI;
  m.id = false;
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c) m.K[l5(r, c)] = Ki[s6(r + 1, c + 1)];
  if (i + 1 < pb.n) {
    SE3<double> gn;
    ld_se3(pb.wt + static_cast<int64_t>(i + 1) * NT + W_G, gn);
    double U[25];
    calc_ublock<double, double>(gn, Ki, U);  // U_i = -H_i^T
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
      for (int c = 0; c < 5; ++c) m.H[5 * r + c] = -U[5 * c + r];
    double zero[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) zero[k] = 0.0;
    calc_dblock<double, double>(&gn, Ki, zero, m.G);  // (X J^{-1} X^T)[1..5][1..5]
  } else {
#pragma unroll
    for (int k = 0; k < 25; ++k) m.H[k] = 0.0;
#pragma unroll
    for (int k = 0; k < 15; ++k) m.G[k] = 0.0;
  }
}

// An affine map x -> M x + v of 6-vectors (M row-major), with a second
// translation v2 for a second right-hand side y -> M y + v2 (MODE_FD2: the
// adjoint's M^{-1} w beside FD; the matrices are the same); id: the identity.
struct AffMap {
  double M[36], v[6], v2[6];
  bool id;
};

__device__ __forceinline__ void aff_store(double *s, const AffMap &a) {
#pragma unroll
  for (int k = 0; k < 36; ++k) s[k] = a.M[k];
#pragma unroll
  for (int k = 0; k < 6; ++k) s[36 + k] = a.v[k];
#pragma unroll
  for (int k = 0; k < 6; ++k) s[42 + k] = a.v2[k];
  s[48] = a.id ? 1.0 : 0.0;
}

__device__ __forceinline__ void aff_load(const double *s, AffMap &a) {
#pragma unroll
  for (int k = 0; k < 36; ++k) a.M[k] = s[k];
#pragma unroll
  for (int k = 0; k < 6; ++k) a.v[k] = s[36 + k];
#pragma unroll
  for (int k = 0; k < 6; ++k) a.v2[k] = s[42 + k];
  a.id = s[48] != 0.0;
}

// a1 <- a1 o a2 (a2 applied first): (M1 M2, M1 v_2 + v_1), the second
// translations alike when TWO
template <bool TWO>
__device__ __forceinline__ void aff_compose(AffMap &a1, const AffMap &a2) {
  if (a2.id) return;
  if (a1.id) {
    a1 = a2;
    return;
  }
  double M[36], v[6], w[6];
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    double s = a1.v[r];
#pragma unroll
    for (int k = 0; k < 6; ++k) s += a1.M[6 * r + k] * a2.v[k];
    v[r] = s;
    if (TWO) {
      double t = a1.v2[r];
#pragma unroll
      for (int k = 0; k < 6; ++k) t += a1.M[6 * r + k] * a2.v2[k];
      w[r] = t;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) t += a1.M[6 * r + k] * a2.M[6 * k + c];
      M[6 * r + c] = t;
    }
  }
#pragma unroll
  for (int k = 0; k < 36; ++k) a1.M[k] = M[k];
#pragma unroll
  for (int k = 0; k < 6; ++k) a1.v[k] = v[k];
  if (TWO) {
#pragma unroll
    for (int k = 0; k < 6; ++k) a1.v2[k] = w[k];
  }
}

// x <- M x + v (second = false) or M x + v2 (second = true)
__device__ __forceinline__ void aff_apply(const AffMap &a, double *x, bool second = false) {
  if (a.id) return;
  double y[6];
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    double s = second ? a.v2[r] : a.v[r];
#pragma unroll
    for (int k = 0; k < 6; ++k) s += a.M[6 * r + k] * x[k];
    y[r] = s;
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) x[k] = y[k];
}

// Kogge-Stone over the team's lanes through shared-memory slots. BACK: lane r
// ends with the composite of lanes r+1 .. P-1 (their maps act before its own in
// the backward recursions), else of lanes 0 .. r-1 (the forward one); `mine`
// holds the lane's own segment map on entry.
template <int P, bool BACK, class Map, class Store, class Load, class Compose>
__device__ __forceinline__ bool team_scan_maps(const Team<P> &tm, double *slot, Map &mine,
                                              Store st, Load ld, Compose comp) {
  bool ok = true;
#pragma unroll 1
  for (int d = 1; d < P; d *= 2) {
    st(slot, mine);
    tm.sync();
    if (BACK ? tm.r + d < P : tm.r >= d) {
      Map other;
      ld(slot + (BACK ? d : -d) * SCAN_SLOT, other);
      ok &= comp(mine, other);  // mine o other: the other lanes' maps act first
    }
    tm.sync();
  }
  // exclusive: the inclusive composite of the neighbour (toward the start)
  st(slot, mine);
  tm.sync();
  if (BACK ? tm.r + 1 < P : tm.r >= 1) ld(slot + (BACK ? 1 : -1) * SCAN_SLOT, mine);
  else mine.id = true;
  tm.sync();
  return ok;
}

// TWO (MODE_FD2): a second right-hand side in4 shares the articulated inertias;
// its bias forces and accelerations ride in the affine maps' second translation
// and give M^{-1} in4 in out4 (the adjoint's linear solve beside FD).
template <int P, bool TWO>
__device__ __forceinline__ void abia_scan_body(const KArgs &A, const Range &rg, double *smem) {
  Team<P> tm;
  Prob<double> pb;
  if (!load_problem<double, P>(A, rg, tm, pb, NT)) return;
  const int n = pb.n, a = pb.a, b = pb.b;
  double *slot = smem + static_cast<int64_t>(threadIdx.x) * SCAN_SLOT;
  double *wa = static_cast<double *>(A.ws_a) + A.state_off[pb.p] * NA_ABIA;
  bool bad = false;
  const double *td2 = TWO ? static_cast<const double *>(A.in4) + A.state_off[pb.p] : nullptr;
  double *out2 = TWO ? static_cast<double *>(A.out4) + A.state_off[pb.p] : nullptr;

  // tau_delta = tau - ID(q, qd, 0) (Algorithm 1's bias torque) and the joint transforms
  id_team<double, P>(tm, pb, A.grav, A.mode);
  tm.sync();

  // 1. the compliances C_i by a backward scan of the Riccati maps
  RicMap seg;
  seg.id = true;
  for (int i = a; i < b; ++i) {  // seg = map_a o ... o map_{b-1}
    RicMap m;
    ric_link(pb, i, m);
    bad |= !ric_compose(seg, m);
  }
  bad |= !team_scan_maps<P, true>(
      tm, slot, seg, [](double *s, const RicMap &m) { ric_store(s, m); },
      [](const double *s, RicMap &m) { ric_load(s, m); },
      [](RicMap &x, const RicMap &y) { return ric_compose(x, y); });
  // C entering the segment (C_b); the composite is constant (it holds the tip's
  // map) unless this lane holds the tip, whose own map is constant
  double C[15];
#pragma unroll
  for (int k = 0; k < 15; ++k) C[k] = (k == 0 || k == 2 || k == 5 || k == 9 || k == 14) ? 1.0 : 0.0;
  bad |= !ric_apply(seg, C);
  // h_i = P_i e_1 and D_i for every link of the segment, from C_{i+1}
  for (int i = b - 1; i >= a; --i) {
    const double *rec = pb.rec + static_cast<int64_t>(i) * REC;
    double h[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) h[k] = rec[REC_J + s6(k, 0)];
    if (i + 1 < n) {
      // + X^T (W S5 W^T) X e_1 with S5 = C_{i+1}^{-1}
      SE3<double> gn;
      ld_se3(pb.wt + static_cast<int64_t>(i + 1) * NT + W_G, gn);
      const double e1[6] = {1.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      double x[6], y[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, t[6];
      adinv(gn, e1, x);
      double L[15], inv[5], r5[5];
      bad |= !chol5(C, L, inv);
#pragma unroll
      for (int k = 0; k < 5; ++k) r5[k] = x[k + 1];
      fwd5(L, inv, r5);
      bwd5(L, inv, r5);
#pragma unroll
      for (int k = 0; k < 5; ++k) y[k + 1] = r5[k];
      adinvT(gn, y, t);
#pragma unroll
      for (int k = 0; k < 6; ++k) h[k] += t[k];
    }
    const double Dinv = rcp_t(h[0]);
    if (!pos_t(h[0])) bad = true;
    double *ra = wa + static_cast<int64_t>(i) * NA_ABIA;
#pragma unroll
    for (int k = 0; k < 6; ++k) ra[A_H + k] = h[k];
    ra[A_DD] = Dinv;
    RicMap m;
    ric_link(pb, i, m);
    bad |= !ric_apply(m, C);  // C_i
  }
  tm.sync();

  // 2. the bias forces p_i = X_{i+1}^T (I - h_{i+1} e_1^T / D_{i+1}) p_{i+1}
  //    + X_{i+1}^T h_{i+1} tau_{i+1} / D_{i+1}, p_{n-1} = 0 (backward scan)
  auto bias_map = [&](int i, AffMap &m) {
    m.id = false;
    if (i + 1 >= n) {
#pragma unroll
      for (int k = 0; k < 36; ++k) m.M[k] = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) m.v[k] = m.v2[k] = 0.0;
      return;
    }
    SE3<double> gn;
    ld_se3(pb.wt + static_cast<int64_t>(i + 1) * NT + W_G, gn);
    const double *rn = wa + static_cast<int64_t>(i + 1) * NA_ABIA;
    double h[6], xh[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) h[k] = rn[A_H + k];
    adinvT(gn, h, xh);  // X^T h
    const double Dinv = rn[A_DD];
    const double td = pb.wt[static_cast<int64_t>(i + 1) * NT + W_TD];
    // columns of X^T, column 0 less X^T h / D
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double e[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, col[6];
      e[c] = 1.0;
      adinvT(gn, e, col);
#pragma unroll
      for (int r = 0; r < 6; ++r) m.M[6 * r + c] = c == 0 ? col[r] - xh[r] * Dinv : col[r];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) m.v[k] = xh[k] * (td * Dinv);
    if (TWO) {
      const double t2 = td2[i + 1];
#pragma unroll
      for (int k = 0; k < 6; ++k) m.v2[k] = xh[k] * (t2 * Dinv);
    }
  };
  AffMap sa;
  sa.id = true;
  for (int i = a; i < b; ++i) {
    AffMap m;
    bias_map(i, m);
    aff_compose<TWO>(sa, m);
  }
  team_scan_maps<P, true>(
      tm, slot, sa, [](double *s, const AffMap &m) { aff_store(s, m); },
      [](const double *s, AffMap &m) { aff_load(s, m); },
      [](AffMap &x, const AffMap &y) { aff_compose<TWO>(x, y); return true; });
  double p[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, p2[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  aff_apply(sa, p);
  if (TWO) aff_apply(sa, p2, true);
  for (int i = b - 1; i >= a; --i) {
    AffMap m;
    bias_map(i, m);
    aff_apply(m, p);  // p_i
    double *ra = wa + static_cast<int64_t>(i) * NA_ABIA;
    ra[A_UU] = (pb.wt[static_cast<int64_t>(i) * NT + W_TD] - p[0]) * ra[A_DD];  // u_i / D_i
    if (TWO) {
      aff_apply(m, p2, true);
      ra[A_UU2] = (td2[i] - p2[0]) * ra[A_DD];
    }
  }
  tm.sync();

  // 3. the accelerations a_i = (I - e_1 h_i^T / D_i) X_i a_{i-1} + e_1 u_i / D_i,
  //    a_{-1} = 0 (forward scan); qdd_i = u_i / D_i - h_i^T X_i a_{i-1} / D_i
  auto acc_map = [&](int i, AffMap &m) {
    m.id = false;
    const double *ri = wa + static_cast<int64_t>(i) * NA_ABIA;
    SE3<double> g;
    ld_se3(pb.wt + static_cast<int64_t>(i) * NT + W_G, g);
    double hx[6];  // X^T h: row 0 of the map is row 0 of X less (X^T h)^T / D
    double h[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) h[k] = ri[A_H + k];
    adinvT(g, h, hx);
    const double Dinv = ri[A_DD];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double e[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, col[6];
      e[c] = 1.0;
      adinv(g, e, col);
#pragma unroll
      for (int r = 0; r < 6; ++r) m.M[6 * r + c] = r == 0 ? col[0] - hx[c] * Dinv : col[r];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) m.v[k] = k == 0 ? ri[A_UU] : 0.0;
    if (TWO) {
#pragma unroll
      for (int k = 0; k < 6; ++k) m.v2[k] = k == 0 ? ri[A_UU2] : 0.0;
    }
  };
  AffMap fa;
  fa.id = true;
  for (int i = a; i < b; ++i) {  // fa = map_{b-1} o ... o map_a
    AffMap m;
    acc_map(i, m);
    aff_compose<TWO>(m, fa);
    fa = m;
  }
  team_scan_maps<P, false>(
      tm, slot, fa, [](double *s, const AffMap &m) { aff_store(s, m); },
      [](const double *s, AffMap &m) { aff_load(s, m); },
      [](AffMap &x, const AffMap &y) { aff_compose<TWO>(x, y); return true; });
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, acc2[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  aff_apply(fa, acc);
  if (TWO) aff_apply(fa, acc2, true);
  for (int i = a; i < b; ++i) {
    const double *ri = wa + static_cast<int64_t>(i) * NA_ABIA;
    SE3<double> g;
    ld_se3(pb.wt + static_cast<int64_t>(i) * NT + W_G, g);
    double ap[6];
    adinv(g, acc, ap);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) s += ri[A_H + k] * ap[k];
    const double qdd = ri[A_UU] - s * ri[A_DD];
    pb.out[i] = qdd;
    if (!finite_t(qdd)) bad = true;
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] = ap[k];
    acc[0] += qdd;
    if (TWO) {
      adinv(g, acc2, ap);
      double s2 = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) s2 += ri[A_H + k] * ap[k];
      const double x = ri[A_UU2] - s2 * ri[A_DD];
      out2[i] = x;
      if (!finite_t(x)) bad = true;
#pragma unroll
      for (int k = 0; k < 6; ++k) acc2[k] = ap[k];
      acc2[0] += x;
    }
  }
  const bool any_bad = tm.any(bad);
  if (tm.r == 0) set_status(A.status, pb.p, any_bad ? 2 : 0);
}

template <int P, bool TWO>
__global__ void __launch_bounds__(block_for<P>()) abia_scan_kernel(KArgs A) {
  extern __shared__ __align__(16) double scan_smem[];
  abia_scan_body<P, TWO>(A, Range{0, 0, A.n_problems}, scan_smem);
}

}  // namespace fdk
