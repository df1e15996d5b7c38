// fd_adjoint.cuh -- reverse-mode inverse dynamics for the adjoint of forward
// dynamics.
//
// Forward dynamics satisfies ID(q, qd, FD(q, qd, tau)) = tau, so for a cotangent
// w of qdd and lambda = M^{-1} w:
//   tau_bar = lambda,  x_bar = -(d ID / d x)^T lambda  for x = q, qd, link masses.
// (d ID / d x)^T lambda is the reverse sweep of Eq. 2a-2d written out by hand in
// canonical frames (S_i = e_1, X_i = Ad_{g_i^{-1}}, dX_i/dq_i = -ad_{e_1} X_i):
//   Fbar_i = X_i Fbar_{i-1} + e_1 lambda_i                       (forward)
//   Abar_i = X_{i+1}^T Abar_{i+1} + J_i Fbar_i                   (backward)
//   Vbar_i = X_{i+1}^T Vbar_{i+1} + ad_{Fbar_i}^T (J_i V_i) - J_i ad_{V_i} Fbar_i
//            - qd_i ad_{e_1}^T Abar_i                             (backward)
//   g_qd_i = Vbar_i[0] + (ad_{V_i} e_1) . Abar_i
//   g_q_i  = -[Vbar_i . ad_{e_1} V_i + Abar_i . ad_{e_1}(A_i - qd_i ad_{V_i} e_1)
//             + (ad_{e_1} Fbar_i) . F_i]
//   g_m_i  = Fbar_i^T J'_i A_i - (ad_{V_i} Fbar_i)^T J'_i V_i,  J' = dJ/dm
// with c (centre of mass) and I_c held fixed: dJ/dm = [[-c^ c^, c^], [-c^, 1]].
// All six recursions are the two operator forms of the forward-dynamics scans.
#pragma once

#include "fd_kernels.cuh"

namespace fdk {

template <class T>
__device__ __forceinline__ T dot6(const T *a, const T *b) {
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 6; ++k) s += a[k] * b[k];
  return s;
}

// y = dJ/dm x for a rigid-body inertia J (J[3..5][3..5] = m 1, J[0..2][3..5] = m c^)
template <class T>
__device__ __forceinline__ void dJdm_apply(const T *J, const T *x, T *y) {
  const T m = J[s6(3, 3)];
  const T inv = T(1) / m;
  // c from the skew block m c^ = [[0, -m cz, m cy], [m cz, 0, -m cx], [-m cy, m cx, 0]]
  const T c[3] = {J[s6(2, 4)] * inv, J[s6(0, 5)] * inv, J[s6(1, 3)] * inv};
  T cxw[3], cxv[3], cxcxw[3];
  cross3(c, x, cxw);          // c^ w
  cross3(c, x + 3, cxv);      // c^ v
  cross3(c, cxw, cxcxw);      // c^ c^ w
  y[0] = -cxcxw[0] + cxv[0];
  y[1] = -cxcxw[1] + cxv[1];
  y[2] = -cxcxw[2] + cxv[2];
  y[3] = -cxw[0] + x[3];
  y[4] = -cxw[1] + x[4];
  y[5] = -cxw[2] + x[5];
}

// The same six recursions on component lanes (teams of 8..32, chains up to the
// inverse dynamics' component-lane length): lanes 0..5 carry the six
// components; the three forward recursions (V, A, Fbar) run in one serial loop
// over the links and the three backward ones (F, Abar, Vbar) in another, one
// transport per recursion per lane per link, while every term that does not
// recur (joint transforms, f_i, J_i Fbar_i, the Vbar term without Abar, and the
// gradients) runs one link per lane. Returns after writing the outputs.
template <class T, int P>
__device__ __forceinline__ void adjoint_lanes(const Team<P> &tm, const Prob<T> &pb,
                                              const KArgs &A, const T *lam, T *qbar, T *qdbar,
                                              T *mbar) {
  const int n = pb.n;
  const int r = tm.r < 6 ? tm.r : 5;
  const bool top = r < 3;
  const int k = top ? r : r - 3;
  const int ka = k == 2 ? 0 : k + 1, kb = k == 0 ? 2 : k - 1;  // k+1, k+2 mod 3
  const bool store = tm.r < 6;
  auto W = [&](int i) { return pb.wt + static_cast<int64_t>(i) * NT_ADJ; };
  auto REC_ = [&](int i) { return pb.rec + static_cast<int64_t>(i) * REC; };

  // joint transforms and R^T p, one link per lane
  for (int i = tm.r; i < n; i += P) {
    SE3<T> g;
    joint_transform(REC_(i), pb.q[i], g);
    st_se3(W(i) + J_G, g);
#pragma unroll
    for (int j = 0; j < 3; ++j)
      W(i)[J_PT + j] = g.R[j] * g.p[0] + g.R[3 + j] * g.p[1] + g.R[6 + j] * g.p[2];
  }
  tm.sync();

  // component k of Ad_{g^-1} x: R^T w (top), R^T v + (R^T w) x (R^T p) (bottom).
  // Every lane runs the same FP64 instructions: operands are picked by selects and
  // the callers pass pa = pbk = 0 on the lanes that take no cross product.
  auto fwd_c = [&](const T *x, T c0, T c1, T c2, T pa, T pbk) {
    const T t = c0 * (top ? x[0] : x[3]) + c1 * (top ? x[1] : x[4]) + c2 * (top ? x[2] : x[5]);
    const T oa = __shfl_sync(tm.mask, t, ka, P), ob = __shfl_sync(tm.mask, t, kb, P);
    return (t + oa * pbk) - ob * pa;
  };
  // component k of Ad_{g^-1}^T y: R n + p x R f (top), R f (bottom)
  auto bwd_c = [&](const T *y, T c0, T c1, T c2, T pa, T pbk) {
    const T t = c0 * (top ? y[0] : y[3]) + c1 * (top ? y[1] : y[4]) + c2 * (top ? y[2] : y[5]);
    const T fa = __shfl_sync(tm.mask, t, 3 + ka, P), fb = __shfl_sync(tm.mask, t, 3 + kb, P);
    return (t + pa * fb) - pbk * fa;
  };
  auto gather = [&](T v, T *full) {
#pragma unroll
    for (int j = 0; j < 6; ++j) full[j] = __shfl_sync(tm.mask, v, j, P);
  };

  // forward: V (Eq. 2a), A (Eq. 2b at qdd = in3), Fbar_i = X_i Fbar_{i-1} + e_1 lambda_i
  {
    T V[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    T Ac[6] = {T(0), T(0), T(0), T(-A.grav[0]), T(-A.grav[1]), T(-A.grav[2])};
    T Fb[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    for (int i = 0; i < n; ++i) {
      T *w = W(i);
      const T c0 = w[J_G + k], c1 = w[J_G + 3 + k], c2 = w[J_G + 6 + k];
      const T pa = top ? T(0) : w[J_PT + ka], pbk = top ? T(0) : w[J_PT + kb];
      const T qdi = pb.qd[i];
      T y = fwd_c(V, c0, c1, c2, pa, pbk) + (r == 0 ? qdi : T(0));
      gather(y, V);
      if (store) w[J_V + r] = y;
      const T cv = neg_if(r == 1 ? V[2] : (r == 2 ? V[1] : (r == 4 ? V[5] : (r == 5 ? V[4] : T(0)))),
                          r == 2 || r == 5);
      y = fwd_c(Ac, c0, c1, c2, pa, pbk) + cv * qdi + (r == 0 ? pb.in3[i] : T(0));
      gather(y, Ac);
      if (store) w[J_A + r] = y;
      y = fwd_c(Fb, c0, c1, c2, pa, pbk) + (r == 0 ? lam[i] : T(0));
      gather(y, Fb);
      if (store) w[J_FB + r] = y;
    }
  }
  tm.sync();

  // terms that do not recur, one link per lane: f_i (into J_F), J_i Fbar_i (into
  // J_AB), ad_{Fbar_i}^T (J_i V_i) - J_i ad_{V_i} Fbar_i (into J_VB)
  for (int i = tm.r; i < n; i += P) {
    T *w = W(i);
    const T *J = REC_(i) + REC_J;
    T V[6], Ai[6], Fb[6], JV[6], t1[6], t2[6], t3[6];
    ldv<T, 6>(w + J_V, V);
    ldv<T, 6>(w + J_A, Ai);
    ldv<T, 6>(w + J_FB, Fb);
    sym6_apply(J, V, JV);
    sym6_apply(J, Ai, t2);
    adT_sub(V, JV, t2);
    stv<T, 6>(w + J_F, t2);   // f_i = J A - ad_V^T J V
    sym6_apply(J, Fb, t2);
    stv<T, 6>(w + J_AB, t2);  // J_i Fbar_i
    ad_apply(V, Fb, t1);      // ad_V Fbar
    sym6_apply(J, t1, t3);    // J ad_V Fbar
    adT_sub(Fb, JV, t3);      // minus the Vbar term: J ad_V Fbar - ad_{Fbar}^T (J V)
    stv<T, 6>(w + J_VB, t3);
  }
  tm.sync();

  // backward: F_i = X_{i+1}^T F_{i+1} + f_i, Abar_i = X_{i+1}^T Abar_{i+1} + J_i Fbar_i,
  // Vbar_i = X_{i+1}^T Vbar_{i+1} + (the Vbar term) - qd_i ad_{e_1}^T Abar_i
  {
    T F[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    T Ab[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    T Vb[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    for (int i = n - 1; i >= 0; --i) {
      T *w = W(i);
      T yF = w[J_F + r], yA = w[J_AB + r], yV;
      const T nv = w[J_VB + r];  // minus the Vbar term
      if (i + 1 < n) {
        const T *wn = W(i + 1);
        const T c0 = wn[J_G + 3 * k], c1 = wn[J_G + 3 * k + 1], c2 = wn[J_G + 3 * k + 2];
        const T pa = top ? wn[J_G + 9 + ka] : T(0), pbk = top ? wn[J_G + 9 + kb] : T(0);
        yF += bwd_c(F, c0, c1, c2, pa, pbk);
        yA += bwd_c(Ab, c0, c1, c2, pa, pbk);
        yV = bwd_c(Vb, c0, c1, c2, pa, pbk) - nv;
      } else {
        yV = -nv;
      }
      gather(yF, F);
      gather(yA, Ab);
      // - qd ad_{e_1}^T Abar = qd (0, -n_z, n_y; 0, -f_z, f_y)
      const T qdi = pb.qd[i];
      const T ca = neg_if(r == 1 ? Ab[2] : (r == 2 ? Ab[1] : (r == 4 ? Ab[5] : (r == 5 ? Ab[4] : T(0)))),
                          r == 1 || r == 4);
      yV += qdi * ca;
      gather(yV, Vb);
      if (store) {
        w[J_F + r] = yF;
        w[J_AB + r] = yA;
        w[J_VB + r] = yV;
      }
    }
  }
  tm.sync();
}

template <class T, int P>
__device__ __forceinline__ void adjoint_body(const KArgs &A, const Range &rg) {
  Team<P> tm;
  Prob<T> pb;
  if (!load_problem<T, P>(A, rg, tm, pb, NT_ADJ)) return;
  const int a = pb.a, b = pb.b;
  const int64_t s0 = A.state_off[pb.p];
  const T *lam = static_cast<const T *>(A.lam) + s0;
  T *qbar = static_cast<T *>(A.out) + s0;
  T *qdbar = static_cast<T *>(A.out2) + s0;
  T *mbar = A.out3 ? static_cast<T *>(A.out3) + s0 : nullptr;
  auto W = [&](int i) { return pb.wt + static_cast<int64_t>(i) * NT_ADJ; };
  auto REC_ = [&](int i) { return pb.rec + static_cast<int64_t>(i) * REC; };
  bool lanes = false;
  if constexpr (P >= 8 && P <= 32) lanes = pb.n <= lanes_id_max_links<P>();
  if (lanes) {
    adjoint_lanes<T, P>(tm, pb, A, lam, qbar, qdbar, mbar);
  } else {
  SegOp<T> op;
  se3_identity(op.h);
  for (int i = a; i < b; ++i) {
    SE3<T> g;
    joint_transform(REC_(i), pb.q[i], g);
    st_se3(W(i) + J_G, g);
    if (P > 1) se3_mul(op.h, g, op.h);
  }
  const T zero6[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  const T base[6] = {T(0), T(0), T(0), T(-A.grav[0]), T(-A.grav[1]), T(-A.grav[2])};

  // generic forward recursion x_i = X_i x_{i-1} + c(i), stored at field `dst`
  auto fwd = [&](const T *x_base, int dst, auto cfun) {
    T x[6];
    if (P > 1) {
      for (int k = 0; k < 6; ++k) x[k] = T(0);
      for (int i = a; i < b; ++i) {
        SE3<T> g;
        ld_se3(W(i) + J_G, g);
        adinv(g, x, x);
        T c[6];
        cfun(i, c);
        for (int k = 0; k < 6; ++k) x[k] += c[k];
      }
      for (int k = 0; k < 6; ++k) op.psi[k] = x[k];
      team_scan_fwd(tm, op, x_base, x);
    } else {
      for (int k = 0; k < 6; ++k) x[k] = x_base[k];
    }
    for (int i = a; i < b; ++i) {
      SE3<T> g;
      ld_se3(W(i) + J_G, g);
      adinv(g, x, x);
      T c[6];
      cfun(i, c);
      for (int k = 0; k < 6; ++k) x[k] += c[k];
      stv<T, 6>(W(i) + dst, x);
    }
  };
  // generic backward recursion y_i = X_{i+1}^T y_{i+1} + l(i), stored at `dst`
  auto bwd = [&](int dst, auto lfun) {
    T y[6];
    if (P > 1) {
      for (int k = 0; k < 6; ++k) y[k] = T(0);
      for (int i = b - 1; i >= a; --i) {
        SE3<T> g;
        ld_se3(W(i) + J_G, g);
        T l[6];
        lfun(i, l);
        for (int k = 0; k < 6; ++k) y[k] += l[k];
        adinvT(g, y, y);
      }
      for (int k = 0; k < 6; ++k) op.psi[k] = y[k];
      team_scan_bwd(tm, op, y);
    } else {
      for (int k = 0; k < 6; ++k) y[k] = T(0);
    }
    for (int i = b - 1; i >= a; --i) {
      SE3<T> g;
      ld_se3(W(i) + J_G, g);
      T l[6];
      lfun(i, l);
      for (int k = 0; k < 6; ++k) y[k] += l[k];
      stv<T, 6>(W(i) + dst, y);
      adinvT(g, y, y);
    }
  };

  // inverse dynamics at (q, qd, qdd): V, A = Vd, F (Eq. 2a-2d)
  fwd(zero6, J_V, [&](int i, T *c) {
    for (int k = 0; k < 6; ++k) c[k] = T(0);
    c[0] = pb.qd[i];
  });
  fwd(base, J_A, [&](int i, T *c) {
    const T *V = W(i) + J_V;
    const T qdi = pb.qd[i];
    c[0] = pb.in3[i];
    c[1] = V[2] * qdi;
    c[2] = -V[1] * qdi;
    c[3] = T(0);
    c[4] = V[5] * qdi;
    c[5] = -V[4] * qdi;
  });
  for (int i = a; i < b; ++i) {  // f_i = J A - ad_V^T J V  (kept in J_FB for now)
    T V[6], Ai[6], JV[6], JA[6], c[6];
    ldv<T, 6>(W(i) + J_V, V);
    ldv<T, 6>(W(i) + J_A, Ai);
    sym6_apply(REC_(i) + REC_J, Ai, JA);
    sym6_apply(REC_(i) + REC_J, V, JV);
    adT_sub(V, JV, JA);
    stv<T, 6>(W(i) + J_FB, JA);
  }
  bwd(J_F, [&](int i, T *l) { ldv<T, 6>(W(i) + J_FB, l); });

  // reverse sweep
  fwd(zero6, J_FB, [&](int i, T *c) {
    for (int k = 0; k < 6; ++k) c[k] = T(0);
    c[0] = lam[i];
  });
  bwd(J_AB, [&](int i, T *l) {
    T Fb[6];
    ldv<T, 6>(W(i) + J_FB, Fb);
    sym6_apply(REC_(i) + REC_J, Fb, l);
  });
  bwd(J_VB, [&](int i, T *l) {
    T V[6], Fb[6], Ab[6], JV[6], t1[6], t2[6], t3[6];
    ldv<T, 6>(W(i) + J_V, V);
    ldv<T, 6>(W(i) + J_FB, Fb);
    ldv<T, 6>(W(i) + J_AB, Ab);
    sym6_apply(REC_(i) + REC_J, V, JV);
    adT_apply(Fb, JV, t1);               // ad_{Fbar}^T (J V)
    ad_apply(V, Fb, t2);                 // ad_V Fbar
    sym6_apply(REC_(i) + REC_J, t2, t3);  // J ad_V Fbar
    // ad_{e_1}^T Abar = (-e_1 x n; -e_1 x f) = (0, n_z, -n_y; 0, f_z, -f_y)
    const T qdi = pb.qd[i];
    l[0] = t1[0] - t3[0];
    l[1] = t1[1] - t3[1] - qdi * Ab[2];
    l[2] = t1[2] - t3[2] + qdi * Ab[1];
    l[3] = t1[3] - t3[3];
    l[4] = t1[4] - t3[4] - qdi * Ab[5];
    l[5] = t1[5] - t3[5] + qdi * Ab[4];
  });
  }

  const int g0 = lanes ? tm.r : a, g1 = lanes ? pb.n : b, gs = lanes ? P : 1;
  for (int i = g0; i < g1; i += gs) {
    const T *w = W(i);
    T V[6], Ai[6], F[6], Fb[6], Ab[6], Vb[6];
    ldv<T, 6>(w + J_V, V);
    ldv<T, 6>(w + J_A, Ai);
    ldv<T, 6>(w + J_F, F);
    ldv<T, 6>(w + J_FB, Fb);
    ldv<T, 6>(w + J_AB, Ab);
    ldv<T, 6>(w + J_VB, Vb);
    const T qdi = pb.qd[i];
    // with ad_V e_1 = (0, w_z, -w_y; 0, v_z, -v_y) and ad_{e_1} x = (0, -x_2, x_1;
    // 0, -x_5, x_4), written out without the zero entries:
    // -g_qd = -Vbar_0 - (ad_V e_1) . Abar
    const T m_gqd = (((-Vb[0] - V[2] * Ab[1]) + V[1] * Ab[2]) - V[5] * Ab[4]) + V[4] * Ab[5];
    // u = A - qd ad_V e_1 (components 1, 2, 4, 5; 0 and 3 are A's)
    const T u1 = Ai[1] - qdi * V[2], u2 = Ai[2] + qdi * V[1];
    const T u4 = Ai[4] - qdi * V[5], u5 = Ai[5] + qdi * V[4];
    // g_q = Vbar . ad_{e_1} V + Abar . ad_{e_1} u + (ad_{e_1} Fbar) . F
    T g_q = ((-Vb[1] * V[2] + Vb[2] * V[1]) - Vb[4] * V[5]) + Vb[5] * V[4];
    g_q = (((g_q - Ab[1] * u2) + Ab[2] * u1) - Ab[4] * u5) + Ab[5] * u4;
    g_q = (((g_q - F[1] * Fb[2]) + F[2] * Fb[1]) - F[4] * Fb[5]) + F[5] * Fb[4];
    // x_bar = -(d ID / d x)^T lambda; d ID / d q carries the minus of dX/dq
    qbar[i] = g_q;
    qdbar[i] = m_gqd;
    if (mbar) {
      T JmA[6], JmV[6], adVFb[6];
      dJdm_apply(REC_(i) + REC_J, Ai, JmA);
      dJdm_apply(REC_(i) + REC_J, V, JmV);
      ad_apply(V, Fb, adVFb);
      mbar[i] = -(dot6(Fb, JmA) - dot6(adVFb, JmV));
    }
  }
}

template <class T, int P>
__global__ void __launch_bounds__(block_for<P>()) adjoint_rnea_kernel(KArgs A) {
  adjoint_body<T, P>(A, Range{0, 0, A.n_problems});
}

// One launch over length classes (see the ClassTable kernels of fd_kernels.cuh).
template <class T>
__global__ void __launch_bounds__(128) adjoint_multi_kernel(KArgs A, ClassTable ct) {
  const int c = class_of_block(ct);
  const Range rg{ct.blk[c], ct.first[c], ct.first[c + 1]};
#define FDK_C(PP) \
  case PP: adjoint_body<T, PP>(A, rg); break;
  FDK_CLASS_TEAMS(FDK_C)
#undef FDK_C
}

}  // namespace fdk
