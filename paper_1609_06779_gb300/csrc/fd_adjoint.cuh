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

// ad_{e_1} x = (e_1 x w; e_1 x v)
template <class T>
__device__ __forceinline__ void ad_e1(const T *x, T *y) {
  y[0] = T(0); y[1] = -x[2]; y[2] = x[1];
  y[3] = T(0); y[4] = -x[5]; y[5] = x[4];
}

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

template <class T, int P>
__global__ void __launch_bounds__(block_for<P>()) adjoint_rnea_kernel(KArgs A) {
  Team<P> tm;
  Prob<T> pb;
  if (!load_problem<T, P>(A, tm, pb, NT_ADJ)) return;
  const int a = pb.a, b = pb.b;
  const int64_t s0 = A.state_off[pb.p];
  const T *lam = static_cast<const T *>(A.lam) + s0;
  T *qbar = static_cast<T *>(A.out) + s0;
  T *qdbar = static_cast<T *>(A.out2) + s0;
  T *mbar = A.out3 ? static_cast<T *>(A.out3) + s0 : nullptr;
  auto W = [&](int i) { return pb.wt + static_cast<int64_t>(i) * NT_ADJ; };
  auto REC_ = [&](int i) { return pb.rec + static_cast<int64_t>(i) * REC; };

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
    adT_apply(V, JV, c);
    for (int k = 0; k < 6; ++k) JA[k] -= c[k];
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

  for (int i = a; i < b; ++i) {
    const T *w = W(i);
    T V[6], Ai[6], F[6], Fb[6], Ab[6], Vb[6];
    ldv<T, 6>(w + J_V, V);
    ldv<T, 6>(w + J_A, Ai);
    ldv<T, 6>(w + J_F, F);
    ldv<T, 6>(w + J_FB, Fb);
    ldv<T, 6>(w + J_AB, Ab);
    ldv<T, 6>(w + J_VB, Vb);
    const T qdi = pb.qd[i];
    // ad_V e_1 = (0, w_z, -w_y; 0, v_z, -v_y)
    const T adVe1[6] = {T(0), V[2], -V[1], T(0), V[5], -V[4]};
    const T g_qd = Vb[0] + dot6(adVe1, Ab);
    T t[6], u[6];
    ad_e1(V, t);
    T g_q = dot6(Vb, t);
    for (int k = 0; k < 6; ++k) u[k] = Ai[k] - qdi * adVe1[k];
    ad_e1(u, t);
    g_q += dot6(Ab, t);
    ad_e1(Fb, t);
    g_q += dot6(t, F);
    // x_bar = -(d ID / d x)^T lambda; d ID / d q carries the minus of dX/dq
    qbar[i] = g_q;
    qdbar[i] = -g_qd;
    if (mbar) {
      T JmA[6], JmV[6], adVFb[6];
      dJdm_apply(REC_(i) + REC_J, Ai, JmA);
      dJdm_apply(REC_(i) + REC_J, V, JmV);
      ad_apply(V, Fb, adVFb);
      mbar[i] = -(dot6(Fb, JmA) - dot6(adVFb, JmV));
    }
  }
}

}  // namespace fdk
