// fd_device.cuh -- device-side building blocks of the forward-dynamics kernels.
//
// Lie-group arithmetic of Section II-A (SE(3), se(3), se(3)*), the team
// primitives used by the segmented scans of Section II-B, and small dense
// symmetric solves (SolvSys of Section IV). Everything is templated on the
// arithmetic type.
//
// Link frames are canonical: the joint axis of link i is the x axis of frame i,
// so S_i = e_1, S_i^T x = x[0] and W_i^T x = x[1..5] (Section III-B).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "fd_layout.h"

namespace fdk {

// ------------------------------------------------------------ math overloads

__device__ __forceinline__ void sincos_t(double x, double *s, double *c) { sincos(x, s, c); }
__device__ __forceinline__ void sincos_t(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
// x > 0 for a pivot, tested on the bit pattern (an integer compare, not an FP64
// one): true for positive numbers and +inf, also for a NaN with a clear sign bit,
// which the kernels' final finiteness check then reports
__device__ __forceinline__ bool pos_t(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool pos_t(float x) { return __float_as_int(x) > 0; }
// -x if f, else x: the sign bit flipped by an integer operation
__device__ __forceinline__ double neg_if(double x, bool f) {
  return __longlong_as_double(static_cast<long long>(
      static_cast<unsigned long long>(__double_as_longlong(x)) ^ (static_cast<unsigned long long>(f) << 63)));
}
__device__ __forceinline__ float neg_if(float x, bool f) {
  return __int_as_float(static_cast<int>(static_cast<unsigned>(__float_as_int(x)) ^
                                         (static_cast<unsigned>(f) << 31)));
}
// 1 / x rounded to nearest (the same value as the IEEE division 1 / x)
__device__ __forceinline__ double rcp_t(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float rcp_t(float x) { return __frcp_rn(x); }

// ------------------------------------------------------------------ indexing

// packed symmetric 6x6, upper triangle row by row (21 entries)
__host__ __device__ constexpr int s6(int i, int j) {
  return i <= j ? i * 6 - (i * (i - 1)) / 2 + (j - i) : j * 6 - (j * (j - 1)) / 2 + (i - j);
}
// packed symmetric / lower-triangular 5x5, lower triangle row by row (15 entries)
__host__ __device__ constexpr int l5(int i, int j) {
  return i >= j ? (i * (i + 1)) / 2 + j : (j * (j + 1)) / 2 + i;
}

// ---------------------------------------------------------------- SE(3) etc.

template <class T>
struct SE3 {
  T R[9];
  T p[3];
};

template <class T>
__device__ __forceinline__ void se3_identity(SE3<T> &g) {
#pragma unroll
  for (int k = 0; k < 9; ++k) g.R[k] = (k % 4 == 0) ? T(1) : T(0);
  g.p[0] = g.p[1] = g.p[2] = T(0);
}

// c = a b  (R_a R_b, R_a p_b + p_a)
template <class T>
__device__ __forceinline__ void se3_mul(const SE3<T> &a, const SE3<T> &b, SE3<T> &c) {
  SE3<T> t;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
      t.R[3 * i + j] = a.R[3 * i] * b.R[j] + a.R[3 * i + 1] * b.R[3 + j] + a.R[3 * i + 2] * b.R[6 + j];
    t.p[i] = a.R[3 * i] * b.p[0] + a.R[3 * i + 1] * b.p[1] + a.R[3 * i + 2] * b.p[2] + a.p[i];
  }
  c = t;
}

template <class T>
__device__ __forceinline__ void cross3(const T *a, const T *b, T *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// y = Ad_{g^{-1}} x: omega' = R^T omega, v' = R^T (v + omega x p)
// (the cross product accumulates onto v in fused multiply-adds)
template <class T>
__device__ __forceinline__ void adinv(const SE3<T> &g, const T *x, T *y) {
  T u[3];
  u[0] = x[3] + x[1] * g.p[2];
  u[0] -= x[2] * g.p[1];
  u[1] = x[4] + x[2] * g.p[0];
  u[1] -= x[0] * g.p[2];
  u[2] = x[5] + x[0] * g.p[1];
  u[2] -= x[1] * g.p[0];
  T o[6];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    o[j] = g.R[j] * x[0] + g.R[3 + j] * x[1] + g.R[6 + j] * x[2];
    o[3 + j] = g.R[j] * u[0] + g.R[3 + j] * u[1] + g.R[6 + j] * u[2];
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) y[k] = o[k];
}

// y = Ad_{g^{-1}}^T x for a wrench x = (n; f): (R n + p x (R f); R f)
template <class T>
__device__ __forceinline__ void adinvT(const SE3<T> &g, const T *x, T *y) {
  T Rn[3], Rf[3], pf[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Rn[i] = g.R[3 * i] * x[0] + g.R[3 * i + 1] * x[1] + g.R[3 * i + 2] * x[2];
    Rf[i] = g.R[3 * i] * x[3] + g.R[3 * i + 1] * x[4] + g.R[3 * i + 2] * x[5];
  }
  // n' = R n + p x (R f), accumulated in fused multiply-adds
  pf[0] = Rn[0] + g.p[1] * Rf[2];
  pf[1] = Rn[1] + g.p[2] * Rf[0];
  pf[2] = Rn[2] + g.p[0] * Rf[1];
  y[0] = pf[0] - g.p[2] * Rf[1];
  y[1] = pf[1] - g.p[0] * Rf[2];
  y[2] = pf[2] - g.p[1] * Rf[0];
  y[3] = Rf[0];
  y[4] = Rf[1];
  y[5] = Rf[2];
}

// y = ad_V x = (w x xw; v x xw + w x xv)
template <class T>
__device__ __forceinline__ void ad_apply(const T *V, const T *x, T *y) {
  T a[3], b[3], c[3];
  cross3(V, x, a);
  cross3(V + 3, x, b);
  cross3(V, x + 3, c);
  y[0] = a[0]; y[1] = a[1]; y[2] = a[2];
  y[3] = b[0] + c[0]; y[4] = b[1] + c[1]; y[5] = b[2] + c[2];
}

// y = ad_V^T x = (-w x n - v x f; -w x f)
template <class T>
__device__ __forceinline__ void adT_apply(const T *V, const T *x, T *y) {
  T a[3], b[3], c[3];
  cross3(V, x, a);
  cross3(V + 3, x + 3, b);
  cross3(V, x + 3, c);
  y[0] = -a[0] - b[0]; y[1] = -a[1] - b[1]; y[2] = -a[2] - b[2];
  y[3] = -c[0]; y[4] = -c[1]; y[5] = -c[2];
}

// y -= ad_V^T x, i.e. y += (w x n + v x f; w x f) for V = (w; v), x = (n; f),
// accumulated in fused multiply-adds (no separate negations)
template <class T>
__device__ __forceinline__ void adT_sub(const T *V, const T *x, T *y) {
  const T *w = V, *v = V + 3, *n = x, *f = x + 3;
  y[0] = (((y[0] + w[1] * n[2]) - w[2] * n[1]) + v[1] * f[2]) - v[2] * f[1];
  y[1] = (((y[1] + w[2] * n[0]) - w[0] * n[2]) + v[2] * f[0]) - v[0] * f[2];
  y[2] = (((y[2] + w[0] * n[1]) - w[1] * n[0]) + v[0] * f[1]) - v[1] * f[0];
  y[3] = (y[3] + w[1] * f[2]) - w[2] * f[1];
  y[4] = (y[4] + w[2] * f[0]) - w[0] * f[2];
  y[5] = (y[5] + w[0] * f[1]) - w[1] * f[0];
}

// y = K x, K packed symmetric 6x6
template <class T, class TK>
__device__ __forceinline__ void sym6_apply(const TK *K, const T *x, T *y) {
  T o[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    T s = T(0);
#pragma unroll
    for (int j = 0; j < 6; ++j) s += T(K[s6(i, j)]) * x[j];
    o[i] = s;
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) y[i] = o[i];
}

// y += K x, K packed symmetric 6x6 (accumulates in fused multiply-adds)
template <class T, class TK>
__device__ __forceinline__ void sym6_apply_add(const TK *K, const T *x, T *y) {
  T o[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    T s = y[i];
#pragma unroll
    for (int j = 0; j < 6; ++j) s += T(K[s6(i, j)]) * x[j];
    o[i] = s;
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) y[i] = o[i];
}

// joint transform in canonical frames: g = (R0 Rot_x(q), p0)
template <class T>
__device__ __forceinline__ void joint_transform(const T *rec, T q, SE3<T> &g) {
  T s, c;
  sincos_t(q, &s, &c);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T r0 = rec[REC_R0 + 3 * i], r1 = rec[REC_R0 + 3 * i + 1], r2 = rec[REC_R0 + 3 * i + 2];
    g.R[3 * i] = r0;
    g.R[3 * i + 1] = c * r1 + s * r2;
    g.R[3 * i + 2] = -s * r1 + c * r2;
    g.p[i] = rec[REC_P0 + i];
  }
}

// ------------------------------------------------------------ load / store

// (converting when the stored type S differs from the arithmetic type T)
template <class S, class T>
__device__ __forceinline__ void ld_se3(const S *src, SE3<T> &g) {
#pragma unroll
  for (int k = 0; k < 9; ++k) g.R[k] = T(src[k]);
#pragma unroll
  for (int k = 0; k < 3; ++k) g.p[k] = T(src[9 + k]);
}
template <class T>
__device__ __forceinline__ void st_se3(T *dst, const SE3<T> &g) {
#pragma unroll
  for (int k = 0; k < 9; ++k) dst[k] = g.R[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) dst[9 + k] = g.p[k];
}
template <class T, int N>
__device__ __forceinline__ void ldv(const T *src, T *x) {
#pragma unroll
  for (int k = 0; k < N; ++k) x[k] = src[k];
}
template <class T, int N>
__device__ __forceinline__ void stv(T *dst, const T *x) {
#pragma unroll
  for (int k = 0; k < N; ++k) dst[k] = x[k];
}

// --------------------------------------------------------------------- teams

// Threads per block for a team of P lanes: teams of up to 128 lanes share
// 128-thread blocks; larger teams are one block each.
template <int P>
__host__ __device__ constexpr int block_for() {
  return P > 128 ? P : 128;
}

// P lanes cooperate on one problem (P a power of two, 1..256). P <= 32: a
// sub-warp, synchronised with __syncwarp and combined with shuffles. P > 32:
// whole warps of one block, synchronised with a named barrier per team and
// combined through shared memory.
template <int P>
struct Team {
  unsigned mask;
  int r;    // lane within the team
  int bar;  // named barrier of the team (P > 32)
  __device__ __forceinline__ Team() {
    const int lane = threadIdx.x & 31;
    if constexpr (P < 32) {
      r = lane & (P - 1);
      mask = ((1u << P) - 1u) << (lane & ~(P - 1));
    } else if constexpr (P == 32) {
      r = lane;
      mask = 0xffffffffu;
    } else {
      r = threadIdx.x & (P - 1);
      mask = 0xffffffffu;
    }
    bar = 1 + static_cast<int>(threadIdx.x) / (P > 32 ? P : 32);
  }
  __device__ __forceinline__ void sync() const {
    if (P > 32) {
      asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(P) : "memory");
    } else if (P > 1) {
      __syncwarp(mask);
    }
  }
  // true on every lane if `b` is true on any lane of the team
  __device__ __forceinline__ bool any(bool b) const {
    if (P > 32) {
      unsigned out;
      asm volatile(
          "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
          "bar.red.or.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
          : "=r"(out)
          : "r"(static_cast<unsigned>(b)), "r"(bar), "r"(P)
          : "memory");
      return out != 0;
    } else if (P > 1) {
      return __any_sync(mask, b);
    }
    return b;
  }
  // shuffles within the warp part of the team (width min(P, 32))
  template <class V>
  __device__ __forceinline__ V up(V v, int d) const {
    return __shfl_up_sync(mask, v, d, P < 32 ? P : 32);
  }
  template <class V>
  __device__ __forceinline__ V down(V v, int d) const {
    return __shfl_down_sync(mask, v, d, P < 32 ? P : 32);
  }
};

// Operator of one lane's segment of a bi-diagonal recursion with the SE(3)
// transports of the chain: forward  x -> Ad_{h^{-1}} x + psi,
//                          backward y -> Ad_{h^{-1}}^T y + psi.
template <class T>
struct SegOp {
  SE3<T> h;
  T psi[6];
};

template <class T>
__device__ __forceinline__ void segop_identity(SegOp<T> &o) {
  se3_identity(o.h);
#pragma unroll
  for (int k = 0; k < 6; ++k) o.psi[k] = T(0);
}

// forward composition: earlier `e`, then later `l`  ->  l (+) e  (into out)
template <class T>
__device__ __forceinline__ void compose_fwd(const SegOp<T> &e, const SegOp<T> &l, SegOp<T> &out) {
  T t[6];
  adinv(l.h, e.psi, t);
  SegOp<T> o;
#pragma unroll
  for (int k = 0; k < 6; ++k) o.psi[k] = t[k] + l.psi[k];
  se3_mul(e.h, l.h, o.h);
  out = o;
}

// backward composition (applied right to left): `m` then the later `l`
template <class T>
__device__ __forceinline__ void compose_bwd(const SegOp<T> &m, const SegOp<T> &l, SegOp<T> &out) {
  T t[6];
  adinvT(m.h, l.psi, t);
  SegOp<T> o;
#pragma unroll
  for (int k = 0; k < 6; ++k) o.psi[k] = t[k] + m.psi[k];
  se3_mul(m.h, l.h, o.h);
  out = o;
}

template <int P, class T>
__device__ __forceinline__ void shfl_op(const Team<P> &tm, const SegOp<T> &a, SegOp<T> &b, int d,
                                        bool up) {
#pragma unroll
  for (int k = 0; k < 9; ++k) b.h.R[k] = up ? tm.up(a.h.R[k], d) : tm.down(a.h.R[k], d);
#pragma unroll
  for (int k = 0; k < 3; ++k) b.h.p[k] = up ? tm.up(a.h.p[k], d) : tm.down(a.h.p[k], d);
#pragma unroll
  for (int k = 0; k < 6; ++k) b.psi[k] = up ? tm.up(a.psi[k], d) : tm.down(a.psi[k], d);
}

// shared-memory slots for the warp aggregates of multi-warp teams
template <class T>
__device__ __forceinline__ SegOp<T> *warp_slots() {
  __shared__ __align__(16) unsigned char raw[32 * sizeof(SegOp<double>)];
  return reinterpret_cast<SegOp<T> *>(raw);
}

// Exclusive forward scan over the team's segments (Section II-B: the operator
// a_{i-1} (+) a_i = a_i a_{i-1}; Kogge-Stone across the lanes of a warp, then
// across the warps of a team). Returns the value entering this lane's segment,
// given x_base entering lane 0.
template <int P, class T>
__device__ __forceinline__ void team_scan_fwd(const Team<P> &tm, SegOp<T> op, const T *x_base,
                                              T *x_in) {
  if constexpr (P == 1) {
#pragma unroll
    for (int k = 0; k < 6; ++k) x_in[k] = x_base[k];
    return;
  } else {
    constexpr int WP = P < 32 ? P : 32;
    const int wl = tm.r & (WP - 1);  // lane within the warp part
#pragma unroll
    for (int d = 1; d < WP; d <<= 1) {
      SegOp<T> o;
      shfl_op(tm, op, o, d, true);
      if (wl >= d) compose_fwd(o, op, op);
    }
    SegOp<T> ex;
    shfl_op(tm, op, ex, 1, true);
    if (wl == 0) segop_identity(ex);
    if constexpr (P > 32) {
      SegOp<T> *slot = warp_slots<T>();
      const int w = static_cast<int>(threadIdx.x) >> 5;  // warp in block
      const int w0 = w - (tm.r >> 5);                      // first warp of the team
      if (wl == 31) slot[w] = op;
      tm.sync();
      SegOp<T> pre;
      segop_identity(pre);
      for (int k = w0; k < w; ++k) compose_fwd(pre, slot[k], pre);
      tm.sync();
      compose_fwd(pre, ex, ex);
    }
    adinv(ex.h, x_base, x_in);
#pragma unroll
    for (int k = 0; k < 6; ++k) x_in[k] += ex.psi[k];
  }
}

// Exclusive backward scan (transposed system, from the tip): returns the value
// entering this lane's segment from the right; nothing enters the last lane.
template <int P, class T>
__device__ __forceinline__ void team_scan_bwd(const Team<P> &tm, SegOp<T> op, T *y_in) {
#pragma unroll
  for (int k = 0; k < 6; ++k) y_in[k] = T(0);
  if constexpr (P > 1) {
    constexpr int WP = P < 32 ? P : 32;
    const int wl = tm.r & (WP - 1);
#pragma unroll
    for (int d = 1; d < WP; d <<= 1) {
      SegOp<T> o;
      shfl_op(tm, op, o, d, false);
      if (wl + d < WP) compose_bwd(op, o, op);
    }
    SegOp<T> ex;
    shfl_op(tm, op, ex, 1, false);
    if (wl == WP - 1) segop_identity(ex);
    if constexpr (P > 32) {
      SegOp<T> *slot = warp_slots<T>();
      const int w = static_cast<int>(threadIdx.x) >> 5;
      const int wend = w - (tm.r >> 5) + P / 32;  // one past the team's last warp
      if (wl == 0) slot[w] = op;
      tm.sync();
      SegOp<T> post;
      segop_identity(post);
      for (int k = wend - 1; k > w; --k) compose_bwd(slot[k], post, post);
      tm.sync();
      compose_bwd(ex, post, ex);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) y_in[k] = ex.psi[k];
  }
}

// ------------------------------------------------------------- 5x5 SolvSys

// Cholesky D = L L^T of a packed symmetric 5x5 (lower triangle). Writes the
// strict lower triangle of L, the reciprocals of its diagonal into inv and (the
// same reciprocals) into L's diagonal slots. Returns false if a pivot is not
// positive.
template <class T>
__device__ __forceinline__ bool chol5(const T *D, T *L, T *inv) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    T d = D[l5(j, j)];
#pragma unroll
    for (int k = 0; k < j; ++k) d -= L[l5(j, k)] * L[l5(j, k)];
    ok = ok && pos_t(d);
    const T r = rsqrt_t(d);  // inf or NaN for a non-positive pivot, flagged by ok
    L[l5(j, j)] = r;  // the diagonal sqrt(d) itself is never read: the solves take 1 / L_jj
    inv[j] = r;
#pragma unroll
    for (int i = j + 1; i < 5; ++i) {
      T s = D[l5(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) s -= L[l5(i, k)] * L[l5(j, k)];
      L[l5(i, j)] = s * r;
    }
  }
  return ok;
}

// x <- L^{-1} x
template <class T>
__device__ __forceinline__ void fwd5(const T *L, const T *inv, T *x) {
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    T s = x[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s -= L[l5(i, k)] * x[k];
    x[i] = s * inv[i];
  }
}

// x <- L^{-T} x
template <class T>
__device__ __forceinline__ void bwd5(const T *L, const T *inv, T *x) {
#pragma unroll
  for (int i = 4; i >= 0; --i) {
    T s = x[i];
#pragma unroll
    for (int k = i + 1; k < 5; ++k) s -= L[l5(k, i)] * x[k];
    x[i] = s * inv[i];
  }
}

// ---------------------------------------------------------------- status

__device__ __forceinline__ void set_status(int32_t *status, int p, int32_t code) {
  if (status) status[p] = code;
}

template <class T>
__device__ __forceinline__ bool finite_t(T x) {
  return isfinite(x);
}

}  // namespace fdk
