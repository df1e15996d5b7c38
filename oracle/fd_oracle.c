/*
 * fd_oracle.c -- plain, slow, FP64 CPU oracle for forward dynamics of serial
 * chains of revolute joints (Yang, Wu & Pan, "A Novel GPU-based Parallel
 * Implementation Scheme and Performance Analysis of Robot Forward Dynamics
 * Algorithms", arXiv 1609.06779).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library. It shares no code with the CUDA path.
 *
 * Everything is dense 6x6 linear algebra in the links' own frames, written so
 * that it can be checked against the paper by eye:
 *   - rnea_chain       Eq. 2a-2d (recursive Newton-Euler; gives the bias torque
 *                      of Eq. 4 with qdd = 0)
 *   - mass_matrix      Section II-C, JSIIA: column k of M(q) is the inverse
 *                      dynamics with qdd = e_k, qdot = 0 and no gravity
 *   - fd_cholesky      Eq. 4: qdd = M(q)^{-1} (tau - tau_bias), M by columns and
 *                      a dense Cholesky factorisation (the plain definition)
 *   - fd_aba           Section II-C, ABIA: articulated-body inertia recursion
 *                      (the standard form the paper cites), direct and serial
 *   - fd_cfa           Section III, Algorithm 1: A, B, C of Eq. cfa-eq2 and
 *                      Eq. fijany-final, the block tri-diagonal solve by odd-even
 *                      elimination (Section IV, Algorithm 2), then CalcAcc
 *
 * Conventions (the readings taken where the paper is silent or inconsistent):
 *   twist V = (omega; v), wrench F = (n; f);
 *   Ad_g = [[R, 0], [p^ R, R]] for g = (R, p); ad_V = [[w^, 0], [v^, w^]];
 *   joint i: g_{i-1,i}(q) = (R0_i, p0_i) * exp([a_i; 0] q), S_i = (a_i; 0);
 *   X_i := Ad_{g_{i-1,i}^{-1}} (the blocks of Gamma);
 *   V_i   = X_i V_{i-1} + S_i qd_i,                       V_0 = 0
 *   Vd_i  = X_i Vd_{i-1} + S_i qdd_i + ad_{V_i} S_i qd_i,  Vd_0 = (0; -g)
 *   F_i   = X_{i+1}^T F_{i+1} + J_i Vd_i - ad_{V_i}^T J_i V_i,  F_{n+1} = 0
 *   tau_i = S_i^T F_i.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_NOT_SPD 2
#define ORC_ERR_ARG 1

/* ------------------------------------------------------------------ small dense */

static void m3_mul(const double *A, const double *B, double *C) {
  double T[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
      T[3 * i + j] = s;
    }
  memcpy(C, T, sizeof T);
}

static void m3_transpose(const double *A, double *B) {
  double T[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) T[3 * j + i] = A[3 * i + j];
  memcpy(B, T, sizeof T);
}

static void m3_vec(const double *A, const double *x, double *y) {
  double t[3];
  for (int i = 0; i < 3; ++i) t[i] = A[3 * i] * x[0] + A[3 * i + 1] * x[1] + A[3 * i + 2] * x[2];
  memcpy(y, t, sizeof t);
}

static void skew3(const double *v, double *S) {
  S[0] = 0.0;   S[1] = -v[2]; S[2] = v[1];
  S[3] = v[2];  S[4] = 0.0;   S[5] = -v[0];
  S[6] = -v[1]; S[7] = v[0];  S[8] = 0.0;
}

/* general dense n x n (row-major) helpers */
static void mat_mul(int r, int k, int c, const double *A, const double *B, double *C) {
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < c; ++j) {
      double s = 0.0;
      for (int t = 0; t < k; ++t) s += A[i * k + t] * B[t * c + j];
      C[i * c + j] = s;
    }
}

static void mat_transpose(int r, int c, const double *A, double *B) {
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < c; ++j) B[j * r + i] = A[i * c + j];
}

static void mat_vec(int r, int c, const double *A, const double *x, double *y) {
  for (int i = 0; i < r; ++i) {
    double s = 0.0;
    for (int j = 0; j < c; ++j) s += A[i * c + j] * x[j];
    y[i] = s;
  }
}

static void mat_tvec(int r, int c, const double *A, const double *x, double *y) {
  for (int j = 0; j < c; ++j) {
    double s = 0.0;
    for (int i = 0; i < r; ++i) s += A[i * c + j] * x[i];
    y[j] = s;
  }
}

/* Cholesky A = L L^T of a dense SPD matrix (L lower, row-major, upper part 0). */
static int cholesky(int n, const double *A, double *L) {
  memset(L, 0, sizeof(double) * (size_t)n * (size_t)n);
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
    if (!(d > 0.0)) return ORC_ERR_NOT_SPD;
    double ljj = sqrt(d);
    L[j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double s = A[i * n + j];
      for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = s / ljj;
    }
  }
  return ORC_OK;
}

/* Solve L L^T x = b given the Cholesky factor. */
static void chol_solve(int n, const double *L, const double *b, double *x) {
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i * n + k] * x[k];
    x[i] = s / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
    x[i] = s / L[i * n + i];
  }
}

/* SolvSys of Section IV: X with D X = Bm, D SPD (n x n), Bm n x m, by Cholesky. */
static int solv_sys(int n, int m, const double *D, const double *Bm, double *X) {
  double L[64], col[8], sol[8];
  if (n > 8) return ORC_ERR_ARG;
  int st = cholesky(n, D, L);
  if (st) return st;
  for (int j = 0; j < m; ++j) {
    for (int i = 0; i < n; ++i) col[i] = Bm[i * m + j];
    chol_solve(n, L, col, sol);
    for (int i = 0; i < n; ++i) X[i * m + j] = sol[i];
  }
  return ORC_OK;
}

/* --------------------------------------------------------------- Lie group */

/* Rodrigues: rotation by angle q about the unit axis a. */
static void rot_axis(const double *a, double q, double *R) {
  double K[9], K2[9];
  skew3(a, K);
  m3_mul(K, K, K2);
  double s = sin(q), c = 1.0 - cos(q);
  for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0 ? 1.0 : 0.0) + s * K[i] + c * K2[i];
}

/* g_{i-1,i}(q) = (R0, p0) exp([a; 0] q) = (R0 Rot(a, q), p0). */
static void joint_transform(const double *frame, const double *axis, double q,
                            double *R, double *p) {
  double Rq[9];
  rot_axis(axis, q, Rq);
  m3_mul(frame, Rq, R);
  p[0] = frame[9]; p[1] = frame[10]; p[2] = frame[11];
}

/* Ad_g = [[R, 0], [p^ R, R]] as a dense 6x6 matrix. */
static void adjoint(const double *R, const double *p, double *A) {
  double P[9], PR[9];
  skew3(p, P);
  m3_mul(P, R, PR);
  memset(A, 0, 36 * sizeof(double));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      A[6 * i + j] = R[3 * i + j];
      A[6 * (i + 3) + j + 3] = R[3 * i + j];
      A[6 * (i + 3) + j] = PR[3 * i + j];
    }
}

/* X = Ad_{g^{-1}}: g^{-1} = (R^T, -R^T p). */
static void adjoint_inv(const double *R, const double *p, double *X) {
  double Rt[9], q[3];
  m3_transpose(R, Rt);
  m3_vec(Rt, p, q);
  q[0] = -q[0]; q[1] = -q[1]; q[2] = -q[2];
  adjoint(Rt, q, X);
}

/* ad_V = [[w^, 0], [v^, w^]]. */
static void ad_matrix(const double *V, double *A) {
  double W[9], U[9];
  skew3(V, W);
  skew3(V + 3, U);
  memset(A, 0, 36 * sizeof(double));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      A[6 * i + j] = W[3 * i + j];
      A[6 * (i + 3) + j + 3] = W[3 * i + j];
      A[6 * (i + 3) + j] = U[3 * i + j];
    }
}

static void joint_twist(const double *axis, double *S) {
  S[0] = axis[0]; S[1] = axis[1]; S[2] = axis[2];
  S[3] = 0.0; S[4] = 0.0; S[5] = 0.0;
}

/* ------------------------------------------------------ inverse dynamics (ID) */

/* Eq. 2a-2d solved by forward and backward substitution of the bi-diagonal
 * systems (I - Gamma) V = S qd + const, (I - Gamma) Vd = S qdd + ad term + const,
 * (I - Gamma)^T F = J Vd - ad^T J V, tau = S^T F.
 * gravity: base acceleration Vd_0 = (0; -g). qd or qdd may be NULL (= 0). */
static int rnea_chain(int n, const double *axes, const double *frames, const double *J,
                      const double *grav, const double *q, const double *qd,
                      const double *qdd, double *tau) {
  double *X = malloc(sizeof(double) * 36 * (size_t)n);
  double *V = malloc(sizeof(double) * 6 * (size_t)n);
  double *Vd = malloc(sizeof(double) * 6 * (size_t)n);
  double *F = malloc(sizeof(double) * 6 * (size_t)n);
  if (!X || !V || !Vd || !F) { free(X); free(V); free(Vd); free(F); return ORC_ERR_ARG; }
  double Vprev[6] = {0, 0, 0, 0, 0, 0};
  double Vdprev[6] = {0, 0, 0, -grav[0], -grav[1], -grav[2]};
  for (int i = 0; i < n; ++i) {
    double R[9], p[3], S[6], ad[36], t[6], u[6];
    joint_transform(frames + 12 * i, axes + 3 * i, q[i], R, p);
    adjoint_inv(R, p, X + 36 * i);
    joint_twist(axes + 3 * i, S);
    double qdi = qd ? qd[i] : 0.0, qddi = qdd ? qdd[i] : 0.0;
    mat_vec(6, 6, X + 36 * i, Vprev, t);
    for (int k = 0; k < 6; ++k) V[6 * i + k] = t[k] + S[k] * qdi;
    ad_matrix(V + 6 * i, ad);
    mat_vec(6, 6, ad, S, u);
    mat_vec(6, 6, X + 36 * i, Vdprev, t);
    for (int k = 0; k < 6; ++k) Vd[6 * i + k] = t[k] + S[k] * qddi + u[k] * qdi;
    memcpy(Vprev, V + 6 * i, sizeof Vprev);
    memcpy(Vdprev, Vd + 6 * i, sizeof Vdprev);
  }
  double Fnext[6] = {0, 0, 0, 0, 0, 0};
  for (int i = n - 1; i >= 0; --i) {
    double a[6], b[6], JV[6], ad[36], c[6];
    const double *Ji = J + 36 * i;
    if (i + 1 < n) mat_tvec(6, 6, X + 36 * (i + 1), Fnext, a);
    else memset(a, 0, sizeof a);
    mat_vec(6, 6, Ji, Vd + 6 * i, b);
    mat_vec(6, 6, Ji, V + 6 * i, JV);
    ad_matrix(V + 6 * i, ad);
    mat_tvec(6, 6, ad, JV, c);
    for (int k = 0; k < 6; ++k) F[6 * i + k] = a[k] + b[k] - c[k];
    memcpy(Fnext, F + 6 * i, sizeof Fnext);
    double S[6];
    joint_twist(axes + 3 * i, S);
    tau[i] = 0.0;
    for (int k = 0; k < 6; ++k) tau[i] += S[k] * F[6 * i + k];
  }
  free(X); free(V); free(Vd); free(F);
  return ORC_OK;
}

/* Section II-C (JSIIA): column k of M(q) = ID(q, qdot = 0, qdd = e_k), no gravity. */
static int mass_matrix_chain(int n, const double *axes, const double *frames,
                             const double *J, const double *q, double *M) {
  double zero_g[3] = {0, 0, 0};
  double *e = calloc((size_t)n, sizeof(double));
  double *col = malloc(sizeof(double) * (size_t)n);
  if (!e || !col) { free(e); free(col); return ORC_ERR_ARG; }
  for (int k = 0; k < n; ++k) {
    e[k] = 1.0;
    rnea_chain(n, axes, frames, J, zero_g, q, NULL, e, col);
    e[k] = 0.0;
    for (int i = 0; i < n; ++i) M[i * n + k] = col[i];
  }
  free(e); free(col);
  return ORC_OK;
}

/* Eq. 4: qdd = M^{-1} (tau - tau_bias), tau_bias = ID(q, qd, 0) with gravity. */
static int fd_cholesky_chain(int n, const double *axes, const double *frames,
                             const double *J, const double *grav, const double *q,
                             const double *qd, const double *tau, double *qdd) {
  double *bias = malloc(sizeof(double) * (size_t)n);
  double *M = malloc(sizeof(double) * (size_t)n * (size_t)n);
  double *L = malloc(sizeof(double) * (size_t)n * (size_t)n);
  if (!bias || !M || !L) { free(bias); free(M); free(L); return ORC_ERR_ARG; }
  rnea_chain(n, axes, frames, J, grav, q, qd, NULL, bias);
  for (int i = 0; i < n; ++i) bias[i] = tau[i] - bias[i];
  mass_matrix_chain(n, axes, frames, J, q, M);
  int st = cholesky(n, M, L);
  if (st == ORC_OK) chol_solve(n, L, bias, qdd);
  free(bias); free(M); free(L);
  return st;
}

/* ----------------------------------------------------------------- ABIA */

/* Articulated-body algorithm (Section II-C; the ABI recursion the paper cites):
 * outward V_i, c_i = ad_{V_i} S_i qd_i, bias wrench p_i = -ad_{V_i}^T J_i V_i;
 * inward  D_i = S^T P_i S, u_i = tau_i - S^T p_i,
 *         Pa = P_i - P_i S D^-1 S^T P_i, pa = p_i + Pa c_i + P_i S D^-1 u_i,
 *         P_{i-1} += X_i^T Pa X_i, p_{i-1} += X_i^T pa;
 * outward a' = X_i a_{i-1} + c_i, qdd_i = D^-1 (u_i - S^T P_i a'), a_i = a' + S qdd_i,
 *         a_0 = (0; -g). */
static int fd_aba_chain(int n, const double *axes, const double *frames, const double *J,
                        const double *grav, const double *q, const double *qd,
                        const double *tau, double *qdd) {
  size_t N = (size_t)n;
  double *X = malloc(sizeof(double) * 36 * N), *S = malloc(sizeof(double) * 6 * N);
  double *c = malloc(sizeof(double) * 6 * N), *P = malloc(sizeof(double) * 36 * N);
  double *pb = malloc(sizeof(double) * 6 * N), *h = malloc(sizeof(double) * 6 * N);
  double *D = malloc(sizeof(double) * N), *u = malloc(sizeof(double) * N);
  if (!X || !S || !c || !P || !pb || !h || !D || !u) {
    free(X); free(S); free(c); free(P); free(pb); free(h); free(D); free(u);
    return ORC_ERR_ARG;
  }
  double Vprev[6] = {0, 0, 0, 0, 0, 0};
  for (int i = 0; i < n; ++i) {
    double R[9], p[3], t[6], V[6], ad[36], JV[6];
    joint_transform(frames + 12 * i, axes + 3 * i, q[i], R, p);
    adjoint_inv(R, p, X + 36 * i);
    joint_twist(axes + 3 * i, S + 6 * i);
    mat_vec(6, 6, X + 36 * i, Vprev, t);
    for (int k = 0; k < 6; ++k) V[k] = t[k] + S[6 * i + k] * qd[i];
    ad_matrix(V, ad);
    mat_vec(6, 6, ad, S + 6 * i, c + 6 * i);
    for (int k = 0; k < 6; ++k) c[6 * i + k] *= qd[i];
    mat_vec(6, 6, J + 36 * i, V, JV);
    mat_tvec(6, 6, ad, JV, pb + 6 * i);
    for (int k = 0; k < 6; ++k) pb[6 * i + k] = -pb[6 * i + k];
    memcpy(P + 36 * i, J + 36 * i, 36 * sizeof(double));
    memcpy(Vprev, V, sizeof V);
  }
  int st = ORC_OK;
  for (int i = n - 1; i >= 0; --i) {
    double *Pi = P + 36 * i, *Si = S + 6 * i, *hi = h + 6 * i;
    mat_vec(6, 6, Pi, Si, hi);
    double d = 0.0, sp = 0.0;
    for (int k = 0; k < 6; ++k) { d += Si[k] * hi[k]; sp += Si[k] * pb[6 * i + k]; }
    if (!(d > 0.0)) { st = ORC_ERR_NOT_SPD; break; }
    D[i] = d;
    u[i] = tau[i] - sp;
    if (i == 0) break;
    double Pa[36], pa[6], Pc[6], T1[36], T2[36], Xt[36], pt[6];
    for (int r = 0; r < 6; ++r)
      for (int k = 0; k < 6; ++k) Pa[6 * r + k] = Pi[6 * r + k] - hi[r] * hi[k] / d;
    mat_vec(6, 6, Pa, c + 6 * i, Pc);
    for (int k = 0; k < 6; ++k) pa[k] = pb[6 * i + k] + Pc[k] + hi[k] * u[i] / d;
    mat_transpose(6, 6, X + 36 * i, Xt);
    mat_mul(6, 6, 6, Xt, Pa, T1);
    mat_mul(6, 6, 6, T1, X + 36 * i, T2);
    for (int k = 0; k < 36; ++k) P[36 * (i - 1) + k] += T2[k];
    mat_tvec(6, 6, X + 36 * i, pa, pt);
    for (int k = 0; k < 6; ++k) pb[6 * (i - 1) + k] += pt[k];
  }
  if (st == ORC_OK) {
    double a[6] = {0, 0, 0, -grav[0], -grav[1], -grav[2]};
    for (int i = 0; i < n; ++i) {
      double ap[6];
      mat_vec(6, 6, X + 36 * i, a, ap);
      double s = 0.0;
      for (int k = 0; k < 6; ++k) { ap[k] += c[6 * i + k]; s += h[6 * i + k] * ap[k]; }
      qdd[i] = (u[i] - s) / D[i];
      for (int k = 0; k < 6; ++k) a[k] = ap[k] + S[6 * i + k] * qdd[i];
    }
  }
  free(X); free(S); free(c); free(P); free(pb); free(h); free(D); free(u);
  return st;
}

/* ------------------------------------------------------------------ CFA */

/* W_i (6x5, row-major): columns (b;0), (c;0), (0;e1), (0;e2), (0;e3) with b, c an
 * orthonormal basis of the plane orthogonal to the joint axis, so W_i^T S_i = 0
 * (Section III-A: the projection that eliminates qdd). */
static void projection_w(const double *axis, double *W) {
  double a[3] = {axis[0], axis[1], axis[2]};
  /* start from the coordinate axis least aligned with a */
  int m = 0;
  if (fabs(a[1]) < fabs(a[m])) m = 1;
  if (fabs(a[2]) < fabs(a[m])) m = 2;
  double e[3] = {0, 0, 0};
  e[m] = 1.0;
  double d = e[0] * a[0] + e[1] * a[1] + e[2] * a[2];
  double b[3] = {e[0] - d * a[0], e[1] - d * a[1], e[2] - d * a[2]};
  double nb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
  b[0] /= nb; b[1] /= nb; b[2] /= nb;
  double c[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
  memset(W, 0, 30 * sizeof(double));
  for (int r = 0; r < 3; ++r) {
    W[5 * r + 0] = b[r];
    W[5 * r + 1] = c[r];
    W[5 * (r + 3) + 2 + r] = 1.0;
  }
}

/* Inverse of a 6x6 SPD matrix by Cholesky solves of the identity columns. */
static int spd_inverse6(const double *A, double *Ai) {
  double L[36], e[6], x[6];
  int st = cholesky(6, A, L);
  if (st) return st;
  for (int j = 0; j < 6; ++j) {
    memset(e, 0, sizeof e);
    e[j] = 1.0;
    chol_solve(6, L, e, x);
    for (int i = 0; i < 6; ++i) Ai[6 * i + j] = x[i];
  }
  return ORC_OK;
}

/* CalcA, CalcB, CalcC of Algorithm 1 with T = (I - Gamma) J^-1 (I - Gamma)^T:
 *   T_ii = J_i^-1 + X_i J_{i-1}^-1 X_i^T, T_{i,i+1} = -J_i^-1 X_{i+1}^T,
 *   T_{i,i-1} = -X_i J_{i-1}^-1;
 *   A = W^T T W (Eq. cfa-eq2): D_i = W_i^T T_ii W_i, U_i = W_i^T T_{i,i+1} W_{i+1};
 *   B = W^T T S (Eq. cfa-eq2): Bb[i][0..2] = W_i^T T_{i,j} S_j for j = i-1, i, i+1;
 *   C = S^T T S (Eq. fijany-final): Cd[i] = S_i^T T_ii S_i,
 *                                   Co[i] = S_i^T T_{i,i+1} S_{i+1}.
 * Outputs: D [n][25], U [n][25] (U[n-1] = 0), Bb [n][3][5], Cd [n], Co [n],
 * W [n][30] (may be NULL). If Win is not NULL it supplies the W_i to use. */
static int cfa_blocks(int n, const double *axes, const double *frames, const double *J,
                      const double *q, const double *Win, double *D, double *U,
                      double *Bb, double *Cd, double *Co, double *Wout) {
  size_t N = (size_t)n;
  double *X = malloc(sizeof(double) * 36 * N), *Ji = malloc(sizeof(double) * 36 * N);
  double *W = malloc(sizeof(double) * 30 * N), *S = malloc(sizeof(double) * 6 * N);
  if (!X || !Ji || !W || !S) { free(X); free(Ji); free(W); free(S); return ORC_ERR_ARG; }
  int st = ORC_OK;
  for (int i = 0; i < n && st == ORC_OK; ++i) {
    double R[9], p[3];
    joint_transform(frames + 12 * i, axes + 3 * i, q[i], R, p);
    adjoint_inv(R, p, X + 36 * i);
    joint_twist(axes + 3 * i, S + 6 * i);
    st = spd_inverse6(J + 36 * i, Ji + 36 * i);
    if (Win) memcpy(W + 30 * i, Win + 30 * i, 30 * sizeof(double));
    else projection_w(axes + 3 * i, W + 30 * i);
  }
  for (int i = 0; i < n && st == ORC_OK; ++i) {
    double Tii[36], Tup[36], Tlo[36], Xt[36], t1[36], t2[36];
    memcpy(Tii, Ji + 36 * i, sizeof Tii);
    if (i > 0) {
      mat_transpose(6, 6, X + 36 * i, Xt);
      mat_mul(6, 6, 6, X + 36 * i, Ji + 36 * (i - 1), t1);
      mat_mul(6, 6, 6, t1, Xt, t2);
      for (int k = 0; k < 36; ++k) Tii[k] += t2[k];
      for (int k = 0; k < 36; ++k) Tlo[k] = -t1[k]; /* T_{i,i-1} = -X_i J_{i-1}^-1 */
    }
    if (i + 1 < n) {
      mat_transpose(6, 6, X + 36 * (i + 1), Xt);
      mat_mul(6, 6, 6, Ji + 36 * i, Xt, t1);
      for (int k = 0; k < 36; ++k) Tup[k] = -t1[k]; /* T_{i,i+1} = -J_i^-1 X_{i+1}^T */
    }
    const double *Wi = W + 30 * i;
    double WtT[30], tmp5[5];
    /* D_i = W_i^T T_ii W_i */
    double Wt[30];
    mat_transpose(6, 5, Wi, Wt);
    mat_mul(5, 6, 6, Wt, Tii, WtT);
    mat_mul(5, 6, 5, WtT, Wi, D + 25 * i);
    /* Bb[i][1] = W_i^T T_ii S_i ; Cd[i] = S_i^T T_ii S_i */
    mat_vec(5, 6, WtT, S + 6 * i, Bb + 15 * i + 5);
    {
      double ts[6];
      mat_vec(6, 6, Tii, S + 6 * i, ts);
      Cd[i] = 0.0;
      for (int k = 0; k < 6; ++k) Cd[i] += S[6 * i + k] * ts[k];
    }
    if (i > 0) {
      mat_mul(5, 6, 6, Wt, Tlo, WtT);
      mat_vec(5, 6, WtT, S + 6 * (i - 1), Bb + 15 * i);
    } else {
      memset(Bb + 15 * i, 0, 5 * sizeof(double));
    }
    if (i + 1 < n) {
      mat_mul(5, 6, 6, Wt, Tup, WtT);
      mat_mul(5, 6, 5, WtT, W + 30 * (i + 1), U + 25 * i);
      mat_vec(5, 6, WtT, S + 6 * (i + 1), Bb + 15 * i + 10);
      double ts[6];
      mat_vec(6, 6, Tup, S + 6 * (i + 1), ts);
      Co[i] = 0.0;
      for (int k = 0; k < 6; ++k) Co[i] += S[6 * i + k] * ts[k];
    } else {
      memset(U + 25 * i, 0, 25 * sizeof(double));
      memset(Bb + 15 * i + 10, 0, 5 * sizeof(double));
      Co[i] = 0.0;
    }
    (void)tmp5;
  }
  if (Wout) memcpy(Wout, W, sizeof(double) * 30 * N);
  free(X); free(Ji); free(W); free(S);
  return st;
}

/* Algorithm 2 (OEESolvBTDSys): odd-even elimination of the symmetric block
 * tri-diagonal system with diagonal blocks D_i, upper blocks U_i (lower = U^T)
 * and right-hand side R_i, block size b (<= 8). Every right-hand side of level j
 * uses level j-1 values. SolvSys is a Cholesky solve. On return F holds the
 * solution; D, U, R hold the level ceil(log2 n) blocks (U then all zero). */
static int oee_solve(int n, int b, double *D, double *U, double *R, double *F) {
  size_t bb = (size_t)b * (size_t)b, N = (size_t)n;
  double *D0 = malloc(sizeof(double) * bb * N), *U0 = malloc(sizeof(double) * bb * N);
  double *R0 = malloc(sizeof(double) * (size_t)b * N);
  double *E = malloc(sizeof(double) * bb * N), *K = malloc(sizeof(double) * bb * N);
  if (!D0 || !U0 || !R0 || !E || !K) {
    free(D0); free(U0); free(R0); free(E); free(K);
    return ORC_ERR_ARG;
  }
  int levels = 0;
  while ((1 << levels) < n) ++levels;
  int st = ORC_OK;
  for (int j = 1; j <= levels && st == ORC_OK; ++j) {
    int d = 1 << (j - 1);
    memcpy(D0, D, sizeof(double) * bb * N);
    memcpy(U0, U, sizeof(double) * bb * N);
    memcpy(R0, R, sizeof(double) * (size_t)b * N);
    /* coefficients for i = 1 .. n - d (0-based: 0 .. n-d-1) */
    for (int i = 0; i + d < n && st == ORC_OK; ++i) {
      double Ut[64], Et[64], Kt[64];
      mat_transpose(b, b, U0 + bb * i, Ut);
      st = solv_sys(b, b, D0 + bb * (i + d), Ut, Et);          /* D_{i+d} E_i^T = U_i^T */
      if (st) break;
      mat_transpose(b, b, Et, E + bb * i);
      st = solv_sys(b, b, D0 + bb * i, U0 + bb * i, Kt);        /* D_i K_i^T = U_i */
      if (st) break;
      mat_transpose(b, b, Kt, K + bb * i);
    }
    if (st) break;
    /* updates of D and R for i = 1 .. n - d */
    for (int i = 0; i + d < n; ++i) {
      double t[64], Ut[64], v[8];
      mat_transpose(b, b, U0 + bb * i, Ut);
      mat_mul(b, b, b, E + bb * i, Ut, t);                       /* E_i U_i^T */
      for (size_t k = 0; k < bb; ++k) D[bb * i + k] -= t[k];
      mat_mul(b, b, b, K + bb * i, U0 + bb * i, t);              /* K_i U_i */
      for (size_t k = 0; k < bb; ++k) D[bb * (i + d) + k] -= t[k];
      mat_vec(b, b, E + bb * i, R0 + (size_t)b * (i + d), v);    /* E_i R_{i+d} */
      for (int k = 0; k < b; ++k) R[(size_t)b * i + k] -= v[k];
      mat_vec(b, b, K + bb * i, R0 + (size_t)b * i, v);          /* K_i R_i */
      for (int k = 0; k < b; ++k) R[(size_t)b * (i + d) + k] -= v[k];
    }
    /* U_i = -E_i U_{i+d} for i = 1 .. n - 2d; the last 2d upper blocks vanish */
    for (int i = 0; i < n; ++i) {
      if (i + 2 * d < n) {
        double t[64];
        mat_mul(b, b, b, E + bb * i, U0 + bb * (i + d), t);
        for (size_t k = 0; k < bb; ++k) U[bb * i + k] = -t[k];
      } else {
        memset(U + bb * i, 0, sizeof(double) * bb);
      }
    }
  }
  for (int i = 0; i < n && st == ORC_OK; ++i)
    st = solv_sys(b, 1, D + bb * i, R + (size_t)b * i, F + (size_t)b * i);
  free(D0); free(U0); free(R0); free(E); free(K);
  return st;
}

/* Algorithm 1 (CalcFwdDyn_CFA): bias torque by ID, tau_delta, A, B, C,
 * R = -B tau_delta, block tri-diagonal solve by OEE, qdd = C tau_delta + B^T F_c.
 * Win [n][30]: the projection W_i of Eq. cfa-eq1 (NULL: projection_w); Fc_out
 * [n][5] (may be NULL) receives the constraint-force coordinates F_c. */
static int fd_cfa_chain(int n, const double *axes, const double *frames, const double *J,
                        const double *grav, const double *q, const double *qd,
                        const double *tau, const double *Win, double *qdd, double *Fc_out) {
  size_t N = (size_t)n;
  double *td = malloc(sizeof(double) * N), *D = malloc(sizeof(double) * 25 * N);
  double *U = malloc(sizeof(double) * 25 * N), *Bb = malloc(sizeof(double) * 15 * N);
  double *Cd = malloc(sizeof(double) * N), *Co = malloc(sizeof(double) * N);
  double *R = malloc(sizeof(double) * 5 * N), *Fc = malloc(sizeof(double) * 5 * N);
  int st = ORC_ERR_ARG;
  if (td && D && U && Bb && Cd && Co && R && Fc) {
    rnea_chain(n, axes, frames, J, grav, q, qd, NULL, td);     /* CalcInvDyn */
    for (int i = 0; i < n; ++i) td[i] = tau[i] - td[i];        /* CalcDiffTorques */
    st = cfa_blocks(n, axes, frames, J, q, Win, D, U, Bb, Cd, Co, NULL);
    if (st == ORC_OK) {
      for (int i = 0; i < n; ++i)                               /* R = -B tau_delta */
        for (int k = 0; k < 5; ++k) {
          double s = Bb[15 * i + 5 + k] * td[i];
          if (i > 0) s += Bb[15 * i + k] * td[i - 1];
          if (i + 1 < n) s += Bb[15 * i + 10 + k] * td[i + 1];
          R[5 * i + k] = -s;
        }
      st = oee_solve(n, 5, D, U, R, Fc);                        /* SolvBTDSys */
    }
    if (st == ORC_OK) {
      for (int j = 0; j < n; ++j) {                             /* CalcAcc */
        double s = Cd[j] * td[j];
        if (j > 0) s += Co[j - 1] * td[j - 1];
        if (j + 1 < n) s += Co[j] * td[j + 1];
        for (int i = j - 1; i <= j + 1; ++i) {
          if (i < 0 || i >= n) continue;
          const double *blk = Bb + 15 * i + 5 * (j - i + 1);     /* B_{i,j} */
          for (int k = 0; k < 5; ++k) s += blk[k] * Fc[5 * i + k];
        }
        qdd[j] = s;
      }
      if (Fc_out) memcpy(Fc_out, Fc, sizeof(double) * 5 * N);
    }
  }
  free(td); free(D); free(U); free(Bb); free(Cd); free(Co); free(R); free(Fc);
  return st;
}

/* ------------------------------------------------------------- exported API */

#define ORC_ALGO_CHOLESKY 0
#define ORC_ALGO_ABA 1
#define ORC_ALGO_CFA 2

/* Single chain entry points (host arrays, n links). */
int orc_rnea(int n, const double *axes, const double *frames, const double *J,
             const double *grav, const double *q, const double *qd, const double *qdd,
             double *tau) {
  if (n < 0) return ORC_ERR_ARG;
  return rnea_chain(n, axes, frames, J, grav, q, qd, qdd, tau);
}

int orc_mass_matrix(int n, const double *axes, const double *frames, const double *J,
                    const double *q, double *M) {
  if (n < 0) return ORC_ERR_ARG;
  return mass_matrix_chain(n, axes, frames, J, q, M);
}

int orc_cfa_blocks(int n, const double *axes, const double *frames, const double *J,
                   const double *q, const double *Win, double *D, double *U, double *Bb,
                   double *Cd, double *Co, double *Wout) {
  if (n < 1) return ORC_ERR_ARG;
  return cfa_blocks(n, axes, frames, J, q, Win, D, U, Bb, Cd, Co, Wout);
}

/* CFA of one chain with the projection W [n][30] (Eq. cfa-eq1; NULL: the
 * default complement); F_c [n][5] may be NULL. */
int orc_fd_cfa_w(int n, const double *axes, const double *frames, const double *J,
                 const double *grav, const double *q, const double *qd, const double *tau,
                 const double *W, double *qdd, double *Fc) {
  if (n < 1) return ORC_ERR_ARG;
  return fd_cfa_chain(n, axes, frames, J, grav, q, qd, tau, W, qdd, Fc);
}

int orc_oee_solve(int n, int b, double *D, double *U, double *R, double *F) {
  if (n < 1 || b < 1 || b > 8) return ORC_ERR_ARG;
  return oee_solve(n, b, D, U, R, F);
}

/* Batched forward dynamics: problem p uses chain chain_of[p] (or p if chain_of is
 * NULL) of a model packed by model_offsets, and its states at state_offsets[p]. */
int orc_fd_batch(int algo, int n_problems, const int32_t *chain_of,
                 const int64_t *model_offsets, const int64_t *state_offsets,
                 const double *axes, const double *frames, const double *J,
                 const double *grav, const double *q, const double *qd, const double *tau,
                 double *qdd, int32_t *status, int n_threads) {
  int bad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(n_threads > 0 ? n_threads : 1) reduction(+ : bad)
#endif
  for (int p = 0; p < n_problems; ++p) {
    int c = chain_of ? chain_of[p] : p;
    int64_t m0 = model_offsets[c], s0 = state_offsets[p];
    int n = (int)(model_offsets[c + 1] - m0);
    int st;
    if (n == 0)
      st = ORC_OK; /* an empty chain has nothing to solve */
    else if (algo == ORC_ALGO_CHOLESKY)
      st = fd_cholesky_chain(n, axes + 3 * m0, frames + 12 * m0, J + 36 * m0, grav, q + s0,
                             qd + s0, tau + s0, qdd + s0);
    else if (algo == ORC_ALGO_ABA)
      st = fd_aba_chain(n, axes + 3 * m0, frames + 12 * m0, J + 36 * m0, grav, q + s0,
                        qd + s0, tau + s0, qdd + s0);
    else if (algo == ORC_ALGO_CFA)
      st = fd_cfa_chain(n, axes + 3 * m0, frames + 12 * m0, J + 36 * m0, grav, q + s0,
                        qd + s0, tau + s0, NULL, qdd + s0, NULL);
    else
      st = ORC_ERR_ARG;
    if (status) status[p] = st;
    bad += st != ORC_OK;
  }
  (void)n_threads;
  return bad;
}

/* Batched inverse dynamics tau = ID(q, qd, qdd) with gravity (Eq. 2a-2d). */
int orc_rnea_batch(int n_problems, const int32_t *chain_of, const int64_t *model_offsets,
                   const int64_t *state_offsets, const double *axes, const double *frames,
                   const double *J, const double *grav, const double *q, const double *qd,
                   const double *qdd, double *tau, int n_threads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(n_threads > 0 ? n_threads : 1)
#endif
  for (int p = 0; p < n_problems; ++p) {
    int c = chain_of ? chain_of[p] : p;
    int64_t m0 = model_offsets[c], s0 = state_offsets[p];
    int n = (int)(model_offsets[c + 1] - m0);
    if (n == 0) continue;
    rnea_chain(n, axes + 3 * m0, frames + 12 * m0, J + 36 * m0, grav, q + s0, qd + s0,
               qdd ? qdd + s0 : NULL, tau + s0);
  }
  (void)n_threads;
  return 0;
}
