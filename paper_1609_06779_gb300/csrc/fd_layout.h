// fd_layout.h -- data layout shared by the host side and the kernels.
//
// Model arena (one record per link, canonical link frames with the joint axis
// along x, so S_i = e_1): REC entries of the arena's type per link,
//   [0, 9)   R0   home rotation parent -> child (row-major)
//   [9, 12)  p0   home translation parent -> child
//   [12, 33) J    spatial inertia at the link origin, packed symmetric 6x6
//   [33, 54) Jinv its inverse, packed symmetric 6x6
//   [54, 56) padding (keeps a record a multiple of 16 bytes in float and double)
// Records of one chain are contiguous; chain k starts at record model_off[k].
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#include <cuda_runtime.h>
#endif

namespace fdk {

constexpr int REC = 56;
constexpr int REC_R0 = 0;
constexpr int REC_P0 = 9;
constexpr int REC_J = 12;
constexpr int REC_JI = 33;

// Per-link workspace fields of the arithmetic type T (inverse-dynamics part).
constexpr int W_G = 0;    // joint transform g_{i-1,i}(q_i): R (9), p (3)
constexpr int W_V = 12;   // twist V_i
constexpr int W_F = 18;   // f_i = J_i Vd_i - ad_{V_i}^T J_i V_i
constexpr int W_TD = 24;  // tau_delta_i (or tau_i for inverse dynamics)
constexpr int W_Z = 25;   // CFA: J^{-1} (I - Gamma)^T F products
constexpr int W_PT = 25;  // R^T p of g_i while the component-lane inverse dynamics runs
                          // (3 entries; CFA overwrites them with its W_Z products later)
constexpr int NT = 32;    // T entries per link

// Per-row workspace of the accumulation type TA for CFA's odd-even elimination.
constexpr int A_D0 = 0;    // D (packed symmetric 5x5), two buffers
constexpr int A_D1 = 15;
constexpr int A_U0 = 30;   // U (row-major 5x5), two buffers
constexpr int A_U1 = 55;
constexpr int A_R0 = 80;   // R (5), two buffers
constexpr int A_R1 = 85;
constexpr int A_L = 90;    // Cholesky factor of D (15) and reciprocal diagonal (5)
constexpr int A_LI = 105;
constexpr int A_FC = 110;  // F_c (5)
constexpr int A_G = 115;   // G = L^{-1} U (row-major 5x5) and g = L^{-1} R of this level
constexpr int A_GR = 140;
constexpr int A_LO = 145;  // cyclic reduction: the lower coupling U_{i-d} kept for back substitution
constexpr int A_Q = 145;   // general projection (odd-even elimination only): Q_i (row-major
                           // 5x5), or for block Jacobi L_i (15) and 1 / L_jj (5)
// a second right-hand side (MODE_FD2: the adjoint's M^{-1} w beside FD)
constexpr int A_R20 = 170;  // R (5), two buffers
constexpr int A_R21 = 175;
constexpr int A_GR2 = 180;  // g = L^{-1} R of this level
constexpr int A_FC2 = 185;  // F_c (5)
constexpr int A_Z2 = 190;   // J^{-1} (I - Gamma)^T F products (6)
constexpr int NA_CFA = 196;

// JSIIA: per-link TA entries (right-hand side 1, h_i = I^c_i e_1 6, the second
// right-hand side of MODE_FD2 1, joint i's axis as a base-frame twist s_i 6) and
// n*n TA entries (M).
constexpr int NA_JSIIA = 14;
constexpr int NSQ_JSIIA = 1;

// ABIA: per-link TA entries: h_i = P_i S_i (6), 1 / D_i (1), u_i / D_i (1), and
// u_i / D_i of the second right-hand side (MODE_FD2).
constexpr int A_H = 0;
constexpr int A_DD = 6;
constexpr int A_UU = 7;
constexpr int A_UU2 = 8;
constexpr int NA_ABIA = 9;

// Kinematic trees (ABIA, JSIIA): per-link TA entries (the layout is in
// fd_tree.cuh); JSIIA adds n*n entries (M) per problem.
constexpr int NA_TREE = 41;
// ... and, for trees closed by loops (JSIIA), per-link loop entries after the
// JSIIA workspace (g_0i 12, five constraint rows and five solves per loop, at
// most four loops a tree)
constexpr int NA_LOOP_LINK = 52;
constexpr int MAX_LOOPS_PER_TREE = 4;

// Adjoint (reverse inverse dynamics) per-link workspace of T.
constexpr int J_G = 0;    // g_i (12)
constexpr int J_V = 12;   // V_i
constexpr int J_A = 18;   // Vd_i
constexpr int J_F = 24;   // F_i
constexpr int J_FB = 30;  // Fbar_i (f_i before the force pass)
constexpr int J_AB = 36;  // Abar_i
constexpr int J_VB = 42;  // Vbar_i
constexpr int J_PT = 48;  // R^T p of g_i (component-lane sweeps)
constexpr int NT_ADJ = 52;

// id_team modes (a zero-initialised KArgs means forward dynamics)
constexpr int MODE_FD = 0;      // tau_delta = tau - ID(q, qd, 0)
constexpr int MODE_ID = 1;      // tau = ID(q, qd, qdd)
constexpr int MODE_LINEAR = 2;  // tau_delta = in3 (solve M x = in3: joint transforms only)
constexpr int MODE_FD2 = 3;     // MODE_FD into out, and M^{-1} in4 into out4 with the same
                                // factorisation (the adjoint's linear solve beside FD)
constexpr int MODE_RES = 4;     // inverse dynamics only (the FP32 CFA refinement pass):
                                // tau_delta = in3 - ID(q, qd, out), the residual of out

// The problems one launch (or one length class of a launch) covers: positions
// t0 .. t1-1 of the processing order, starting at block blk0 of the grid.
struct Range {
  int32_t blk0;
  int32_t t0, t1;
};

// A launch split into length classes: class c takes blocks blk[c] .. blk[c+1]-1
// and problems first[c] .. first[c+1]-1 of the processing order (longest first,
// so a class is a contiguous range), with a team of team[c] lanes per problem.
constexpr int MAX_CLASSES = 24;
struct ClassTable {
  int32_t n;
  int32_t blk[MAX_CLASSES + 1];
  int32_t first[MAX_CLASSES + 1];
  int32_t team[MAX_CLASSES];
};

struct KArgs {
  const void *model;         // [L][REC] of T
  const void *model64;       // [L][REC] of double (the FP64 copy; mixed-precision CFA blocks)
  const int64_t *model_off;  // [K + 1]
  const int32_t *prob_chain; // [N] chain of each problem, or null: problem p is chain p
  const int64_t *state_off;  // [N + 1]
  const int64_t *sq_off;     // [N + 1] prefix sums of n_p^2
  const int32_t *order;      // [N] processing order (longest first)
  int32_t n_problems;
  int32_t team;
  const void *q;
  const void *qd;
  const void *in3;  // tau (forward dynamics) or qdd (inverse dynamics)
  void *out;        // qdd (forward dynamics) or tau (inverse dynamics)
  void *ws_t;       // per-link T workspace
  void *ws_a;       // TA workspace
  int32_t *status;  // [N] or null
  double grav[3];
  int32_t mode;     // MODE_FD (default) or MODE_LINEAR for the forward-dynamics kernels
  const void *lam;  // adjoint: lambda = M^{-1} qdd_bar
  void *out2;       // adjoint: qdot_bar
  void *out3;       // adjoint: mass_bar (or null)
  const void *in4;  // MODE_FD2: second right-hand side w
  void *out4;       // MODE_FD2: M^{-1} w
  // CFA with a general projection W_i = Wc_i Q_i (Wc_i = e_2 .. e_6 of the
  // canonical frame): WPROJ_GIVEN takes Q_i from wq ([L][25] double, row-major,
  // by the model's link index), WPROJ_BLOCK_JACOBI forms Q_i = L_i^{-T} from
  // D_i = L_i L_i^T
  const double *wq;
  int32_t wmode;
  // kinematic trees: each link's parent within its tree (-1: the base), by the
  // model's link index; null for serial chains
  const int32_t *parent;
  // closed loops of kinematic trees: loops of chain c are loop_off[c] ..
  // loop_off[c+1]-1; per loop its links a, b (loop_ab) and the two joint frames
  // in canonical link coordinates (loop_T, 24 doubles); loop_ws: where the loop
  // workspace starts in ws_a (elements)
  const int32_t *loop_off;
  const int32_t *loop_ab;
  const double *loop_T;
  int64_t loop_ws;
};

constexpr int WPROJ_GIVEN = 1;
constexpr int WPROJ_BLOCK_JACOBI = 2;

}  // namespace fdk
