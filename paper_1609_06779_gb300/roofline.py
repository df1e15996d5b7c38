"""Algorithmic work per problem, for the roofline of each kernel.

Counts are the floating-point operations of the method as the kernels carry it
out in canonical link frames (S_i = e_1), with a fused multiply-add counted as 2
and every other add, multiply, divide or reciprocal square root as 1; sin/cos of
the joint angles are not counted. The serial (team = 1) schedule is the
reference: the scan's extra compositions for team > 1 are overhead, not work.

Primitive costs (flops): Ad_{g^-1} x or Ad_{g^-1}^T x = 42, symmetric 6x6 times
a vector = 66, ad_V^T x = 33, joint transform = 18; 5x5 Cholesky = 60, one 5x5
triangular solve = 25.

Bytes: the model record (56 entries of the arithmetic type per link) and the
four state vectors (q, qdot, tau in, qdd out) per link; the workspace is
intermediate traffic, not algorithmic.
"""
from __future__ import annotations

import math

ADJ, SYM6, ADT, JT = 42, 66, 33, 18
CHOL5, TRI5 = 60, 25


def id_flops(n: int) -> int:
    """Eq. 2a-2d: transform 18, twist 43, acceleration 50, f_i 171, force 49."""
    return n * (JT + (ADJ + 1) + (ADJ + 8) + (2 * SYM6 + ADT + 6) + (ADJ + 7))


# X^T P X + J in rotated 3x3 blocks (R A, R B, R C 135; B' 45; C' 30;
# B'' = B' + p^ C' 36; top-left block with its cross terms 84; + J 15)
CONG_BLOCKS = 345
# the same with row and column 0 of P zero (the articulated inertia, Pa S = 0):
# R A 18 and R B 27 instead of 45 each, A' 24 instead of 36
CONG_BLOCKS_ART = CONG_BLOCKS - 57


def abia_flops(n: int) -> int:
    """ID + articulated-inertia recursion (Pa on its 15 nonzero entries 45 + 1,
    pa 18, congruence with J in blocks and the zero row and column of Pa 288, bias
    transport 42) for n-1 links + forward pass 56."""
    per_abi = 46 + 18 + CONG_BLOCKS_ART + ADJ
    return id_flops(n) + max(n - 1, 0) * per_abi + n * (ADJ + 14)


def jsiia_flops(n: int) -> int:
    """ID + the composite inertias of the unit-acceleration columns (n - 1
    congruences X^T I X: 12 transports, + J 21) + the entries of M below the
    diagonal as base-frame pairings (per link: forward kinematics 63, the joint
    axis as a base-frame twist 9, the composite force to the base frame 42; per
    entry a 6-term dot product 11) + Cholesky n^3/3 + two triangular solves 2 n^2."""
    composite = max(n - 1, 0) * (12 * ADJ + 21)
    entries = n * (63 + 9 + ADJ) + 11 * n * (n - 1) // 2
    return id_flops(n) + composite + entries + (n ** 3) // 3 + 2 * n * n


def oee_flops(n: int) -> int:
    """Odd-even elimination (Algorithm 2): ceil(log2 n) levels; per row and
    level the Cholesky factor of D (60) and g = L^{-1} R (25), and while the row
    has an upper neighbour G = L^{-1} U (125); the E part (Z = U L^{-T} 125,
    Z Z^T 165, Z g 50) and, while row i + 2d exists, Z G (250); the K part
    (G^T G 165, G^T g 55); then the final block solves (110 per row)."""
    levels = math.ceil(math.log2(n)) if n > 1 else 0
    f = 0
    for j in range(1, levels + 1):
        d = 1 << (j - 1)
        pairs = max(n - d, 0)            # rows with an upper neighbour (= with a lower one)
        f += n * (CHOL5 + TRI5) + pairs * 5 * TRI5
        f += pairs * (5 * TRI5 + 165 + 50)
        f += max(n - 2 * d, 0) * 250
        f += pairs * (165 + 55)
    return f + n * (CHOL5 + 2 * TRI5)


# D_i = (X K X^T)[1..5][1..5] + K_self in rotated 3x3 blocks: Bt = B + A p^ 36,
# Cs = C - p^ B + Bt^T p^ 48, A R_{:,1..2} 30 + its 3 entries 18, rows 1..2 of
# R^T Bt 30 + its 6 entries 36, R^T Cs 45 + its 6 entries 36 (each entry with its
# addition into K_self)
D_BLOCKS = 36 + 48 + 48 + 66 + 81
# U_i: columns 1, 2 of Ad^T have three nonzeros (5 rows x 5 flops); columns 3..5
# are (p x x; x), and k_top . (p x x) + k_bot . x = (k_top x p + k_bot) . x (per
# row 12 for that vector, then 5 per column)
U_BLOCK = 2 * 25 + 5 * (12 + 3 * 5)


def cfa_flops(n: int) -> int:
    """ID + A blocks (D in rotated blocks 279; U 185: rows 1..5 of J^{-1} times
    the sparse columns of Ad^T) + R = -B tau (J^{-1} on three nonzero components
    30 + 6, one transport 42) + OEE + CalcAcc (120)."""
    return id_flops(n) + n * (D_BLOCKS + U_BLOCK + 78) + oee_flops(n) + n * 120


def cr_flops(n: int) -> int:
    """Block cyclic reduction of the same system: at each level the eliminated
    rows factor themselves (60 + 25, and G = L^{-1} U 125 when they have an upper
    neighbour) and the kept rows take the OEE row update (E part 340 + Z G 250,
    K part 220); back substitution 150 per row; the root row solves directly."""
    levels = math.ceil(math.log2(n)) if n > 1 else 0
    f = 0
    for j in range(1, levels + 1):
        d = 1 << (j - 1)
        for i in range(d - 1, n, d):
            if ((i + 1) // d) % 2 == 1:        # eliminated at this level
                f += CHOL5 + TRI5 + (5 * TRI5 if i + d < n else 0)
                f += 150
            else:                              # kept: updated
                if i + d < n:
                    f += 5 * TRI5 + 165 + 50 + (250 if i + 2 * d < n else 0)
                if i - d >= 0:
                    f += 165 + 55
    roots = 1 if n >= 1 and (n & (n - 1)) == 0 else 0
    return f + roots * (CHOL5 + 2 * TRI5)


def cfa_cr_flops(n: int) -> int:
    return id_flops(n) + n * (D_BLOCKS + U_BLOCK + 78) + cr_flops(n) + n * 120


def hybrid_flops(n: int) -> int:
    """The hybrid partition / cyclic-reduction solve at the serial schedule (one
    segment: every row but the first and the last is interior): per interior row
    the Cholesky factor 60, G1 = L^{-1} F^T and G2 = L^{-1} U 250, g 25, the
    updates of the first row and the next row (G1^T G1, G2^T G2 150 each, G1^T g,
    G2^T g 50 each), the moved coupling F = -G1^T G2 250, and the back
    substitution 125; the two kept rows by cyclic reduction."""
    if n <= 2:
        return cr_flops(n)
    return (n - 2) * (60 + 250 + 25 + 300 + 100 + 250 + 125) + cr_flops(2)


def cfa_hybrid_flops(n: int) -> int:
    return id_flops(n) + n * (D_BLOCKS + U_BLOCK + 78) + hybrid_flops(n) + n * 120


FLOPS = {"id": id_flops, "abia": abia_flops, "jsiia": jsiia_flops, "cfa": cfa_flops,
         "cfa_cr": cfa_cr_flops, "cfa_hybrid": cfa_hybrid_flops,
         # the ABI scan computes the ABIA: its useful work is ABIA's serial count
         # (the scan's compositions are the price of the depth, not work)
         "abia_scan": abia_flops}


def flops(algo: str, lengths) -> int:
    f = FLOPS[algo]
    return int(sum(f(int(n)) for n in lengths))


def bytes_per_link(prec: str) -> int:
    es = 8 if prec == "fp64" else 4
    return 56 * es + 4 * es
