"""H-matrix approximation of the L1 matrix R, Section 3 (oracle; test infrastructure only).

Steps, in the paper's order:

1. Block tree (Section 3, construction paragraph and Fig. 2): start from the whole index
   set {1..M} x {1..M}; a block whose columns all lie above the diagonal is a zero block;
   an admissible block becomes a low-rank (Rk) block; any other block is split 2 x 2 by
   bisecting its row and column index ranges, until it is no larger than ``leaf`` and is
   then kept as a full (dense) block.
2. Admissibility (Definition 3.1): the rows of theta are the points t_m (the supports of the
   Dirac test functions) and span I_t = [a, b]; the columns of sigma are hat functions
   phi_j with supports [t_{j-1}, t_{j+1}] and span I_s = [c, d].  The block is admissible if
   d < a and diam(I_t) = b - a <= dist(I_s, I_t) = a - d.
3. Taylor degenerate kernel about the centre t_c = (a + b)/2 of I_t, k terms
   (Eq. degenerate_kernel and the Taylor display of Section 3), with
   c_nu = (1/nu!) prod_{l=1}^{nu} (1 - alpha - l).
4. Rk factors (Eqs. A_elements, B_elements):
       A[m, nu] = (t_m - t_c)^nu / Gamma(1 - alpha),
       B[j, nu] = int q_nu(s) phi_j'(s) ds,   q_nu(s) = c_nu (t_c - s)^-(alpha+nu).
   The printed closed form of B cancels catastrophically far from the diagonal in double
   precision, so B is evaluated here in its integrated-by-parts form (the one used in the
   proof of Theorem 3.1):  B[j, nu] = -c_nu (alpha + nu) int (t_c - s)^(-1-alpha-nu) phi_j(s) ds,
   by Gauss-Legendre on each half of the hat.  Both factors are rescaled by rho^nu,
   rho = (b - a)/2 (A by rho^-nu, B by rho^nu), which leaves A B^T unchanged and keeps both
   in floating-point range on strongly graded meshes.

The approximated matrix R~ is returned densely (dense blocks hold the exact entries of R), so
that the oracle's smoother and defect can use it with plain dense linear algebra.  The bound
of Theorem 3.1 is provided for the pin that checks the factors.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Block:
    r0: int   # first row index (0-based, row m = r0 + 1)
    r1: int   # one past the last row
    c0: int   # first column index (0-based, column j = c0 + 1)
    c1: int
    kind: str  # "zero", "dense", "rk"


def _interval_rows(t: np.ndarray, r0: int, r1: int) -> tuple[float, float]:
    """I_t = [a, b] spanned by the points t_m, m = r0+1 .. r1."""
    return t[r0 + 1], t[r1]


def _interval_cols(t: np.ndarray, c0: int, c1: int) -> tuple[float, float]:
    """I_s = [c, d] spanned by the supports [t_{j-1}, t_{j+1}], j = c0+1 .. c1."""
    M = len(t) - 1
    return t[c0], t[min(c1 + 1, M)]


def admissible(t: np.ndarray, blk: Block) -> bool:
    a, b = _interval_rows(t, blk.r0, blk.r1)
    c, d = _interval_cols(t, blk.c0, blk.c1)
    return d < a and (b - a) <= (a - d)


def block_tree(t: np.ndarray, leaf: int) -> list[Block]:
    """Leaves of the block tree of R (step 1 above)."""
    M = len(t) - 1
    out: list[Block] = []

    def rec(r0, r1, c0, c1):
        blk = Block(r0, r1, c0, c1, "")
        if c0 >= r1:                      # every column j > every row m: zero block
            blk.kind = "zero"
            out.append(blk)
            return
        if admissible(t, blk):
            blk.kind = "rk"
            out.append(blk)
            return
        if (r1 - r0) <= leaf or (c1 - c0) <= leaf:
            blk.kind = "dense"
            out.append(blk)
            return
        rm = (r0 + r1) // 2
        cm = (c0 + c1) // 2
        rec(r0, rm, c0, cm)
        rec(r0, rm, cm, c1)
        rec(rm, r1, c0, cm)
        rec(rm, r1, cm, c1)

    rec(0, M, 0, M)
    return out


def taylor_coeff(alpha: float, nu: int) -> float:
    """c_nu = (1/nu!) prod_{l=1}^{nu} (1 - alpha - l)."""
    c = 1.0
    for l in range(1, nu + 1):
        c *= (1.0 - alpha - l) / l
    return c


def rk_factors(t: np.ndarray, alpha: float, blk: Block, k: int, nq: int = 24):
    """Scaled Taylor factors (A, B) of one admissible block: R~|block = A @ B.T."""
    a, b = _interval_rows(t, blk.r0, blk.r1)
    tc = 0.5 * (a + b)
    rho = 0.5 * (b - a)
    if rho == 0.0:
        rho = 1.0
    rows = np.arange(blk.r0 + 1, blk.r1 + 1)
    cols = np.arange(blk.c0 + 1, blk.c1 + 1)
    nus = np.arange(k)
    A = ((t[rows][:, None] - tc) / rho) ** nus[None, :] / math.gamma(1.0 - alpha)
    xg, wg = np.polynomial.legendre.leggauss(nq)
    up = 0.5 * (1.0 + xg)
    tau_l = t[cols] - t[cols - 1]
    tau_r = t[cols + 1] - t[cols]
    sl = t[cols - 1][:, None] + tau_l[:, None] * up[None, :]    # nodes, rising half
    sr = t[cols][:, None] + tau_r[:, None] * up[None, :]        # nodes, falling half
    B = np.empty((len(cols), k))
    for nu in nus:
        c_nu = taylor_coeff(alpha, int(nu))
        fl = (tc - sl) ** (-1.0 - alpha) * (rho / (tc - sl)) ** nu
        fr = (tc - sr) ** (-1.0 - alpha) * (rho / (tc - sr)) ** nu
        il = 0.5 * tau_l * (fl * up[None, :] * wg[None, :]).sum(axis=1)
        ir = 0.5 * tau_r * (fr * (1.0 - up)[None, :] * wg[None, :]).sum(axis=1)
        B[:, nu] = -c_nu * (alpha + nu) * (il + ir)
    return A, B


def approximate(t: np.ndarray, alpha: float, R: np.ndarray, leaf: int, k: int):
    """R~ (dense array) and the block list: dense blocks copied from R, Rk blocks A B^T."""
    blocks = block_tree(t, leaf)
    Rt = np.zeros_like(R)
    for blk in blocks:
        if blk.kind == "dense":
            Rt[blk.r0:blk.r1, blk.c0:blk.c1] = R[blk.r0:blk.r1, blk.c0:blk.c1]
        elif blk.kind == "rk":
            A, B = rk_factors(t, alpha, blk, k)
            Rt[blk.r0:blk.r1, blk.c0:blk.c1] = A @ B.T
    return Rt, blocks


def theorem31_bound(t: np.ndarray, alpha: float, blk: Block, k: int) -> np.ndarray:
    """Entry-wise bound of Theorem 3.1 for an admissible block, shape (rows, cols):
    (tau_{j-1} + tau_j) / (2 Gamma(1-alpha) (|a-t_c| + |a-d|)^(1+alpha)) * 3^-k (3/2 (alpha+k) + 3/4)."""
    a, b = _interval_rows(t, blk.r0, blk.r1)
    c, d = _interval_cols(t, blk.c0, blk.c1)
    tc = 0.5 * (a + b)
    cols = np.arange(blk.c0 + 1, blk.c1 + 1)
    supp = t[cols + 1] - t[cols - 1]
    pref = supp / (2.0 * math.gamma(1.0 - alpha) * (abs(a - tc) + abs(a - d)) ** (1.0 + alpha))
    series = 3.0 ** (-k) * (1.5 * (alpha + k) + 0.75)
    return np.broadcast_to(pref[None, :] * series, (blk.r1 - blk.r0, len(cols)))
