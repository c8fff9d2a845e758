"""Host side of the split outer defect (no GPU): the BF16 digit tiles of R~ that the tensor cores
multiply (fhmg_hmatrix_split_digits).  The tiles are decoded through the layout the header states
and checked against the library's dense R~: every row is the 49-bit rounding of R~ 2^(49 - E_m)
written exactly in seven balanced base-2^7 digits, E_m is the binary exponent of the row's largest
entry, every stored value is an exact BF16 integer, the upper triangle is zero, and the block table
lists exactly the digit tiles that hold a nonzero digit."""
import math

import numpy as np
import pytest

import paper_1706_07632_gb300 as fh

G, TR, TK = 7, 128, 64


def bf16_to_float(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def tile_index(r, k):
    """uint16 index of entry (r, k) in a 128 x 64 K-major tile with the 128-byte swizzle."""
    return (r // 8) * 512 + (r % 8) * 64 + (((k // 8) ^ (r % 8)) & 7) * 8 + k % 8


def decode(H):
    """digits d[a, m, k] of R~ from the tiles (zero where a block lists no tile for digit a)."""
    tiles, pairs, rexp = H.split_digits()
    M = H.M
    nI = M // TR
    r, k = np.meshgrid(np.arange(TR), np.arange(TK), indexing="ij")
    idx = tile_index(r, k)
    assert np.unique(idx).size == TR * TK  # the layout is a permutation of the tile
    d = np.zeros((G, M, M))
    nxt = 0
    q = 0
    for I in range(nI):
        for J in range(2 * I + 2):
            mask, first, z0, z1 = (int(v) for v in pairs[q])
            assert (z0, z1) == (0, 0)
            assert first == nxt  # tiles of consecutive blocks are contiguous, in digit order
            for a in range(G):
                if (mask >> a) & 1:
                    vals = bf16_to_float(tiles[nxt][idx])
                    assert np.all(vals == np.round(vals))  # exact small integers
                    assert np.any(vals != 0)  # listed tiles hold a nonzero digit
                    d[a, I * TR:(I + 1) * TR, J * TK:(J + 1) * TK] = vals
                    nxt += 1
            q += 1
    assert nxt == tiles.shape[0] and q == pairs.shape[0]
    return d, rexp


@pytest.mark.parametrize("alpha,gamma,M,rank,tol", [(0.55, 2.0, 512, 0, 1e-10), (0.3, 1.7 / 0.3, 256, 0, 0.0),
                                                    (0.8, 1.5, 128, 12, 0.0), (0.5, 3.0, 128, 0, 1e-10)])
def test_split_digits_reconstruct_rounded_rows(alpha, gamma, M, rank, tol):
    leaf = 32 if gamma == 3.0 else 64
    H = fh.HMatrix(alpha, gamma, 1.0, M, leaf, rank, tol)
    R = H.dense()
    d, rexp = decode(H)
    # digit ranges: balanced digits below the top one, the top one within 129
    assert np.all(d[1:] >= -64) and np.all(d[1:] <= 63)
    assert np.all(np.abs(d[0]) <= 129)
    # the upper triangle (k > m) carries no digit
    assert np.all(d[:, np.triu_indices(M, 1)[0], np.triu_indices(M, 1)[1]] == 0)
    for m in range(M):
        mx = float(np.abs(R[m, :m + 1]).max())
        E = math.frexp(mx)[1] if mx > 0 else 0
        assert rexp[m] == E
        # X = sum_a d_a 2^(7 (6 - a)) as exact Python integers
        X = [sum(int(d[a, m, k]) << (7 * (G - 1 - a)) for a in range(G)) for k in range(m + 1)]
        want = [int(round(math.ldexp(float(R[m, k]), 49 - E))) for k in range(m + 1)]
        assert X == want
        # hence |R~ - X 2^(E - 49)| <= 2^(E - 50), and zero rows stay zero
        err = np.abs(np.array([math.ldexp(x, E - 49) for x in X]) - R[m, :m + 1])
        assert float(err.max()) <= math.ldexp(1.0, E - 50)


def test_split_digit_masks_are_exact():
    """A block's mask bit a is set exactly when one of its entries has a nonzero digit a: the
    decoder above already rejects listed all-zero tiles; here every unlisted tile must be zero."""
    M = 256
    H = fh.HMatrix(0.4, 2.5, 1.0, M, 64, 0, 1e-10)
    R = H.dense()
    tiles, pairs, rexp = H.split_digits()
    d, _ = decode(H)
    # digits recomputed from R~ directly, without the tiles
    full = np.zeros((G, M, M))
    for m in range(M):
        E = int(rexp[m])
        for k in range(m + 1):
            X = int(round(math.ldexp(float(R[m, k]), 49 - E)))
            for a in range(G - 1, 0, -1):
                dg = ((X + 64) & 127) - 64
                full[a, m, k] = dg
                X = (X - dg) >> 7
            full[0, m, k] = X
    assert np.array_equal(d, full)
    q = 0
    for I in range(M // TR):
        for J in range(2 * I + 2):
            blk = full[:, I * TR:(I + 1) * TR, J * TK:(J + 1) * TK]
            want = sum(1 << a for a in range(G) if np.any(blk[a] != 0))
            assert int(pairs[q][0]) == want
            q += 1


@pytest.mark.parametrize("M", [64, 1024, 2048])
def test_split_digits_rejects_unsupported_sizes(M):
    H = fh.HMatrix(0.5, 2.0, 1.0, M, 64 if M >= 128 else 32, 0, 1e-10)
    with pytest.raises(fh.FhmgError):
        H.split_digits()
