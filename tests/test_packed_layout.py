"""Host-side check of the packed-triangle digit layout of the Cholesky vectors (no GPU).

The layout stores, for every b^L, the lower 128 x 128 tiles (I >= J) of its full 128-row blocks,
the diagonal tiles whole, as 8 K blocks of 128 rows x 16 (tile (I, J) of L at index
L T + I(I+1)/2 + J, T = nb1(nb1+1)/2), and the rows past the last whole block whole (rows (L, j)
of all X r, K-blocked with the row count padded to 384).  This test restates that storage order
and the three tile reads of the half transform (a stored tile as is, a stored tile transposed,
the ragged rows transposed), with the coordinates the loading thread computes once per tile,
and checks that every stage of every row tile sees b^L(mu, nu) in the orientation its MMA reads,
for sizes with no whole block, whole blocks only, and 1 to 127 ragged rows."""
import numpy as np
import pytest

BK, BM, ROWPAD = 16, 128, 384


def _storage(B):
    """Tile and ragged-row arrays of one digit plane, in the kernels' storage order."""
    X, n, _ = B.shape
    nb1 = n // 128
    T = nb1 * (nb1 + 1) // 2
    n1, r = 128 * nb1, n - 128 * nb1
    # tiles: [X*T tiles][8 K blocks][128 rows][16]
    tiles = np.zeros((X * T, 8, 128, 16))
    for L in range(X):
        for I in range(nb1):
            for J in range(I + 1):
                blk = B[L, 128 * I:128 * I + 128, 128 * J:128 * J + 128]     # rows mu, cols nu
                tiles[L * T + I * (I + 1) // 2 + J] = blk.reshape(128, 8, 16).transpose(1, 0, 2)
    rpad = (X * r + ROWPAD - 1) // ROWPAD * ROWPAD if r else 0
    nkb = (n + BK - 1) // BK
    rag = np.zeros((nkb, rpad, 16))            # [K block][rows (L, j)][16]
    for L in range(X):
        rows = np.zeros((r, nkb * BK))
        rows[:, :n] = B[L, n1:, :]
        rag[:, L * r:L * r + r, :] = rows.reshape(r, nkb, 16).transpose(1, 0, 2)
    return tiles.reshape(-1, 16), rag, nb1, T, r, rpad, nkb


def _box_direct(flat_rows, y):
    """3D box {16, 128} at row y of the K-blocked rows: A[m][k] = row y + m, column k."""
    return flat_rows[y:y + 128]


def _box_mn(planes, rpad, y, z):
    """4D box {16, 16, 8} at (0, y, z) of dims {16, rpad, nkb}, read MN-major:
    A[m][k] with m = 16 kb' + c (stored K) and k = stored row y + k."""
    A = np.zeros((128, 16))
    nkb = planes.shape[0] // rpad
    for kb2 in range(8):
        if z + kb2 >= nkb:
            continue
        blk = planes[(z + kb2) * rpad + y:(z + kb2) * rpad + y + 16]   # [16 rows][16]
        rows = min(16, max(0, rpad - y))
        A[kb2 * 16:kb2 * 16 + 16, :rows] = blk[:rows].T
    return A


@pytest.mark.parametrize("n", [100, 129, 256, 300, 383])
def test_packed_tiles_feed_every_stage(n):
    rng = np.random.default_rng(n)
    X = 3
    B = rng.standard_normal((X, n, n))
    B = B + B.transpose(0, 2, 1)
    tiles, rag, nb1, T, r, rpad, nkb_r = _storage(B)
    rag_flat = rag.reshape(-1, 16)
    kb_total = (n + BK - 1) // BK
    for L in range(X):
        for R in range(nb1):
            # per-tile coordinates of the loading thread
            pk_row = (L * T + R * (R + 1) // 2) * 8
            pk_col = L * T + R
            pk_rag = L * r - 8 * nb1 * BK
            for kb in range(kb_total):
                J = kb >> 3
                if J <= R:
                    A = _box_direct(tiles, (pk_row + kb) * BM)
                elif J < nb1:
                    A = _box_mn(tiles, 128, (kb & 7) * BK, (pk_col + J * (J + 1) // 2) * 8)
                else:
                    A = _box_mn(rag_flat, rpad, pk_rag + kb * BK, R * (BM // BK))
                # the stage is MN-major exactly from K block 8 (R + 1) on
                assert (kb >= 8 * (R + 1)) == (J > R)
                nu = 16 * kb + np.arange(16)
                ok = nu < n
                want = B[L, 128 * R:128 * R + 128][:, nu[ok]]
                assert np.array_equal(A[:, ok], want)
    # the ragged rows as the rows of their own product (K-major, rows (L, j))
    for L in range(X):
        for j in range(r):
            row = np.concatenate([rag[kb, L * r + j] for kb in range(nkb_r)])[:n]
            assert np.array_equal(row, B[L, 128 * nb1 + j])


@pytest.mark.parametrize("n", [100, 1200])
def test_packed_bytes(n):
    """Digits held per L: T tiles of 128 x 128 plus r ragged rows of n, against n rows of n."""
    nb1 = n // 128
    T, r = nb1 * (nb1 + 1) // 2, n - 128 * nb1
    packed, full = T * 128 * 128 + r * n, n * n
    assert packed <= full
    if n == 1200:   # 45 tiles and 48 ragged rows: 0.55 of the full rows
        assert (T, r) == (45, 48) and abs(packed / full - 0.552) < 1e-3
