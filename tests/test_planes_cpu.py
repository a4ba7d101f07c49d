"""The bit-plane build of the large-window strategy, emulated on the CPU:
32 lanes each pack one column of 32 / NB consecutive rows into a word, a
warp-wide 32x32 bit transpose (five rounds of lane-pair exchanges, as the
kernel's warp_transpose32 does with shuffles) leaves in lane q * NB + b the
plane word of bit b of row q, and that word must equal the ballot definition
of a bit plane: bit l set iff bit b of the pixel in column l is set."""
import numpy as np
import pytest

MASKS = (0x0000FFFF, 0x00FF00FF, 0x0F0F0F0F, 0x33333333, 0x55555555)


def transpose32(x):
    """x: 32 uint32 lane words; returns the lane words after the five rounds."""
    x = x.astype(np.uint64)
    lanes = np.arange(32)
    for i, m in enumerate(MASKS):
        s = 16 >> i
        y = x[lanes ^ s]
        hi = (lanes & s) != 0
        keep_hi = (x & ~np.uint64(m) & np.uint64(0xFFFFFFFF)) | ((y >> np.uint64(s)) & np.uint64(m))
        keep_lo = (x & np.uint64(m)) | ((y << np.uint64(s)) & ~np.uint64(m) & np.uint64(0xFFFFFFFF))
        x = np.where(hi, keep_hi, keep_lo)
    return x.astype(np.uint32)


def test_transpose_is_the_bit_matrix_transpose():
    rng = np.random.default_rng(7)
    for _ in range(50):
        x = rng.integers(0, 2**32, 32, dtype=np.uint64).astype(np.uint32)
        bits = (x[:, None] >> np.arange(32, dtype=np.uint32)[None, :]) & 1   # bits[l, j] = bit j of lane l
        t = transpose32(x)
        want = (bits.T.astype(np.uint64) << np.arange(32, dtype=np.uint64)[None, :]).sum(axis=1)
        assert np.array_equal(t, want.astype(np.uint32))


@pytest.mark.parametrize("nb", [8, 16])
def test_packed_rows_give_the_ballot_planes(nb):
    rng = np.random.default_rng(nb)
    p = 32 // nb
    px = rng.integers(0, 2**nb, (p, 32), dtype=np.uint64)           # rows x columns of one 32-column word
    x = np.zeros(32, dtype=np.uint64)
    for j in range(p):
        x |= px[j] << np.uint64(nb * j)
    t = transpose32(x.astype(np.uint32))
    for lane in range(32):
        b, q = lane % nb, lane // nb
        want = sum(int((px[q, l] >> b) & 1) << l for l in range(32))
        assert int(t[lane]) == want, (lane, b, q)
