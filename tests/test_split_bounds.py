"""The bounds the exact tensor-core environment update rests on, checked on the host.

The update splits every FP64 block, scaled by 2^-e with e the smallest exponent such that
|x| < 2^e over the block, into six integer slices of 7 bits: v = a + lo with a = fl32(v) and
lo = fl32(v - a), then slices from a by exact FP32 steps (w *= 2^7, q = rint(w), w -= q),
with lo joining the remainder after the third slice.  This test runs those steps in
NumPy float32/float64 arithmetic (an emulation of the algorithm, not of the kernel, which
the GPU tests compare against the FP64 path) and checks what the kernel relies on:
  * every slice is an integer of magnitude <= 128 (the first), <= 72 (the fourth) or <= 64,
    hence exact in BF16 (8-bit significand: every integer up to 256);
  * the slices reproduce v to below 2^-42 of the block scale;
  * the sum over at most 128 columns of the products of one level i + j (at most six
    pairs) stays below 2^24, so the FP32 accumulator holds it exactly.
"""
import numpy as np

BITS = 7
NSL = 6


def split_block(x):
    """Slices (NSL x shape) and exponent of one block, by the steps described above."""
    m = np.max(np.abs(x))
    e = int(np.frexp(m)[1]) if m > 0 else 0
    v = np.ldexp(x, -e)
    a = v.astype(np.float32)
    lo = (v - a.astype(np.float64)).astype(np.float32)
    w = a.copy()
    out = np.zeros((NSL,) + x.shape, dtype=np.float32)
    for s in range(NSL):
        if s == 3:
            w = (w + lo * np.float32(2.0 ** (3 * BITS))).astype(np.float32)
        w = (w * np.float32(2.0 ** BITS)).astype(np.float32)
        q = np.rint(w).astype(np.float32)
        out[s] = q
        w = (w - q).astype(np.float32)
    return out, e


def blocks(rng):
    yield rng.standard_normal((40, 130))
    # wide dynamic range inside one block
    yield rng.standard_normal((64, 64)) * np.exp(rng.uniform(-30, 5, (64, 64)))
    # values just below a power of two (v rounds to 1.0 in FP32)
    yield np.full((8, 16), 1.0 - 2.0 ** -60) * 3.0
    yield rng.standard_normal((1, 1)) * 1e-200
    yield np.zeros((3, 5))


def test_slices_are_small_integers_and_reproduce_the_block():
    rng = np.random.default_rng(1605)
    for x in blocks(rng):
        d, e = split_block(x)
        assert np.all(d == np.rint(d))
        lim = np.array([128, 64, 64, 72, 64, 64], dtype=np.float32)
        assert np.all(np.abs(d) <= lim[:, None, None])
        recon = sum(d[s].astype(np.float64) * 2.0 ** (-BITS * (s + 1)) for s in range(NSL))
        err = np.max(np.abs(np.ldexp(x, -e) - recon)) if x.size else 0.0
        assert err <= 2.0 ** -42, err


def test_level_sums_stay_below_two_to_the_24():
    rng = np.random.default_rng(1606)
    # worst magnitudes the bounds allow, and random slices of real blocks
    worst = np.array([128, 64, 64, 72, 64, 64], dtype=np.float64)
    for lev in range(NSL):
        pairs = [(i, lev - i) for i in range(lev + 1) if lev - i < NSL]
        bound = 128 * sum(worst[i] * worst[j] for i, j in pairs)
        assert bound < 2 ** 24, (lev, bound)
    a, _ = split_block(rng.standard_normal((128, 128)))
    b, _ = split_block(rng.standard_normal((128, 128)))
    for lev in range(NSL):
        acc = np.zeros((128, 128))
        for i in range(lev + 1):
            j = lev - i
            if j < NSL:
                acc += a[i].astype(np.float64) @ b[j].astype(np.float64).T
        assert np.max(np.abs(acc)) < 2 ** 24
        # the FP32 sum of the same products is exact (an integer below 2^24)
        acc32 = np.zeros((128, 128), dtype=np.float32)
        for i in range(lev + 1):
            j = lev - i
            if j < NSL:
                acc32 += a[i] @ b[j].T
        assert np.array_equal(acc32.astype(np.float64), acc)


def test_levels_rebuild_the_fp64_product():
    """Sum over levels of 2^(eA + eB - 7 (l + 2)) x level sum reproduces A B^T to the
    bound of the dropped terms (pairs i + j >= 6 and the splitting remainders)."""
    rng = np.random.default_rng(1607)
    A = rng.standard_normal((64, 100))
    B = rng.standard_normal((48, 100)) * 1e3
    a, ea = split_block(A)
    b, eb = split_block(B)
    out = np.zeros((64, 48))
    for lev in range(NSL):
        s = np.zeros((64, 48))
        for i in range(lev + 1):
            j = lev - i
            s += a[i].astype(np.float64) @ b[j].astype(np.float64).T
        out += np.ldexp(s, ea + eb - BITS * (lev + 2))
    ref = A @ B.T
    scale = 2.0 ** (ea + eb) * A.shape[1]
    assert np.max(np.abs(out - ref)) <= 8 * 2.0 ** -42 * scale
