"""The exact 0/1 arithmetic the tensor-core subset test relies on (CPU).

The tcgen05 kernels (subset_tc.cu) test p inside r as a 0/1 GEMM of kind
f8f6f4: D[p, r] = sum over items l of p_l * (1 - r_l) counts the items of p
missing from r, so p is inside r exactly when D = 0.  The operands are E4M3
bytes: 0x38 (1.0) for a set item in the dense form, 0x08 (2^-6) in the fused
form, where each product is 2^-12.  With at most 512 items per test (K <= 8
words) every partial sum is a multiple of 2^-12 below 2^-3, exact in the FP32
accumulator in any order, and D = 0 only when no item is missing.

Checked here from the E4M3 definition (1 sign, 4 exponent bits with bias 7,
3 mantissa bits; subnormals at exponent 0) and IEEE float32 sums in numpy:
the two operand bytes, the exactness of every count up to 512 under
shuffled accumulation orders, the complement identity on random itemsets,
and the fused kernel's spread of four items into four operand bytes by one
multiply and one mask.
"""
import numpy as np
import pytest


def e4m3(byte: int) -> float:
    s = -1.0 if byte & 0x80 else 1.0
    e, m = (byte >> 3) & 0xF, byte & 0x7
    if e == 0:
        return s * (m / 8.0) * 2.0 ** (1 - 7)
    return s * (1.0 + m / 8.0) * 2.0 ** (e - 7)


def test_operand_bytes():
    assert e4m3(0x38) == 1.0
    assert e4m3(0x08) == 2.0 ** -6
    assert e4m3(0x00) == 0.0
    assert np.float32(e4m3(0x08)) * np.float32(e4m3(0x08)) == np.float32(2.0 ** -12)


@pytest.mark.parametrize("unit", [1.0, 2.0 ** -12])
def test_counts_up_to_512_are_exact_in_fp32(unit):
    rng = np.random.default_rng(7)
    for count in list(range(0, 40)) + [255, 256, 257, 511, 512]:
        terms = np.zeros(512, np.float32)
        terms[:count] = np.float32(unit)
        for _ in range(4):
            acc = np.float32(0.0)
            for t in rng.permutation(terms):
                acc = np.float32(acc + t)
            assert acc == np.float32(count * unit)
            assert (acc == 0) == (count == 0)


def test_complement_counts_missing_items():
    rng = np.random.default_rng(8)
    for _ in range(200):
        L = int(rng.choice([64, 256, 512]))
        p = rng.random(L) < rng.uniform(0.01, 0.3)
        r = rng.random(L) < rng.uniform(0.1, 0.9)
        if rng.random() < 0.3:
            r |= p                                   # make p inside r
        A = np.where(p, np.float32(e4m3(0x08)), np.float32(0))
        B = np.where(r, np.float32(0), np.float32(e4m3(0x08)))   # complemented record
        D = np.float32(0)
        for a, b in zip(A, B):
            D = np.float32(D + a * b)
        missing = int((p & ~r).sum())
        assert D == np.float32(missing * 2.0 ** -12)
        assert (D == 0) == bool(np.all(~p | r))


def spread_nibble(n: int) -> int:
    """The fused kernel's expansion of 4 items into 4 E4M3 bytes (uint32)."""
    return (n * 0x01020408) & 0x08080808 & 0xFFFFFFFF


def test_nibble_spread_gives_one_byte_per_item():
    for n in range(16):
        v = spread_nibble(n)
        assert [(v >> (8 * b)) & 0xFF for b in range(4)] == \
            [0x08 if (n >> b) & 1 else 0x00 for b in range(4)]
        # the shifted copies of n do not overlap, so the product has no carries
        assert n * 0x01020408 == sum(n << s for s in (3, 10, 17, 24)) < 1 << 32
