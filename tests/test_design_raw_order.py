"""The bit identities behind the raw-bit compares of round 1 and the level-0
contraction, checked on the CPU against the oracle's own order key (pinned by
test_order_key_total_order): for FP32 weights whose sign bit is clear,

- raw bits compare as unsigned integers in the order of their minimax keys,
  and the key is the raw pattern with its top bit set;
- for the widest order the key is the complement of the raw pattern with its
  top bit cleared, so the complemented raw bits compare in key order;

and a single weight with its sign bit set (-0.0 included) breaks the first
identity, which is why one such weight sends the kernels back to keys."""
import numpy as np

import oracle


def _patterns(rng, count):
    """Non-negative FP32 bit patterns: +0, subnormals, normals, +inf, NaNs."""
    special = np.array([0x00000000, 0x00000001, 0x007FFFFF, 0x00800000, 0x3F800000, 0x7F7FFFFF,
                        0x7F800000, 0x7F800001, 0x7FC00000, 0x7FFFFFFF], dtype=np.uint32)
    rnd = rng.integers(0, 1 << 31, size=count, dtype=np.uint64).astype(np.uint32)
    return np.concatenate([special, rnd])


def _keys(bits, widest):
    dt = oracle.F32 | (oracle.WIDEST if widest else 0)
    return np.array([oracle.order_key(int(b), dt) for b in bits], dtype=np.uint64)


def test_minimax_keys_of_non_negative_floats_are_raw_bits_with_the_top_bit():
    rng = np.random.default_rng(11)
    bits = _patterns(rng, 3000)
    k = _keys(bits, widest=False)
    assert np.array_equal(k, bits.astype(np.uint64) | 0x80000000)
    # the same order: sorting by raw bits sorts by key
    order = np.argsort(bits, kind="stable")
    assert np.all(np.diff(k[order].astype(np.int64)) >= 0)


def test_widest_keys_of_non_negative_floats_are_complemented_raw_bits():
    rng = np.random.default_rng(12)
    bits = _patterns(rng, 3000)
    k = _keys(bits, widest=True)
    comp = (~bits).astype(np.uint64) & 0xFFFFFFFF
    assert np.array_equal(k, comp & 0x7FFFFFFF)
    order = np.argsort(comp, kind="stable")
    assert np.all(np.diff(k[order].astype(np.int64)) >= 0)


def test_a_sign_bit_breaks_the_raw_order():
    # -0.0 and -1.0 sit below +0.0 in key order but above every
    # non-negative float as raw unsigned bits
    for neg in (0x80000000, 0xBF800000):
        kn = oracle.order_key(neg, oracle.F32)
        kz = oracle.order_key(0x00000000, oracle.F32)
        assert kn < kz and neg > 0x7FFFFFFF
