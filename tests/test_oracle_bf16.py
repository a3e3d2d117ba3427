"""Pins of the oracle's BF16 storage model (anchor + offset means, BF16
attributes, Morton spatial order): round-to-nearest-even on hand-checked bit
patterns, the nearest-neighbour property on random values, Morton codes of a
grid, and the error bound of the stored means."""
import numpy as np

import oracle
import synth


def test_bf16_rounding_hand_cases():
    """1 + 2^-8 is halfway between 1 and 1 + 2^-7 and rounds to the even
    mantissa (1.0); 1 + 3 2^-8 rounds up to 1 + 2^-6; exact values stay."""
    x = np.float32([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 0.15625, 3.0e38])
    b = oracle.bf16_bits(x)
    assert b.tolist() == [0x3F80, 0x3F80, 0x3F82, 0xC020, 0x3E20, 0x7F62]
    assert oracle.bf16_value(b)[:5].tolist() == [1.0, 1.0, 1 + 2 ** -6, -2.5, 0.15625]


def test_bf16_is_nearest_with_ties_to_even():
    rng = np.random.default_rng(1500)
    x = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-6, 6, 20000)).astype(np.float32)
    b = oracle.bf16_bits(x)
    v = oracle.bf16_value(b).astype(np.float64)
    up = oracle.bf16_value(b.astype(np.uint32) + 1).astype(np.float64)
    dn = oracle.bf16_value(b.astype(np.uint32) - 1).astype(np.float64)
    e = np.abs(x - v)
    assert np.all(e <= np.abs(x - up)) and np.all(e <= np.abs(x - dn))
    assert np.all(e <= np.abs(x) * 2.0 ** -8 + 1e-300)  # half an ulp of an 8-bit significand
    tie = (e == np.abs(x - up)) | (e == np.abs(x - dn))
    assert np.all(b[tie] % 2 == 0)


def test_morton_order_of_a_grid():
    """A 2x2x2 grid of points at the corners of their box: codes interleave x
    (bit 0), y (bit 1), z (bit 2), so the order is x fastest, then y, then z;
    repeated points keep index order."""
    pts = np.array([[x, y, z] for z in (0, 1) for y in (0, 1) for x in (0, 1)], np.float32) * 2.0
    rng = np.random.default_rng(3)
    shuffled = rng.permutation(8)
    perm = oracle.spatial_order(pts[shuffled])
    assert np.array_equal(shuffled[perm], np.arange(8))
    dup = np.array([[1, 1, 1], [0, 0, 0], [1, 1, 1], [0, 0, 0]], np.float32)
    assert oracle.spatial_order(dup).tolist() == [1, 3, 0, 2]
    # a flat axis quantises to 0
    flat = np.array([[0, 5, 1], [1, 5, 0], [0, 5, 0]], np.float32)
    assert oracle.spatial_order(flat).tolist() == [2, 1, 0]


def test_packed_means_error_bound_and_roundtrip():
    """Stored mean = lo + step q with step = chunk extent / 65535: |error| <=
    step / 2 plus FP32 rounding of the product and the sum; chunks in Morton
    order are compact (um steps), in random order they span the room."""
    sc = synth.room_scene(200_000, seed=1005)
    perm = oracle.spatial_order(sc.means)
    anchors, packed = oracle.pack_bf16(sc, perm)
    dec = oracle.unpack_bf16(anchors, packed)
    m = np.asarray(sc.means, np.float32)[perm].astype(np.float64)
    step = anchors[np.arange(sc.n) // oracle.BF16_CHUNK, 3:6].astype(np.float64)
    err = np.abs(dec.means - m)
    assert np.all(err <= 0.5 * step + 2.0 ** -23 * (np.abs(m) + 65535 * step))
    assert err.max() < 1e-4
    a2, p2 = oracle.pack_bf16(sc, None)
    e2 = np.abs(oracle.unpack_bf16(a2, p2).means - np.asarray(sc.means, np.float32))
    assert np.median(e2) > 10 * np.median(err)
    # the box corners are stored exactly: q = 0 at lo, 65535 at hi
    assert packed[:, 0:3].min() == 0 and packed[:, 0:3].max() == 65535
    # other attributes: relative 2^-8 (half an ulp of an 8-bit significand)
    for k in ("log_scales", "quats", "colors"):
        x = np.asarray(getattr(sc, k), np.float32)[perm].astype(np.float64)
        assert np.all(np.abs(getattr(dec, k) - x) <= np.abs(x) * 2.0 ** -8 + 1e-30)
