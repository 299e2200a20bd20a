"""The assembly's float -> double widening of normal numbers (assemble.cuh,
widen): the high word ((|u| >> 3) + (896 << 20)) | sign and the low word
u << 29 of the double, selected when |u| - 0x00800000 < 0x7f000000 as
unsigned 32-bit values.  Checked here against the IEEE conversion (numpy) on
random bit patterns and on every exponent's edges; the predicate must select
exactly the normal numbers (zeros, subnormals, infinities and NaNs take the
general path)."""
import numpy as np


def fast_bits(u):
    mag = u & np.uint32(0x7FFFFFFF)
    hi = ((mag >> np.uint32(3)).astype(np.uint64) + np.uint64(896 << 20)) | (u & np.uint32(0x80000000)).astype(np.uint64)
    lo = (u.astype(np.uint64) << np.uint64(29)) & np.uint64(0xFFFFFFFF)
    return (hi << np.uint64(32)) | lo


def selected(u):
    mag = u & np.uint32(0x7FFFFFFF)
    return (mag - np.uint32(0x00800000)) < np.uint32(0x7F000000)   # unsigned wrap-around


def test_fast_path_selects_exactly_the_normal_numbers():
    rng = np.random.default_rng(7)
    u = rng.integers(0, 2 ** 32, size=1 << 20, dtype=np.uint64).astype(np.uint32)
    edges = []
    for e in (0, 1, 2, 127, 253, 254, 255):
        for m in (0, 1, 0x7FFFFF, 0x400000):
            for s in (0, 1):
                edges.append((s << 31) | (e << 23) | m)
    u = np.concatenate([u, np.array(edges, dtype=np.uint32)])
    f = u.view(np.float32)
    sel = selected(u)
    assert np.array_equal(sel, np.isfinite(f) & (np.abs(f) >= np.finfo(np.float32).tiny))


def test_fast_path_bits_equal_the_ieee_conversion():
    rng = np.random.default_rng(11)
    u = rng.integers(0, 2 ** 32, size=1 << 21, dtype=np.uint64).astype(np.uint32)
    edges = [(s << 31) | (e << 23) | m for s in (0, 1) for e in (1, 2, 126, 127, 128, 253, 254)
             for m in (0, 1, 2, 3, 7, 8, 0x3FFFFF, 0x7FFFFF)]
    u = np.concatenate([u, np.array(edges, dtype=np.uint32)])
    u = u[selected(u)]
    ref = u.view(np.float32).astype(np.float64).view(np.uint64)
    assert np.array_equal(fast_bits(u), ref)
