"""The orderings the kernels rely on, checked on the encodings themselves
(re-expressed here with numpy bit views):

- the NCP profile takes a minimum of FP64 conductances with an unsigned
  64-bit atomic minimum, through the map b -> (b >> 63) ? ~b : b | 2^63 of the
  double's bit pattern b, which must order as the doubles do (negatives
  included: a directed graph can give a negative cut);
- the NCP sweep orders vertices by the 64-bit key ((~(bits(key) + 1)) << 32 | v)
  for FP32 keys >= 0, whose ascending order must be key descending, then id
  ascending (key 0.0 included: a positive p can give a key that rounds to 0).
"""
import numpy as np


def _dbl_enc(x):
    b = np.asarray(x, dtype=np.float64).view(np.uint64)
    sign = (b >> np.uint64(63)).astype(bool)
    return np.where(sign, ~b, b | np.uint64(1 << 63))


def test_double_map_orders_as_the_doubles():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(100_000) * 10.0 ** rng.integers(-300, 300, 100_000),
                        [0.0, -0.0, np.inf, -np.inf, 1.0, -1.0, 5e-324, -5e-324, 1 / 7, 0.5]])
    x = x[np.isfinite(x) | np.isinf(x)]
    order_x = np.argsort(x, kind="stable")
    enc = _dbl_enc(x)
    xs, es = x[order_x], enc[order_x]
    # strictly increasing doubles give strictly increasing codes (-0.0 and 0.0 aside)
    strict = xs[1:] > xs[:-1]
    assert np.all(es[1:][strict] > es[:-1][strict])


def _sort_key(key, v):
    enc = key.astype(np.float32).view(np.uint32).astype(np.uint64) + np.uint64(1)
    return ((~enc) & np.uint64(0xFFFFFFFF)) << np.uint64(32) | v.astype(np.uint64)


def test_sweep_key_orders_by_key_then_id():
    rng = np.random.default_rng(2)
    n = 50_000
    key = (rng.random(n) * 2.0 ** rng.integers(-140, 20, n)).astype(np.float32)
    key[:500] = 0.0                      # keys that round to zero
    key[500:1500] = np.float32(0.125)    # exact ties
    v = rng.permutation(n).astype(np.uint32)
    got = np.argsort(_sort_key(key, v), kind="stable")
    exp = np.lexsort((v, -key.astype(np.float64)))  # key descending, then id ascending
    assert np.array_equal(got, exp)
