"""The NCP sweep skips an element without dividing when p < (K (1 - 2^-20)) * d
in FP32 (K the current threshold key, d the degree): the claim is that such
an element's key RN(p / d) is below K, so skipping never drops a candidate.

Checked here in IEEE FP32 arithmetic (numpy's float32 products and quotients
round to nearest, as the kernel's __fmul_rn / __fdiv_rn do): the condition
under which the kernel applies the test (K (1 - 2^-20) normal, the product
finite) and random keys over many octaves, plus adversarial elements placed
just below the cut.
"""
import numpy as np

F32 = np.float32
C = F32(1.0) - F32(2.0) ** -20          # 1 - 2^-20, exact in FP32
FLT_MIN = np.finfo(np.float32).tiny


def _rejects(p, d, K):
    kc = F32(K) * C
    if not kc >= FLT_MIN:
        return np.zeros_like(p, dtype=bool)
    lim = kc * d.astype(np.float32)
    return np.isfinite(lim) & (p < lim)


def test_random_keys_over_many_octaves():
    rng = np.random.default_rng(2021)
    rejected = 0
    for _ in range(20):
        n = 200_000
        p = (rng.random(n) * 2.0 ** rng.integers(-60, 10, n)).astype(np.float32)
        p[p == 0] = F32(1e-30)
        d = rng.integers(1, 1 << 22, n).astype(np.uint32)
        kp, kd = F32(rng.random() * 2.0 ** rng.integers(-60, 10)), F32(rng.integers(1, 1 << 20))
        K = kp / kd
        rej = _rejects(p, d, K)
        keys = p / d.astype(np.float32)
        assert np.all(keys[rej] < K)
        rejected += int(rej.sum())
    assert rejected > 0  # the test exercises the skip


def test_adversarial_elements_just_below_the_cut():
    rng = np.random.default_rng(7)
    K = (F32(0.3) / F32(7.0))
    d = rng.integers(1, 1 << 20, 100_000).astype(np.uint32)
    df = d.astype(np.float64)
    for rel in (1 - 2.0 ** -19, 1 - 2.0 ** -20, 1 - 2.0 ** -21, 1 - 2.0 ** -22, 1 - 2.0 ** -24, 1.0):
        p = (float(K) * df * rel).astype(np.float32)  # p / d within a few ulps of K
        for step in (-2, -1, 0, 1, 2):
            pp = np.nextafter(p, np.float32(np.inf) if step > 0 else np.float32(0), dtype=np.float32) \
                if step != 0 else p
            rej = _rejects(pp, d, K)
            keys = pp / d.astype(np.float32)
            assert np.all(keys[rej] < K)
            if rel <= 1 - 2.0 ** -19 and step <= 0:
                assert rej.all()  # far enough below the cut: every element is skipped
