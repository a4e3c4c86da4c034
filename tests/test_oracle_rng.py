"""Pins of the oracle's random-number path (CPU only).

* Philox4x32-10 against the cuRAND host-side generator, run as a black-box
  library: for seed S its output block k*65536 + t is Philox of counter
  (k mod 2^32, k >> 32, t, 0) under key (lo32 S, hi32 S); the generator offset
  moves k.  This pins counter words 0-2, both key words and all ten rounds.
* An independent restatement in Python integers (cross-check of the C).
* Box-Muller normals: moments, a Kolmogorov-Smirnov test against Phi, and
  independence of the two members of a pair.
"""
import ctypes
import ctypes.util

import numpy as np
import pytest

import oracle


def _curand():
    for c in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if not c:
            continue
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


def _curand_host_philox(seed: int, offset: int, n: int) -> np.ndarray:
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    g = ctypes.c_void_p()
    rc = lib.curandCreateGeneratorHost(ctypes.byref(g), 161)  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    if rc != 0:
        pytest.skip(f"cuRAND host generator unavailable ({rc})")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(g, ctypes.c_ulonglong(offset)) == 0
        buf = np.empty(n, np.uint32)
        assert lib.curandGenerate(g, buf.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(g)
    return buf


@pytest.mark.parametrize("seed,k0", [(0, 0), (0x0123456789ABCDEF, 0), (0xFEDCBA9876543210, (1 << 32) + 5),
                                     (2**64 - 1, 2**32 - 1)])
def test_philox_matches_curand_host(seed, k0):
    T = 65536
    K = 2
    buf = _curand_host_philox(seed, 4 * T * k0, 4 * T * K).reshape(K, T, 4)
    k = (k0 + np.arange(K, dtype=np.uint64))[:, None] * np.ones(T, dtype=np.uint64)[None, :]
    t = np.broadcast_to(np.arange(T, dtype=np.uint64)[None, :], (K, T))
    ctr = np.stack([k & 0xFFFFFFFF, k >> 32, t, np.zeros_like(t)], axis=-1).astype(np.uint32).reshape(-1, 4)
    key = np.tile(np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32), (ctr.shape[0], 1))
    got = oracle.philox(ctr, key).reshape(K, T, 4)
    assert np.array_equal(got, buf)


# --- independent restatement in Python integers -----------------------------

def _philox_py(ctr, key):
    M0, M1, W0, W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85
    c0, c1, c2, c3 = ctr
    k0, k1 = key
    for r in range(10):
        p0 = M0 * c0
        p1 = M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0), p1 & 0xFFFFFFFF, ((p0 >> 32) ^ c3 ^ k1), p0 & 0xFFFFFFFF
        k0 = (k0 + W0) & 0xFFFFFFFF
        k1 = (k1 + W1) & 0xFFFFFFFF
    return [c0, c1, c2, c3]


def test_philox_python_restatement_all_words():
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2**32, size=(500, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(500, 2), dtype=np.uint64).astype(np.uint32)
    got = oracle.philox(ctr, key)
    for i in range(500):
        assert list(got[i]) == _philox_py([int(v) for v in ctr[i]], [int(v) for v in key[i]])


# --- Box-Muller normals -----------------------------------------------------

@pytest.mark.parametrize("ubits", [32, 23])
def test_normals_moments_and_ks(ubits):
    from scipy import stats
    z = np.concatenate([oracle.normals(11, s, p, 0, 2000, ubits=ubits) for s in range(3) for p in range(20)])
    n = z.size  # 1.44e6
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    kurt = np.mean(z**4) / np.mean(z**2) ** 2
    assert abs(kurt - 3.0) < 5 * np.sqrt(96.0 / n)
    assert stats.kstest(z[:200000], "norm").pvalue > 1e-4
    pairs = z.reshape(-1, 2)
    r = np.corrcoef(pairs[:, 0], pairs[:, 1])[0, 1]
    assert abs(r) < 5 / np.sqrt(pairs.shape[0])
    # independence of squares too (catches r shared across the pair wrongly)
    r2 = np.corrcoef(pairs[:, 0] ** 2, pairs[:, 1] ** 2)[0, 1]
    assert abs(r2) < 5 / np.sqrt(pairs.shape[0])


def test_normals_block_layout():
    """Block b of path (s,p) uses counters (3b+i, p, s, tag); pair i takes
    words (2i, 2i+1) with cosine first (restated here with numpy)."""
    seed, s, p, b = 0x1234_5678_9ABC_DEF0, 5, 77, 9
    key = np.array([[seed & 0xFFFFFFFF, seed >> 32]] * 3, dtype=np.uint32)
    ctr = np.array([[3 * b + i, p, s, 0] for i in range(3)], dtype=np.uint32)
    w = oracle.philox(ctr, key).ravel().astype(np.float64)
    u = (w + 0.5) * 2.0**-32
    r = np.sqrt(-2 * np.log(u[0::2]))
    zz = np.empty(12)
    zz[0::2] = r * np.cos(2 * np.pi * u[1::2])
    zz[1::2] = r * np.sin(2 * np.pi * u[1::2])
    got = oracle.normals(seed, s, p, b, 1)
    np.testing.assert_allclose(got, zz, rtol=0, atol=1e-14)
