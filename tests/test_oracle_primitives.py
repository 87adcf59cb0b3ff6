"""Pins of the oracle's primitives against things other than itself:
library primality tests, brute force on small moduli, the convolution
theorem against schoolbook negacyclic products, the cuRAND Philox generator,
high-precision recomputation of the Gaussian table, and the evaluation-point
definition of the Galois automorphism."""
import ctypes
import math
import os

import numpy as np
import pytest
import sympy

import oracle

# ---------------------------------------------------------------- primes


@pytest.mark.parametrize("bits,log_n,count", [(30, 6, 4), (40, 12, 8), (50, 16, 6), (60, 16, 4)])
def test_primes_are_the_first_ntt_primes_below_2_to_bits(bits, log_n, count):
    two_n = 2 << log_n
    ps = oracle.gen_primes(bits, log_n, count)
    assert len(ps) == count
    # every candidate k*2N+1 between 2^bits and the last prime is tested with sympy:
    # the kept ones are exactly the primes, in decreasing order
    k = ((1 << bits) - 2) // two_n
    expect = []
    while len(expect) < count:
        q = k * two_n + 1
        if sympy.isprime(q):
            expect.append(q)
        k -= 1
    assert ps == expect
    assert all(p < (1 << bits) and p % two_n == 1 for p in ps)


def test_special_primes_skip_the_limbs():
    limbs = oracle.gen_primes(40, 10, 3)
    sp = oracle.gen_primes(40, 10, 2, exclude=limbs)
    assert not set(sp) & set(limbs)
    assert sp == oracle.gen_primes(40, 10, 5)[3:]


def test_miller_rabin_vs_sympy():
    rng = np.random.default_rng(1)
    cands = [int(x) | 1 for x in rng.integers(1 << 40, 1 << 62, 400, dtype=np.int64)]
    # Carmichael numbers and strong pseudoprimes to small bases
    cands += [561, 1105, 1729, 2047, 1373653, 25326001, 3215031751, 2152302898747,
              3474749660383, 341550071728321, 3825123056546413051, (1 << 61) - 1]
    for n in cands:
        assert oracle.is_prime(n) == sympy.isprime(n), n


# ---------------------------------------------------------------- roots


def test_min_root_brute_force_small_moduli():
    for log_n in (2, 3, 4, 5):
        for q in oracle.gen_primes(16, log_n, 3):
            n = 1 << log_n
            brute = next(x for x in range(2, q) if pow(x, n, q) == q - 1)
            assert oracle.min_root(q, log_n) == brute


@pytest.mark.parametrize("bits,log_n", [(40, 12), (60, 16)])
def test_min_root_is_a_primitive_2n_th_root(bits, log_n):
    q = oracle.gen_primes(bits, log_n, 1)[0]
    psi = oracle.min_root(q, log_n)
    n = 1 << log_n
    assert pow(psi, n, q) == q - 1 and pow(psi, 2 * n, q) == 1


def test_min_root_is_the_least_among_all_roots_of_x_n_plus_1():
    log_n = 6
    q = oracle.gen_primes(30, log_n, 1)[0]
    roots = sympy.ntheory.residue_ntheory.nthroot_mod(q - 1, 1 << log_n, q, all_roots=True)
    assert len(roots) == 1 << log_n
    assert oracle.min_root(q, log_n) == min(roots)


# ---------------------------------------------------------------- NTT


def schoolbook_negacyclic(a, b, q):
    n = len(a)
    out = [0] * n
    for i in range(n):
        for j in range(n):
            k = i + j
            if k < n:
                out[k] += int(a[i]) * int(b[j])
            else:
                out[k - n] -= int(a[i]) * int(b[j])
    return [x % q for x in out]


@pytest.mark.parametrize("log_n", [2, 3, 4, 5, 6, 7, 8])
def test_ntt_definition_gives_negacyclic_convolution(log_n):
    q = oracle.gen_primes(40, log_n, 1)[0]
    psi = oracle.min_root(q, log_n)
    rng = np.random.default_rng(log_n)
    a = rng.integers(0, q, 1 << log_n, dtype=np.uint64)
    b = rng.integers(0, q, 1 << log_n, dtype=np.uint64)
    A = oracle.ntt_def(a, log_n, q, psi)
    B = oracle.ntt_def(b, log_n, q, psi)
    C = np.array([(int(x) * int(y)) % q for x, y in zip(A, B)], dtype=np.uint64)
    c = oracle.intt_def(C, log_n, q, psi)
    assert [int(x) for x in c] == schoolbook_negacyclic(a, b, q)


@pytest.mark.parametrize("log_n", [1, 2, 5, 8, 10])
def test_radix2_matches_definition(log_n):
    q = oracle.gen_primes(59, log_n, 1)[0]
    psi = oracle.min_root(q, log_n)
    a = np.random.default_rng(7).integers(0, q, 1 << log_n, dtype=np.uint64)
    A = oracle.ntt_def(a, log_n, q, psi)
    assert np.array_equal(oracle.ntt_r2(a, log_n, q, psi), A)
    assert np.array_equal(oracle.intt_r2(A, log_n, q, psi), a)
    assert np.array_equal(oracle.intt_def(A, log_n, q, psi), a)


def test_ntt_evaluates_at_the_odd_powers():
    # the NTT of a polynomial evaluated directly (Horner, Python ints) at each
    # odd power psi^e lands in slot j with e = 2 brv(j) + 1
    log_n = 5
    n = 1 << log_n
    q = oracle.gen_primes(40, log_n, 1)[0]
    psi = oracle.min_root(q, log_n)
    a = [int(x) for x in np.random.default_rng(3).integers(0, q, n, dtype=np.uint64)]
    A = oracle.ntt_def(np.array(a, dtype=np.uint64), log_n, q, psi)
    for j in range(n):
        e = 2 * int(format(j, f"0{log_n}b")[::-1], 2) + 1
        x = pow(psi, e, q)
        v = 0
        for c in reversed(a):
            v = (v * x + c) % q
        assert int(A[j]) == v


# ---------------------------------------------------------------- Philox


def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so"):
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    return None


@pytest.mark.parametrize("seed", [0, 0x0123456789ABCDEF, 42])
def test_philox_matches_curand_host_generator(seed):
    # cuRAND's host Philox4x32-10 generator emits block b from the counter
    # (b // 65536, 0, b % 65536, 0) under the key (seed low, seed high); the
    # blocks around 65536 exercise the first counter word as well.
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    count = 4 * (65536 + 16)
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(count, dtype=np.uint32)
        assert lib.curandGenerate(gen, ctypes.c_void_p(out.ctypes.data),
                                  ctypes.c_size_t(count)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    blocks = out.reshape(-1, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for b in list(range(16)) + list(range(65536, 65552)) + [777, 40000]:
        want = [int(x) for x in blocks[b]]
        assert [int(x) for x in oracle.philox([b // 65536, 0, b % 65536, 0], key)] == want, b


def test_philox_zero_block():
    # Philox4x32-10 of the all-zero counter under the all-zero key
    assert [int(x) for x in oracle.philox([0, 0, 0, 0], [0, 0])] == [
        0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]


# ---------------------------------------------------------------- samplers


def test_gauss_table_vs_high_precision():
    import mpmath
    mpmath.mp.prec = 200
    sigma = 3.2
    T = oracle.gauss_table(sigma)
    K = math.ceil(6 * sigma)
    assert len(T) == K
    rho = [mpmath.exp(-mpmath.mpf(k * k) / (2 * mpmath.mpf(sigma) ** 2)) for k in range(K + 1)]
    z = rho[0] + 2 * sum(rho[1:])
    cum = rho[0]
    for k in range(K):
        if k:
            cum += 2 * rho[k]
        exact = int(mpmath.floor(cum / z * mpmath.mpf(2) ** 64))
        assert abs(int(T[k]) - exact) <= 1 << 13  # double precision of the cumulative sum
    assert all(int(T[k]) < int(T[k + 1]) for k in range(K - 1))


def test_gaussian_moments():
    x = oracle.sample(0, "gauss", sid=5, dom=3, count=200000)
    assert abs(x.mean()) < 0.03
    assert abs(x.var() - 3.2 ** 2) < 0.15
    assert np.abs(x).max() <= 20
    # symmetric: P(x = k) ~ P(x = -k)
    assert abs(np.mean(x > 0) - np.mean(x < 0)) < 0.01


def test_ternary_is_uniform():
    x = oracle.sample(0, "ternary", sid=0, dom=1, count=300000)
    counts = np.array([(x == v).sum() for v in (-1, 0, 1)])
    assert counts.sum() == len(x)
    chi2 = ((counts - len(x) / 3) ** 2 / (len(x) / 3)).sum()
    assert chi2 < 13.8  # 99.9% quantile, 2 degrees of freedom


def test_uniform_residues():
    q = oracle.gen_primes(60, 12, 1)[0]
    x = oracle.sample(3, "uniform", sid=1, dom=2, count=100000, limb=2, q=q).astype(np.uint64)
    assert int(x.max()) < q
    assert abs(float(np.mean(x.astype(np.float64))) / q - 0.5) < 0.005
    # wiring: the residue is the 128-bit word of that counter's block mod q
    w = oracle.philox([17, 2, 1, 2], [3, 0])
    v = (int(w[3]) << 96) | (int(w[2]) << 64) | (int(w[1]) << 32) | int(w[0])
    assert int(x[17]) == v % q


# ---------------------------------------------------------------- automorphism


def test_galois_elements():
    log_n = 10
    m = 2 << log_n
    for r in (0, 1, 2, 5, 100, -1, -3):
        k = oracle.galois_elt(log_n, r)
        assert k == pow(5, r % (1 << (log_n - 1)), m)
    assert oracle.galois_elt(log_n, 1 << (log_n - 1)) == 1


def test_automorphism_coefficient_form_by_evaluation():
    # a(X^k) evaluated at x equals a evaluated at x^k, for the roots of X^N + 1
    log_n = 5
    n = 1 << log_n
    q = oracle.gen_primes(40, log_n, 1)[0]
    psi = oracle.min_root(q, log_n)
    a = [int(v) for v in np.random.default_rng(9).integers(0, q, n, dtype=np.uint64)]
    for k in (5, 25, 2 * n - 1, 3):
        b = [int(v) for v in oracle.automorph_coef(np.array(a, dtype=np.uint64), log_n, q, k)]
        for e in (1, 3, 7, 2 * n - 1):
            x = pow(psi, e, q)
            lhs = sum(c * pow(x, i, q) for i, c in enumerate(b)) % q
            rhs = sum(c * pow(x, i * k, q) for i, c in enumerate(a)) % q
            assert lhs == rhs


def test_automorphism_evaluation_form_is_the_transformed_coefficient_form():
    o = oracle.Oracle(6, 2, 30, 1, 40, 2.0 ** 20)
    rng = np.random.default_rng(4)
    coef = np.stack([rng.integers(0, q, o.n, dtype=np.uint64) for q in o.primes[:2]])
    ev = np.stack([oracle.ntt_def(coef[t], o.log_n, o.primes[t], o.roots[t]) for t in range(2)])
    for k in (5, 25, 3, 2 * o.n - 1):
        got = o.automorph(ev, 2, k)
        for t in range(2):
            want = oracle.ntt_def(oracle.automorph_coef(coef[t], o.log_n, o.primes[t], k),
                                  o.log_n, o.primes[t], o.roots[t])
            assert np.array_equal(got[t], want)
