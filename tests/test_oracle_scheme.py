"""Pins of the oracle's scheme-level functions: exact big-integer checks of
encryption, basis conversion, rescaling and key switching on tiny rings, the
homomorphism property (Eq. 1-2) against FP64, the canonical-embedding encoder
against numpy's FFT and a closed form, and the logistic-regression step
against the FP64 update of Eq. 5-8 with the Table 2 polynomial."""
import math

import numpy as np
import pytest

import oracle
import paper_2006_10091_gb300 as he
from paper_2006_10091_gb300 import workloads
from tests.lr_reference import lr_step_fp64, table2

# ------------------------------------------------------------------ helpers


def to_coef(o, polys, nlimbs):
    """Evaluation form -> coefficient residues, limb by limb, by the O(N^2)
    inverse definition."""
    return np.stack([oracle.intt_def(polys[t], o.log_n, o.primes[t], o.roots[t])
                     for t in range(nlimbs)])


def to_eval(o, coef, prime_indices):
    return np.stack([oracle.ntt_def(coef[i], o.log_n, o.primes[t], o.roots[t])
                     for i, t in enumerate(prime_indices)])


def crt(residues, primes):
    """Integer in [0, prod) with the given residues (Python ints)."""
    Q = math.prod(primes)
    x = 0
    for r, q in zip(residues, primes):
        Qi = Q // q
        x += int(r) * Qi * pow(Qi, -1, q)
    return x % Q


def centered(x, Q):
    return x - Q if x > Q // 2 else x


def negacyclic(a, b):
    n = len(a)
    out = [0] * n
    for i in range(n):
        if a[i] == 0:
            continue
        for j in range(n):
            k = i + j
            if k < n:
                out[k] += a[i] * b[j]
            else:
                out[k - n] -= a[i] * b[j]
    return out


@pytest.fixture(scope="module")
def tiny():
    # N = 32, six 30-bit limbs, two 40-bit special primes: digits of two limbs
    return oracle.Oracle(5, 6, 30, 2, 40, 2.0 ** 20, seed=11, rot_steps=[1, 3, -1])


# ------------------------------------------------------------------ encode


def test_encode_matches_numpy_fft():
    o = oracle.Oracle(8, 2, 30, 1, 40, 2.0 ** 30)
    rng = np.random.default_rng(0)
    z = rng.uniform(-1, 1, o.n // 2) + 1j * rng.uniform(-1, 1, o.n // 2)
    raw = o.encode_raw(z.real, z.imag, scale=2.0 ** 30)
    # slot j sits at the 2N-th root of unity exp(i pi e_j / N), e_j = 5^j mod 2N, its
    # conjugate at 2N - e_j; the coefficients are (Delta/N) Re(DFT_2N(v))[i]
    m = 2 * o.n
    v = np.zeros(m, dtype=complex)
    for j in range(o.n // 2):
        e = pow(5, j, m)
        v[e] = z[j]
        v[m - e] = np.conj(z[j])
    want = (2.0 ** 30 / o.n) * np.fft.fft(v)[: o.n].real
    assert np.max(np.abs(raw - want)) < 1e-5
    coeffs = o.encode(z.real, z.imag, scale=2.0 ** 30)
    assert np.array_equal(coeffs, np.round(raw).astype(np.int64)) or \
        np.max(np.abs(coeffs - raw)) <= 0.5 + 1e-9


def test_encode_decode_roundtrip():
    o = oracle.Oracle(10, 2, 40, 1, 60, 2.0 ** 40)
    z = workloads.uniform_slots(1, o.n // 2)
    m = o.encode(z)
    re, im = o.decode(m.astype(np.float64), 2.0 ** 40)
    assert np.max(np.abs(re - z)) < 2.0 ** -(40 - 10 - 2)
    assert np.max(np.abs(im)) < 2.0 ** -(40 - 10 - 2)


@pytest.mark.parametrize("g,logms", [(1, 40), (2, 40), (4, 40), (8, 40), (8, 27), (4, 27), (8, 30)])
def test_mask_encoding_closed_form(g, logms):
    """The mask (1 on slots = 0 mod g) encodes to the polynomial with
    coefficient (Delta/g) cos(pi i / N) at i = 0 mod N/(2g) and 0 elsewhere:
    the slot positions = 0 mod g are the 2N-th roots exp(i pi t/N) with
    t = +-1 mod 4g, and summing over that coset leaves only those terms."""
    import mpmath
    mpmath.mp.prec = 120
    log_n = 11
    o = oracle.Oracle(log_n, 2, 40, 1, 60, 2.0 ** 40)
    ms = 2.0 ** logms
    got = o.lr_mask(g, ms)
    step = o.n // (2 * g)
    for i in range(o.n):
        if i % step:
            assert got[i] == 0
        else:
            exact = mpmath.mpf(ms) / g * mpmath.cos(mpmath.pi * i / o.n)
            frac = exact - mpmath.floor(exact)
            assert abs(frac - 0.5) > 1e-3  # far from a rounding tie
            assert got[i] == int(mpmath.nint(exact))


# ------------------------------------------------------------------ encryption


def test_secret_key_encryption_is_exact(tiny):
    o = tiny
    m = workloads.int_poly(5, o.n, 1 << 20)
    ct = o.encrypt(m, 4, use_sk=True, cid=9)
    dec = o.decrypt_coeffs(ct, exact=True)
    e = oracle.sample(o.seed, "gauss", sid=9, dom=7, count=o.n)
    assert [d - int(x) for d, x in zip(dec, m)] == [int(x) for x in e]
    assert max(abs(int(x)) for x in e) <= 20


def test_public_key_encryption_is_exact(tiny):
    """Dec(Enc_pk(m)) - m = v e_pk + e0 + e1 s, recomputed with Python
    integers from the sampled streams and the secret key."""
    o = tiny
    m = workloads.int_poly(6, o.n, 1 << 20)
    ct = o.encrypt(m, 5, use_sk=False, cid=4)
    dec = o.decrypt_coeffs(ct, exact=True)
    s = [int(x) for x in o.secret()]
    e_pk = [int(x) for x in oracle.sample(o.seed, "gauss", sid=0, dom=3, count=o.n)]
    v = [int(x) for x in oracle.sample(o.seed, "ternary", sid=4, dom=6, count=o.n)]
    e0 = [int(x) for x in oracle.sample(o.seed, "gauss", sid=4, dom=7, count=o.n)]
    e1 = [int(x) for x in oracle.sample(o.seed, "gauss", sid=4, dom=8, count=o.n)]
    ve = negacyclic(v, e_pk)
    e1s = negacyclic(e1, s)
    want = [ve[i] + e0[i] + e1s[i] for i in range(o.n)]
    assert [d - int(x) for d, x in zip(dec, m)] == want
    assert set(s) <= {-1, 0, 1}


# ------------------------------------------------------------------ basis conversion


def test_modup_is_x_plus_small_multiple_of_qj(tiny):
    o = tiny
    level = 5  # digits {0,1}, {2,3}, {4}
    rng = np.random.default_rng(2)
    x = np.stack([rng.integers(0, q, o.n, dtype=np.uint64) for q in o.primes[:level]])
    for j, digit in enumerate([(0, 1), (2, 3), (4,)]):
        qj = [o.primes[i] for i in digit]
        Qj = math.prod(qj)
        targets = [t for t in list(range(level)) + [6, 7] if t not in digit]
        ys = {t: o.modup_coef(x, level, j, t) for t in targets}
        for k in range(o.n):
            xv = crt([x[i, k] for i in digit], qj)
            us = set()
            for t in targets:
                c = o.primes[t]
                cand = [u for u in range(len(digit)) if (xv + u * Qj) % c == int(ys[t][k])]
                assert cand, (j, t, k)
                us.add(tuple(cand))
            assert len(us) == 1


def test_moddown_conversion_is_exact(tiny):
    """The P -> q_t conversion of ModDown is the exact lift to [0, P): the
    CRT integer of the special residues, reduced mod q_t (no multiple of P),
    including the residues that lift next to 0 and next to P."""
    o = tiny
    rng = np.random.default_rng(3)
    ps = o.primes[6:8]
    P = ps[0] * ps[1]
    ints = [int(v) for v in rng.integers(0, 2 ** 62, o.n - 4)] + [0, 1, P - 2, P - 1]
    ints = [v % P for v in ints]
    y = np.array([[v % p for v in ints] for p in ps], dtype=np.uint64)
    for t in range(6):
        conv = o.moddown_conv(y, t)
        for k in range(o.n):
            assert crt(y[:, k], ps) == ints[k]
            assert int(conv[k]) == ints[k] % o.primes[t]


@pytest.mark.parametrize("merged", [False, True])
def test_moddown_rounds_boundary_lifts(tiny, merged):
    """ModDown on accumulators chosen as integers X whose (X + h) mod D lifts
    to 0, 1, 2, D - 2 or D - 1 (D = P, or P q_{l-1} merged with the rescale):
    every output coefficient is floor((X + h) / D), the rounded quotient,
    residue by residue (Python integers)."""
    from tests import moddown_inputs as mi
    o = tiny
    level = 5
    acc, d01, X, D = mi.accumulator(o, level, seed=17, merged=merged)
    lt = level - 1 if merged else level
    want = mi.expected_coef(X, D, o.primes[:lt])
    if merged:
        got = o.moddown_rescale(acc, d01, level)
    else:
        got = np.stack(o.moddown(acc, level))
    for p in range(2):
        gotc = to_coef(o, got[p], lt)
        for t in range(lt):
            assert [int(v) for v in gotc[t]] == want[p][t], (p, t)


# ------------------------------------------------------------------ rescale


def test_rescale_is_rounded_division(tiny):
    o = tiny
    level = 4
    data = workloads.residues(7, o.primes[:level], o.n, parts=2)
    ct = oracle.Ciphertext(data, level, 2.0 ** 40)
    out = o.rescale(ct)
    ql = o.primes[level - 1]
    for p in range(2):
        coef = to_coef(o, data[p], level)
        got = to_coef(o, out.data[p], level - 1)
        for k in range(o.n):
            c = crt(coef[:, k], o.primes[:level])
            r = (c + (ql - 1) // 2) // ql  # round(c / q_last), q_last odd
            for t in range(level - 1):
                assert int(got[t, k]) == r % o.primes[t]


# ------------------------------------------------------------------ tensor / key switching


def test_tensor_is_the_product_of_decryptions(tiny):
    o = tiny
    level = 3
    a = workloads.residues(8, o.primes[:level], o.n, parts=2)
    b = workloads.residues(9, o.primes[:level], o.n, parts=2)
    d = o.tensor(oracle.Ciphertext(a, level, 1.0), oracle.Ciphertext(b, level, 1.0))
    s = [int(x) for x in o.secret()]
    for t in range(level):
        q = o.primes[t]
        sv = oracle.ntt_def(np.array([x % q for x in s], dtype=np.uint64), o.log_n, q, o.roots[t])
        for k in range(o.n):
            sk = int(sv[k])
            lhs = (int(d[0, t, k]) + int(d[1, t, k]) * sk + int(d[2, t, k]) * sk * sk) % q
            rhs = ((int(a[0, t, k]) + int(a[1, t, k]) * sk) * (int(b[0, t, k]) + int(b[1, t, k]) * sk)) % q
            assert lhs == rhs


def _switch_error(o, d, level, k0, k1, sprime_eval):
    """max |k0 + k1 s - d s'| over coefficients, centered mod Q_level."""
    s = [int(x) for x in o.secret()]
    Q = math.prod(o.primes[:level])
    diff = np.zeros((level, o.n), dtype=np.uint64)
    for t in range(level):
        q = o.primes[t]
        sv = oracle.ntt_def(np.array([x % q for x in s], dtype=np.uint64), o.log_n, q, o.roots[t])
        for k in range(o.n):
            v = (int(k0[t, k]) + int(k1[t, k]) * int(sv[k]) - int(d[t, k]) * int(sprime_eval[t][k])) % q
            diff[t, k] = v
    coef = to_coef(o, diff, level)
    return max(abs(centered(crt(coef[:, k], o.primes[:level]), Q)) for k in range(o.n))


def _bound(o, level):
    # ModDown divides sum_j d~_j e_j (|d~_j| < |D_j| Q_j, |e_j| <= 20, N terms per
    # coefficient) by P and adds the conversion's error (< alpha per coefficient,
    # times the ternary secret's N terms for the second part)
    P = o.primes[o.L] * o.primes[o.L + 1]
    qmax = max(o.primes[:level])
    beta = -(-level // o.alpha)
    return beta * o.n * 20 * o.alpha * qmax ** o.alpha / P + o.alpha * (o.n + 1) + 1


@pytest.mark.parametrize("level", [6, 5, 2])
def test_relinearisation_key_switch_error_is_small(tiny, level):
    o = tiny
    d = workloads.residues(10 + level, o.primes[:level], o.n)[0]
    k0, k1 = o.keyswitch(d, level, -1)
    s = [int(x) for x in o.secret()]
    s2 = []
    for t in range(level):
        q = o.primes[t]
        sv = oracle.ntt_def(np.array([x % q for x in s], dtype=np.uint64), o.log_n, q, o.roots[t])
        s2.append([(int(v) * int(v)) % q for v in sv])
    err = _switch_error(o, d, level, k0, k1, s2)
    assert err <= _bound(o, level)


def test_galois_key_switch_error_is_small(tiny):
    o = tiny
    level = 4
    d = workloads.residues(20, o.primes[:level], o.n)[0]
    k = oracle.galois_elt(o.log_n, 3)
    key_id = o.gal_order.index(k)
    k0, k1 = o.keyswitch(d, level, key_id)
    s = [int(x) for x in o.secret()]
    sk = []
    for t in range(level):
        q = o.primes[t]
        sv = oracle.ntt_def(np.array([x % q for x in s], dtype=np.uint64), o.log_n, q, o.roots[t])
        sk.append([int(v) for v in o.automorph(sv[None, :], 1, k)[0]])
    assert _switch_error(o, d, level, k0, k1, sk) <= _bound(o, level)


# ------------------------------------------------------------------ homomorphism (Eq. 1-2)


@pytest.fixture(scope="module")
def mid():
    return oracle.Oracle(10, 5, 40, 1, 60, 2.0 ** 40, seed=3, rot_steps=[1, 2, 5, -1, -7])


def _enc(o, z, level, cid, scale=None, use_sk=False):
    scale = scale or o.scale
    return o.encrypt(o.encode(z, scale=scale), level, use_sk=use_sk, cid=cid, scale=scale)


def test_add_and_multiply_are_homomorphic(mid):
    o = mid
    z1 = workloads.uniform_slots(1, o.n // 2)
    z2 = workloads.uniform_slots(2, o.n // 2)
    a, b = _enc(o, z1, 5, 1), _enc(o, z2, 5, 2, use_sk=True)
    re, _ = o.decrypt(o.add(a, b))
    assert np.max(np.abs(re - (z1 + z2))) < 2.0 ** -20
    c = o.mul_relin_rescale(a, b)
    assert c.level == 4 and c.scale == a.scale * b.scale / o.primes[4]
    re, _ = o.decrypt(c)
    assert np.max(np.abs(re - z1 * z2)) < 2.0 ** -20
    # depth 2
    d = o.mul_relin_rescale(c, o.drop(b, 4))
    re, _ = o.decrypt(d)
    assert np.max(np.abs(re - z1 * z2 * z2)) < 2.0 ** -18


def test_constant_and_plaintext_products(mid):
    o = mid
    z = workloads.uniform_slots(3, o.n // 2)
    w = workloads.uniform_slots(4, o.n // 2)
    a = _enc(o, z, 4, 5)
    k = round(0.75 * o.primes[3])
    c = o.rescale(o.mul_int(a, k, o.primes[3]))
    re, _ = o.decrypt(c)
    assert np.max(np.abs(re - 0.75 * z)) < 2.0 ** -20
    re, _ = o.decrypt(o.add_int(a, round(-0.3 * a.scale)))
    assert np.max(np.abs(re - (z - 0.3))) < 2.0 ** -20
    pm = o.encode(w, scale=o.primes[3])
    c = o.rescale(o.mul_plain(a, pm, o.primes[3]))
    re, _ = o.decrypt(c)
    assert np.max(np.abs(re - z * w)) < 2.0 ** -20


@pytest.mark.parametrize("r", [1, 2, 5, -1, -7])
def test_rotation_is_a_cyclic_slot_shift(mid, r):
    o = mid
    z = workloads.uniform_slots(5, o.n // 2)
    a = _enc(o, z, 3, 6)
    re, _ = o.decrypt(o.rotate(a, r))
    assert np.max(np.abs(re - np.roll(z, -r))) < 2.0 ** -20


def test_rotation_without_key_is_refused(mid):
    with pytest.raises(KeyError):
        mid.rotate(_enc(mid, np.zeros(4), 2, 7), 3)


# ------------------------------------------------------------------ LR step (Eq. 5-8)


def test_table2_golden_values():
    t = table2()
    assert t["binomial"] == [0.5, -0.0843, 0.0, 0.0002]
    assert t["hinge"] == [0.5875, -0.1005, 0.0008, -0.00039]
    assert t["huber"] == [2.0, -0.1311, 0.0, 0.00005]


@pytest.mark.parametrize("loss", ["binomial", "hinge"])
def test_lr_step_matches_fp64_update(loss):
    log_n, g = 10, 4
    n_slots = (1 << log_n) // 2
    F = n_slots // g
    data = workloads.LRData(seed=0, n_samples=16, n_features=100)
    o = oracle.Oracle(log_n, 7, 40, 1, 60, 2.0 ** 40, seed=1, rot_steps=he.lr_rot_steps(n_slots, g))
    coeffs = table2()[loss]
    lr = 1.0 / data.n
    Z = [_enc(o, v, 7, 100 + k) for k, v in enumerate(workloads.pack_samples(data.X, data.y, n_slots, g))]
    W = _enc(o, workloads.pack_weights(data.w0, n_slots, g), 7, 99)
    out = o.lr_gradient_step(Z, W, coeffs, lr, g, 2.0 ** 40)
    assert out.level == 2 and out.scale == W.scale
    re, _ = o.decrypt(out)
    w1 = lr_step_fp64(data.X, data.y, data.w0, coeffs, lr)
    want = workloads.pack_weights(w1, n_slots, g)
    rel = np.max(np.abs(re - want)) / np.max(np.abs(want))
    assert rel < 2.0 ** -20, rel


@pytest.mark.parametrize("l2", [0.5, 3.0])
def test_lr_step_with_l2_regulariser_matches_fp64_update(l2):
    """The step with the regulariser of Eq. 4 (R = (l2/2) |w|^2, so the
    gradient of Eq. 6/8 gains l2 w) decrypts to the FP64 update
    w + lr (sum p(.) y x - l2 w), and differs from the unregularised step by
    -lr l2 w slot by slot (a dropped or sign-flipped term fails both)."""
    log_n, g = 10, 4
    n_slots = (1 << log_n) // 2
    data = workloads.LRData(seed=3, n_samples=16, n_features=100)
    o = oracle.Oracle(log_n, 7, 40, 1, 60, 2.0 ** 40, seed=1, rot_steps=he.lr_rot_steps(n_slots, g))
    coeffs = table2()["binomial"]
    lr = 1.0 / data.n
    Z = [_enc(o, v, 7, 100 + k) for k, v in enumerate(workloads.pack_samples(data.X, data.y, n_slots, g))]
    W = _enc(o, workloads.pack_weights(data.w0, n_slots, g), 7, 99)
    out = o.lr_gradient_step(Z, W, coeffs, lr, g, 2.0 ** 40, l2=l2)
    assert out.level == 2 and out.scale == W.scale
    re, _ = o.decrypt(out)
    want = workloads.pack_weights(lr_step_fp64(data.X, data.y, data.w0, coeffs, lr, l2=l2), n_slots, g)
    assert np.max(np.abs(re - want)) / np.max(np.abs(want)) < 2.0 ** -20
    re0, _ = o.decrypt(o.lr_gradient_step(Z, W, coeffs, lr, g, 2.0 ** 40))
    delta = -lr * l2 * workloads.pack_weights(data.w0, n_slots, g)
    assert np.max(np.abs((re - re0) - delta)) < 2.0 ** -20 * np.max(np.abs(want))
    assert np.max(np.abs(delta)) > 1e-3  # the term is far above the tolerance


def test_keyswitch_equals_big_integer_definition(tiny):
    """Hybrid key switching recomputed with Python integers from its
    definition: per digit the approximate ModUp y_j = sum_i [x_i (Q_j/q_i)^-1]_{q_i}
    (Q_j/q_i) (an integer equal to [x]_{Q_j} + u Q_j), the products with the key
    over the integers mod X^N + 1, then the division by P with rounding:
    out = floor((acc + h) / P) = round(acc / P), h = (P-1)/2.  Must equal the
    oracle's residues."""
    o = tiny
    level, n, L, alpha = 5, o.n, o.L, o.alpha
    q = o.primes
    P = math.prod(q[L:L + alpha])
    h = (P - 1) // 2
    d = workloads.residues(91, q[:level], n)[0]
    k0, k1 = o.keyswitch(d, level, -1)
    dc = to_coef(o, d, level)
    key = o.key(1)  # [beta][2][np][N], evaluation form
    targets = list(range(level)) + list(range(L, L + alpha))
    mod = math.prod(q[t] for t in targets)
    acc = [[0] * n, [0] * n]
    for j in range((level + alpha - 1) // alpha):
        digit = list(range(j * alpha, min((j + 1) * alpha, level)))
        Qj = math.prod(q[i] for i in digit)
        y = [0] * n
        for i in digit:
            qhat = Qj // q[i]
            inv = pow(qhat, -1, q[i])
            for c in range(n):
                y[c] += (int(dc[i][c]) * inv % q[i]) * qhat
        for p in range(2):
            kc = [oracle.intt_def(key[j, p, t], o.log_n, q[t], o.roots[t]) for t in targets]
            kint = [crt([kc[ti][c] for ti in range(len(targets))], [q[t] for t in targets]) for c in range(n)]
            prod = negacyclic(y, kint)
            acc[p] = [(a + b) % mod for a, b in zip(acc[p], prod)]
    for p, got in enumerate((k0, k1)):
        gotc = to_coef(o, got, level)
        for c in range(n):
            out = (acc[p][c] + h) // P
            for t in range(level):
                assert int(gotc[t][c]) == out % q[t], (p, c, t)


def test_mul_relin_rescale_equals_big_integer_definition(tiny):
    """Multiplication recomputed with Python integers: the tensor's parts
    (d0, d1, d2) residue by residue, the integer ModUp of d2 and its products
    with the relinearisation key over Q_level P (as in the key-switch pin),
    V = P (d0, d1) + those products, and one division with rounding by
    P q_{level-1}: out = floor((V + h) / (P q_{level-1})), h = (P q_{level-1}
    - 1)/2.  Must equal the oracle's residues."""
    o = tiny
    level, n, L, alpha = 5, o.n, o.L, o.alpha
    q = o.primes
    P = math.prod(q[L:L + alpha])
    D = P * q[level - 1]
    h = (D - 1) // 2
    a = workloads.residues(97, q[:level], n, parts=2)
    b = workloads.residues(98, q[:level], n, parts=2)
    out = o.mul_relin_rescale(oracle.Ciphertext(a, level, o.scale), oracle.Ciphertext(b, level, o.scale))
    d0 = np.stack([(a[0][t].astype(object) * b[0][t].astype(object)) % q[t] for t in range(level)])
    d1 = np.stack([(a[0][t].astype(object) * b[1][t].astype(object) + a[1][t].astype(object) * b[0][t].astype(object))
                   % q[t] for t in range(level)])
    d2 = np.stack([(a[1][t].astype(object) * b[1][t].astype(object)) % q[t] for t in range(level)])
    as_u64 = lambda x: np.array(x, dtype=np.uint64)
    d2c = to_coef(o, as_u64(d2), level)
    targets = list(range(level)) + list(range(L, L + alpha))
    mod = math.prod(q[t] for t in targets)
    key = o.key(1)
    acc = [[0] * n, [0] * n]
    for j in range((level + alpha - 1) // alpha):
        digit = list(range(j * alpha, min((j + 1) * alpha, level)))
        Qj = math.prod(q[i] for i in digit)
        y = [0] * n
        for i in digit:
            qhat = Qj // q[i]
            inv = pow(qhat, -1, q[i])
            for c in range(n):
                y[c] += (int(d2c[i][c]) * inv % q[i]) * qhat
        for p in range(2):
            kc = [oracle.intt_def(key[j, p, t], o.log_n, q[t], o.roots[t]) for t in targets]
            kint = [crt([kc[ti][c] for ti in range(len(targets))], [q[t] for t in targets]) for c in range(n)]
            acc[p] = [(x + v) % mod for x, v in zip(acc[p], negacyclic(y, kint))]
    for p, dp in enumerate((d0, d1)):
        dc = to_coef(o, as_u64(dp), level)
        dint = [crt([dc[t][c] for t in range(level)], q[:level]) for c in range(n)]
        gotc = to_coef(o, out.data[p], level - 1)
        for c in range(n):
            V = (P * dint[c] + acc[p][c]) % mod
            want = (V + h) // D
            for t in range(level - 1):
                assert int(gotc[t][c]) == want % q[t], (p, c, t)


def _kappa_int(y, k, n):
    """X -> X^k on integer coefficients, X^N = -1."""
    z = [0] * n
    for i, v in enumerate(y):
        e = i * k % (2 * n)
        if e < n:
            z[e] += v
        else:
            z[e - n] -= v
    return z


@pytest.mark.parametrize("steps", [[1, 3], [-1], [3, 1, -1]])
def test_rotate_sum_equals_big_integer_definition(tiny, steps):
    """The hoisted rotate-and-sum recomputed with Python integers: the digits
    y_j of a1 are raised once (the integer ModUp of the key-switch pin above),
    rotation s puts kappa_s(y_j) (X -> X^k_s over the integers) into its
    products with its Galois key, all products are summed mod Q_level P and
    divided by P once, with rounding; the addends are a0 + sum_s kappa_s(a0)
    and a1.  Must equal the oracle's residues."""
    o = tiny
    level, n, L, alpha = 5, o.n, o.L, o.alpha
    q = o.primes
    P = math.prod(q[L:L + alpha])
    h = (P - 1) // 2
    a = workloads.residues(94, q[:level], n, parts=2)
    out = o.rotate_sum(oracle.Ciphertext(a, level, o.scale), steps)
    dc = [to_coef(o, a[p], level) for p in range(2)]
    targets = list(range(level)) + list(range(L, L + alpha))
    mod = math.prod(q[t] for t in targets)
    ks = [oracle.galois_elt(o.log_n, s) for s in steps]
    acc = [[0] * n, [0] * n]
    for k in ks:
        key = o.key(2 + o.gal_order.index(k))
        for j in range((level + alpha - 1) // alpha):
            digit = list(range(j * alpha, min((j + 1) * alpha, level)))
            Qj = math.prod(q[i] for i in digit)
            y = [0] * n
            for i in digit:
                qhat = Qj // q[i]
                inv = pow(qhat, -1, q[i])
                for c in range(n):
                    y[c] += (int(dc[1][i][c]) * inv % q[i]) * qhat
            yk = _kappa_int(y, k, n)
            for p in range(2):
                kc = [oracle.intt_def(key[j, p, t], o.log_n, q[t], o.roots[t]) for t in targets]
                kint = [crt([kc[ti][c] for ti in range(len(targets))], [q[t] for t in targets]) for c in range(n)]
                prod = negacyclic(yk, kint)
                acc[p] = [(x + v) % mod for x, v in zip(acc[p], prod)]
    for p in range(2):
        gotc = to_coef(o, out.data[p], level)
        for t in range(level):
            addend = [int(v) for v in dc[p][t]]
            if p == 0:
                for k in ks:
                    addend = [x + v for x, v in zip(addend, _kappa_int([int(v) for v in dc[0][t]], k, n))]
            for c in range(n):
                want = ((acc[p][c] + h) // P + addend[c]) % q[t]
                assert int(gotc[t][c]) == want, (p, t, c)


@pytest.mark.parametrize("steps", [[1, 2], [5, -7, -1], [2]])
def test_rotate_sum_decrypts_to_the_sum_of_shifts(mid, steps):
    o = mid
    z = workloads.uniform_slots(7, o.n // 2)
    a = _enc(o, z, 4, 8)
    re, _ = o.decrypt(o.rotate_sum(a, steps))
    want = z + sum(np.roll(z, -s) for s in steps)
    assert np.max(np.abs(re - want)) < 2.0 ** -20


def test_rotate_sum_refuses_missing_keys_and_zero_steps(mid):
    a = _enc(mid, workloads.uniform_slots(8, mid.n // 2), 3, 9)
    with pytest.raises(KeyError):
        mid.rotate_sum(a, [3])
    with pytest.raises(KeyError):
        mid.rotate_sum(a, [1, 0])


def test_lr_inference_matches_fp64_polynomial():
    log_n, g = 10, 4
    n_slots = (1 << log_n) // 2
    F = n_slots // g
    data = workloads.LRData(seed=2, n_samples=8, n_features=90)
    o = oracle.Oracle(log_n, 6, 40, 1, 60, 2.0 ** 40, seed=4, rot_steps=he.lr_rot_steps(n_slots, g))
    coeffs = table2()["binomial"]
    Z = [_enc(o, v, 5, 300 + k) for k, v in enumerate(workloads.pack_samples(data.X, data.y, n_slots, g))]
    W = _enc(o, workloads.pack_weights(data.w0, n_slots, g), 5, 299)
    S = o.lr_inference(Z, W, coeffs, 1.0, g)
    assert S[0].level == 2 and abs(S[0].scale / W.scale - 1) < 1e-12
    m = data.y * (data.X @ data.w0)
    p = coeffs[0] + coeffs[1] * m + coeffs[3] * m ** 3
    for k, ct in enumerate(S):
        re, _ = o.decrypt(ct)
        for s in range(g):
            i = k * g + s
            assert np.max(np.abs(re[s::g] - p[i])) < 2.0 ** -20


def test_results_do_not_depend_on_thread_count():
    """Keys, key switching and the gradient step over five data ciphertexts
    (the step's parallel loop) give the same residues on one thread and on
    every thread."""
    log_n, g = 9, 4
    n_slots = (1 << log_n) // 2
    rots = he.lr_rot_steps(n_slots, g)
    data = workloads.LRData(seed=8, n_samples=5 * g, n_features=60)
    outs = []
    threads = oracle.get_threads()
    try:
        for nt in (1, max(2, threads)):
            oracle.set_threads(nt)
            o = oracle.Oracle(log_n, 7, 40, 2, 50, 2.0 ** 40, seed=4, rot_steps=rots)
            Z = [_enc(o, v, 7, 10 + k) for k, v in enumerate(workloads.pack_samples(data.X, data.y, n_slots, g))]
            W = _enc(o, workloads.pack_weights(data.w0, n_slots, g), 7, 9)
            assert len(Z) == 5
            step = o.lr_gradient_step(Z, W, table2()["binomial"], 1.0 / 20, g, 2.0 ** 30, l2=0.25)
            outs.append((o.key(1), o.key(2), step.data))
    finally:
        oracle.set_threads(threads)
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
