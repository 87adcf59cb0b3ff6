"""Parity of the sm_103a library with the CPU oracle, through the C ABI.

Residues must match bit for bit (integer work); encoding (floating point
deciding an integer) must match except where the oracle's unrounded value
lies within 1e-6 of a rounding tie; decryption to doubles within 1e-12
relative.  Sizes span several NTT tiles and ragged batch counts."""
import math

import numpy as np
import pytest

import oracle
from paper_2006_10091_gb300 import workloads
from tests.gpu_util import Pair, assert_same_residues, gpu_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def he():
    return gpu_lib()


@pytest.fixture(scope="module")
def small():
    # N = 2^10, five 40-bit limbs, one 60-bit special prime
    return Pair(10, 5, 40, 1, 60, 2.0 ** 40, seed=3, rots=[1, 2, 5, -1, -7])


@pytest.fixture(scope="module")
def digits():
    # N = 2^11, seven 45-bit limbs, two 50-bit special primes: digits of two limbs,
    # a partial last digit at odd levels
    return Pair(11, 7, 45, 2, 50, 2.0 ** 45, seed=5, rots=[3, -2])


# ------------------------------------------------------------------ parameters / NTT


def test_primes_match(small, digits):
    assert small.g.primes == small.o.primes
    assert digits.g.primes == digits.o.primes
    assert small.g.beta == small.o.beta and digits.g.beta == digits.o.beta


@pytest.mark.parametrize("log_n", [4, 7, 10, 12, 13, 14, 15, 16])
def test_ntt_matches_oracle(he, log_n):
    import torch
    L = 3
    ctx = he.Context(log_n, L, 50, 1, 60, 2.0 ** 40, seed=1)
    n = 1 << log_n
    npolys = 3  # ragged: three polynomials of L + 1 limbs
    data = workloads.residues(log_n, ctx.primes, n, parts=npolys)  # [npolys][np][n]
    want = [[oracle.ntt_r2(data[p, limb], log_n, ctx.primes[limb], oracle.min_root(ctx.primes[limb], log_n))
             for limb in range(L + 1)] for p in range(npolys)]
    for shape in ((0, 1, 2) if log_n >= 12 else (0,)):  # every compiled tile shape
        he.he_set_tuning(ctx, "ntt_shape", shape)
        t = torch.from_numpy(data.view(np.int64).copy()).cuda()
        he.he_ntt(ctx, t, npolys, (L + 1) * n, L + 1, 0, False)
        got = t.cpu().numpy().view(np.uint64)
        for p in range(npolys):
            for limb in range(L + 1):
                assert np.array_equal(got[p, limb], want[p][limb]), (shape, p, limb)
        he.he_ntt(ctx, t, npolys, (L + 1) * n, L + 1, 0, True)
        assert np.array_equal(t.cpu().numpy().view(np.uint64), data)
    he.he_set_tuning(ctx, "ntt_shape", 0)


@pytest.mark.parametrize("log_n", [13, 16])
def test_ntt_several_polynomials_per_cta(he, log_n):
    """Large ragged batches, where NTT CTAs transform several polynomials of
    one limb: every shape and grouping agrees with the runtime-shaped kernel."""
    import torch
    ctx = he.Context(log_n, 3, 45, 1, 60, 2.0 ** 40, seed=4)
    n = 1 << log_n
    npolys = 321 if log_n == 13 else 41
    data = workloads.residues(7 + log_n, ctx.primes, n, parts=npolys)
    t0 = torch.from_numpy(data.view(np.int64).copy()).cuda()
    he.he_set_tuning(ctx, "ntt_generic", True)
    he.he_ntt(ctx, t0, npolys, 4 * n, 4, 0, False)
    ref = t0.cpu().numpy()
    he.he_set_tuning(ctx, "ntt_generic", False)
    for shape in (0, 1, 2):
        for pb in (1, 8):
            he.he_set_tuning(ctx, "ntt_shape", shape)
            he.he_set_tuning(ctx, "ntt_pb_max", pb)
            t = torch.from_numpy(data.view(np.int64).copy()).cuda()
            he.he_ntt(ctx, t, npolys, 4 * n, 4, 0, False)
            assert np.array_equal(t.cpu().numpy(), ref), (shape, pb)
            he.he_ntt(ctx, t, npolys, 4 * n, 4, 0, True)
            assert np.array_equal(t.cpu().numpy().view(np.uint64), data), (shape, pb)
    he.he_set_tuning(ctx, "ntt_shape", 0)
    he.he_set_tuning(ctx, "ntt_pb_max", 8)


@pytest.mark.parametrize("log_n", [12, 13, 14, 15, 16])
def test_both_ntt_kernels_agree(he, log_n):
    """The compile-time-shaped and the runtime-shaped transforms give the same
    residues, on limb primes (lazy forward butterflies) and the 60-bit special
    prime (corrected butterflies), with skipped digit limbs left untouched."""
    import torch
    ctx = he.Context(log_n, 4, 45, 1, 60, 2.0 ** 40, seed=3)
    n = 1 << log_n
    data = workloads.residues(100 + log_n, ctx.primes, n, parts=5)
    outs = []
    for generic in (False, True):
        he.he_set_tuning(ctx, "ntt_generic", generic)
        t = torch.from_numpy(data.view(np.int64).copy()).cuda()
        he.he_ntt(ctx, t, 5, 5 * n, 5, 0, False)
        fwd = t.cpu().numpy().copy()
        he.he_ntt(ctx, t, 5, 5 * n, 5, 0, True)
        assert np.array_equal(t.cpu().numpy().view(np.uint64), data)
        outs.append(fwd)
    he.he_set_tuning(ctx, "ntt_generic", False)
    assert np.array_equal(outs[0], outs[1])


def test_ntt_limb_subset_and_prime_offset(he):
    import torch
    log_n, L = 12, 4
    ctx = he.Context(log_n, L, 45, 2, 55, 2.0 ** 40, seed=2)
    n = 1 << log_n
    data = workloads.residues(9, ctx.primes[2:5], n, parts=2)
    t = torch.from_numpy(data.view(np.int64).copy()).cuda()
    he.he_ntt(ctx, t, 2, 3 * n, 3, 2, False)  # limbs use primes 2, 3, 4
    got = t.cpu().numpy().view(np.uint64)
    for p in range(2):
        for k in range(3):
            q = ctx.primes[2 + k]
            assert np.array_equal(got[p, k], oracle.ntt_r2(data[p, k], log_n, q, oracle.min_root(q, log_n)))


# ------------------------------------------------------------------ encryption / keys


@pytest.mark.parametrize("use_sk", [False, True])
@pytest.mark.parametrize("level", [1, 3, 5])
def test_encryption_is_bit_exact(small, he, use_sk, level):
    m = workloads.int_poly(level, small.n, 1 << 35)
    g = small.gpu_enc(m, level, cid=17 + level, use_sk=use_sk)
    o = small.orc_enc(m, level, cid=17 + level, use_sk=use_sk)
    assert_same_residues(g, o, he, small.g)


def test_encryption_into_larger_buffer(small, he):
    m = workloads.int_poly(4, small.n, 1 << 30)
    g = small.gpu_enc(m, 3, cid=4, cap=5)
    assert_same_residues(g, small.orc_enc(m, 3, cid=4), he, small.g)


@pytest.mark.parametrize("level", [7, 6, 3, 1])
def test_keyswitch_relin_bit_exact(digits, he, level):
    import torch
    d = workloads.residues(40 + level, digits.o.primes[:level], digits.n)[0]
    k0, k1 = digits.o.keyswitch(d, level, -1)
    dt = torch.from_numpy(d.view(np.int64).copy()).cuda()
    o0 = torch.empty_like(dt)
    o1 = torch.empty_like(dt)
    he.he_keyswitch(digits.g, dt, level, 0, o0, o1)
    assert np.array_equal(o0.cpu().numpy().view(np.uint64), k0)
    assert np.array_equal(o1.cpu().numpy().view(np.uint64), k1)


def test_keyswitch_galois_bit_exact(digits, he):
    import torch
    level = 5
    d = workloads.residues(77, digits.o.primes[:level], digits.n)[0]
    gal = oracle.galois_elt(11, -2)
    k0, k1 = digits.o.keyswitch(d, level, digits.o.gal_order.index(gal))
    dt = torch.from_numpy(d.view(np.int64).copy()).cuda()
    o0, o1 = torch.empty_like(dt), torch.empty_like(dt)
    he.he_keyswitch(digits.g, dt, level, gal, o0, o1)
    assert np.array_equal(o0.cpu().numpy().view(np.uint64), k0)
    assert np.array_equal(o1.cpu().numpy().view(np.uint64), k1)


# ------------------------------------------------------------------ ciphertext operations


def _ct_pair(pair, seed, level, scale=None):
    m = workloads.int_poly(seed, pair.n, 1 << 30)
    return (pair.gpu_enc(m, level, cid=seed, scale=scale),
            pair.orc_enc(m, level, cid=seed, scale=scale))


@pytest.mark.parametrize("pair_name,level", [("small", 5), ("small", 2), ("digits", 7), ("digits", 4)])
def test_mul_relin_rescale_bit_exact(request, he, pair_name, level):
    pair = request.getfixturevalue(pair_name)
    ga, oa = _ct_pair(pair, 101, level)
    gb, ob = _ct_pair(pair, 102, level)
    out = pair.g.new_ct(level)
    he.he_mul_relin_rescale(pair.g, ga, gb, out)
    assert_same_residues(out, pair.o.mul_relin_rescale(oa, ob), he, pair.g)
    out2 = pair.g.new_ct(level)
    he.he_mul_relin(pair.g, ga, gb, out2)
    assert_same_residues(out2, pair.o.mul_relin(oa, ob), he, pair.g)


@pytest.mark.parametrize("count", [1, 3, 16])
def test_batched_mul_matches_single(small, he, count):
    level = 4
    ms = [workloads.int_poly(200 + i, small.n, 1 << 30) for i in range(2 * count)]
    A = small.g.new_ct(level, count)
    B = small.g.new_ct(level, count)
    for i in range(count):
        he.he_encrypt_poly(small.g, ms[i], small.g.scale, level, A[i], cid=300 + i)
        he.he_encrypt_poly(small.g, ms[count + i], small.g.scale, level, B[i], cid=400 + i)
    O = small.g.new_ct(level, count)
    he.he_mul_relin_rescale_batch(small.g, A, B, O)
    for i in range(count):
        oa = small.orc_enc(ms[i], level, cid=300 + i)
        ob = small.orc_enc(ms[count + i], level, cid=400 + i)
        assert_same_residues(O[i], small.o.mul_relin_rescale(oa, ob), he, small.g)


def test_batched_mul_non_uniform_buffers(small, he):
    level = 3
    A = [small.gpu_enc(workloads.int_poly(i, small.n, 1 << 20), level, cid=i) for i in range(3)]
    B = [small.gpu_enc(workloads.int_poly(9 + i, small.n, 1 << 20), level, cid=9 + i) for i in range(3)]
    O = [small.g.new_ct(level + 1) for _ in range(3)]  # separate allocations, larger capacity
    he.he_mul_relin_rescale_batch(small.g, A, B, O)
    for i in range(3):
        oa = small.orc_enc(workloads.int_poly(i, small.n, 1 << 20), level, cid=i)
        ob = small.orc_enc(workloads.int_poly(9 + i, small.n, 1 << 20), level, cid=9 + i)
        assert_same_residues(O[i], small.o.mul_relin_rescale(oa, ob), he, small.g)


@pytest.mark.parametrize("r", [1, 2, 5, -1, -7])
def test_rotation_bit_exact(small, he, r):
    ga, oa = _ct_pair(small, 500, 4)
    out = small.g.new_ct(4)
    he.he_rotate(small.g, ga, r, out)
    assert_same_residues(out, small.o.rotate(oa, r), he, small.g)


def test_rotation_batch_and_digits(digits, he):
    count, level = 5, 5
    ms = [workloads.int_poly(600 + i, digits.n, 1 << 30) for i in range(count)]
    A = digits.g.new_ct(level, count)
    for i in range(count):
        he.he_encrypt_poly(digits.g, ms[i], digits.g.scale, level, A[i], cid=600 + i)
    O = digits.g.new_ct(level, count)
    he.he_rotate_batch(digits.g, A, 3, O)
    for i in range(count):
        want = digits.o.rotate(digits.orc_enc(ms[i], level, cid=600 + i), 3)
        assert_same_residues(O[i], want, he, digits.g)


def test_rescale_add_sub_drop_bit_exact(small, he):
    ga, oa = _ct_pair(small, 700, 5)
    gb, ob = _ct_pair(small, 701, 5)
    out = small.g.new_ct(5)
    he.he_rescale(small.g, ga, out)
    assert_same_residues(out, small.o.rescale(oa), he, small.g)
    he.he_add(small.g, ga, gb, out)
    assert_same_residues(out, small.o.add(oa, ob), he, small.g)
    he.he_sub(small.g, ga, gb, out)
    assert_same_residues(out, small.o.sub(oa, ob), he, small.g)
    he.he_drop_level(small.g, ga, 2, out)
    assert_same_residues(out, small.o.drop(oa, 2), he, small.g)
    # in place
    c = small.gpu_ct(oa)
    he.he_add(small.g, c, gb, c)
    assert_same_residues(c, small.o.add(oa, ob), he, small.g)


def test_constant_and_plaintext_ops_bit_exact(small, he):
    ga, oa = _ct_pair(small, 800, 4)
    out = small.g.new_ct(4)
    he.he_mul_const(small.g, ga, -0.3125, 2.0 ** 38, out)
    assert_same_residues(out, small.o.mul_int(oa, round(-0.3125 * 2 ** 38), 2.0 ** 38), he, small.g)
    he.he_add_const(small.g, ga, 0.7, out)
    want = small.o.add_int(oa, int(np.round(0.7 * oa.scale)))
    assert_same_residues(out, want, he, small.g)
    pt = workloads.int_poly(801, small.n, 1 << 38)
    he.he_mul_plain(small.g, ga, pt, 2.0 ** 38, out)
    assert_same_residues(out, small.o.mul_plain(oa, pt, 2.0 ** 38), he, small.g)


# ------------------------------------------------------------------ encode / decrypt


@pytest.mark.parametrize("log_n,logscale", [(10, 40), (12, 30), (14, 40), (16, 50)])
def test_encode_matches_oracle_away_from_ties(he, log_n, logscale):
    ctx = he.Context(log_n, 2, 50, 1, 60, 2.0 ** logscale)
    o = oracle.Oracle(log_n, 2, 50, 1, 60, 2.0 ** logscale)
    z = workloads.uniform_slots(log_n, ctx.n // 2)
    got = he.he_encode(ctx, z, 2.0 ** logscale)
    raw = o.encode_raw(z, scale=2.0 ** logscale)
    want = o.encode(z, scale=2.0 ** logscale)
    # the two sides sum in different orders; both round half away from zero
    # unrounded values agree to a few units in the last place of Delta-sized doubles
    tol = max(1e-6, 2.0 ** (logscale - 52) * log_n * 4)
    frac = np.abs(np.abs(raw - np.trunc(raw)) - 0.5)
    near_tie = frac < tol
    assert np.array_equal(got[~near_tie], want[~near_tie])
    assert np.all(np.abs(got - want) <= max(1, math.ceil(tol)))


def test_decrypt_matches_oracle(small, he):
    for level in (1, 3, 5):
        ga, oa = _ct_pair(small, 900 + level, level)
        got = he.he_decrypt_poly(small.g, ga)
        want = small.o.decrypt_coeffs(oa)
        assert np.allclose(got, want, rtol=1e-12, atol=0)
        # decoding: compare with the oracle's decode of the same coefficients
        re = he.he_decrypt_decode(small.g, ga)
        ore, _ = small.o.decode(want, oa.scale)
        assert np.max(np.abs(re - ore)) < 1e-9


# ------------------------------------------------------------------ accuracy (decrypted vs FP64)


def test_cfg1_mul_accuracy_and_parity(he):
    """N = 2^12, three ~40-bit limbs + one special prime, 2^30 scale, 16 pairs
    of 2048 uniform slots: each product within 1e-4 of FP64.  The second
    operand is encoded at the prime the rescale divides by, so the product
    lands back at scale 2^30."""
    p = Pair(12, 3, 40, 1, 60, 2.0 ** 30, seed=0)
    level, count = 3, 16
    qlast = float(p.g.primes[level - 1])
    A = p.g.new_ct(level, count)
    B = p.g.new_ct(level, count)
    zs = []
    for i in range(count):
        za = workloads.uniform_slots(2 * i, 2048)
        zb = workloads.uniform_slots(2 * i + 1, 2048)
        zs.append((za, zb))
        he.he_encode_encrypt(p.g, za, 2.0 ** 30, level, A[i], cid=2 * i)
        he.he_encode_encrypt(p.g, zb, qlast, level, B[i], cid=2 * i + 1)
    O = p.g.new_ct(level, count)
    he.he_mul_relin_rescale_batch(p.g, A, B, O)
    worst = 0.0
    for i in range(count):
        assert O[i].scale == pytest.approx(2.0 ** 30, rel=1e-12)
        got = he.he_decrypt_decode(p.g, O[i], 2048)
        worst = max(worst, float(np.max(np.abs(got - zs[i][0] * zs[i][1]))))
    assert worst < 1e-4, worst
    # bit-exact against the oracle on the first pair, inputs from the oracle encoder
    ma = p.o.encode(zs[0][0], scale=2.0 ** 30)
    mb = p.o.encode(zs[0][1], scale=qlast)
    oa = p.o.encrypt(ma, level, cid=50, scale=2.0 ** 30)
    ob = p.o.encrypt(mb, level, cid=51, scale=qlast)
    ga, gb = p.gpu_enc(ma, level, 50, scale=2.0 ** 30), p.gpu_enc(mb, level, 51, scale=qlast)
    out = p.g.new_ct(level)
    he.he_mul_relin_rescale(p.g, ga, gb, out)
    assert_same_residues(out, p.o.mul_relin_rescale(oa, ob), he, p.g)


def test_rotation_accuracy(small, he):
    z = workloads.uniform_slots(11, small.n // 2)
    a = small.g.new_ct(3)
    he.he_encode_encrypt(small.g, z, 2.0 ** 40, 3, a, cid=11)
    out = small.g.new_ct(3)
    for r in (1, -7):
        he.he_rotate(small.g, a, r, out)
        got = he.he_decrypt_decode(small.g, out)
        assert np.max(np.abs(got - np.roll(z, -r))) < 2.0 ** -20


def test_refresh_round_trip(small, he):
    z = workloads.uniform_slots(12, small.n // 2)
    a = small.g.new_ct(5)
    he.he_encode_encrypt(small.g, z, 2.0 ** 40, 2, a, cid=12)
    out = small.g.new_ct(5)
    he.he_refresh(small.g, a, 5, 2.0 ** 40, 99, out)
    assert out.level == 5 and out.scale == 2.0 ** 40
    got = he.he_decrypt_decode(small.g, out)
    assert np.max(np.abs(got - z)) < 2.0 ** -20


# ------------------------------------------------------------------ errors


def test_errors_are_reported(small, he):
    ga, _ = _ct_pair(small, 1000, 3)
    out = small.g.new_ct(3)
    with pytest.raises(he.HeError) as e:
        he.he_rotate(small.g, ga, 3, out)  # no key for step 3
    assert e.value.code == he.HE_ENOKEY
    one = small.g.new_ct(1)
    gb = small.gpu_enc(workloads.int_poly(1, small.n, 10), 1, cid=1)
    with pytest.raises(he.HeError) as e:
        he.he_mul_relin_rescale(small.g, gb, gb, one)
    assert e.value.code == he.HE_ELEVEL
    gc = small.gpu_enc(workloads.int_poly(2, small.n, 10), 3, cid=2, scale=2.0 ** 20)
    with pytest.raises(he.HeError) as e:
        he.he_add(small.g, ga, gc, out)
    assert e.value.code == he.HE_ESCALE
    small_out = small.g.new_ct(1)
    with pytest.raises(he.HeError) as e:
        he.he_add(small.g, ga, ga, small_out)
    assert e.value.code == he.HE_EINVAL


# ------------------------------------------------------------------ fused key switching (N >= 2^12)


@pytest.fixture(scope="module")
def wide():
    # N = 2^12, six 45-bit limbs, two 55-bit special primes (digits of two limbs)
    return Pair(12, 6, 45, 2, 55, 2.0 ** 45, seed=8, rots=[5, -3])


@pytest.mark.parametrize("level", [6, 5, 2])
def test_fused_keyswitch_bit_exact(wide, he, level):
    import torch
    d = workloads.residues(500 + level, wide.o.primes[:level], wide.n)[0]
    k0, k1 = wide.o.keyswitch(d, level, -1)
    dt = torch.from_numpy(d.view(np.int64).copy()).cuda()
    # fused kernels (every tile shape), then the unfused sequence
    for generic, shape in ((False, 0), (False, 1), (False, 2), (True, 0)):
        he.he_set_tuning(wide.g, "ntt_generic", generic)
        he.he_set_tuning(wide.g, "ntt_shape", shape)
        o0, o1 = torch.empty_like(dt), torch.empty_like(dt)
        he.he_keyswitch(wide.g, dt, level, 0, o0, o1)
        assert np.array_equal(o0.cpu().numpy().view(np.uint64), k0)
        assert np.array_equal(o1.cpu().numpy().view(np.uint64), k1)
    he.he_set_tuning(wide.g, "ntt_generic", False)
    he.he_set_tuning(wide.g, "ntt_shape", 0)


def test_autotune_keeps_results(wide, he):
    """The autotuner picks knobs among its candidates; a rotation and a
    multiplication after it still match the oracle bit for bit."""
    res = he.he_autotune(wide.g, 6, 8)
    assert res["ntt_shape"] in (0, 1, 2) and res["ntt_pb_max"] in (1, 4, 8)
    assert res["ms_per_keyswitch"] > 0
    m1, m2 = workloads.int_poly(81, wide.n, 1 << 36), workloads.int_poly(82, wide.n, 1 << 36)
    ga, oa = wide.gpu_enc(m1, 6, 81), wide.orc_enc(m1, 6, 81)
    gb, ob = wide.gpu_enc(m2, 6, 82), wide.orc_enc(m2, 6, 82)
    out = wide.g.new_ct(6)
    he.he_rotate(wide.g, ga, 5, out)
    assert_same_residues(out, wide.o.rotate(oa, 5), he, wide.g)
    he.he_mul_relin_rescale(wide.g, ga, gb, out)
    assert_same_residues(out, wide.o.mul_relin_rescale(oa, ob), he, wide.g)
    for k, v in (("ntt_shape", 0), ("ntt_pb_max", 8)):
        he.he_set_tuning(wide.g, k, v)
    with pytest.raises(he.HeError):
        he.he_autotune(wide.g, 0, 8)


def test_fused_keyswitch_many_digits(he):
    """Nine one-limb digits and a 60-bit special prime: the fused inner
    product sums nine full products below 2^120 in 128 bits per residue
    before its one reduction."""
    import torch
    p = Pair(12, 9, 40, 1, 60, 2.0 ** 40, seed=12)
    d = workloads.residues(900, p.o.primes[:9], p.n)[0]
    k0, k1 = p.o.keyswitch(d, 9, -1)
    dt = torch.from_numpy(d.view(np.int64).copy()).cuda()
    o0, o1 = torch.empty_like(dt), torch.empty_like(dt)
    he.he_keyswitch(p.g, dt, 9, 0, o0, o1)
    assert np.array_equal(o0.cpu().numpy().view(np.uint64), k0)
    assert np.array_equal(o1.cpu().numpy().view(np.uint64), k1)


@pytest.mark.parametrize("log_n", [14, 16])
def test_ntt_largest_primes(he, log_n):
    """Limb primes just below 2^58 (the largest whose forward butterflies skip
    the correction: values reach 33q) and special primes just below 2^61 (the
    largest allowed: corrected butterflies reach 4q), on inputs all q - 1 and
    on uniform ones: bit-exact against the oracle's radix-2 transform, and the
    inverse restores the input, for every compiled tile shape."""
    import torch
    ctx = he.Context(log_n, 2, 58, 1, 61, 2.0 ** 40, seed=5)
    n = 1 << log_n
    data = workloads.residues(300 + log_n, ctx.primes, n, parts=2)
    for k, q in enumerate(ctx.primes):
        data[0, k, :] = q - 1
    assert ctx.primes[0] > 2 ** 57 and ctx.primes[2] > 2 ** 60
    want = [[oracle.ntt_r2(data[p, k], log_n, q, oracle.min_root(q, log_n)) for k, q in enumerate(ctx.primes)]
            for p in range(2)]
    for shape in (0, 1, 2):
        he.he_set_tuning(ctx, "ntt_shape", shape)
        t = torch.from_numpy(data.view(np.int64).copy()).cuda()
        he.he_ntt(ctx, t, 2, 3 * n, 3, 0, False)
        got = t.cpu().numpy().view(np.uint64)
        for p in range(2):
            for k in range(3):
                assert np.array_equal(got[p, k], want[p][k]), (shape, p, k)
        he.he_ntt(ctx, t, 2, 3 * n, 3, 0, True)
        assert np.array_equal(t.cpu().numpy().view(np.uint64), data), shape
    he.he_set_tuning(ctx, "ntt_shape", 0)


def test_keyswitch_largest_primes(he):
    """Key switching, rotation and multiplication with 58-bit limbs and a
    61-bit special prime (fused conversions and transforms at the largest
    prime of each butterfly kind), on a digit input of all q - 1 as well."""
    import torch
    p = Pair(14, 3, 58, 1, 61, 2.0 ** 40, seed=21, rots=[1])
    for fill in (False, True):
        d = workloads.residues(910, p.o.primes[:3], p.n)[0]
        if fill:
            for k in range(3):
                d[k, :] = p.o.primes[k] - 1
        k0, k1 = p.o.keyswitch(d, 3, -1)
        dt = torch.from_numpy(d.view(np.int64).copy()).cuda()
        o0, o1 = torch.empty_like(dt), torch.empty_like(dt)
        he.he_keyswitch(p.g, dt, 3, 0, o0, o1)
        assert np.array_equal(o0.cpu().numpy().view(np.uint64), k0), fill
        assert np.array_equal(o1.cpu().numpy().view(np.uint64), k1), fill
    m1, m2 = workloads.int_poly(71, p.n, 1 << 36), workloads.int_poly(72, p.n, 1 << 36)
    ga, oa = p.gpu_enc(m1, 3, 71), p.orc_enc(m1, 3, 71)
    gb, ob = p.gpu_enc(m2, 3, 72), p.orc_enc(m2, 3, 72)
    out = p.g.new_ct(3)
    he.he_rotate(p.g, ga, 1, out)
    assert_same_residues(out, p.o.rotate(oa, 1), he, p.g)
    he.he_mul_relin_rescale(p.g, ga, gb, out)
    assert_same_residues(out, p.o.mul_relin_rescale(oa, ob), he, p.g)


def test_moddown_fused_and_unfused_after_fused_keyswitch(he):
    """N = 2^15 with four special primes: in the (8, 4) column shape the
    conversion kernel would need more shared memory than it may take, so a
    fused decomposition and row kernel are followed by the unfused ModDown
    (full inverse transform first); in the other shapes the conversion kernel
    finishes the dropped limbs' inverse transform itself.  Key switching, the
    multiplication (ModDown merged with the rescale), a rescale, a rotation
    and a hoisted rotate-and-sum, bit-exact in every shape."""
    import torch
    p = Pair(15, 3, 40, 4, 50, 2.0 ** 40, seed=31, rots=[1, 2, 3])
    d = workloads.residues(930, p.o.primes[:3], p.n)[0]
    k0, k1 = p.o.keyswitch(d, 3, -1)
    m1, m2 = workloads.int_poly(931, p.n, 1 << 36), workloads.int_poly(932, p.n, 1 << 36)
    ga, oa = p.gpu_enc(m1, 3, 931), p.orc_enc(m1, 3, 931)
    gb, ob = p.gpu_enc(m2, 3, 932), p.orc_enc(m2, 3, 932)
    want_mul = p.o.mul_relin_rescale(oa, ob)
    want_rs = p.o.rescale(oa)
    want_rot = p.o.rotate(oa, 2)
    want_sum = p.o.rotate_sum(oa, [1, 2, 3])
    dt = torch.from_numpy(d.view(np.int64).copy()).cuda()
    for shape in (0, 1, 2):
        he.he_set_tuning(p.g, "ntt_shape", shape)
        o0, o1 = torch.empty_like(dt), torch.empty_like(dt)
        he.he_keyswitch(p.g, dt, 3, 0, o0, o1)
        assert np.array_equal(o0.cpu().numpy().view(np.uint64), k0), shape
        assert np.array_equal(o1.cpu().numpy().view(np.uint64), k1), shape
        out = p.g.new_ct(3)
        he.he_mul_relin_rescale(p.g, ga, gb, out)
        assert_same_residues(out, want_mul, he, p.g)
        he.he_rescale(p.g, ga, out)
        assert_same_residues(out, want_rs, he, p.g)
        he.he_rotate(p.g, ga, 2, out)
        assert_same_residues(out, want_rot, he, p.g)
        he.he_rotate_sum(p.g, ga, [1, 2, 3], out)
        assert_same_residues(out, want_sum, he, p.g)
    he.he_set_tuning(p.g, "ntt_shape", 0)


def test_fused_rotation_and_mul_bit_exact(wide, he):
    m1, m2 = workloads.int_poly(61, wide.n, 1 << 36), workloads.int_poly(62, wide.n, 1 << 36)
    ga, oa = wide.gpu_enc(m1, 5, 61), wide.orc_enc(m1, 5, 61)
    gb, ob = wide.gpu_enc(m2, 5, 62), wide.orc_enc(m2, 5, 62)
    out = wide.g.new_ct(5)
    he.he_rotate(wide.g, ga, -3, out)
    assert_same_residues(out, wide.o.rotate(oa, -3), he, wide.g)
    he.he_mul_relin_rescale(wide.g, ga, gb, out)
    assert_same_residues(out, wide.o.mul_relin_rescale(oa, ob), he, wide.g)


@pytest.mark.parametrize("level", [6, 3, 2])
def test_fused_rescale_bit_exact(wide, he, level):
    """The rescale runs as a ModDown by q_{l-1} through the fused kernels at
    N >= 2^12; out of place and in place."""
    m = workloads.int_poly(64 + level, wide.n, 1 << 40)
    ga, oa = wide.gpu_enc(m, level, 64 + level), wide.orc_enc(m, level, 64 + level)
    want = wide.o.rescale(oa)
    out = wide.g.new_ct(level)
    he.he_rescale(wide.g, ga, out)
    assert_same_residues(out, want, he, wide.g)
    he.he_rescale(wide.g, ga, ga)
    assert_same_residues(ga, want, he, wide.g)


def test_fused_rotation_in_place(wide, he):
    """The fused rotation reads its input through the automorphism while it
    writes the output; an output that overlaps the input takes the path with
    a separate automorphism and gives the same residues."""
    m = workloads.int_poly(63, wide.n, 1 << 36)
    ga, oa = wide.gpu_enc(m, 5, 63), wide.orc_enc(m, 5, 63)
    want = wide.o.rotate(oa, 5)
    he.he_rotate(wide.g, ga, 5, ga)
    assert_same_residues(ga, want, he, wide.g)


def test_fused_single_special_prime_n13(he):
    p = Pair(13, 4, 40, 1, 60, 2.0 ** 40, seed=9, rots=[1])
    m1, m2 = workloads.int_poly(71, p.n, 1 << 30), workloads.int_poly(72, p.n, 1 << 30)
    ga, oa = p.gpu_enc(m1, 4, 71), p.orc_enc(m1, 4, 71)
    gb, ob = p.gpu_enc(m2, 4, 72), p.orc_enc(m2, 4, 72)
    out = p.g.new_ct(4)
    he.he_mul_relin_rescale(p.g, ga, gb, out)
    assert_same_residues(out, p.o.mul_relin_rescale(oa, ob), he, p.g)
    he.he_rotate(p.g, ga, 1, out)
    assert_same_residues(out, p.o.rotate(oa, 1), he, p.g)


@pytest.mark.parametrize("log_n", [15, 16])
def test_fused_matches_unfused_large(he, log_n):
    """At the large ring sizes with four special primes (the tile shapes where
    ModDown's conversion may not fit in shared memory) every fused variant
    gives the residues of the unfused sequence, which the oracle pins at small
    N; relinearisation and rotation."""
    import torch
    ctx = he.Context(log_n, 8, 50, 4, 60, 2.0 ** 50, seed=23, rot_steps=[3, 1, 2, 64, 128, 192])
    n = ctx.n
    d = workloads.residues(31 + log_n, ctx.primes[:8], n)[0]
    dt = torch.from_numpy(d.view(np.int64).copy()).cuda()
    outs = {}
    for generic, shape in ((True, 0), (False, 0), (False, 1), (False, 2)):
        he.he_set_tuning(ctx, "ntt_generic", generic)
        he.he_set_tuning(ctx, "ntt_shape", shape)
        o0, o1 = torch.empty_like(dt), torch.empty_like(dt)
        he.he_keyswitch(ctx, dt, 8, 0, o0, o1)
        outs[(generic, shape)] = (o0.cpu().numpy(), o1.cpu().numpy())
        ct = ctx.new_ct(8)
        he.he_encrypt_poly(ctx, workloads.int_poly(5, n, 1 << 40), 2.0 ** 50, 8, ct, cid=5)
        rot = ctx.new_ct(8)
        he.he_rotate(ctx, ct, 3, rot)
        outs[(generic, shape, "rot")] = he.he_ct_export(ctx, rot)
        he.he_rotate_sum(ctx, ct, [1, 2, 3], rot)
        outs[(generic, shape, "rotsum")] = he.he_ct_export(ctx, rot)
        he.he_rotate_sum(ctx, ct, [64, 128, 192], rot)
        outs[(generic, shape, "rotsum64")] = he.he_ct_export(ctx, rot)
    he.he_set_tuning(ctx, "ntt_generic", False)
    he.he_set_tuning(ctx, "ntt_shape", 0)
    for shape in (0, 1, 2):
        for k in range(2):
            assert np.array_equal(outs[(False, shape)][k], outs[(True, 0)][k]), (shape, k)
        assert np.array_equal(outs[(False, shape, "rot")], outs[(True, 0, "rot")]), shape
        assert np.array_equal(outs[(False, shape, "rotsum")], outs[(True, 0, "rotsum")]), shape
        assert np.array_equal(outs[(False, shape, "rotsum64")], outs[(True, 0, "rotsum64")]), shape


@pytest.fixture(scope="module")
def hoist():
    # N = 2^12, six 45-bit limbs, two 55-bit special primes
    return Pair(12, 6, 45, 2, 55, 2.0 ** 45, seed=14, rots=[1, 2, 3, 5, -3, -1, -2, 4, 6, 8, 16, 24])


@pytest.mark.parametrize("level,steps", [(6, [1, 2, 3]), (5, [5, -3]), (2, [-1, -2, 5]), (1, [3]), (4, [2, 4, 6]),
                                         (6, [8, 16, 24]), (3, [16])])
def test_rotate_sum_bit_exact(hoist, he, level, steps):
    """The hoisted rotate-and-sum against the oracle's: fused kernels in every
    tile shape, the unfused sequence, and in place.  Even steps map every row
    tile of the fused row pass at N = 2^12 onto itself (the kernel then sums
    the rotations in registers); odd ones move rows between tiles (one
    accumulator per rotation)."""
    m = workloads.int_poly(90 + level, hoist.n, 1 << 36)
    ga, oa = hoist.gpu_enc(m, level, 90 + level), hoist.orc_enc(m, level, 90 + level)
    want = hoist.o.rotate_sum(oa, steps)
    for generic, shape in ((False, 0), (False, 1), (False, 2), (True, 0)):
        he.he_set_tuning(hoist.g, "ntt_generic", generic)
        he.he_set_tuning(hoist.g, "ntt_shape", shape)
        out = hoist.g.new_ct(level)
        he.he_rotate_sum(hoist.g, ga, steps, out)
        assert_same_residues(out, want, he, hoist.g)
    he.he_set_tuning(hoist.g, "ntt_generic", False)
    he.he_set_tuning(hoist.g, "ntt_shape", 0)
    he.he_rotate_sum(hoist.g, ga, steps, ga)
    assert_same_residues(ga, want, he, hoist.g)


def test_rotate_sum_batch_and_errors(hoist, he):
    count, level = 5, 4
    ms = [workloads.int_poly(950 + i, hoist.n, 1 << 30) for i in range(count)]
    A = hoist.g.new_ct(level, count)
    for i in range(count):
        he.he_encrypt_poly(hoist.g, ms[i], hoist.g.scale, level, A[i], cid=950 + i)
    O = hoist.g.new_ct(level, count)
    he.he_rotate_sum_batch(hoist.g, A, [1, 2, 3], O)
    for i in range(count):
        want = hoist.o.rotate_sum(hoist.orc_enc(ms[i], level, cid=950 + i), [1, 2, 3])
        assert_same_residues(O[i], want, he, hoist.g)
    for steps, code in (([7], he.HE_ENOKEY), ([1, 0], he.HE_EINVAL), ([1] * 17, he.HE_EINVAL)):
        with pytest.raises(he.HeError) as e:
            he.he_rotate_sum(hoist.g, A[0], steps, O[0])
        assert e.value.code == code
    with pytest.raises(he.HeError) as e:  # an output over another input
        he.he_rotate_sum_batch(hoist.g, [A[0], A[1]], [1], [A[1], O[1]])
    assert e.value.code == he.HE_EINVAL


@pytest.fixture(scope="module")
def wide58():
    # N = 2^12, four 58-bit limbs, one 61-bit special prime
    return Pair(12, 4, 58, 1, 61, 2.0 ** 40, seed=31, rots=[2, 4, 6, 8, 10, 12])


def split_sums(bits: int, nrot: int, beta: int) -> bool:
    """Whether the product kernel sums a closed stage's key products on a
    prime of `bits` bits as split sums: 2 ceil(bits/2) + 2 + bitlen(nrot beta) <= 64."""
    sb = (bits + 1) // 2
    return 2 * sb + 2 + (nrot * beta).bit_length() <= 64


@pytest.mark.parametrize("level,steps,limb_split", [(4, [2, 4, 6, 8, 10, 12], False), (3, [2, 4, 6, 8], True),
                                                    (2, [2, 4], True)])
def test_rotate_sum_wide_primes_bit_exact(wide58, he, level, steps, limb_split):
    """Closed hoisted stages on 58-bit limbs and a 61-bit special prime, on
    uniform residues and on residues all q - 1: with 24 key products per
    residue the limbs' sums are 128-bit multiply-accumulates and part 0 goes
    through the rotations in the ModDown combine; with 12 the limbs take the
    split sums at the edge of their 64-bit bound (2*29 + 2 + 4 = 64) and part 0
    is added in the product kernel, while the special prime stays on 128-bit
    sums; with 4, both.  Every tile shape, equal to the oracle."""
    beta = level  # one special prime: digits of one limb
    assert split_sums(58, len(steps), beta) == limb_split and not split_sums(61, len(steps), beta)
    assert all(q.bit_length() == 58 for q in wide58.o.primes[:4]) and wide58.o.primes[4].bit_length() == 61
    for fill in (False, True):
        data = workloads.residues(3100 + level, wide58.o.primes[:level], wide58.n, parts=2)
        if fill:
            for k in range(level):
                data[:, k, :] = wide58.o.primes[k] - 1
        oa = oracle.Ciphertext(data, level, wide58.o.scale)
        want = wide58.o.rotate_sum(oa, steps)
        ga = wide58.gpu_ct(oa)
        for shape in (0, 1, 2):
            he.he_set_tuning(wide58.g, "ntt_shape", shape)
            out = wide58.g.new_ct(level)
            he.he_rotate_sum(wide58.g, ga, steps, out)
            assert_same_residues(out, want, he, wide58.g)
    he.he_set_tuning(wide58.g, "ntt_shape", 0)


@pytest.mark.parametrize("ks_ct", [1, 2, 4])
def test_key_products_per_cta_bit_exact(hoist, he, ks_ct):
    """The product kernel with 1, 2 or 4 ciphertexts per CTA (each key word
    serving that many): a ragged batch of 7 (a tail CTA with fewer) through a
    closed hoisted stage (steps 8, 16, 24), a relinearising multiplication and
    a single rotation, in every tile shape, equal to the oracle."""
    count, level = 7, 5
    ms = [workloads.int_poly(1700 + i, hoist.n, 1 << 30) for i in range(count)]
    A = hoist.g.new_ct(level, count)
    for i in range(count):
        he.he_encrypt_poly(hoist.g, ms[i], hoist.g.scale, level, A[i], cid=1700 + i)
    orc = [hoist.orc_enc(ms[i], level, cid=1700 + i) for i in range(count)]
    want_sum = [hoist.o.rotate_sum(o, [8, 16, 24]) for o in orc]
    want_mul = [hoist.o.mul_relin_rescale(o, orc[(i + 1) % count]) for i, o in enumerate(orc)]
    want_rot = [hoist.o.rotate(o, 8) for o in orc]
    B = [A[(i + 1) % count] for i in range(count)]
    he.he_set_tuning(hoist.g, "ks_ct", ks_ct)
    try:
        for shape in (0, 1, 2):
            he.he_set_tuning(hoist.g, "ntt_shape", shape)
            O = hoist.g.new_ct(level, count)
            he.he_rotate_sum_batch(hoist.g, A, [8, 16, 24], O)
            for i in range(count):
                assert_same_residues(O[i], want_sum[i], he, hoist.g)
            he.he_mul_relin_rescale_batch(hoist.g, A, B, O)
            for i in range(count):
                assert_same_residues(O[i], want_mul[i], he, hoist.g)
            he.he_rotate_batch(hoist.g, A, 8, O)
            for i in range(count):
                assert_same_residues(O[i], want_rot[i], he, hoist.g)
    finally:
        he.he_set_tuning(hoist.g, "ks_ct", 0)
        he.he_set_tuning(hoist.g, "ntt_shape", 0)


def test_rotate_sum_accuracy(hoist, he):
    z = workloads.uniform_slots(96, hoist.n // 2)
    a = hoist.g.new_ct(4)
    he.he_encode_encrypt(hoist.g, z, 2.0 ** 45, 4, a, cid=96)
    out = hoist.g.new_ct(4)
    he.he_rotate_sum(hoist.g, a, [1, 2, 3], out)
    got = he.he_decrypt_decode(hoist.g, out)
    want = z + np.roll(z, -1) + np.roll(z, -2) + np.roll(z, -3)
    assert np.max(np.abs(got - want)) < 2.0 ** -20


def test_rotate_sum_many_digits_unfused(he):
    """Twenty-two one-limb digits: their row tiles exceed the shared memory
    of the fused hoisted row pass, so the stage runs the unfused ModUp and
    inner products; same residues as the oracle."""
    p = Pair(12, 22, 40, 1, 60, 2.0 ** 40, seed=15, rots=[1, 2])
    m = workloads.int_poly(97, p.n, 1 << 30)
    ga, oa = p.gpu_enc(m, 22, 97), p.orc_enc(m, 22, 97)
    out = p.g.new_ct(22)
    he.he_rotate_sum(p.g, ga, [1, 2], out)
    assert_same_residues(out, p.o.rotate_sum(oa, [1, 2]), he, p.g)


def test_alu_probes_run(he):
    """The throughput probes behind the integer roof return positive rates in
    the expected order (a Shoup product costs several multiply-adds)."""
    r = [he.he_probe_alu(k) for k in range(5)]
    assert all(x["per_second"] > 0 and x["per_clock_per_sm"] > 0 for x in r)
    assert r[0]["per_clock_per_sm"] > 4 * r[1]["per_clock_per_sm"]
    with pytest.raises(he.HeError):
        he.he_probe_alu(7)


def test_library_owned_ciphertexts(small, he):
    """Handles from he_ct_alloc serve every entry point like caller-owned
    buffers: encrypt into two, multiply into a third, equal to the oracle;
    he_ct_free releases them; a capacity outside [1, L] is refused."""
    ma, mb = workloads.int_poly(61, small.n, 1 << 30), workloads.int_poly(62, small.n, 1 << 30)
    a, b, out = he.he_ct_alloc(small.g, 5), he.he_ct_alloc(small.g, 5), he.he_ct_alloc(small.g, 4)
    assert a.level == 0
    he.he_encrypt_poly(small.g, ma, small.g.scale, 5, a, cid=61)
    he.he_encrypt_poly(small.g, mb, small.g.scale, 5, b, cid=62)
    he.he_mul_relin_rescale(small.g, a, b, out)
    want = small.o.mul_relin_rescale(small.orc_enc(ma, 5, 61), small.orc_enc(mb, 5, 62))
    assert (out.level, out.scale) == (want.level, pytest.approx(want.scale, rel=1e-15))
    assert np.array_equal(he.he_ct_export(small.g, out), want.data)
    for h in (a, b, out):
        h.close()
    for cap in (0, small.L + 1):
        with pytest.raises(he.HeError) as e:
            he.he_ct_alloc(small.g, cap)
        assert e.value.code == he.HE_EINVAL


def test_empty_and_degenerate_inputs(small, he):
    """Empty batches are no-ops; a rotation by 0 or by N/2 slots (the identity
    automorphism) returns the input's residues; operations on one-limb
    ciphertexts that need none of the consumed limbs work at level 1 and
    equal the oracle; an empty sum is refused."""
    he.he_mul_relin_rescale_batch(small.g, [], [], [])
    he.he_rotate_batch(small.g, [], 1, [])
    he.he_rotate_sum_batch(small.g, [], [1], [])
    ga, oa = _ct_pair(small, 1300, 3)
    for steps in (0, small.n // 2):
        out = small.g.new_ct(3)
        he.he_rotate(small.g, ga, steps, out)
        assert np.array_equal(he.he_ct_export(small.g, out), oa.data)
    g1, o1 = _ct_pair(small, 1301, 1)
    out = small.g.new_ct(1)
    he.he_rotate(small.g, g1, 1, out)  # key switching with a single limb
    assert_same_residues(out, small.o.rotate(o1, 1), he, small.g)
    he.he_add(small.g, g1, g1, out)
    assert_same_residues(out, small.o.add(o1, o1), he, small.g)
    with pytest.raises(he.HeError) as e:
        he.he_sum(small.g, [], out)
    assert e.value.code == he.HE_EINVAL
