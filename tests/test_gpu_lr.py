"""The encrypted logistic-regression step (Eq. 5-8, Table 2) on the GPU:
residues bit-exact against the oracle's op-for-op evaluation, and the
decrypted weights against the FP64 update."""
import math

import numpy as np
import pytest

import oracle
from paper_2006_10091_gb300 import workloads
from tests.gpu_util import Pair, assert_same_residues, gpu_lib
from tests.lr_reference import lr_step_fp64, table2

pytestmark = pytest.mark.gpu


def rot_steps(n_slots, g):
    return gpu_lib().lr_rot_steps(n_slots, g)


@pytest.fixture(scope="module")
def lr_pair():
    log_n, g = 10, 4
    return Pair(log_n, 7, 40, 1, 60, 2.0 ** 40, seed=1, rots=rot_steps((1 << log_n) // 2, g)), g


@pytest.mark.parametrize("loss", ["binomial", "hinge", "huber"])
def test_lr_step_bit_exact(lr_pair, loss):
    pair, g = lr_pair
    he = pair.he
    nZ, level = 5, 7  # ragged: not a power of two
    coeffs = table2()[loss]
    lr = 1.0 / (nZ * g)
    ms = [workloads.int_poly(10 + k, pair.n, 1 << 28) for k in range(nZ)]
    mw = workloads.int_poly(9, pair.n, 1 << 28)
    Zg = pair.g.new_ct(level, nZ)
    for k in range(nZ):
        he.he_encrypt_poly(pair.g, ms[k], 2.0 ** 40, level, Zg[k], cid=100 + k)
    Wg = pair.gpu_enc(mw, level, 99, scale=2.0 ** 40)
    Zo = [pair.orc_enc(ms[k], level, 100 + k, scale=2.0 ** 40) for k in range(nZ)]
    Wo = pair.orc_enc(mw, level, 99, scale=2.0 ** 40)
    out = pair.g.new_ct(level)
    he.he_lr_gradient_step(pair.g, Zg, Wg, he.lr_config(coeffs, lr, g, 2.0 ** 40), out)
    want = pair.o.lr_gradient_step(Zo, Wo, coeffs, lr, g, 2.0 ** 40)
    assert out.level == level - 5
    assert_same_residues(out, want, he, pair.g)


@pytest.mark.parametrize("l2", [0.5, 3.0])
def test_lr_step_with_l2_regulariser_bit_exact(lr_pair, l2):
    """The step with the L2 regulariser's gradient (Eq. 4, 6: grad R = l2 w)
    equals the oracle's residues, and decrypts to w + lr (sum p y x - l2 w)."""
    pair, g = lr_pair
    he = pair.he
    n_slots = pair.n // 2
    data = workloads.LRData(seed=3, n_samples=16, n_features=100)
    coeffs = table2()["binomial"]
    lr = 1.0 / data.n
    zs = workloads.pack_samples(data.X, data.y, n_slots, g)
    ms = [pair.o.encode(v, scale=2.0 ** 40) for v in zs]
    mw = pair.o.encode(workloads.pack_weights(data.w0, n_slots, g), scale=2.0 ** 40)
    Zg = pair.g.new_ct(7, len(ms))
    for k, m in enumerate(ms):
        he.he_encrypt_poly(pair.g, m, 2.0 ** 40, 7, Zg[k], cid=100 + k)
    Wg = pair.gpu_enc(mw, 7, 99, scale=2.0 ** 40)
    out = pair.g.new_ct(7)
    he.he_lr_gradient_step(pair.g, Zg, Wg, he.lr_config(coeffs, lr, g, 2.0 ** 40, l2=l2), out)
    Zo = [pair.orc_enc(m, 7, 100 + k, scale=2.0 ** 40) for k, m in enumerate(ms)]
    want = pair.o.lr_gradient_step(Zo, pair.orc_enc(mw, 7, 99, scale=2.0 ** 40), coeffs, lr, g, 2.0 ** 40, l2=l2)
    assert_same_residues(out, want, he, pair.g)
    got = he.he_decrypt_decode(pair.g, out)
    ref = workloads.pack_weights(lr_step_fp64(data.X, data.y, data.w0, coeffs, lr, l2=l2), n_slots, g)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 2.0 ** -20


def test_lr_step_refuses_negative_l2(lr_pair):
    pair, g = lr_pair
    he = pair.he
    Z = pair.g.new_ct(7, 1)
    he.he_encrypt_poly(pair.g, workloads.int_poly(1, pair.n, 100), 2.0 ** 40, 7, Z[0], cid=1)
    W = pair.gpu_enc(workloads.int_poly(2, pair.n, 100), 7, 2, scale=2.0 ** 40)
    out = pair.g.new_ct(7)
    with pytest.raises(he.HeError) as e:
        he.he_lr_gradient_step(pair.g, Z, W, he.lr_config(table2()["binomial"], 0.1, g, 2.0 ** 40, l2=-1.0), out)
    assert e.value.code == he.HE_EINVAL


def test_lr_step_refuses_empty_data(lr_pair):
    pair, g = lr_pair
    he = pair.he
    W = pair.gpu_enc(workloads.int_poly(7, pair.n, 100), 7, 7, scale=2.0 ** 40)
    out = pair.g.new_ct(7)
    with pytest.raises(he.HeError) as e:
        he.he_lr_gradient_step(pair.g, [], W, he.lr_config(table2()["binomial"], 0.1, g, 2.0 ** 40), out)
    assert e.value.code == he.HE_EINVAL
    with pytest.raises(he.HeError) as e:  # a worker without data in a batched call
        he.he_lr_gradient_step_workers(pair.g, [([], W, out)], he.lr_config(table2()["binomial"], 0.1, g, 2.0 ** 40))
    assert e.value.code == he.HE_EINVAL


def test_lr_step_non_uniform_inputs(lr_pair):
    pair, g = lr_pair
    he = pair.he
    coeffs = table2()["binomial"]
    ms = [workloads.int_poly(30 + k, pair.n, 1 << 28) for k in range(3)]
    Zg = [pair.gpu_enc(m, 6, 200 + k, scale=2.0 ** 40, cap=7) for k, m in enumerate(ms)]
    mw = workloads.int_poly(31, pair.n, 1 << 28)
    Wg = pair.gpu_enc(mw, 6, 199, scale=2.0 ** 40)
    out = pair.g.new_ct(6)
    he.he_lr_gradient_step(pair.g, Zg, Wg, he.lr_config(coeffs, 0.1, g, 2.0 ** 40), out)
    Zo = [pair.orc_enc(m, 6, 200 + k, scale=2.0 ** 40) for k, m in enumerate(ms)]
    want = pair.o.lr_gradient_step(Zo, pair.orc_enc(mw, 6, 199, scale=2.0 ** 40), coeffs, 0.1, g,
                                   2.0 ** 40)
    assert_same_residues(out, want, he, pair.g)


@pytest.mark.parametrize("loss", ["binomial", "huber"])
def test_lr_step_accuracy_vs_fp64(lr_pair, loss):
    pair, g = lr_pair
    he = pair.he
    n_slots = pair.n // 2
    data = workloads.LRData(seed=4, n_samples=24, n_features=100)
    coeffs = table2()[loss]
    lr = 1.0 / data.n
    zs = workloads.pack_samples(data.X, data.y, n_slots, g)
    Z = pair.g.new_ct(7, len(zs))
    for k, v in enumerate(zs):
        he.he_encode_encrypt(pair.g, v, 2.0 ** 40, 7, Z[k], cid=300 + k)
    W = pair.g.new_ct(7)
    he.he_encode_encrypt(pair.g, workloads.pack_weights(data.w0, n_slots, g), 2.0 ** 40, 7, W, cid=299)
    out = pair.g.new_ct(7)
    he.he_lr_gradient_step(pair.g, Z, W, he.lr_config(coeffs, lr, g, 2.0 ** 40), out)
    got = he.he_decrypt_decode(pair.g, out)
    want = workloads.pack_weights(lr_step_fp64(data.X, data.y, data.w0, coeffs, lr), n_slots, g)
    rel = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert rel < 2.0 ** -20, rel


def test_lr_step_refuses_low_level(lr_pair):
    pair, g = lr_pair
    he = pair.he
    Z = pair.g.new_ct(5, 2)
    for k in range(2):
        he.he_encrypt_poly(pair.g, workloads.int_poly(k, pair.n, 100), 2.0 ** 40, 5, Z[k], cid=k)
    W = pair.gpu_enc(workloads.int_poly(5, pair.n, 100), 5, 5, scale=2.0 ** 40)
    out = pair.g.new_ct(5)
    with pytest.raises(he.HeError) as e:
        he.he_lr_gradient_step(pair.g, Z, W, he.lr_config(table2()["binomial"], 0.1, g, 2.0 ** 40), out)
    assert e.value.code == he.HE_ELEVEL


# ------------------------------------------------------------------ several workers in one call


def _workers_inputs(pair, sizes, levels, seed0):
    he = pair.he
    out = []
    for k, (nz, wl) in enumerate(zip(sizes, levels)):
        Z = pair.g.new_ct(7, nz)
        for i in range(nz):
            he.he_encrypt_poly(pair.g, workloads.int_poly(seed0 + 100 * k + i, pair.n, 1 << 28), 2.0 ** 40, 7,
                               Z[i], cid=seed0 + 100 * k + i)
        W = pair.gpu_enc(workloads.int_poly(seed0 + 100 * k + 99, pair.n, 1 << 28), wl, seed0 + 100 * k + 99,
                         scale=2.0 ** 40, cap=7)
        out.append((Z, W, pair.g.new_ct(7)))
    return out


@pytest.mark.parametrize("graph", [False, True])
def test_workers_match_separate_calls(lr_pair, graph):
    """Shards of uneven size at two levels in one call give the residues of
    one call per shard (each of which is bit-exact against the oracle)."""
    pair, g = lr_pair
    he = pair.he
    cfg = he.lr_config(table2()["hinge"], 0.05, g, 2.0 ** 40)
    shards = _workers_inputs(pair, [3, 1, 5, 2], [7, 6, 7, 6], 5000)
    import torch
    side = torch.cuda.Stream()  # graph capture needs a non-default stream
    torch.cuda.synchronize()
    he.he_set_stream(pair.g, side.cuda_stream)
    try:
        for _ in range(2 if graph else 1):  # a graph call captures, the next one replays
            he.he_lr_gradient_step_workers(pair.g, shards, cfg, graph=graph)
        he.he_sync(pair.g)
    finally:
        he.he_set_stream(pair.g, torch.cuda.current_stream().cuda_stream)
    for Z, W, W_out in shards:
        Zv = [Z_i for Z_i in Z]
        if W.level < 7:
            Zd = pair.g.new_ct(7, len(Z))
            for i, z in enumerate(Z):
                he.he_drop_level(pair.g, z, W.level, Zd[i])
            Zv = Zd
        single = pair.g.new_ct(7)
        he.he_lr_gradient_step(pair.g, Zv, W, cfg, single)
        assert W_out.level == W.level - 5
        assert np.array_equal(he.he_ct_export(pair.g, W_out), he.he_ct_export(pair.g, single))


@pytest.mark.parametrize("graph", [False, True])
def test_workers_match_oracle(lr_pair, graph):
    """Three workers of 1, 3 and 2 data ciphertexts, weights at levels 7, 7
    and 6 (no refresh), in one batched call (eager, and captured then
    replayed as a CUDA graph): each worker's new weights equal the oracle's
    step on that worker's data, residue for residue."""
    pair, g = lr_pair
    he = pair.he
    coeffs, lr, ms = table2()["huber"], 0.05, 2.0 ** 40
    sizes, wlevels = [1, 3, 2], [7, 7, 6]
    shards, wants = [], []
    for k, (nz, wl) in enumerate(zip(sizes, wlevels)):
        mz = [workloads.int_poly(9000 + 100 * k + i, pair.n, 1 << 28) for i in range(nz)]
        mw = workloads.int_poly(9000 + 100 * k + 99, pair.n, 1 << 28)
        Z = pair.g.new_ct(7, nz)
        for i, m in enumerate(mz):
            he.he_encrypt_poly(pair.g, m, 2.0 ** 40, 7, Z[i], cid=9000 + 100 * k + i)
        W = pair.gpu_enc(mw, wl, 9000 + 100 * k + 99, scale=2.0 ** 40, cap=7)
        shards.append((Z, W, pair.g.new_ct(7)))
        Zo = [pair.orc_enc(m, 7, 9000 + 100 * k + i, scale=2.0 ** 40) for i, m in enumerate(mz)]
        Zo = [oracle.Ciphertext(np.ascontiguousarray(z.data[:, :wl]), wl, z.scale) for z in Zo]
        Wo = pair.orc_enc(mw, wl, 9000 + 100 * k + 99, scale=2.0 ** 40)
        wants.append(pair.o.lr_gradient_step(Zo, Wo, coeffs, lr, g, ms))
    cfg = he.lr_config(coeffs, lr, g, ms)
    import torch
    side = torch.cuda.Stream()  # graph capture needs a non-default stream
    torch.cuda.synchronize()
    he.he_set_stream(pair.g, side.cuda_stream)
    try:
        for _ in range(2 if graph else 1):  # a graph call captures, the next one replays
            he.he_lr_gradient_step_workers(pair.g, shards, cfg, graph=graph)
        he.he_sync(pair.g)
    finally:
        he.he_set_stream(pair.g, torch.cuda.current_stream().cuda_stream)
    for (Z, W, W_out), want in zip(shards, wants):
        assert_same_residues(W_out, want, he, pair.g)


def test_workers_refresh_low_levels(lr_pair):
    """A worker whose weights have too few limbs left is refreshed by the
    in-process key holder first (Algorithm 1); the decrypted
    result still matches the FP64 update."""
    pair, g = lr_pair
    he = pair.he
    n_slots = pair.n // 2
    coeffs = table2()["binomial"]
    shards, datas = [], []
    for k, wl in enumerate([3, 7]):
        data = workloads.LRData(seed=20 + k, n_samples=12, n_features=60)
        datas.append(data)
        zs = workloads.pack_samples(data.X, data.y, n_slots, g)
        Z = pair.g.new_ct(7, len(zs))
        for i, v in enumerate(zs):
            he.he_encode_encrypt(pair.g, v, 2.0 ** 40, 7, Z[i], cid=700 + 10 * k + i)
        W = pair.g.new_ct(7)
        he.he_encode_encrypt(pair.g, workloads.pack_weights(data.w0, n_slots, g), 2.0 ** 40, wl, W, cid=690 + k)
        shards.append((Z, W, pair.g.new_ct(7)))
    with pytest.raises(he.HeError) as e:
        he.he_lr_gradient_step_workers(pair.g, shards, he.lr_config(coeffs, 1 / 12, g, 2.0 ** 40))
    assert e.value.code == he.HE_ELEVEL
    he.he_lr_gradient_step_workers(pair.g, shards, he.lr_config(coeffs, 1 / 12, g, 2.0 ** 40), refresh_level=7)
    for (Z, W, W_out), data in zip(shards, datas):
        assert W_out.level == 2
        got = he.he_decrypt_decode(pair.g, W_out)
        want = workloads.pack_weights(lr_step_fp64(data.X, data.y, data.w0, coeffs, 1 / 12), n_slots, g)
        assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 2.0 ** -20


# ------------------------------------------------------------------ inference


def test_inference_bit_exact_and_accurate(lr_pair):
    pair, g = lr_pair
    he = pair.he
    n_slots = pair.n // 2
    coeffs = table2()["hinge"]
    ms = [workloads.int_poly(80 + k, pair.n, 1 << 28) for k in range(3)]
    mw = workloads.int_poly(89, pair.n, 1 << 28)
    Z = pair.g.new_ct(7, 3)
    for k, m in enumerate(ms):
        he.he_encrypt_poly(pair.g, m, 2.0 ** 40, 6, Z[k], cid=80 + k)
    W = pair.gpu_enc(mw, 6, 89, scale=2.0 ** 40)
    S = pair.g.new_ct(7, 3)
    he.he_lr_inference_workers(pair.g, [(Z, W, S)], he.lr_config(coeffs, 1.0, g, 2.0 ** 40))
    Zo = [pair.orc_enc(m, 6, 80 + k, scale=2.0 ** 40) for k, m in enumerate(ms)]
    want = pair.o.lr_inference(Zo, pair.orc_enc(mw, 6, 89, scale=2.0 ** 40), coeffs, 1.0, g)
    for k in range(3):
        assert_same_residues(S[k], want[k], he, pair.g)
    # accuracy on real data
    data = workloads.LRData(seed=9, n_samples=2 * g, n_features=90)
    zs = workloads.pack_samples(data.X, data.y, n_slots, g)
    Z2 = pair.g.new_ct(7, len(zs))
    for k, v in enumerate(zs):
        he.he_encode_encrypt(pair.g, v, 2.0 ** 40, 7, Z2[k], cid=900 + k)
    W2 = pair.g.new_ct(7)
    he.he_encode_encrypt(pair.g, workloads.pack_weights(data.w0, n_slots, g), 2.0 ** 40, 7, W2, cid=899)
    S2 = pair.g.new_ct(7, len(zs))
    he.he_lr_inference_workers(pair.g, [(Z2, W2, S2)], he.lr_config(coeffs, 1.0, g, 2.0 ** 40))
    m = data.y * (data.X @ data.w0)
    p = coeffs[0] + coeffs[1] * m + coeffs[2] * m * m + coeffs[3] * m ** 3
    for k in range(len(zs)):
        assert S2[k].level == 4
        got = he.he_decrypt_decode(pair.g, S2[k])
        for s in range(g):
            assert np.max(np.abs(got[s::g] - p[k * g + s])) < 2.0 ** -20


@pytest.mark.parametrize("g", [1, 128])
def test_extreme_packings_bit_exact(g):
    """One sample per ciphertext (g = 1: no per-feature sum, no replication)
    and 128 samples of 4 features each: both kinds against the oracle."""
    log_n = 10
    n_slots = (1 << log_n) // 2
    pair = Pair(log_n, 7, 40, 1, 60, 2.0 ** 40, seed=5, rots=rot_steps(n_slots, g))
    he = pair.he
    coeffs = table2()["hinge"]
    ms = [workloads.int_poly(500 + k, pair.n, 1 << 28) for k in range(2)]
    mw = workloads.int_poly(509, pair.n, 1 << 28)
    Zg = pair.g.new_ct(7, 2)
    for k, m in enumerate(ms):
        he.he_encrypt_poly(pair.g, m, 2.0 ** 40, 7, Zg[k], cid=500 + k)
    Wg = pair.gpu_enc(mw, 7, 509, scale=2.0 ** 40)
    Zo = [pair.orc_enc(m, 7, 500 + k, scale=2.0 ** 40) for k, m in enumerate(ms)]
    Wo = pair.orc_enc(mw, 7, 509, scale=2.0 ** 40)
    out = pair.g.new_ct(7)
    he.he_lr_gradient_step(pair.g, Zg, Wg, he.lr_config(coeffs, 0.25, g, 2.0 ** 40), out)
    assert_same_residues(out, pair.o.lr_gradient_step(Zo, Wo, coeffs, 0.25, g, 2.0 ** 40), he, pair.g)
    S = pair.g.new_ct(7, 2)
    he.he_lr_inference_workers(pair.g, [(Zg, Wg, S)], he.lr_config(coeffs, 1.0, g, 2.0 ** 40))
    want = pair.o.lr_inference(Zo, Wo, coeffs, 1.0, g)
    for k in range(2):
        assert_same_residues(S[k], want[k], he, pair.g)


def test_host_input_step_matches_device_step():
    """The step on host buffers (copies overlapped with the circuit, in chunks
    of 5 and in the library's own short first chunk and budget-sized rest)
    gives the residues of the step on device buffers, at a ring size with the
    fused kernels and a ragged number of data ciphertexts."""
    import torch
    log_n, g = 12, 8
    n_slots = (1 << log_n) // 2
    he = gpu_lib()
    ctx = he.Context(log_n, 7, 40, 2, 55, 2.0 ** 40, seed=21, rot_steps=rot_steps(n_slots, g))
    nZ = 37
    Z = ctx.new_ct(7, nZ)
    for k in range(nZ):
        he.he_encrypt_poly(ctx, workloads.int_poly(700 + k, ctx.n, 1 << 28), 2.0 ** 40, 7, Z[k], cid=700 + k)
    W = ctx.new_ct(7)
    he.he_encrypt_poly(ctx, workloads.int_poly(799, ctx.n, 1 << 28), 2.0 ** 40, 7, W, cid=799)
    cfg = he.lr_config(table2()["binomial"], 1.0 / (nZ * g), g, 2.0 ** 27)
    he.he_set_tuning(ctx, "lr_chunk", 5)
    out = ctx.new_ct(7)
    he.he_lr_gradient_step(ctx, Z, W, cfg, out)
    want = he.he_ct_export(ctx, out)
    zh = torch.empty((nZ, 2, 7, ctx.n), dtype=torch.int64, pin_memory=True)
    he.he_ct_export_batch(ctx, Z, zh)
    wh = he.he_ct_export(ctx, W)
    oh = np.zeros((2, 2, ctx.n), dtype=np.uint64)
    # chunks of 5; then the library's own: a first chunk of one 16-ciphertext
    # piece, the rest in one chunk of the budget
    for chunk in (5, 0):
        he.he_set_tuning(ctx, "lr_chunk", chunk)
        for _ in range(2):  # the second call reuses the device buffers and events
            oh[:] = 0
            level, scale = he.he_lr_gradient_step_host(ctx, zh, 7, 2.0 ** 40, wh, 7, 2.0 ** 40, cfg, oh)
            assert level == 2 and scale == out.scale
            assert np.array_equal(oh, want), chunk
    with pytest.raises(he.HeError) as e:
        he.he_lr_gradient_step_host(ctx, zh, 7, 2.0 ** 40, wh[:, :5].copy(), 5, 2.0 ** 40, cfg, oh)
    assert e.value.code == he.HE_ELEVEL


def test_batched_import_export_round_trip():
    """Uniform batches move in one copy per contiguous run; ciphertexts with
    spare capacity or in separate buffers still land limb by limb."""
    he = gpu_lib()
    ctx = he.Context(11, 5, 40, 1, 60, 2.0 ** 40, seed=22)
    data = workloads.residues(5, ctx.primes[:4], ctx.n, parts=2 * 6).reshape(6, 2, 4, ctx.n)
    uni = ctx.new_ct(4, 6)
    he.he_ct_import_batch(ctx, data, 4, 2.0 ** 40, uni)
    mixed = [ctx.new_ct(5) for _ in range(3)] + ctx.new_ct(4, 3)
    he.he_ct_import_batch(ctx, data, 4, 2.0 ** 40, mixed)
    for cts in (uni, mixed):
        for i, ct in enumerate(cts):
            assert np.array_equal(he.he_ct_export(ctx, ct), data[i])
        back = np.zeros_like(data)
        he.he_ct_export_batch(ctx, cts, back)
        assert np.array_equal(back, data)


def test_lr_step_and_inference_bit_exact_fused_kernels():
    """At N = 2^12 the step runs on the fused kernels (key switch, ModDown,
    rescale, rotate-and-add) with two special primes: residues equal the
    oracle's op-for-op evaluation."""
    log_n, g = 12, 8
    n_slots = (1 << log_n) // 2
    pair = Pair(log_n, 7, 40, 2, 55, 2.0 ** 40, seed=13, rots=rot_steps(n_slots, g))
    he = pair.he
    coeffs = table2()["huber"]
    ms = [workloads.int_poly(600 + k, pair.n, 1 << 28) for k in range(3)]
    mw = workloads.int_poly(609, pair.n, 1 << 28)
    Zg = pair.g.new_ct(7, 3)
    for k, m in enumerate(ms):
        he.he_encrypt_poly(pair.g, m, 2.0 ** 40, 7, Zg[k], cid=600 + k)
    Wg = pair.gpu_enc(mw, 7, 609, scale=2.0 ** 40)
    Zo = [pair.orc_enc(m, 7, 600 + k, scale=2.0 ** 40) for k, m in enumerate(ms)]
    Wo = pair.orc_enc(mw, 7, 609, scale=2.0 ** 40)
    out = pair.g.new_ct(7)
    he.he_lr_gradient_step(pair.g, Zg, Wg, he.lr_config(coeffs, 0.125, g, 2.0 ** 30), out)
    assert_same_residues(out, pair.o.lr_gradient_step(Zo, Wo, coeffs, 0.125, g, 2.0 ** 30), he, pair.g)
    S = pair.g.new_ct(7, 3)
    he.he_lr_inference_workers(pair.g, [(Zg, Wg, S)], he.lr_config(coeffs, 1.0, g, 2.0 ** 40))
    want = pair.o.lr_inference(Zo, Wo, coeffs, 1.0, g)
    for k in range(3):
        assert_same_residues(S[k], want[k], he, pair.g)


@pytest.mark.parametrize("refresh_every,top,iterations", [(1, 11, 3), (2, 11, 3), (3, 16, 6), (5, 26, 5)])
def test_training_loop_matches_fp64_algorithm(refresh_every, top, iterations):
    """Algorithms 1 and 2: two workers with their own data run their steps,
    the key holder averages their weights every `refresh_every` steps (the
    paper's l = 1, 3, 5) and after the last; the decrypted result equals the
    same procedure in FP64 within 2^-20 of the weights."""
    he = gpu_lib()
    log_n, g = 12, 8
    n_slots = (1 << log_n) // 2
    ctx = he.Context(log_n, top, 40, 2, 55, 2.0 ** 40, seed=17, rot_steps=rot_steps(n_slots, g))
    coeffs = table2()["binomial"]
    lr = 1.0 / 16
    w0 = workloads.LRData(seed=40, n_samples=16, n_features=200).w0
    datas = [workloads.LRData(seed=41 + k, n_samples=16, n_features=200) for k in range(2)]
    workers = []
    for k, d in enumerate(datas):
        zs = workloads.pack_samples(d.X, d.y, n_slots, g)
        Z = ctx.new_ct(top, len(zs))
        for i, v in enumerate(zs):
            he.he_encode_encrypt(ctx, v, 2.0 ** 40, top, Z[i], cid=100 * k + i)
        W = ctx.new_ct(top)
        he.he_encode_encrypt(ctx, workloads.pack_weights(w0, n_slots, g), 2.0 ** 40, top, W, cid=100 * k + 99)
        workers.append((Z, W))
    out = ctx.new_ct(top)
    cfg = he.lr_config(coeffs, lr, g, 2.0 ** 27)
    he.he_lr_train(ctx, workers, cfg, iterations, refresh_every, top, out)
    assert out.level == top
    ws = [w0.copy() for _ in datas]
    for it in range(1, iterations + 1):
        ws = [lr_step_fp64(d.X, d.y, w, coeffs, lr) for d, w in zip(datas, ws)]
        if it % refresh_every == 0 or it == iterations:
            avg = sum(ws) / len(ws)
            ws = [avg.copy() for _ in ws]
    want = workloads.pack_weights(ws[0], n_slots, g)
    got = he.he_decrypt_decode(ctx, out)
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 2.0 ** -20
    with pytest.raises(he.HeError) as e:  # the limbs hold fewer steps than that between refreshes
        he.he_lr_train(ctx, workers, cfg, iterations, (top - 1) // 5 + 1, top, out)
    assert e.value.code == he.HE_ELEVEL


def test_sum_of_weights_equals_oracle_additions(lr_pair):
    """he_sum (the aggregation of Algorithm 2) of four ciphertexts, uniform and
    not, equals the oracle's chained additions residue for residue."""
    pair, g = lr_pair
    he = pair.he
    ms = [workloads.int_poly(300 + k, pair.n, 1 << 30) for k in range(4)]
    want = pair.orc_enc(ms[0], 6, 300)
    for k in range(1, 4):
        want = pair.o.add(want, pair.orc_enc(ms[k], 6, 300 + k))
    uni = pair.g.new_ct(7, 4)
    for k, m in enumerate(ms):
        he.he_encrypt_poly(pair.g, m, 2.0 ** 40, 6, uni[k], cid=300 + k)
    loose = [pair.gpu_enc(m, 6, 300 + k) for k, m in enumerate(ms)]
    for cts in (uni, loose):
        out = pair.g.new_ct(7)
        he.he_sum(pair.g, cts, out)
        assert_same_residues(out, want, he, pair.g)
    he.he_sum(pair.g, loose, loose[0])  # in place on the first
    assert_same_residues(loose[0], want, he, pair.g)


def test_sharded_training_loop_one_rank_matches_fp64():
    """The sharded Algorithms 1-2 loop on one process (three workers, the
    key holder's average taken as the decrypted modular sum of their
    weights): within 2^-20 of the FP64 procedure."""
    from paper_2006_10091_gb300 import sharding
    he = gpu_lib()
    log_n, g, top = 12, 8, 11
    n_slots = (1 << log_n) // 2
    ctx = he.Context(log_n, top, 40, 2, 55, 2.0 ** 40, seed=17, rot_steps=rot_steps(n_slots, g))
    coeffs = table2()["binomial"]
    lr = 1.0 / 16
    w0 = workloads.LRData(seed=40, n_samples=16, n_features=200).w0
    datas = [workloads.LRData(seed=51 + k, n_samples=8 * (k + 1), n_features=200) for k in range(3)]
    parts = sharding.partition_shards([len(d.y) // g for d in datas], 1)
    assert parts == [[0, 1, 2]]
    workers = []
    for k, d in enumerate(datas):
        zs = workloads.pack_samples(d.X, d.y, n_slots, g)
        Z = ctx.new_ct(top, len(zs))
        for i, v in enumerate(zs):
            he.he_encode_encrypt(ctx, v, 2.0 ** 40, top, Z[i], cid=100 * k + i)
        W = ctx.new_ct(top)
        he.he_encode_encrypt(ctx, workloads.pack_weights(w0, n_slots, g), 2.0 ** 40, top, W, cid=100 * k + 99)
        workers.append((Z, W))
    cfg = he.lr_config(coeffs, lr, g, 2.0 ** 27)
    out = sharding.train_sharded(ctx, workers, cfg, 3, 2, top, 5000, len(workers))
    assert out.level == top
    ws = [w0.copy() for _ in datas]
    for it in range(1, 4):
        ws = [lr_step_fp64(d.X, d.y, w, coeffs, lr) for d, w in zip(datas, ws)]
        if it % 2 == 0 or it == 3:
            avg = sum(ws) / len(ws)
            ws = [avg.copy() for _ in ws]
    want = workloads.pack_weights(ws[0], n_slots, g)
    got = he.he_decrypt_decode(ctx, out)
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 2.0 ** -20
