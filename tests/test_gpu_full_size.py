"""Full-size checks, in the launch configuration the benchmark times: the
encrypted LR step over 4096 samples x 784 features at N = 2^14 (512 data
ciphertexts, 8 limbs + 2 special primes, one batch), and multiplication and
rotation at N = 2^16 with 24 limbs and 4 special primes.  The oracle cannot
run these sizes whole, so they are checked through properties: decryption
against FP64 within the 2^-20 gate; the device step, the host-input step and
the many-worker entry point giving identical residues; and sampled key-switch
outputs recomputed by the oracle at the same parameters (one coefficient
column at a time is not separable, so the oracle key-switches one input)."""
import math

import numpy as np
import pytest

from paper_2006_10091_gb300 import workloads
from tests.gpu_util import gpu_lib
from tests.lr_reference import lr_step_fp64, table2

pytestmark = pytest.mark.gpu


def test_full_size_step_accuracy_and_entry_points_agree():
    import torch
    he = gpu_lib()
    log_n, L, g = 14, 8, 8
    n_slots = (1 << log_n) // 2
    F = n_slots // g
    ctx = he.Context(log_n, L, 40, 2, 59, 2.0 ** 40, seed=0, rot_steps=he.lr_rot_steps(n_slots, g))
    he.he_autotune(ctx, L - 1, 64)
    data = workloads.LRData(seed=0, n_samples=4096, n_features=784)
    zs = workloads.pack_samples(data.X, data.y, n_slots, g)
    assert len(zs) == 512
    Z = ctx.new_ct(L, len(zs))
    for k, v in enumerate(zs):
        he.he_encode_encrypt(ctx, v, 2.0 ** 40, L, Z[k], cid=1000 + k)
    W = ctx.new_ct(L)
    he.he_encode_encrypt(ctx, workloads.pack_weights(data.w0, n_slots, g), 2.0 ** 40, L, W, cid=999)
    coeffs = table2()["binomial"]
    cfg = he.lr_config(coeffs, 1.0 / 4096, g, 2.0 ** 27)
    out = ctx.new_ct(L)
    he.he_lr_gradient_step(ctx, Z, W, cfg, out)
    got = he.he_decrypt_decode(ctx, out)
    want = workloads.pack_weights(lr_step_fp64(data.X, data.y, data.w0, coeffs, 1.0 / 4096), n_slots, g)
    rel = float(np.max(np.abs(got - want)) / np.max(np.abs(want)))
    assert rel < 2.0 ** -20, rel
    ref = he.he_ct_export(ctx, out)
    # host buffers, copies overlapped
    zh = torch.empty((512, 2, L, ctx.n), dtype=torch.int64, pin_memory=True)
    he.he_ct_export_batch(ctx, Z, zh)
    oh = np.zeros((2, L - 5, ctx.n), dtype=np.uint64)
    for _ in range(3):  # later calls size the first chunk from the previous call's timings
        oh[:] = 0
        he.he_lr_gradient_step_host(ctx, zh, L, 2.0 ** 40, he.he_ct_export(ctx, W), L, 2.0 ** 40, cfg, oh)
        assert np.array_equal(oh, ref)
    # the same shard as one of several workers, graph-captured
    other = ctx.new_ct(L, 8)
    for k in range(8):
        he.he_encrypt_poly(ctx, workloads.int_poly(5000 + k, ctx.n, 1 << 28), 2.0 ** 40, L, other[k], cid=5000 + k)
    W2, O1, O2 = ctx.new_ct(L), ctx.new_ct(L), ctx.new_ct(L)
    he.he_encrypt_poly(ctx, workloads.int_poly(5100, ctx.n, 1 << 28), 2.0 ** 40, L, W2, cid=5100)
    for graph in (False, True):
        he.he_lr_gradient_step_workers(ctx, [(Z, W, O1), (other, W2, O2)], cfg, graph=graph)
        assert np.array_equal(he.he_ct_export(ctx, O1), ref)


def test_large_parameters_mul_rotate_accuracy():
    """N = 2^16, 24 x ~50-bit limbs, 4 special primes (dnum 6), scale 2^50:
    mul+relin+rescale and a 1024-slot rotate-and-sum decrypt within 1e-8 of
    FP64 at the top level and after several levels."""
    he = gpu_lib()
    stages = he.rotsum_stages(1, 10)
    rots = [1 << t for t in range(10)]
    rots += [r for st in stages for r in st if r not in rots]
    ctx = he.Context(16, 24, 50, 4, 60, 2.0 ** 50, seed=1, rot_steps=rots)
    n_slots = ctx.n // 2
    za, zb = workloads.uniform_slots(1, n_slots), workloads.uniform_slots(2, n_slots)
    a, b, c = ctx.new_ct(24), ctx.new_ct(24), ctx.new_ct(24)
    he.he_encode_encrypt(ctx, za, 2.0 ** 50, 24, a, cid=1)
    he.he_encode_encrypt(ctx, zb, float(ctx.primes[23]), 24, b, cid=2)
    he.he_mul_relin_rescale(ctx, a, b, c)
    assert c.level == 23
    assert float(np.max(np.abs(he.he_decrypt_decode(ctx, c) - za * zb))) < 1e-8
    # rotate-and-sum over 1024 positions at level 23: one rotation and one
    # addition at a time, and in hoisted stages (in place)
    c2 = ctx.new_ct(24)
    he.he_ct_import(ctx, he.he_ct_export(ctx, c), 23, c.scale, c2)
    t = ctx.new_ct(24)
    for s in range(10):
        he.he_rotate(ctx, c, 1 << s, t)
        he.he_add(ctx, c, t, c)
    want = sum(np.roll(za * zb, -k) for k in range(1024))
    assert float(np.max(np.abs(he.he_decrypt_decode(ctx, c) - want))) < 1e-7
    for st in stages:
        he.he_rotate_sum(ctx, c2, st, c2)
    assert float(np.max(np.abs(he.he_decrypt_decode(ctx, c2) - want))) < 1e-7


def test_full_size_keyswitch_matches_oracle():
    """The relinearisation key switch at the step's parameters (N = 2^14, 8
    limbs, 2 special primes), level 7, with the autotuned kernel knobs,
    against the oracle's residues."""
    import torch
    from tests.gpu_util import Pair
    pair = Pair(14, 8, 40, 2, 59, 2.0 ** 40, seed=0)
    he = pair.he
    he.he_autotune(pair.g, 7, 64)
    d = workloads.residues(77, pair.o.primes[:7], pair.n)[0]
    k0, k1 = pair.o.keyswitch(d, 7, -1)
    dt = torch.from_numpy(d.view(np.int64).copy()).cuda()
    o0, o1 = torch.empty_like(dt), torch.empty_like(dt)
    he.he_keyswitch(pair.g, dt, 7, 0, o0, o1)
    assert np.array_equal(o0.cpu().numpy().view(np.uint64), k0)
    assert np.array_equal(o1.cpu().numpy().view(np.uint64), k1)
