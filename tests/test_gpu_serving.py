"""The continuous-batching request loop: requests of two ring sizes and both
kinds (gradient step, inference), some with weights too low for the circuit
(refreshed in-process first), submitted together to a server with several
concurrent waves, give exactly the residues they give when served one at a
time; the decrypted results match FP64; the device memory held stays within
the budget."""
import math

import numpy as np
import pytest

from paper_2006_10091_gb300 import workloads
from tests.gpu_util import Pair, gpu_lib
from tests.lr_reference import lr_step_fp64, table2

pytestmark = pytest.mark.gpu


def rots(he, n_slots, g):
    return he.lr_rot_steps(n_slots, g)


@pytest.fixture(scope="module")
def setup():
    he = gpu_lib()
    # 16 samples of 64 (N = 2^11) or 128 (N = 2^12) feature positions per ciphertext
    ctxs = [he.Context(11, 7, 40, 1, 60, 2.0 ** 40, seed=31, rot_steps=rots(he, 1 << 10, 16)),
            he.Context(12, 7, 40, 2, 50, 2.0 ** 40, seed=32, rot_steps=rots(he, 1 << 11, 16))]
    coeffs = table2()["binomial"]
    reqs = []
    for r in range(10):
        ci = r % 2
        ctx = ctxs[ci]
        n_slots = ctx.n // 2
        feats = 64 if ci == 0 else 128  # 16 samples per ciphertext in both rings
        g = n_slots // feats
        kind = he.HE_REQ_GRADIENT if r % 3 else he.HE_REQ_INFERENCE
        nz = 1 + r % 3
        w_level = [7, 3, 6, 2, 7][r % 5]
        data = workloads.LRData(seed=200 + r, n_samples=nz * g, n_features=feats - 3)
        zs = workloads.pack_samples(data.X, data.y, n_slots, g)
        Z = ctx.new_ct(7, nz)
        for k, v in enumerate(zs):
            he.he_encode_encrypt(ctx, v, 2.0 ** 40, 7, Z[k], cid=1000 * r + k)
        W = ctx.new_ct(7)
        he.he_encode_encrypt(ctx, workloads.pack_weights(data.w0, n_slots, g), 2.0 ** 40, w_level, W, cid=1000 * r + 99)
        Zh = np.stack([he.he_ct_export(ctx, z) for z in Z])
        Wh = he.he_ct_export(ctx, W)
        lr = 1.0 / 64 if kind == he.HE_REQ_GRADIENT else 1.0
        cfg = he.lr_config(coeffs, lr, g, 2.0 ** 27 if kind == he.HE_REQ_GRADIENT else 2.0 ** 40)
        # some steps ask for a spare limb: weights below 7 limbs are refreshed
        min_w = 7 if kind == he.HE_REQ_GRADIENT and r % 2 == 0 else 0
        need = max(6 if kind == he.HE_REQ_GRADIENT else 5, min_w)
        l0 = w_level if w_level >= need else 7
        l_out = l0 - (5 if kind == he.HE_REQ_GRADIENT else 3)
        shape = (2, l_out, ctx.n) if kind == he.HE_REQ_GRADIENT else (nz, 2, l_out, ctx.n)
        reqs.append(dict(ci=ci, kind=kind, Zh=Zh, Wh=Wh, w_level=w_level, cfg=cfg, shape=shape, data=data,
                         g=g, lr=lr, nz=nz, l_out=l_out, cid=77000 + r, min_w=min_w))
    return he, ctxs, reqs, coeffs


def serve(he, ctxs, reqs, budget, inflight, wave, one_at_a_time):
    srv = he.Server(ctxs, budget, max_inflight=inflight, max_wave=wave)
    outs, ids = {}, {}
    try:
        for i, r in enumerate(reqs):
            out = np.zeros(r["shape"], dtype=np.uint64)
            rid = srv.submit(r["ci"], r["kind"], r["Zh"], 7, 2.0 ** 40, r["Wh"], r["w_level"], 2.0 ** 40,
                             r["cfg"], out, refresh_cid=r["cid"], min_w_level=r["min_w"])
            outs[rid] = out
            ids[rid] = i
            if one_at_a_time:
                srv.drain()
        srv.drain()
        res = srv.poll()
        stats = srv.stats()
    finally:
        srv.close()
    assert len(res) == len(reqs)
    by_index = {}
    for x in res:
        assert x["status"] == 0, x
        by_index[ids[x["id"]]] = (outs[x["id"]], x)
    return by_index, stats


def test_results_are_the_same_alone_and_in_the_mix(setup):
    he, ctxs, reqs, coeffs = setup
    alone, _ = serve(he, ctxs, reqs, 1 << 34, 1, 1, True)
    mixed, stats = serve(he, ctxs, reqs, 1 << 34, 3, 4, False)
    for i in range(len(reqs)):
        assert np.array_equal(alone[i][0], mixed[i][0]), i
        assert alone[i][1]["level"] == mixed[i][1]["level"] == reqs[i]["l_out"]
    assert stats["waves"] < len(reqs)  # requests that arrived together shared a wave
    # decrypted results against FP64
    for i, r in enumerate(reqs):
        ctx = ctxs[r["ci"]]
        n_slots = ctx.n // 2
        out, info = mixed[i]
        if r["kind"] == he.HE_REQ_GRADIENT:
            ct = ctx.new_ct(r["l_out"])
            he.he_ct_import(ctx, out, r["l_out"], info["scale"], ct)
            got = he.he_decrypt_decode(ctx, ct)
            d = r["data"]
            want = workloads.pack_weights(lr_step_fp64(d.X, d.y, d.w0, coeffs, r["lr"]), n_slots, r["g"])
            assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 2.0 ** -20
        else:
            d = r["data"]
            m = d.y * (d.X @ d.w0)
            p = coeffs[0] + coeffs[1] * m + coeffs[2] * m * m + coeffs[3] * m ** 3
            for k in range(r["nz"]):
                ct = ctx.new_ct(r["l_out"])
                he.he_ct_import(ctx, out[k], r["l_out"], info["scale"], ct)
                got = he.he_decrypt_decode(ctx, ct)
                for s in range(r["g"]):
                    assert np.max(np.abs(got[s::r["g"]] - p[k * r["g"] + s])) < 2.0 ** -20


def test_budget_bounds_device_memory(setup):
    he, ctxs, reqs, _ = setup
    budget = 256 << 20
    _, stats = serve(he, ctxs, reqs[:6], budget, 3, 4, False)
    assert stats["used"] == 0 or stats["used"] <= stats["peak_used"]
    assert stats["peak_used"] <= budget


def test_served_results_equal_the_oracle():
    """A gradient request and an inference request (N = 2^12, two special
    primes, weights at the data's level: no refresh), served together and
    each alone: the result residues equal the oracle's step and inference on
    the same ciphertexts."""
    he = gpu_lib()
    g, n_slots = 16, 1 << 11
    pair = Pair(12, 7, 40, 2, 50, 2.0 ** 40, seed=32, rots=rots(he, n_slots, g))
    coeffs = table2()["binomial"]
    data = workloads.LRData(seed=400, n_samples=2 * g, n_features=125)
    zs = workloads.pack_samples(data.X, data.y, n_slots, g)
    Zo = [pair.orc_enc(pair.o.encode(v, scale=2.0 ** 40), 7, 500 + k, scale=2.0 ** 40) for k, v in enumerate(zs)]
    Wo = pair.orc_enc(pair.o.encode(workloads.pack_weights(data.w0, n_slots, g), scale=2.0 ** 40), 7, 499,
                      scale=2.0 ** 40)
    Zh = np.ascontiguousarray(np.stack([z.data for z in Zo]))
    Wh = np.ascontiguousarray(Wo.data)
    grad_cfg = he.lr_config(coeffs, 1.0 / 64, g, 2.0 ** 27)
    inf_cfg = he.lr_config(coeffs, 1.0, g, 2.0 ** 40)
    want_grad = pair.o.lr_gradient_step(Zo, Wo, coeffs, 1.0 / 64, g, 2.0 ** 27)
    want_inf = pair.o.lr_inference(Zo, Wo, coeffs, 1.0, g)
    for together in (True, False):
        srv = he.Server([pair.g], 1 << 34, max_inflight=2, max_wave=4)
        try:
            out_g = np.zeros((2, 2, pair.n), dtype=np.uint64)
            out_i = np.zeros((len(zs), 2, 4, pair.n), dtype=np.uint64)
            srv.submit(0, he.HE_REQ_GRADIENT, Zh, 7, 2.0 ** 40, Wh, 7, 2.0 ** 40, grad_cfg, out_g)
            if not together:
                srv.drain()
            srv.submit(0, he.HE_REQ_INFERENCE, Zh, 7, 2.0 ** 40, Wh, 7, 2.0 ** 40, inf_cfg, out_i)
            srv.drain()
            res = srv.poll()
        finally:
            srv.close()
        assert [r["status"] for r in res] == [0, 0]
        assert np.array_equal(out_g, want_grad.data)
        for k in range(len(zs)):
            assert np.array_equal(out_i[k], want_inf[k].data), k


def test_request_larger_than_the_budget_is_refused(setup):
    """A request whose own buffers and workspace exceed the whole budget is
    refused at submit with HE_ENOMEM instead of being admitted alone."""
    he, ctxs, reqs, _ = setup
    srv = he.Server(ctxs, 1 << 20, max_inflight=1, max_wave=1)
    try:
        r = reqs[1]
        out = np.zeros(r["shape"], dtype=np.uint64)
        with pytest.raises(he.HeError) as e:
            srv.submit(r["ci"], r["kind"], r["Zh"], 7, 2.0 ** 40, r["Wh"], r["w_level"], 2.0 ** 40, r["cfg"], out,
                       refresh_cid=r["cid"], min_w_level=r["min_w"])
        assert e.value.code == he.HE_ENOMEM
        srv.drain()
        assert srv.stats()["peak_used"] == 0
    finally:
        srv.close()
