"""Helpers for the GPU parity tests: a CPU oracle context and a GPU context
built from the same parameters and seed (hence the same primes and keys)."""
import functools

import numpy as np
import pytest

import oracle


@functools.lru_cache(maxsize=None)
def gpu_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_10091_gb300 import build as B
    B.build()
    import paper_2006_10091_gb300 as he
    he.load()
    return he


class Pair:
    def __init__(self, log_n, L, limb_bits, alpha, special_bits, scale, seed=0, rots=(), sigma=3.2):
        he = gpu_lib()
        self.he = he
        self.o = oracle.Oracle(log_n, L, limb_bits, alpha, special_bits, scale, sigma=sigma, seed=seed,
                               rot_steps=rots)
        self.g = he.Context(log_n, L, limb_bits, alpha, special_bits, scale, sigma=sigma, seed=seed,
                            rot_steps=rots)
        assert self.g.primes == self.o.primes
        self.n, self.L = 1 << log_n, L

    def gpu_ct(self, ct: "oracle.Ciphertext", cap=None):
        """Import oracle residues into a fresh GPU buffer."""
        out = self.g.new_ct(cap or ct.level)
        self.he.he_ct_import(self.g, ct.data, ct.level, ct.scale, out)
        return out

    def gpu_enc(self, m, level, cid, use_sk=False, scale=None, cap=None):
        out = self.g.new_ct(cap or level)
        self.he.he_encrypt_poly(self.g, m, scale or self.g.scale, level, out, use_sk=use_sk, cid=cid)
        return out

    def orc_enc(self, m, level, cid, use_sk=False, scale=None):
        return self.o.encrypt(m, level, use_sk=use_sk, cid=cid, scale=scale or self.o.scale)


def assert_same_residues(gpu_ct, orc_ct, he, ctx):
    got = he.he_ct_export(ctx, gpu_ct)
    assert gpu_ct.level == orc_ct.level
    want = np.asarray(orc_ct.data, dtype=np.uint64)
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        raise AssertionError(f"{len(bad)} residues differ, first at {bad[0].tolist()}: "
                             f"{got[tuple(bad[0])]} vs {want[tuple(bad[0])]}")
    assert gpu_ct.scale == pytest.approx(orc_ct.scale, rel=1e-15)
