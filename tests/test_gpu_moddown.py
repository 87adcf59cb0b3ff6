"""ModDown on the GPU equals the oracle's exact-lift ModDown on accumulators
whose dropped part lifts to 0, 1, 2, D - 2 or D - 1 after adding h = (D - 1)/2
(D = P for a key switch, P q_{l-1} for the multiplication's ModDown merged
with its rescale), through the C ABI's he_moddown, in the fused kernels and
in the separate-kernel path, from two to eight dropped primes, including the
LR step's parameters (N = 2^14, eight 40-bit limbs, two 59-bit special
primes).  Residues must be equal bit for bit."""
import numpy as np
import pytest

import oracle
from tests import moddown_inputs as mi
from tests.gpu_util import Pair, gpu_lib

pytestmark = pytest.mark.gpu

CONFIGS = {
    # name: (log_n, L, limb_bits, alpha, special_bits, levels)
    "n12_a2": (12, 6, 40, 2, 59, (6, 3)),
    "n13_a4": (13, 8, 40, 4, 50, (8, 5)),
    "n12_a7": (12, 8, 50, 7, 61, (8, 2)),  # merged: eight dropped primes, the tables' limit
    "n14_step": (14, 8, 40, 2, 59, (8, 7)),
}


@pytest.fixture(scope="module", params=sorted(CONFIGS))
def pair(request):
    log_n, L, lb, alpha, sb, levels = CONFIGS[request.param]
    return Pair(log_n, L, lb, alpha, sb, 2.0 ** 40, seed=21), levels


def _run(pr, acc, level, d01):
    import torch
    he, g = pr.he, pr.g
    t = torch.from_numpy(np.ascontiguousarray(acc).view(np.int64).copy()).cuda()
    lt = level - 1 if d01 is not None else level
    out = g.new_ct(lt)
    if d01 is None:
        he.he_moddown(g, t, level, out)
    else:
        d = pr.gpu_ct(oracle.Ciphertext(d01, level, 2.0 ** 40))
        he.he_moddown(g, t, level, out, d01=d)
    assert out.level == lt
    return he.he_ct_export(g, out)


@pytest.mark.parametrize("merged", [False, True])
@pytest.mark.parametrize("generic", [False, True])
def test_moddown_boundary_lifts_bit_exact(pair, merged, generic):
    pr, levels = pair
    he = gpu_lib()
    he.he_set_tuning(pr.g, "ntt_generic", 1 if generic else 0)
    try:
        for level in levels:
            acc, d01, X, D = mi.accumulator(pr.o, level, seed=31 + level, merged=merged)
            want = pr.o.moddown_rescale(acc, d01, level) if merged else np.stack(pr.o.moddown(acc, level))
            got = _run(pr, acc, level, d01)
            if not np.array_equal(got, want):
                bad = np.argwhere(got != want)
                raise AssertionError(f"level {level}: {len(bad)} residues differ, first at {bad[0].tolist()}")
    finally:
        he.he_set_tuning(pr.g, "ntt_generic", 0)


def test_moddown_errors(pair):
    import torch
    pr, levels = pair
    he = gpu_lib()
    g = pr.g
    t = torch.zeros(2 * (g.L + g.alpha) * g.n, dtype=torch.int64, device="cuda")
    out = g.new_ct(g.L)
    with pytest.raises(he.HeError):
        he.he_moddown(g, t, 0, out)
    with pytest.raises((he.HeError, ValueError)):  # refused by the binding's size check or the library
        he.he_moddown(g, t, g.L + 1, out)
    d = g.new_ct(1)
    d.level = 1
    with pytest.raises(he.HeError):  # the merged form needs two limbs
        he.he_moddown(g, t, 1, out, d01=d)
