"""Bit-exact parity with the oracle at the parameters the benchmark times.

- The LR gradient step (Eq. 7-8, Table 2 binomial row) at the benchmark's
  ring and moduli: N = 2^14, eight 40-bit limbs, two 59-bit special primes,
  scale 2^40, g = 8 samples per ciphertext, mask scale 2^27, learning rate
  1/4096, on two data ciphertexts of the synthetic 784-feature data (the
  oracle encodes them; both sides encrypt the same integer coefficients).
  Every compiled tile shape runs the same step.
- Multiplication (Sec. 3: tensor, relinearisation, rescale), rotation and a
  hoisted rotate-and-sum at the large configuration (N = 2^16, 24 limbs of
  ~50 bits, four 60-bit special primes, scale 2^50) and at N = 2^15 (20
  limbs, four special primes), one ciphertext each, every tile shape.

The oracle needs one to two minutes for each configuration (key generation
dominates); every residue is compared."""
import numpy as np
import pytest

from paper_2006_10091_gb300 import workloads
from tests.gpu_util import Pair, assert_same_residues, gpu_lib
from tests.lr_reference import table2

pytestmark = pytest.mark.gpu


def test_step_at_benchmark_parameters_matches_oracle():
    he = gpu_lib()
    log_n, L, g = 14, 8, 8
    n_slots = (1 << log_n) // 2
    pair = Pair(log_n, L, 40, 2, 59, 2.0 ** 40, seed=0, rots=he.lr_rot_steps(n_slots, g))
    data = workloads.LRData(seed=0, n_samples=2 * g, n_features=784)
    zs = workloads.pack_samples(data.X, data.y, n_slots, g)
    assert len(zs) == 2
    coeffs = table2()["binomial"]
    cfg = he.lr_config(coeffs, 1.0 / 4096, g, 2.0 ** 27)
    ms = [pair.o.encode(v, scale=2.0 ** 40) for v in zs]
    mw = pair.o.encode(workloads.pack_weights(data.w0, n_slots, g), scale=2.0 ** 40)
    Zo = [pair.orc_enc(m, L, 1000 + k, scale=2.0 ** 40) for k, m in enumerate(ms)]
    Wo = pair.orc_enc(mw, L, 999, scale=2.0 ** 40)
    want = pair.o.lr_gradient_step(Zo, Wo, coeffs, 1.0 / 4096, g, 2.0 ** 27)
    Z = pair.g.new_ct(L, len(ms))
    for k, m in enumerate(ms):
        he.he_encrypt_poly(pair.g, m, 2.0 ** 40, L, Z[k], cid=1000 + k)
    W = pair.gpu_enc(mw, L, 999, scale=2.0 ** 40)
    for shape in (0, 1, 2):
        he.he_set_tuning(pair.g, "ntt_shape", shape)
        out = pair.g.new_ct(L)
        he.he_lr_gradient_step(pair.g, Z, W, cfg, out)
        assert out.level == L - 5
        assert_same_residues(out, want, he, pair.g)
    he.he_set_tuning(pair.g, "ntt_shape", 0)


LARGE = {
    # name: (log_n, L, limb bits, alpha, special bits, scale, rotate-and-sum steps)
    "n16_l24": (16, 24, 50, 4, 60, 2.0 ** 50, list(range(1, 16))),
    "n15_l20": (15, 20, 50, 4, 60, 2.0 ** 50, list(range(1, 8))),
    # the serving mix's other rings: rotations that move rows between tiles
    # at N = 2^13, a closed stage (every row tile onto itself: split sums,
    # part 0 in the product kernel) at N = 2^14 with five four-limb digits
    "n13_l20": (13, 20, 50, 4, 60, 2.0 ** 50, list(range(1, 8))),
    "n14_l20_closed": (14, 20, 50, 4, 60, 2.0 ** 50, [8, 16, 24, 32, 40, 48, 56]),
}


@pytest.mark.parametrize("name", sorted(LARGE))
def test_large_ring_ops_match_oracle(name):
    he = gpu_lib()
    log_n, L, lb, alpha, sb, scale, steps = LARGE[name]
    pair = Pair(log_n, L, lb, alpha, sb, scale, seed=0, rots=steps)
    ma = workloads.int_poly(1, pair.n, 1 << 40)
    mb = workloads.int_poly(2, pair.n, 1 << 40)
    ao = pair.orc_enc(ma, L, 1, scale=scale)
    bo = pair.orc_enc(mb, L, 2, scale=scale)
    want_mul = pair.o.mul_relin_rescale(ao, bo)
    want_rot = pair.o.rotate(ao, steps[0])
    want_sum = pair.o.rotate_sum(ao, steps)
    a = pair.gpu_enc(ma, L, 1, scale=scale)
    b = pair.gpu_enc(mb, L, 2, scale=scale)
    for shape in (0, 1, 2):
        he.he_set_tuning(pair.g, "ntt_shape", shape)
        out = pair.g.new_ct(L)
        he.he_mul_relin_rescale(pair.g, a, b, out)
        assert_same_residues(out, want_mul, he, pair.g)
        he.he_rotate(pair.g, a, steps[0], out)
        assert_same_residues(out, want_rot, he, pair.g)
        he.he_rotate_sum(pair.g, a, steps, out)
        assert_same_residues(out, want_sum, he, pair.g)
    he.he_set_tuning(pair.g, "ntt_shape", 0)
