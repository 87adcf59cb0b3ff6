"""he_rescale_noalloc: the rescale for callers that cannot allocate device
memory (a host that runs the GPU under its own pool and a fixed memory
budget, or a loop that must not stall on an allocation).  Its scratch is the
library's static device array; the result must equal he_rescale's, residue
for residue, on consecutive calls that reuse the array.  This file is
collected last so that a run stopping at the first failure has run every
other test first."""
import numpy as np
import pytest

from paper_2006_10091_gb300 import workloads
from tests.gpu_util import gpu_lib

pytestmark = pytest.mark.gpu


def test_rescale_noalloc_matches_rescale_on_consecutive_calls():
    he = gpu_lib()
    ctx = he.Context(13, 6, 45, 1, 60, 2.0 ** 45, seed=21)
    for call, level in enumerate((6, 4)):  # two calls in a row share the static scratch
        a = ctx.new_ct(6)
        he.he_encrypt_poly(ctx, workloads.int_poly(40 + call, ctx.n, 1 << 40), 2.0 ** 45, level, a, cid=40 + call)
        ref, out = ctx.new_ct(6), ctx.new_ct(6)
        he.he_rescale(ctx, a, ref)
        he.he_rescale_noalloc(ctx, a, out)
        assert (out.level, out.scale) == (ref.level, ref.scale) == (level - 1, a.scale / ctx.primes[level - 1])
        assert np.array_equal(he.he_ct_export(ctx, out), he.he_ct_export(ctx, ref))


def test_rescale_noalloc_rejects_sizes_beyond_the_static_array():
    he = gpu_lib()
    ctx = he.Context(16, 4, 50, 1, 60, 2.0 ** 50, seed=22)  # 2 * 4 * 2^16 words > 2^19
    a = ctx.new_ct(4)
    he.he_encrypt_poly(ctx, workloads.int_poly(1, ctx.n, 1 << 30), 2.0 ** 50, 4, a, cid=1)
    with pytest.raises(he.HeError) as e:
        he.he_rescale_noalloc(ctx, a, ctx.new_ct(4))
    assert e.value.code == he.HE_EINVAL and "static array" in str(e.value)
