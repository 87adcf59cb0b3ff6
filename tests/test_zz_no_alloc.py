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


def test_rescale_noalloc_never_asks_the_workspace():
    """On a fresh context (no rescale run yet) the entry point neither grows
    the context's workspace nor asks it for scratch at all (a fallback to the
    workspace would count a request), and its result equals he_rescale's,
    which does ask."""
    he = gpu_lib()
    ctx = he.Context(13, 6, 45, 1, 60, 2.0 ** 45, seed=23)
    host = workloads.residues(5, ctx.primes[:6], ctx.n, parts=2)
    a = ctx.new_ct(6)
    he.he_ct_import(ctx, host, 6, 2.0 ** 45, a)
    before = he.he_ctx_workspace(ctx)
    out = ctx.new_ct(6)
    he.he_rescale_noalloc(ctx, a, out)
    he.he_sync(ctx)
    assert he.he_ctx_workspace(ctx) == before
    ref = ctx.new_ct(6)
    he.he_rescale(ctx, a, ref)
    assert he.he_ctx_workspace(ctx)["requests"] == before["requests"] + 1
    assert np.array_equal(he.he_ct_export(ctx, out), he.he_ct_export(ctx, ref))


def test_rescale_noalloc_at_the_size_limit():
    """N = 2^14: level 15 needs 2*15*N + 64 words, within the 2^19 of the
    array, and matches he_rescale; level 16 needs 2^19 + 64 and is refused."""
    he = gpu_lib()
    ctx = he.Context(14, 16, 40, 1, 60, 2.0 ** 40, seed=24)
    for level, ok in ((15, True), (16, False)):
        host = workloads.residues(60 + level, ctx.primes[:level], ctx.n, parts=2)
        a = ctx.new_ct(level)
        he.he_ct_import(ctx, host, level, 2.0 ** 40, a)
        out = ctx.new_ct(level)
        if not ok:
            with pytest.raises(he.HeError) as e:
                he.he_rescale_noalloc(ctx, a, out)
            assert e.value.code == he.HE_EINVAL
            continue
        he.he_rescale_noalloc(ctx, a, out)
        ref = ctx.new_ct(level)
        he.he_rescale(ctx, a, ref)
        assert np.array_equal(he.he_ct_export(ctx, out), he.he_ct_export(ctx, ref))


def test_rescale_noalloc_rejects_sizes_beyond_the_static_array():
    he = gpu_lib()
    ctx = he.Context(16, 4, 50, 1, 60, 2.0 ** 50, seed=22)  # 2 * 4 * 2^16 words > 2^19
    a = ctx.new_ct(4)
    he.he_encrypt_poly(ctx, workloads.int_poly(1, ctx.n, 1 << 30), 2.0 ** 50, 4, a, cid=1)
    with pytest.raises(he.HeError) as e:
        he.he_rescale_noalloc(ctx, a, ctx.new_ct(4))
    assert e.value.code == he.HE_EINVAL and "static array" in str(e.value)
