// ntt2.cu -- entry points of the two-pass NTT with compile-time tile shapes
// (kernels in ntt2_impl.cuh, instantiated per ring size in ntt2_n12.cu ..
// ntt2_n16.cu).  Three tile shapes per ring size (column pass bits, rows per
// tile | row pass bits, rows per tile); c->ntt_shape picks one (the
// autotuner times them).  The fused key-switching kernels use the same
// pairs.  (Radix-16 rounds, Shape's LOG_V = 4 with 128-thread CTAs, measured
// slower than these.)
#include "ntt2_impl.cuh"

namespace he {

int ntt2_inverse_rows(he_ctx* c, const PolyBatch& b) {
  switch (c->log_n) {
    case 12: return ntt2_inv_rows_n12(c, b);
    case 13: return ntt2_inv_rows_n13(c, b);
    case 14: return ntt2_inv_rows_n14(c, b);
    case 15: return ntt2_inv_rows_n15(c, b);
    case 16: return ntt2_inv_rows_n16(c, b);
    default: return fail(HE_EINVAL, "ntt2_inverse_rows: no compiled shape");
  }
}

int ntt2(he_ctx* c, const PolyBatch& b, bool inv, bool* handled) {
  *handled = true;
  switch (c->log_n) {
    case 12: return ntt2_n12(c, b, inv);
    case 13: return ntt2_n13(c, b, inv);
    case 14: return ntt2_n14(c, b, inv);
    case 15: return ntt2_n15(c, b, inv);
    case 16: return ntt2_n16(c, b, inv);
    default: *handled = false; return HE_OK;
  }
}

}  // namespace he
