// ntt2_n12.cu -- the compile-time-shaped NTT instantiated for N = 2^12.
#include "ntt2_impl.cuh"

namespace he {

int ntt2_n12(he_ctx* c, const PolyBatch& b, bool inv) {
  const int sh = c->ntt_shape;
  return sh == 1 ? run2_dir<12, 5, 6, 7, 4>(c, b, inv) : sh == 2 ? run2_dir<12, 3, 8, 9, 2>(c, b, inv) : run2_dir<12, 6, 5, 6, 5>(c, b, inv);
}

int ntt2_inv_rows_n12(he_ctx* c, const PolyBatch& b) {
  const int sh = c->ntt_shape;
  return sh == 1 ? run2_inv_rows<12, 5, 6, 7, 4>(c, b) : sh == 2 ? run2_inv_rows<12, 3, 8, 9, 2>(c, b)
                                                   : run2_inv_rows<12, 6, 5, 6, 5>(c, b);
}

}  // namespace he
