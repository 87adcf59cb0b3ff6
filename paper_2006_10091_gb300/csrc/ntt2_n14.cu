// ntt2_n14.cu -- the compile-time-shaped NTT instantiated for N = 2^14.
#include "ntt2_impl.cuh"

namespace he {

int ntt2_n14(he_ctx* c, const PolyBatch& b, bool inv) {
  const int sh = c->ntt_shape;
  return sh == 1 ? run2_dir<14, 8, 3, 6, 5>(c, b, inv) : sh == 2 ? run2_dir<14, 5, 6, 9, 2>(c, b, inv) : run2_dir<14, 7, 4, 7, 4>(c, b, inv);
}

int ntt2_inv_rows_n14(he_ctx* c, const PolyBatch& b) {
  const int sh = c->ntt_shape;
  return sh == 1 ? run2_inv_rows<14, 8, 3, 6, 5>(c, b) : sh == 2 ? run2_inv_rows<14, 5, 6, 9, 2>(c, b)
                                                   : run2_inv_rows<14, 7, 4, 7, 4>(c, b);
}

}  // namespace he
