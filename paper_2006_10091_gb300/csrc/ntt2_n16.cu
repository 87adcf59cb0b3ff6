// ntt2_n16.cu -- the compile-time-shaped NTT instantiated for N = 2^16.
#include "ntt2_impl.cuh"

namespace he {

int ntt2_n16(he_ctx* c, const PolyBatch& b, bool inv) {
  const int sh = c->ntt_shape;
  return sh == 1 ? run2_dir<16, 7, 4, 9, 2>(c, b, inv) : sh == 2 ? run2_dir<16, 6, 5, 10, 1>(c, b, inv) : run2_dir<16, 8, 4, 8, 3>(c, b, inv);
}

int ntt2_inv_rows_n16(he_ctx* c, const PolyBatch& b) {
  const int sh = c->ntt_shape;
  return sh == 1 ? run2_inv_rows<16, 7, 4, 9, 2>(c, b) : sh == 2 ? run2_inv_rows<16, 6, 5, 10, 1>(c, b)
                                                   : run2_inv_rows<16, 8, 4, 8, 3>(c, b);
}

}  // namespace he
