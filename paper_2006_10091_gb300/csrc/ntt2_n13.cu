// ntt2_n13.cu -- the compile-time-shaped NTT instantiated for N = 2^13.
#include "ntt2_impl.cuh"

namespace he {

int ntt2_n13(he_ctx* c, const PolyBatch& b, bool inv) {
  const int sh = c->ntt_shape;
  return sh == 1 ? run2_dir<13, 6, 5, 7, 4>(c, b, inv) : sh == 2 ? run2_dir<13, 4, 7, 9, 2>(c, b, inv) : run2_dir<13, 7, 4, 6, 5>(c, b, inv);
}

int ntt2_inv_rows_n13(he_ctx* c, const PolyBatch& b) {
  const int sh = c->ntt_shape;
  return sh == 1 ? run2_inv_rows<13, 6, 5, 7, 4>(c, b) : sh == 2 ? run2_inv_rows<13, 4, 7, 9, 2>(c, b)
                                                   : run2_inv_rows<13, 7, 4, 6, 5>(c, b);
}

}  // namespace he
