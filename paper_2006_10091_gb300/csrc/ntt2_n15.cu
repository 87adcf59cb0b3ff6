// ntt2_n15.cu -- the compile-time-shaped NTT instantiated for N = 2^15.
#include "ntt2_impl.cuh"

namespace he {

int ntt2_n15(he_ctx* c, const PolyBatch& b, bool inv) {
  const int sh = c->ntt_shape;
  return sh == 1 ? run2_dir<15, 7, 4, 8, 3>(c, b, inv) : sh == 2 ? run2_dir<15, 6, 5, 9, 2>(c, b, inv) : run2_dir<15, 8, 4, 7, 4>(c, b, inv);
}

int ntt2_inv_rows_n15(he_ctx* c, const PolyBatch& b) {
  const int sh = c->ntt_shape;
  return sh == 1 ? run2_inv_rows<15, 7, 4, 8, 3>(c, b) : sh == 2 ? run2_inv_rows<15, 6, 5, 9, 2>(c, b)
                                                   : run2_inv_rows<15, 8, 4, 7, 4>(c, b);
}

}  // namespace he
