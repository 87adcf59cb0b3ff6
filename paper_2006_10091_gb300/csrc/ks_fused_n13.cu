// ks_fused_n13.cu -- the fused key-switching kernels instantiated for N = 2^13
// (the three tile shapes of ntt2.cu).
#include "ks_fused.cuh"

namespace he {

int ks_rot_n13(he_ctx* c, const KsRotArgs& a, uint32_t count, bool* handled, int* closed) {
  const int sh = c->ntt_shape;
  return sh == 1 ? ks_rot_run<13, 6, 5, 7, 4>(c, a, count, handled, closed)
       : sh == 2 ? ks_rot_run<13, 4, 7, 9, 2>(c, a, count, handled, closed) : ks_rot_run<13, 7, 4, 6, 5>(c, a, count, handled, closed);
}

size_t ks_rot_smem_n13(const he_ctx* c, uint32_t beta) {
  const int sh = c->ntt_shape;
  return sh == 1 ? ks_rot_smem<13, 7, 4>(beta) : sh == 2 ? ks_rot_smem<13, 9, 2>(beta) : ks_rot_smem<13, 6, 5>(beta);
}

int md_fused_n13(he_ctx* c, const MdArgs& a, uint32_t count, bool* handled) {
  const int sh = c->ntt_shape;
  return sh == 1 ? md_fused_run<13, 6, 5, 7, 4>(c, a, count, handled)
       : sh == 2 ? md_fused_run<13, 4, 7, 9, 2>(c, a, count, handled) : md_fused_run<13, 7, 4, 6, 5>(c, a, count, handled);
}

size_t md_col_smem_n13(const he_ctx* c, uint32_t nd) {
  const int sh = c->ntt_shape;
  return sh == 1 ? md_col_smem<13, 6, 5>(nd)
       : sh == 2 ? md_col_smem<13, 4, 7>(nd) : md_col_smem<13, 7, 4>(nd);
}

size_t ks_all_smem_n13(const he_ctx* c, uint32_t beta, const uint32_t* cnt) {
  const int sh = c->ntt_shape;
  return sh == 1 ? ks_all_smem<13, 6, 5>(c, beta, cnt)
       : sh == 2 ? ks_all_smem<13, 4, 7>(c, beta, cnt) : ks_all_smem<13, 7, 4>(c, beta, cnt);
}

}  // namespace he
