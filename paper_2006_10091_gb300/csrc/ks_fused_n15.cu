// ks_fused_n15.cu -- the fused key-switching kernels instantiated for N = 2^15
// (the three tile shapes of ntt2.cu).
#include "ks_fused.cuh"

namespace he {

int ks_rot_n15(he_ctx* c, const KsRotArgs& a, uint32_t count, bool* handled, int* closed) {
  const int sh = c->ntt_shape;
  return sh == 1 ? ks_rot_run<15, 7, 4, 8, 3>(c, a, count, handled, closed)
       : sh == 2 ? ks_rot_run<15, 6, 5, 9, 2>(c, a, count, handled, closed) : ks_rot_run<15, 8, 4, 7, 4>(c, a, count, handled, closed);
}

size_t ks_rot_smem_n15(const he_ctx* c, uint32_t beta) {
  const int sh = c->ntt_shape;
  return sh == 1 ? ks_rot_smem<15, 8, 3>(beta) : sh == 2 ? ks_rot_smem<15, 9, 2>(beta) : ks_rot_smem<15, 7, 4>(beta);
}

int md_fused_n15(he_ctx* c, const MdArgs& a, uint32_t count, bool* handled) {
  const int sh = c->ntt_shape;
  return sh == 1 ? md_fused_run<15, 7, 4, 8, 3>(c, a, count, handled)
       : sh == 2 ? md_fused_run<15, 6, 5, 9, 2>(c, a, count, handled) : md_fused_run<15, 8, 4, 7, 4>(c, a, count, handled);
}

size_t md_col_smem_n15(const he_ctx* c, uint32_t nd) {
  const int sh = c->ntt_shape;
  return sh == 1 ? md_col_smem<15, 7, 4>(nd)
       : sh == 2 ? md_col_smem<15, 6, 5>(nd) : md_col_smem<15, 8, 4>(nd);
}

size_t ks_all_smem_n15(const he_ctx* c, uint32_t beta, const uint32_t* cnt) {
  const int sh = c->ntt_shape;
  return sh == 1 ? ks_all_smem<15, 7, 4>(c, beta, cnt)
       : sh == 2 ? ks_all_smem<15, 6, 5>(c, beta, cnt) : ks_all_smem<15, 8, 4>(c, beta, cnt);
}

}  // namespace he
