// ks_fused_n16.cu -- the fused key-switching kernels instantiated for N = 2^16
// (the three tile shapes of ntt2.cu).
#include "ks_fused.cuh"

namespace he {

int ks_rot_n16(he_ctx* c, const KsRotArgs& a, uint32_t count, bool* handled, int* closed) {
  const int sh = c->ntt_shape;
  return sh == 1 ? ks_rot_run<16, 7, 4, 9, 2>(c, a, count, handled, closed)
       : sh == 2 ? ks_rot_run<16, 6, 5, 10, 1>(c, a, count, handled, closed) : ks_rot_run<16, 8, 4, 8, 3>(c, a, count, handled, closed);
}

size_t ks_rot_smem_n16(const he_ctx* c, uint32_t beta) {
  const int sh = c->ntt_shape;
  return sh == 1 ? ks_rot_smem<16, 9, 2>(beta) : sh == 2 ? ks_rot_smem<16, 10, 1>(beta) : ks_rot_smem<16, 8, 3>(beta);
}

int md_fused_n16(he_ctx* c, const MdArgs& a, uint32_t count, bool* handled) {
  const int sh = c->ntt_shape;
  return sh == 1 ? md_fused_run<16, 7, 4, 9, 2>(c, a, count, handled)
       : sh == 2 ? md_fused_run<16, 6, 5, 10, 1>(c, a, count, handled) : md_fused_run<16, 8, 4, 8, 3>(c, a, count, handled);
}

size_t md_col_smem_n16(const he_ctx* c, uint32_t nd) {
  const int sh = c->ntt_shape;
  return sh == 1 ? md_col_smem<16, 7, 4>(nd)
       : sh == 2 ? md_col_smem<16, 6, 5>(nd) : md_col_smem<16, 8, 4>(nd);
}

size_t ks_all_smem_n16(const he_ctx* c, uint32_t beta, const uint32_t* cnt) {
  const int sh = c->ntt_shape;
  return sh == 1 ? ks_all_smem<16, 7, 4>(c, beta, cnt)
       : sh == 2 ? ks_all_smem<16, 6, 5>(c, beta, cnt) : ks_all_smem<16, 8, 4>(c, beta, cnt);
}

}  // namespace he
