// ks_fused_n12.cu -- the fused key-switching kernels instantiated for N = 2^12
// (the three tile shapes of ntt2.cu).
#include "ks_fused.cuh"

namespace he {

int ks_rot_n12(he_ctx* c, const KsRotArgs& a, uint32_t count, bool* handled, int* closed) {
  const int sh = c->ntt_shape;
  return sh == 1 ? ks_rot_run<12, 5, 6, 7, 4>(c, a, count, handled, closed)
       : sh == 2 ? ks_rot_run<12, 3, 8, 9, 2>(c, a, count, handled, closed) : ks_rot_run<12, 6, 5, 6, 5>(c, a, count, handled, closed);
}

size_t ks_rot_smem_n12(const he_ctx* c, uint32_t beta) {
  const int sh = c->ntt_shape;
  return sh == 1 ? ks_rot_smem<12, 7, 4>(beta) : sh == 2 ? ks_rot_smem<12, 9, 2>(beta) : ks_rot_smem<12, 6, 5>(beta);
}

int md_fused_n12(he_ctx* c, const MdArgs& a, uint32_t count, bool* handled) {
  const int sh = c->ntt_shape;
  return sh == 1 ? md_fused_run<12, 5, 6, 7, 4>(c, a, count, handled)
       : sh == 2 ? md_fused_run<12, 3, 8, 9, 2>(c, a, count, handled) : md_fused_run<12, 6, 5, 6, 5>(c, a, count, handled);
}

size_t md_col_smem_n12(const he_ctx* c, uint32_t nd) {
  const int sh = c->ntt_shape;
  return sh == 1 ? md_col_smem<12, 5, 6>(nd)
       : sh == 2 ? md_col_smem<12, 3, 8>(nd) : md_col_smem<12, 6, 5>(nd);
}

size_t ks_all_smem_n12(const he_ctx* c, uint32_t beta, const uint32_t* cnt) {
  const int sh = c->ntt_shape;
  return sh == 1 ? ks_all_smem<12, 5, 6>(c, beta, cnt)
       : sh == 2 ? ks_all_smem<12, 3, 8>(c, beta, cnt) : ks_all_smem<12, 6, 5>(c, beta, cnt);
}

}  // namespace he
