// Adjoint launcher of the shape-specialised second-order frequential kernels (templates
// in jtfs_freq_ct.cuh); a separate translation unit so the two compile in
// parallel.
#include "jtfs_freq_ct.cuh"

namespace jtfs {

bool launch_freq_adj_ct(int mode, const FreqArgs& A, int lF, unsigned grid, size_t smem, cudaStream_t s,
                        const Tile* tiles, const float* S1, const float2* Y2, const float* dout, float* dS1,
                        float2* dY2) {
#define JTFS_CT_ADJ(LN, LW, LFv)                                                                     \
  if (A.logNfr == LN && A.logW == LW && lF == LFv) {                                                 \
    if (mode != 2) return false;                                                                     \
    opt_in_smem<k_freq_adj_ct<2, LN, LW, LFv>>();                                                    \
    k_freq_adj_ct<2, LN, LW, LFv><<<grid, kThreads, smem, s>>>(A, tiles, S1, Y2, dout, dS1, dY2);     \
    return true;                                                                                     \
  }
  JTFS_CT_ADJ(8, 3, 3)
  JTFS_CT_ADJ(6, 4, 2)
#undef JTFS_CT_ADJ
  return launch_freq_adj_ct_long(mode, A, lF, grid, smem, s, tiles, S1, Y2, dout, dS1, dY2);
}

}  // namespace jtfs
