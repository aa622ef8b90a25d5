// Forward launcher of the shape-specialised second-order frequential kernels (templates
// in jtfs_freq_ct.cuh); a separate translation unit so the two compile in
// parallel.
#include "jtfs_freq_ct.cuh"

namespace jtfs {

bool launch_freq_fwd_ct(int mode, const FreqArgs& A, int lF, unsigned grid, size_t smem, cudaStream_t s,
                        const Tile* tiles, const float* S1, const float2* Y2, float* out) {
#define JTFS_CT_FWD(LN, LW, LFv)                                                               \
  if (A.logNfr == LN && A.logW == LW && lF == LFv) {                                           \
    if (mode != 2) return false;                                                               \
    opt_in_smem<k_freq_fwd_ct<2, LN, LW, LFv>>();                                              \
    k_freq_fwd_ct<2, LN, LW, LFv><<<grid, kThreads, smem, s>>>(A, tiles, S1, Y2, out);          \
    return true;                                                                               \
  }
  JTFS_CT_FWD(8, 4, 3)
  JTFS_CT_FWD(8, 3, 3)
  JTFS_CT_FWD(6, 4, 2)
#undef JTFS_CT_FWD
  return launch_freq_fwd_ct_long(mode, A, lF, grid, smem, s, tiles, S1, Y2, out);
}

}  // namespace jtfs
