// Forward launcher of the shape-specialised second-order frequential kernel for
// N_fr = 512 frequential bins with log2 F = 4 on 8-column tiles (long signals:
// 191 first-order paths padded to 512); a translation unit of its own so it
// compiles beside the others.
#include "jtfs_freq_ct.cuh"

namespace jtfs {

bool launch_freq_fwd_ct_long(int mode, const FreqArgs& A, int lF, unsigned grid, size_t smem, cudaStream_t s,
                             const Tile* tiles, const float* S1, const float2* Y2, float* out) {
  if (mode != 2 || A.logNfr != 9 || A.logW != 3 || lF != 4) return false;
  opt_in_smem<k_freq_fwd_ct<2, 9, 3, 4>>();
  k_freq_fwd_ct<2, 9, 3, 4><<<grid, kThreads, smem, s>>>(A, tiles, S1, Y2, out);
  return true;
}

}  // namespace jtfs
