// Adjoint launcher of the shape-specialised second-order frequential kernel for
// N_fr = 512 frequential bins with log2 F = 4 on 4-column tiles (long signals);
// a translation unit of its own so it compiles beside the others.
#include "jtfs_freq_ct.cuh"

namespace jtfs {

bool launch_freq_adj_ct_long(int mode, const FreqArgs& A, int lF, unsigned grid, size_t smem, cudaStream_t s,
                             const Tile* tiles, const float* S1, const float2* Y2, const float* dout, float* dS1,
                             float2* dY2) {
  if (mode != 2 || A.logNfr != 9 || A.logW != 2 || lF != 4) return false;
  opt_in_smem<k_freq_adj_ct<2, 9, 2, 4>>();
  k_freq_adj_ct<2, 9, 2, 4><<<grid, kThreads, smem, s>>>(A, tiles, S1, Y2, dout, dS1, dY2);
  return true;
}

}  // namespace jtfs
