// Device helpers shared by the CUDA translation units of the JTFS library:
// complex arithmetic, register DFTs, and the argument block and
// shared-memory staging of the frequential kernels.  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "jtfs_internal.h"

namespace jtfs {

constexpr int kThreads = 256;
constexpr int kMaxSmem = 227 * 1024;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// ---------------------------------------------------------------------------
// Register DFTs of size 2, 4, 8, 16 (natural order in and out).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {  // * (-i) forward, * (+i) inverse
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// exp(-2 pi i m / 16) (forward) or its conjugate; m is a compile-time constant after unrolling.
template <bool INV>
__device__ __forceinline__ float2 w16(int m) {
  constexpr float C1 = 0.92387953251128674f, S1 = 0.38268343236508978f, H = 0.70710678118654752f;
  const float c[16] = {1.f, C1, H, S1, 0.f, -S1, -H, -C1, -1.f, -C1, -H, -S1, 0.f, S1, H, C1};
  const float sn[16] = {0.f, S1, H, C1, 1.f, C1, H, S1, 0.f, -S1, -H, -C1, -1.f, -C1, -H, -S1};
  return make_float2(c[m & 15], INV ? sn[m & 15] : -sn[m & 15]);
}
template <bool INV>
__device__ __forceinline__ void dft4(float2& v0, float2& v1, float2& v2, float2& v3) {
  const float2 s02 = cadd(v0, v2), d02 = csub(v0, v2), s13 = cadd(v1, v3), d13 = mul_mi<INV>(csub(v1, v3));
  v0 = cadd(s02, s13);
  v2 = csub(s02, s13);
  v1 = cadd(d02, d13);
  v3 = csub(d02, d13);
}
template <bool INV, int R>
__device__ __forceinline__ void dft_reg(float2* v) {
  if constexpr (R == 2) {
    const float2 t = v[0];
    v[0] = cadd(t, v[1]);
    v[1] = csub(t, v[1]);
  } else if constexpr (R == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    // n = 2 n1 + n2, k = k1 + 4 k2: DFT4 over n1, twiddle W8^(n2 k1), DFT2 over n2.
    dft4<INV>(v[0], v[2], v[4], v[6]);
    dft4<INV>(v[1], v[3], v[5], v[7]);
    float2 b[4] = {v[1], cmul(v[3], w16<INV>(2)), mul_mi<INV>(v[5]), cmul(v[7], w16<INV>(6))};
    float2 a[4] = {v[0], v[2], v[4], v[6]};
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      v[k1] = cadd(a[k1], b[k1]);
      v[k1 + 4] = csub(a[k1], b[k1]);
    }
  } else {  // R == 16: n = 4 n1 + n2, k = k1 + 4 k2
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
    // now Y[n2][k1] sits at v[4 k1 + n2]; twiddle by W16^(n2 k1)
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1)
#pragma unroll
      for (int n2 = 1; n2 < 4; ++n2) v[4 * k1 + n2] = cmul(v[4 * k1 + n2], w16<INV>(n2 * k1));
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    // X[k1 + 4 k2] sits at v[4 k1 + k2]: transpose the 4 x 4 register block
    float2 t[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[4 * k1 + k2];
  }
}

// ---------------------------------------------------------------------------
// Frequential scattering (§3.4) fused with modulus and phi_F averaging:
// argument block and shared-memory staging common to all its kernels.
// ---------------------------------------------------------------------------
struct FreqArgs {
  int N1, N_fr, logNfr, R_out, logRout, n_frames, logN, W, logW, n_beta1, n_beta2, n_ftab;
  int64_t phi_size, phi1_off, y2_tot, v2_tot;
  const FiltD* beta;
  FiltD phiF;
  const float* ftab;
  const FreqChunk* chunks;
  int n_chunks;
  const int* s2;
  const int* n1max_act;
  const int64_t* y2_off;
  const int64_t* v2_off;
  const float2* tw;
  int twlog;
  // compact tables (see Plan::h_ftabc); tab_smem = 1 stages them in shared memory
  const float* ftabc;
  const int* ftabc_off;
  int n_ftabc, ftabc_phi, tab_smem;
  int ftabc_lev[16];
  // Unpooled along n1 (no phi_F): each path's |Y_fr| rows start at row_off[beta].
  int unpooled_f;
  const int* row_off;
};

// Shared-memory layout of the frequential kernels (all in float2 units):
//   tw    [N_fr]                twiddles exp(-2 pi i e / N_fr)
//   bufs  nbuf x [W * N_fr]     interleaved transforms
//   band  [n_beta2] int2        (lo, hi) of each frequential filter
//   chk   [n_chunks] FreqChunk
//   toff  [n_beta2] int         offset of each filter's band in the compact table
//   tc    [n_ftabc] float       compact table (16-byte aligned), when A.tab_smem
struct FreqSmem {
  float2* tw;
  float2* buf;
  const float* tab;  // global (read through L1): [n_ftab][N_fr]
  int2* band;
  FreqChunk* chk;
  int* toff;
  const float* tc;   // compact table: shared memory if A.tab_smem, else global
};

__device__ __forceinline__ FreqSmem freq_smem_carve(const FreqArgs& A, float2* sm, int nbuf) {
  FreqSmem S;
  const int WN = A.W * A.N_fr;
  S.tw = sm;
  S.buf = sm + A.N_fr;
  S.tab = A.ftab;
  S.band = reinterpret_cast<int2*>(S.buf + nbuf * WN);
  S.chk = reinterpret_cast<FreqChunk*>(S.band + A.n_beta2);
  S.toff = reinterpret_cast<int*>(S.chk + A.n_chunks);
  float* tcs = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(S.toff + A.n_beta2) + 15) & ~uintptr_t(15));
  S.tc = A.tab_smem ? tcs : A.ftabc;
  return S;
}

__device__ __forceinline__ void freq_stage_tables(const FreqArgs& A, const FreqSmem& S) {
  const int sh = A.twlog - A.logNfr;
  for (int i = threadIdx.x; i < A.N_fr; i += blockDim.x) S.tw[i] = __ldg(A.tw + (i << sh));
  for (int i = threadIdx.x; i < A.n_beta2; i += blockDim.x) S.band[i] = make_int2(A.beta[i].lo, A.beta[i].hi);
  const int* csrc = reinterpret_cast<const int*>(A.chunks);
  int* cdst = reinterpret_cast<int*>(S.chk);
  for (int i = threadIdx.x; i < A.n_chunks * static_cast<int>(sizeof(FreqChunk) / sizeof(int)); i += blockDim.x)
    cdst[i] = csrc[i];
  for (int i = threadIdx.x; i < A.n_beta2; i += blockDim.x) S.toff[i] = __ldg(A.ftabc_off + i);
  if (A.tab_smem) {
    float* tcs = const_cast<float*>(S.tc);
    for (int i = threadIdx.x; i < A.n_ftabc; i += blockDim.x) tcs[i] = __ldg(A.ftabc + i);
  }
}

// Columns of the tile into interleaved layout dst[r * W + w], zero-padded to N_fr rows.
template <int MODE>
__device__ __forceinline__ void freq_load_columns(const FreqArgs& A, const Tile& tl, const float* S1,
                                                  const float2* Y2, float2* dst, int& stride, int& n1m) {
  const float2* ysrc = nullptr;
  const float* ssrc = nullptr;
  if (MODE == 1) {
    n1m = A.N1;
    stride = A.n_frames;
    ssrc = S1 + static_cast<int64_t>(tl.b) * A.N1 * A.n_frames + tl.t0;
  } else {
    n1m = A.n1max_act[tl.a];
    stride = 1 << (A.logN - A.s2[tl.a]);
    ysrc = Y2 + static_cast<int64_t>(tl.b) * A.y2_tot + A.y2_off[tl.a] + tl.t0;
  }
  for (int i = threadIdx.x; i < A.W * A.N_fr; i += blockDim.x) {
    const int w = i & (A.W - 1), r = i >> A.logW;
    float2 v = make_float2(0.f, 0.f);
    if (r < n1m && w < tl.ncols) {
      if (MODE == 1) v = make_float2(ssrc[static_cast<int64_t>(r) * stride + w], 0.f);
      else v = ysrc[static_cast<int64_t>(r) * stride + w];
    }
    dst[i] = v;
  }
}

__host__ __device__ __forceinline__ int ceil_log2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}


// Shape-specialised frequential kernels (jtfs_freq_ct_fwd.cu, jtfs_freq_ct_adj.cu;
// the N_fr = 512 shapes in jtfs_freq_ct_long_*.cu).  Each returns false,
// launching nothing, when no specialisation matches the plan's (N_fr, columns
// per tile, log2 F).
bool launch_freq_fwd_ct(int mode, const FreqArgs& A, int lF, unsigned grid, size_t smem, cudaStream_t s,
                        const Tile* tiles, const float* S1, const float2* Y2, float* out);
bool launch_freq_adj_ct(int mode, const FreqArgs& A, int lF, unsigned grid, size_t smem, cudaStream_t s,
                        const Tile* tiles, const float* S1, const float2* Y2, const float* dout, float* dS1,
                        float2* dY2);
bool launch_freq_fwd_ct_long(int mode, const FreqArgs& A, int lF, unsigned grid, size_t smem, cudaStream_t s,
                             const Tile* tiles, const float* S1, const float2* Y2, float* out);
bool launch_freq_adj_ct_long(int mode, const FreqArgs& A, int lF, unsigned grid, size_t smem, cudaStream_t s,
                             const Tile* tiles, const float* S1, const float2* Y2, const float* dout, float* dS1,
                             float2* dY2);

}  // namespace jtfs
