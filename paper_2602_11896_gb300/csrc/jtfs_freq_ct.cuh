// Shape-specialised frequential scattering kernels (§3.4 with the modulus and
// phi_F averaging of Eq. (5)), forward and adjoint.
//
// Same computation as the generic kernels of jtfs_cuda.cu, but the
// frequential length N_fr, the columns per tile W and the averaging level
// log2 F are template parameters, and each chunk of frequential filters is
// dispatched to a body whose transform size R and interleave count are
// compile-time constants.  Every shift, mask, loop bound and stride is then a
// constant, so a radix pass is loads at immediate offsets, FP arithmetic and
// stores; the generic kernels spend most of their instructions on runtime
// index arithmetic.  Data layout, interleaving and pairing are described in
// jtfs_device.cuh / jtfs_cuda.cu.
#pragma once

#include <cuda_runtime.h>

#include "jtfs_device.cuh"

namespace jtfs {
namespace {

__host__ __device__ constexpr int radix_log(int rem) {
  return (rem == 3 || rem == 5 || rem == 6 || rem == 9) ? 3 : (rem >= 4 ? 4 : rem);
}

// One radix pass over 2^LCNT interleaved transforms of size 2^LOGN; twiddle
// table of 2^LOGTW entries.  When the pass has at least one pair of adjacent
// transforms per thread, each thread takes two (16-byte accesses, shared
// index arithmetic and twiddles); otherwise one, to keep more threads busy.
template <bool INV, int LOGN, int LCNT, int LNS, int LOGTW>
__device__ __forceinline__ void ct_pass(const float2* __restrict__ src, float2* __restrict__ dst,
                                        const float2* __restrict__ tw) {
  constexpr int LR = radix_log(LOGN - LNS);
  constexpr int R = 1 << LR;
  constexpr int LQ = LOGN - LR;
  constexpr int NS = 1 << LNS;
  constexpr int SHIFT = LOGTW - (LNS + LR);
  constexpr bool PAIR = (1 << (LQ + LCNT - 1)) >= kThreads;
  if constexpr (PAIR) {
    constexpr int LP = LCNT - 1;
    constexpr int TOTAL = 1 << (LQ + LP);
    constexpr int SSTRIDE = 1 << (LQ + LP);
    constexpr int DSTRIDE = NS << LP;
    constexpr int ITERS = (TOTAL + kThreads - 1) / kThreads;
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll 1
    for (int it = 0; it < ITERS; ++it) {
      const int idx = static_cast<int>(threadIdx.x) + it * kThreads;
      if ((TOTAL % kThreads) != 0 && idx >= TOTAL) break;
      const int fp = idx & ((1 << LP) - 1), j = idx >> LP;
      const int k = j & (NS - 1);
      float2 va[R], vb[R];
      const float4* sp = s4 + ((j << LP) + fp);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float4 t = sp[r * SSTRIDE];
        va[r] = make_float2(t.x, t.y);
        vb[r] = make_float2(t.z, t.w);
      }
      if constexpr (LNS > 0) {
        const int e = k << SHIFT;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[r * e];
          if (INV) w.y = -w.y;
          va[r] = cmul(va[r], w);
          vb[r] = cmul(vb[r], w);
        }
      }
      dft_reg<INV, R>(va);
      dft_reg<INV, R>(vb);
      float4* dp = d4 + (((((j - k) << LR) + k) << LP) + fp);
#pragma unroll
      for (int q = 0; q < R; ++q) dp[q * DSTRIDE] = make_float4(va[q].x, va[q].y, vb[q].x, vb[q].y);
    }
  } else {
    constexpr int TOTAL = 1 << (LQ + LCNT);
    constexpr int SSTRIDE = 1 << (LQ + LCNT);
    constexpr int DSTRIDE = NS << LCNT;
    constexpr int ITERS = (TOTAL + kThreads - 1) / kThreads;
#pragma unroll 1
    for (int it = 0; it < ITERS; ++it) {
      const int idx = static_cast<int>(threadIdx.x) + it * kThreads;
      if ((TOTAL % kThreads) != 0 && idx >= TOTAL) break;
      const int f = idx & ((1 << LCNT) - 1), j = idx >> LCNT;
      const int k = j & (NS - 1);
      float2 v[R];
      const float2* sp = src + ((j << LCNT) + f);
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = sp[r * SSTRIDE];
      if constexpr (LNS > 0) {
        const int e = k << SHIFT;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[r * e];
          if (INV) w.y = -w.y;
          v[r] = cmul(v[r], w);
        }
      }
      dft_reg<INV, R>(v);
      float2* dp = dst + (((((j - k) << LR) + k) << LCNT) + f);
#pragma unroll
      for (int q = 0; q < R; ++q) dp[q * DSTRIDE] = v[q];
    }
  }
}

template <bool INV, int LOGN, int LCNT, int LNS, int LOGTW>
struct CtFft {
  static __device__ __forceinline__ float2* run(float2* a, float2* b, const float2* tw) {
    if constexpr (LNS >= LOGN) {
      return a;
    } else {
      ct_pass<INV, LOGN, LCNT, LNS, LOGTW>(a, b, tw);
      __syncthreads();
      return CtFft<INV, LOGN, LCNT, LNS + radix_log(LOGN - LNS), LOGTW>::run(b, a, tw);
    }
  }
};

// Columns of the tile into interleaved layout [r][w], zero-padded to N_fr rows.
template <int MODE, int LOGNFR, int LOGW>
__device__ __forceinline__ void ct_load_columns(const FreqArgs& A, const Tile& tl, const float* S1, const float2* Y2,
                                                float2* dst, int& stride, int& n1m) {
  constexpr int W = 1 << LOGW, NFR = 1 << LOGNFR;
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
#pragma unroll 1
  for (int i = threadIdx.x; i < W * NFR; i += kThreads) {
    const int w = i & (W - 1), r = i >> LOGW;
    float2 v = make_float2(0.f, 0.f);
    if (r < n1m && w < tl.ncols) {
      if (MODE == 1) v = make_float2(ssrc[static_cast<int64_t>(r) * stride + w], 0.f);
      else v = ysrc[static_cast<int64_t>(r) * stride + w];
    }
    dst[i] = v;
  }
}

// Fold of the chunk's filter products onto R = N_fr / 2^K bins (see freq_fold).
template <int LOGNFR, int LOGW, int K, int LC>
__device__ __forceinline__ void ct_fold(const FreqSmem& S, const FreqChunk& ch, const float2* yh, float2* out) {
  constexpr int NFR = 1 << LOGNFR, LR = LOGNFR - K, R = 1 << LR, LP = LC - 1, LWP = LOGW - 1;
  constexpr float INV = 1.f / NFR;
  const float4* y4 = reinterpret_cast<const float4*>(yh);
  float4* o4 = reinterpret_cast<float4*>(out);
#pragma unroll 2
  for (int i = threadIdx.x; i < (R << LP); i += kThreads) {
    const int fp = i & ((1 << LP) - 1), m = i >> LP;
    const int bc = fp >> LWP, wp = fp & ((1 << LWP) - 1);
    const int b = bc < ch.n ? ch.beta[bc] : -1;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (b >= 0) {
      const int2 bd = S.band[b];
      const float* t = S.tc + S.toff[b] - bd.x;  // t[sb] = filter at signed bin sb of its band
      const float4* yc = y4 + wp;
      for (int sb = bd.x + ((m - bd.x) & (R - 1)); sb <= bd.y; sb += R) {
        const int q = sb & (NFR - 1);
        const float g = t[sb];
        const float4 y = yc[q << LWP];
        acc.x += g * y.x;
        acc.y += g * y.y;
        acc.z += g * y.z;
        acc.w += g * y.w;
      }
    }
    o4[i] = make_float4(acc.x * INV, acc.y * INV, acc.z * INV, acc.w * INV);
  }
}

// phi_F averaging fold onto R_out bins (see freq_pool_fold).
template <int LOGNFR, int LF, int K, int LC>
__device__ __forceinline__ void ct_pool_fold(const FreqArgs& A, const FreqSmem& S, const float2* uh, float2* out) {
  constexpr int NFR = 1 << LOGNFR, LR = LOGNFR - K, R = 1 << LR, LRO = LOGNFR - LF, RO = 1 << LRO, LP = LC - 1;
  constexpr float INV = 1.f / R;
  const float* t = S.tc + A.ftabc_phi - A.phiF.lo;  // t[sb] = phi_F at signed bin sb of its band
  const float4* u4 = reinterpret_cast<const float4*>(uh);
  float4* o4 = reinterpret_cast<float4*>(out);
#pragma unroll 2
  for (int i = threadIdx.x; i < (RO << LP); i += kThreads) {
    const int fp = i & ((1 << LP) - 1), m = i >> LP;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int sb = A.phiF.lo + ((m - A.phiF.lo) & (RO - 1)); sb <= A.phiF.hi; sb += RO) {
      const float g = t[sb];
      const float4 v = u4[((sb & (R - 1)) << LP) + fp];
      acc.x += g * v.x;
      acc.y += g * v.y;
      acc.z += g * v.z;
      acc.w += g * v.w;
    }
    o4[i] = make_float4(acc.x * INV, acc.y * INV, acc.z * INV, acc.w * INV);
  }
}

// ---------------------------------------------------------------------------
// Forward chunk: fold, inverse FFT, modulus, FFT, phi_F fold, inverse FFT, store.
// ---------------------------------------------------------------------------
template <int MODE, int LOGNFR, int LOGW, int LF, int K, int LCADD>
__device__ __forceinline__ void fwd_chunk(const FreqArgs& A, const FreqSmem& S, const FreqChunk& ch, const Tile& tl,
                                          int stride, const float2* yh, float2* f1, float2* f2, float* out) {
  constexpr int W = 1 << LOGW, LR = LOGNFR - K, LC = LOGW + LCADD, LRO = LOGNFR - LF, RO = 1 << LRO;
  constexpr int CNT = 1 << LC;
  ct_fold<LOGNFR, LOGW, K, LC>(S, ch, yh, f1);
  __syncthreads();
  float2* z = CtFft<true, LR, LC, 0, LOGNFR>::run(f1, f2, S.tw);
  {
    float4* z4 = reinterpret_cast<float4*>(z);
#pragma unroll 4
    for (int i = threadIdx.x; i < (1 << (LR + LC - 1)); i += kThreads) {
      const float4 v = z4[i];
      z4[i] = make_float4(sqrtf(v.x * v.x + v.y * v.y), 0.f, sqrtf(v.z * v.z + v.w * v.w), 0.f);
    }
  }
  __syncthreads();
  float2* zo = (z == f1) ? f2 : f1;
  float2* uh = CtFft<false, LR, LC, 0, LOGNFR>::run(z, zo, S.tw);
  float2* g = (uh == f1) ? f2 : f1;
  ct_pool_fold<LOGNFR, LF, K, LC>(A, S, uh, g);
  __syncthreads();
  float2* pr = CtFft<true, LRO, LC, 0, LOGNFR>::run(g, uh, S.tw);
#pragma unroll 4
  for (int i = threadIdx.x; i < (RO << LC); i += kThreads) {
    const int f = i & (CNT - 1), row = i >> LC;
    const int bc = f >> LOGW, w = f & (W - 1);
    if (bc < ch.n && w < tl.ncols) {
      const int b = ch.beta[bc];
      const float v = pr[i].x;
      if (MODE == 1)
        out[static_cast<int64_t>(tl.b) * A.phi_size + A.phi1_off + (static_cast<int64_t>(b) * RO + row) * A.n_frames +
            tl.t0 + w] = v;
      else
        out[static_cast<int64_t>(tl.b) * A.v2_tot + A.v2_off[tl.a] + (static_cast<int64_t>(b) * RO + row) * stride +
            tl.t0 + w] = v;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Adjoint chunk (see k_freq_adj): recompute z, then F(dw), unfold with the
// phi_F level, inverse FFT, modulus adjoint, FFT, scatter into D.
// ---------------------------------------------------------------------------
template <int MODE, int LOGNFR, int LOGW, int LF, int K, int LCADD>
__device__ __forceinline__ void adj_chunk(const FreqArgs& A, const FreqSmem& S, const FreqChunk& ch, const Tile& tl,
                                          int stride, const float2* yh, float2* D, float2* zb, float2* f1, float2* f2,
                                          const float* dout) {
  constexpr int NFR = 1 << LOGNFR, W = 1 << LOGW, LR = LOGNFR - K, R = 1 << LR, LC = LOGW + LCADD;
  constexpr int LRO = LOGNFR - LF, RO = 1 << LRO, CNT = 1 << LC, LP = LC - 1, LWP = LOGW - 1;
  constexpr float INVR = 1.f / R, INVNFR = 1.f / NFR;
  ct_fold<LOGNFR, LOGW, K, LC>(S, ch, yh, f1);
  __syncthreads();
  float2* z = CtFft<true, LR, LC, 0, LOGNFR>::run(f1, f2, S.tw);
  float2* dwb = (z == f1) ? f2 : f1;
  {
    const float4* z4 = reinterpret_cast<const float4*>(z);
    float4* zb4 = reinterpret_cast<float4*>(zb);
#pragma unroll 4
    for (int i = threadIdx.x; i < (R << LP); i += kThreads) zb4[i] = z4[i];
  }
#pragma unroll 4
  for (int i = threadIdx.x; i < (RO << LC); i += kThreads) {
    const int f = i & (CNT - 1), row = i >> LC;
    const int bc = f >> LOGW, w = f & (W - 1);
    float v = 0.f;
    if (bc < ch.n && w < tl.ncols) {
      const int b = ch.beta[bc];
      if (MODE == 1)
        v = dout[static_cast<int64_t>(tl.b) * A.phi_size + A.phi1_off + (static_cast<int64_t>(b) * RO + row) * A.n_frames +
                 tl.t0 + w];
      else
        v = dout[static_cast<int64_t>(tl.b) * A.v2_tot + A.v2_off[tl.a] + (static_cast<int64_t>(b) * RO + row) * stride +
                 tl.t0 + w];
    }
    dwb[i] = make_float2(v, 0.f);
  }
  __syncthreads();
  float2* dW = CtFft<false, LRO, LC, 0, LOGNFR>::run(dwb, z, S.tw);
  float2* X = (dW == dwb) ? z : dwb;
  {
    const float* lev = S.tc + A.ftabc_lev[K];
    const float4* dW4 = reinterpret_cast<const float4*>(dW);
    float4* X4 = reinterpret_cast<float4*>(X);
#pragma unroll 4
    for (int i = threadIdx.x; i < (R << LP); i += kThreads) {
      const int fp = i & ((1 << LP) - 1), m = i >> LP;
      const float sc = lev[m] * INVR;
      const float4 v = dW4[((m & (RO - 1)) << LP) + fp];
      X4[i] = make_float4(v.x * sc, v.y * sc, v.z * sc, v.w * sc);
    }
  }
  __syncthreads();
  float2* du = CtFft<true, LR, LC, 0, LOGNFR>::run(X, dW, S.tw);
  {
    float4* du4 = reinterpret_cast<float4*>(du);
    const float4* zb4 = reinterpret_cast<const float4*>(zb);
#pragma unroll 4
    for (int i = threadIdx.x; i < (R << LP); i += kThreads) {
      const float4 d = du4[i];
      const float4 v = zb4[i];
      const float m0 = sqrtf(v.x * v.x + v.y * v.y), m1 = sqrtf(v.z * v.z + v.w * v.w);
      const float g0 = m0 > 0.f ? d.x / m0 : 0.f, g1 = m1 > 0.f ? d.z / m1 : 0.f;
      du4[i] = make_float4(g0 * v.x, g0 * v.y, g1 * v.z, g1 * v.w);
    }
  }
  __syncthreads();
  float2* other = (du == X) ? dW : X;
  float2* dZ = CtFft<false, LR, LC, 0, LOGNFR>::run(du, other, S.tw);
  {
    const float4* dZ4 = reinterpret_cast<const float4*>(dZ);
    float4* D4 = reinterpret_cast<float4*>(D);
#pragma unroll 2
    for (int i = threadIdx.x; i < ((W * NFR) >> 1); i += kThreads) {
      const int wp = i & ((1 << LWP) - 1), m = i >> LWP;
      const int sgn = m < (NFR >> 1) ? m : m - NFR;
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int bc = 0; bc < ch.n; ++bc) {
        const int b = ch.beta[bc];
        const int2 bd = S.band[b];
        if (sgn < bd.x || sgn > bd.y) continue;
        const float gg = S.tc[S.toff[b] + (sgn - bd.x)];
        const float4 v = dZ4[((m & (R - 1)) << LP) + (bc << LWP) + wp];
        acc.x += gg * v.x;
        acc.y += gg * v.y;
        acc.z += gg * v.z;
        acc.w += gg * v.w;
      }
      float4 d = D4[i];
      d.x += acc.x * INVNFR;
      d.y += acc.y * INVNFR;
      d.z += acc.z * INVNFR;
      d.w += acc.w * INVNFR;
      D4[i] = d;
    }
  }
  __syncthreads();
}

// Compile-time dispatch over (K, LCADD) with LCADD <= min(K, 4), K <= LF.
template <int MODE, int LOGNFR, int LOGW, int LF, int K, int LCADD>
__device__ __forceinline__ void fwd_dispatch(int k, int lcadd, const FreqArgs& A, const FreqSmem& S,
                                             const FreqChunk& ch, const Tile& tl, int stride, const float2* yh,
                                             float2* f1, float2* f2, float* out) {
  if (k == K && lcadd == LCADD) {
    fwd_chunk<MODE, LOGNFR, LOGW, LF, K, LCADD>(A, S, ch, tl, stride, yh, f1, f2, out);
  } else if constexpr (LCADD < K && LCADD < 4) {
    fwd_dispatch<MODE, LOGNFR, LOGW, LF, K, LCADD + 1>(k, lcadd, A, S, ch, tl, stride, yh, f1, f2, out);
  } else if constexpr (K < LF) {
    fwd_dispatch<MODE, LOGNFR, LOGW, LF, K + 1, 0>(k, lcadd, A, S, ch, tl, stride, yh, f1, f2, out);
  }
}

template <int MODE, int LOGNFR, int LOGW, int LF, int K, int LCADD>
__device__ __forceinline__ void adj_dispatch(int k, int lcadd, const FreqArgs& A, const FreqSmem& S,
                                             const FreqChunk& ch, const Tile& tl, int stride, const float2* yh,
                                             float2* D, float2* zb, float2* f1, float2* f2, const float* dout) {
  if (k == K && lcadd == LCADD) {
    adj_chunk<MODE, LOGNFR, LOGW, LF, K, LCADD>(A, S, ch, tl, stride, yh, D, zb, f1, f2, dout);
  } else if constexpr (LCADD < K && LCADD < 4) {
    adj_dispatch<MODE, LOGNFR, LOGW, LF, K, LCADD + 1>(k, lcadd, A, S, ch, tl, stride, yh, D, zb, f1, f2, dout);
  } else if constexpr (K < LF) {
    adj_dispatch<MODE, LOGNFR, LOGW, LF, K + 1, 0>(k, lcadd, A, S, ch, tl, stride, yh, D, zb, f1, f2, dout);
  }
}

template <int MODE, int LOGNFR, int LOGW, int LF>
__global__ void __launch_bounds__(kThreads, 2)
k_freq_fwd_ct(FreqArgs A, const Tile* __restrict__ tiles, const float* __restrict__ S1,
              const float2* __restrict__ Y2, float* __restrict__ out) {
  extern __shared__ float2 sm[];
  constexpr int W = 1 << LOGW, NFR = 1 << LOGNFR, WN = W * NFR;
  const Tile tl = tiles[blockIdx.x];
  const FreqSmem S = freq_smem_carve(A, sm, 3);
  float2* buf0 = S.buf;
  float2* buf1 = buf0 + WN;
  float2* buf2 = buf1 + WN;
  freq_stage_tables(A, S);
  int stride, n1m;
  ct_load_columns<MODE, LOGNFR, LOGW>(A, tl, S1, Y2, buf0, stride, n1m);
  __syncthreads();
  float2* yh = CtFft<false, LOGNFR, LOGW, 0, LOGNFR>::run(buf0, buf1, S.tw);
  float2* f1 = (yh == buf0) ? buf1 : buf0;
  for (int c = 0; c < A.n_chunks; ++c) {
    const FreqChunk& ch = S.chk[c];
    fwd_dispatch<MODE, LOGNFR, LOGW, LF, 0, 0>(ch.k, ceil_log2(ch.n), A, S, ch, tl, stride, yh, f1, buf2, out);
  }
}

template <int MODE, int LOGNFR, int LOGW, int LF>
__global__ void __launch_bounds__(kThreads, 2)
k_freq_adj_ct(FreqArgs A, const Tile* __restrict__ tiles, const float* S1, const float2* __restrict__ Y2,
              const float* __restrict__ dout, float* dS1, float2* __restrict__ dY2) {
  extern __shared__ float2 sm[];
  constexpr int W = 1 << LOGW, NFR = 1 << LOGNFR, WN = W * NFR;
  const Tile tl = tiles[blockIdx.x];
  const FreqSmem S = freq_smem_carve(A, sm, 5);
  float2* buf0 = S.buf;
  float2* buf1 = buf0 + WN;
  float2* zb = buf1 + WN;
  float2* f1 = zb + WN;
  float2* f2 = f1 + WN;
  freq_stage_tables(A, S);
  int stride, n1m;
  ct_load_columns<MODE, LOGNFR, LOGW>(A, tl, S1, Y2, buf0, stride, n1m);
  __syncthreads();
  float2* yh = CtFft<false, LOGNFR, LOGW, 0, LOGNFR>::run(buf0, buf1, S.tw);
  float2* D = (yh == buf0) ? buf1 : buf0;
  {
    float4* D4 = reinterpret_cast<float4*>(D);
    for (int i = threadIdx.x; i < (WN >> 1); i += kThreads) D4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (int c = 0; c < A.n_chunks; ++c) {
    const FreqChunk& ch = S.chk[c];
    adj_dispatch<MODE, LOGNFR, LOGW, LF, 0, 0>(ch.k, ceil_log2(ch.n), A, S, ch, tl, stride, yh, D, zb, f1, f2, dout);
  }
  float2* dy = CtFft<true, LOGNFR, LOGW, 0, LOGNFR>::run(D, f1, S.tw);
  for (int i = threadIdx.x; i < n1m * W; i += kThreads) {
    const int w = i & (W - 1), r = i >> LOGW;
    if (w < tl.ncols) {
      const float2 v = dy[i];
      if (MODE == 1)
        dS1[(static_cast<int64_t>(tl.b) * A.N1 + r) * A.n_frames + tl.t0 + w] = v.x;
      else
        dY2[static_cast<int64_t>(tl.b) * A.y2_tot + A.y2_off[tl.a] + static_cast<int64_t>(r) * stride + tl.t0 + w] = v;
    }
  }
}

template <auto Kernel>
void opt_in_smem() {
  static const cudaError_t once = [] {
    const cudaError_t e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    cudaGetLastError();
    return e;
  }();
  (void)once;
}

// Specialised shapes, (log2 N_fr, log2 W, log2 F), are listed in the two
// launchers (jtfs_freq_ct_fwd.cu, jtfs_freq_ct_adj.cu): second-order kernels
// only; the first-order ones process N/T columns per clip and use the generic
// kernels.

}  // namespace
}  // namespace jtfs
