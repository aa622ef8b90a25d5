// Second-order frequential scattering on the 5th-generation tensor cores
// (§3.4 with the modulus of Eq. (2) and the phi_F averaging of Eq. (5)), and
// its adjoint (§2.3, Eq. (7)).
//
// Per time column t of one second-order path group (n2), the frequential
// step is two linear maps around a modulus:
//   Z_beta[r]  = sum_{n < n1max} H_beta[r][n] Y2[n][t]            (complex)
//   V_beta[ro] = sum_r P_k[ro][r] |Z_beta[r]|                      (real)
// with H_beta[r][n] = h_beta((2^k r - n) mod N_fr), h_beta the impulse
// response of the frequential filter on the N_fr grid (the band-limited
// table the FFT kernels fold), and P_k the phi_F averaging at level k
// (periodised onto N_fr / 2^k bins, then decimated to R_out rows).  Every
// column of a group shares H and P, so a tile of 128 columns is a pair of
// GEMMs:
//   GEMM1  D1[128 x 2 rc] = Y[128 x 2 n1] . B1^T   (real/imaginary interleaved)
//   GEMM2  D2[128 x R_out] += |D1| [128 x rc] . P^T   (accumulated over a filter's chunks)
// and the adjoint recomputes D1, then
//   GEMM2' dA[128 x rc] = dV [128 x R_out] . P        (d|Z|)
//   GEMM3  dY[128 x 2 n1] += (Z / |Z| dA) [128 x 2 rc] . B1   (accumulated over all chunks)
// FP32 accuracy from BF16 operands: every operand is split v = hi + lo (two
// BF16, relative residue ~2^-18) and each product is hi.hi + lo.hi + hi.lo
// (three MMAs into the same FP32 accumulator, ~1e-5 relative error).
//
// One CTA per tile of 128 columns (MMA M = 128 = TMEM lanes), 320 threads:
// warps 0-7 load and convert the operands written by threads and run the
// epilogues (warp w reads TMEM lanes 32 (w % 4) .. + 31, half w / 4 of the
// columns), warp 8 lane 0 issues the TMA loads of the constant tables into
// rings of shared-memory stages, warp 9 lane 0 issues tcgen05.mma (one chunk
// of GEMM1 ahead of GEMM2 / GEMM3; TMEM accumulators double-buffered).  All
// hand-offs are mbarriers; every wait is bounded and an expired wait aborts
// the CTA (TMA copies drained, MMAs completed, TMEM freed) and raises a flag
// read by jtfs_tc_error().
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "jtfs.h"
#include "jtfs_internal.h"
#include "jtfs_umma.cuh"

namespace jtfs {
namespace {

__device__ int g_tc_err;
// First expired wait since the last jtfs_tc_error() (diagnostics): CTA, thread,
// barrier offset inside the CTA's control block, parity.
__device__ int g_tc_err_info[4];

constexpr int kTcM = 128;                // columns per tile
constexpr int kS2 = 2;                   // stages of the pooling-table ring (4 KB each)

struct TcArgs {
  const TcChunk* chunks;
  int n_chunks;
  const Tile* tiles;
  const int* n1max_act;
  const int* s2;
  const int64_t* y2_off;
  const int64_t* v2_off;
  int64_t y2_tot, v2_tot;
  int logN, RO, nr1;
  const float2* Y2;
  float* V2;         // forward output
  const float* dV2;  // adjoint input
  float2* dY2;       // adjoint output
};

struct TcCtl {
  unsigned long long b1_full[16], b1_empty[16], b2_full[4], b2_empty[4], b3_full[8], b3_empty[8];
  unsigned long long a1_full, d1_full[2], d1_empty[2], a2_full[2], a2_empty[2], d2_full[2], d2_empty[2];
  unsigned long long dv_full[2], dv_empty[2], d3_full, drain[3];
  uint32_t tmem;
  int abort;
};

__device__ __forceinline__ void st_shared_v4(uint32_t addr, const uint32_t (&v)[4]) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
               : "memory");
}
__device__ __forceinline__ uint64_t kdesc(uint32_t addr) { return sdesc(addr, 16, 1024); }

// Wait on an mbarrier phase regardless of the abort flag (teardown only), bounded.
__device__ __forceinline__ void mbar_wait_drain(uint32_t bar, uint32_t parity) {
  for (uint32_t i = 0; i < kSpinLimit && !mbar_try_wait(bar, parity); ++i) __nanosleep(64);
}

// Records the first expired wait since the last jtfs_tc_error_info() (kept out
// of line: it runs at most once per CTA).
__device__ __noinline__ void tc_wait_expired(uint32_t bar, uint32_t parity) {
  if (atomicCAS(&g_tc_err_info[0], 0, int(blockIdx.x) + 1) == 0) {
    extern __shared__ uint8_t smem_raw[];
    g_tc_err_info[1] = int(threadIdx.x);
    g_tc_err_info[2] = int(bar - smem_u32(smem_raw));
    g_tc_err_info[3] = int(parity);
  }
}

// Bounded mbarrier wait: at most c_wait_polls polls (see mbar_wait); gives up
// early once another role of the CTA aborted.
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  const uint32_t polls = c_wait_polls;
  for (uint32_t i = 0; i < polls; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    if (i >= 8) __nanosleep(64);
  }
  *abort = 1;
  tc_wait_expired(bar, parity);
  return false;
}

// |x + iy| from the hardware reciprocal square root (a few ulp; the epilogues
// are instruction-bound and the correctly rounded sqrtf costs a long sequence).
__device__ __forceinline__ float modulus(float x, float y) {
  const float m2 = x * x + y * y;
  return m2 > 0.f ? m2 * rsqrtf(m2) : 0.f;
}

// Bounded wait taken by a whole epilogue warp: the tcgen05.ld that follow are
// warp-collective, so every lane must make the same decision.
__device__ __forceinline__ bool wait_warp(uint32_t bar, uint32_t parity, volatile int* abort) {
  const bool ok = tc_wait(bar, parity, abort);
  return __all_sync(0xffffffffu, ok);
}

// Y2 tile -> A1 in tensor memory: lane c (this warp's 32 lanes), column word n
// holds (Re, Im) of Y2 row n as BF16 hi at a1 + n and lo at a1 + 32 KA + n (K
// index 2n + (re, im)).  Warp-collective: words
// 4g .. 4g + 3 for g = part, part + nparts, ...; rows n >= n1max are zero.
template <int KA>
__device__ __forceinline__ void load_a1_tmem(const TcArgs& A, const Tile& tl, int n1m, int ks1, uint32_t a1, int c,
                                             int part, int nparts) {
  const int L2 = 1 << (A.logN - A.s2[tl.a]);
  const float2* ysrc = A.Y2 + int64_t(tl.b) * A.y2_tot + A.y2_off[tl.a] + tl.t0 + c;
  const bool colok = c < tl.ncols;
  for (int g = part; g < 2 * ks1; g += nparts) {
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int n = 4 * g + e;
      float2 v = make_float2(0.f, 0.f);
      if (colok && n < n1m) v = ysrc[int64_t(n) * L2];
      split2(v.x, v.y, hi[e], lo[e]);
    }
    tmem_st4(a1 + uint32_t(4 * g), hi);
    tmem_st4(a1 + uint32_t(32 * KA + 4 * g), lo);
  }
}

// GEMM1 of one chunk with A1 in tensor memory (hi at a1, lo at a1 + 32 KA).
template <int KA, int S1>
__device__ __forceinline__ bool issue_g1_ts(TcCtl* ctl, const TcChunk& c, int ks1, uint32_t a1, uint32_t sB1,
                                            uint32_t d, int& c1, volatile int* abort) {
  const uint32_t idesc = idesc_bf16_n(2 * c.rc);
  const int na = (ks1 + 3) >> 2;
  for (int a = 0; a < na; ++a) {
    const int s = c1 % S1;
    if (!tc_wait(smem_u32(&ctl->b1_full[s]), (c1 / S1) & 1, abort)) return false;
    tc_fence_after();
    const uint64_t bh = kdesc(sB1 + uint32_t(s) * 16384u), bl = bh + (8192u >> 4);
    const int kn = min(4, ks1 - a * 4);
    for (int kk = 0; kk < kn; ++kk) {
      const uint64_t o = uint64_t(kk) * 2u;            // 32 bytes in 16-byte descriptor units
      const uint32_t ah = a1 + uint32_t(32 * a + 8 * kk), al = ah + uint32_t(32 * KA);  // 8 words = 16 K
      umma_bf16_ts(d, ah, bh + o, idesc, (a | kk) != 0);
      umma_bf16_ts(d, al, bh + o, idesc, 1);
      umma_bf16_ts(d, ah, bl + o, idesc, 1);
    }
    umma_commit(smem_u32(&ctl->b1_empty[s]));
    ++c1;
  }
  return true;
}

// ---------------------------------------------------------------------------
// Thread roles of both kernels: warps 0-15 are two epilogue groups of 8 warps
// (group g takes the chunks i with i % 2 == g; inside a group warp w reads TMEM
// lanes 32 (w % 4) .. + 31 and half (w % 8) / 4 of the chunk's columns),
// warp 16 lane 0 issues the TMA loads, warps 17, 18 (and 19 in the adjoint)
// lane 0 each issue one GEMM, so that their barrier waits overlap.  Chunk
// descriptors are read one chunk ahead (a global read on the issue path costs
// more than the MMAs it feeds).
// ---------------------------------------------------------------------------
constexpr int kGrp = 256;                 // threads per epilogue group
constexpr int kEpiAll = 2 * kGrp;         // epilogue threads
constexpr int kWarpTma = 16, kWarpG1 = 17, kWarpG2 = 18, kWarpG3 = 19;

__device__ __forceinline__ void init_barriers(TcCtl* ctl, int n_epi) {
  for (int s = 0; s < 16; ++s) {
    mbar_init(smem_u32(&ctl->b1_full[s]), 1);
    mbar_init(smem_u32(&ctl->b1_empty[s]), 1);
  }
  for (int s = 0; s < 8; ++s) {
    mbar_init(smem_u32(&ctl->b3_full[s]), 1);
    mbar_init(smem_u32(&ctl->b3_empty[s]), 1);
  }
  for (int s = 0; s < kS2; ++s) {
    mbar_init(smem_u32(&ctl->b2_full[s]), 1);
    mbar_init(smem_u32(&ctl->b2_empty[s]), 1);
  }
  for (int s = 0; s < 2; ++s) {
    mbar_init(smem_u32(&ctl->d1_full[s]), 1);
    mbar_init(smem_u32(&ctl->d1_empty[s]), kGrp);
    mbar_init(smem_u32(&ctl->a2_full[s]), kGrp);
    mbar_init(smem_u32(&ctl->a2_empty[s]), 1);
    mbar_init(smem_u32(&ctl->d2_full[s]), 1);
    mbar_init(smem_u32(&ctl->d2_empty[s]), kGrp);
    mbar_init(smem_u32(&ctl->dv_full[s]), kGrp);
    mbar_init(smem_u32(&ctl->dv_empty[s]), 1);
  }
  mbar_init(smem_u32(&ctl->a1_full), n_epi);
  mbar_init(smem_u32(&ctl->d3_full), 1);
  for (int s = 0; s < 3; ++s) mbar_init(smem_u32(&ctl->drain[s]), 1);
  ctl->abort = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// TMA loads of one chunk's GEMM1 table rows (one stage per K atom used).
template <int S1>
__device__ __forceinline__ bool load_b1(TcCtl* ctl, const CUtensorMap* tm, const TcChunk& c, int ks1, int nr1,
                                        uint32_t sB1, int& n1, volatile int* abort) {
  const int na = (ks1 + 3) >> 2;
  for (int a = 0; a < na; ++a) {
    const int s = n1 % S1;
    if (n1 >= S1 && !tc_wait(smem_u32(&ctl->b1_empty[s]), ((n1 / S1) - 1) & 1, abort)) return false;
    const uint32_t bar = smem_u32(&ctl->b1_full[s]);
    mbar_expect_tx(bar, 16384u);
    tma_load_2d(sB1 + uint32_t(s) * 16384u, tm, bar, a * 64, c.b1row);
    tma_load_2d(sB1 + uint32_t(s) * 16384u + 8192u, tm, bar, a * 64, nr1 + c.b1row);
    ++n1;
  }
  return true;
}

__device__ __forceinline__ TcChunk ld_chunk(const TcChunk* p, int i, int n) {
  TcChunk c{};
  if (i < n) {
    const int4* q = reinterpret_cast<const int4*>(p + i);
    const int4 x = __ldg(q), y = __ldg(q + 1);
    c = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
  }
  return c;
}

// ---------------------------------------------------------------------------
// Forward: V2 of one tile of 128 columns.
// Shared memory: B1 ring S1 x 16 KB (64 table rows hi | lo), B2 ring kS2 x 4 KB
// (R_out rows, hi|lo packed in each 128-byte row), A2 2 x 16 KB (|Z| hi|lo
// packed, one per group).
// TMEM: D1 2 x 64 columns at 0, D2 2 x 32 columns at 128, A1 (the Y2 tile, as
// in the adjoint: 32 KA hi + 32 KA lo columns) at 192: 256 columns in all for
// KA = 1 (two CTAs per SM), 512 for KA = 2 .. 5 (n1max up to 160).
// ---------------------------------------------------------------------------
// Forward threads with NG epilogue groups: 8 NG epilogue warps, then the TMA
// warp and the two issuing warps.  NG = 1 runs two CTAs per SM (two
// independent hand-off chains per SM instead of two groups in one CTA).
template <int NG>
constexpr int tc_fwd_threads() { return (8 * NG + 3) * 32; }
constexpr int kTcAdjThreads = 20 * 32;

template <int KA, int S1>
constexpr size_t tc_fwd_smem() {
  return sizeof(TcCtl) + 1024 + size_t(S1) * 16384 + size_t(kS2) * 4096 + 2 * 16384;
}
template <int KA> __host__ __device__ constexpr uint32_t fwd_a1_col() { return 192u; }
template <int KA> __host__ __device__ constexpr uint32_t fwd_tmem_cols() { return KA == 1 ? 256u : 512u; }

template <int KA, int S1, int NG>
__global__ void __launch_bounds__(tc_fwd_threads<NG>(), NG == 1 ? 2 : 1)
k_freq_tc_fwd(const __grid_constant__ CUtensorMap tmB1, const __grid_constant__ CUtensorMap tmB2, const TcArgs A) {
  constexpr int wTma = 8 * NG, wG1 = wTma + 1, wG2 = wTma + 2;
  extern __shared__ uint8_t smem_raw[];
  TcCtl* ctl = reinterpret_cast<TcCtl*>(smem_raw);
  const uint32_t base = (smem_u32(smem_raw) + sizeof(TcCtl) + 1023u) & ~1023u;
  const uint32_t sB1 = base;
  constexpr uint32_t kA1 = fwd_a1_col<KA>(), kCols = fwd_tmem_cols<KA>();
  const uint32_t sB2 = sB1 + uint32_t(S1) * 16384u;
  const uint32_t sA2 = sB2 + uint32_t(kS2) * 4096u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Tile tl = A.tiles[blockIdx.x];
  const int n1m = A.n1max_act[tl.a];
  const int ks1 = (2 * n1m + 15) >> 4;
  const int nch = A.n_chunks, RO = A.RO;
  volatile int* abort = &ctl->abort;
  if (threadIdx.x == 0) init_barriers(ctl, kGrp * NG);
  if (warp == wG1) tmem_alloc(smem_u32(&ctl->tmem), kCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem;
  int n1 = 0, n2 = 0;  // TMA stages issued (producer)
  bool issued = false;

  if (warp == wTma) {
    if (lane == 0) {
      TcChunk nx = ld_chunk(A.chunks, 0, nch);
      bool ok = load_b1<S1>(ctl, &tmB1, nx, ks1, A.nr1, sB1, n1, abort);
      TcChunk cur = nx;
      for (int i = 0; ok && i < nch; ++i) {
        nx = ld_chunk(A.chunks, i + 1, nch);
        if (i + 1 < nch) ok = load_b1<S1>(ctl, &tmB1, nx, ks1, A.nr1, sB1, n1, abort);
        if (!ok) break;
        const int s = n2 % kS2;
        if (n2 >= kS2 && !tc_wait(smem_u32(&ctl->b2_empty[s]), ((n2 / kS2) - 1) & 1, abort)) break;
        const uint32_t bar = smem_u32(&ctl->b2_full[s]);
        mbar_expect_tx(bar, uint32_t(RO) * 128u);
        tma_load_2d(sB2 + uint32_t(s) * 4096u, &tmB2, bar, 64 * (cur.r0 >> 5), cur.k * RO);
        ++n2;
        cur = nx;
      }
    }
  } else if (warp == wG1) {
    if (lane == 0) {  // GEMM1: D1[i & 1] = Y . B1 (chunk i)
      issued = true;
      int c1 = 0;
      bool ok = tc_wait(smem_u32(&ctl->a1_full), 0, abort);
      tc_fence_after();
      TcChunk nx = ld_chunk(A.chunks, 0, nch);
      for (int i = 0; ok && i < nch; ++i) {
        const TcChunk c = nx;
        nx = ld_chunk(A.chunks, i + 1, nch);
        const int j = i & 1;
        if (i >= 2) {
          if (!tc_wait(smem_u32(&ctl->d1_empty[j]), ((i >> 1) - 1) & 1, abort)) break;
          tc_fence_after();
        }
        if (!issue_g1_ts<KA, S1>(ctl, c, ks1, tmem + kA1, sB1, tmem + uint32_t(j) * 64u, c1, abort)) break;
        umma_commit(smem_u32(&ctl->d1_full[j]));
      }
    }
  } else if (warp == wG2) {
    if (lane == 0) {  // GEMM2: D2[beta & 1] += |Z| . P^T (chunk i)
      issued = true;
      int c2 = 0;
      const uint32_t idesc2 = idesc_bf16_n(RO);
      TcChunk nx = ld_chunk(A.chunks, 0, nch);
      for (int i = 0; i < nch; ++i) {
        const TcChunk c = nx;
        nx = ld_chunk(A.chunks, i + 1, nch);
        const int ja = i & 1, s = c2 % kS2, bj = c.beta & 1;
        if (!tc_wait(smem_u32(&ctl->a2_full[ja]), (i >> 1) & 1, abort)) break;
        if (!tc_wait(smem_u32(&ctl->b2_full[s]), (c2 / kS2) & 1, abort)) break;
        if (c.first && c.beta >= 2 && !tc_wait(smem_u32(&ctl->d2_empty[bj]), ((c.beta >> 1) - 1) & 1, abort)) break;
        tc_fence_after();
        const uint32_t d = tmem + 128u + uint32_t(bj) * 32u;
        const uint64_t a2 = kdesc(sA2 + uint32_t(ja) * 16384u), b2 = kdesc(sB2 + uint32_t(s) * 4096u);
        for (int kk = 0; kk < (c.rc >> 4); ++kk) {
          const uint64_t o = uint64_t(kk) * 2u;
          umma_bf16(d, a2 + o, b2 + o, idesc2, !(c.first && kk == 0));
          umma_bf16(d, a2 + 4u + o, b2 + o, idesc2, 1);
          umma_bf16(d, a2 + o, b2 + 4u + o, idesc2, 1);
        }
        umma_commit(smem_u32(&ctl->a2_empty[ja]));
        umma_commit(smem_u32(&ctl->b2_empty[s]));
        if (c.last) umma_commit(smem_u32(&ctl->d2_full[bj]));
        ++c2;
      }
    }
  } else if (warp < wTma) {
    // Epilogue groups.
    const int g = warp >> 3, q = warp & 3, h = (warp >> 2) & 1;
    const int c = q * 32 + lane;
    const uint32_t lane_off = uint32_t(q * 32) << 16;
    const bool colok = c < tl.ncols;
    const int L2 = 1 << (A.logN - A.s2[tl.a]);
    float* vdst = A.V2 + int64_t(tl.b) * A.v2_tot + A.v2_off[tl.a] + tl.t0 + c;
    load_a1_tmem<KA>(A, tl, n1m, ks1, tmem + lane_off + kA1, c, (warp >> 2) & (2 * NG - 1), 2 * NG);
    tmem_st_wait();
    tc_fence_before();
    mbar_arrive(smem_u32(&ctl->a1_full));
    auto store_v2 = [&](int beta) -> bool {
      const int bj = beta & 1;
      if (!wait_warp(smem_u32(&ctl->d2_full[bj]), (beta >> 1) & 1, abort)) return false;
      tc_fence_after();
      const int half = RO >> 1;
      const uint32_t taddr = tmem + lane_off + 128u + uint32_t(bj) * 32u + uint32_t(h * half);
      float v[16];
      if (half == 16) {
        uint32_t r[16];
        tmem_ld16_nowait(taddr, r);
        tmem_ld_wait();
        tmem_regs_ready(r);
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(r[e]);
      } else {
        uint32_t r[8];
        tmem_ld8_nowait(taddr, r);
        tmem_ld_wait();
        tmem_regs_ready(r);
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(r[e]);
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&ctl->d2_empty[bj]));
      if (colok) {
        float* o = vdst + (int64_t(beta) * RO + h * half) * L2;
#pragma unroll
        for (int e = 0; e < 16; ++e)
          if (e < half) o[int64_t(e) * L2] = v[e];
      }
      return true;
    };
    // V2 of a filter is stored after this group's next chunk, not at once: GEMM2 of the filter's last chunk
    // needs the |Z| this group has just written, and waiting for it here would leave the group idle for
    // that GEMM's whole latency.  D2[beta & 1] is free again once stored, before GEMM2 of beta + 2 needs it.
    int pend = -1;
    bool eok = true;
    TcChunk nx = ld_chunk(A.chunks, g, nch);
    for (int i = g; i < nch; i += NG) {
      const TcChunk ch = nx;
      nx = ld_chunk(A.chunks, i + NG, nch);
      const int j = i & 1;
      if (!wait_warp(smem_u32(&ctl->d1_full[j]), (i >> 1) & 1, abort)) { eok = false; break; }
      tc_fence_after();
      // D1 columns [h rc, h rc + rc): rc / 2 complex values, rows r = h rc / 2 + e.
      const uint32_t taddr = tmem + lane_off + uint32_t(j) * 64u + uint32_t(h * ch.rc);
      float mag[16];
      if (ch.rc == 32) {
        float z[32];
        tmem_ld32(taddr, z);
#pragma unroll
        for (int e = 0; e < 16; ++e) mag[e] = modulus(z[2 * e], z[2 * e + 1]);
      } else {
        uint32_t r[16];
        tmem_ld16_nowait(taddr, r);
        tmem_ld_wait();
        tmem_regs_ready(r);
#pragma unroll
        for (int e = 0; e < 8; ++e) mag[e] = modulus(__uint_as_float(r[2 * e]), __uint_as_float(r[2 * e + 1]));
#pragma unroll
        for (int e = 8; e < 16; ++e) mag[e] = 0.f;
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&ctl->d1_empty[j]));
      // |Z| rows into this group's A2 (hi at K = r, lo at K = 32 + r) once GEMM2 of chunk i - 2 has read it.
      if (i >= 2 && !wait_warp(smem_u32(&ctl->a2_empty[j]), ((i >> 1) - 1) & 1, abort)) { eok = false; break; }
      const uint32_t a2 = sA2 + uint32_t(j) * 16384u;
      const int nck = ch.rc >> 4, ck0 = h * nck;
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        if (t < nck) {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) split2(mag[8 * t + 2 * e], mag[8 * t + 2 * e + 1], hi[e], lo[e]);
          st_shared_v4(a2 + swz128(c, ck0 + t), hi);
          st_shared_v4(a2 + swz128(c, 4 + ck0 + t), lo);
        }
      }
      fence_proxy_async();
      mbar_arrive(smem_u32(&ctl->a2_full[j]));
      if (pend >= 0 && !store_v2(pend)) { eok = false; break; }
      pend = ch.last ? ch.beta : -1;
    }
    if (eok && pend >= 0) store_v2(pend);
  }

  // Teardown: no TMA copy or MMA of this CTA may be in flight when it exits.
  if (warp == wTma && lane == 0 && *abort) {
    for (int t = max(0, n1 - S1); t < n1; ++t) mbar_wait_drain(smem_u32(&ctl->b1_full[t % S1]), (t / S1) & 1);
    for (int t = max(0, n2 - kS2); t < n2; ++t) mbar_wait_drain(smem_u32(&ctl->b2_full[t % kS2]), (t / kS2) & 1);
  }
  if ((warp == wG1 || warp == wG2) && lane == 0 && issued) {
    const uint32_t dr = smem_u32(&ctl->drain[warp - wG1]);
    umma_commit(dr);
    mbar_wait_drain(dr, 0);
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort) atomicExch(&g_tc_err, 1);
  if (warp == wG1) {
    __syncwarp();
    tmem_dealloc(tmem, kCols);
  }
}

// ---------------------------------------------------------------------------
// Adjoint: dY2 of one tile of 128 columns, from Y2 (recomputed Z) and dV2.
// The two data operands that are M x K tiles of the tile's columns, A1 (the Y2
// tile, for GEMM1) and A3 (dZ of a chunk, for GEMM3), live in tensor memory:
// an MMA at N = 64 reading a 4 KB A tile and a 2 KB B tile from shared memory
// each time is bound by shared-memory bandwidth once the three GEMMs, the TMA
// writes and the epilogue share it; from TMEM only B is read there, and the
// epilogue writes dZ with tcgen05.st instead of shared-memory stores.
// Shared memory: B1 ring S1 x 16 KB, B2' ring kS2 x 4 KB (32 table rows, hi|lo
// packed), dV 2 x 16 KB (hi|lo packed), B3 ring S3 x 16 KA KB (64 KA rows
// (n, re/im) x 64 K, hi then lo; GEMM3 runs at N = 2 n1max).
// TMEM (512 columns): D1 2 x 64 at 0, D2' 2 x 32 at 128, then
//   KA = 1: D3 (<= 64) at 192, A1 (32 hi + 32 lo) at 256, A3 NA3 x 64 at 320;
//   KA = 2: A3 (one, 64) at 192, D3 (<= 128) at 256, A1 (64 hi + 64 lo) at 384.
// ---------------------------------------------------------------------------
template <int KA, int S1, int S3>
constexpr size_t tc_adj_smem() {
  return sizeof(TcCtl) + 1024 + size_t(S1) * 16384 + size_t(kS2) * 4096 + 2 * 16384 + size_t(S3) * 16384 * KA;
}
template <int KA> __host__ __device__ constexpr uint32_t adj_d3_col() { return KA == 1 ? 192u : 256u; }
template <int KA> __host__ __device__ constexpr uint32_t adj_a1_col() { return KA == 1 ? 256u : 384u; }
template <int KA> __host__ __device__ constexpr uint32_t adj_a3_col() { return KA == 1 ? 320u : 192u; }

template <int KA, int S1, int S3, int NA3>
__global__ void __launch_bounds__(kTcAdjThreads, 1)
k_freq_tc_adj(const __grid_constant__ CUtensorMap tmB1, const __grid_constant__ CUtensorMap tmB2t,
              const __grid_constant__ CUtensorMap tmB3, const TcArgs A) {
  static_assert(NA3 >= 1 && NA3 <= (KA == 1 ? 2 : 1), "A3 buffers must fit the TMEM map");
  extern __shared__ uint8_t smem_raw[];
  TcCtl* ctl = reinterpret_cast<TcCtl*>(smem_raw);
  const uint32_t base = (smem_u32(smem_raw) + sizeof(TcCtl) + 1023u) & ~1023u;
  const uint32_t sB1 = base;
  const uint32_t sB2 = sB1 + uint32_t(S1) * 16384u;
  const uint32_t sDV = sB2 + uint32_t(kS2) * 4096u;
  const uint32_t sB3 = sDV + 2u * 16384u;  // ring of S3 stages of 16 KB x KA
  constexpr uint32_t kD3 = adj_d3_col<KA>(), kA1 = adj_a1_col<KA>(), kA3 = adj_a3_col<KA>();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Tile tl = A.tiles[blockIdx.x];
  const int n1m = A.n1max_act[tl.a];
  const int ks1 = (2 * n1m + 15) >> 4;
  const int k1pad = 16 * ks1;               // GEMM3 N (columns (n, re/im) kept)
  constexpr uint32_t kB3 = 16384u * KA;     // B3 stage: 64 KA rows (n, re/im) x 64 K, hi then lo
  const int nch = A.n_chunks, RO = A.RO;
  const int nbeta = ld_chunk(A.chunks, nch - 1, nch).beta + 1;
  volatile int* abort = &ctl->abort;
  if (threadIdx.x == 0) init_barriers(ctl, kEpiAll);
  if (warp == kWarpG1) tmem_alloc(smem_u32(&ctl->tmem), 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem;
  int n1 = 0, n2 = 0, n3 = 0;
  bool issued = false;

  if (warp == kWarpTma) {
    if (lane == 0) {
      auto load_b2 = [&](const TcChunk& c) -> bool {
        const int s = n2 % kS2;
        if (n2 >= kS2 && !tc_wait(smem_u32(&ctl->b2_empty[s]), ((n2 / kS2) - 1) & 1, abort)) return false;
        const uint32_t bar = smem_u32(&ctl->b2_full[s]);
        mbar_expect_tx(bar, 4096u);
        tma_load_2d(sB2 + uint32_t(s) * 4096u, &tmB2t, bar, 0, c.prow);
        ++n2;
        return true;
      };
      auto load_b3 = [&](const TcChunk& c) -> bool {  // one stage: hi rows [0, 64 KA), then lo rows
        const int s = n3 % S3;
        if (n3 >= S3 && !tc_wait(smem_u32(&ctl->b3_empty[s]), ((n3 / S3) - 1) & 1, abort)) return false;
        const uint32_t bar = smem_u32(&ctl->b3_full[s]), st = sB3 + uint32_t(s) * kB3;
        mbar_expect_tx(bar, kB3);
        for (int u = 0; u < KA; ++u) {
          tma_load_2d(st + 8192u * u, &tmB3, bar, c.b1row, 64 * u);
          tma_load_2d(st + 8192u * (KA + u), &tmB3, bar, c.b1row, 128 + 64 * u);
        }
        ++n3;
        return true;
      };
      TcChunk cur = ld_chunk(A.chunks, 0, nch);
      bool ok = load_b1<S1>(ctl, &tmB1, cur, ks1, A.nr1, sB1, n1, abort) && load_b2(cur);
      for (int i = 0; ok && i < nch; ++i) {
        const TcChunk nx = ld_chunk(A.chunks, i + 1, nch);
        if (i + 1 < nch) ok = load_b1<S1>(ctl, &tmB1, nx, ks1, A.nr1, sB1, n1, abort) && load_b2(nx);
        if (ok) ok = load_b3(cur);
        cur = nx;
      }
    }
  } else if (warp == kWarpG1) {
    if (lane == 0) {  // GEMM1 (recompute Z): D1[i & 1]
      issued = true;
      int c1 = 0;
      bool ok = tc_wait(smem_u32(&ctl->a1_full), 0, abort);
      tc_fence_after();
      TcChunk nx = ld_chunk(A.chunks, 0, nch);
      for (int i = 0; ok && i < nch; ++i) {
        const TcChunk c = nx;
        nx = ld_chunk(A.chunks, i + 1, nch);
        const int j = i & 1;
        if (i >= 2) {
          if (!tc_wait(smem_u32(&ctl->d1_empty[j]), ((i >> 1) - 1) & 1, abort)) break;
          tc_fence_after();
        }
        if (!issue_g1_ts<KA, S1>(ctl, c, ks1, tmem + kA1, sB1, tmem + uint32_t(j) * 64u, c1, abort)) break;
        umma_commit(smem_u32(&ctl->d1_full[j]));
      }
    }
  } else if (warp == kWarpG2) {
    if (lane == 0) {  // GEMM2': d|Z| = dV . P into D2'[i & 1]
      issued = true;
      int c2 = 0;
      TcChunk nx = ld_chunk(A.chunks, 0, nch);
      for (int i = 0; i < nch; ++i) {
        const TcChunk c = nx;
        nx = ld_chunk(A.chunks, i + 1, nch);
        const int bj = c.beta & 1, j = i & 1, s = c2 % kS2;
        if (c.first && !tc_wait(smem_u32(&ctl->dv_full[bj]), (c.beta >> 1) & 1, abort)) break;
        if (i >= 2) {
          if (!tc_wait(smem_u32(&ctl->d2_empty[j]), ((i >> 1) - 1) & 1, abort)) break;
          tc_fence_after();
        }
        if (!tc_wait(smem_u32(&ctl->b2_full[s]), (c2 / kS2) & 1, abort)) break;
        tc_fence_after();
        const uint32_t d = tmem + 128u + uint32_t(j) * 32u;
        const uint32_t idesc = idesc_bf16_n(c.rc);
        const uint64_t a = kdesc(sDV + uint32_t(bj) * 16384u), b = kdesc(sB2 + uint32_t(s) * 4096u);
        for (int kk = 0; kk < (RO >> 4); ++kk) {
          const uint64_t o = uint64_t(kk) * 2u;
          umma_bf16(d, a + o, b + o, idesc, kk != 0);
          umma_bf16(d, a + 4u + o, b + o, idesc, 1);
          umma_bf16(d, a + o, b + 4u + o, idesc, 1);
        }
        umma_commit(smem_u32(&ctl->b2_empty[s]));
        umma_commit(smem_u32(&ctl->d2_full[j]));
        if (c.last) umma_commit(smem_u32(&ctl->dv_empty[bj]));
        ++c2;
      }
    }
  } else if (warp == kWarpG3) {
    if (lane == 0) {  // GEMM3: D3 += dZ . B1 (rows of chunk i); A3 buffers use the a2 barriers.
      issued = true;
      int c3 = 0;
      TcChunk nx = ld_chunk(A.chunks, 0, nch);
      for (int i = 0; i < nch; ++i) {
        const TcChunk c = nx;
        nx = ld_chunk(A.chunks, i + 1, nch);
        const int ja = i % NA3;
        if (!tc_wait(smem_u32(&ctl->a2_full[ja]), (i / NA3) & 1, abort)) break;
        tc_fence_after();
        const uint32_t a3 = tmem + kA3 + uint32_t(ja) * 64u;  // dZ hi words 0..31, lo 32..63
        // N = k1pad (all (n, re/im) columns kept) in one MMA per term and K step.
        const int s = c3 % S3;
        if (!tc_wait(smem_u32(&ctl->b3_full[s]), (c3 / S3) & 1, abort)) break;
        tc_fence_after();
        const uint64_t bh = kdesc(sB3 + uint32_t(s) * kB3), bl = bh + ((8192u * KA) >> 4);
        const uint32_t d = tmem + kD3;
        const uint32_t idesc = idesc_bf16_n(k1pad);
        for (int kk = 0; kk < (c.rc >> 3); ++kk) {  // K = 2 rc
          const uint64_t o = uint64_t(kk) * 2u;
          const uint32_t ah = a3 + uint32_t(8 * kk), al = ah + 32u;
          umma_bf16_ts(d, ah, bh + o, idesc, (i | kk) != 0);
          umma_bf16_ts(d, al, bh + o, idesc, 1);
          umma_bf16_ts(d, ah, bl + o, idesc, 1);
        }
        umma_commit(smem_u32(&ctl->b3_empty[s]));
        ++c3;
        umma_commit(smem_u32(&ctl->a2_empty[i & 1]));  // keyed on the chunk, not the buffer
        if (i == nch - 1) umma_commit(smem_u32(&ctl->d3_full));
      }
    }
  } else if (warp < kWarpTma) {
    // Epilogue groups.
    const int g = warp >> 3, q = warp & 3, h = (warp >> 2) & 1;
    const int c = q * 32 + lane;
    const uint32_t lane_off = uint32_t(q * 32) << 16;
    const bool colok = c < tl.ncols;
    const int L2 = 1 << (A.logN - A.s2[tl.a]);
    const float* vsrc = A.dV2 + int64_t(tl.b) * A.v2_tot + A.v2_off[tl.a] + tl.t0 + c;
    // dV of filter beta (R_out rows) into dV buffer beta & 1: hi at K = ro, lo at K = 32 + ro.
    auto load_dv = [&](int beta) {
      const int half = RO >> 1;
      const float* src = vsrc + (int64_t(beta) * RO + h * half) * L2;
      float v[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) v[e] = (colok && e < half) ? src[int64_t(e) * L2] : 0.f;
      const uint32_t dv = sDV + uint32_t(beta & 1) * 16384u;
      const int nck = half >> 3, ck0 = h * nck;
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        if (t < nck) {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) split2(v[8 * t + 2 * e], v[8 * t + 2 * e + 1], hi[e], lo[e]);
          st_shared_v4(dv + swz128(c, ck0 + t), hi);
          st_shared_v4(dv + swz128(c, 4 + ck0 + t), lo);
        }
      }
    };
    load_a1_tmem<KA>(A, tl, n1m, ks1, tmem + lane_off + kA1, c, (warp >> 2) & 3, 4);
    tmem_st_wait();
    if (g == 0) load_dv(0);
    fence_proxy_async();
    tc_fence_before();
    mbar_arrive(smem_u32(&ctl->a1_full));
    if (g == 0) mbar_arrive(smem_u32(&ctl->dv_full[0]));
    bool ok = true;
    TcChunk nx = ld_chunk(A.chunks, g, nch);
    for (int i = g; i < nch; i += 2) {
      const TcChunk ch = nx;
      nx = ld_chunk(A.chunks, i + 2, nch);
      const int j = i & 1;
      if (ch.first && ch.beta + 1 < nbeta) {
        const int nb = ch.beta + 1, bj = nb & 1;
        if (nb >= 2 && !wait_warp(smem_u32(&ctl->dv_empty[bj]), ((nb >> 1) - 1) & 1, abort)) { ok = false; break; }
        load_dv(nb);
        fence_proxy_async();
        mbar_arrive(smem_u32(&ctl->dv_full[bj]));
      }
      if (!wait_warp(smem_u32(&ctl->d1_full[j]), (i >> 1) & 1, abort)) { ok = false; break; }
      if (!wait_warp(smem_u32(&ctl->d2_full[j]), (i >> 1) & 1, abort)) { ok = false; break; }
      tc_fence_after();
      // Z rows r = h rc / 2 + e (D1 columns [h rc, h rc + rc)) and d|Z| (D2' columns [h rc / 2, ...)).
      float z[32], gz[16];
      if (ch.rc == 32) {
        uint32_t r[32], r16[16];
        tmem_ld16_nowait(tmem + lane_off + uint32_t(j) * 64u + uint32_t(h * 32), *reinterpret_cast<uint32_t(*)[16]>(r));
        tmem_ld16_nowait(tmem + lane_off + uint32_t(j) * 64u + uint32_t(h * 32 + 16),
                         *reinterpret_cast<uint32_t(*)[16]>(r + 16));
        tmem_ld16_nowait(tmem + lane_off + 128u + uint32_t(j) * 32u + uint32_t(h * 16), r16);
        tmem_ld_wait();
        tmem_regs_ready(r);
        tmem_regs_ready(r16);
#pragma unroll
        for (int e = 0; e < 32; ++e) z[e] = __uint_as_float(r[e]);
#pragma unroll
        for (int e = 0; e < 16; ++e) gz[e] = __uint_as_float(r16[e]);
      } else {
        uint32_t r[16], r8[8];
        tmem_ld16_nowait(tmem + lane_off + uint32_t(j) * 64u + uint32_t(h * 16), r);
        tmem_ld8_nowait(tmem + lane_off + 128u + uint32_t(j) * 32u + uint32_t(h * 8), r8);
        tmem_ld_wait();
        tmem_regs_ready(r);
        tmem_regs_ready(r8);
#pragma unroll
        for (int e = 0; e < 16; ++e) z[e] = __uint_as_float(r[e]);
#pragma unroll
        for (int e = 16; e < 32; ++e) z[e] = 0.f;
#pragma unroll
        for (int e = 0; e < 8; ++e) gz[e] = __uint_as_float(r8[e]);
#pragma unroll
        for (int e = 8; e < 16; ++e) gz[e] = 0.f;
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&ctl->d1_empty[j]));
      mbar_arrive(smem_u32(&ctl->d2_empty[j]));
      // dZ = Z / |Z| * d|Z| (0 where |Z| = 0), K index 2 r + (re, im) of the chunk.
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const float m2 = z[2 * e] * z[2 * e] + z[2 * e + 1] * z[2 * e + 1];
        const float sc = m2 > 0.f ? gz[e] * rsqrtf(m2) : 0.f;
        z[2 * e] *= sc;
        z[2 * e + 1] *= sc;
      }
      // dZ into A3 buffer i % NA3 once GEMM3 has read chunk w = i - NA3, the last chunk that used it.
      // a2_empty[w & 1] completes its phase (w >> 1) when GEMM3 has read chunk w.  This group has already
      // seen chunk w - 2 read (its previous wait), and chunk w + 2 cannot have been written yet, so the
      // phase parity names chunk w without ambiguity.  (Waiting on one barrier for the shared buffer's
      // last use would not: with NA3 = 1 its parity is the same after chunk i - 1 and after chunk i - 3.)
      const int ja = i % NA3, w = i - NA3;
      if (w >= 0 && !wait_warp(smem_u32(&ctl->a2_empty[w & 1]), (w >> 1) & 1, abort)) { ok = false; break; }
      tc_fence_after();
      // Row r = h rc / 2 + e of the chunk is word r of the A3 buffer: hi at + r, lo at + 32 + r.
      const uint32_t a3 = tmem + lane_off + kA3 + uint32_t(ja) * 64u;
      if (ch.rc == 32) {
        uint32_t hi[16], lo[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) split2(z[2 * e], z[2 * e + 1], hi[e], lo[e]);
        tmem_st16(a3 + uint32_t(16 * h), hi);
        tmem_st16(a3 + 32u + uint32_t(16 * h), lo);
      } else {
        uint32_t hi[8], lo[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) split2(z[2 * e], z[2 * e + 1], hi[e], lo[e]);
        tmem_st8(a3 + uint32_t(8 * h), hi);
        tmem_st8(a3 + 32u + uint32_t(8 * h), lo);
      }
      tmem_st_wait();
      tc_fence_before();
      mbar_arrive(smem_u32(&ctl->a2_full[ja]));
    }
    if (g == 0 && ok && wait_warp(smem_u32(&ctl->d3_full), 0, abort)) {
      tc_fence_after();
      // D3 columns (n, re/im): this half holds n in [h k1pad / 4, (h + 1) k1pad / 4).
      const int64_t ybase = int64_t(tl.b) * A.y2_tot + A.y2_off[tl.a] + tl.t0 + c;
      const int ncol = k1pad >> 1;
      for (int b8 = 0; b8 < ncol; b8 += 8) {
        uint32_t r[8];
        tmem_ld8_nowait(tmem + lane_off + kD3 + uint32_t(h * ncol + b8), r);
        tmem_ld_wait();
        tmem_regs_ready(r);
        const int n0 = (h * ncol + b8) >> 1;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int n = n0 + e;
          if (colok && n < n1m)
            A.dY2[ybase + int64_t(n) * L2] = make_float2(__uint_as_float(r[2 * e]), __uint_as_float(r[2 * e + 1]));
        }
      }
    }
  }

  if (warp == kWarpTma && lane == 0 && *abort) {
    for (int t = max(0, n1 - S1); t < n1; ++t) mbar_wait_drain(smem_u32(&ctl->b1_full[t % S1]), (t / S1) & 1);
    for (int t = max(0, n2 - kS2); t < n2; ++t) mbar_wait_drain(smem_u32(&ctl->b2_full[t % kS2]), (t / kS2) & 1);
    for (int t = max(0, n3 - S3); t < n3; ++t) mbar_wait_drain(smem_u32(&ctl->b3_full[t % S3]), (t / S3) & 1);
  }
  if (warp >= kWarpG1 && warp <= kWarpG3 && lane == 0 && issued) {
    const uint32_t dr = smem_u32(&ctl->drain[warp - kWarpG1]);
    umma_commit(dr);
    mbar_wait_drain(dr, 0);
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort) atomicExch(&g_tc_err, 1);
  if (warp == kWarpG1) {
    __syncwarp();
    tmem_dealloc(tmem, 512);
  }
}

}  // namespace
}  // namespace jtfs

// ===========================================================================
// Host side: operand tables, tiles, tensor maps, launchers.
// ===========================================================================
namespace jtfs {
namespace {

uint16_t bf16_rn(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return static_cast<uint16_t>(u >> 16);  // inf / nan unchanged
  u += 0x7fffu + ((u >> 16) & 1u);
  return static_cast<uint16_t>(u >> 16);
}
float bf16_f(uint16_t h) {
  const uint32_t u = uint32_t(h) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
// v = hi + lo to ~2^-18 relative (both BF16, round to nearest even).
void split_bf16(double v, uint16_t& hi, uint16_t& lo) {
  hi = bf16_rn(static_cast<float>(v));
  lo = bf16_rn(static_cast<float>(v - double(bf16_f(hi))));
}

constexpr int kFwdS1[2] = {4, 8};  // n1max <= 32: two CTAs per SM
constexpr int kFwdS1Wide[4] = {8, 9, 8, 10};  // table ring stages for KA = 2 .. 5 (>= 2 chunks of KA atoms)
constexpr int kTcMaxKA = 5;
constexpr int kTcWideMinTiles = 148;  // tiles (one per SM) a group with KA >= 3 needs to take the tensor cores
constexpr int kAdjS1[2] = {6, 6}, kAdjS3[2] = {4, 2}, kAdjNA3[2] = {2, 1};

PFN_cuTensorMapEncodeTiled_v12000 tc_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      ptr = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }();
  return fn;
}

// 2-D BF16 table [rows][cols] (row-major), boxes of box_rows x 64 columns, 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* base, uint64_t cols, uint64_t rows, uint32_t box_rows) {
  auto fn = tc_encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(base) & 15u) || (cols * 2) % 16) return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * 2};
  const cuuint32_t box[2] = {64, box_rows};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

TcArgs tc_args(const Plan& p) {
  TcArgs A{};
  A.chunks = p.d_tc_chunks;
  A.n_chunks = static_cast<int>(p.tc_chunks.size());
  A.n1max_act = p.d_n1max_act;
  A.s2 = p.d_s2;
  A.y2_off = p.d_y2_off;
  A.v2_off = p.d_v2_off;
  A.y2_tot = p.y2_tot;
  A.v2_tot = p.v2_tot;
  A.logN = p.logN;
  A.RO = p.R_out;
  A.nr1 = p.tc_nr1;
  return A;
}

template <auto Kernel>
cudaError_t tc_opt_in(size_t smem) {
  static const cudaError_t e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    static_cast<int>(smem));
  return e;
}

}  // namespace

void tc_build(Plan& p) {
  p.tc_ok = false;
  p.tc_chunks.clear();
  for (auto& t : p.tc_tiles) t.clear();
  p.tc_b1.clear();
  p.tc_b2.clear();
  p.tc_b2t.clear();
  p.tc_b3.clear();
  p.tiles2_fft = p.tiles2_fft_f = p.tiles2;
  p.tiles2w_fft = p.tiles2w_fft_f = p.tiles2w;
  const int RO = p.R_out, NF = p.N_fr;
  if (p.n_active == 0 || (RO != 16 && RO != 32) || NF < 64 || NF > 1024) return;
  if (p.unpooled_f) return;  // the GEMM tables include the phi_F averaging
  // K atoms of A1 per group: the forward takes n1max <= 160 (KA <= 5), the adjoint n1max <= 64 (KA <= 2:
  // its D3 of 2 n1max TMEM columns and the rest leave no room for more).
  std::vector<int> ka(p.n_active, 0);
  int ka_max = 0;
  for (int a = 0; a < p.n_active; ++a) {
    const int n1 = p.n1max[p.active[a]];
    const int64_t L2 = p.N >> p.s2[a];
    ka[a] = L2 < kTcM || n1 > 32 * kTcMaxKA ? 0 : (n1 + 31) / 32;
    // A wide group runs 3-5x the MMAs per tile of a KA = 1 group; with fewer tiles than SMs its few long
    // CTAs are slower than the FFT kernels' many short ones (measured on the 8 x 2^16 chirp plan).
    if (ka[a] >= 3 && int64_t(p.batch) * L2 < int64_t(kTcWideMinTiles) * kTcM) ka[a] = 0;
    ka_max = std::max(ka_max, ka[a]);
  }
  if (!ka_max) return;
  auto ka_adj = [&](int a) { return ka[a] <= 2 ? ka[a] : 0; };

  // Chunks of up to 32 rows per filter, in filter order.
  std::vector<int> rowP(p.lF + 2, 0);
  for (int k = 0; k <= p.lF; ++k) rowP[k + 1] = rowP[k] + (NF >> k);
  std::vector<int> rowB(p.n_beta2, 0);
  int nr = 0;
  for (int b = 0; b < p.n_beta2; ++b) {
    const int k = p.beta_k[b], R = NF >> k, rc = std::min(R, 32);
    rowB[b] = nr;
    for (int r0 = 0; r0 < R; r0 += rc)
      p.tc_chunks.push_back({b, k, r0, rc, 2 * (nr + r0), rowP[k] + r0, r0 == 0 ? 1 : 0, r0 + rc == R ? 1 : 0});
    nr += R;
  }
  const int nr1 = 2 * nr;
  p.tc_nr1 = nr1;

  // Impulse responses h_beta[t] = (1/N_fr) sum_{sb in band} g_beta[sb] e^{2 pi i sb t / N_fr}, from the same
  // band-limited tables the FFT kernels fold.
  const double two_pi = 2.0 * M_PI;
  std::vector<double> hr(size_t(p.n_beta2) * NF), hi(size_t(p.n_beta2) * NF);
  for (int b = 0; b < p.n_beta2; ++b) {
    const FiltD& f = p.h_beta[b];
    const float* g = p.h_ftabc.data() + p.h_ftabc_off[b];
    for (int t = 0; t < NF; ++t) {
      double sr = 0.0, si = 0.0;
      for (int sb = f.lo; sb <= f.hi; ++sb) {
        const double w = two_pi * double((int64_t(sb) * t) % NF) / double(NF);
        sr += double(g[sb - f.lo]) * std::cos(w);
        si += double(g[sb - f.lo]) * std::sin(w);
      }
      hr[size_t(b) * NF + t] = sr / NF;
      hi[size_t(b) * NF + t] = si / NF;
    }
  }
  // GEMM1 table B1 [(beta, r, re/im)][(n, re/im)], n < W1 / 2: [Zr, Zi] = Yr [Hr, Hi] + Yi [-Hi, Hr].
  const int W1 = 64 * std::max(2, ka_max);
  p.tc_w1 = W1;
  p.tc_b1.assign(size_t(2) * nr1 * W1, 0);
  p.tc_b3.assign(size_t(256) * nr1, 0);
  for (int b = 0; b < p.n_beta2; ++b) {
    const int k = p.beta_k[b], R = NF >> k;
    for (int r = 0; r < R; ++r)
      for (int n = 0; n < W1 / 2; ++n) {
        const int t = (((r << k) - n) % NF + NF) % NF;
        const double vr = hr[size_t(b) * NF + t], vi = hi[size_t(b) * NF + t];
        const int row = 2 * (rowB[b] + r);
        const double v[2][2] = {{vr, -vi}, {vi, vr}};  // [x = re/im of Z][y = re/im of Y]
        for (int x = 0; x < 2; ++x)
          for (int y = 0; y < 2; ++y) {
            uint16_t h16, l16;
            split_bf16(v[x][y], h16, l16);
            const int rr = row + x, cc = 2 * n + y;
            p.tc_b1[size_t(rr) * W1 + cc] = h16;
            p.tc_b1[size_t(nr1 + rr) * W1 + cc] = l16;
            if (n < 64) {
              p.tc_b3[size_t(cc) * nr1 + rr] = h16;          // transposed: rows (n, y), columns (r, x)
              p.tc_b3[size_t(128 + cc) * nr1 + rr] = l16;
            }
          }
      }
  }
  // phi_F averaging P_k[ro][r] = (1/R) sum_{sb in band} phi[sb] cos(2 pi sb (ro D - r) / R), D = R / R_out.
  p.tc_kp2 = 64 * (NF / 32);
  p.tc_np2 = rowP[p.lF + 1];
  p.tc_b2.assign(size_t(p.lF + 1) * RO * p.tc_kp2, 0);
  p.tc_b2t.assign(size_t(p.tc_np2) * 64, 0);
  const float* phi = p.h_ftabc.data() + p.ftabc_phi;
  for (int k = 0; k <= p.lF; ++k) {
    const int R = NF >> k, D = R / RO;
    for (int ro = 0; ro < RO; ++ro)
      for (int r = 0; r < R; ++r) {
        const int64_t t = ((int64_t(ro) * D - r) % R + R) % R;
        double acc = 0.0;
        for (int sb = p.h_phiF.lo; sb <= p.h_phiF.hi; ++sb)
          acc += double(phi[sb - p.h_phiF.lo]) * std::cos(two_pi * double(((int64_t(sb) * t) % R + R) % R) / R);
        acc /= R;
        uint16_t h16, l16;
        split_bf16(acc, h16, l16);
        const size_t frow = size_t(k * RO + ro) * p.tc_kp2 + 64 * (r >> 5) + (r & 31);
        p.tc_b2[frow] = h16;
        p.tc_b2[frow + 32] = l16;
        const size_t arow = size_t(rowP[k] + r) * 64 + ro;
        p.tc_b2t[arow] = h16;
        p.tc_b2t[arow + 32] = l16;
      }
  }
  // Tiles of 128 columns for the tensor-core groups; the FFT kernels keep the others.
  p.tiles2_fft.clear();
  p.tiles2w_fft.clear();
  p.tiles2_fft_f.clear();
  p.tiles2w_fft_f.clear();
  for (const Tile& t : p.tiles2) {
    if (!ka_adj(t.a)) p.tiles2_fft.push_back(t);
    if (!ka[t.a]) p.tiles2_fft_f.push_back(t);
  }
  for (const Tile& t : p.tiles2w) {
    if (!ka_adj(t.a)) p.tiles2w_fft.push_back(t);
    if (!ka[t.a]) p.tiles2w_fft_f.push_back(t);
  }
  for (int b = 0; b < p.batch; ++b)
    for (int a = 0; a < p.n_active; ++a) {
      if (!ka[a]) continue;
      const int L2 = static_cast<int>(p.N >> p.s2[a]);
      for (int t0 = 0; t0 < L2; t0 += kTcM) p.tc_tiles[ka[a] - 1].push_back({b, a, t0, std::min(kTcM, L2 - t0)});
    }
  p.tc_ok = true;
}

int tc_upload(Plan& p) {
  if (!p.tc_ok) return JTFS_OK;
  struct Part { const void* src; size_t bytes; size_t off; };
  std::vector<Part> parts;
  size_t total = 0;
  auto put = [&](const void* src, size_t bytes) {
    const size_t off = total;
    parts.push_back({src, bytes, off});
    total = (total + std::max<size_t>(bytes, 1) + 1023) & ~size_t(1023);
    return off;
  };
  const size_t o_b1 = put(p.tc_b1.data(), p.tc_b1.size() * 2);
  const size_t o_b2 = put(p.tc_b2.data(), p.tc_b2.size() * 2);
  const size_t o_b2t = put(p.tc_b2t.data(), p.tc_b2t.size() * 2);
  const size_t o_b3 = put(p.tc_b3.data(), p.tc_b3.size() * 2);
  const size_t o_ch = put(p.tc_chunks.data(), p.tc_chunks.size() * sizeof(TcChunk));
  size_t o_t[5];
  for (int k = 0; k < 5; ++k) o_t[k] = put(p.tc_tiles[k].data(), p.tc_tiles[k].size() * sizeof(Tile));
  const size_t o_f = put(p.tiles2_fft.data(), p.tiles2_fft.size() * sizeof(Tile));
  const size_t o_fw = put(p.tiles2w_fft.data(), p.tiles2w_fft.size() * sizeof(Tile));
  const size_t o_ff = put(p.tiles2_fft_f.data(), p.tiles2_fft_f.size() * sizeof(Tile));
  const size_t o_ffw = put(p.tiles2w_fft_f.data(), p.tiles2w_fft_f.size() * sizeof(Tile));
  void* blob = nullptr;
  if (cudaMalloc(&blob, total) != cudaSuccess) return JTFS_ERR_NOMEM;
  std::vector<unsigned char> host(total, 0);
  for (auto& pt : parts)
    if (pt.bytes) std::memcpy(host.data() + pt.off, pt.src, pt.bytes);
  if (cudaMemcpy(blob, host.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(blob);
    return JTFS_ERR_CUDA;
  }
  unsigned char* at = static_cast<unsigned char*>(blob);
  p.d_tc = blob;
  p.d_tc_chunks = reinterpret_cast<const TcChunk*>(at + o_ch);
  for (int k = 0; k < 5; ++k) p.d_tc_tiles[k] = reinterpret_cast<const Tile*>(at + o_t[k]);
  p.d_tiles2_fft = reinterpret_cast<const Tile*>(at + o_f);
  p.d_tiles2w_fft = reinterpret_cast<const Tile*>(at + o_fw);
  p.d_tiles2_fft_f = reinterpret_cast<const Tile*>(at + o_ff);
  p.d_tiles2w_fft_f = reinterpret_cast<const Tile*>(at + o_ffw);
  const bool ok = make_map(&p.tc_map[0], at + o_b1, uint64_t(p.tc_w1), uint64_t(2) * p.tc_nr1, 64) &&
                  make_map(&p.tc_map[1], at + o_b2, p.tc_kp2, uint64_t(p.lF + 1) * p.R_out, p.R_out) &&
                  make_map(&p.tc_map[2], at + o_b2t, 64, p.tc_np2, 32) &&
                  make_map(&p.tc_map[3], at + o_b3, p.tc_nr1, 256, 64);
  if (!ok) {
    // No tensor maps (driver without the entry point): keep the FFT kernels for every group.
    cudaFree(blob);
    p.d_tc = nullptr;
    p.tc_ok = false;
    p.tiles2_fft = p.tiles2_fft_f = p.tiles2;
    p.tiles2w_fft = p.tiles2w_fft_f = p.tiles2w;
  }
  return JTFS_OK;
}

void tc_release(Plan& p) {
  if (p.d_tc) cudaFree(p.d_tc);
  p.d_tc = nullptr;
}

bool tc_has_groups(const Plan& p, int which) { return p.tc_ok && p.tune_tc && !p.tc_tiles[which].empty(); }

// Forward tiles of the groups with KA > 1 (one CTA per SM, two epilogue groups, 512 TMEM columns).
template <int KA>
int launch_fwd_wide(const Plan& p, TcArgs A, cudaStream_t s) {
  if (p.tc_tiles[KA - 1].empty()) return JTFS_OK;
  constexpr int S1 = kFwdS1Wide[KA - 2];
  constexpr size_t smem = tc_fwd_smem<KA, S1>();
  static_assert(smem + 1024 <= 227 * 1024 && S1 <= 16 && fwd_a1_col<KA>() + 64 * KA <= 512, "forward budget");
  if (tc_opt_in<k_freq_tc_fwd<KA, S1, 2>>(smem) != cudaSuccess) return JTFS_ERR_CUDA;
  A.tiles = p.d_tc_tiles[KA - 1];
  k_freq_tc_fwd<KA, S1, 2><<<static_cast<unsigned>(p.tc_tiles[KA - 1].size()), tc_fwd_threads<2>(), smem, s>>>(
      p.tc_map[0], p.tc_map[1], A);
  return cudaGetLastError() == cudaSuccess ? JTFS_OK : JTFS_ERR_CUDA;
}

int tc_forward(const Plan& p, const float2* Y2, float* V2, cudaStream_t s, cudaStream_t s2) {
  if (!p.tc_ok || !p.tune_tc) return JTFS_OK;
  TcArgs A = tc_args(p);
  A.Y2 = Y2;
  A.V2 = V2;
  if (!p.tc_tiles[0].empty()) {
    constexpr size_t smem = tc_fwd_smem<1, kFwdS1[0]>();
    static_assert(2 * (smem + 1024) <= 228 * 1024, "two forward CTAs per SM");
    if (tc_opt_in<k_freq_tc_fwd<1, kFwdS1[0], 1>>(smem) != cudaSuccess) return JTFS_ERR_CUDA;
    A.tiles = p.d_tc_tiles[0];
    k_freq_tc_fwd<1, kFwdS1[0], 1><<<static_cast<unsigned>(p.tc_tiles[0].size()), tc_fwd_threads<1>(), smem, s>>>(
        p.tc_map[0], p.tc_map[1], A);
    if (cudaGetLastError() != cudaSuccess) return JTFS_ERR_CUDA;
  }
  // The wider groups, one after another on s2.
  int rc = JTFS_OK;
  if (rc == JTFS_OK) rc = launch_fwd_wide<2>(p, A, s2);
  if (rc == JTFS_OK) rc = launch_fwd_wide<3>(p, A, s2);
  if (rc == JTFS_OK) rc = launch_fwd_wide<4>(p, A, s2);
  if (rc == JTFS_OK) rc = launch_fwd_wide<5>(p, A, s2);
  return rc;
}

int tc_adjoint(const Plan& p, const float2* Y2, const float* dV2, float2* dY2, cudaStream_t s, cudaStream_t s2) {
  if (!p.tc_ok || !p.tune_tc) return JTFS_OK;
  TcArgs A = tc_args(p);
  A.Y2 = Y2;
  A.dV2 = dV2;
  A.dY2 = dY2;
  if (!p.tc_tiles[0].empty()) {
    constexpr size_t smem = tc_adj_smem<1, kAdjS1[0], kAdjS3[0]>();
    if (tc_opt_in<k_freq_tc_adj<1, kAdjS1[0], kAdjS3[0], kAdjNA3[0]>>(smem) != cudaSuccess) return JTFS_ERR_CUDA;
    A.tiles = p.d_tc_tiles[0];
    k_freq_tc_adj<1, kAdjS1[0], kAdjS3[0], kAdjNA3[0]>
        <<<static_cast<unsigned>(p.tc_tiles[0].size()), kTcAdjThreads, smem, s>>>(p.tc_map[0], p.tc_map[2],
                                                                               p.tc_map[3], A);
    if (cudaGetLastError() != cudaSuccess) return JTFS_ERR_CUDA;
  }
  if (!p.tc_tiles[1].empty()) {
    constexpr size_t smem = tc_adj_smem<2, kAdjS1[1], kAdjS3[1]>();
    if (tc_opt_in<k_freq_tc_adj<2, kAdjS1[1], kAdjS3[1], kAdjNA3[1]>>(smem) != cudaSuccess) return JTFS_ERR_CUDA;
    A.tiles = p.d_tc_tiles[1];
    k_freq_tc_adj<2, kAdjS1[1], kAdjS3[1], kAdjNA3[1]>
        <<<static_cast<unsigned>(p.tc_tiles[1].size()), kTcAdjThreads, smem, s2>>>(p.tc_map[0], p.tc_map[2],
                                                                               p.tc_map[3], A);
    if (cudaGetLastError() != cudaSuccess) return JTFS_ERR_CUDA;
  }
  return JTFS_OK;
}

}  // namespace jtfs

// ---------------------------------------------------------------------------
// C ABI (include/jtfs.h).
// ---------------------------------------------------------------------------
extern "C" int jtfs_tc_error(void) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, jtfs::g_tc_err, sizeof(int)) != cudaSuccess) return JTFS_ERR_CUDA;
  const int zero[4] = {0, 0, 0, 0};
  if (v && cudaMemcpyToSymbol(jtfs::g_tc_err, zero, sizeof(int)) != cudaSuccess) return JTFS_ERR_CUDA;
  const int vp = jtfs::pool_tc_error();
  if (vp < 0) return vp;
  return v | vp;
}

namespace jtfs {
int set_wait_polls_freq(int64_t polls) {
  const uint32_t v = polls < 0 ? kSpinLimit : static_cast<uint32_t>(polls < int64_t(kSpinLimit) ? polls : kSpinLimit);
  return cudaMemcpyToSymbol(c_wait_polls, &v, sizeof(v)) == cudaSuccess ? JTFS_OK : JTFS_ERR_CUDA;
}
}  // namespace jtfs

extern "C" int jtfs_tc_error_info(int64_t* info, int n) {
  int v[4];
  if (cudaMemcpyFromSymbol(v, jtfs::g_tc_err_info, sizeof(v)) != cudaSuccess) return JTFS_ERR_CUDA;
  for (int i = 0; i < n && i < 4 && info; ++i) info[i] = i == 0 ? int64_t(v[0]) - 1 : v[i];
  const int zero[4] = {0, 0, 0, 0};
  if (cudaMemcpyToSymbol(jtfs::g_tc_err_info, zero, sizeof(zero)) != cudaSuccess) return JTFS_ERR_CUDA;
  return 4;
}

extern "C" int64_t jtfs_tc_table(jtfs_plan_t plan, int which, float* out, int64_t n) {
  if (!plan || (which != 0 && which != 1) || n < 0) return JTFS_ERR_ARG;
  const jtfs::Plan& p = plan->p;
  if (p.tc_b1.empty()) return JTFS_ERR_SHAPE;
  auto f = [](uint16_t h) {
    const uint32_t u = uint32_t(h) << 16;
    float v;
    std::memcpy(&v, &u, 4);
    return v;
  };
  if (which == 0) {  // the first 128 columns (n < 64) of each row of the GEMM1 table
    const int64_t total = int64_t(p.tc_nr1) * 128, W1 = p.tc_w1, half = int64_t(p.tc_nr1) * W1;
    for (int64_t i = 0; out && i < std::min(n, total); ++i) {
      const int64_t o = (i / 128) * W1 + i % 128;
      out[i] = f(p.tc_b1[size_t(o)]) + f(p.tc_b1[size_t(half + o)]);
    }
    return total;
  }
  const int RO = p.R_out, NF = p.N_fr;
  const int64_t total = int64_t(p.lF + 1) * RO * NF;
  for (int64_t i = 0; out && i < std::min(n, total); ++i) {
    const int r = int(i % NF), ro = int((i / NF) % RO), k = int(i / (int64_t(NF) * RO));
    float v = 0.f;
    if (r < (NF >> k)) {
      const size_t o = size_t(k * RO + ro) * p.tc_kp2 + 64 * (r >> 5) + (r & 31);
      v = f(p.tc_b2[o]) + f(p.tc_b2[o + 32]);
    }
    out[i] = v;
  }
  return total;
}
