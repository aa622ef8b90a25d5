// Time averaging of the second-order paths on the 5th-generation tensor cores
// (the phi_T average of Eq. (5), at stride T).
//
// For one clip and one path group (n2) of level s (rows at stride 2^s, L =
// N / 2^s samples), every pooled row is
//   Phi2[r][f] = sum_t V2[r][t] g_s[(f D - t) mod L],   D = 2^(log2 T - s),
// with g_s the phi_T taps at level s.  All rows share the tap matrix
// G[f][t] = g_s[(f D - t) mod L], so a tile of 128 rows is the GEMM
//   D[128 x F] = V[128 x K] . G^T[K x F]         (F = N / T frames, K = time)
// over a split of the time axis, written as partial sums into the slots of the
// fixed-order reduction (k_pool_reduce) that the FMA kernels also use.
// FP32 accuracy from BF16 operands: each operand is split v = hi + lo and each
// product is hi.hi + lo.hi + hi.lo (three MMAs into one FP32 accumulator).
//
// One CTA per (clip, group, 128 rows, time split), 288 threads: warps 0-7 turn
// 64-sample blocks of V2 (a half-warp per row and load, 4 samples a thread, the
// next block's loads in flight while the current one is converted) and of the taps
// into BF16 hi/lo operand tiles (128-byte swizzle, two shared-memory stages)
// and then read the accumulator (warp w: TMEM lanes 32 (w % 4) .. + 31, half
// w / 4 of the frames); warp 8 lane 0 issues tcgen05.mma.
// Every wait is bounded: an expired wait stops the CTA (MMAs completed, TMEM
// freed) and raises a flag read through jtfs_tc_error().
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "jtfs.h"
#include "jtfs_internal.h"
#include "jtfs_umma.cuh"

namespace jtfs {
namespace {

__device__ int g_pt_err;

constexpr int kPtThreads = 288;
constexpr int kPtProd = 256;  // producer / epilogue threads (warps 0-7)
constexpr int kPtWarpMma = 8;
constexpr int kPtRows = 128;  // rows per tile (MMA M)
constexpr int kPtK = 64;      // samples per operand block (one 128-byte swizzle atom of BF16)
static_assert(kPtProd == 2 * kPtRows, "two producer threads per tile row");

struct PtArgs {
  const float* V2;
  float* part;
  const int4* tiles;      // (clip, active group, first 64-row slot, split) or, banded, (..., 32-frame block)
  const int* tile0;       // first partial slot of each (clip, group)
  const int* s2;
  const int64_t* v2_off;
  const float* taps;
  const int64_t* tap_off;
  int64_t v2_tot;
  int logN, lT, n_frames, rows, n_active, split_len;
  // Banded groups: reach of phi_T's taps per group, and Phi written directly.
  const int* pool_w;
  const int* band_S;      // banded adjoint: samples per CTA of each active group
  float* phi;
  int64_t phi_size;
  const int64_t* phi2_off;
};

struct PtCtl {
  unsigned long long full[2], empty[2], done, sub_full[2], sub_empty[2];
  uint32_t tmem;
  int abort;
};

// Banded windows are accumulated in sub-windows of kPtSubK blocks (4096 samples), alternating between two
// TMEM accumulators; the producer warps add each finished sub-window into FP32 registers.  One FP32
// accumulator taking tens of thousands of MMAs drifts (3.7e-4 relative on a 2.2e5-sample window); sums of
// at most 4096 samples stay within the dense path's bound.
constexpr int kPtSubK = 64;

__device__ __forceinline__ bool pt_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  const uint32_t polls = c_wait_polls;
  for (uint32_t i = 0; i < polls; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    if (i >= 8) __nanosleep(64);
  }
  *abort = 1;
  return false;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, const uint32_t (&v)[4]) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
               : "memory");
}

__device__ __forceinline__ float ld_shared_f32(uint32_t addr) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void st_shared_f32(uint32_t addr, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ float4 ld_shared_v4f(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr)
               : "memory");
  return v;
}
__device__ __forceinline__ void st_shared_v2(uint32_t addr, const uint32_t (&v)[2]) {
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(v[0]), "r"(v[1]) : "memory");
}

// Banded tiles with long windows (SUBW) add the producers' running sums of finished sub-windows: 16 floats
// per producer thread.
template <int F, bool SUBW = false>
constexpr size_t pt_smem() {
  return sizeof(PtCtl) + 1024 + 2 * (2 * 16384 + 2 * size_t(F) * 128) + (SUBW ? size_t(kPtProd) * 16 * 4 : 0);
}

// BAND: a group where phi_T's reach is short against the circle; the CTA
// computes 32 frames f0 .. f0 + 31 of 128 rows from the samples within reach
// only (t from f0 D - W to (f0 + 31) D + W, widened to whole 64-sample blocks;
// the extra samples enter with their own exact taps), read circularly, and
// writes Phi directly (no split, no reduction); windows longer than kPtSubK
// blocks are summed sub-window by sub-window.
template <int F, bool BAND = false, bool SUBW = false>
__global__ void __launch_bounds__(kPtThreads, 2)
k_pool_tc_fwd(const PtArgs A) {
  extern __shared__ uint8_t smem_raw[];
  PtCtl* ctl = reinterpret_cast<PtCtl*>(smem_raw);
  constexpr uint32_t kA = 16384u, kB = uint32_t(F) * 128u, kStage = 2 * kA + 2 * kB;
  const uint32_t base = (smem_u32(smem_raw) + sizeof(PtCtl) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  const int4 tl = A.tiles[blockIdx.x];
  const int b = tl.x, a = tl.y, slot = tl.z, sp = tl.w;
  const int s = A.s2[a], lL = A.logN - s, L = 1 << lL, D = 1 << (A.lT - s);
  const int f0 = BAND ? sp * 32 : 0;   // first frame of the tile
  int tbeg, tend;
  if (BAND) {
    const int W = A.pool_w[a];
    tbeg = ((f0 * D - W) >> 6) << 6;                          // floor to a 64-sample block
    tend = ((((f0 + 31) * D + W + 1) + 63) >> 6) << 6;
  } else {
    tbeg = sp * A.split_len;
    tend = min(L, tbeg + A.split_len);
  }
  const int nkb = (tend - tbeg + kPtK - 1) / kPtK;
  // Banded: blocks per sub-window (a window of up to kPtSubK + 2 blocks stays one sub-window; without
  // SUBW every window is one, which the host allows only when none is longer).
  const int subk = SUBW && nkb > kPtSubK + 2 ? kPtSubK : max(nkb, 1);
  const int nsplit = BAND ? 1 : (L + A.split_len - 1) / A.split_len;
  const int r0 = slot * 64;
  volatile int* abort = &ctl->abort;
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&ctl->full[i]), kPtProd);
      mbar_init(smem_u32(&ctl->empty[i]), 1);
    }
    mbar_init(smem_u32(&ctl->done), 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&ctl->sub_full[i]), 1);
      mbar_init(smem_u32(&ctl->sub_empty[i]), kPtProd);
    }
    ctl->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  constexpr uint32_t kCols = SUBW ? 2 * F : (F < 32 ? 32 : F);
  if (warp == kPtWarpMma) tmem_alloc(smem_u32(&ctl->tmem), kCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem;
  bool issued = false;
  // Banded: warp w's share of the finished sub-windows (rows 32 (w % 4) + lane, frames w / 4 * F / 2 ..),
  // summed in this thread's shared-memory slots (element e at word e * kPtProd + tid).
  constexpr int FH = F / 2;
  static_assert(!SUBW || (BAND && FH == 16), "sub-windows are for banded tiles of 32 frames");
  const uint32_t racc = base + 2u * kStage + uint32_t(tid) * 4u;
  int q_read = 0;  // sub-windows already added into racc
  auto add_sub = [&](int q) {  // warp-collective: sub-window q's accumulator into racc
    uint32_t v[16];
    tmem_ld16_nowait(tmem + (uint32_t((warp & 3) * 32) << 16) + uint32_t((q & 1) * F + (warp >> 2) * FH), v);
    tmem_ld_wait();
    tmem_regs_ready(v);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const uint32_t a4 = racc + uint32_t(e * kPtProd * 4);
      st_shared_f32(a4, (q == 0 ? 0.f : ld_shared_f32(a4)) + __uint_as_float(v[e]));
    }
  };

  if (warp < kPtWarpMma) {
    // Producer: half-warps run along the samples, so each load instruction of a warp reads two rows' 256
    // contiguous bytes.  Thread (warp w, lane l) takes samples 4 (l % 16) .. + 3 of the rows
    // 2 (w + 8 i) + l / 16, i = 0 .. 7, of every 64-sample block.
    const int c4 = lane & 15, sub = lane >> 4;
    const float* vbase = A.V2 + static_cast<int64_t>(b) * A.v2_tot + A.v2_off[a];
    const float* g = A.taps + A.tap_off[s];
    const bool vec = L >= kPtK;  // whole 64-sample blocks inside the row: 16-byte loads
    float4 nxt[8];
    const int rw = r0 + 2 * warp + sub;        // row of i = 0; row i is rw + 16 i
    const float* vrow0 = vbase + static_cast<int64_t>(rw) * L;
    auto load_v = [&](int t0) {
      const int t = t0 + 4 * c4;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = rw + 16 * i;
        const float* vrow = vrow0 + static_cast<int64_t>(16 * i) * L;
        if (r >= A.rows || t >= tend) {
          nxt[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        } else if (BAND) {   // whole 64-sample blocks, circular
          nxt[i] = __ldg(reinterpret_cast<const float4*>(vrow + (t & (L - 1))));
        } else if (vec) {
          nxt[i] = __ldg(reinterpret_cast<const float4*>(vrow + t));
        } else {
          nxt[i] = make_float4(vrow[t], t + 1 < tend ? vrow[t + 1] : 0.f, t + 2 < tend ? vrow[t + 2] : 0.f,
                               t + 3 < tend ? vrow[t + 3] : 0.f);
        }
      }
    };
    load_v(tbeg);
    for (int kb = 0; kb < nkb; ++kb) {
      const int st = kb & 1;
      const int t0 = tbeg + kb * kPtK;
      if (SUBW && kb % subk == 2 && kb > subk) {
        // Sub-window q - 1 is complete once its MMAs are (at most two blocks behind this producer).
        const int q = kb / subk - 1;
        const bool okw = __all_sync(0xffffffffu, pt_wait(smem_u32(&ctl->sub_full[q & 1]), (q >> 1) & 1, abort));
        if (!okw) break;
        tc_fence_after();
        add_sub(q);
        q_read = q + 1;
        tc_fence_before();
        mbar_arrive(smem_u32(&ctl->sub_empty[q & 1]));
      }
      float4 cur[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) cur[c] = nxt[c];
      if (kb + 1 < nkb) load_v(t0 + kPtK);
      if (kb >= 2 && !pt_wait(smem_u32(&ctl->empty[st]), ((kb >> 1) - 1) & 1, abort)) break;
      const uint32_t sA = base + uint32_t(st) * kStage, sAl = sA + kA, sB = sA + 2 * kA, sBl = sB + kB;
#pragma unroll
      for (int i = 0; i < 8; ++i) {  // 4 samples = the half of 16-byte chunk c4 / 2 selected by c4 % 2
        const int rr = 2 * (warp + 8 * i) + sub;
        const float4 p = cur[i];
        uint32_t hi[2], lo[2];
        split2(p.x, p.y, hi[0], lo[0]);
        split2(p.z, p.w, hi[1], lo[1]);
        const uint32_t off = swz128(rr, c4 >> 1) + 8u * uint32_t(c4 & 1);
        st_shared_v2(sA + off, hi);
        st_shared_v2(sAl + off, lo);
      }
      // Taps: row f, samples t0 .. t0 + 63 of G[f][t] = g[(f D - t) mod L] = g[(t - f D) mod L] (g is
      // even).  With D a multiple of 8 the 8 samples of a chunk are 8 consecutive, 32-byte aligned taps.
      for (int q = tid; q < F * 8; q += kPtProd) {
        const int f = q >> 3, ch = q & 7;
        const int tc = t0 + 8 * ch;
        float v[8];
        if (f0 + f >= A.n_frames) {
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = 0.f;
        } else if (D >= 8 && tc + 8 <= tend) {
          const float4* src = reinterpret_cast<const float4*>(g + ((tc - (f0 + f) * D) & (L - 1)));
          const float4 x = __ldg(src), y = __ldg(src + 1);
          v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
          v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = tc + e < tend ? __ldg(g + ((tc + e - (f0 + f) * D) & (L - 1))) : 0.f;
        }
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split2(v[2 * e], v[2 * e + 1], hi[e], lo[e]);
        st_shared_v4(sB + swz128(f, ch), hi);
        st_shared_v4(sBl + swz128(f, ch), lo);
      }
      fence_proxy_async();
      mbar_arrive(smem_u32(&ctl->full[st]));
    }
  } else if (warp == kPtWarpMma && lane == 0) {
    issued = true;
    const uint32_t idesc = idesc_bf16_n(F);
    for (int kb = 0; kb < nkb; ++kb) {
      const int st = kb & 1;
      const int q = SUBW ? kb / subk : 0;
      const bool first = SUBW ? kb % subk == 0 : kb == 0;
      // Accumulator q & 1 last held sub-window q - 2: the producers have read it.
      if (SUBW && first && q >= 2 && !pt_wait(smem_u32(&ctl->sub_empty[q & 1]), ((q - 2) >> 1) & 1, abort)) break;
      if (!pt_wait(smem_u32(&ctl->full[st]), (kb >> 1) & 1, abort)) break;
      tc_fence_after();
      const uint32_t sA = base + uint32_t(st) * kStage;
      const uint64_t ah = sdesc(sA, 16, 1024), al = sdesc(sA + kA, 16, 1024);
      const uint64_t bh = sdesc(sA + 2 * kA, 16, 1024), bl = sdesc(sA + 2 * kA + kB, 16, 1024);
      const uint32_t d = tmem + uint32_t((q & 1) * F);
#pragma unroll
      for (int kk = 0; kk < kPtK / 16; ++kk) {
        const uint64_t o = uint64_t(kk) * 2u;  // 32 bytes in 16-byte descriptor units
        umma_bf16(d, ah + o, bh + o, idesc, !(first && kk == 0));
        umma_bf16(d, al + o, bh + o, idesc, 1);
        umma_bf16(d, ah + o, bl + o, idesc, 1);
      }
      umma_commit(smem_u32(&ctl->empty[st]));
      if (SUBW && (kb % subk == subk - 1 || kb == nkb - 1)) umma_commit(smem_u32(&ctl->sub_full[q & 1]));
    }
    umma_commit(smem_u32(&ctl->done));  // completes once every issued MMA has completed
  }

  if (warp < kPtWarpMma) {
    const bool ok = pt_wait(smem_u32(&ctl->done), 0, abort);
    const bool all = __all_sync(0xffffffffu, ok) && !*abort;
    tc_fence_after();
    if (all) {
      // Warp w: rows 32 (w % 4) + lane of the tile (its TMEM lanes), frames [w / 4 * F / 2, + F / 2).
      const int q4 = warp & 3, fh = warp >> 2;
      const int r = r0 + 32 * q4 + lane;
      float4* out;
      if (BAND) {
        out = reinterpret_cast<float4*>(A.phi + static_cast<int64_t>(b) * A.phi_size + A.phi2_off[a] +
                                        static_cast<int64_t>(r) * A.n_frames + f0 + fh * FH);
      } else {
        const int64_t ba = static_cast<int64_t>(b) * A.n_active + a;
        const int64_t t = A.tile0[ba] + static_cast<int64_t>(r >> 6) * nsplit + sp;
        out = reinterpret_cast<float4*>(A.part + (t * 64 + (r & 63)) * A.n_frames + fh * FH);
      }
      const uint32_t taddr = tmem + (uint32_t(q4 * 32) << 16) + uint32_t(fh * FH);
      if (SUBW && subk < nkb) {
        // Every MMA has completed (done): add the sub-windows not yet read.
        const int nsub = (nkb + subk - 1) / subk;
        for (int q = q_read; q < nsub; ++q) add_sub(q);
        if (r < A.rows) {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            out[e] = make_float4(ld_shared_f32(racc + uint32_t((4 * e) * kPtProd * 4)),
                                 ld_shared_f32(racc + uint32_t((4 * e + 1) * kPtProd * 4)),
                                 ld_shared_f32(racc + uint32_t((4 * e + 2) * kPtProd * 4)),
                                 ld_shared_f32(racc + uint32_t((4 * e + 3) * kPtProd * 4)));
        }
      } else if (FH == 16) {
        uint32_t v[16];
        tmem_ld16_nowait(taddr, v);
        tmem_ld_wait();
        tmem_regs_ready(v);
        if (r < A.rows) {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            out[e] = make_float4(__uint_as_float(v[4 * e]), __uint_as_float(v[4 * e + 1]),
                                 __uint_as_float(v[4 * e + 2]), __uint_as_float(v[4 * e + 3]));
        }
      } else {
#pragma unroll
        for (int j = 0; j < FH / 32; ++j) {
          float v[32];
          tmem_ld32(taddr + uint32_t(32 * j), v);
          if (r < A.rows) {
#pragma unroll
            for (int e = 0; e < 8; ++e)
              out[8 * j + e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
          }
        }
      }
    }
  }
  if (warp == kPtWarpMma && lane == 0 && issued && *abort) {
    // The done commit above already covers every issued MMA; wait for it before freeing TMEM.
    for (uint32_t i = 0; i < kSpinLimit && !mbar_try_wait(smem_u32(&ctl->done), 0); ++i) __nanosleep(64);
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && *abort) atomicExch(&g_pt_err, 1);
  if (warp == kPtWarpMma) {
    __syncwarp();
    tmem_dealloc(tmem, kCols);
  }
}

// ---------------------------------------------------------------------------
// Adjoint: dV2[r][t] = sum_f dPhi2[r][f] G[f][t] for 128 rows and a block of
// kPtTb samples: D[128 x 128] = dPhi [128 x F] . G [F x 128] per 128-sample
// block (MMA N = 128), K = F frames.  Operand rows (K-major, 128-byte swizzle):
// F = 32 packs hi (K 0..31) and lo into one 128-byte row; F = 64, 128 use F / 64
// atoms of hi then as many of lo.  The dPhi tile is split once; each block's
// tap tile G^T[t][f] = g[(f D - t) mod L] is built by the same 8 warps, which
// then store the finished block (TMEM double-buffered, 2 x 128 columns).
// ---------------------------------------------------------------------------
constexpr int kPtTb = 1024;   // samples per adjoint CTA (8 blocks of 128)

struct PaCtl {
  unsigned long long a_full, b_full[2], d_full[2], d_empty[2], done;
  uint32_t tmem;
  int abort;
};

template <int F>
__host__ __device__ constexpr uint32_t pa_tile() { return F == 32 ? 16384u : uint32_t(F / 64) * 2u * 16384u; }  // 128 rows, hi + lo

// Tiles that store dV2 through the per-warp transposing tile (8 warps x 32 rows x 36 floats).
template <int F, bool BAND>
__host__ __device__ constexpr bool pa_staged() { return F == 32 || BAND; }
template <int F, bool BAND = false>
constexpr size_t pa_smem() {
  return sizeof(PaCtl) + 1024 + 3 * size_t(pa_tile<F>()) + (pa_staged<F, BAND>() ? 8 * 4608 : 0);
}

// Byte offsets of K-step kk (16 K) inside a hi + lo operand tile.
template <int F>
__device__ __forceinline__ uint32_t pa_hi(int kk) {
  return F == 32 ? uint32_t(kk) * 32u : uint32_t(kk >> 2) * 16384u + uint32_t(kk & 3) * 32u;
}
template <int F>
__device__ __forceinline__ uint32_t pa_lo(int kk) {
  return F == 32 ? 64u + uint32_t(kk) * 32u : uint32_t(F / 64) * 16384u + pa_hi<F>(kk);
}
// Shared-memory byte address of the 16-byte chunk holding K = 8 c .. 8 c + 7 of row `row`, hi or lo.
template <int F>
__device__ __forceinline__ uint32_t pa_chunk(uint32_t tile, int row, int c, bool lo) {
  if (F == 32) return tile + swz128(row, c + (lo ? 4 : 0));
  return tile + (lo ? uint32_t(F / 64) * 16384u : 0u) + uint32_t(c >> 3) * 16384u + swz128(row, c & 7);
}

// BAND: a group where phi_T's reach is short against the circle; the CTA covers band_S[a] samples from
// t0 (tile.w) and only the F frames fa .. fa + F - 1 (mod n_frames), fa = floor((t0 - W) / D), that
// can reach them (band_S is chosen so that every frame within reach is among them; the others enter
// with their exact taps).
template <int F, bool BAND = false>
__global__ void __launch_bounds__(kPtThreads)
k_pool_tc_adj(const PtArgs A, const float* __restrict__ dphi, int64_t phi_size, const int64_t* __restrict__ phi2_off,
              float* __restrict__ dV2) {
  extern __shared__ uint8_t smem_raw[];
  PaCtl* ctl = reinterpret_cast<PaCtl*>(smem_raw);
  constexpr uint32_t kT = pa_tile<F>();
  const uint32_t base = (smem_u32(smem_raw) + sizeof(PaCtl) + 1023u) & ~1023u;
  const uint32_t sA = base, sB0 = base + kT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  const int4 tl = A.tiles[blockIdx.x];  // (clip, active group, first 64-row slot, block of kPtTb samples or t0)
  const int b = tl.x, a = tl.y, r0 = tl.z * 64, tb0 = BAND ? tl.w : tl.w * kPtTb;
  const int s = A.s2[a], L = 1 << (A.logN - s), D = 1 << (A.lT - s);
  const int nblk = (min(L - tb0, BAND ? A.band_S[a] : kPtTb) + 127) / 128;
  // First frame of the K range: 0, or for banded tiles floor((t0 - W) / D) (t0 - W may be negative).
  const int fa = BAND ? -((A.pool_w[a] - tb0 + D - 1) >> (A.lT - s)) : 0;
  volatile int* abort = &ctl->abort;
  if (tid == 0) {
    mbar_init(smem_u32(&ctl->a_full), kPtProd);
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&ctl->b_full[i]), kPtProd);
      mbar_init(smem_u32(&ctl->d_full[i]), 1);
      mbar_init(smem_u32(&ctl->d_empty[i]), kPtProd);
    }
    mbar_init(smem_u32(&ctl->done), 1);
    ctl->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kPtWarpMma) tmem_alloc(smem_u32(&ctl->tmem), 256);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem;
  bool issued = false;

  if (warp < kPtWarpMma) {
    const float* g = A.taps + A.tap_off[s];
    // Tap tile of block j: row t (0..127) = sample tb0 + 128 j + t, K = frame f.
    // Lanes run along the rows (samples), so each tap load of a warp reads 32 consecutive taps
    // g[(t - f D) mod L] (= g[(f D - t) mod L], g is even).
    auto build_b = [&](int j) {
      const uint32_t tile = sB0 + uint32_t(j & 1) * kT;
      const int tj = tb0 + 128 * j;
      for (int q = tid; q < 128 * (F / 8); q += kPtProd) {
        const int row = q & 127, c = q >> 7;
        const int t = tj + row;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int f = fa + 8 * c + e;
          v[e] = (t < L && 8 * c + e < A.n_frames) ? __ldg(g + ((t - f * D) & (L - 1))) : 0.f;
        }
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split2(v[2 * e], v[2 * e + 1], hi[e], lo[e]);
        st_shared_v4(pa_chunk<F>(tile, row, c, false), hi);
        st_shared_v4(pa_chunk<F>(tile, row, c, true), lo);
      }
      fence_proxy_async();
      mbar_arrive(smem_u32(&ctl->b_full[j & 1]));
    };
    // dPhi tile: row r0 + q / (F / 8), frames 8 (q % (F / 8)) .. + 7.
    const float* dp = dphi + static_cast<int64_t>(b) * phi_size + phi2_off[a];
    for (int q = tid; q < 128 * (F / 8); q += kPtProd) {
      const int row = q / (F / 8), c = q % (F / 8);
      const int r = r0 + row;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f), y = x;
      if (r < A.rows && BAND) {  // frames fa + 8 c .. + 7, taken mod n_frames
        const float* src = dp + static_cast<int64_t>(r) * A.n_frames;
        const int m = A.n_frames - 1, f = fa + 8 * c;
        x = make_float4(__ldg(src + (f & m)), __ldg(src + ((f + 1) & m)), __ldg(src + ((f + 2) & m)),
                        __ldg(src + ((f + 3) & m)));
        y = make_float4(__ldg(src + ((f + 4) & m)), __ldg(src + ((f + 5) & m)), __ldg(src + ((f + 6) & m)),
                        __ldg(src + ((f + 7) & m)));
      } else if (r < A.rows) {
        const float4* src = reinterpret_cast<const float4*>(dp + static_cast<int64_t>(r) * A.n_frames + 8 * c);
        x = __ldg(src);
        y = __ldg(src + 1);
      }
      uint32_t hi[4], lo[4];
      split2(x.x, x.y, hi[0], lo[0]);
      split2(x.z, x.w, hi[1], lo[1]);
      split2(y.x, y.y, hi[2], lo[2]);
      split2(y.z, y.w, hi[3], lo[3]);
      st_shared_v4(pa_chunk<F>(sA, row, c, false), hi);
      st_shared_v4(pa_chunk<F>(sA, row, c, true), lo);
    }
    fence_proxy_async();
    mbar_arrive(smem_u32(&ctl->a_full));
    build_b(0);
    if (nblk > 1) build_b(1);
    // Epilogue of block j: warp w stores rows 32 (w % 4) + lane, samples 64 (w / 4) .. + 63 of the block.
    // For F = 32 each 32 x 32 piece goes through a padded per-warp shared-memory tile (rows of 36
    // floats), so that the global stores run along the rows: 8 lanes x 16 bytes per row, 4 rows per
    // store instruction, instead of one row per lane.
    const int q4 = warp & 3, hh = warp >> 2;
    const int r = r0 + 32 * q4 + lane;
    float* orow = dV2 + static_cast<int64_t>(b) * A.v2_tot + A.v2_off[a] + static_cast<int64_t>(r < A.rows ? r : 0) * L;
    float* vbase = dV2 + static_cast<int64_t>(b) * A.v2_tot + A.v2_off[a];
    const uint32_t stg = sB0 + 2 * kT + uint32_t(warp) * 4608u;
    for (int j = 0; j < nblk; ++j) {
      const int jb = j & 1;
      const bool ok = pt_wait(smem_u32(&ctl->d_full[jb]), (j >> 1) & 1, abort);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const int t = tb0 + 128 * j + 64 * hh;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float v[32];
        tmem_ld32(tmem + (uint32_t(q4 * 32) << 16) + uint32_t(jb * 128 + 64 * hh + 32 * h), v);
        if (pa_staged<F, BAND>()) {
          const int tt = t + 32 * h;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const uint32_t w4[4] = {__float_as_uint(v[4 * e]), __float_as_uint(v[4 * e + 1]),
                                    __float_as_uint(v[4 * e + 2]), __float_as_uint(v[4 * e + 3])};
            st_shared_v4(stg + uint32_t(lane) * 144u + 16u * e, w4);
          }
          __syncwarp();
          const int tl = tt + 4 * (lane & 7);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int rho = 4 * k + (lane >> 3), rg = r0 + 32 * q4 + rho;
            const float4 x = ld_shared_v4f(stg + uint32_t(rho) * 144u + 16u * uint32_t(lane & 7));
            if (rg < A.rows) {
              float* o = vbase + static_cast<int64_t>(rg) * L + tl;
              if (tl + 4 <= L) {
                *reinterpret_cast<float4*>(o) = x;
              } else {
                if (tl < L) o[0] = x.x;
                if (tl + 1 < L) o[1] = x.y;
                if (tl + 2 < L) o[2] = x.z;
              }
            }
          }
          __syncwarp();
        } else if (r < A.rows) {
          const int tt = t + 32 * h;
          if (tt + 32 <= L) {
            float4* o = reinterpret_cast<float4*>(orow + tt);
#pragma unroll
            for (int e = 0; e < 8; ++e) o[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
          } else {
#pragma unroll
            for (int e = 0; e < 32; ++e)
              if (tt + e < L) orow[tt + e] = v[e];
          }
        }
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&ctl->d_empty[jb]));
      // Block j + 2 reuses tap stage jb: its MMAs (block j) have completed (d_full above).
      if (j + 2 < nblk) build_b(j + 2);
    }
  } else if (warp == kPtWarpMma && lane == 0) {
    issued = true;
    const uint32_t idesc = idesc_bf16_n(128);
    bool ok = pt_wait(smem_u32(&ctl->a_full), 0, abort);
    tc_fence_after();
    for (int j = 0; ok && j < nblk; ++j) {
      const int jb = j & 1;
      if (!pt_wait(smem_u32(&ctl->b_full[jb]), (j >> 1) & 1, abort)) break;
      if (j >= 2 && !pt_wait(smem_u32(&ctl->d_empty[jb]), ((j >> 1) - 1) & 1, abort)) break;
      tc_fence_after();
      const uint32_t sB = sB0 + uint32_t(jb) * kT;
      const uint32_t d = tmem + uint32_t(jb) * 128u;
#pragma unroll
      for (int kk = 0; kk < F / 16; ++kk) {
        const uint64_t ah = sdesc(sA + pa_hi<F>(kk), 16, 1024), al = sdesc(sA + pa_lo<F>(kk), 16, 1024);
        const uint64_t bh = sdesc(sB + pa_hi<F>(kk), 16, 1024), bl = sdesc(sB + pa_lo<F>(kk), 16, 1024);
        umma_bf16(d, ah, bh, idesc, kk != 0);
        umma_bf16(d, al, bh, idesc, 1);
        umma_bf16(d, ah, bl, idesc, 1);
      }
      umma_commit(smem_u32(&ctl->d_full[jb]));
    }
    umma_commit(smem_u32(&ctl->done));  // completes once every issued MMA has completed
    // TMEM is freed below: wait for that completion (bounded), also after an abort.
    for (uint32_t i = 0; i < kSpinLimit && !mbar_try_wait(smem_u32(&ctl->done), 0); ++i) __nanosleep(64);
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && *abort) atomicExch(&g_pt_err, 1);
  if (warp == kPtWarpMma) {
    __syncwarp();
    tmem_dealloc(tmem, 256);
  }
}

template <auto Kernel>
cudaError_t pt_opt_in(size_t smem) {
  return cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
}

template <int F, bool BAND = false, bool SUBW = false>
int launch_pt(const PtArgs& A, unsigned grid, cudaStream_t s) {
  constexpr size_t smem = pt_smem<F, SUBW>();
  if (pt_opt_in<k_pool_tc_fwd<F, BAND, SUBW>>(smem) != cudaSuccess) return JTFS_ERR_CUDA;
  k_pool_tc_fwd<F, BAND, SUBW><<<grid, kPtThreads, smem, s>>>(A);
  return cudaGetLastError() == cudaSuccess ? JTFS_OK : JTFS_ERR_CUDA;
}

template <int F, bool BAND = false>
int launch_pa(const PtArgs& A, const float* dphi, int64_t phi_size, const int64_t* phi2_off, float* dV2,
              unsigned grid, cudaStream_t s) {
  constexpr size_t smem = pa_smem<F, BAND>();
  if (pt_opt_in<k_pool_tc_adj<F, BAND>>(smem) != cudaSuccess) return JTFS_ERR_CUDA;
  k_pool_tc_adj<F, BAND><<<grid, kPtThreads, smem, s>>>(A, dphi, phi_size, phi2_off, dV2);
  return cudaGetLastError() == cudaSuccess ? JTFS_OK : JTFS_ERR_CUDA;
}

}  // namespace

int pool_tc_adjoint(const Plan& p, const float* dphi, float* dV2, cudaStream_t s) {
  if (p.pool_tc_adj_tiles.empty()) return JTFS_OK;
  PtArgs A{};
  A.tiles = p.d_pool_tc_adj_tiles;
  A.s2 = p.d_s2;
  A.v2_off = p.d_v2_off;
  A.taps = p.d_taps;
  A.tap_off = p.d_tap_off;
  A.v2_tot = p.v2_tot;
  A.logN = p.logN;
  A.lT = p.lT;
  A.n_frames = p.n_frames;
  A.rows = p.rows2;
  A.n_active = p.n_active;
  const unsigned grid = static_cast<unsigned>(p.pool_tc_adj_tiles.size());
  switch (p.n_frames) {
    case 32: return launch_pa<32>(A, dphi, p.phi_size, p.d_phi2_off, dV2, grid, s);
    case 64: return launch_pa<64>(A, dphi, p.phi_size, p.d_phi2_off, dV2, grid, s);
    case 128: return launch_pa<128>(A, dphi, p.phi_size, p.d_phi2_off, dV2, grid, s);
    default: return JTFS_ERR_SHAPE;
  }
}

int pool_tc_band_adjoint(const Plan& p, const float* dphi, float* dV2, cudaStream_t s) {
  if (p.pool_tc_band_adj_tiles.empty()) return JTFS_OK;
  PtArgs A{};
  A.tiles = p.d_pool_tc_band_adj_tiles;
  A.s2 = p.d_s2;
  A.v2_off = p.d_v2_off;
  A.taps = p.d_taps;
  A.tap_off = p.d_tap_off;
  A.v2_tot = p.v2_tot;
  A.logN = p.logN;
  A.lT = p.lT;
  A.n_frames = p.n_frames;
  A.rows = p.rows2;
  A.n_active = p.n_active;
  A.pool_w = p.d_pool_w;
  A.band_S = p.d_pool_band_S;
  return launch_pa<kPoolBandAdjF, true>(A, dphi, p.phi_size, p.d_phi2_off, dV2,
                                     static_cast<unsigned>(p.pool_tc_band_adj_tiles.size()), s);
}

bool pool_tc_dense(const Plan& p) { return p.n_frames == 32 || p.n_frames == 64 || p.n_frames == 128; }

bool pool_tc_supported(const Plan& p) { return pool_tc_dense(p) || !p.pool_tc_band_tiles.empty(); }

int pool_tc_band(const Plan& p, const float* V2, float* phi, cudaStream_t s) {
  if (p.pool_tc_band_tiles.empty()) return JTFS_OK;
  PtArgs A{};
  A.V2 = V2;
  A.tiles = p.d_pool_tc_band_tiles;
  A.s2 = p.d_s2;
  A.v2_off = p.d_v2_off;
  A.taps = p.d_taps;
  A.tap_off = p.d_tap_off;
  A.v2_tot = p.v2_tot;
  A.logN = p.logN;
  A.lT = p.lT;
  A.n_frames = p.n_frames;
  A.rows = p.rows2;
  A.n_active = p.n_active;
  A.pool_w = p.d_pool_w;
  A.phi = phi;
  A.phi_size = p.phi_size;
  A.phi2_off = p.d_phi2_off;
  const unsigned grid = static_cast<unsigned>(p.pool_tc_band_tiles.size());
  return p.pool_tc_band_long ? launch_pt<32, true, true>(A, grid, s) : launch_pt<32, true, false>(A, grid, s);
}

int pool_tc_forward(const Plan& p, const float* V2, float* part, int si, cudaStream_t s) {
  if (p.pool_tc_tiles[si].empty()) return JTFS_OK;
  PtArgs A{};
  A.V2 = V2;
  A.part = part;
  A.tiles = p.d_pool_tc_tiles[si];
  A.tile0 = p.d_pool_tile0[si];
  A.s2 = p.d_s2;
  A.v2_off = p.d_v2_off;
  A.taps = p.d_taps;
  A.tap_off = p.d_tap_off;
  A.v2_tot = p.v2_tot;
  A.logN = p.logN;
  A.lT = p.lT;
  A.n_frames = p.n_frames;
  A.rows = p.rows2;
  A.n_active = p.n_active;
  A.split_len = kPoolSplits[si];
  const unsigned grid = static_cast<unsigned>(p.pool_tc_tiles[si].size());
  switch (p.n_frames) {
    case 32: return launch_pt<32>(A, grid, s);
    case 64: return launch_pt<64>(A, grid, s);
    case 128: return launch_pt<128>(A, grid, s);
    default: return JTFS_ERR_SHAPE;
  }
}

int pool_tc_error() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_pt_err, sizeof(int)) != cudaSuccess) return JTFS_ERR_CUDA;
  const int zero = 0;
  if (v && cudaMemcpyToSymbol(g_pt_err, &zero, sizeof(int)) != cudaSuccess) return JTFS_ERR_CUDA;
  return v;
}

int set_wait_polls_pool(int64_t polls) {
  const uint32_t v = polls < 0 ? kSpinLimit : static_cast<uint32_t>(polls < int64_t(kSpinLimit) ? polls : kSpinLimit);
  return cudaMemcpyToSymbol(c_wait_polls, &v, sizeof(v)) == cudaSuccess ? JTFS_OK : JTFS_ERR_CUDA;
}

}  // namespace jtfs
