// Learned initialiser layers: transposed 1-D convolution (stride 2, kernel 9,
// padding 4, output padding 1) with its data and weight gradients, BF16
// operands and FP32 accumulation, activations channels-last ([B][T][C]).
//
// Output time t = 2v + p (parity p) of a layer sees input samples v + 2 - j:
//   z[b][2v+p][co] = bias[co] + sum_{j<5, ci} x[b][v+2-j][ci] W[ci][co][2j+p]   (2j+p <= 8)
//   dx[b][u][ci]   = sum_{k<9, co} g[b][2u-4+k][co] W[ci][co][k]
//   dW[ci][co][k]  = sum_{b, u} x[b][u][ci] g[b][2u-4+k][co]
// With g [B][2T][C] read as [B][T][2C] (row u holds times 2u and 2u+1), time
// 2u-4+k is row u-2+m, half q, for k = 2m+q.  Every shift is therefore a shift
// of whole rows, which a TMA tile load takes as its row coordinate (rows outside
// the clip read as zero), so the three products are GEMMs on the 5th-generation
// tensor cores with no gather:
//   forward   M = 128 positions v, N = 256 = (p, co), K = (ci block, j)
//   data grad M = 128 positions u, N = 128 = ci,      K = (k, co block)
//   weight    M = 128 channels ci, N = 256 = (q, co), K = positions (split, fixed-order reduction)
// One CTA of 4 warps per output tile: thread 0 issues TMA loads into a ring of
// shared-memory stages, thread 32 issues tcgen05.mma (accumulator in TMEM) and
// frees each stage with tcgen05.commit, then all four warps read the
// accumulator back with tcgen05.ld and run the fused epilogue (bias + GELU,
// GELU', or the split-K partial store).  Every mbarrier wait is bounded; a
// wait that runs out sets an abort flag, the CTA drains and frees its TMEM,
// and jtfs_decoder_error() reports it.
//
// The output layer (128 -> 1 channel) is too narrow for the tensor cores and
// runs as plain FMA kernels.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "jtfs.h"
#include "jtfs_umma.cuh"

namespace {

constexpr int kC = 128;                    // hidden width (tensor-core layers)

__device__ int g_decoder_err;


__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// ---------------------------------------------------------------------------
// The tensor-core GEMM skeleton.
// ---------------------------------------------------------------------------
struct Ctl {
  unsigned long long full[4], empty[4], done;
  uint32_t tmem;
  int abort;
};

template <class Op>
constexpr size_t umma_smem_bytes() {
  return sizeof(Ctl) + 1024 + size_t(Op::kStages) * (128 * 64 * 2 + Op::kBN * 64 * 2);
}

template <class Op>
__global__ void __launch_bounds__(128, 1)
k_umma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const Op op) {
  constexpr int S = Op::kStages, BN = Op::kBN;
  constexpr uint32_t kA = 128 * 64 * 2, kB = BN * 64 * 2, kStage = kA + kB;
  extern __shared__ uint8_t smem_raw[];
  Ctl* ctl = reinterpret_cast<Ctl*>(smem_raw);
  const uint32_t base = (smem_u32(smem_raw) + sizeof(Ctl) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = op.num_kblocks();
  volatile int* abort = &ctl->abort;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&ctl->full[s]), 1);
      mbar_init(smem_u32(&ctl->empty[s]), 1);
    }
    mbar_init(smem_u32(&ctl->done), 1);
    ctl->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) tmem_alloc(smem_u32(&ctl->tmem), BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem;

  int issued = 0;
  if (threadIdx.x == 0) {  // TMA producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % S;
      if (kb >= S && !mbar_wait(smem_u32(&ctl->empty[s]), ((kb / S) - 1) & 1, abort)) break;
      const uint32_t bar = smem_u32(&ctl->full[s]);
      mbar_expect_tx(bar, kStage);
      op.load(kb, &tmA, &tmB, base + s * kStage, base + s * kStage + kA, bar);
      issued = kb + 1;
    }
  } else if (threadIdx.x == 32) {  // MMA issuer
    constexpr uint32_t idesc = idesc_bf16(BN, Op::kAMN, Op::kBMN);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % S;
      if (!mbar_wait(smem_u32(&ctl->full[s]), (kb / S) & 1, abort)) break;
      tc_fence_after();
      const uint32_t a = base + s * kStage, b = a + kA;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) umma_bf16(tmem, Op::adesc(a, kk), Op::bdesc(b, kk), idesc, (kb | kk) != 0);
      umma_commit(smem_u32(&ctl->empty[s]));
    }
    umma_commit(smem_u32(&ctl->done));  // arrives once every MMA issued above has completed
  }
  const bool got = mbar_wait(smem_u32(&ctl->done), 0, abort);
  tc_fence_after();
  const int good = __syncthreads_and(got && !*abort && nk > 0);
  if (good) {
    op.epilogue(tmem, warp, lane);
  } else if (threadIdx.x == 32) {
    // Every MMA issued above must complete before TMEM is freed (the wait above gives up early on abort).
    for (uint32_t i = 0; i < kSpinLimit && !mbar_try_wait(smem_u32(&ctl->done), 0); ++i) __nanosleep(64);
  }
  tc_fence_before();
  __syncthreads();
  if (!good && threadIdx.x == 0) {
    // Let this thread's TMA copies still in flight land before the CTA exits.
    for (int kb = max(0, issued - S); kb < issued; ++kb) {
      const uint32_t bar = smem_u32(&ctl->full[kb % S]);
      for (uint32_t i = 0; i < kSpinLimit && !mbar_try_wait(bar, (kb / S) & 1); ++i) __nanosleep(64);
    }
    if (nk > 0) atomicExch(&g_decoder_err, 1);
  }
  if (warp == 2) tmem_dealloc(tmem, BN);
}

// Epilogue store helpers: 32 consecutive values of one row.
__device__ __forceinline__ void store32_f32(float* dst, const float (&v)[32]) {
  float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int i = 0; i < 8; ++i) d[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}
__device__ __forceinline__ void store32_bf16(uint16_t* dst, const float (&v)[32]) {
  uint4* d = reinterpret_cast<uint4*>(dst);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      w[k] = uint32_t(f2bf(v[8 * i + 2 * k])) | (uint32_t(f2bf(v[8 * i + 2 * k + 1])) << 16);
    d[i] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Forward: grid (ceil(T / 128), B).  A = x rows v0 + 2 - j (box 64 ch x 128 rows),
// B = Wf [(p, co)][(j, ci)] (box 64 x 256).
struct FwdOp {
  static constexpr int kBN = 256, kStages = 2;
  static constexpr bool kAMN = false, kBMN = false;
  int T, Cip;
  const float* bias;
  float* z;
  uint16_t* h;
  __device__ int num_kblocks() const { return 5 * (Cip / 64); }
  __device__ void load(int kb, const CUtensorMap* ta, const CUtensorMap* tb, uint32_t sa, uint32_t sb,
                       uint32_t bar) const {
    const int c = kb / 5, j = kb % 5;
    tma_load_3d(sa, ta, bar, c * 64, int(blockIdx.x) * 128 + 2 - j, int(blockIdx.y));
    tma_load_2d(sb, tb, bar, j * Cip + c * 64, 0);
  }
  __device__ static uint64_t adesc(uint32_t a, int kk) { return sdesc(a + kk * 32, 16, 1024); }
  __device__ static uint64_t bdesc(uint32_t b, int kk) { return sdesc(b + kk * 32, 16, 1024); }
  __device__ void epilogue(uint32_t tmem, int warp, int lane) const {
    const int v = int(blockIdx.x) * 128 + warp * 32 + lane;
    const bool valid = v < T;
    const int64_t row0 = (int64_t(blockIdx.y) * 2 * T + 2 * int64_t(v)) * kC;
#pragma unroll 1
    for (int col = 0; col < 2 * kC; col += 32) {
      float acc[32];
      tmem_ld32(tmem + (uint32_t(warp * 32) << 16) + col, acc);
      const int p = col / kC, co = col % kC;
      const float4* bb = reinterpret_cast<const float4*>(bias + co);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float4 q = bb[i];
        acc[4 * i] += q.x;
        acc[4 * i + 1] += q.y;
        acc[4 * i + 2] += q.z;
        acc[4 * i + 3] += q.w;
      }
      if (valid) {
        const int64_t off = row0 + int64_t(p) * kC + co;
        if (z) store32_f32(z + off, acc);
        if (h) {
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[i] = gelu(acc[i]);
          store32_bf16(h + off, acc);
        }
      }
    }
  }
};

// Data gradient: grid (ceil(T / 128), B).  A = g read as [B][T][256], rows
// u0 - 2 + m, half q (box 64 x 128 rows); B = Wd [ci][(k, co)] (box 64 x 128).
struct BwdDataOp {
  static constexpr int kBN = 128, kStages = 3;
  static constexpr bool kAMN = false, kBMN = false;
  int T;
  const float* zprev;  // GELU' applied when non-null
  float* g32;
  uint16_t* g16;
  __device__ int num_kblocks() const { return 9 * (kC / 64); }
  __device__ void load(int kb, const CUtensorMap* ta, const CUtensorMap* tb, uint32_t sa, uint32_t sb,
                       uint32_t bar) const {
    const int k = kb / (kC / 64), c = kb % (kC / 64);
    const int m = k >> 1, q = k & 1;
    tma_load_3d(sa, ta, bar, q * kC + c * 64, int(blockIdx.x) * 128 - 2 + m, int(blockIdx.y));
    tma_load_2d(sb, tb, bar, k * kC + c * 64, 0);
  }
  __device__ static uint64_t adesc(uint32_t a, int kk) { return sdesc(a + kk * 32, 16, 1024); }
  __device__ static uint64_t bdesc(uint32_t b, int kk) { return sdesc(b + kk * 32, 16, 1024); }
  __device__ void epilogue(uint32_t tmem, int warp, int lane) const {
    const int u = int(blockIdx.x) * 128 + warp * 32 + lane;
    const bool valid = u < T;
    const int64_t row = (int64_t(blockIdx.y) * T + u) * kC;
#pragma unroll 1
    for (int col = 0; col < kC; col += 32) {
      float acc[32];
      tmem_ld32(tmem + (uint32_t(warp * 32) << 16) + col, acc);
      if (valid) {
        if (zprev) {
          const float4* zz = reinterpret_cast<const float4*>(zprev + row + col);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float4 q = zz[i];
            acc[4 * i] *= gelu_grad(q.x);
            acc[4 * i + 1] *= gelu_grad(q.y);
            acc[4 * i + 2] *= gelu_grad(q.z);
            acc[4 * i + 3] *= gelu_grad(q.w);
          }
        }
        if (g32) store32_f32(g32 + row + col, acc);
        if (g16) store32_bf16(g16 + row + col, acc);
      }
    }
  }
};

// Weight gradient: grid (5, Cip / 128, splits).  blockIdx.x = m (taps 2m, 2m+1),
// blockIdx.z = (clip, position chunk).  A = x [positions][ci] MN-major (two
// boxes 64 ch x 64 rows), B = g as [B][T][256] rows u - 2 + m MN-major (four
// boxes 64 x 64 rows).  Partial sums D[ci][(q, co)] go to part[split][m][ci][256].
struct DwOp {
  static constexpr int kBN = 256, kStages = 2;
  static constexpr bool kAMN = true, kBMN = true;
  int T, Cip, chunk, spc;  // spc = chunks per clip
  float* part;
  __device__ int u_begin() const { return (int(blockIdx.z) % spc) * chunk; }
  __device__ int num_kblocks() const { return (min(chunk, T - u_begin()) + 63) / 64; }
  __device__ void load(int kb, const CUtensorMap* ta, const CUtensorMap* tb, uint32_t sa, uint32_t sb,
                       uint32_t bar) const {
    const int b = int(blockIdx.z) / spc, u = u_begin() + kb * 64, m = int(blockIdx.x);
    const int ci0 = int(blockIdx.y) * 128;
    tma_load_3d(sa, ta, bar, ci0, u, b);
    tma_load_3d(sa + 8192, ta, bar, ci0 + 64, u, b);
#pragma unroll
    for (int n = 0; n < 4; ++n) tma_load_3d(sb + n * 8192, tb, bar, n * 64, u - 2 + m, b);
  }
  __device__ static uint64_t adesc(uint32_t a, int kk) { return sdesc(a + kk * 2048, 8192, 1024); }
  __device__ static uint64_t bdesc(uint32_t b, int kk) { return sdesc(b + kk * 2048, 8192, 1024); }
  __device__ void epilogue(uint32_t tmem, int warp, int lane) const {
    const int ci = int(blockIdx.y) * 128 + warp * 32 + lane;
    float* dst = part + ((int64_t(blockIdx.z) * 5 + blockIdx.x) * Cip + ci) * 256;
#pragma unroll 1
    for (int col = 0; col < 256; col += 32) {
      float acc[32];
      tmem_ld32(tmem + (uint32_t(warp * 32) << 16) + col, acc);
      store32_f32(dst + col, acc);
    }
  }
};

// dW[ci][co][k] = sum over splits (ascending) of part[split][k/2][ci][(k%2) C + co], ci < Ci.
__global__ void k_dw_reduce(const float* __restrict__ part, float* __restrict__ dw, int Ci, int Cip, int splits) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(Ci) * kC * 9) return;
  const int k = int(idx % 9), co = int((idx / 9) % kC), ci = int(idx / (9 * kC));
  const int64_t step = int64_t(5) * Cip * 256;
  const float* p = part + (int64_t(k >> 1) * Cip + ci) * 256 + (k & 1) * kC + co;
  float acc = 0.f;
  for (int s = 0; s < splits; ++s) acc += p[s * step];
  dw[idx] = acc;
}

// ---------------------------------------------------------------------------
// Output layer (C -> 1 channel): plain FMA kernels.
// ---------------------------------------------------------------------------
constexpr int kOutV = 64;  // positions per CTA

// y[b][2v+p] = bias + sum_{j, ci} x[b][v+2-j][ci] w[ci][2j+p]; grid (ceil(T/64), B), 128 threads.
__global__ void __launch_bounds__(128)
k_out_fwd(const uint16_t* __restrict__ x, const float* __restrict__ w, const float* __restrict__ bias,
          float* __restrict__ y, int T) {
  __shared__ float xs[kC][kOutV + 5];
  __shared__ float ws[kC][9];
  const int b = blockIdx.y, v0 = blockIdx.x * kOutV;
  for (int i = threadIdx.x; i < kC * 9; i += blockDim.x) ws[i / 9][i % 9] = w[i];
  for (int i = threadIdx.x; i < (kOutV + 4) * kC; i += blockDim.x) {
    const int r = i / kC, ci = i % kC, v = v0 - 2 + r;
    xs[ci][r] = (v >= 0 && v < T) ? bf2f(x[(int64_t(b) * T + v) * kC + ci]) : 0.f;
  }
  __syncthreads();
  const int vl = threadIdx.x >> 1, p = threadIdx.x & 1, v = v0 + vl;
  float acc = bias[0];
  for (int ci = 0; ci < kC; ++ci) {
#pragma unroll
    for (int j = 0; j < 5; ++j)
      if (2 * j + p <= 8) acc += xs[ci][vl + 4 - j] * ws[ci][2 * j + p];
  }
  if (v < T) y[int64_t(b) * 2 * T + 2 * v + p] = acc;
}

// g[b][u][ci] = (sum_k dy[b][2u-4+k] w[ci][k]) * GELU'(zprev[b][u][ci]).  One warp per
// position (b, u), four channels per lane (16-byte loads and stores).
__global__ void __launch_bounds__(256)
k_out_bwd_data(const float* __restrict__ dy, const float* __restrict__ w, const float* __restrict__ zprev,
               float* __restrict__ g32, uint16_t* __restrict__ g16, int T, int64_t rows) {
  __shared__ float4 ws[9][kC / 4];
  for (int i = threadIdx.x; i < 9 * (kC / 4); i += blockDim.x) {
    const int k = i / (kC / 4), c = 4 * (i % (kC / 4));
    ws[k][i % (kC / 4)] = make_float4(w[c * 9 + k], w[(c + 1) * 9 + k], w[(c + 2) * 9 + k], w[(c + 3) * 9 + k]);
  }
  __syncthreads();
  const int64_t row = int64_t(blockIdx.x) * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (row >= rows) return;
  const int c4 = threadIdx.x & 31;
  const int u = int(row % T);
  const float* d = dy + (row / T) * 2 * T;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int t = 2 * u - 4 + k;
    if (t >= 0 && t < 2 * T) {
      const float dv = d[t];
      const float4 q = ws[k][c4];
      acc.x += dv * q.x;
      acc.y += dv * q.y;
      acc.z += dv * q.z;
      acc.w += dv * q.w;
    }
  }
  const int64_t i4 = row * (kC / 4) + c4;
  if (zprev) {
    const float4 z = reinterpret_cast<const float4*>(zprev)[i4];
    acc.x *= gelu_grad(z.x);
    acc.y *= gelu_grad(z.y);
    acc.z *= gelu_grad(z.z);
    acc.w *= gelu_grad(z.w);
  }
  if (g32) reinterpret_cast<float4*>(g32)[i4] = acc;
  if (g16)
    reinterpret_cast<uint2*>(g16)[i4] = make_uint2(uint32_t(f2bf(acc.x)) | (uint32_t(f2bf(acc.y)) << 16),
                                                   uint32_t(f2bf(acc.z)) | (uint32_t(f2bf(acc.w)) << 16));
}

constexpr int kOutChunk = 256;  // positions per CTA of the output layer's weight gradient

// part[chunk][ci][k] = sum over the chunk's u of x[b][u][ci] dy[b][2u-4+k];
// part_db[chunk] = sum of dy over the chunk's times [2 u0, 2 uend).  grid (ceil(T/256), B).
__global__ void __launch_bounds__(128)
k_out_bwd_weight(const uint16_t* __restrict__ x, const float* __restrict__ dy, float* __restrict__ part,
                 float* __restrict__ part_db, int T) {
  __shared__ float ds[2 * kOutChunk + 8];
  __shared__ float red[128];
  const int b = blockIdx.y, u0 = blockIdx.x * kOutChunk;
  const float* d = dy + int64_t(b) * 2 * T;
  for (int i = threadIdx.x; i < 2 * kOutChunk + 8; i += blockDim.x) {
    const int t = 2 * u0 - 4 + i;
    ds[i] = (t >= 0 && t < 2 * T) ? d[t] : 0.f;
  }
  __syncthreads();
  const int ci = threadIdx.x;
  float acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.f;
  const int uend = min(T, u0 + kOutChunk);
  for (int u = u0; u < uend; ++u) {
    const float xv = bf2f(x[(int64_t(b) * T + u) * kC + ci]);
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] += xv * ds[2 * (u - u0) + k];
  }
  const int64_t chunk = int64_t(blockIdx.y) * gridDim.x + blockIdx.x;
#pragma unroll
  for (int k = 0; k < 9; ++k) part[(chunk * kC + ci) * 9 + k] = acc[k];
  // bias: this chunk's times, fixed-order tree
  float s = 0.f;
  for (int i = threadIdx.x; i < 2 * (uend - u0); i += blockDim.x) s += ds[4 + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part_db[chunk] = red[0];
}

__global__ void k_out_reduce(const float* __restrict__ part, const float* __restrict__ part_db,
                             float* __restrict__ dw, float* __restrict__ db, int chunks) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kC * 9) {
    float acc = 0.f;
    for (int c = 0; c < chunks; ++c) acc += part[int64_t(c) * kC * 9 + i];
    dw[i] = acc;
  } else if (i == kC * 9 && db) {
    float acc = 0.f;
    for (int c = 0; c < chunks; ++c) acc += part_db[c];
    db[0] = acc;
  }
}

// ---------------------------------------------------------------------------
// Bias gradient of a tensor-core layer, packing, cast, Adam.
// ---------------------------------------------------------------------------
constexpr int kColChunk = 512;  // rows per CTA

__global__ void __launch_bounds__(128)
k_colsum(const float* __restrict__ g, int64_t rows, float* __restrict__ part) {
  const int64_t r0 = int64_t(blockIdx.x) * kColChunk;
  const int64_t r1 = min(rows, r0 + kColChunk);
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;  // four interleaved partial sums, combined in fixed order
  const float* p = g + threadIdx.x;
  int64_t r = r0;
  for (; r + 4 <= r1; r += 4) {
    a0 += p[r * kC];
    a1 += p[(r + 1) * kC];
    a2 += p[(r + 2) * kC];
    a3 += p[(r + 3) * kC];
  }
  for (; r < r1; ++r) a0 += p[r * kC];
  part[int64_t(blockIdx.x) * kC + threadIdx.x] = (a0 + a1) + (a2 + a3);
}

__global__ void k_colsum_reduce(const float* __restrict__ part, float* __restrict__ db, int chunks) {
  const int c = threadIdx.x;
  float acc = 0.f;
  for (int i = 0; i < chunks; ++i) acc += part[int64_t(i) * kC + c];
  db[c] = acc;
}

// x[b][t][c] = bf16(phi[b][c][t] * s[c]) for c < C, 0 for C <= c < Cip.  32 x 32 tiles.
__global__ void k_pack_input(const float* __restrict__ phi, const float* __restrict__ s, uint16_t* __restrict__ x,
                             int C, int Cip, int T) {
  __shared__ float tile[32][33];
  const int b = blockIdx.z, c0 = blockIdx.y * 32, t0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 256 threads: 8 rows per pass
  for (int r = ty; r < 32; r += 8) {
    const int c = c0 + r, t = t0 + tx;
    tile[r][tx] = (c < C && t < T) ? phi[(int64_t(b) * C + c) * T + t] * s[c] : 0.f;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int t = t0 + r, c = c0 + tx;
    if (t < T && c < Cip) x[(int64_t(b) * T + t) * Cip + c] = f2bf(tile[tx][r]);
  }
}

// wf[(p, co)][(j, ci)] = W[ci][co][2j+p] (0 where 2j+p > 8 or ci >= Ci), [2C][5 Cip].
__global__ void k_pack_wf(const float* __restrict__ w, uint16_t* __restrict__ wf, int Ci, int Cip) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t n = int64_t(2 * kC) * 5 * Cip;
  if (i >= n) return;
  const int col = int(i % (5 * Cip)), row = int(i / (5 * Cip));
  const int p = row / kC, co = row % kC, j = col / Cip, ci = col % Cip;
  const int k = 2 * j + p;
  wf[i] = (k <= 8 && ci < Ci) ? f2bf(w[(int64_t(ci) * kC + co) * 9 + k]) : uint16_t(0);
}

// wd[ci][(k, co)] = W[ci][co][k], [C][9 C].
__global__ void k_pack_wd(const float* __restrict__ w, uint16_t* __restrict__ wd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kC * 9 * kC) return;
  const int col = i % (9 * kC), ci = i / (9 * kC);
  const int k = col / kC, co = col % kC;
  wd[i] = f2bf(w[(ci * kC + co) * 9 + k]);
}

__global__ void k_cast_bf16(const float* __restrict__ x, uint16_t* __restrict__ y, int64_t n) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) y[i] = f2bf(x[i]);
}

__global__ void k_adam_params(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                              float* __restrict__ v, uint16_t* __restrict__ pb, int64_t n, float lr, float c1,
                              float c2) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
  p[i] = pi;
  if (pb) pb[i] = f2bf(pi);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
int ok() { return cudaGetLastError() == cudaSuccess ? JTFS_OK : JTFS_ERR_CUDA; }
unsigned blocks(int64_t n) { return static_cast<unsigned>((n + 255) / 256); }
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// BF16 tensor map with 128-byte swizzle over a [d2][d1][d0] array (d0 innermost).
bool make_map(CUtensorMap* m, const void* base, int rank, uint64_t d0, uint64_t d1, uint64_t d2, uint32_t b0,
              uint32_t b1) {
  auto fn = encode_fn();
  if (!fn || !aligned16(base)) return false;
  const cuuint64_t dims[3] = {d0, d1, d2};
  const cuuint64_t strides[2] = {d0 * 2, d0 * d1 * 2};
  const cuuint32_t box[3] = {b0, b1, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class Op>
int launch_umma(const CUtensorMap& ta, const CUtensorMap& tb, const Op& op, dim3 grid, cudaStream_t s) {
  constexpr size_t smem = umma_smem_bytes<Op>();
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_umma<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (attr != cudaSuccess) return JTFS_ERR_CUDA;
  k_umma<Op><<<grid, 128, smem, s>>>(ta, tb, op);
  return ok();
}

bool bad(int B, int T) { return B < 1 || T < 1 || int64_t(B) * T > (int64_t(1) << 28) || T > (1 << 24); }

// Weight-gradient split: about 8 waves of 152 CTAs, chunks of whole 64-row blocks within one clip.
void dw_split(int B, int Cip, int T, int* chunk, int* spc) {
  const int64_t per_clip = std::max<int64_t>(1, std::llround(1216.0 / (5.0 * (Cip / 128) * B)));
  *chunk = static_cast<int>(cdiv(cdiv(T, per_clip), 64) * 64);
  *spc = static_cast<int>(cdiv(T, *chunk));
}

}  // namespace

extern "C" int jtfs_convt_padded_channels(int C) { return C < 1 ? 0 : static_cast<int>(cdiv(C, 128) * 128); }

extern "C" int jtfs_convt_pack_input(const float* phi, const float* row_scale, uint16_t* x, int B, int C, int T,
                                     void* stream) {
  if (!phi || !row_scale || !x || C < 1 || bad(B, T)) return JTFS_ERR_ARG;
  const int Cip = jtfs_convt_padded_channels(C);
  dim3 grid(static_cast<unsigned>(cdiv(T, 32)), static_cast<unsigned>(cdiv(Cip, 32)), static_cast<unsigned>(B));
  k_pack_input<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(phi, row_scale, x, C, Cip, T);
  return ok();
}

extern "C" int jtfs_convt_pack_weights(const float* w, uint16_t* wf, uint16_t* wd, int Ci, int Co, void* stream) {
  if (!w || !wf || Ci < 1 || Co != kC || (wd && Ci != kC)) return JTFS_ERR_ARG;
  const int Cip = jtfs_convt_padded_channels(Ci);
  auto s = static_cast<cudaStream_t>(stream);
  k_pack_wf<<<blocks(int64_t(2 * kC) * 5 * Cip), 256, 0, s>>>(w, wf, Ci, Cip);
  if (wd) k_pack_wd<<<blocks(kC * 9 * kC), 256, 0, s>>>(w, wd);
  return ok();
}

extern "C" int jtfs_convt_forward(const uint16_t* x, const uint16_t* wf, const float* bias, float* z, uint16_t* h,
                                  int B, int Cip, int Co, int T, void* stream) {
  if (!x || !wf || !bias || (!z && !h) || Co != kC || Cip < 128 || Cip % 128 || bad(B, T)) return JTFS_ERR_ARG;
  if (!aligned16(bias) || (z && !aligned16(z)) || (h && !aligned16(h))) return JTFS_ERR_ARG;
  CUtensorMap ta, tb;
  if (!make_map(&ta, x, 3, Cip, T, B, 64, 128) || !make_map(&tb, wf, 2, 5 * Cip, 2 * kC, 1, 64, 2 * kC))
    return JTFS_ERR_ARG;
  FwdOp op{T, Cip, bias, z, h};
  return launch_umma(ta, tb, op, dim3(static_cast<unsigned>(cdiv(T, 128)), static_cast<unsigned>(B)),
                     static_cast<cudaStream_t>(stream));
}

extern "C" int jtfs_convt_backward_data(const uint16_t* g, const uint16_t* wd, const float* zprev, float* g_prev,
                                        uint16_t* g_prev_bf16, int B, int Ci, int Co, int T, void* stream) {
  if (!g || !wd || (!g_prev && !g_prev_bf16) || Ci != kC || Co != kC || bad(B, T)) return JTFS_ERR_ARG;
  if ((zprev && !aligned16(zprev)) || (g_prev && !aligned16(g_prev)) || (g_prev_bf16 && !aligned16(g_prev_bf16)))
    return JTFS_ERR_ARG;
  CUtensorMap ta, tb;
  if (!make_map(&ta, g, 3, 2 * kC, T, B, 64, 128) || !make_map(&tb, wd, 2, 9 * kC, kC, 1, 64, kC))
    return JTFS_ERR_ARG;
  BwdDataOp op{T, zprev, g_prev, g_prev_bf16};
  return launch_umma(ta, tb, op, dim3(static_cast<unsigned>(cdiv(T, 128)), static_cast<unsigned>(B)),
                     static_cast<cudaStream_t>(stream));
}

extern "C" size_t jtfs_convt_weight_workspace_bytes(int B, int Cip, int Co, int T) {
  if (Co != kC || Cip < 128 || Cip % 128 || bad(B, T)) return 0;
  int chunk, spc;
  dw_split(B, Cip, T, &chunk, &spc);
  return size_t(B) * spc * 5 * Cip * 256 * sizeof(float);
}

extern "C" int jtfs_convt_backward_weight(const uint16_t* x, const uint16_t* g, float* dw, int B, int Ci, int Cip,
                                          int Co, int T, void* workspace, void* stream) {
  if (!x || !g || !dw || !workspace || Co != kC || Ci < 1 || Ci > Cip || Cip % 128 || bad(B, T))
    return JTFS_ERR_ARG;
  if (!aligned16(workspace)) return JTFS_ERR_ARG;
  int chunk, spc;
  dw_split(B, Cip, T, &chunk, &spc);
  CUtensorMap ta, tb;
  if (!make_map(&ta, x, 3, Cip, T, B, 64, 64) || !make_map(&tb, g, 3, 2 * kC, T, B, 64, 64)) return JTFS_ERR_ARG;
  float* part = static_cast<float*>(workspace);
  DwOp op{T, Cip, chunk, spc, part};
  auto s = static_cast<cudaStream_t>(stream);
  const int rc =
      launch_umma(ta, tb, op, dim3(5, static_cast<unsigned>(Cip / 128), static_cast<unsigned>(B * spc)), s);
  if (rc != JTFS_OK) return rc;
  k_dw_reduce<<<blocks(int64_t(Ci) * kC * 9), 256, 0, s>>>(part, dw, Ci, Cip, B * spc);
  return ok();
}

extern "C" size_t jtfs_convt_bias_workspace_bytes(int64_t rows) {
  return rows < 1 ? 0 : size_t(cdiv(rows, kColChunk)) * kC * sizeof(float);
}

extern "C" int jtfs_convt_bias_grad(const float* g, float* db, int64_t rows, int Co, void* workspace, void* stream) {
  if (!g || !db || !workspace || Co != kC || rows < 1) return JTFS_ERR_ARG;
  const int chunks = static_cast<int>(cdiv(rows, kColChunk));
  auto s = static_cast<cudaStream_t>(stream);
  float* part = static_cast<float*>(workspace);
  k_colsum<<<chunks, kC, 0, s>>>(g, rows, part);
  k_colsum_reduce<<<1, kC, 0, s>>>(part, db, chunks);
  return ok();
}

extern "C" int jtfs_convt_out_forward(const uint16_t* x, const float* w, const float* bias, float* y, int B, int Ci,
                                      int T, void* stream) {
  if (!x || !w || !bias || !y || Ci != kC || bad(B, T)) return JTFS_ERR_ARG;
  dim3 grid(static_cast<unsigned>(cdiv(T, kOutV)), static_cast<unsigned>(B));
  k_out_fwd<<<grid, 128, 0, static_cast<cudaStream_t>(stream)>>>(x, w, bias, y, T);
  return ok();
}

extern "C" int jtfs_convt_out_backward_data(const float* dy, const float* w, const float* zprev, float* g_prev,
                                            uint16_t* g_prev_bf16, int B, int Ci, int T, void* stream) {
  if (!dy || !w || (!g_prev && !g_prev_bf16) || Ci != kC || bad(B, T)) return JTFS_ERR_ARG;
  if ((zprev && !aligned16(zprev)) || (g_prev && !aligned16(g_prev)) || (g_prev_bf16 && !aligned16(g_prev_bf16)))
    return JTFS_ERR_ARG;
  const int64_t rows = int64_t(B) * T;
  k_out_bwd_data<<<static_cast<unsigned>(cdiv(rows, 8)), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      dy, w, zprev, g_prev, g_prev_bf16, T, rows);
  return ok();
}

extern "C" size_t jtfs_convt_out_workspace_bytes(int B, int T) {
  if (bad(B, T)) return 0;
  const int64_t chunks = int64_t(B) * cdiv(T, kOutChunk);
  return size_t(chunks) * (kC * 9 + 1) * sizeof(float);
}

extern "C" int jtfs_convt_out_backward_weight(const uint16_t* x, const float* dy, float* dw, float* db, int B,
                                              int Ci, int T, void* workspace, void* stream) {
  if (!x || !dy || !dw || !workspace || Ci != kC || bad(B, T)) return JTFS_ERR_ARG;
  const int per = static_cast<int>(cdiv(T, kOutChunk));
  const int chunks = B * per;
  auto s = static_cast<cudaStream_t>(stream);
  float* part = static_cast<float*>(workspace);
  float* part_db = part + int64_t(chunks) * kC * 9;
  k_out_bwd_weight<<<dim3(per, B), 128, 0, s>>>(x, dy, part, part_db, T);
  k_out_reduce<<<static_cast<unsigned>(cdiv(kC * 9 + 1, 256)), 256, 0, s>>>(part, part_db, dw, db, chunks);
  return ok();
}

namespace jtfs {
int set_wait_polls_decoder(int64_t polls) {
  const uint32_t v = polls < 0 ? kSpinLimit : static_cast<uint32_t>(polls < int64_t(kSpinLimit) ? polls : kSpinLimit);
  return cudaMemcpyToSymbol(c_wait_polls, &v, sizeof(v)) == cudaSuccess ? JTFS_OK : JTFS_ERR_CUDA;
}
}  // namespace jtfs

extern "C" int jtfs_decoder_error(void) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_decoder_err, sizeof(int)) != cudaSuccess) return JTFS_ERR_CUDA;
  const int zero = 0;
  if (v && cudaMemcpyToSymbol(g_decoder_err, &zero, sizeof(int)) != cudaSuccess) return JTFS_ERR_CUDA;
  return v;
}

extern "C" int jtfs_cast_bf16(const float* x, uint16_t* y, int64_t n, void* stream) {
  if (!x || !y || n < 0) return JTFS_ERR_ARG;
  if (n) k_cast_bf16<<<blocks(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, y, n);
  return ok();
}

extern "C" int jtfs_adam_update(float* param, const float* grad, float* m, float* v, uint16_t* param_bf16, int64_t n,
                                float lr, int step, void* stream) {
  if (!param || !grad || !m || !v || n < 0 || step < 1 || !(lr > 0.f)) return JTFS_ERR_ARG;
  const float c1 = static_cast<float>(1.0 / (1.0 - std::pow(0.9, step)));
  const float c2 = static_cast<float>(1.0 / (1.0 - std::pow(0.999, step)));
  if (n) k_adam_params<<<blocks(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(param, grad, m, v, param_bf16, n, lr, c1,
                                                                                c2);
  return ok();
}
