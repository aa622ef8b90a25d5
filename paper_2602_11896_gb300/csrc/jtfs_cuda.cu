// CUDA kernels (sm_103a) and the compute entry points of the JTFS C ABI.
//
// Every filtering step of the method (Eqs. (1)-(5); §3.2-§3.5) is done in
// the Fourier domain: a loader evaluates the analytic filter on the bins
// where it is not negligible and folds them onto the decimated grid
// ("subsample_fourier", §3.2: periodisation of the spectrum, which equals
// time-domain decimation), a shared-memory Stockham FFT transforms, and a
// storer writes.  The frequential scattering (§3.4) with its modulus and
// phi_F averaging runs fused per tile of time columns; phi_T averaging of the
// second order is a decimating FIR.  The adjoint chain (§2.3, Eqs. (6)-(8))
// transposes each step: periodisation becomes tiling, filters multiply again
// (they are real in the Fourier domain), the modulus becomes z/|z|.
//
// FFT convention: F (sign -1) and F^H (sign +1), both unnormalised; every
// 1/n factor is applied by a loader.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "jtfs.h"
#include "jtfs_device.cuh"
#include "jtfs_internal.h"

namespace jtfs {
namespace {

// ---------------------------------------------------------------------------
// Complex helpers and filters
// ---------------------------------------------------------------------------
// Filter value at signed bin s of its grid (see FiltD).
__device__ __forceinline__ float fval(const FiltD& f, int s) {
  const float d = static_cast<float>(s) - f.c0;
  float v = expf(-d * d * f.a);
  if (f.kappa != 0.f) {
    const float sf = static_cast<float>(s);
    v -= f.kappa * expf(-sf * sf * f.a);
  }
  return v;
}

// sum over signed bins s in [f.lo, f.hi] with s = m (mod Ld) of
// src[s mod Ls] * value(s): a filter product folded onto Ld bins.
__device__ __forceinline__ float2 band_gather(const float2* __restrict__ src, int Ls, int Ld, int m,
                                              const FiltD& f) {
  float2 acc = make_float2(0.f, 0.f);
  for (int s = f.lo + ((m - f.lo) & (Ld - 1)); s <= f.hi; s += Ld) {
    const float g = fval(f, s);
    const float2 v = src[s & (Ls - 1)];
    acc.x += g * v.x;
    acc.y += g * v.y;
  }
  return acc;
}

// sum over signed bins s in [f.lo, f.hi] with s = m (mod L) of value(s):
// the filter periodised onto L bins ("levels", read as a sum of aliases).
__device__ __forceinline__ float band_lev(int m, int L, const FiltD& f) {
  float acc = 0.f;
  for (int s = f.lo + ((m - f.lo) & (L - 1)); s <= f.hi; s += L) acc += fval(f, s);
  return acc;
}

template <bool INV>
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int e) {
  float2 w = __ldg(tw + e);
  if (INV) w.y = -w.y;
  return w;
}

// ---------------------------------------------------------------------------
// CTA-wide batched Stockham FFT in shared memory.
// `count` transforms of size 2^logn; transform f lives at a + f*bstride.
// Mixed radix: one radix-2 pass when logn is odd, then radix-4 passes.
// Returns the buffer (a or b) holding the natural-order result.  Must be
// called by every thread of the block.
// ---------------------------------------------------------------------------
template <bool INV>
__device__ float2* cta_fft(float2* a, float2* b, int logn, int count, int bstride,
                           const float2* __restrict__ tw, int twlog) {
  const int n = 1 << logn;
  int lNs = 0;
  if (logn & 1) {
    const int lq = logn - 1, q = n >> 1;
    const int total = count << lq;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int f = i >> lq, j = i & (q - 1);
      const float2* src = a + f * bstride;
      float2* dst = b + f * bstride;
      const float2 v0 = src[j], v1 = src[j + q];
      dst[2 * j] = make_float2(v0.x + v1.x, v0.y + v1.y);
      dst[2 * j + 1] = make_float2(v0.x - v1.x, v0.y - v1.y);
    }
    __syncthreads();
    float2* t = a; a = b; b = t;
    lNs = 1;
  }
  while (lNs < logn) {
    const int lq = logn - 2, q = n >> 2;
    const int total = count << lq;
    const int Ns = 1 << lNs;
    const int shift = twlog - (lNs + 2);
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int f = i >> lq, j = i & (q - 1);
      const float2* src = a + f * bstride;
      float2* dst = b + f * bstride;
      const int k = j & (Ns - 1);
      float2 v0 = src[j], v1 = src[j + q], v2 = src[j + 2 * q], v3 = src[j + 3 * q];
      if (lNs > 0) {
        v1 = cmul(v1, twiddle<INV>(tw, k << shift));
        v2 = cmul(v2, twiddle<INV>(tw, (2 * k) << shift));
        v3 = cmul(v3, twiddle<INV>(tw, (3 * k) << shift));
      }
      const float2 s02 = make_float2(v0.x + v2.x, v0.y + v2.y);
      const float2 d02 = make_float2(v0.x - v2.x, v0.y - v2.y);
      const float2 s13 = make_float2(v1.x + v3.x, v1.y + v3.y);
      const float2 d13 = make_float2(v1.x - v3.x, v1.y - v3.y);
      float2 y1, y3;
      if (!INV) {  // W_4 = -i
        y1 = make_float2(d02.x + d13.y, d02.y - d13.x);
        y3 = make_float2(d02.x - d13.y, d02.y + d13.x);
      } else {
        y1 = make_float2(d02.x - d13.y, d02.y + d13.x);
        y3 = make_float2(d02.x + d13.y, d02.y - d13.x);
      }
      const int d = ((j - k) << 2) + k;
      dst[d] = make_float2(s02.x + s13.x, s02.y + s13.y);
      dst[d + Ns] = y1;
      dst[d + 2 * Ns] = make_float2(s02.x - s13.x, s02.y - s13.y);
      dst[d + 3 * Ns] = y3;
    }
    __syncthreads();
    float2* t = a; a = b; b = t;
    lNs += 2;
  }
  return a;
}

// ---------------------------------------------------------------------------
// Register DFTs of size 2, 4, 8, 16 (natural order in and out) and a
// batched Stockham FFT over *interleaved* transforms: element i of transform
// f lives at a[i * cnt + f].  Consecutive threads take consecutive f, so every
// load and store of a pass is contiguous across the warp (no bank conflicts
// whatever the Stockham stride), and all threads of a warp read the same
// twiddle (a broadcast).  Twiddles come from a shared-memory table.
// ---------------------------------------------------------------------------
// One radix-R pass over interleaved transforms, two adjacent transforms per
// thread (16-byte accesses; both share index arithmetic and twiddles).
template <bool INV, int R, int LR>
__device__ __forceinline__ void il_pass(const float2* __restrict__ src, float2* __restrict__ dst, int logn,
                                        int lcnt, int lNs, const float2* __restrict__ tw, int twlog) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
  float4* d4 = reinterpret_cast<float4*>(dst);
  const int lq = logn - LR;
  const int lp = lcnt - 1;                 // log2(pairs per bin)
  const int total = 1 << (lq + lp);
  const int Ns = 1 << lNs;
  const int shift = twlog - (lNs + LR);
  const int sstride = 1 << (lq + lp);      // float4 stride between the R inputs
  const int dstride = Ns << lp;            // float4 stride between the R outputs
  for (int idx = threadIdx.x; idx < total; idx += kThreads) {
    const int fp = idx & ((1 << lp) - 1), j = idx >> lp;
    const int k = j & (Ns - 1);
    float2 va[R], vb[R];
    const float4* sp = s4 + ((j << lp) + fp);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4 t = sp[r * sstride];
      va[r] = make_float2(t.x, t.y);
      vb[r] = make_float2(t.z, t.w);
    }
    if (lNs > 0) {
      const int e = k << shift;
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
    float4* dp = d4 + (((((j - k) << LR) + k) << lp) + fp);
#pragma unroll
    for (int q = 0; q < R; ++q) dp[q * dstride] = make_float4(va[q].x, va[q].y, vb[q].x, vb[q].y);
  }
}

// 2^lcnt (>= 2) interleaved transforms of size 2^logn; tw = shared table of
// exp(-2 pi i e / 2^twlog), 2^twlog >= 2^logn.  Returns the result buffer.
template <bool INV>
__device__ float2* cta_fft_il(float2* a, float2* b, int logn, int lcnt, const float2* __restrict__ tw, int twlog) {
  int lNs = 0;
  while (lNs < logn) {
    const int rem = logn - lNs;
    int lr;
    if (rem == 5 || rem == 6 || rem == 9 || rem == 3) {
      il_pass<INV, 8, 3>(a, b, logn, lcnt, lNs, tw, twlog);
      lr = 3;
    } else if (rem >= 4) {
      il_pass<INV, 16, 4>(a, b, logn, lcnt, lNs, tw, twlog);
      lr = 4;
    } else if (rem == 2) {
      il_pass<INV, 4, 2>(a, b, logn, lcnt, lNs, tw, twlog);
      lr = 2;
    } else {
      il_pass<INV, 2, 1>(a, b, logn, lcnt, lNs, tw, twlog);
      lr = 1;
    }
    __syncthreads();
    float2* t = a; a = b; b = t;
    lNs += lr;
  }
  return a;
}

// ---------------------------------------------------------------------------
// Loaders: element idx of the input of the FFT described by a job.
// ---------------------------------------------------------------------------
struct LdReal {  // real row -> complex
  const float* s;
  __device__ float2 operator()(const Job& jb, int idx, int) const {
    return make_float2(s[jb.src + idx], 0.f);
  }
};
struct LdC {  // complex row
  const float2* s;
  __device__ float2 operator()(const Job& jb, int idx, int) const { return s[jb.src + idx]; }
};
struct LdMod {  // |z| of a complex row (the modulus of §2.1)
  const float2* s;
  __device__ float2 operator()(const Job& jb, int idx, int) const {
    const float2 v = s[jb.src + idx];
    return make_float2(sqrtf(v.x * v.x + v.y * v.y), 0.f);
  }
};
// Filter product folded onto 2^logn bins, scaled by 1/Ls (Ls = source row
// length): with an unnormalised inverse FFT this yields the decimated
// filtered signal (§3.2 cdgmm + subsample_fourier + ifft).
struct LdBand {
  const float2* s;
  const FiltD* table;  // per-job filter table[jb.filt], or NULL: `fixed`
  FiltD fixed;
  __device__ float2 operator()(const Job& jb, int idx, int logn) const {
    const FiltD f = table ? table[jb.filt] : fixed;
    const int Ls = 1 << jb.lslog;
    return cscale(band_gather(s + jb.src, Ls, 1 << logn, idx, f), 1.f / static_cast<float>(Ls));
  }
};
// Adjoint of the modulus: dz = du * z / |z| (0 where z = 0); du is the real
// part of a complex row.
struct LdDz {
  const float2* du;
  const float2* z;
  __device__ float2 operator()(const Job& jb, int idx, int) const {
    const float g = du[jb.src + idx].x;
    const float2 v = z[jb.src + idx];
    const float m = sqrtf(v.x * v.x + v.y * v.y);
    return m > 0.f ? make_float2(g * v.x / m, g * v.y / m) : make_float2(0.f, 0.f);
  }
};

// Band product of the coloured initialisation (§2.3): g = a * z, with the
// envelope a the real part of a complex row and z the band-passed noise.
struct LdLin {
  const float2* a;
  const float2* z;
  __device__ float2 operator()(const Job& jb, int idx, int) const {
    const float s = a[jb.src + idx].x;
    const float2 v = z[jb.src + idx];
    return make_float2(s * v.x, s * v.y);
  }
};

struct StC {
  float2* d;
  __device__ void operator()(const Job& jb, int idx, float2 v) const { d[jb.dst + idx] = v; }
};
struct StR {  // real part
  float* d;
  __device__ void operator()(const Job& jb, int idx, float2 v) const { d[jb.dst + idx] = v.x; }
};

}  // namespace
}  // namespace jtfs

#include "jtfs_tfft.cuh"

namespace jtfs {
namespace {

// ---------------------------------------------------------------------------
// Batched FFT kernels.
// ---------------------------------------------------------------------------
template <bool INV, class Ld, class St>
__global__ void __launch_bounds__(kThreads)
k_fft_small(Ld ld, St st, const Job* __restrict__ jobs, int njobs, int logn, int per_cta,
            const float2* __restrict__ tw, int twlog) {
  extern __shared__ float2 sm[];
  const int n = 1 << logn;
  const int j0 = blockIdx.x * per_cta;
  const int nj = min(per_cta, njobs - j0);
  float2* a = sm;
  float2* b = sm + per_cta * n;
  for (int i = threadIdx.x; i < nj * n; i += blockDim.x) a[i] = ld(jobs[j0 + (i >> logn)], i & (n - 1), logn);
  __syncthreads();
  float2* r = cta_fft<INV>(a, b, logn, nj, n, tw, twlog);
  for (int i = threadIdx.x; i < nj * n; i += blockDim.x) st(jobs[j0 + (i >> logn)], i & (n - 1), r[i]);
}

// Four-step FFT for 2^logn > 2^kSmallLogMax: n = na * nb, na = 2^la.
// Pass 1: for each column c < nb, FFT of size na over x[c + nb*i], times
// W_n^{c k}, into scratch row-major [k][c].  Pass 2: for each row k, FFT of
// size nb over c; output index k + na*q.  CB columns / rows per CTA.
template <bool INV, int CB, class Ld>
__global__ void __launch_bounds__(kThreads)
k_fft4_pass1(Ld ld, const Job* __restrict__ jobs, int logn, int la, float2* __restrict__ scr,
             const float2* __restrict__ tw, int twlog) {
  extern __shared__ float2 sm[];
  const int lb = logn - la, na = 1 << la, nb = 1 << lb;
  const int groups = nb / CB;
  const int jl = blockIdx.x / groups;
  const int c0 = (blockIdx.x % groups) * CB;
  const Job jb = jobs[jl];
  const int bs = na + 1;
  float2* a = sm;
  float2* b = sm + CB * bs;
  for (int i = threadIdx.x; i < CB * na; i += blockDim.x) {
    const int cc = i % CB, ii = i / CB;
    a[cc * bs + ii] = ld(jb, (c0 + cc) + (ii << lb), logn);
  }
  __syncthreads();
  float2* r = cta_fft<INV>(a, b, la, CB, bs, tw, twlog);
  const int tshift = twlog - logn;
  float2* out = scr + (static_cast<int64_t>(jl) << logn);
  for (int i = threadIdx.x; i < CB * na; i += blockDim.x) {
    const int cc = i % CB, k = i / CB;
    const float2 v = cmul(r[cc * bs + k], twiddle<INV>(tw, ((c0 + cc) * k) << tshift));
    out[(static_cast<int64_t>(k) << lb) + c0 + cc] = v;
  }
}

template <bool INV, int CB, class St>
__global__ void __launch_bounds__(kThreads)
k_fft4_pass2(St st, const Job* __restrict__ jobs, int logn, int la, const float2* __restrict__ scr,
             const float2* __restrict__ tw, int twlog) {
  extern __shared__ float2 sm[];
  const int lb = logn - la, na = 1 << la, nb = 1 << lb;
  const int groups = na / CB;
  const int jl = blockIdx.x / groups;
  const int k0 = (blockIdx.x % groups) * CB;
  const Job jb = jobs[jl];
  const int bs = nb + 1;
  float2* a = sm;
  float2* b = sm + CB * bs;
  const float2* in = scr + (static_cast<int64_t>(jl) << logn);
  for (int i = threadIdx.x; i < CB * nb; i += blockDim.x) {
    const int kk = i >> lb, c = i & (nb - 1);
    a[kk * bs + c] = in[(static_cast<int64_t>(k0 + kk) << lb) + c];
  }
  __syncthreads();
  float2* r = cta_fft<INV>(a, b, lb, CB, bs, tw, twlog);
  for (int i = threadIdx.x; i < CB * nb; i += blockDim.x) {
    const int kk = i % CB, q = i / CB;
    st(jb, (k0 + kk) + (q << la), r[kk * bs + q]);
  }
}

// Opt in to large dynamic shared memory once per kernel (keyed on the kernel
// itself: instantiations that differ only in INV or MODE share a type).
template <auto Kernel>
void allow_big_smem() {
  static const cudaError_t once = [] {
    // Static shared memory counts against the same per-block limit.
    cudaFuncAttributes fa{};
    int stat = 0;
    if (cudaFuncGetAttributes(&fa, Kernel) == cudaSuccess) stat = static_cast<int>(fa.sharedSizeBytes);
    const cudaError_t e =
        cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem - stat);
    cudaGetLastError();  // do not leave a sticky error for the next launch check
    return e;
  }();
  (void)once;
}

// One launch of the batched / four-step kernels.
template <bool INV, class Ld, class St>
int run_fft_launch(const Plan& p, const FftLaunch& l, const Ld& ld, const St& st, float2* scr, cudaStream_t s) {
  {
    const Job* jobs = p.d_jobs + l.job0;
    if (l.logn <= kSmallLogMax) {
      const int n = 1 << l.logn;
      const int per = std::max(1, std::min(p.tune_fft_points, 1 << kSmallLogMax) >> l.logn);
      const int grid = (l.njobs + per - 1) / per;
      const size_t smem = 2 * size_t(per) * n * sizeof(float2);
      allow_big_smem<k_fft_small<INV, Ld, St>>();
      k_fft_small<INV, Ld, St><<<grid, kThreads, smem, s>>>(ld, st, jobs, l.njobs, l.logn, per, p.d_tw,
                                                             p.twlog);
    } else {
      const int la = l.logn / 2, lb = l.logn - la;
      if (la <= 9 && lb <= 9) {
        constexpr int CB = 16;
        const size_t sm1 = 2 * size_t(CB) * ((1 << la) + 1) * sizeof(float2);
        const size_t sm2 = 2 * size_t(CB) * ((1 << lb) + 1) * sizeof(float2);
        allow_big_smem<k_fft4_pass1<INV, CB, Ld>>();
        allow_big_smem<k_fft4_pass2<INV, CB, St>>();
        k_fft4_pass1<INV, CB, Ld><<<l.njobs * ((1 << lb) / CB), kThreads, sm1, s>>>(ld, jobs, l.logn, la, scr,
                                                                                  p.d_tw, p.twlog);
        k_fft4_pass2<INV, CB, St><<<l.njobs * ((1 << la) / CB), kThreads, sm2, s>>>(st, jobs, l.logn, la, scr,
                                                                                  p.d_tw, p.twlog);
      } else {
        constexpr int CB = 8;
        const size_t sm1 = 2 * size_t(CB) * ((1 << la) + 1) * sizeof(float2);
        const size_t sm2 = 2 * size_t(CB) * ((1 << lb) + 1) * sizeof(float2);
        allow_big_smem<k_fft4_pass1<INV, CB, Ld>>();
        allow_big_smem<k_fft4_pass2<INV, CB, St>>();
        k_fft4_pass1<INV, CB, Ld><<<l.njobs * ((1 << lb) / CB), kThreads, sm1, s>>>(ld, jobs, l.logn, la, scr,
                                                                                  p.d_tw, p.twlog);
        k_fft4_pass2<INV, CB, St><<<l.njobs * ((1 << la) / CB), kThreads, sm2, s>>>(st, jobs, l.logn, la, scr,
                                                                                  p.d_tw, p.twlog);
      }
    }
    if (cudaGetLastError() != cudaSuccess) return JTFS_ERR_CUDA;
  }
  return JTFS_OK;
}

// One launch description of 2^17 .. 2^20 points on the FFT engine (two passes through the scratch).
template <bool INV, class Ld, class St>
int run_tfft_big(const Plan& p, const FftLaunch& l, const Ld& ld, const St& st, float2* scr, cudaStream_t s) {
  allow_big_smem<k_tfft_big1<INV, Ld>>();
  allow_big_smem<k_tfft_big2<INV, St>>();
  const unsigned grid = static_cast<unsigned>(l.njobs) << (l.logn - kTfLogP);
  k_tfft_big1<INV, Ld><<<grid, kTfThreads, kTfSmem, s>>>(ld, p.d_jobs, l.job0, l.logn, scr);
  k_tfft_big2<INV, St><<<grid, kTfThreads, kTfSmem, s>>>(st, p.d_jobs, l.job0, l.logn, scr);
  return cudaGetLastError() == cudaSuccess ? JTFS_OK : JTFS_ERR_CUDA;
}

// Transforms of one stage on the time-axis FFT engine (jtfs_tfft.cuh): every
// size up to 2^13 in one launch of k_tfft, each size 2^14 .. 2^16 in one
// cluster launch, larger ones on the four-step kernels.
template <bool INV, class Ld, class St>
int run_tfft(const Plan& p, const std::vector<FftLaunch>& L, const Ld& ld, const St& st, float2* scr,
             cudaStream_t s) {
  // One launch per run of consecutive items (the plan gives every stage a single run).
  int i0 = -1, i1 = -1;
  auto flush = [&]() -> int {
    if (i1 <= i0) return JTFS_OK;
    allow_big_smem<k_tfft<INV, Ld, St>>();
    k_tfft<INV, Ld, St><<<static_cast<unsigned>(i1 - i0), kTfThreads, kTfSmem, s>>>(ld, st, p.d_jobs,
                                                                                  p.d_tf_items + i0);
    return cudaGetLastError() == cudaSuccess ? JTFS_OK : JTFS_ERR_CUDA;
  };
  for (const FftLaunch& l : L) {
    if (l.logn > kTfLogP || l.n_items == 0) continue;
    if (l.item0 != i1) {
      const int rc = flush();
      if (rc != JTFS_OK) return rc;
      i0 = l.item0;
    }
    i1 = l.item0 + l.n_items;
  }
  {
    const int rc = flush();
    if (rc != JTFS_OK) return rc;
  }
  for (const FftLaunch& l : L) {
    if (l.logn <= kTfLogP) continue;
    if (l.logn > kTfLogP + 3) {
      const int rc = l.logn <= kTfLogP + 7 ? run_tfft_big<INV>(p, l, ld, st, scr, s)
                                           : run_fft_launch<INV>(p, l, ld, st, scr, s);
      if (rc != JTFS_OK) return rc;
      continue;
    }
    allow_big_smem<k_tfft_cluster<INV, Ld, St>>();
    const unsigned C = 1u << (l.logn - kTfLogP);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(static_cast<unsigned>(l.njobs) * C);
    cfg.blockDim = dim3(kTfThreads);
    cfg.dynamicSmemBytes = kTfSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_tfft_cluster<INV, Ld, St>, ld, st, p.d_jobs, l.job0, l.logn) != cudaSuccess)
      return JTFS_ERR_CUDA;
  }
  return JTFS_OK;
}

template <bool INV, class Ld, class St>
int run_fft(const Plan& p, const std::vector<FftLaunch>& L, const Ld& ld, const St& st, float2* scr,
            cudaStream_t s) {
  if (p.tune_tfft) return run_tfft<INV>(p, L, ld, st, scr, s);
  for (const FftLaunch& l : L) {
    const int rc = run_fft_launch<INV>(p, l, ld, st, scr, s);
    if (rc != JTFS_OK) return rc;
  }
  return JTFS_OK;
}

// ---------------------------------------------------------------------------
// Frequential scattering (§3.4) fused with modulus and phi_F averaging.
// One CTA per tile of W time columns; every column is zero-padded to N_fr
// rows, transformed once, then for each frequential filter beta:
// product + fold to R = N_fr/2^k bins, inverse FFT, modulus, FFT, phi_F
// product + fold to R_out bins, inverse FFT, real part.
// MODE 1: first order, input S1 (real), betas {phi_F, +xi}, output Phi.
// MODE 2: second order, input Y2 (complex), all betas, output V2.
// ---------------------------------------------------------------------------
// Z[m][f] = (1/N_fr) sum_{s in band, s = m mod R} yhat[s][w] psi_beta(s), transform f = bc*W + w.
// Two adjacent transforms (same filter) per thread.
__device__ __forceinline__ void freq_fold(const FreqArgs& A, const FreqSmem& S, const FreqChunk& ch, int lc,
                                          const float2* yh, float2* out, int lR) {
  const int R = 1 << lR, Nfr = A.N_fr;
  const float inv = 1.f / static_cast<float>(Nfr);
  const int lp = lc - 1;
  const float4* y4 = reinterpret_cast<const float4*>(yh);
  float4* o4 = reinterpret_cast<float4*>(out);
  const int lWp = A.logW - 1;
  for (int i = threadIdx.x; i < (R << lp); i += kThreads) {
    const int fp = i & ((1 << lp) - 1), m = i >> lp;
    const int bc = fp >> lWp, wp = fp & ((1 << lWp) - 1);
    const int b = bc < ch.n ? ch.beta[bc] : -1;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (b >= 0) {
      const int2 bd = S.band[b];
      const float* t = S.tab + b * Nfr;
      const float4* yc = y4 + wp;
      for (int sb = bd.x + ((m - bd.x) & (R - 1)); sb <= bd.y; sb += R) {
        const int q = sb & (Nfr - 1);
        const float g = __ldg(t + q);
        const float4 y = yc[q << lWp];
        acc.x += g * y.x;
        acc.y += g * y.y;
        acc.z += g * y.z;
        acc.w += g * y.w;
      }
    }
    o4[i] = make_float4(acc.x * inv, acc.y * inv, acc.z * inv, acc.w * inv);
  }
}

// W[m][f] = (1/R) sum_{s in phi_F band, s = m mod R_out} uhat[s mod R][f] phi_F(s).
__device__ __forceinline__ void freq_pool_fold(const FreqArgs& A, const FreqSmem& S, int lc, const float2* uh,
                                               float2* out, int lR) {
  const int R = 1 << lR, Nfr = A.N_fr, Ro = A.R_out;
  const float* t = S.tab + A.n_beta2 * Nfr;
  const float inv = 1.f / static_cast<float>(R);
  const int lp = lc - 1;
  const float4* u4 = reinterpret_cast<const float4*>(uh);
  float4* o4 = reinterpret_cast<float4*>(out);
  for (int i = threadIdx.x; i < (Ro << lp); i += kThreads) {
    const int fp = i & ((1 << lp) - 1), m = i >> lp;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int sb = A.phiF.lo + ((m - A.phiF.lo) & (Ro - 1)); sb <= A.phiF.hi; sb += Ro) {
      const float g = __ldg(t + (sb & (Nfr - 1)));
      const float4 v = u4[((sb & (R - 1)) << lp) + fp];
      acc.x += g * v.x;
      acc.y += g * v.y;
      acc.z += g * v.z;
      acc.w += g * v.w;
    }
    o4[i] = make_float4(acc.x * inv, acc.y * inv, acc.z * inv, acc.w * inv);
  }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads)
k_freq_fwd(FreqArgs A, const Tile* __restrict__ tiles, const float* __restrict__ S1,
           const float2* __restrict__ Y2, float* __restrict__ out) {
  extern __shared__ float2 sm[];
  const Tile tl = tiles[blockIdx.x];
  const int W = A.W, WN = W * A.N_fr;
  const FreqSmem S = freq_smem_carve(A, sm, 3);
  float2* buf0 = S.buf;
  float2* buf1 = buf0 + WN;
  float2* buf2 = buf1 + WN;
  freq_stage_tables(A, S);
  int stride, n1m;
  freq_load_columns<MODE>(A, tl, S1, Y2, buf0, stride, n1m);
  __syncthreads();
  float2* yh = cta_fft_il<false>(buf0, buf1, A.logNfr, A.logW, S.tw, A.logNfr);
  float2* f1 = (yh == buf0) ? buf1 : buf0;
  float2* f2 = buf2;
  const int Ro = A.R_out, lRo = A.logRout;
  for (int c = 0; c < A.n_chunks; ++c) {
    const FreqChunk& ch = S.chk[c];
    const int lR = A.logNfr - ch.k;
    const int lc = ceil_log2(ch.n) + A.logW;
    freq_fold(A, S, ch, lc, yh, f1, lR);
    __syncthreads();
    float2* z = cta_fft_il<true>(f1, f2, lR, lc, S.tw, A.logNfr);
    {
      float4* z4 = reinterpret_cast<float4*>(z);
      for (int i = threadIdx.x; i < (1 << (lR + lc - 1)); i += kThreads) {
        const float4 v = z4[i];
        z4[i] = make_float4(sqrtf(v.x * v.x + v.y * v.y), 0.f, sqrtf(v.z * v.z + v.w * v.w), 0.f);
      }
    }
    __syncthreads();
    if (A.unpooled_f) {  // |Y_fr| rows as they are: no phi_F
      for (int i = threadIdx.x; i < (1 << (lR + lc)); i += blockDim.x) {
        const int f = i & ((1 << lc) - 1), row = i >> lc;
        const int bc = f >> A.logW, w = f & (W - 1);
        if (bc < ch.n && w < tl.ncols) {
          const int b = ch.beta[bc];
          const int64_t r = A.row_off[b] + row;
          if (MODE == 1)
            out[static_cast<int64_t>(tl.b) * A.phi_size + A.phi1_off + r * A.n_frames + tl.t0 + w] = z[i].x;
          else
            out[static_cast<int64_t>(tl.b) * A.v2_tot + A.v2_off[tl.a] + r * stride + tl.t0 + w] = z[i].x;
        }
      }
      __syncthreads();
      continue;
    }
    float2* zo = (z == f1) ? f2 : f1;
    float2* uh = cta_fft_il<false>(z, zo, lR, lc, S.tw, A.logNfr);
    float2* g = (uh == f1) ? f2 : f1;
    freq_pool_fold(A, S, lc, uh, g, lR);
    __syncthreads();
    float2* pr = cta_fft_il<true>(g, uh, lRo, lc, S.tw, A.logNfr);
    for (int i = threadIdx.x; i < (Ro << lc); i += blockDim.x) {
      const int f = i & ((1 << lc) - 1), row = i >> lc;
      const int bc = f >> A.logW, w = f & (W - 1);
      if (bc < ch.n && w < tl.ncols) {
        const int b = ch.beta[bc];
        const float v = pr[i].x;
        if (MODE == 1)
          out[static_cast<int64_t>(tl.b) * A.phi_size + A.phi1_off +
              (static_cast<int64_t>(b) * Ro + row) * A.n_frames + tl.t0 + w] = v;
        else
          out[static_cast<int64_t>(tl.b) * A.v2_tot + A.v2_off[tl.a] +
              (static_cast<int64_t>(b) * Ro + row) * stride + tl.t0 + w] = v;
      }
    }
    __syncthreads();
  }
}

// Adjoint of k_freq_fwd at the same input (recomputed): given the gradient
// of its outputs (dPhi first-order block for MODE 1, dV2 for MODE 2), writes
// the gradient of its input columns (dS1 real for MODE 1, dY2 for MODE 2).
template <int MODE>
__global__ void __launch_bounds__(kThreads)
k_freq_adj(FreqArgs A, const Tile* __restrict__ tiles, const float* S1, const float2* __restrict__ Y2,
           const float* __restrict__ dout, float* dS1, float2* __restrict__ dY2) {
  extern __shared__ float2 sm[];
  const Tile tl = tiles[blockIdx.x];
  const int W = A.W, Nfr = A.N_fr, WN = W * Nfr;
  const FreqSmem S = freq_smem_carve(A, sm, 5);
  float2* buf0 = S.buf;
  float2* buf1 = buf0 + WN;
  float2* zb = buf1 + WN;
  float2* f1 = zb + WN;
  float2* f2 = f1 + WN;
  freq_stage_tables(A, S);
  int stride, n1m;
  freq_load_columns<MODE>(A, tl, S1, Y2, buf0, stride, n1m);
  __syncthreads();
  float2* yh = cta_fft_il<false>(buf0, buf1, A.logNfr, A.logW, S.tw, A.logNfr);
  float2* D = (yh == buf0) ? buf1 : buf0;
  for (int i = threadIdx.x; i < WN; i += blockDim.x) D[i] = make_float2(0.f, 0.f);
  const float invNfr = 1.f / static_cast<float>(Nfr);
  const int Ro = A.R_out, lRo = A.logRout;
  for (int c = 0; c < A.n_chunks; ++c) {
    const FreqChunk& ch = S.chk[c];
    const int lR = A.logNfr - ch.k, R = 1 << lR;
    const int lc = ceil_log2(ch.n) + A.logW, cnt = 1 << lc;
    const float invR = 1.f / static_cast<float>(R);
    // Recompute z and keep it in zb.
    freq_fold(A, S, ch, lc, yh, f1, lR);
    __syncthreads();
    float2* z = cta_fft_il<true>(f1, f2, lR, lc, S.tw, A.logNfr);
    float2* dwb = (z == f1) ? f2 : f1;
    for (int i = threadIdx.x; i < (R << lc); i += blockDim.x) zb[i] = z[i];
    float2* du;
    float2* other;
    if (A.unpooled_f) {  // no phi_F: the output gradient is d|Y_fr| itself
      for (int i = threadIdx.x; i < (R << lc); i += blockDim.x) {
        const int f = i & (cnt - 1), row = i >> lc;
        const int bc = f >> A.logW, w = f & (W - 1);
        float v = 0.f;
        if (bc < ch.n && w < tl.ncols) {
          const int b = ch.beta[bc];
          const int64_t r = A.row_off[b] + row;
          if (MODE == 1)
            v = dout[static_cast<int64_t>(tl.b) * A.phi_size + A.phi1_off + r * A.n_frames + tl.t0 + w];
          else
            v = dout[static_cast<int64_t>(tl.b) * A.v2_tot + A.v2_off[tl.a] + r * stride + tl.t0 + w];
        }
        dwb[i] = make_float2(v, 0.f);
      }
      __syncthreads();
      du = dwb;
      other = z;
    } else {
    // dw: the output gradient of the chunk, interleaved [row][f].
    for (int i = threadIdx.x; i < (Ro << lc); i += blockDim.x) {
      const int f = i & (cnt - 1), row = i >> lc;
      const int bc = f >> A.logW, w = f & (W - 1);
      float v = 0.f;
      if (bc < ch.n && w < tl.ncols) {
        const int b = ch.beta[bc];
        if (MODE == 1)
          v = dout[static_cast<int64_t>(tl.b) * A.phi_size + A.phi1_off +
                   (static_cast<int64_t>(b) * Ro + row) * A.n_frames + tl.t0 + w];
        else
          v = dout[static_cast<int64_t>(tl.b) * A.v2_tot + A.v2_off[tl.a] +
                   (static_cast<int64_t>(b) * Ro + row) * stride + tl.t0 + w];
      }
      dwb[i] = make_float2(v, 0.f);
    }
    __syncthreads();
    float2* dW = cta_fft_il<false>(dwb, z, lRo, lc, S.tw, A.logNfr);
    float2* X = (dW == dwb) ? z : dwb;
    // du_hat[m] = (1/R) phi_F level_k(m) dW[m mod R_out]   (adjoint of the pooling fold)
    const float* lev = S.tab + (A.n_beta2 + 1 + ch.k) * Nfr;
    {
      const int lp = lc - 1;
      const float4* dW4 = reinterpret_cast<const float4*>(dW);
      float4* X4 = reinterpret_cast<float4*>(X);
      for (int i = threadIdx.x; i < (R << lp); i += kThreads) {
        const int fp = i & ((1 << lp) - 1), m = i >> lp;
        const float sc = __ldg(lev + m) * invR;
        const float4 v = dW4[((m & (Ro - 1)) << lp) + fp];
        X4[i] = make_float4(v.x * sc, v.y * sc, v.z * sc, v.w * sc);
      }
    }
    __syncthreads();
    du = cta_fft_il<true>(X, dW, lR, lc, S.tw, A.logNfr);
    other = (du == X) ? dW : X;
    }
    // dz = Re(du) z / |z|  (0 where z = 0)
    for (int i = threadIdx.x; i < (R << lc); i += kThreads) {
      const float gr = du[i].x;
      const float2 v = zb[i];
      const float mg = sqrtf(v.x * v.x + v.y * v.y);
      du[i] = mg > 0.f ? make_float2(gr * v.x / mg, gr * v.y / mg) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* dZ = cta_fft_il<false>(du, other, lR, lc, S.tw, A.logNfr);
    // D[m][w] += (1/N_fr) sum_beta psi_beta(s(m)) dZ_beta[m mod R][w]
    {
      const int lWp = A.logW - 1, lp = lc - 1;
      const float4* dZ4 = reinterpret_cast<const float4*>(dZ);
      float4* D4 = reinterpret_cast<float4*>(D);
      for (int i = threadIdx.x; i < (WN >> 1); i += kThreads) {
        const int wp = i & ((1 << lWp) - 1), m = i >> lWp;
        const int sgn = m < (Nfr >> 1) ? m : m - Nfr;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int bc = 0; bc < ch.n; ++bc) {
          const int b = ch.beta[bc];
          const int2 bd = S.band[b];
          if (sgn < bd.x || sgn > bd.y) continue;
          const float gg = __ldg(S.tab + b * Nfr + m);
          const float4 v = dZ4[((m & (R - 1)) << lp) + (bc << lWp) + wp];
          acc.x += gg * v.x;
          acc.y += gg * v.y;
          acc.z += gg * v.z;
          acc.w += gg * v.w;
        }
        float4 d = D4[i];
        d.x += acc.x * invNfr;
        d.y += acc.y * invNfr;
        d.z += acc.z * invNfr;
        d.w += acc.w * invNfr;
        D4[i] = d;
      }
    }
    __syncthreads();
  }
  float2* dy = cta_fft_il<true>(D, f1, A.logNfr, A.logW, S.tw, A.logNfr);
  for (int i = threadIdx.x; i < n1m * W; i += blockDim.x) {
    const int w = i & (W - 1), r = i >> A.logW;
    if (w < tl.ncols) {
      const float2 v = dy[i];
      if (MODE == 1)
        dS1[(static_cast<int64_t>(tl.b) * A.N1 + r) * A.n_frames + tl.t0 + w] = v.x;
      else
        dY2[static_cast<int64_t>(tl.b) * A.y2_tot + A.y2_off[tl.a] + static_cast<int64_t>(r) * stride + tl.t0 + w] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// phi_T averaging of the second order (Eq. (5)) as a decimating FIR and its
// adjoint.  out[f] = sum_t v[t] g_s[(f D - t) mod L], L = N/2^s, D = T/2^s.
// ---------------------------------------------------------------------------
struct PoolArgs {
  int logN, lT, n_frames, R_out, n_beta2, n_active;
  int rows2;  // rows of one second-order block (n_beta2 R_out when pooled along n1)
  int64_t phi_size, v2_tot;
  const int* s2;
  const int64_t* v2_off;
  const int64_t* phi2_off;
  const float* taps;
  const int64_t* tap_off;
  const int* pool_w;  // per active n2: banded half-width, 0 = dense
};

// Both directions are dense products with the tap matrix
// G[t][f] = g_s[(f D - t) mod L]:  Phi2[rows x nf] = V2[rows x L] G and
// dV2[rows x L] = dPhi2[rows x nf] G^T, where rows = (1+2K) R_out paths-rows
// of one (clip, n2).  Register-blocked SIMT tiles; V2 is read once.
constexpr int kPoolRows = 64;   // rows per CTA
constexpr int kPoolK = 32;      // time samples per shared-memory stage (forward)
constexpr int kPoolT = 64;      // time samples per CTA (adjoint)

// Forward, split over time: a CTA owns a 64-row x 8*FPT-frame tile of one
// (clip, n2) and the time samples [split * split_len, +split_len); thread
// (ty = tid / 8, tx = tid % 8) owns rows ty + 32 i (i < 2) and frames
// tx + 8 j (j < FPT).  Partial sums go to `part`, reduced in a fixed order
// by k_pool_reduce (deterministic).
template <int FPT>
__global__ void __launch_bounds__(kThreads)
k_pool_fwd(PoolArgs A, const float* __restrict__ V2, float* __restrict__ part, const int4* __restrict__ tiles,
           int split_len) {
  __shared__ float Vs[kPoolK][kPoolRows + 1];
  __shared__ float Gs[kPoolK][8 * FPT];
  const int4 tl = tiles[blockIdx.x];  // (clip, active n2, row tile, split)
  const int b = tl.x, a = tl.y, split = tl.w;
  const int fb = blockIdx.y * 8 * FPT;
  const int s = A.s2[a];
  const int lL = A.logN - s, L = 1 << lL;
  const int D = 1 << (A.lT - s);
  const int rows = A.rows2;
  const int r0 = tl.z * kPoolRows;
  const int tbeg = split * split_len, tend = min(L, tbeg + split_len);
  const float* v = V2 + static_cast<int64_t>(b) * A.v2_tot + A.v2_off[a];
  const float* g = A.taps + A.tap_off[s];
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  float acc[2][FPT];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < FPT; ++j) acc[i][j] = 0.f;
  for (int t0 = tbeg; t0 < tend; t0 += kPoolK) {
    for (int i = threadIdx.x; i < kPoolRows * kPoolK; i += blockDim.x) {
      const int rr = i / kPoolK, tt = i % kPoolK;
      const int r = r0 + rr;
      Vs[tt][rr] = (r < rows && t0 + tt < tend) ? v[static_cast<int64_t>(r) * L + t0 + tt] : 0.f;
    }
    for (int i = threadIdx.x; i < kPoolK * 8 * FPT; i += blockDim.x) {
      const int tt = i % kPoolK, ff = i / kPoolK;  // consecutive threads: consecutive taps
      const int f = fb + ff;
      Gs[tt][ff] = (f < A.n_frames && t0 + tt < tend) ? g[(f * D - (t0 + tt)) & (L - 1)] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int tt = 0; tt < kPoolK; ++tt) {
      const float v0 = Vs[tt][ty], v1 = Vs[tt][ty + 32];
#pragma unroll
      for (int j = 0; j < FPT; ++j) {
        const float gg = Gs[tt][tx + 8 * j];
        acc[0][j] += v0 * gg;
        acc[1][j] += v1 * gg;
      }
    }
    __syncthreads();
  }
  // partial layout: [tile index][64 rows][n_frames]
  float* out = part + static_cast<int64_t>(blockIdx.x) * kPoolRows * A.n_frames;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int rr = ty + 32 * i;
#pragma unroll
    for (int j = 0; j < FPT; ++j) {
      const int f = fb + tx + 8 * j;
      if (f < A.n_frames) out[rr * A.n_frames + f] = acc[i][j];
    }
  }
}

// Forward, split over time, register-blocked: a CTA of 4 FR threads owns a
// 64-row x FR-frame tile of one (clip, n2) and the time samples
// [split * split_len, +split_len).  Warp w accumulates frames 8 w .. 8 w + 7
// and lane l rows 2 l, 2 l + 1: per time sample one float2 of V2 rows and two
// warp-broadcast float4 of taps feed 16 FMAs.  Shared layouts are swizzled so
// that neither the transposing stores nor the reads conflict:
//   Vs[t][2 ((r >> 1) ^ sv(t)) + (r & 1)],  sv(t) = 2 ((t >> 2) & 7)
//   Gs[t][f ^ (8 (t & 3))]
// The next chunk's V2 and taps are read into registers while the current one
// is used.  Partial sums as k_pool_fwd (reduced by k_pool_reduce).
template <int FR>
__global__ void __launch_bounds__(4 * FR)
k_pool_fwd2(PoolArgs A, const float* __restrict__ V2, float* __restrict__ part, const int4* __restrict__ tiles,
            int split_len) {
  constexpr int NT = 4 * FR;                          // threads
  constexpr int VPT = (kPoolRows * kPoolK / 4) / NT;  // float4 of V2 per thread per chunk (>= 1)
  __shared__ __align__(16) float Vs[kPoolK][kPoolRows];
  __shared__ __align__(16) float Gs[kPoolK][FR];
  const int4 tl = tiles[blockIdx.x];  // (clip, active n2, row tile, split)
  const int b = tl.x, a = tl.y, split = tl.w;
  const int fb = blockIdx.y * FR;
  const int s = A.s2[a];
  const int lL = A.logN - s, L = 1 << lL;
  const int D = 1 << (A.lT - s);
  const int rows = A.rows2;
  const int r0 = tl.z * kPoolRows;
  const int tbeg = split * split_len, tend = min(L, tbeg + split_len);
  const float* v = V2 + static_cast<int64_t>(b) * A.v2_tot + A.v2_off[a];
  const float* g = A.taps + A.tap_off[s];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[2][8];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  // V2 chunk: float4 q = row q / 8, samples 4 (q % 8) .. + 3 (coalesced rows).
  float4 pre[VPT];
  auto load_v = [&](int t0) {
#pragma unroll
    for (int u = 0; u < VPT; ++u) {
      const int q = threadIdx.x + u * NT;
      const int rr = q >> 3, tq = (q & 7) * 4;
      const int r = r0 + rr;
      pre[u] = (r < rows && t0 + tq < tend)
                   ? *reinterpret_cast<const float4*>(v + static_cast<int64_t>(r) * L + t0 + tq)
                   : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  // Taps: element e = tid + u NT, block e / 32 covers samples 4 (blk % 8) .. + 3
  // and frames 8 (blk / 8) .. + 7; lane: sample + (lane & 3), frame + (lane >> 2).
  float gpre[8];
  auto load_g = [&](int t0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = threadIdx.x + u * NT, blk = e >> 5, ln = e & 31;
      const int tt = 4 * (blk & 7) + (ln & 3), ff = 8 * (blk >> 3) + (ln >> 2);
      const int f = fb + ff;
      gpre[u] = (f < A.n_frames && t0 + tt < tend) ? __ldg(g + ((f * D - (t0 + tt)) & (L - 1))) : 0.f;
    }
  };
  load_v(tbeg);
  load_g(tbeg);
  for (int t0 = tbeg; t0 < tend; t0 += kPoolK) {
#pragma unroll
    for (int u = 0; u < VPT; ++u) {
      const int q = threadIdx.x + u * NT;
      const int rr = q >> 3, tq = (q & 7) * 4;
      const float x[4] = {pre[u].x, pre[u].y, pre[u].z, pre[u].w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int t = tq + e;
        Vs[t][2 * ((rr >> 1) ^ (2 * ((t >> 2) & 7))) + (rr & 1)] = x[e];
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = threadIdx.x + u * NT, blk = e >> 5, ln = e & 31;
      const int tt = 4 * (blk & 7) + (ln & 3), ff = 8 * (blk >> 3) + (ln >> 2);
      Gs[tt][ff ^ (8 * (tt & 3))] = gpre[u];
    }
    __syncthreads();
    if (t0 + kPoolK < tend) {
      load_v(t0 + kPoolK);
      load_g(t0 + kPoolK);
    }
#pragma unroll 8
    for (int tt = 0; tt < kPoolK; ++tt) {
      const float2 vv = *reinterpret_cast<const float2*>(&Vs[tt][2 * (lane ^ (2 * ((tt >> 2) & 7)))]);
      const int gc = (8 * warp) ^ (8 * (tt & 3));
      const float4 g0 = *reinterpret_cast<const float4*>(&Gs[tt][gc]);
      const float4 g1 = *reinterpret_cast<const float4*>(&Gs[tt][gc + 4]);
      const float gf[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        acc[0][j] = fmaf(vv.x, gf[j], acc[0][j]);
        acc[1][j] = fmaf(vv.y, gf[j], acc[1][j]);
      }
    }
    __syncthreads();
  }
  // partial layout: [tile index][64 rows][n_frames]
  float* out = part + static_cast<int64_t>(blockIdx.x) * kPoolRows * A.n_frames;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int rr = 2 * lane + i;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int f = fb + 8 * warp + j;
      if (f < A.n_frames) out[rr * A.n_frames + f] = acc[i][j];
    }
  }
}

// Phi2[b][a][r][f] = sum over splits (ascending) of the partials.
__global__ void __launch_bounds__(kThreads)
k_pool_reduce(PoolArgs A, const float* __restrict__ part, float* __restrict__ phi, const int* __restrict__ tile0,
              int split_len, int64_t total) {
  const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int rows = A.rows2;
  const int64_t per_a = static_cast<int64_t>(rows) * A.n_frames;
  const int64_t ba = idx / per_a;
  const int rf = static_cast<int>(idx % per_a);
  const int r = rf / A.n_frames, f = rf % A.n_frames;
  const int a = static_cast<int>(ba % A.n_active), b = static_cast<int>(ba / A.n_active);
  if (A.pool_w[a]) return;  // written by k_pool_fwd_band
  const int L = 1 << (A.logN - A.s2[a]);
  const int nsplit = (L + split_len - 1) / split_len;
  // tiles of (b, a) start at tile0[ba]; ordered by row tile then split
  const int64_t t = tile0[ba] + static_cast<int64_t>(r / kPoolRows) * nsplit;
  const float* pp = part + (t * kPoolRows + (r % kPoolRows)) * A.n_frames + f;
  float acc = 0.f;
  for (int sp = 0; sp < nsplit; ++sp) acc += pp[static_cast<int64_t>(sp) * kPoolRows * A.n_frames];
  phi[static_cast<int64_t>(b) * A.phi_size + A.phi2_off[a] + static_cast<int64_t>(r) * A.n_frames + f] = acc;
}

// Banded forward: a CTA owns 64 rows x 32 frames f0 .. f0+31 of one (clip,
// n2) and sums over the window t in [f0 D - W, (f0+31) D + W] (mod L), the
// only samples whose taps reach those frames (taps beyond W are below 2^-40 of
// the peak).  Writes Phi2 directly.  Thread mapping as k_pool_fwd<4>.
__global__ void __launch_bounds__(kThreads)
k_pool_fwd_band(PoolArgs A, const float* __restrict__ V2, float* __restrict__ phi, const int4* __restrict__ tiles) {
  constexpr int FPT = 4;
  __shared__ float Vs[kPoolK][kPoolRows + 1];
  __shared__ float Gs[kPoolK][8 * FPT];
  const int4 tl = tiles[blockIdx.x];  // (clip, active n2, row tile, frame block)
  const int b = tl.x, a = tl.y;
  const int f0 = tl.w * 8 * FPT;
  const int s = A.s2[a];
  const int lL = A.logN - s, L = 1 << lL;
  const int D = 1 << (A.lT - s);
  const int W = A.pool_w[a];
  const int rows = A.rows2;
  const int r0 = tl.z * kPoolRows;
  const int tbeg = f0 * D - W, tend = (f0 + 8 * FPT - 1) * D + W + 1;
  const float* v = V2 + static_cast<int64_t>(b) * A.v2_tot + A.v2_off[a];
  const float* g = A.taps + A.tap_off[s];
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  float acc[2][FPT];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < FPT; ++j) acc[i][j] = 0.f;
  for (int t0 = tbeg; t0 < tend; t0 += kPoolK) {
    for (int i = threadIdx.x; i < kPoolRows * kPoolK; i += blockDim.x) {
      const int rr = i / kPoolK, tt = i % kPoolK;
      const int r = r0 + rr;
      Vs[tt][rr] = (r < rows && t0 + tt < tend) ? v[static_cast<int64_t>(r) * L + ((t0 + tt) & (L - 1))] : 0.f;
    }
    for (int i = threadIdx.x; i < kPoolK * 8 * FPT; i += blockDim.x) {
      const int tt = i % kPoolK, ff = i / kPoolK;
      const int f = f0 + ff;
      Gs[tt][ff] = (f < A.n_frames && t0 + tt < tend) ? g[(f * D - (t0 + tt)) & (L - 1)] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int tt = 0; tt < kPoolK; ++tt) {
      const float v0 = Vs[tt][ty], v1 = Vs[tt][ty + 32];
#pragma unroll
      for (int j = 0; j < FPT; ++j) {
        const float gg = Gs[tt][tx + 8 * j];
        acc[0][j] += v0 * gg;
        acc[1][j] += v1 * gg;
      }
    }
    __syncthreads();
  }
  float* out = phi + static_cast<int64_t>(b) * A.phi_size + A.phi2_off[a];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int r = r0 + ty + 32 * i;
    if (r >= rows) continue;
#pragma unroll
    for (int j = 0; j < FPT; ++j) {
      const int f = f0 + tx + 8 * j;
      if (f < A.n_frames) out[static_cast<int64_t>(r) * A.n_frames + f] = acc[i][j];
    }
  }
}

// Adjoint: a CTA owns 64 rows x 64 time samples; thread (ty = tid / 16,
// tx = tid % 16) computes rows ty + 16 i (i < 4) and times tx + 16 j (j < 4).
// Adjoint, dense groups: dV2[rows x L] = dPhi2[rows x nf] G^T on tiles of 64
// rows x (kPoolAdjSub x 128) samples: the CTA loads its dPhi2 rows once, then
// walks its 128-sample sub-tiles, gathering the next sub-tile's taps into
// registers while it computes the current one.  Thread (tr = tid % 16,
// tt = tid / 16) owns rows 4 tr .. 4 tr + 3 and samples 8 tt .. 8 tt + 7 of a
// sub-tile (one float4 of dPhi2 rows and two of taps per frame), written as
// float4 pairs.  Frames are taken 32 at a time.
constexpr int kPoolAdjSub = 4;

__global__ void __launch_bounds__(kThreads)
k_pool_adj2(PoolArgs A, const float* __restrict__ dphi, float* __restrict__ dV2, const int4* __restrict__ tiles) {
  __shared__ __align__(16) float Ps[32][kPoolRows + 4];
  __shared__ __align__(16) float Gs[32][128 + 4];
  const int4 tl = tiles[blockIdx.x];  // (b, a, row tile, group of kPoolAdjSub 128-sample tiles)
  const int b = tl.x, a = tl.y;
  const int s = A.s2[a];
  const int lL = A.logN - s, L = 1 << lL;
  const int D = 1 << (A.lT - s);
  const int rows = A.rows2;
  const int r0 = tl.z * kPoolRows;
  const float* dp = dphi + static_cast<int64_t>(b) * A.phi_size + A.phi2_off[a];
  const float* g = A.taps + A.tap_off[s];
  float* out = dV2 + static_cast<int64_t>(b) * A.v2_tot + A.v2_off[a];
  const int tr = threadIdx.x & 15, tt = threadIdx.x >> 4;
  float gpre[16];
  auto load_g = [&](int f0, int t0) {  // 32 frames x 128 samples: element i = (frame i / 128, sample i % 128)
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int i = threadIdx.x + u * kThreads;
      const int f = f0 + (i >> 7), t = t0 + (i & 127);
      gpre[u] = (f < A.n_frames && t < L) ? __ldg(g + ((f * D - t) & (L - 1))) : 0.f;
    }
  };
  const int tbase = tl.w * (kPoolAdjSub * 128);
  const int nsub = min(kPoolAdjSub, (L - tbase + 127) / 128);
  for (int f0 = 0; f0 < A.n_frames; f0 += 32) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 8; ++u) {  // 64 rows x 32 frames
      const int i = threadIdx.x + u * kThreads;
      const int rr = i >> 5, ff = i & 31;
      const int r = r0 + rr, f = f0 + ff;
      Ps[ff][rr] = (r < rows && f < A.n_frames) ? dp[static_cast<int64_t>(r) * A.n_frames + f] : 0.f;
    }
    load_g(f0, tbase);
    for (int sub = 0; sub < nsub; ++sub) {
      const int t0 = tbase + sub * 128;
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int i = threadIdx.x + u * kThreads;
        Gs[i >> 7][i & 127] = gpre[u];
      }
      __syncthreads();
      if (sub + 1 < nsub) load_g(f0, t0 + 128);
      float acc[4][8];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll 8
      for (int ff = 0; ff < 32; ++ff) {
        const float4 pv = *reinterpret_cast<const float4*>(&Ps[ff][4 * tr]);
        const float4 g0 = *reinterpret_cast<const float4*>(&Gs[ff][8 * tt]);
        const float4 g1 = *reinterpret_cast<const float4*>(&Gs[ff][8 * tt + 4]);
        const float pr[4] = {pv.x, pv.y, pv.z, pv.w};
        const float gt[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(pr[i], gt[j], acc[i][j]);
      }
      // More than 32 frames: accumulate this frame block into dV2 (first block stores).
      const int t = t0 + 8 * tt;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = r0 + 4 * tr + i;
        if (r >= rows || t >= L) continue;
        float* o = out + static_cast<int64_t>(r) * L + t;
        if (L >= 8) {  // L is a power of two: t + 8 <= L and 16-byte aligned rows
          float4* o4 = reinterpret_cast<float4*>(o);
          float4 x0 = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
          float4 x1 = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
          if (f0 > 0) {
            const float4 y0 = o4[0], y1 = o4[1];
            x0 = make_float4(y0.x + x0.x, y0.y + x0.y, y0.z + x0.z, y0.w + x0.w);
            x1 = make_float4(y1.x + x1.x, y1.y + x1.y, y1.z + x1.z, y1.w + x1.w);
          }
          o4[0] = x0;
          o4[1] = x1;
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (t + j < L) o[j] = (f0 > 0 ? o[j] : 0.f) + acc[i][j];
        }
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads)
k_pool_adj(PoolArgs A, const float* __restrict__ dphi, float* __restrict__ dV2, const int4* __restrict__ tiles) {
  __shared__ float Ps[32][kPoolRows + 1];
  __shared__ float Gs[32][kPoolT + 1];
  const int4 tl = tiles[blockIdx.x];  // (b, a, row tile, time tile)
  const int b = tl.x, a = tl.y;
  const int s = A.s2[a];
  const int lL = A.logN - s, L = 1 << lL;
  const int D = 1 << (A.lT - s);
  const int rows = A.rows2;
  const int r0 = tl.z * kPoolRows, t0 = tl.w * kPoolT;
  const float* dp = dphi + static_cast<int64_t>(b) * A.phi_size + A.phi2_off[a];
  const float* g = A.taps + A.tap_off[s];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  // Frames whose taps reach [t0, t0 + 64): all of them (dense), or the band
  // f D in [t0 - W, t0 + 63 + W], taken mod n_frames (banded).
  const int W = A.pool_w[a];
  const int fbeg = W ? -((W - t0 + D - 1) >> (A.lT - s)) : 0;  // floor((t0 - W) / D); t0 - W may be < 0
  const int fend = W ? ((t0 + kPoolT - 1 + W) >> (A.lT - s)) + 1 : A.n_frames;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int f0 = fbeg; f0 < fend; f0 += 32) {
    for (int i = threadIdx.x; i < kPoolRows * 32; i += blockDim.x) {
      const int rr = i / 32, ff = i % 32;
      const int r = r0 + rr, f = f0 + ff;
      Ps[ff][rr] = (r < rows && f < fend) ? dp[static_cast<int64_t>(r) * A.n_frames + (f & (A.n_frames - 1))] : 0.f;
    }
    for (int i = threadIdx.x; i < 32 * kPoolT; i += blockDim.x) {
      const int ff = i / kPoolT, tt = i % kPoolT;
      const int f = f0 + ff, t = t0 + tt;
      Gs[ff][tt] = (f < fend && t < L) ? g[(f * D - t) & (L - 1)] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int ff = 0; ff < 32; ++ff) {
      float pv[4], gv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) pv[i] = Ps[ff][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) gv[j] = Gs[ff][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += pv[i] * gv[j];
    }
    __syncthreads();
  }
  float* out = dV2 + static_cast<int64_t>(b) * A.v2_tot + A.v2_off[a];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty + 16 * i;
    if (r >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int t = t0 + tx + 16 * j;
      if (t < L) out[static_cast<int64_t>(r) * L + t] = acc[i][j];
    }
  }
}

// ---------------------------------------------------------------------------
// Adjoint gathers of the time-axis filterings.
// ---------------------------------------------------------------------------
struct GradArgs {
  int logN, N1, n_frames, n_active;
  int64_t u1_tot, y2_tot;
  const FiltD* psi1;
  const FiltD* psi2;
  FiltD phiT;
  const int* s2;
  const int* n1max_act;
  const int* act_n2;
  const int64_t* y2_off;
  const int64_t* u1_off;
};

// dU1hat[b][n1][m] = (1/L1) [ sum_{n2: n1 < n1max} lev_{psi_n2}(m) dZ2[n2][n1][m mod L2]
//                             + lev_{phi_T}(m) dS1hat[n1][m mod N/T] ]
__global__ void __launch_bounds__(kThreads)
k_dU1(GradArgs A, const Job* __restrict__ jobs, const int2* __restrict__ blocks, const float2* __restrict__ dZ2,
      const float2* __restrict__ dS1h, float2* __restrict__ dU1h) {
  // blocks: (job, block in its row) per block of a 1-D grid; null: a 2-D grid of (block, job).
  const int2 bk = blocks ? blocks[blockIdx.x] : make_int2(int(blockIdx.y), int(blockIdx.x));
  const Job jb = jobs[bk.x];
  const int lL1 = jb.lslog, L1 = 1 << lL1;
  const int m = bk.y * blockDim.x + threadIdx.x;
  if (m >= L1) return;
  const int n1 = jb.filt, b = jb.b;
  float2 acc = make_float2(0.f, 0.f);
  for (int a = 0; a < A.n_active; ++a) {
    if (n1 >= A.n1max_act[a]) continue;
    const int L2 = 1 << (A.logN - A.s2[a]);
    const float lev = band_lev(m, L1, A.psi2[A.act_n2[a]]);
    if (lev != 0.f) {
      const float2 v = dZ2[static_cast<int64_t>(b) * A.y2_tot + A.y2_off[a] + static_cast<int64_t>(n1) * L2 +
                           (m & (L2 - 1))];
      acc.x += lev * v.x;
      acc.y += lev * v.y;
    }
  }
  {
    const float lev = band_lev(m, L1, A.phiT);
    if (lev != 0.f) {
      const float2 v = dS1h[(static_cast<int64_t>(b) * A.N1 + n1) * A.n_frames + (m & (A.n_frames - 1))];
      acc.x += lev * v.x;
      acc.y += lev * v.y;
    }
  }
  dU1h[jb.dst + m] = cscale(acc, 1.f / static_cast<float>(L1));
}

// dXhat[b][m] = (1/N) [ sum_n1 psi_n1(s) dZ1[n1][m mod L1] + phi_T(s) dS0hat[m mod N/T] ]
__global__ void __launch_bounds__(kThreads)
k_dX(GradArgs A, int64_t total, const float2* __restrict__ dZ1, const float2* __restrict__ dS0h,
     float2* __restrict__ dXh) {
  const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int N = 1 << A.logN;
  const int b = static_cast<int>(idx >> A.logN);
  const int m = static_cast<int>(idx & (N - 1));
  const int s = m < (N >> 1) ? m : m - N;
  float2 acc = make_float2(0.f, 0.f);
  for (int n1 = 0; n1 < A.N1; ++n1) {
    const FiltD f = A.psi1[n1];
    if (s < f.lo || s > f.hi) continue;
    const int L1 = 1 << (A.logN - f.k);
    const float g = fval(f, s);
    const float2 v = dZ1[static_cast<int64_t>(b) * A.u1_tot + A.u1_off[n1] + (m & (L1 - 1))];
    acc.x += g * v.x;
    acc.y += g * v.y;
  }
  if (dS0h && s >= A.phiT.lo && s <= A.phiT.hi) {
    const float g = fval(A.phiT, s);
    const float2 v = dS0h[static_cast<int64_t>(b) * A.n_frames + (m & (A.n_frames - 1))];
    acc.x += g * v.x;
    acc.y += g * v.y;
  }
  dXh[idx] = cscale(acc, 1.f / static_cast<float>(N));
}

// ---------------------------------------------------------------------------
// Loss E_b = sum (phi - target)^2 and dphi = 2 (phi - target); fixed-order
// block reduction (deterministic).  A NaN or infinite E_b sets g_nonfinite,
// which jtfs_status reports.
// ---------------------------------------------------------------------------
__device__ int g_nonfinite;

__global__ void __launch_bounds__(512)
k_loss(const float* __restrict__ phi, const float* __restrict__ tgt, float* __restrict__ dphi,
       float* __restrict__ loss, int64_t size) {
  __shared__ double red[512];
  const int b = blockIdx.x;
  const float* p = phi + static_cast<int64_t>(b) * size;
  const float* t = tgt + static_cast<int64_t>(b) * size;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < size; i += blockDim.x) {
    const float d = p[i] - t[i];
    if (dphi) dphi[static_cast<int64_t>(b) * size + i] = 2.f * d;
    acc += static_cast<double>(d) * d;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    loss[b] = static_cast<float>(red[0]);
    if (!isfinite(red[0])) atomicOr(&g_nonfinite, 1);
  }
}

// Large Phi: the same loss over `parts` CTAs per clip.  Part j of clip b
// sums entries [j chunk, (j+1) chunk) into part_sum[b][j] (double, fixed
// order); k_loss_sum then adds the parts of each clip in a fixed order.
__global__ void __launch_bounds__(512)
k_loss_part(const float* __restrict__ phi, const float* __restrict__ tgt, float* __restrict__ dphi,
            double* __restrict__ part_sum, int64_t size, int64_t chunk) {
  __shared__ double red[512];
  const int b = blockIdx.y;
  const int64_t lo = static_cast<int64_t>(blockIdx.x) * chunk, hi = min(size, lo + chunk);
  const float* p = phi + static_cast<int64_t>(b) * size;
  const float* t = tgt + static_cast<int64_t>(b) * size;
  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const float d = p[i] - t[i];
    if (dphi) dphi[static_cast<int64_t>(b) * size + i] = 2.f * d;
    acc += static_cast<double>(d) * d;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part_sum[static_cast<int64_t>(b) * gridDim.x + blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(256)
k_loss_sum(const double* __restrict__ part_sum, float* __restrict__ loss, int parts) {
  __shared__ double red[256];
  const double* ps = part_sum + static_cast<int64_t>(blockIdx.x) * parts;
  double acc = 0.0;
  for (int j = threadIdx.x; j < parts; j += blockDim.x) acc += ps[j];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    loss[blockIdx.x] = static_cast<float>(red[0]);
    if (!isfinite(red[0])) atomicOr(&g_nonfinite, 1);
  }
}

__global__ void __launch_bounds__(kThreads)
k_adam(float* __restrict__ y, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
       int64_t n, float lr, float c1, float c2) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  y[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
}

// Adam with the 1-based step index read from device memory (graph replay).
// The bias corrections are computed once per block in double, as metamer_step
// computes them on the host, so both give the same iterates.
__global__ void __launch_bounds__(kThreads)
k_adam_counted(float* __restrict__ y, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
               int64_t n, float lr, const int* __restrict__ step) {
  __shared__ float corr[2];
  if (threadIdx.x == 0) {
    const double t = static_cast<double>(*step);
    corr[0] = static_cast<float>(1.0 / (1.0 - pow(0.9, t)));
    corr[1] = static_cast<float>(1.0 / (1.0 - pow(0.999, t)));
  }
  __syncthreads();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float c1 = corr[0], c2 = corr[1];
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  y[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
}

__global__ void k_step_next(int* step) { *step += 1; }

// ---------------------------------------------------------------------------
// Reconstruction variant of §2.3: coloured initialisation and momentum
// descent with the bold-driver step size.
// ---------------------------------------------------------------------------

// Per clip b (blockIdx.y): dst[b dst_stride + dst_off + i] (+)= src[b src_stride + src_off + i], i < len.
// Moves blocks between Phi and the workspace for the unpooled outputs.
__global__ void __launch_bounds__(kThreads)
k_copy_block(const float* __restrict__ src, int64_t src_stride, int64_t src_off, float* __restrict__ dst,
             int64_t dst_stride, int64_t dst_off, int64_t len, int accumulate) {
  const float* a = src + static_cast<int64_t>(blockIdx.y) * src_stride + src_off;
  float* d = dst + static_cast<int64_t>(blockIdx.y) * dst_stride + dst_off;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < len;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    d[i] = accumulate ? d[i] + a[i] : a[i];
}

// rows[r][t] *= gain[r mod n_rows] over `total` = batch * n_rows * row_len entries.
__global__ void __launch_bounds__(kThreads)
k_scale_rows(float* __restrict__ rows, const float* __restrict__ gain, int n_rows, int log_len, int64_t total) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= total) return;
  rows[i] *= gain[static_cast<int>((i >> log_len) % n_rows)];
}

// Per clip b (one CTA): y[b] *= ||x[b]|| / ||y[b]|| (y[b] = 0 when ||y[b]|| = 0);
// both squared norms summed in double in a fixed order.
__global__ void __launch_bounds__(512)
k_energy_match(const float* __restrict__ x, float* __restrict__ y, int64_t n) {
  __shared__ double red[2][512];
  const float* xb = x + static_cast<int64_t>(blockIdx.x) * n;
  float* yb = y + static_cast<int64_t>(blockIdx.x) * n;
  double sx = 0.0, sy = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double a = xb[i], b = yb[i];
    sx += a * a;
    sy += b * b;
  }
  red[0][threadIdx.x] = sx;
  red[1][threadIdx.x] = sy;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  const float scale = red[1][0] > 0.0 ? static_cast<float>(sqrt(red[0][0] / red[1][0])) : 0.f;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) yb[i] *= scale;
}

// Bold-driver decision per clip: state[b] = (mu, E_acc, accepted, evaluations).
// Accept when E <= E_acc (E_acc = +inf before the first evaluation; NaN is
// rejected): mu grows by 1.1 unless it is the first evaluation, E_acc = E.
// Otherwise mu halves.
__global__ void k_bold_decide(float4* __restrict__ state, const float* __restrict__ loss, int batch) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  float4 st = state[b];
  const float E = loss[b];
  const bool acc = E <= st.y;
  if (acc) {
    if (isfinite(st.y)) st.x *= 1.1f;
    st.y = E;
  } else {
    st.x *= 0.5f;
  }
  st.z = acc ? 1.f : 0.f;
  st.w += 1.f;
  state[b] = st;
}

// Momentum update after k_bold_decide (one thread per sample, clip = i >> log_n):
//   accepted: g_acc = g, u = m u - mu g, y += u;
//   rejected: y -= u (back to the accepted point), u = -mu g_acc, y += u.
__global__ void __launch_bounds__(kThreads)
k_momentum(float* __restrict__ y, float* __restrict__ u, float* __restrict__ g_acc, const float* __restrict__ g,
           const float4* __restrict__ state, int log_n, int64_t total, float m) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const float4 st = state[i >> log_n];
  float yi = y[i];
  float ui;
  if (st.z != 0.f) {
    const float gi = g[i];
    g_acc[i] = gi;
    ui = m * u[i] - st.x * gi;
  } else {
    yi -= u[i];
    ui = -st.x * g_acc[i];
  }
  u[i] = ui;
  y[i] = yi + ui;
}

// ---------------------------------------------------------------------------
// Orchestration.
// ---------------------------------------------------------------------------
struct Bufs {
  float2 *Xh, *U1h, *Zs, *dS1h, *Y2, *dY2, *dXh, *dS0h, *scr;
  float *S1, *V2, *phi, *dphi, *dy, *part;
  double* lossp;
};

Bufs bufs(const Plan& p, void* ws) {
  auto* c = static_cast<unsigned char*>(ws);
  Bufs w;
  w.Xh = reinterpret_cast<float2*>(c + p.ws_Xh);
  w.U1h = reinterpret_cast<float2*>(c + p.ws_U1h);
  w.Zs = reinterpret_cast<float2*>(c + p.ws_Zs);
  w.S1 = reinterpret_cast<float*>(c + p.ws_S1);
  w.dS1h = reinterpret_cast<float2*>(c + p.ws_dS1h);
  w.Y2 = reinterpret_cast<float2*>(c + p.ws_Y2);
  w.dY2 = reinterpret_cast<float2*>(c + p.ws_dY2);
  w.V2 = reinterpret_cast<float*>(c + p.ws_V2);
  w.phi = reinterpret_cast<float*>(c + p.ws_phi);
  w.dphi = reinterpret_cast<float*>(c + p.ws_dphi);
  w.dXh = reinterpret_cast<float2*>(c + p.ws_dXh);
  w.dS0h = reinterpret_cast<float2*>(c + p.ws_dS0h);
  w.dy = reinterpret_cast<float*>(c + p.ws_dy);
  w.scr = reinterpret_cast<float2*>(c + p.ws_scr);
  w.part = reinterpret_cast<float*>(c + p.ws_part);
  w.lossp = reinterpret_cast<double*>(c + p.ws_lossp);
  return w;
}

FreqArgs freq_args(const Plan& p, int mode) {
  FreqArgs A{};
  A.chunks = mode == 1 ? p.d_chunks1 : p.d_chunks2;
  A.n_chunks = static_cast<int>(mode == 1 ? p.chunks1.size() : p.chunks2.size());
  A.N1 = p.N1;
  A.N_fr = p.N_fr;
  A.logNfr = p.logNfr;
  A.R_out = p.R_out;
  A.logRout = p.logNfr - p.lF;
  A.n_frames = p.n_frames;
  A.logN = p.logN;
  A.W = p.freq_cols;
  int lw = 0;
  while ((1 << lw) < A.W) ++lw;
  A.logW = lw;
  A.n_beta1 = p.n_beta1;
  A.n_beta2 = p.n_beta2;
  A.n_ftab = p.n_ftab;
  A.ftab = p.d_ftab;
  A.phi_size = p.phi_size;
  A.phi1_off = p.phi1_off;
  A.y2_tot = p.y2_tot;
  A.v2_tot = p.v2_tot;
  A.beta = p.d_beta;
  A.phiF = p.h_phiF;
  A.s2 = p.d_s2;
  A.n1max_act = p.d_n1max_act;
  A.y2_off = p.d_y2_off;
  A.v2_off = p.d_v2_off;
  A.tw = p.d_tw;
  A.twlog = p.twlog;
  A.ftabc = p.d_ftabc;
  A.ftabc_off = p.d_ftabc_off;
  A.n_ftabc = static_cast<int>(p.h_ftabc.size());
  A.ftabc_phi = p.ftabc_phi;
  A.tab_smem = 0;
  for (int k = 0; k < 16; ++k) A.ftabc_lev[k] = p.ftabc_lev[k];
  A.unpooled_f = p.unpooled_f ? 1 : 0;
  A.row_off = p.d_row_off;
  return A;
}

PoolArgs pool_args(const Plan& p) {
  PoolArgs A{};
  A.logN = p.logN;
  A.lT = p.lT;
  A.n_frames = p.n_frames;
  A.R_out = p.R_out;
  A.n_beta2 = p.n_beta2;
  A.rows2 = p.rows2;
  A.n_active = p.n_active;
  A.phi_size = p.phi_size;
  A.v2_tot = p.v2_tot;
  A.s2 = p.d_s2;
  A.v2_off = p.d_v2_off;
  A.phi2_off = p.d_phi2_off;
  A.taps = p.d_taps;
  A.pool_w = p.d_pool_w;
  A.tap_off = p.d_tap_off;
  return A;
}

GradArgs grad_args(const Plan& p) {
  GradArgs A{};
  A.logN = p.logN;
  A.N1 = p.N1;
  A.n_frames = p.n_frames;
  A.n_active = p.n_active;
  A.u1_tot = p.u1_tot;
  A.y2_tot = p.y2_tot;
  A.psi1 = p.d_psi1;
  A.psi2 = p.d_psi2;
  A.phiT = p.h_phiT;
  A.s2 = p.d_s2;
  A.n1max_act = p.d_n1max_act;
  A.act_n2 = p.d_act_n2;
  A.y2_off = p.d_y2_off;
  A.u1_off = p.d_u1_off;
  return A;
}

#define JTFS_TRY(expr)            \
  do {                            \
    const int rc_ = (expr);       \
    if (rc_ != JTFS_OK) return rc_; \
  } while (0)

int check_launch() { return cudaGetLastError() == cudaSuccess ? JTFS_OK : JTFS_ERR_CUDA; }

int copy_block(const Plan& p, const float* src, int64_t src_stride, int64_t src_off, float* dst, int64_t dst_stride,
               int64_t dst_off, int64_t len, bool accumulate, cudaStream_t s) {
  const unsigned gx = static_cast<unsigned>(std::min<int64_t>((len + kThreads - 1) / kThreads, 4096));
  k_copy_block<<<dim3(std::max(gx, 1u), static_cast<unsigned>(p.batch)), kThreads, 0, s>>>(
      src, src_stride, src_off, dst, dst_stride, dst_off, len, accumulate ? 1 : 0);
  return check_launch();
}

// Bracket one launch of `stage` with the caller's events, if registered.
void prof_begin(const Plan& p, int stage, cudaStream_t s) {
  const auto& ev = p.prof_events[stage];
  const int i = p.prof_next[stage];
  if (2 * i + 1 < static_cast<int>(ev.size())) cudaEventRecord(static_cast<cudaEvent_t>(ev[2 * i]), s);
}
void prof_end(const Plan& p, int stage, cudaStream_t s) {
  const auto& ev = p.prof_events[stage];
  const int i = p.prof_next[stage];
  if (2 * i + 1 < static_cast<int>(ev.size())) {
    cudaEventRecord(static_cast<cudaEvent_t>(ev[2 * i + 1]), s);
    p.prof_next[stage] = i + 1;
  }
}

// Fork / join of independent launches of one stage: branch k runs on the plan's auxiliary stream k,
// which waits for the work already on the caller's stream; leaving the scope makes the caller's
// stream wait for every branch used.  With stage events registered (jtfs_profile_stage) or without
// auxiliary streams everything stays on the caller's stream, in order.
class Fork {
 public:
  Fork(const Plan& p, cudaStream_t s) : p_(p), s_(s) {
    bool prof = false;
    for (const auto& e : p.prof_events) prof = prof || !e.empty();
    on_ = p.aux[0] && p.aux_mu && !prof;
    if (on_) {
      lock_ = std::unique_lock<std::mutex>(*p.aux_mu);
      on_ = cudaEventRecord(p.ev_fork, s) == cudaSuccess;
    }
  }
  cudaStream_t branch(int k) {
    if (!on_) return s_;
    if (!(used_ & (1 << k))) {
      if (cudaStreamWaitEvent(p_.aux[k], p_.ev_fork, 0) != cudaSuccess) return s_;
      used_ |= 1 << k;
    }
    return p_.aux[k];
  }
  void join() {
    for (int k = 0; k < 3; ++k)
      if (used_ & (1 << k)) {
        cudaEventRecord(p_.ev_join[k], p_.aux[k]);
        cudaStreamWaitEvent(s_, p_.ev_join[k], 0);
      }
    used_ = 0;
  }
  ~Fork() { join(); }

 private:
  const Plan& p_;
  cudaStream_t s_;
  bool on_ = false;
  int used_ = 0;
  std::unique_lock<std::mutex> lock_;
};

int64_t fft_launches(const Plan& p, const std::vector<FftLaunch>& L) {
  int64_t n = 0;
  int end = -1;
  for (const FftLaunch& l : L) {
    if (p.tune_tfft && l.logn <= kTfLogP) {
      if (l.n_items > 0 && l.item0 != end) ++n;   // a new run of items: one more launch
      if (l.n_items > 0) end = l.item0 + l.n_items;
    } else if (p.tune_tfft && l.logn <= kTfLogP + 3) {
      n += 1;
    } else {
      n += l.logn <= kSmallLogMax ? 1 : 2;
    }
  }
  return n;
}

// Launches of the second-order frequential stage (forward or adjoint): the
// tensor-core kernels of the groups they handle plus one FFT-kernel launch.
int64_t freq2_launches(const Plan& p, bool fwd) {
  if (!(p.tc_ok && p.tune_tc)) return 1;
  int64_t n = 0;
  for (int k = 0; k < (fwd ? 5 : 2); ++k) n += int64_t(!p.tc_tiles[k].empty());
  return n + int64_t(!(fwd ? p.tiles2_fft_f : p.tiles2_fft).empty());
}

int64_t forward_launches(const Plan& p, bool full) {
  int64_t n = fft_launches(p, p.L_x) + fft_launches(p, p.L_u1) + fft_launches(p, p.L_u1inplace) + fft_launches(p, p.L_s1);
  if (full) n += (p.unpooled_t ? 1 : fft_launches(p, p.L_s0)) + 1;
  if (p.n_active > 0) n += fft_launches(p, p.L_y2) + (full ? (p.unpooled_t ? 1 : 2) + freq2_launches(p, true) : 0);
  return n;
}

int64_t backward_launches(const Plan& p) {
  int64_t n = 1 + fft_launches(p, p.L_ds1) + (p.L_u1inplace.empty() ? 0 : 1) +
              2 * fft_launches(p, p.L_u1inplace) + (p.unpooled_t ? 1 : fft_launches(p, p.L_ds0)) + 1 + fft_launches(p, p.L_x);
  if (p.n_active > 0) n += 1 + freq2_launches(p, false) + fft_launches(p, p.L_y2inplace);
  return n;
}

size_t freq_smem(const Plan& p, int nbuf, int cols = 0) {
  if (cols == 0) cols = p.freq_cols;
  return size_t(p.N_fr) * sizeof(float2) + size_t(nbuf) * cols * p.N_fr * sizeof(float2) +
         size_t(p.n_beta2) * sizeof(int2) +
         std::max(p.chunks1.size(), p.chunks2.size()) * sizeof(FreqChunk) + size_t(p.n_beta2) * sizeof(int) + 16;
}

// Shared memory of a specialised second-order launch: with the compact filter
// tables staged (A.tab_smem = 1) when two CTAs still fit on an SM, else without.
size_t ct_smem(const Plan& p, int nbuf, int cols, FreqArgs& A) {
  constexpr size_t kTwoCtas = 113 * 1024;
  const size_t base = freq_smem(p, nbuf, cols);
  const size_t with = base + p.h_ftabc.size() * sizeof(float);
  A.tab_smem = with <= kTwoCtas ? 1 : 0;
  return A.tab_smem ? with : base;
}

// Forward stages.  `full` = false stops after what the adjoint needs
// (Xhat, U1hat, S1, Y2) and skips writing Phi.
// ---------------------------------------------------------------------------
// Several plans run stage by stage (run_forward_multi in jtfs_internal.h);
// a single plan is the case n = 1 without merged tables.
// ---------------------------------------------------------------------------
// One plan of a run, with its workspace buffers and inputs / outputs.
struct Member {
  const Plan* p;
  Bufs w;
  const float* x;
  float* phi;
  const float* dphi;
  float* dx;
};

// Per-plan loaders / stores of a merged launch, chosen by the job's `pad`
// (the kernels take them as __grid_constant__, so the table is indexed in
// place).
template <class F>
struct GLd {
  F f[kMaxGroups];
  __device__ __forceinline__ float2 operator()(const Job& jb, int idx, int logn) const {
    return f[jb.pad](jb, idx, logn);
  }
};
template <class F>
struct GSt {
  F f[kMaxGroups];
  __device__ __forceinline__ void operator()(const Job& jb, int idx, float2 v) const { f[jb.pad](jb, idx, v); }
};

// One time-axis FFT stage of every member: the merged launches of the FFT
// engine when `merged` is given, else each plan's own launches.
template <bool INV, class MkLd, class MkSt>
int run_stage(const Member* m, int n, const FftMerged* merged, int stage, MkLd mkld, MkSt mkst, cudaStream_t s) {
  using Ld = decltype(mkld(m[0]));
  using St = decltype(mkst(m[0]));
  if (!merged) {
    for (int i = 0; i < n; ++i)
      JTFS_TRY((run_fft<INV>(*m[i].p, stage_launches(*m[i].p, stage), mkld(m[i]), mkst(m[i]), m[i].w.scr, s)));
    return JTFS_OK;
  }
  GLd<Ld> gl{};
  GSt<St> gs{};
  for (int i = 0; i < n; ++i) {
    gl.f[i] = mkld(m[i]);
    gs.f[i] = mkst(m[i]);
  }
  const FftMerged& fm = merged[stage];
  if (fm.n_items > 0) {
    allow_big_smem<k_tfft<INV, GLd<Ld>, GSt<St>>>();
    k_tfft<INV, GLd<Ld>, GSt<St>><<<static_cast<unsigned>(fm.n_items), kTfThreads, kTfSmem, s>>>(gl, gs, fm.jobs,
                                                                                               fm.items);
    JTFS_TRY(check_launch());
  }
  for (const FftLaunch& l : fm.cluster) {
    allow_big_smem<k_tfft_cluster<INV, GLd<Ld>, GSt<St>>>();
    const unsigned C = 1u << (l.logn - kTfLogP);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(static_cast<unsigned>(l.njobs) * C);
    cfg.blockDim = dim3(kTfThreads);
    cfg.dynamicSmemBytes = kTfSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_tfft_cluster<INV, GLd<Ld>, GSt<St>>, gl, gs, fm.jobs, l.job0, l.logn) !=
        cudaSuccess)
      return JTFS_ERR_CUDA;
  }
  // Sizes above 2^16: each plan's two-pass launches (they need its scratch).
  for (int i = 0; i < n; ++i)
    for (const FftLaunch& l : stage_launches(*m[i].p, stage))
      if (l.logn > kTfLogP + 3) JTFS_TRY((run_tfft_big<INV>(*m[i].p, l, mkld(m[i]), mkst(m[i]), m[i].w.scr, s)));
  return JTFS_OK;
}

// STAGE(inverse?, stage, loader, store): loader and store expressions in
// terms of `g` (the member), `p` (its plan) and `w` (its buffers).
#define STAGE(INV, ST, LD_EXPR, ST_EXPR)                                                                 \
  JTFS_TRY((run_stage<INV>(                                                                            \
      m, n, merged, ST,                                                                                \
      [&](const Member& g) { const Plan& p = *g.p; const Bufs& w = g.w; (void)p; (void)w; return LD_EXPR; }, \
      [&](const Member& g) { const Plan& p = *g.p; const Bufs& w = g.w; (void)p; (void)w; return ST_EXPR; }, s)))
#define EACH for (int gi_ = 0; gi_ < n; ++gi_)
#define PLAN                     \
  const Plan& p = *m[gi_].p;     \
  const Bufs& w = m[gi_].w;      \
  (void)p;                       \
  (void)w

int forward_multi(const Member* m, int n, const FftMerged* merged, bool full, cudaStream_t s) {
  // The band signals x * psi_n1 (decimated) stay in Zs for the adjoint's
  // modulus derivative; U1h receives the FFT of their modulus.
  STAGE(false, FS_X, LdReal{g.x}, StC{w.Xh});
  STAGE(true, FS_U1, (LdBand{w.Xh, p.d_psi1, FiltD{}}), StC{w.Zs});
  STAGE(false, FS_U1IP, LdMod{w.Zs}, StC{w.U1h});
  if (full) {
    if (m[0].p->unpooled_t) {  // zeroth order = x (batches refuse the unpooled flags)
      EACH {
        PLAN;
        JTFS_TRY(copy_block(p, m[gi_].x, p.N, 0, m[gi_].phi, p.phi_size, 0, p.N, false, s));
      }
    } else {
      STAGE(true, FS_S0, (LdBand{w.Xh, nullptr, p.h_phiT}), StR{g.phi});
    }
  }
  STAGE(true, FS_S1, (LdBand{w.U1h, nullptr, p.h_phiT}), StR{w.S1});
  if (full) {
    EACH {
      PLAN;
      float* phi = m[gi_].phi;
      const FreqArgs FA = freq_args(p, 1);
      if (p.unpooled_f || !launch_freq_fwd_ct(1, FA, p.lF, static_cast<unsigned>(p.tiles1.size()), freq_smem(p, 3), s,
                                              p.d_tiles1, w.S1, nullptr, phi)) {
        allow_big_smem<k_freq_fwd<1>>();
        k_freq_fwd<1><<<static_cast<unsigned>(p.tiles1.size()), kThreads, freq_smem(p, 3), s>>>(
            FA, p.d_tiles1, w.S1, nullptr, phi);
      }
      JTFS_TRY(check_launch());
    }
  }
  STAGE(true, FS_Y2, (LdBand{w.U1h, p.d_psi2, FiltD{}}), StC{w.Y2});
  if (full) {
    EACH {
      PLAN;
      float* phi = m[gi_].phi;
      if (p.n_active == 0) continue;
      const FreqArgs FA2 = freq_args(p, 2);
      allow_big_smem<k_freq_fwd<2>>();
      prof_begin(p, JTFS_STAGE_FREQ2_FWD, s);
      FreqArgs FA2w = FA2, FA2n = FA2;
      FA2w.W = p.freq_cols_wide;
      FA2w.logW = ceil_log2(p.freq_cols_wide);
      const size_t smem_w = ct_smem(p, 3, p.freq_cols_wide, FA2w);
      const size_t smem_n = ct_smem(p, 3, p.freq_cols, FA2n);
      // Groups with at most 64 rows n1 on the tensor cores, the others on the FFT kernels; the three
      // launches touch disjoint groups and run concurrently.
      const bool tc = p.tc_ok && p.tune_tc;
      {
        Fork fk(p, s);
        if (tc) {
          prof_begin(p, JTFS_STAGE_FREQ2_FWD_TC, s);
          bool more = false;
          for (int k = 1; k < 5; ++k) more = more || tc_has_groups(p, k);
          JTFS_TRY(tc_forward(p, w.Y2, w.V2, s, more ? fk.branch(0) : s));
          prof_end(p, JTFS_STAGE_FREQ2_FWD_TC, s);
        }
        const Tile* t2 = tc ? p.d_tiles2_fft_f : p.d_tiles2;
        const Tile* t2w = tc ? p.d_tiles2w_fft_f : p.d_tiles2w;
        const unsigned n2 = static_cast<unsigned>(tc ? p.tiles2_fft_f.size() : p.tiles2.size());
        const unsigned n2w = static_cast<unsigned>(tc ? p.tiles2w_fft_f.size() : p.tiles2w.size());
        if (n2 > 0) {
          const cudaStream_t cs = fk.branch(1);
          if (p.unpooled_f ||
              (!(p.tune_wide && launch_freq_fwd_ct(2, FA2w, p.lF, n2w, smem_w, cs, t2w, nullptr, w.Y2, w.V2)) &&
               !launch_freq_fwd_ct(2, FA2n, p.lF, n2, smem_n, cs, t2, nullptr, w.Y2, w.V2)))
            k_freq_fwd<2><<<n2, kThreads, freq_smem(p, 3), cs>>>(FA2, t2, nullptr, w.Y2, w.V2);
        }
        JTFS_TRY(check_launch());
      }
      prof_end(p, JTFS_STAGE_FREQ2_FWD, s);
      if (p.unpooled_t) {  // second-order blocks = V2 (no phi_T)
        JTFS_TRY(copy_block(p, w.V2, p.v2_tot, 0, phi, p.phi_size, p.phi2_base, p.v2_tot, false, s));
        continue;
      }
      const PoolArgs PA = pool_args(p);
      const int fpt = p.n_frames >= 128 ? 16 : p.n_frames >= 64 ? 8 : p.n_frames >= 32 ? 4 : p.n_frames >= 16 ? 2 : 1;
      const int si = p.tune_split;
      const int split_len = kPoolSplits[si];
      dim3 grid(static_cast<unsigned>(p.pool_fwd_tiles[si].size()),
                static_cast<unsigned>((p.n_frames + 8 * fpt - 1) / (8 * fpt)));
      prof_begin(p, JTFS_STAGE_POOL_FWD, s);
      const int4* pt = p.d_pool_fwd_tiles[si];
      if (!p.pool_band_tiles.empty()) {
        // Banded groups: on the tensor cores where the widened sample range fits the circle.
        const bool tcb = p.tune_pool_tc && !p.pool_tc_band_tiles.empty();
        if (tcb) JTFS_TRY(pool_tc_band(p, w.V2, phi, s));
        const auto& bt = tcb ? p.pool_band_rest : p.pool_band_tiles;
        if (!bt.empty()) {
          k_pool_fwd_band<<<static_cast<unsigned>(bt.size()), kThreads, 0, s>>>(
              PA, w.V2, phi, tcb ? p.d_pool_band_rest : p.d_pool_band_tiles);
          JTFS_TRY(check_launch());
        }
      }
      if (grid.x && p.tune_pool_tc && pool_tc_dense(p)) {
        // Tensor cores: 128 rows x all frames per CTA, partials into the same slots.
        JTFS_TRY(pool_tc_forward(p, w.V2, w.part, si, s));
      } else if (grid.x && p.n_frames >= 32) {
        // 16-byte register-blocked kernel: 32, 64 or 128 frames per CTA.
        const int fr = p.n_frames >= 128 ? 128 : p.n_frames >= 64 ? 64 : 32;
        const dim3 g2(grid.x, static_cast<unsigned>((p.n_frames + fr - 1) / fr));
        if (fr == 128) k_pool_fwd2<128><<<g2, 512, 0, s>>>(PA, w.V2, w.part, pt, split_len);
        else if (fr == 64) k_pool_fwd2<64><<<g2, 256, 0, s>>>(PA, w.V2, w.part, pt, split_len);
        else k_pool_fwd2<32><<<g2, 128, 0, s>>>(PA, w.V2, w.part, pt, split_len);
        JTFS_TRY(check_launch());
      } else if (grid.x) {
        switch (fpt) {
          case 16: k_pool_fwd<16><<<grid, kThreads, 0, s>>>(PA, w.V2, w.part, pt, split_len); break;
          case 8: k_pool_fwd<8><<<grid, kThreads, 0, s>>>(PA, w.V2, w.part, pt, split_len); break;
          case 4: k_pool_fwd<4><<<grid, kThreads, 0, s>>>(PA, w.V2, w.part, pt, split_len); break;
          case 2: k_pool_fwd<2><<<grid, kThreads, 0, s>>>(PA, w.V2, w.part, pt, split_len); break;
          default: k_pool_fwd<1><<<grid, kThreads, 0, s>>>(PA, w.V2, w.part, pt, split_len); break;
        }
        JTFS_TRY(check_launch());
      }
      if (grid.x) {
        const int64_t total = int64_t(p.batch) * p.n_active * p.rows2 * p.n_frames;
        k_pool_reduce<<<static_cast<unsigned>((total + kThreads - 1) / kThreads), kThreads, 0, s>>>(
            PA, w.part, phi, p.d_pool_tile0[si], split_len, total);
      }
      prof_end(p, JTFS_STAGE_POOL_FWD, s);
      JTFS_TRY(check_launch());
    }
  }
  return JTFS_OK;
}

// Backward stages from dphi (device, [batch][phi_size]) to dx.  Requires
// forward_stages(full or not) to have filled Zs, U1h, S1 and Y2.
int backward_multi(const Member* m, int n, const FftMerged* merged, cudaStream_t s) {
  EACH {
    PLAN;
    const float* dphi = m[gi_].dphi;
    const FreqArgs FA = freq_args(p, 1);
    const FreqArgs FA2 = freq_args(p, 2);
    if (p.n_active > 0) {
      const PoolArgs PA = pool_args(p);
      prof_begin(p, JTFS_STAGE_POOL_ADJ, s);
      if (p.unpooled_t)  // dV2 = the second-order blocks of dPhi
        JTFS_TRY(copy_block(p, dphi, p.phi_size, p.phi2_base, w.V2, p.v2_tot, 0, p.v2_tot, false, s));
      if (!p.pool_tiles2.empty()) {
        if (p.tune_pool_tc && pool_tc_dense(p))  // dense groups on the tensor cores
          JTFS_TRY(pool_tc_adjoint(p, dphi, w.V2, s));
        else
          k_pool_adj2<<<static_cast<unsigned>(p.pool_tiles2.size()), kThreads, 0, s>>>(PA, dphi, w.V2,
                                                                                       p.d_pool_tiles2);
      }
      if (!p.pool_tiles.empty()) {
        // Banded groups: on the tensor cores where 64 frames cover a tile's reach, the rest on the FMA kernel.
        const bool tcb = p.tune_pool_tc && !p.pool_tc_band_adj_tiles.empty();
        if (tcb) JTFS_TRY(pool_tc_band_adjoint(p, dphi, w.V2, s));
        const auto& bt = tcb ? p.pool_tiles_rest : p.pool_tiles;
        if (!bt.empty())
          k_pool_adj<<<static_cast<unsigned>(bt.size()), kThreads, 0, s>>>(PA, dphi, w.V2,
                                                                          tcb ? p.d_pool_tiles_rest : p.d_pool_tiles);
      }
      prof_end(p, JTFS_STAGE_POOL_ADJ, s);
      JTFS_TRY(check_launch());
      allow_big_smem<k_freq_adj<2>>();
      allow_big_smem<k_freq_adj<1>>();
      prof_begin(p, JTFS_STAGE_FREQ2_ADJ, s);
      FreqArgs FA2c = FA2;
      const size_t smem_c = ct_smem(p, 5, p.freq_cols, FA2c);
      const bool tc = p.tc_ok && p.tune_tc;
      {
        // The tensor-core groups, the FFT groups and the first-order adjoint (which reads dphi and S1
        // only) touch disjoint data and run concurrently.
        Fork fk(p, s);
        if (tc) {
          prof_begin(p, JTFS_STAGE_FREQ2_ADJ_TC, s);
          JTFS_TRY(tc_adjoint(p, w.Y2, w.V2, w.dY2, s, tc_has_groups(p, 1) ? fk.branch(0) : s));
          prof_end(p, JTFS_STAGE_FREQ2_ADJ_TC, s);
        }
        const Tile* t2 = tc ? p.d_tiles2_fft : p.d_tiles2;
        const unsigned n2 = static_cast<unsigned>(tc ? p.tiles2_fft.size() : p.tiles2.size());
        if (n2 > 0) {
          const cudaStream_t cs = fk.branch(1);
          if (p.unpooled_f ||
              !launch_freq_adj_ct(2, FA2c, p.lF, n2, smem_c, cs, t2, nullptr, w.Y2, w.V2, nullptr, w.dY2))
            k_freq_adj<2><<<n2, kThreads, freq_smem(p, 5), cs>>>(FA2, t2, nullptr, w.Y2, w.V2, nullptr, w.dY2);
        }
        JTFS_TRY(check_launch());
        prof_end(p, JTFS_STAGE_FREQ2_ADJ, s);
        const cudaStream_t s1 = fk.branch(2);
        if (p.unpooled_f || !launch_freq_adj_ct(1, FA, p.lF, static_cast<unsigned>(p.tiles1.size()),
                                                freq_smem(p, 5), s1, p.d_tiles1, w.S1, nullptr, dphi, w.S1, nullptr))
          k_freq_adj<1><<<static_cast<unsigned>(p.tiles1.size()), kThreads, freq_smem(p, 5), s1>>>(
              FA, p.d_tiles1, w.S1, nullptr, dphi, w.S1, nullptr);
        JTFS_TRY(check_launch());
      }
    } else {
      allow_big_smem<k_freq_adj<1>>();
      if (p.unpooled_f || !launch_freq_adj_ct(1, FA, p.lF, static_cast<unsigned>(p.tiles1.size()), freq_smem(p, 5),
                                              s, p.d_tiles1, w.S1, nullptr, dphi, w.S1, nullptr))
        k_freq_adj<1><<<static_cast<unsigned>(p.tiles1.size()), kThreads, freq_smem(p, 5), s>>>(
            FA, p.d_tiles1, w.S1, nullptr, dphi, w.S1, nullptr);
      JTFS_TRY(check_launch());
    }
  }
  STAGE(false, FS_Y2IP, LdC{w.dY2}, StC{w.dY2});
  STAGE(false, FS_DS1, LdReal{w.S1}, StC{w.dS1h});
  EACH {
    PLAN;
    // Every level in one launch: one block per kThreads samples of every U1 row (the block table).
    static_assert(kDU1Block == kThreads, "block table built for kThreads-thread blocks");
    const GradArgs GA = grad_args(p);
    if (!p.du1_blocks.empty()) {
      k_dU1<<<static_cast<unsigned>(p.du1_blocks.size()), kThreads, 0, s>>>(
          GA, p.d_jobs + p.L_u1inplace.front().job0, p.d_du1_blocks, w.dY2, w.dS1h, w.U1h);
      JTFS_TRY(check_launch());
    }
  }
  STAGE(true, FS_U1IP, LdC{w.U1h}, StC{w.U1h});
  STAGE(false, FS_U1IP, (LdDz{w.U1h, w.Zs}), StC{w.Zs});
  if (!m[0].p->unpooled_t) STAGE(false, FS_DS0, LdReal{g.dphi}, StC{w.dS0h});
  EACH {
    PLAN;
    const GradArgs GA = grad_args(p);
    const int64_t total = int64_t(p.batch) * p.N;
    k_dX<<<static_cast<unsigned>((total + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        GA, total, w.Zs, p.unpooled_t ? nullptr : w.dS0h, w.dXh);
    JTFS_TRY(check_launch());
  }
  STAGE(true, FS_X, LdC{w.dXh}, StR{g.dx});
  EACH {
    PLAN;
    if (p.unpooled_t)  // the zeroth order is x: its gradient adds directly
      JTFS_TRY(copy_block(p, m[gi_].dphi, p.phi_size, 0, m[gi_].dx, p.N, 0, p.N, true, s));
  }
  return JTFS_OK;
}

int forward_stages(const Plan& p, const float* x, float* phi, const Bufs& w, bool full, cudaStream_t s) {
  const Member m{&p, w, x, phi, nullptr, nullptr};
  return forward_multi(&m, 1, nullptr, full, s);
}

int backward_stages(const Plan& p, const float* dphi, float* dx, const Bufs& w, cudaStream_t s) {
  const Member m{&p, w, nullptr, nullptr, dphi, dx};
  return backward_multi(&m, 1, nullptr, s);
}

// Coloured initialisation (§2.3): y0 = ||x|| y~ / ||y~||,
// y~ = sum_l c_l Psi_l^T (A_l . Psi_l w), A_l = 2^(lT-k1) P_l^T S1x(., l).
// The chain is the first-layer part of the adjoint with the envelope in place
// of dU1 and a linear band product in place of the modulus adjoint.
int coloured_init_stages(const Plan& p, const float* x, const float* w_noise, float* y0, const Bufs& w,
                         cudaStream_t s) {
  // S1 of the target: first layer and phi_T pooling (§3.2, Eq. (4)).
  JTFS_TRY((run_fft<false>(p, p.L_x, LdReal{x}, StC{w.Xh}, w.scr, s)));
  JTFS_TRY((run_fft<true>(p, p.L_u1, LdBand{w.Xh, p.d_psi1, FiltD{}}, StC{w.U1h}, w.scr, s)));
  JTFS_TRY((run_fft<false>(p, p.L_u1inplace, LdMod{w.U1h}, StC{w.U1h}, w.scr, s)));
  JTFS_TRY((run_fft<true>(p, p.L_s1, LdBand{w.U1h, nullptr, p.h_phiT}, StR{w.S1}, w.scr, s)));
  // Envelopes c_l A_l at the U1 rate: gains, then the adjoint of the pooling.
  {
    const int64_t total = int64_t(p.batch) * p.N1 * p.n_frames;
    k_scale_rows<<<static_cast<unsigned>((total + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        w.S1, p.d_cinit, p.N1, p.log_frames, total);
    JTFS_TRY(check_launch());
  }
  JTFS_TRY((run_fft<false>(p, p.L_ds1, LdReal{w.S1}, StC{w.dS1h}, w.scr, s)));
  GradArgs GA = grad_args(p);
  GradArgs GA1 = GA;
  GA1.n_active = 0;  // no second-order term
  for (const FftLaunch& l : p.L_u1inplace) {
    dim3 grid((1u << l.logn) / kThreads + 1, l.njobs);
    k_dU1<<<grid, kThreads, 0, s>>>(GA1, p.d_jobs + l.job0, nullptr, nullptr, w.dS1h, w.U1h);
    JTFS_TRY(check_launch());
  }
  JTFS_TRY((run_fft<true>(p, p.L_u1inplace, LdC{w.U1h}, StC{w.U1h}, w.scr, s)));
  // Band-passed noise Psi_l w, band products, and the filterbank adjoint.
  JTFS_TRY((run_fft<false>(p, p.L_x, LdReal{w_noise}, StC{w.Xh}, w.scr, s)));
  JTFS_TRY((run_fft<true>(p, p.L_u1, LdBand{w.Xh, p.d_psi1, FiltD{}}, StC{w.Zs}, w.scr, s)));
  JTFS_TRY((run_fft<false>(p, p.L_u1inplace, LdLin{w.U1h, w.Zs}, StC{w.Zs}, w.scr, s)));
  {
    const int64_t total = int64_t(p.batch) * p.N;
    k_dX<<<static_cast<unsigned>((total + kThreads - 1) / kThreads), kThreads, 0, s>>>(GA, total, w.Zs, nullptr,
                                                                                       w.dXh);
    JTFS_TRY(check_launch());
  }
  JTFS_TRY((run_fft<true>(p, p.L_x, LdC{w.dXh}, StR{y0}, w.scr, s)));
  k_energy_match<<<p.batch, 512, 0, s>>>(x, y0, p.N);
  return check_launch();
}

int momentum_update(float* y, float* u, float* g_acc, const float* g, float* state, const float* loss, int batch,
                    int64_t n, float m, cudaStream_t s) {
  k_bold_decide<<<(batch + 127) / 128, 128, 0, s>>>(reinterpret_cast<float4*>(state), loss, batch);
  JTFS_TRY(check_launch());
  int log_n = 0;
  while ((int64_t(1) << log_n) < n) ++log_n;
  const int64_t total = int64_t(batch) * n;
  k_momentum<<<static_cast<unsigned>((total + kThreads - 1) / kThreads), kThreads, 0, s>>>(
      y, u, g_acc, g, reinterpret_cast<const float4*>(state), log_n, total, m);
  return check_launch();
}

int check_call(const Plan& p, void* ws) {
  if (!p.on_device) return JTFS_ERR_NODEVICE;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return JTFS_ERR_WORKSPACE;
  return JTFS_OK;
}

bool misaligned(const void* ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15) != 0; }

}  // namespace

const std::vector<FftLaunch>& stage_launches(const Plan& p, int stage) {
  switch (stage) {
    case FS_X: return p.L_x;
    case FS_U1: return p.L_u1;
    case FS_U1IP: return p.L_u1inplace;
    case FS_S0: return p.L_s0;
    case FS_S1: return p.L_s1;
    case FS_Y2: return p.L_y2;
    case FS_Y2IP: return p.L_y2inplace;
    case FS_DS1: return p.L_ds1;
    default: return p.L_ds0;
  }
}

void merge_fft_stages(const Plan* const* plans, int n, std::vector<Job>& jobs, std::vector<int4>& items,
                      FftMerged (&out)[FS_COUNT], int (&job0)[FS_COUNT], int (&item0)[FS_COUNT]) {
  jobs.clear();
  items.clear();
  for (int st = 0; st < FS_COUNT; ++st) {
    FftMerged& fm = out[st];
    fm.cluster.clear();
    job0[st] = static_cast<int>(jobs.size());
    item0[st] = static_cast<int>(items.size());
    // Sizes up to 2^13: every plan's items, their jobs copied behind (pad = the plan).
    for (int g = 0; g < n; ++g)
      for (const FftLaunch& l : stage_launches(*plans[g], st)) {
        if (l.logn > kTfLogP) continue;
        const int base = static_cast<int>(jobs.size()) - job0[st];
        for (int j = 0; j < l.njobs; ++j) {
          Job jb = plans[g]->jobs[size_t(l.job0 + j)];
          jb.pad = g;
          jobs.push_back(jb);
        }
        for (int it = 0; it < l.n_items; ++it) {
          int4 v = plans[g]->tf_items[size_t(l.item0 + it)];
          v.x = base + (v.x - l.job0);   // relative to the stage's first job
          items.push_back(v);
        }
      }
    fm.n_items = static_cast<int>(items.size()) - item0[st];
    // 2^14 .. 2^16: one cluster launch per size over every plan's jobs of that size.
    for (int lg = kTfLogP + 1; lg <= kTfLogP + 3; ++lg) {
      const int first = static_cast<int>(jobs.size()) - job0[st];
      for (int g = 0; g < n; ++g)
        for (const FftLaunch& l : stage_launches(*plans[g], st)) {
          if (l.logn != lg) continue;
          for (int j = 0; j < l.njobs; ++j) {
            Job jb = plans[g]->jobs[size_t(l.job0 + j)];
            jb.pad = g;
            jobs.push_back(jb);
          }
        }
      const int cnt = static_cast<int>(jobs.size()) - job0[st] - first;
      if (cnt > 0) fm.cluster.push_back({lg, cnt, first, 0, 0});
    }
  }
}

namespace {
std::vector<Member> members(const Plan* const* plans, const float* const* x, float* const* phi,
                            const float* const* dphi, float* const* dx, void* const* ws, int n) {
  std::vector<Member> m(static_cast<size_t>(n));
  for (int i = 0; i < n; ++i)
    m[size_t(i)] = {plans[i], bufs(*plans[i], ws[i]), x ? x[i] : nullptr, phi ? phi[i] : nullptr,
                    dphi ? dphi[i] : nullptr, dx ? dx[i] : nullptr};
  return m;
}
}  // namespace

int run_forward_multi(const Plan* const* plans, const float* const* x, float* const* phi, void* const* ws, int n,
                      const FftMerged* merged, bool full, cudaStream_t s) {
  if (n < 1 || n > kMaxGroups) return JTFS_ERR_ARG;
  const std::vector<Member> m = members(plans, x, phi, nullptr, nullptr, ws, n);
  return forward_multi(m.data(), n, merged, full, s);
}

int run_backward_multi(const Plan* const* plans, const float* const* dphi, float* const* dx, void* const* ws, int n,
                       const FftMerged* merged, cudaStream_t s) {
  if (n < 1 || n > kMaxGroups) return JTFS_ERR_ARG;
  const std::vector<Member> m = members(plans, nullptr, nullptr, dphi, dx, ws, n);
  return backward_multi(m.data(), n, merged, s);
}

int run_forward(const Plan& p, const float* x, float* phi, void* ws, bool full, cudaStream_t s) {
  return forward_stages(p, x, phi, bufs(p, ws), full, s);
}
int run_backward(const Plan& p, const float* dphi, float* dx, void* ws, cudaStream_t s) {
  return backward_stages(p, dphi, dx, bufs(p, ws), s);
}

}  // namespace jtfs


using jtfs::Bufs;

extern "C" int jtfs_forward(jtfs_plan_t plan, const float* x, float* phi, void* workspace, void* stream) {
  if (!plan || !x || !phi || jtfs::misaligned(x) || jtfs::misaligned(phi)) return JTFS_ERR_ARG;
  const jtfs::Plan& p = plan->p;
  JTFS_TRY(jtfs::check_call(p, workspace));
  const Bufs w = jtfs::bufs(p, workspace);
  return jtfs::forward_stages(p, x, phi, w, true, static_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------------------
// No-allocation forward: scratch in a fixed array of the library image.
// ---------------------------------------------------------------------------
namespace jtfs {
namespace {

// File-scope device array used as the workspace of jtfs_forward_noalloc.  In
// host code `g_noalloc_scratch` names a host-side stand-in, never a device
// address: the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[JTFS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::once_flag g_scratch_once[kMaxDevices];
void* g_scratch_ptr[kMaxDevices] = {};
cudaError_t g_scratch_err[kMaxDevices] = {};

// Device address of the array on the current device (looked up once per device).
int noalloc_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return JTFS_ERR_ARG;
  std::call_once(g_scratch_once[dev], [dev] {
    void* ptr = nullptr;
    g_scratch_err[dev] = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (g_scratch_err[dev] == cudaSuccess) g_scratch_ptr[dev] = ptr;
    else cudaGetLastError();
  });
  if (g_scratch_err[dev] != cudaSuccess || !g_scratch_ptr[dev]) return JTFS_ERR_CUDA;
  *out = g_scratch_ptr[dev];
  return JTFS_OK;
}

}  // namespace
}  // namespace jtfs

extern "C" int jtfs_forward_noalloc(jtfs_plan_t plan, const float* x, float* phi, void* stream) {
  if (!plan || !x || !phi || jtfs::misaligned(x) || jtfs::misaligned(phi)) return JTFS_ERR_ARG;
  const jtfs::Plan& p = plan->p;
  if (!p.on_device) return JTFS_ERR_NODEVICE;
  if (p.ws_bytes > JTFS_NOALLOC_SCRATCH_BYTES) return JTFS_ERR_TOOBIG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p.device) return JTFS_ERR_ARG;
  void* scratch = nullptr;
  JTFS_TRY(jtfs::noalloc_scratch(dev, &scratch));
  const Bufs w = jtfs::bufs(p, scratch);
  return jtfs::forward_stages(p, x, phi, w, true, static_cast<cudaStream_t>(stream));
}

extern "C" int jtfs_backward(jtfs_plan_t plan, const float* x, const float* dphi, float* dx, void* workspace,
                             void* stream) {
  if (!plan || !x || !dphi || !dx || jtfs::misaligned(x) || jtfs::misaligned(dphi) || jtfs::misaligned(dx))
    return JTFS_ERR_ARG;
  const jtfs::Plan& p = plan->p;
  JTFS_TRY(jtfs::check_call(p, workspace));
  const Bufs w = jtfs::bufs(p, workspace);
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  JTFS_TRY(jtfs::forward_stages(p, x, nullptr, w, false, s));
  return jtfs::backward_stages(p, dphi, dx, w, s);
}

extern "C" int jtfs_loss_grad(jtfs_plan_t plan, const float* y, const float* phi_target, float* loss, float* dy,
                              void* workspace, void* stream) {
  if (!plan || !y || !phi_target || !loss || jtfs::misaligned(y) || jtfs::misaligned(phi_target) ||
      (dy && jtfs::misaligned(dy)))
    return JTFS_ERR_ARG;
  const jtfs::Plan& p = plan->p;
  JTFS_TRY(jtfs::check_call(p, workspace));
  const Bufs w = jtfs::bufs(p, workspace);
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  JTFS_TRY(jtfs::forward_stages(p, y, w.phi, w, true, s));
  if (p.loss_parts <= 1) {
    jtfs::k_loss<<<p.batch, 512, 0, s>>>(w.phi, phi_target, dy ? w.dphi : nullptr, loss, p.phi_size);
  } else {
    const int64_t chunk = (p.phi_size + p.loss_parts - 1) / p.loss_parts;
    jtfs::k_loss_part<<<dim3(p.loss_parts, p.batch), 512, 0, s>>>(w.phi, phi_target, dy ? w.dphi : nullptr,
                                                                  w.lossp, p.phi_size, chunk);
    JTFS_TRY(jtfs::check_launch());
    jtfs::k_loss_sum<<<p.batch, 256, 0, s>>>(w.lossp, loss, p.loss_parts);
  }
  JTFS_TRY(jtfs::check_launch());
  if (!dy) return JTFS_OK;
  return jtfs::backward_stages(p, w.dphi, dy, w, s);
}

extern "C" int metamer_step(jtfs_plan_t plan, float* y, const float* phi_target, float* adam_m, float* adam_v,
                            int step, float lr, float* loss_out, void* workspace, void* stream) {
  if (!plan || !y || !phi_target || !adam_m || !adam_v || !loss_out || step < 1 || !(lr > 0.f) ||
      jtfs::misaligned(adam_m) || jtfs::misaligned(adam_v))
    return JTFS_ERR_ARG;
  const jtfs::Plan& p = plan->p;
  JTFS_TRY(jtfs::check_call(p, workspace));
  const Bufs w = jtfs::bufs(p, workspace);
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  JTFS_TRY(jtfs_loss_grad(plan, y, phi_target, loss_out, w.dy, workspace, stream));
  const int64_t n = int64_t(p.batch) * p.N;
  const float c1 = static_cast<float>(1.0 / (1.0 - std::pow(0.9, step)));
  const float c2 = static_cast<float>(1.0 / (1.0 - std::pow(0.999, step)));
  jtfs::k_adam<<<static_cast<unsigned>((n + jtfs::kThreads - 1) / jtfs::kThreads), jtfs::kThreads, 0, s>>>(
      y, adam_m, adam_v, w.dy, n, lr, c1, c2);
  return jtfs::check_launch();
}

extern "C" int metamer_step_counted(jtfs_plan_t plan, float* y, const float* phi_target, float* adam_m,
                                    float* adam_v, int32_t* step, float lr, float* loss_out, void* workspace,
                                    void* stream) {
  if (!plan || !y || !phi_target || !adam_m || !adam_v || !step || !loss_out || !(lr > 0.f) ||
      jtfs::misaligned(adam_m) || jtfs::misaligned(adam_v))
    return JTFS_ERR_ARG;
  const jtfs::Plan& p = plan->p;
  JTFS_TRY(jtfs::check_call(p, workspace));
  const Bufs w = jtfs::bufs(p, workspace);
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  JTFS_TRY(jtfs_loss_grad(plan, y, phi_target, loss_out, w.dy, workspace, stream));
  const int64_t n = int64_t(p.batch) * p.N;
  jtfs::k_adam_counted<<<static_cast<unsigned>((n + jtfs::kThreads - 1) / jtfs::kThreads), jtfs::kThreads, 0, s>>>(
      y, adam_m, adam_v, w.dy, n, lr, step);
  JTFS_TRY(jtfs::check_launch());
  jtfs::k_step_next<<<1, 1, 0, s>>>(step);
  return jtfs::check_launch();
}

extern "C" int jtfs_status(void* stream) {
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return JTFS_ERR_CUDA;
  int nf = 0;
  if (cudaMemcpyFromSymbol(&nf, jtfs::g_nonfinite, sizeof(int)) != cudaSuccess) return JTFS_ERR_CUDA;
  const int zero = 0;
  if (nf && cudaMemcpyToSymbol(jtfs::g_nonfinite, &zero, sizeof(int)) != cudaSuccess) return JTFS_ERR_CUDA;
  const int nfb = jtfs::batch_nonfinite_take();
  const int tc = jtfs_tc_error();
  const int dec = jtfs_decoder_error();
  if (nfb < 0 || tc < 0 || dec < 0) return JTFS_ERR_CUDA;
  if (tc || dec) return JTFS_ERR_TIMEOUT;
  if (nf || nfb) return JTFS_ERR_NONFINITE;
  return JTFS_OK;
}

extern "C" int jtfs_set_wait_limit(int64_t polls) {
  JTFS_TRY(jtfs::set_wait_polls_freq(polls));
  JTFS_TRY(jtfs::set_wait_polls_pool(polls));
  return jtfs::set_wait_polls_decoder(polls);
}

extern "C" int jtfs_coloured_init(jtfs_plan_t plan, const float* x, const float* w_noise, float* y0,
                                  void* workspace, void* stream) {
  if (!plan || !x || !w_noise || !y0 || jtfs::misaligned(x) || jtfs::misaligned(w_noise) || jtfs::misaligned(y0))
    return JTFS_ERR_ARG;
  const jtfs::Plan& p = plan->p;
  JTFS_TRY(jtfs::check_call(p, workspace));
  return jtfs::coloured_init_stages(p, x, w_noise, y0, jtfs::bufs(p, workspace), static_cast<cudaStream_t>(stream));
}

extern "C" int jtfs_momentum_update(float* y, float* u, float* g_acc, const float* g, float* state,
                                    const float* loss, int batch, int64_t n, float m, void* stream) {
  if (!y || !u || !g_acc || !g || !state || !loss || batch < 1 || n < 1 || (n & (n - 1)) ||
      (reinterpret_cast<uintptr_t>(state) & 15) || !(m >= 0.f && m < 1.f))
    return JTFS_ERR_ARG;
  return jtfs::momentum_update(y, u, g_acc, g, state, loss, batch, n, m, static_cast<cudaStream_t>(stream));
}

extern "C" int metamer_step_momentum(jtfs_plan_t plan, float* y, const float* phi_target, float* u, float* g_acc,
                                     float* state, float m, float* loss_out, void* workspace, void* stream) {
  if (!plan || !y || !phi_target || !u || !g_acc || !state || !loss_out || jtfs::misaligned(u) ||
      jtfs::misaligned(g_acc) || (reinterpret_cast<uintptr_t>(state) & 15) || !(m >= 0.f && m < 1.f))
    return JTFS_ERR_ARG;
  const jtfs::Plan& p = plan->p;
  JTFS_TRY(jtfs::check_call(p, workspace));
  const Bufs w = jtfs::bufs(p, workspace);
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  JTFS_TRY(jtfs_loss_grad(plan, y, phi_target, loss_out, w.dy, workspace, stream));
  return jtfs::momentum_update(y, u, g_acc, w.dy, state, loss_out, p.batch, p.N, m, s);
}

extern "C" int64_t jtfs_init_gains(jtfs_plan_t plan, float* out, int64_t n) {
  if (!plan) return JTFS_ERR_ARG;
  const auto& g = plan->p.h_cinit;
  if (out) {
    if (n < static_cast<int64_t>(g.size())) return JTFS_ERR_ARG;
    std::copy(g.begin(), g.end(), out);
  }
  return static_cast<int64_t>(g.size());
}

extern "C" int jtfs_profile_stage(jtfs_plan_t plan, int stage, void** events, int count) {
  if (!plan || stage < 0 || stage >= JTFS_STAGE_COUNT || count < 0 || (count > 0 && !events)) return JTFS_ERR_ARG;
  const jtfs::Plan& p = plan->p;
  p.prof_events[stage].assign(events ? events : nullptr, events ? events + count : nullptr);
  p.prof_next[stage] = 0;
  return JTFS_OK;
}

extern "C" int64_t jtfs_launch_count(jtfs_plan_t plan, int call) {
  if (!plan) return JTFS_ERR_ARG;
  const jtfs::Plan& p = plan->p;
  switch (call) {
    case 0: return jtfs::forward_launches(p, true);
    case 1: return jtfs::forward_launches(p, false) + jtfs::backward_launches(p);
    case 2: return jtfs::forward_launches(p, true) + (p.loss_parts > 1 ? 2 : 1) + jtfs::backward_launches(p);
    case 3: return jtfs::forward_launches(p, true) + (p.loss_parts > 1 ? 3 : 2) + jtfs::backward_launches(p);
    default: return JTFS_ERR_ARG;
  }
}

// ---------------------------------------------------------------------------
// Autotuning of execution choices that do not change results.
// ---------------------------------------------------------------------------
extern "C" int jtfs_get_tuning(jtfs_plan_t plan, int64_t* choice, int n) {
  if (!plan) return JTFS_ERR_ARG;
  const jtfs::Plan& p = plan->p;
  const int64_t v[6] = {p.tune_wide, jtfs::kPoolSplits[p.tune_split], p.tune_fft_points,
                        (p.tc_ok && p.tune_tc) ? 1 : 0, (p.tune_pool_tc && jtfs::pool_tc_supported(p)) ? 1 : 0,
                        p.tune_tfft};
  for (int i = 0; i < n && i < 6 && choice; ++i) choice[i] = v[i];
  return 6;
}

extern "C" int jtfs_set_tuning(jtfs_plan_t plan, const int64_t* choice, int n) {
  if (!plan || !choice || n < 3) return JTFS_ERR_ARG;
  int si = -1;
  for (int i = 0; i < 3; ++i)
    if (jtfs::kPoolSplits[i] == choice[1]) si = i;
  const int64_t pts = choice[2];
  if ((choice[0] != 0 && choice[0] != 1) || si < 0 || pts < 1024 || pts > 8192 || (pts & (pts - 1))) return JTFS_ERR_ARG;
  const jtfs::Plan& p = plan->p;
  if (n >= 4 && choice[3] != 0 && choice[3] != 1) return JTFS_ERR_ARG;
  if (n >= 5 && choice[4] != 0 && choice[4] != 1) return JTFS_ERR_ARG;
  if (n >= 6 && choice[5] != 0 && choice[5] != 1) return JTFS_ERR_ARG;
  p.tune_wide = static_cast<int>(choice[0]);
  p.tune_split = si;
  p.tune_fft_points = static_cast<int>(pts);
  if (n >= 4) p.tune_tc = static_cast<int>(choice[3]);
  if (n >= 5) p.tune_pool_tc = static_cast<int>(choice[4]);
  if (n >= 6) p.tune_tfft = static_cast<int>(choice[5]);
  return 6;
}

extern "C" int jtfs_autotune(jtfs_plan_t plan, const float* y, const float* phi_target, float* loss, float* dy,
                             void* workspace, void* stream, int64_t* choice, int n) {
  if (!plan || !y || !phi_target || !loss || !dy) return JTFS_ERR_ARG;
  const jtfs::Plan& p = plan->p;
  JTFS_TRY(jtfs::check_call(p, workspace));
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return JTFS_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return JTFS_ERR_CUDA;
  }
  auto time_it = [&](float* ms) -> int {
    JTFS_TRY(jtfs_loss_grad(plan, y, phi_target, loss, dy, workspace, stream));  // warm-up / set-up
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
      if (cudaEventRecord(e0, s) != cudaSuccess) return JTFS_ERR_CUDA;
      JTFS_TRY(jtfs_loss_grad(plan, y, phi_target, loss, dy, workspace, stream));
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return JTFS_ERR_CUDA;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      best = std::min(best, t);
    }
    *ms = best;
    return JTFS_OK;
  };
  int rc = JTFS_OK;
  if (p.tc_ok) {
    float best = 1e30f, t = 0.f;
    int best_tc = p.tune_tc;
    for (int v : {1, 0}) {
      p.tune_tc = v;
      if ((rc = time_it(&t)) != JTFS_OK) break;
      if (t < best) best = t, best_tc = v;
    }
    p.tune_tc = best_tc;
  }
  if (rc == JTFS_OK) {
    float best = 1e30f, t = 0.f;
    int best_v = p.tune_tfft;
    for (int v : {1, 0}) {
      p.tune_tfft = v;
      if ((rc = time_it(&t)) != JTFS_OK) break;
      if (t < best) best = t, best_v = v;
    }
    p.tune_tfft = best_v;
  }
  if (rc == JTFS_OK && jtfs::pool_tc_supported(p)) {
    float best = 1e30f, t = 0.f;
    int best_v = p.tune_pool_tc;
    for (int v : {1, 0}) {
      p.tune_pool_tc = v;
      if ((rc = time_it(&t)) != JTFS_OK) break;
      if (t < best) best = t, best_v = v;
    }
    p.tune_pool_tc = best_v;
  }
  if (rc == JTFS_OK && !p.tune_tfft) {
    float best = 1e30f, t = 0.f;
    int best_pts = p.tune_fft_points;
    for (int pts : {1024, 2048, 4096, 8192}) {
      p.tune_fft_points = pts;
      if ((rc = time_it(&t)) != JTFS_OK) break;
      if (t < best) best = t, best_pts = pts;
    }
    p.tune_fft_points = best_pts;
  }
  if (rc == JTFS_OK) {
    float best = 1e30f, t = 0.f;
    int best_si = p.tune_split;
    for (int si = 0; si < 3; ++si) {
      p.tune_split = si;
      if ((rc = time_it(&t)) != JTFS_OK) break;
      if (t < best) best = t, best_si = si;
    }
    p.tune_split = best_si;
  }
  if (rc == JTFS_OK) {
    float best = 1e30f, t = 0.f;
    int best_w = p.tune_wide;
    for (int wv : {0, 1}) {
      p.tune_wide = wv;
      if ((rc = time_it(&t)) != JTFS_OK) break;
      if (t < best) best = t, best_w = wv;
    }
    p.tune_wide = best_w;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != JTFS_OK) return rc;
  return jtfs_get_tuning(plan, choice, n);
}
