// Time-axis FFT engine of the first and second layers (§3.2-§3.3: the
// transforms around every filter product, modulus and their adjoints).
//
// One CTA holds up to kTfP = 8192 complex points in shared memory and
// transforms them in place with radix-16 register passes (a radix-2/4/8 pass
// last when log2 n is not a multiple of 4): every thread reads the 16 points
// of its butterflies into registers, the CTA synchronises, and the results are
// written back to the Stockham output positions.  Shared memory is padded by
// one float2 every 16 (index i lives at i + i / 16), which makes both the
// unit-stride reads and the stride-16 writes of a pass conflict-free for
// 64-bit accesses.  Twiddles are computed with sincospif (exact arguments:
// the angles are dyadic fractions of a turn): w, w^2, w^4, w^8 directly, the
// other powers as products of at most three of them.
//
// * Transforms of up to 2^13 points: k_tfft, one launch per stage for all its
//   sizes (levels); CTA i takes item (first job, count, log2 n), count jobs of
//   one size with count * n <= kTfP.
// * 2^14, 2^15, 2^16 points: k_tfft_cluster, a cluster of C = n / 2^13 CTAs
//   per transform (decimation in time over the cluster): CTA c transforms the
//   subsequence x[c + C m] in its shared memory, then, after a cluster
//   barrier, takes the outputs k in [c 2^13 / C, (c + 1) 2^13 / C) of every
//   sub-transform: X[k + 2^13 q] = sum_c W_n^(c k) W_C^(c q) X_c[k], the
//   X_c[k] read from the other CTAs' shared memory (distributed shared
//   memory); a second cluster barrier keeps every CTA's memory alive until all
//   reads are done.  Inputs are read before the first barrier and outputs
//   written after it, so a stage may transform a buffer in place.
// * 2^17 .. 2^20 points: the same decimation over C = 16 .. 128 CTAs in two
//   launches through a global scratch (k_tfft_big1: the sub-transforms and
//   their twiddles; k_tfft_big2: the C-point transforms over them, in the same
//   shared-memory engine), since clusters hold at most 8 (16) CTAs.
// Loaders and stores are the functors of the four-step kernels (element idx
// of the transform described by a job), passed as __grid_constant__ so that
// the per-plan functor tables of a multi-plan run are indexed in place.
#pragma once

#include <cooperative_groups.h>

namespace jtfs {
namespace {

constexpr int kTfLogP = 13;
constexpr int kTfP = 1 << kTfLogP;        // points per CTA
constexpr int kTfThreads = kTfP / 16;     // one radix-16 butterfly per thread
constexpr int kTfMaxJobs = 256;           // jobs per CTA (sizes >= 2^5)
constexpr size_t kTfSmem = size_t(kTfP + kTfP / 16) * sizeof(float2);

__device__ __forceinline__ int tf_pad(int i) { return i + (i >> 4); }

// exp(-2 pi i x / 2) forward, its conjugate inverse (x in half turns).
template <bool INV>
__device__ __forceinline__ float2 tf_cis(float x) {
  float s, c;
  sincospif(x, &s, &c);
  return make_float2(c, INV ? s : -s);
}

// v[r] *= w^r, w = exp(-+2 pi i t), t = k / m turns, for r < R.
template <bool INV, int R>
__device__ __forceinline__ void tf_twiddle(float2 (&v)[R], int k, int lm) {
  const float x = ldexpf(static_cast<float>(2 * k), -lm);   // 2 k / m half turns, exact
  const float2 w1 = tf_cis<INV>(x);
  v[1] = cmul(v[1], w1);
  if constexpr (R >= 4) {
    const float2 w2 = tf_cis<INV>(2.f * x);
    const float2 w3 = cmul(w1, w2);
    v[2] = cmul(v[2], w2);
    v[3] = cmul(v[3], w3);
    if constexpr (R >= 8) {
      const float2 w4 = tf_cis<INV>(4.f * x);
      v[4] = cmul(v[4], w4);
      v[5] = cmul(v[5], cmul(w1, w4));
      v[6] = cmul(v[6], cmul(w2, w4));
      v[7] = cmul(v[7], cmul(w3, w4));
      if constexpr (R == 16) {
        const float2 w8 = tf_cis<INV>(8.f * x);
        v[8] = cmul(v[8], w8);
        v[9] = cmul(v[9], cmul(w1, w8));
        v[10] = cmul(v[10], cmul(w2, w8));
        v[11] = cmul(v[11], cmul(w3, w8));
        const float2 w12 = cmul(w4, w8);
        v[12] = cmul(v[12], w12);
        v[13] = cmul(v[13], cmul(w1, w12));
        v[14] = cmul(v[14], cmul(w2, w12));
        v[15] = cmul(v[15], cmul(w3, w12));
      }
    }
  }
}

// One in-place radix-R Stockham pass over `total` points = jobs of 2^logn
// (job f at [f n, (f + 1) n)), sub-transform size Ns = 2^lNs before the pass.
template <bool INV, int R, int LR>
__device__ __forceinline__ void tf_pass(float2* s, int logn, int total, int lNs) {
  constexpr int NB = 16 / R;                 // butterflies per thread
  const int lq = logn - LR, q = 1 << lq, Ns = 1 << lNs;
  const int nbf = total >> LR;
  float2 v[NB][R];
  int out[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int t = threadIdx.x + b * kTfThreads;
    out[b] = -1;
    if (t < nbf) {
      const int f = t >> lq, j = t & (q - 1), k = j & (Ns - 1);
      const int in0 = (f << logn) + j;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = s[tf_pad(in0 + r * q)];
      if (lNs > 0) tf_twiddle<INV, R>(v[b], k, lNs + LR);
      dft_reg<INV, R>(v[b]);
      out[b] = (f << logn) + ((j - k) << LR) + k;
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < NB; ++b)
    if (out[b] >= 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) s[tf_pad(out[b] + r * Ns)] = v[b][r];
    }
  __syncthreads();
}

// In-place FFT of total / 2^logn transforms of 2^logn points (natural order
// in and out); every thread of the CTA must call it.
template <bool INV>
__device__ void tf_fft(float2* s, int logn, int total) {
  int lNs = 0;
  for (; logn - lNs >= 4; lNs += 4) tf_pass<INV, 16, 4>(s, logn, total, lNs);
  switch (logn - lNs) {
    case 3: tf_pass<INV, 8, 3>(s, logn, total, lNs); break;
    case 2: tf_pass<INV, 4, 2>(s, logn, total, lNs); break;
    case 1: tf_pass<INV, 2, 1>(s, logn, total, lNs); break;
    default: break;
  }
}

// Transforms of up to kTfP points: item (job0, count, log2 n) per CTA.
template <bool INV, class Ld, class St>
__global__ void __launch_bounds__(kTfThreads, 2)
k_tfft(const __grid_constant__ Ld ld, const __grid_constant__ St st, const Job* __restrict__ jobs,
       const int4* __restrict__ items) {
  extern __shared__ float2 tf_sm[];
  __shared__ Job sj[kTfMaxJobs];
  const int4 it = items[blockIdx.x];
  const int job0 = it.x, cnt = it.y, logn = it.z;
  const int n = 1 << logn, total = cnt << logn;
  for (int i = threadIdx.x; i < cnt; i += kTfThreads) sj[i] = jobs[job0 + i];
  __syncthreads();
  for (int i = threadIdx.x; i < total; i += kTfThreads) tf_sm[tf_pad(i)] = ld(sj[i >> logn], i & (n - 1), logn);
  __syncthreads();
  tf_fft<INV>(tf_sm, logn, total);
  for (int i = threadIdx.x; i < total; i += kTfThreads) st(sj[i >> logn], i & (n - 1), tf_sm[tf_pad(i)]);
}

// One transform of n = C 2^13 points per cluster of C CTAs (C = 2, 4, 8).
template <bool INV, class Ld, class St>
__global__ void __launch_bounds__(kTfThreads, 2)
k_tfft_cluster(const __grid_constant__ Ld ld, const __grid_constant__ St st, const Job* __restrict__ jobs, int job0,
               int logn) {
  namespace cg = cooperative_groups;
  extern __shared__ float2 tf_sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int lC = logn - kTfLogP, C = 1 << lC;
  const int c = static_cast<int>(cl.block_rank());
  const Job jb = jobs[job0 + static_cast<int>(blockIdx.x >> lC)];
  for (int i = threadIdx.x; i < kTfP; i += kTfThreads) tf_sm[tf_pad(i)] = ld(jb, c + (i << lC), logn);
  __syncthreads();
  tf_fft<INV>(tf_sm, kTfLogP, kTfP);
  cl.sync();
  const int kc = kTfP >> lC;                 // outputs k of this CTA
  for (int t = threadIdx.x; t < kc; t += kTfThreads) {
    const int k = c * kc + t;
    float2 v[8];
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      if (cc < C) {
        const float2* rs = cl.map_shared_rank(tf_sm, cc);
        const float2 x = rs[tf_pad(k)];
        v[cc] = cc == 0 ? x : cmul(x, tf_cis<INV>(ldexpf(static_cast<float>(2 * cc * k), -logn)));
      }
    }
    if (C == 2) {
      float2 u[2] = {v[0], v[1]};
      dft_reg<INV, 2>(u);
      st(jb, k, u[0]);
      st(jb, k + kTfP, u[1]);
    } else if (C == 4) {
      float2 u[4] = {v[0], v[1], v[2], v[3]};
      dft_reg<INV, 4>(u);
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) st(jb, k + qq * kTfP, u[qq]);
    } else {
      dft_reg<INV, 8>(v);
#pragma unroll
      for (int qq = 0; qq < 8; ++qq) st(jb, k + qq * kTfP, v[qq]);
    }
  }
  cl.sync();
}

// n = C 2^13 points with C = 16 .. 128 (2^17 .. 2^20), in two launches through
// a global scratch of n points per job.
// Pass 1, CTA (job, c): the 2^13-point transform X_c of x[c + C m], times the
// twiddles W_n^(c k), into scratch [job][c][k].
template <bool INV, class Ld>
__global__ void __launch_bounds__(kTfThreads, 2)
k_tfft_big1(const __grid_constant__ Ld ld, const Job* __restrict__ jobs, int job0, int logn,
            float2* __restrict__ scr) {
  extern __shared__ float2 tf_sm[];
  const int lC = logn - kTfLogP;
  const int jl = static_cast<int>(blockIdx.x >> lC), c = static_cast<int>(blockIdx.x & ((1u << lC) - 1));
  const Job jb = jobs[job0 + jl];
  for (int i = threadIdx.x; i < kTfP; i += kTfThreads) tf_sm[tf_pad(i)] = ld(jb, c + (i << lC), logn);
  __syncthreads();
  tf_fft<INV>(tf_sm, kTfLogP, kTfP);
  float2* out = scr + (static_cast<int64_t>(jl) << logn) + (static_cast<int64_t>(c) << kTfLogP);
  for (int k = threadIdx.x; k < kTfP; k += kTfThreads) {
    const float2 v = tf_sm[tf_pad(k)];
    out[k] = c == 0 ? v : cmul(v, tf_cis<INV>(ldexpf(static_cast<float>(2 * c * k), -logn)));
  }
}

// Pass 2, CTA (job, block of K = 2^13 / C outputs k): the C-point transforms
// over c of the twiddled X_c[k], X[k + 2^13 q] = sum_c W_C^(c q) u_c[k].
template <bool INV, class St>
__global__ void __launch_bounds__(kTfThreads, 2)
k_tfft_big2(const __grid_constant__ St st, const Job* __restrict__ jobs, int job0, int logn,
            const float2* __restrict__ scr) {
  extern __shared__ float2 tf_sm[];
  const int lC = logn - kTfLogP, lK = kTfLogP - lC;
  const int jl = static_cast<int>(blockIdx.x >> lC), kb = static_cast<int>(blockIdx.x & ((1u << lC) - 1));
  const Job jb = jobs[job0 + jl];
  const int k0 = kb << lK;
  const float2* in = scr + (static_cast<int64_t>(jl) << logn);
  for (int i = threadIdx.x; i < kTfP; i += kTfThreads) {   // i = c K + j: u_c[k0 + j] -> element c of job j
    const int c = i >> lK, j = i & ((1 << lK) - 1);
    tf_sm[tf_pad((j << lC) + c)] = in[(static_cast<int64_t>(c) << kTfLogP) + k0 + j];
  }
  __syncthreads();
  tf_fft<INV>(tf_sm, lC, kTfP);
  for (int i = threadIdx.x; i < kTfP; i += kTfThreads) {   // i = q K + j
    const int q = i >> lK, j = i & ((1 << lK) - 1);
    st(jb, k0 + j + (q << kTfLogP), tf_sm[tf_pad((j << lC) + q)]);
  }
}

}  // namespace
}  // namespace jtfs
