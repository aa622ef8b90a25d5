// Learned initialiser layers: transposed 1-D convolution (stride 2, kernel 9,
// padding 4, output padding 1), its data and weight gradients, GELU, and an
// Adam update, on BF16 operands with FP32 accumulation.
//
// The three convolution products are implicit GEMMs run on the tensor cores
// with mma.sync m16n8k16 (BF16 in, FP32 accumulate).  A CTA of 4 warps owns a
// 64 x 64 output tile; operands are gathered through small functors (zero
// outside the signal) into shared memory, 32 reduction steps at a time.
//
//   forward, parity p of the output time t = 2v + p:
//     y[b][co][2v+p] = bias[co] + sum_{ci, j<5} W[ci][co][p + 8 - 2j] x[b][ci][v + j - 2]
//   data gradient:
//     dx[b][ci][u] = sum_{co, k<9} W[ci][co][k] dy[b][co][2u - 4 + k]
//   weight gradient (split over b, u; fixed-order reduction):
//     dW[ci][co][k] = sum_{b, u} x[b][ci][u] dy[b][co][2u - 4 + k]
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "jtfs.h"

namespace {

constexpr int BM = 64, BN = 64, BK = 32, kGemmThreads = 128;
constexpr int kDwSplit = 4096;  // reduction length per CTA of the weight gradient

__device__ __forceinline__ uint16_t f2bf(float f) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[m][n] = sum_k A(m, k) B(k, n) over the CTA's 64 x 64 tile and the
// reduction range [k_begin, k_end); epilogue epi(m, n, value).
template <class LA, class LB, class EPI>
__global__ void __launch_bounds__(kGemmThreads)
k_gemm_bf16(LA la, LB lb, EPI epi, int M, int N, int k_len_per_z, int K_total) {
  __shared__ __align__(16) uint16_t As[BM][BK + 8];
  __shared__ __align__(16) uint16_t Bs[BN][BK + 8];  // stored [n][k]
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int k_begin = blockIdx.z * k_len_per_z;
  const int k_end = min(K_total, k_begin + k_len_per_z);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, tg = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  for (int k0 = k_begin; k0 < k_end; k0 += BK) {
    for (int i = threadIdx.x; i < BM * BK; i += kGemmThreads) {
      const int mm = i / BK, kk = i % BK;
      const int m = m0 + mm, k = k0 + kk;
      As[mm][kk] = (m < M && k < k_end) ? la(m, k) : uint16_t(0);
    }
    for (int i = threadIdx.x; i < BN * BK; i += kGemmThreads) {
      const int nn = i % BN, kk = i / BN;
      const int n = n0 + nn, k = k0 + kk;
      Bs[nn][kk] = (n < N && k < k_end) ? lb(k, n) : uint16_t(0);
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + i * 16 + g;
        af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * tg]);
        af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * tg]);
        af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * tg + 8]);
        af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * tg + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + j * 8 + g;
        bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + 2 * tg]);
        bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + 2 * tg + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = m0 + wm + i * 16 + g, c = n0 + wn + j * 8 + 2 * tg;
      if (r < M && c < N) epi(r, c, acc[i][j][0]);
      if (r < M && c + 1 < N) epi(r, c + 1, acc[i][j][1]);
      if (r + 8 < M && c < N) epi(r + 8, c, acc[i][j][2]);
      if (r + 8 < M && c + 1 < N) epi(r + 8, c + 1, acc[i][j][3]);
    }
}

// ---- forward ---------------------------------------------------------------
struct FwdA {  // A_p[co][ci*5 + j] = W[ci][co][p + 8 - 2j] (0 outside the kernel)
  const uint16_t* w;
  int Co, p;
  __device__ uint16_t operator()(int co, int kk) const {
    const int ci = kk / 5, j = kk % 5, k = p + 8 - 2 * j;
    return (k >= 0 && k < 9) ? w[(static_cast<int64_t>(ci) * Co + co) * 9 + k] : uint16_t(0);
  }
};
struct FwdB {  // B[ci*5 + j][b*T + v] = x[b][ci][v + j - 2]
  const uint16_t* x;
  int Ci, T;
  __device__ uint16_t operator()(int kk, int n) const {
    const int ci = kk / 5, j = kk % 5, b = n / T, v = n % T, u = v + j - 2;
    return (u >= 0 && u < T) ? x[(static_cast<int64_t>(b) * Ci + ci) * T + u] : uint16_t(0);
  }
};
struct FwdEpi {  // y[b][co][2v + p] = acc + bias[co]
  float* y;
  const float* bias;
  int Co, T, p;
  __device__ void operator()(int co, int n, float v) const {
    const int b = n / T, vv = n % T;
    y[(static_cast<int64_t>(b) * Co + co) * (2 * T) + 2 * vv + p] = v + (bias ? bias[co] : 0.f);
  }
};

// ---- data gradient ----------------------------------------------------------
struct DxA {  // A[ci][co*9 + k] = W[ci][co][k]
  const uint16_t* w;
  int Co;
  __device__ uint16_t operator()(int ci, int kk) const { return w[static_cast<int64_t>(ci) * Co * 9 + kk]; }
};
struct DxB {  // B[co*9 + k][b*T + u] = dy[b][co][2u - 4 + k]
  const uint16_t* dy;
  int Co, T;
  __device__ uint16_t operator()(int kk, int n) const {
    const int co = kk / 9, k = kk % 9, b = n / T, u = n % T, t = 2 * u - 4 + k;
    return (t >= 0 && t < 2 * T) ? dy[(static_cast<int64_t>(b) * Co + co) * (2 * T) + t] : uint16_t(0);
  }
};
struct DxEpi {
  float* dx;
  int Ci, T;
  __device__ void operator()(int ci, int n, float v) const {
    const int b = n / T, u = n % T;
    dx[(static_cast<int64_t>(b) * Ci + ci) * T + u] = v;
  }
};

// ---- weight gradient --------------------------------------------------------
struct DwA {  // A[ci][b*T + u] = x[b][ci][u]
  const uint16_t* x;
  int Ci, T;
  __device__ uint16_t operator()(int ci, int kk) const {
    const int b = kk / T, u = kk % T;
    return x[(static_cast<int64_t>(b) * Ci + ci) * T + u];
  }
};
struct DwB {  // B[b*T + u][co] = dy[b][co][2u - 4 + k]
  const uint16_t* dy;
  int Co, T, k;
  __device__ uint16_t operator()(int kk, int co) const {
    const int b = kk / T, u = kk % T, t = 2 * u - 4 + k;
    return (t >= 0 && t < 2 * T) ? dy[(static_cast<int64_t>(b) * Co + co) * (2 * T) + t] : uint16_t(0);
  }
};
struct DwEpi {  // partial[split][ci][co] for tap k
  float* part;
  int Ci, Co;
  int64_t split_stride;
  __device__ void operator()(int ci, int co, float v) const {
    part[static_cast<int64_t>(blockIdx.z) * split_stride + static_cast<int64_t>(ci) * Co + co] = v;
  }
};

__global__ void k_dw_reduce(const float* __restrict__ part, float* __restrict__ dw, int Ci, int Co, int k, int nsplit) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t cc = static_cast<int64_t>(Ci) * Co;
  if (i >= cc) return;
  float acc = 0.f;
  for (int s = 0; s < nsplit; ++s) acc += part[s * cc + i];
  dw[i * 9 + k] = acc;
}

// db[co] = sum_{b, t} dy[b][co][t]; one block per co, fixed-order reduction.
__global__ void k_bias_grad(const float* __restrict__ dy, float* __restrict__ db, int B, int Co, int L) {
  __shared__ float red[256];
  const int co = blockIdx.x;
  float acc = 0.f;
  for (int64_t i = threadIdx.x; i < static_cast<int64_t>(B) * L; i += blockDim.x) {
    const int64_t b = i / L, t = i % L;
    acc += dy[(b * Co + co) * L + t];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[co] = red[0];
}

__global__ void k_gelu_fwd(const float* __restrict__ z, uint16_t* __restrict__ h, int64_t n) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = z[i];
  h[i] = f2bf(0.5f * v * (1.f + erff(v * 0.70710678118654752f)));
}

// dz = dh * GELU'(z), GELU'(z) = (1 + erf(z/sqrt2))/2 + z exp(-z^2/2)/sqrt(2 pi)
__global__ void k_gelu_bwd(const float* __restrict__ dh, const float* __restrict__ z, float* __restrict__ dz,
                           int64_t n) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = z[i];
  const float d = 0.5f * (1.f + erff(v * 0.70710678118654752f)) + v * expf(-0.5f * v * v) * 0.39894228040143268f;
  dz[i] = dh[i] * d;
}

__global__ void k_cast_bf16(const float* __restrict__ x, uint16_t* __restrict__ y, int64_t n) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) y[i] = f2bf(x[i]);
}

__global__ void k_cast_bf16_rows(const float* __restrict__ x, const float* __restrict__ s, uint16_t* __restrict__ y,
                                 int C, int64_t T, int64_t n) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) y[i] = f2bf(x[i] * s[(i / T) % C]);
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

int ok() { return cudaGetLastError() == cudaSuccess ? JTFS_OK : JTFS_ERR_CUDA; }
unsigned blocks(int64_t n) { return static_cast<unsigned>((n + 255) / 256); }

bool bad_dims(int B, int Ci, int Co, int T) {
  return B < 1 || Ci < 1 || Co < 1 || T < 1 || static_cast<int64_t>(B) * T > (int64_t(1) << 30) ||
         static_cast<int64_t>(Ci) * 9 > (int64_t(1) << 30);
}

}  // namespace

extern "C" int jtfs_convt_forward(const uint16_t* x, const uint16_t* w, const float* bias, float* y, int B, int Ci,
                                  int Co, int T, void* stream) {
  if (!x || !w || !y || bad_dims(B, Ci, Co, T)) return JTFS_ERR_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int N = B * T, K = Ci * 5;
  dim3 grid((N + BN - 1) / BN, (Co + BM - 1) / BM, 1);
  for (int p = 0; p < 2; ++p)
    k_gemm_bf16<<<grid, kGemmThreads, 0, s>>>(FwdA{w, Co, p}, FwdB{x, Ci, T}, FwdEpi{y, bias, Co, T, p}, Co, N, K, K);
  return ok();
}

extern "C" int jtfs_convt_backward_data(const uint16_t* dy, const uint16_t* w, float* dx, int B, int Ci, int Co,
                                        int T, void* stream) {
  if (!dy || !w || !dx || bad_dims(B, Ci, Co, T)) return JTFS_ERR_ARG;
  const int N = B * T, K = Co * 9;
  dim3 grid((N + BN - 1) / BN, (Ci + BM - 1) / BM, 1);
  k_gemm_bf16<<<grid, kGemmThreads, 0, static_cast<cudaStream_t>(stream)>>>(DxA{w, Co}, DxB{dy, Co, T},
                                                                            DxEpi{dx, Ci, T}, Ci, N, K, K);
  return ok();
}

extern "C" size_t jtfs_convt_weight_workspace_bytes(int B, int Ci, int Co, int T) {
  if (bad_dims(B, Ci, Co, T)) return 0;
  const int64_t K = static_cast<int64_t>(B) * T;
  const int64_t nsplit = (K + kDwSplit - 1) / kDwSplit;
  return static_cast<size_t>(nsplit) * Ci * Co * sizeof(float);
}

extern "C" int jtfs_convt_backward_weight(const uint16_t* x, const uint16_t* dy, const float* dy_f32, float* dw,
                                          float* db, int B, int Ci, int Co, int T, void* workspace, void* stream) {
  if (!x || !dy || !dw || !workspace || bad_dims(B, Ci, Co, T)) return JTFS_ERR_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int K = B * T;
  const int nsplit = (K + kDwSplit - 1) / kDwSplit;
  float* part = static_cast<float*>(workspace);
  const int64_t cc = static_cast<int64_t>(Ci) * Co;
  dim3 grid((Co + BN - 1) / BN, (Ci + BM - 1) / BM, nsplit);
  for (int k = 0; k < 9; ++k) {
    k_gemm_bf16<<<grid, kGemmThreads, 0, s>>>(DwA{x, Ci, T}, DwB{dy, Co, T, k}, DwEpi{part, Ci, Co, cc}, Ci, Co,
                                              kDwSplit, K);
    if (ok() != JTFS_OK) return JTFS_ERR_CUDA;
    k_dw_reduce<<<blocks(cc), 256, 0, s>>>(part, dw, Ci, Co, k, nsplit);
    if (ok() != JTFS_OK) return JTFS_ERR_CUDA;
  }
  if (db && dy_f32) k_bias_grad<<<Co, 256, 0, s>>>(dy_f32, db, B, Co, 2 * T);
  return ok();
}

extern "C" int jtfs_gelu_forward(const float* z, uint16_t* h, int64_t n, void* stream) {
  if (!z || !h || n < 0) return JTFS_ERR_ARG;
  if (n) k_gelu_fwd<<<blocks(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(z, h, n);
  return ok();
}

extern "C" int jtfs_gelu_backward(const float* dh, const float* z, float* dz, int64_t n, void* stream) {
  if (!dh || !z || !dz || n < 0) return JTFS_ERR_ARG;
  if (n) k_gelu_bwd<<<blocks(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(dh, z, dz, n);
  return ok();
}

extern "C" int jtfs_cast_bf16(const float* x, uint16_t* y, int64_t n, void* stream) {
  if (!x || !y || n < 0) return JTFS_ERR_ARG;
  if (n) k_cast_bf16<<<blocks(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, y, n);
  return ok();
}

extern "C" int jtfs_cast_bf16_rows(const float* x, const float* row_scale, uint16_t* y, int B, int C, int64_t T,
                                   void* stream) {
  if (!x || !row_scale || !y || B < 0 || C < 1 || T < 0) return JTFS_ERR_ARG;
  const int64_t n = static_cast<int64_t>(B) * C * T;
  if (n) k_cast_bf16_rows<<<blocks(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, row_scale, y, C, T, n);
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
