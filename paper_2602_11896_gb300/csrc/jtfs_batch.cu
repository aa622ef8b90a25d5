// Ragged batches: clips of any lengths, grouped by padded length, each group
// on its own plan.  A clip of length L is zero-padded on the right to the
// next power of two >= max(L, T) (§3.2's padding, periodic boundary), its Phi
// computed there and cropped to the first ceil(L/T) frames of every row; the
// loss runs over the kept frames only, so the crop's adjoint fills zeros.
// With JTFS_BATCH_REFLECT the padding is on both sides instead (§3.2's
// padding and unpadding): P samples per side, P where the slowest time
// envelope exp(-2 pi^2 sigma^2 t^2) of psi1, psi2 and phi_T drops below 1e-3,
// padded length n = next power of two >= L + 2P, left pad p0 = T floor((n -
// L) / 2T), mirror extension without repeating the edge samples; the kept
// frames start at p0 / T and the gradient folds the mirrored samples back.
// Packed layouts are described in include/jtfs.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <new>
#include <vector>

#include "jtfs.h"
#include "jtfs_internal.h"

namespace jtfs {
namespace {

constexpr int kThreadsB = 256;

// Per clip (device copy): packed offsets, offsets of its group's buffers in
// the workspace (in floats), sizes.
struct ClipD {
  int64_t so;     // packed samples
  int64_t po;     // packed Phi
  int64_t ypad;   // padded input row
  int64_t phi;    // full (uncropped) Phi
  int64_t dphi;   // its gradient
  int64_t dy;     // gradient w.r.t. the padded row
  int L, N, nf, nf_full, rows, pad;
  int f0;         // first kept frame
  int p0;         // left pad (samples)
  int refl;       // 1: mirror padding on both sides, 0: zeros on the right
  int pad2;
  int64_t g;      // gradient w.r.t. the clip's samples (offset in floats)
};

struct Group {
  Plan plan;
  std::vector<int> clips;
  size_t ws_off = 0, ypad_off = 0, phi_off = 0, dphi_off = 0, dy_off = 0;
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Index into a clip of L samples of position u relative to its first sample,
// mirrored without repeating the edge samples (period 2(L-1)).
__device__ __forceinline__ int mirror(int u, int L) {
  if (L == 1) return 0;
  const int per = 2 * (L - 1);
  int r = u % per;
  if (r < 0) r += per;
  return r < L ? r : per - r;
}

// Padded rows from packed samples: zeros beyond L, or the mirror extension.
__global__ void __launch_bounds__(kThreadsB) k_gather(const ClipD* __restrict__ clips, const float* __restrict__ y,
                                                     float* __restrict__ ws) {
  const ClipD c = clips[blockIdx.y];
  for (int t = blockIdx.x * kThreadsB + threadIdx.x; t < c.N; t += gridDim.x * kThreadsB)
    ws[c.ypad + t] = c.refl ? y[c.so + mirror(t - c.p0, c.L)] : (t < c.L ? y[c.so + t] : 0.f);
}

// Adjoint of the mirror extension: sample t of a reflect clip collects every
// padded position that copies it (positions p0 + t + k per, and p0 - t + k per
// for 0 < t < L-1), summed in ascending order; written over the padded row,
// which the backward pass no longer reads.
__global__ void __launch_bounds__(kThreadsB) k_fold(const ClipD* __restrict__ clips, float* ws) {
  const ClipD c = clips[blockIdx.y];
  if (!c.refl) return;
  const float* d = ws + c.dy;
  const int per = c.L == 1 ? 1 : 2 * (c.L - 1);
  for (int t = blockIdx.x * kThreadsB + threadIdx.x; t < c.L; t += gridDim.x * kThreadsB) {
    float acc = 0.f;
    for (int s = ((c.p0 + t) % per + per) % per; s < c.N; s += per) acc += d[s];
    if (t > 0 && t < c.L - 1)
      for (int s = ((c.p0 - t) % per + per) % per; s < c.N; s += per) acc += d[s];
    ws[c.g + t] = acc;
  }
}

// Set by k_masked_loss_sum when a clip's loss is NaN or infinite (jtfs_status).
__device__ int g_batch_nonfinite;

// Loss over the kept frames, dPhi = 2 (Phi - target) there and 0 on cropped
// frames: kLossParts CTAs per clip each sum a fixed range of its entries in
// double, then k_masked_loss_sum adds the parts of each clip in a fixed order
// (deterministic).
constexpr int kLossParts = 16;

__global__ void __launch_bounds__(512) k_masked_loss_part(const ClipD* __restrict__ clips,
                                                         const float* __restrict__ tgt, float* ws,
                                                         double* __restrict__ part) {
  __shared__ double red[512];
  const ClipD c = clips[blockIdx.y];
  const int lnf = __ffs(c.nf_full) - 1;   // N / T frames: a power of two
  const int64_t total = static_cast<int64_t>(c.rows) << lnf;
  const int64_t chunk = (total + kLossParts - 1) / kLossParts;
  const int64_t lo = static_cast<int64_t>(blockIdx.x) * chunk, hi = min(total, lo + chunk);
  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const int r = static_cast<int>(i >> lnf), f = static_cast<int>(i & (c.nf_full - 1));
    float d = 0.f;
    if (f >= c.f0 && f < c.f0 + c.nf) {
      d = ws[c.phi + i] - tgt[c.po + static_cast<int64_t>(r) * c.nf + (f - c.f0)];
      acc += static_cast<double>(d) * d;
    }
    ws[c.dphi + i] = 2.f * d;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[static_cast<int64_t>(blockIdx.y) * kLossParts + blockIdx.x] = red[0];
}

__global__ void k_masked_loss_sum(const double* __restrict__ part, float* __restrict__ loss, int count) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count) return;
  double acc = 0.0;
  for (int q = 0; q < kLossParts; ++q) acc += part[static_cast<int64_t>(b) * kLossParts + q];
  loss[b] = static_cast<float>(acc);
  if (!isfinite(acc)) atomicOr(&g_batch_nonfinite, 1);
}

// Cropped Phi, packed.
__global__ void __launch_bounds__(kThreadsB) k_crop(const ClipD* __restrict__ clips, const float* __restrict__ ws,
                                                   float* __restrict__ phi) {
  const ClipD c = clips[blockIdx.y];
  const int64_t total = static_cast<int64_t>(c.rows) * c.nf;
  for (int64_t i = blockIdx.x * kThreadsB + threadIdx.x; i < total; i += static_cast<int64_t>(gridDim.x) * kThreadsB) {
    const int64_t r = i / c.nf, f = i % c.nf;
    phi[c.po + i] = ws[c.phi + r * c.nf_full + c.f0 + f];
  }
}

// Adam on the packed samples (gradient = first L samples of the padded
// gradient); the 1-based step index is read from device memory.
__global__ void __launch_bounds__(kThreadsB) k_adam_packed(const ClipD* __restrict__ clips, const float* __restrict__ ws,
                                                          float* __restrict__ y, float* __restrict__ m,
                                                          float* __restrict__ v, const int* __restrict__ step,
                                                          float lr) {
  const ClipD c = clips[blockIdx.y];
  const int t_step = *step;
  const float c1 = 1.f / (1.f - powf(0.9f, static_cast<float>(t_step)));
  const float c2 = 1.f / (1.f - powf(0.999f, static_cast<float>(t_step)));
  for (int t = blockIdx.x * kThreadsB + threadIdx.x; t < c.L; t += gridDim.x * kThreadsB) {
    const int64_t i = c.so + t;
    const float g = ws[c.g + t];
    const float mi = 0.9f * m[i] + 0.1f * g;
    const float vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    y[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
  }
}

__global__ void k_step_increment(int* step) { *step += 1; }

}  // namespace

int batch_nonfinite_take() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_batch_nonfinite, sizeof(int)) != cudaSuccess) return JTFS_ERR_CUDA;
  const int zero = 0;
  if (v && cudaMemcpyToSymbol(g_batch_nonfinite, &zero, sizeof(int)) != cudaSuccess) return JTFS_ERR_CUDA;
  return v;
}

}  // namespace jtfs

struct jtfs_batch_s {
  std::vector<int64_t> lengths, so, po;
  std::vector<jtfs::Group> groups;
  std::vector<jtfs::ClipD> clips;
  jtfs::ClipD* d_clips = nullptr;
  size_t ws_bytes = 0;
  int max_blocks_x = 1;
  bool on_device = false;
  // Time-axis FFT stages of all groups merged (one launch per stage, one
  // cluster launch per size 2^14 .. 2^16); empty with more than kMaxGroups
  // groups, which then run one after another.
  size_t lossp_off = 0;   // per-clip partial loss sums (kLossParts doubles per clip)
  bool merged_ok = false;
  jtfs::FftMerged merged[jtfs::FS_COUNT];
  void* d_merged = nullptr;
};

namespace {

void destroy_batch(jtfs_batch_s* b) {
  if (!b) return;
  for (auto& g : b->groups) jtfs::release_plan(g.plan);
  if (b->d_clips) cudaFree(b->d_clips);
  if (b->d_merged) cudaFree(b->d_merged);
  delete b;
}

}  // namespace

extern "C" int jtfs_batch_create(jtfs_batch_t* out, const int64_t* lengths, int count, int J, int Q, int Q2,
                                 int J_fr, int Q_fr, int64_t T, int F, uint32_t flags) {
  if (!out || !lengths || count < 1) return JTFS_ERR_ARG;
  *out = nullptr;
  if (T < 2 || (T & (T - 1))) return JTFS_ERR_SHAPE;
  // The crop and the masked loss index Phi as rows x frames: unpooled layouts are not batched.
  if (flags & (JTFS_PLAN_UNPOOLED_T | JTFS_PLAN_UNPOOLED_F)) return JTFS_ERR_ARG;
  const bool refl = (flags & JTFS_BATCH_REFLECT) != 0;
  flags &= ~JTFS_BATCH_REFLECT;
  jtfs_batch_s* b = new (std::nothrow) jtfs_batch_s();
  if (!b) return JTFS_ERR_NOMEM;
  int rc = JTFS_OK;
  try {
    // Mirror pad width from the filterbanks (independent of the length).
    int64_t P = 0;
    if (refl) {
      jtfs::Plan probe;
      const int64_t n_probe = std::max<int64_t>({T, int64_t(1) << std::min(J + 1, 20), 16});
      rc = jtfs::build_plan(probe, n_probe, J, Q, Q2, J_fr, Q_fr, T, F, 1, JTFS_PLAN_HOST_ONLY);
      if (rc == JTFS_OK) {
        double sig = probe.phiT.sigma;
        for (const auto& f : probe.psi1) sig = std::min(sig, f.sigma);
        for (const auto& f : probe.psi2) sig = std::min(sig, f.sigma);
        P = static_cast<int64_t>(std::ceil(std::sqrt(std::log(1000.0) / 2.0) / (M_PI * sig)));
      }
    }
    std::map<int64_t, std::vector<int>> by_n;
    for (int i = 0; i < count && rc == JTFS_OK; ++i) {
      const int64_t L = lengths[i];
      if (L < 1 || L > (int64_t(1) << 20)) {
        rc = JTFS_ERR_SHAPE;
        break;
      }
      int64_t n = 1;
      while (n < std::max<int64_t>(refl ? L + 2 * P : L, T)) n <<= 1;
      if (n > (int64_t(1) << 20)) {
        rc = JTFS_ERR_SHAPE;
        break;
      }
      by_n[n].push_back(i);
      b->lengths.push_back(L);
    }
    if (rc == JTFS_OK) {
      b->groups.resize(by_n.size());
      size_t gi = 0, off = 0;
      b->clips.assign(count, jtfs::ClipD{});
      for (auto& kv : by_n) {
        jtfs::Group& g = b->groups[gi++];
        g.clips = kv.second;
        rc = jtfs::build_plan(g.plan, kv.first, J, Q, Q2, J_fr, Q_fr, T, F, static_cast<int>(g.clips.size()), flags);
        if (rc != JTFS_OK) break;
        if (!(flags & JTFS_PLAN_HOST_ONLY)) {
          rc = jtfs::upload_plan(g.plan);
          if (rc != JTFS_OK) break;
        }
        const size_t B = g.clips.size(), N = static_cast<size_t>(kv.first), Pz = static_cast<size_t>(g.plan.phi_size);
        g.ws_off = off;
        off = jtfs::align256(off + g.plan.ws_bytes);
        g.ypad_off = off;
        off = jtfs::align256(off + B * N * sizeof(float));
        g.phi_off = off;
        off = jtfs::align256(off + B * Pz * sizeof(float));
        g.dphi_off = off;
        off = jtfs::align256(off + B * Pz * sizeof(float));
        g.dy_off = off;
        off = jtfs::align256(off + B * N * sizeof(float));
        for (size_t k = 0; k < B; ++k) {
          jtfs::ClipD& c = b->clips[g.clips[k]];
          c.L = static_cast<int>(lengths[g.clips[k]]);
          c.N = static_cast<int>(N);
          c.nf_full = g.plan.n_frames;
          c.nf = static_cast<int>((c.L + T - 1) / T);
          c.rows = static_cast<int>(Pz / g.plan.n_frames);
          c.refl = refl ? 1 : 0;
          c.p0 = refl ? static_cast<int>(T * ((static_cast<int64_t>(N) - c.L) / (2 * T))) : 0;
          c.f0 = static_cast<int>(c.p0 / T);
          c.ypad = static_cast<int64_t>(g.ypad_off / sizeof(float) + k * N);
          c.phi = static_cast<int64_t>(g.phi_off / sizeof(float) + k * Pz);
          c.dphi = static_cast<int64_t>(g.dphi_off / sizeof(float) + k * Pz);
          c.dy = static_cast<int64_t>(g.dy_off / sizeof(float) + k * N);
          c.g = refl ? c.ypad : c.dy;
        }
        b->max_blocks_x = std::max<int>(b->max_blocks_x, static_cast<int>((N + 255) / 256));
      }
      b->lossp_off = off;
      off = jtfs::align256(off + size_t(count) * jtfs::kLossParts * sizeof(double));
      b->ws_bytes = off;
      b->so.assign(count + 1, 0);
      b->po.assign(count + 1, 0);
      for (int i = 0; i < count && rc == JTFS_OK; ++i) {
        jtfs::ClipD& c = b->clips[i];
        b->so[i + 1] = b->so[i] + c.L;
        b->po[i + 1] = b->po[i] + static_cast<int64_t>(c.rows) * c.nf;
        c.so = b->so[i];
        c.po = b->po[i];
      }
      if (rc == JTFS_OK && !(flags & JTFS_PLAN_HOST_ONLY)) {
        if (cudaMalloc(&b->d_clips, count * sizeof(jtfs::ClipD)) != cudaSuccess) rc = JTFS_ERR_NOMEM;
        else if (cudaMemcpy(b->d_clips, b->clips.data(), count * sizeof(jtfs::ClipD), cudaMemcpyHostToDevice) !=
                 cudaSuccess)
          rc = JTFS_ERR_CUDA;
        b->on_device = rc == JTFS_OK;
      }
      if (rc == JTFS_OK && b->on_device && b->groups.size() <= size_t(jtfs::kMaxGroups)) {
        // Merged job and item tables of the time-axis FFT stages.
        std::vector<const jtfs::Plan*> plans;
        for (const auto& g : b->groups) plans.push_back(&g.plan);
        std::vector<jtfs::Job> mj;
        std::vector<int4> mi;
        int j0[jtfs::FS_COUNT], i0[jtfs::FS_COUNT];
        jtfs::merge_fft_stages(plans.data(), static_cast<int>(plans.size()), mj, mi, b->merged, j0, i0);
        const size_t jb = mj.size() * sizeof(jtfs::Job), ib = mi.size() * sizeof(int4);
        if (cudaMalloc(&b->d_merged, jtfs::align256(jb) + std::max<size_t>(ib, 16)) != cudaSuccess) {
          rc = JTFS_ERR_NOMEM;
        } else {
          auto* at = static_cast<unsigned char*>(b->d_merged);
          auto* dj = reinterpret_cast<jtfs::Job*>(at);
          auto* di = reinterpret_cast<int4*>(at + jtfs::align256(jb));
          if ((jb && cudaMemcpy(dj, mj.data(), jb, cudaMemcpyHostToDevice) != cudaSuccess) ||
              (ib && cudaMemcpy(di, mi.data(), ib, cudaMemcpyHostToDevice) != cudaSuccess))
            rc = JTFS_ERR_CUDA;
          for (int st = 0; st < jtfs::FS_COUNT; ++st) {
            b->merged[st].jobs = dj + j0[st];
            b->merged[st].items = di + i0[st];
          }
          b->merged_ok = rc == JTFS_OK;
        }
      }
    }
  } catch (...) {
    rc = JTFS_ERR_NOMEM;
  }
  if (rc != JTFS_OK) {
    destroy_batch(b);
    return rc;
  }
  *out = b;
  return JTFS_OK;
}

extern "C" int jtfs_plan_ragged(jtfs_batch_t* out, const int64_t* lengths, int count, int J, int Q, int Q2,
                                int J_fr, int Q_fr, int64_t T, int F, uint32_t flags) {
  return jtfs_batch_create(out, lengths, count, J, Q, Q2, J_fr, Q_fr, T, F, flags);
}

extern "C" int jtfs_batch_destroy(jtfs_batch_t batch) {
  destroy_batch(batch);
  return JTFS_OK;
}

extern "C" int jtfs_batch_layout(jtfs_batch_t batch, int64_t* sample_off, int64_t* phi_off) {
  if (!batch) return JTFS_ERR_ARG;
  const int n = static_cast<int>(batch->lengths.size());
  for (int i = 0; i <= n; ++i) {
    if (sample_off) sample_off[i] = batch->so[i];
    if (phi_off) phi_off[i] = batch->po[i];
  }
  return n;
}

extern "C" size_t jtfs_batch_workspace_bytes(jtfs_batch_t batch) { return batch ? batch->ws_bytes : 0; }

namespace {

int batch_check(jtfs_batch_t b, void* ws) {
  if (!b) return JTFS_ERR_ARG;
  if (!b->on_device) return JTFS_ERR_NODEVICE;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return JTFS_ERR_WORKSPACE;
  return JTFS_OK;
}

int launched() { return cudaGetLastError() == cudaSuccess ? JTFS_OK : JTFS_ERR_CUDA; }

int gather_and_forward(jtfs_batch_t b, const float* x, void* ws, bool full, cudaStream_t s) {
  auto* base = static_cast<unsigned char*>(ws);
  const int count = static_cast<int>(b->lengths.size());
  jtfs::k_gather<<<dim3(std::min(b->max_blocks_x, 1024), count), jtfs::kThreadsB, 0, s>>>(
      b->d_clips, x, reinterpret_cast<float*>(base));
  if (launched() != JTFS_OK) return JTFS_ERR_CUDA;
  if (b->merged_ok) {
    const int n = static_cast<int>(b->groups.size());
    const jtfs::Plan* plans[jtfs::kMaxGroups];
    const float* x_g[jtfs::kMaxGroups];
    float* phi_g[jtfs::kMaxGroups];
    void* ws_g[jtfs::kMaxGroups];
    for (int i = 0; i < n; ++i) {
      const auto& g = b->groups[size_t(i)];
      plans[i] = &g.plan;
      x_g[i] = reinterpret_cast<const float*>(base + g.ypad_off);
      phi_g[i] = reinterpret_cast<float*>(base + g.phi_off);
      ws_g[i] = base + g.ws_off;
    }
    return jtfs::run_forward_multi(plans, x_g, phi_g, ws_g, n, b->merged, full, s);
  }
  for (const auto& g : b->groups) {
    const int rc = jtfs::run_forward(g.plan, reinterpret_cast<const float*>(base + g.ypad_off),
                                     reinterpret_cast<float*>(base + g.phi_off), base + g.ws_off, full, s);
    if (rc != JTFS_OK) return rc;
  }
  return JTFS_OK;
}

int backward_all(jtfs_batch_t b, void* ws, cudaStream_t s) {
  auto* base = static_cast<unsigned char*>(ws);
  if (b->merged_ok) {
    const int n = static_cast<int>(b->groups.size());
    const jtfs::Plan* plans[jtfs::kMaxGroups];
    const float* dphi_g[jtfs::kMaxGroups];
    float* dy_g[jtfs::kMaxGroups];
    void* ws_g[jtfs::kMaxGroups];
    for (int i = 0; i < n; ++i) {
      const auto& g = b->groups[size_t(i)];
      plans[i] = &g.plan;
      dphi_g[i] = reinterpret_cast<const float*>(base + g.dphi_off);
      dy_g[i] = reinterpret_cast<float*>(base + g.dy_off);
      ws_g[i] = base + g.ws_off;
    }
    return jtfs::run_backward_multi(plans, dphi_g, dy_g, ws_g, n, b->merged, s);
  }
  for (const auto& g : b->groups) {
    const int rc = jtfs::run_backward(g.plan, reinterpret_cast<const float*>(base + g.dphi_off),
                                      reinterpret_cast<float*>(base + g.dy_off), base + g.ws_off, s);
    if (rc != JTFS_OK) return rc;
  }
  return JTFS_OK;
}

}  // namespace

extern "C" int jtfs_batch_forward(jtfs_batch_t batch, const float* x, float* phi, void* workspace, void* stream) {
  const int rc0 = batch_check(batch, workspace);
  if (rc0 != JTFS_OK) return rc0;
  if (!x || !phi) return JTFS_ERR_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = gather_and_forward(batch, x, workspace, true, s);
  if (rc != JTFS_OK) return rc;
  const int count = static_cast<int>(batch->lengths.size());
  jtfs::k_crop<<<dim3(64, count), jtfs::kThreadsB, 0, s>>>(batch->d_clips, static_cast<const float*>(workspace), phi);
  return launched();
}

extern "C" int jtfs_batch_metamer_step(jtfs_batch_t batch, float* y, const float* phi_target, float* adam_m,
                                       float* adam_v, int32_t* step, float lr, float* loss, void* workspace,
                                       void* stream) {
  const int rc0 = batch_check(batch, workspace);
  if (rc0 != JTFS_OK) return rc0;
  if (!y || !phi_target || !adam_m || !adam_v || !step || !loss || !(lr > 0.f)) return JTFS_ERR_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto* base = static_cast<unsigned char*>(workspace);
  const int count = static_cast<int>(batch->lengths.size());
  int rc = gather_and_forward(batch, y, workspace, true, s);
  if (rc != JTFS_OK) return rc;
  jtfs::k_masked_loss_part<<<dim3(jtfs::kLossParts, count), 512, 0, s>>>(
      batch->d_clips, phi_target, reinterpret_cast<float*>(base), reinterpret_cast<double*>(base + batch->lossp_off));
  if (launched() != JTFS_OK) return JTFS_ERR_CUDA;
  jtfs::k_masked_loss_sum<<<(count + 127) / 128, 128, 0, s>>>(reinterpret_cast<const double*>(base + batch->lossp_off),
                                                               loss, count);
  if (launched() != JTFS_OK) return JTFS_ERR_CUDA;
  rc = backward_all(batch, workspace, s);
  if (rc != JTFS_OK) return rc;
  jtfs::k_fold<<<dim3(std::min(batch->max_blocks_x, 1024), count), jtfs::kThreadsB, 0, s>>>(
      batch->d_clips, reinterpret_cast<float*>(base));
  if (launched() != JTFS_OK) return JTFS_ERR_CUDA;
  jtfs::k_adam_packed<<<dim3(std::min(batch->max_blocks_x, 1024), count), jtfs::kThreadsB, 0, s>>>(
      batch->d_clips, reinterpret_cast<const float*>(base), y, adam_m, adam_v, step, lr);
  if (launched() != JTFS_OK) return JTFS_ERR_CUDA;
  jtfs::k_step_increment<<<1, 1, 0, s>>>(step);
  return launched();
}
