// Internal definitions shared by the host plan (jtfs_plan.cpp) and the CUDA
// kernels (jtfs_cuda.cu).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

namespace jtfs {

// A filter as the kernels evaluate it on a grid of n bins (signed bin s,
// frequency s/n): value(s) = exp(-(s - c0)^2 * a) - kappa * exp(-s^2 * a),
// with c0 = xi * n and a = 1 / (2 (sigma n)^2); kappa = 0 for low-pass
// filters.  Outside the band [lo, hi] (signed bins, clipped to
// [-n/2, n/2 - 1]) the value is below exp(-72) and treated as 0.
struct FiltD {
  float c0;
  float a;
  float kappa;
  int lo;
  int hi;
  int k;   // dyadic subsampling applied after this filter (stride level)
  int j;
  int pad;
};

// One FFT of a batched launch: where its input row and output row start
// (element offsets into the launch's source / destination buffers), which
// filter its loader applies and log2 of the source row length.
constexpr int kDU1Block = 256;
constexpr int kPoolBandAdjF = 64;  // frames per CTA of the banded tensor-core pooling adjoint  // threads per block of the U1-row gradient gather (k_dU1)

struct Job {
  int64_t src;
  int64_t dst;
  int32_t filt;
  int32_t lslog;
  int32_t b;
  int32_t pad;
};

// A tile of columns for the frequential kernels.
struct Tile {
  int b;      // clip
  int a;      // active second-order index (-1: first order)
  int t0;     // first column
  int ncols;  // columns in this tile
};

// Frequential filters of equal stride level k processed together by the
// frequential kernels: `n` filter indices (<= 16), each folded onto
// N_fr / 2^k bins.
struct FreqChunk {
  int k;
  int n;
  int beta[16];
};

// A batched FFT launch: `njobs` transforms of size 2^logn described by
// jobs[job0 .. job0 + njobs).
struct FftLaunch {
  int logn;
  int njobs;
  int job0;
  int item0;    // this launch's CTAs in the merged small-transform launch of its stage (logn <= 13)
  int n_items;
};

// Tensor-core frequential scattering (jtfs_freq_tc.cu): one chunk is up to 32
// consecutive output rows r of one frequential filter beta, i.e. 2 rc rows
// (real, imaginary) of the GEMM1 table.
struct TcChunk {
  int beta;   // filter index
  int k;      // its stride level
  int r0;     // first row of the chunk in [0, N_fr / 2^k)
  int rc;     // rows in this chunk (16 or 32)
  int b1row;  // first row of the chunk in the GEMM1 table
  int prow;   // first row of the chunk in the adjoint pooling table
  int first;  // first chunk of its filter
  int last;   // last chunk of its filter
};

struct FilterH {
  double xi;
  double sigma;
  int j;
};

// Number of sigmas beyond which a Gaussian term is dropped (exp(-72)).
constexpr double kBandSigmas = 12.0;
// Largest FFT done by one CTA in shared memory (2^13 complex, ping-pong).
constexpr int kSmallLogMax = 13;
// Columns per CTA in the frequential kernels (at most; fewer for long N_fr).
constexpr int kFreqCols = 16;
// Candidate time samples per forward time-pooling CTA (split over time); the
// plan's tuning state picks one.
constexpr int kPoolSplits[3] = {1024, 2048, 4096};

struct Plan {
  // Parameters.
  int64_t N = 0;
  int J = 0, Q = 0, Q2 = 0, J_fr = 0, Q_fr = 0;
  int64_t T = 0;
  int F = 0;
  int batch = 0;
  uint32_t flags = 0;

  // Output variants (JTFS_PLAN_UNPOOLED_T / _F): no phi_T averaging of the
  // second order (stride 2^j2, zeroth order = x), no phi_F averaging.
  bool unpooled_t = false, unpooled_f = false;
  int64_t phi2_base = 0;  // start of the second-order blocks inside Phi
  // Rows n1 of each frequential path, as offsets: path beta (second-order
  // order: phi_F, +xi, -xi; the first order uses the first 1 + K) starts at
  // row_off[beta] of its block; R_out per path unless unpooled along n1.
  std::vector<int> row_off;
  int rows1 = 0, rows2 = 0;  // rows of the first-order block, of one second-order block
  const int* d_row_off = nullptr;

  // Derived sizes.
  int logN = 0, lT = 0, lF = 0;
  int N1 = 0, N2 = 0, K = 0;
  int N_fr = 0, logNfr = 0, R_out = 0;
  int n_frames = 0, log_frames = 0;
  int n_active = 0;
  int n_beta1 = 0, n_beta2 = 0;
  int64_t phi_size = 0;

  // Filterbanks.
  std::vector<FilterH> psi1, psi2, psifr;
  FilterH phiT{}, phiF{};
  std::vector<int> k1;        // per n1: min(j1, log2 T)
  std::vector<int> n1max;     // per n2
  std::vector<int> active;    // active n2 indices
  std::vector<int> s2;        // per active index: min(j2, log2 T)
  std::vector<int> beta_k;    // per second-order beta: frequential stride level

  // Per-clip layouts (element counts).
  std::vector<int64_t> u1_off;  // per n1, in complex elements
  int64_t u1_tot = 0;
  std::vector<int64_t> y2_off;  // per active index, start of its [n1max][L2] block
  int64_t y2_tot = 0;
  std::vector<int64_t> v2_off;  // per active index, start of [n_beta2][R_out][L2]
  int64_t v2_tot = 0;
  std::vector<int64_t> phi2_off;  // per active index, offset inside Phi
  int64_t phi1_off = 0;
  std::vector<int64_t> tap_off;   // per level s in [0, lT]: time-pooling taps
  int64_t tap_tot = 0;

  // Workspace layout (byte offsets).
  size_t ws_Xh = 0, ws_U1h = 0, ws_Zs = 0, ws_S1 = 0, ws_dS1h = 0, ws_Y2 = 0,
         ws_dY2 = 0, ws_V2 = 0, ws_phi = 0, ws_dphi = 0, ws_scr = 0,
         ws_dXh = 0, ws_dS0h = 0, ws_dy = 0, ws_part = 0, ws_lossp = 0, ws_bytes = 0;
  int loss_parts = 1;  // CTAs per clip of the loss reduction (large Phi: several)
  int64_t scr_elems = 0;  // four-step scratch, complex elements

  // Launch descriptions.
  std::vector<Job> jobs;
  std::vector<FftLaunch> L_x;        // F0: FFT of x
  std::vector<FftLaunch> L_u1;       // F1: per k1 level
  std::vector<FftLaunch> L_s0;       // F2
  std::vector<FftLaunch> L_s1;       // F3
  std::vector<FftLaunch> L_y2;       // F5: per s2 level
  std::vector<FftLaunch> L_u1inplace;// B6a/B6c: rows of U1h / Zs in place (per k1 level)
  std::vector<FftLaunch> L_y2inplace;// B4: rows of dY2 in place (per s2 level)
  std::vector<FftLaunch> L_ds1;      // B4b: FFT of dS1 rows
  std::vector<FftLaunch> L_ds0;      // B7a: FFT of dS0
  std::vector<Tile> tiles1, tiles2;
  int freq_cols = kFreqCols;
  std::vector<Tile> tiles2w;  // second order, twice the columns (forward kernel)
  int freq_cols_wide = kFreqCols;
  std::vector<FreqChunk> chunks1, chunks2;
  std::vector<int4> pool_tiles;   // adjoint time pooling, banded groups: (clip, active n2, row tile, 64-sample tile)
  std::vector<int4> pool_tiles2;  // adjoint time pooling, dense groups: (clip, active n2, row tile, 512-sample tile)
  std::vector<int4> pool_fwd_tiles[3];  // forward time pooling per split: (clip, active n2, row tile, split)
  std::vector<int> pool_tile0[3];       // per split and (clip, active n2): first forward tile
  std::vector<int4> pool_tc_tiles[3];   // tensor-core forward pooling per split: (clip, active n2, even 64-row tile, split)
  std::vector<int4> pool_tc_adj_tiles;  // tensor-core adjoint pooling: (clip, active n2, even 64-row tile, 1024-sample block)
  const int4* d_pool_tc_adj_tiles = nullptr;
  const int4* d_pool_tc_tiles[3] = {nullptr, nullptr, nullptr};
  mutable int tune_pool_tc = 1;         // time pooling forward on the tensor cores where supported
  // Banded time pooling: per active n2 the tap half-width W (level samples)
  // beyond which g_s is below 2^-40 g_s[0], or 0 where the dense product is
  // used; forward tiles of the banded levels: (clip, active n2, row tile, 32-frame block).
  std::vector<int> pool_w;
  std::vector<int4> pool_band_tiles;
  // Banded groups whose widened sample range fits the circle (31 D + 2 W + 128 <= L): tiles of the
  // tensor-core banded pooling (clip, group, even 64-row slot, 32-frame block), and the FMA tiles of
  // the other banded groups.
  std::vector<int4> pool_tc_band_tiles, pool_band_rest;
  bool pool_tc_band_long = false;      // some banded tensor-core window exceeds 4096 + 128 samples
  // Banded adjoint on the tensor cores: samples per CTA of each active group (0: FMA kernel), its tiles
  // (clip, group, even 64-row slot, first sample), and the FMA kernel's tiles of the other banded groups.
  std::vector<int> pool_band_S;
  std::vector<int4> pool_tc_band_adj_tiles, pool_tiles_rest;
  const int* d_pool_band_S = nullptr;
  const int4* d_pool_tc_band_adj_tiles = nullptr;
  const int4* d_pool_tiles_rest = nullptr;
  const int4* d_pool_tc_band_tiles = nullptr;
  const int4* d_pool_band_rest = nullptr;
  // Frequential tables on the N_fr grid, one row of N_fr floats each:
  // rows [0, n_beta2): psi_beta; row n_beta2: phi_F; row n_beta2 + 1 + k:
  // phi_F periodised onto N_fr / 2^k bins (k = 0 .. log2 F).
  std::vector<float> h_ftab;
  int n_ftab = 0;
  // The same tables restricted to what the specialised kernels read: each
  // second-order beta over its band [lo, hi] (offset ftabc_off[b]), phi_F over
  // its band (offset ftabc_phi), and the phi_F level rows (offset ftabc_lev[k]).
  std::vector<float> h_ftabc;
  std::vector<int> h_ftabc_off;
  int ftabc_phi = 0;
  int ftabc_lev[16] = {};

  // Host copies of the device tables.
  std::vector<FiltD> h_psi1, h_psi2, h_beta;  // psi1/psi2 on grid N; beta on N_fr
  FiltD h_phiT{}, h_phiF{};                   // phi_T on grid N, phi_F on grid N_fr
  std::vector<float> h_taps;
  // Per n1: gain of band n1 in the coloured initialisation (§2.3),
  // 2^(lT+1) / sqrt(mean_m psi_hat(m)^6): c = 2^(k1+1) / sqrt(...) times the
  // 2^(lT-k1) that makes the adjoint of the phi_T pooling an interpolation.
  std::vector<float> h_cinit;

  // Device side.
  bool on_device = false;
  int device = -1;
  void* d_blob = nullptr;
  const float2* d_tw = nullptr;
  int twlog = 0;
  const FiltD* d_psi1 = nullptr;
  const FiltD* d_psi2 = nullptr;
  const FiltD* d_beta = nullptr;
  const float* d_taps = nullptr;
  const Job* d_jobs = nullptr;
  const Tile* d_tiles1 = nullptr;
  const Tile* d_tiles2 = nullptr;
  const Tile* d_tiles2w = nullptr;
  const FreqChunk* d_chunks1 = nullptr;
  const FreqChunk* d_chunks2 = nullptr;
  const float* d_ftab = nullptr;
  const float* d_ftabc = nullptr;
  const int* d_ftabc_off = nullptr;
  const int4* d_pool_tiles = nullptr;
  const int4* d_pool_tiles2 = nullptr;
  const int4* d_pool_fwd_tiles[3] = {nullptr, nullptr, nullptr};
  const int* d_pool_tile0[3] = {nullptr, nullptr, nullptr};

  // Tuning state (jtfs_autotune / jtfs_set_tuning): wide forward tiles for the
  // second-order frequential kernel, index into kPoolSplits, and the points
  // per CTA of batched small FFTs.
  mutable int tune_wide = 1;
  mutable int tune_split = 1;
  mutable int tune_fft_points = 4096;
  // Time-axis FFT engine (jtfs_tfft.cuh, tuning choice 6): 1 = in-place
  // radix-16 CTA transforms with all sizes <= 2^13 of a stage in one launch
  // and 2^14..2^16 on CTA clusters; 0 = the batched / four-step kernels.
  mutable int tune_tfft = 1;
  std::vector<int4> tf_items;          // (first job, jobs, log2 n, 0) per CTA
  const int4* d_tf_items = nullptr;
  std::vector<int2> du1_blocks;        // k_dU1: (U1 job - first U1 job, block of kDU1Block in its row)
  const int2* d_du1_blocks = nullptr;
  const int* d_s2 = nullptr;          // per active index
  const int* d_pool_w = nullptr;      // per active index
  const int4* d_pool_band_tiles = nullptr;
  const int* d_n1max_act = nullptr;   // per active index
  const int64_t* d_y2_off = nullptr;  // per active index
  const int64_t* d_v2_off = nullptr;
  const int64_t* d_phi2_off = nullptr;
  const int64_t* d_u1_off = nullptr;  // per n1
  const int* d_k1 = nullptr;          // per n1
  const int* d_act_n2 = nullptr;      // per active index: n2
  const int64_t* d_tap_off = nullptr; // per level s
  const float* d_cinit = nullptr;     // per n1

  // Tensor-core frequential path of the second order (jtfs_freq_tc.cu): BF16
  // hi/lo operand tables of the filter matrices (GEMM1 [tc_nr1 rows x 128],
  // forward pooling [(lF + 1) R_out rows x tc_kp2], adjoint pooling
  // [tc_np2 rows x 64], GEMM1 transposed [256 rows x tc_nr1]), the chunk
  // list, the tiles of the groups it handles (n1max <= 32, <= 64) and the
  // tiles the FFT kernels keep.
  bool tc_ok = false;
  int tc_nr1 = 0, tc_kp2 = 0, tc_np2 = 0;
  std::vector<uint16_t> tc_b1, tc_b2, tc_b2t, tc_b3;
  std::vector<TcChunk> tc_chunks;
  // Tiles of the tensor-core groups by K atoms of A1 (KA = 1 .. 5: n1max <= 32, 64, 96, 128, 160); the
  // adjoint takes KA <= 2. The FFT kernels keep the other groups: of the adjoint (tiles2_fft, wide
  // tiles2w_fft) and of the forward (the _f lists).
  std::vector<Tile> tc_tiles[5];
  std::vector<Tile> tiles2_fft, tiles2w_fft, tiles2_fft_f, tiles2w_fft_f;
  int tc_w1 = 128;                     // columns (n, re/im) of the GEMM1 table
  mutable int tune_tc = 1;
  void* d_tc = nullptr;
  const TcChunk* d_tc_chunks = nullptr;
  const Tile* d_tc_tiles[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  const Tile* d_tiles2_fft = nullptr;
  const Tile* d_tiles2w_fft = nullptr;
  const Tile* d_tiles2_fft_f = nullptr;
  const Tile* d_tiles2w_fft_f = nullptr;
  CUtensorMap tc_map[4];  // GEMM1 table, forward pooling, adjoint pooling, GEMM1 transposed

  // Measurement hook (jtfs_profile_stage): events per stage and next index.
  mutable std::vector<void*> prof_events[6];
  mutable int prof_next[6] = {0, 0, 0, 0, 0, 0};

  // The second-order frequential stage's launches are independent of one another (the two tensor-core
  // kernels, the FFT kernels of the larger groups, the first-order adjoint): they run on auxiliary
  // streams forked from and joined to the caller's stream by events, created with the plan on its
  // device (null: the launches stay on the caller's stream).  The mutex orders the event records of
  // host threads sharing the plan.
  cudaStream_t aux[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[3] = {nullptr, nullptr, nullptr};
  std::shared_ptr<std::mutex> aux_mu;
};

// Host plan construction (jtfs_plan.cpp).  Returns 0 or a JTFS_ERR_* code.
int build_plan(Plan& p, int64_t N, int J, int Q, int Q2, int J_fr, int Q_fr,
               int64_t T, int F, int batch, uint32_t flags);
int upload_plan(Plan& p);
void release_plan(Plan& p);

// Tensor-core time pooling of the second order (jtfs_pool_tc.cu): whether the
// plan's frame count has a kernel (32, 64 or 128 frames), the forward
// launch (partials in the slots of k_pool_reduce), and its expired-wait flag
// (read and cleared).
bool pool_tc_supported(const Plan& p);   // dense groups (32, 64, 128 frames) or banded tiles on tensor cores
bool pool_tc_dense(const Plan& p);       // the dense kernels apply (32, 64 or 128 frames)
int pool_tc_band_adjoint(const Plan& p, const float* dphi, float* dV2, cudaStream_t s);
// Banded groups on the tensor cores: 32 frames x 128 rows per CTA, Phi written directly.
int pool_tc_band(const Plan& p, const float* V2, float* phi, cudaStream_t s);
int pool_tc_forward(const Plan& p, const float* V2, float* part, int si, cudaStream_t s);
int pool_tc_adjoint(const Plan& p, const float* dphi, float* dV2, cudaStream_t s);
int pool_tc_error();
// Device-side status (jtfs_status): each translation unit with flags in
// device memory reads and clears its own, or sets its copy of the bounded
// waits' poll limit (c_wait_polls; polls < 0: the default bound).
int batch_nonfinite_take();
int set_wait_polls_pool(int64_t polls);
int set_wait_polls_freq(int64_t polls);
int set_wait_polls_decoder(int64_t polls);

// Tensor-core frequential path (jtfs_freq_tc.cu): host tables at plan
// construction, device copies and tensor maps at upload, release.  tc_build
// leaves tc_ok false (and the FFT tiles equal to the full lists) for shapes it
// does not handle.
void tc_build(Plan& p);
int tc_upload(Plan& p);
void tc_release(Plan& p);
// Launch the second-order forward (V2 from Y2) / adjoint (dY2 from Y2, dV2)
// on the tensor-core groups; no-ops when the plan has no such group.
// The groups with n1max <= 32 run on s, those with 33..64 rows on s2.
int tc_forward(const Plan& p, const float2* Y2, float* V2, cudaStream_t s, cudaStream_t s2);
int tc_adjoint(const Plan& p, const float2* Y2, const float* dV2, float2* dY2, cudaStream_t s, cudaStream_t s2);
bool tc_has_groups(const Plan& p, int which);  // which = KA - 1: n1max <= 32, 33..64, .., 129..160

// Stages of one plan on a caller workspace (jtfs_cuda.cu).  run_forward with
// full = false computes only what run_backward needs (phi may be NULL);
// run_backward needs a preceding run_forward on the same workspace.
int run_forward(const Plan& p, const float* x, float* phi, void* ws, bool full, cudaStream_t s);
int run_backward(const Plan& p, const float* dphi, float* dx, void* ws, cudaStream_t s);

// Several plans run stage by stage (the groups of a ragged batch): each
// time-axis FFT stage of all plans is one launch of the FFT engine (plus one
// cluster launch per size 2^14 .. 2^16) over merged job tables, in which a
// job's `pad` field names its plan; the other stages launch per plan.
constexpr int kMaxGroups = 8;
enum FftStage { FS_X, FS_U1, FS_U1IP, FS_S0, FS_S1, FS_Y2, FS_Y2IP, FS_DS1, FS_DS0, FS_COUNT };
const std::vector<FftLaunch>& stage_launches(const Plan& p, int stage);
struct FftMerged {
  const Job* jobs = nullptr;          // device
  const int4* items = nullptr;        // device: (first job, jobs, log2 n, 0) per CTA, sizes <= 2^13
  int n_items = 0;
  std::vector<FftLaunch> cluster;     // one per size 2^14 .. 2^16: (log2 n, jobs, first job)
};
// Host side of the merged tables of `n` plans (job / item arrays of every
// stage concatenated); `jobs` / `items` receive the arrays to upload, and
// `out[stage]` their ranges (pointers filled by the caller after upload).
void merge_fft_stages(const Plan* const* plans, int n, std::vector<Job>& jobs, std::vector<int4>& items,
                      FftMerged (&out)[FS_COUNT], int (&job0)[FS_COUNT], int (&item0)[FS_COUNT]);
int run_forward_multi(const Plan* const* plans, const float* const* x, float* const* phi, void* const* ws,
                      int n, const FftMerged* merged, bool full, cudaStream_t s);
int run_backward_multi(const Plan* const* plans, const float* const* dphi, float* const* dx, void* const* ws,
                       int n, const FftMerged* merged, cudaStream_t s);

}  // namespace jtfs

// Opaque handle of the C ABI.
struct jtfs_plan_s {
  jtfs::Plan p;
};
