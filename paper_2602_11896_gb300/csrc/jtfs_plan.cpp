// Host side of a JTFS plan: filterbank design (§3.1), the multirate schedule
// of §3.2-§3.5, per-clip layouts, workspace layout, the job tables of every
// batched FFT launch, and the upload of the small device tables.
//
// Readings of passages the paper leaves open (shared with nothing else in
// this library; the CUDA kernels only consume the tables built here):
//  - §3.1 listing uses an undefined `r`: taken as r_psi = sqrt(1/2).
//  - filter field 'j': the largest k with 2^k (xi + 3 sigma) <= 1/2 (>= 0).
//  - phi_T has sigma = 0.1/T cycles/sample, phi_F sigma = 0.1/F cycles/bin;
//    output strides are T in time and 2^floor(log2 F) along n1.
//  - strides: k1 = min(j1, log2 T); second-order rows j1 < j2 at total stride
//    s2 = min(j2, log2 T); frequential k_fr = min(j_fr, floor(log2 F)).
//  - N_fr = next power of two >= N1 + 2^(J_fr + 1).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "jtfs.h"
#include "jtfs_internal.h"

namespace jtfs {
namespace {

constexpr double kSigma0 = 0.1;  // §3.1 listing

// §3.1 generator: constant-Q geometric progression down to the elbow
// sigma_min = sigma0 / 2^J, then Q-1 constant-bandwidth filters.
std::vector<FilterH> filterbank(int J, int Q) {
  std::vector<FilterH> out;
  const double r_psi = std::sqrt(0.5);
  double xi = std::max(1.0 / (1.0 + std::pow(2.0, 3.0 / Q)), 0.35);
  const double factor = 1.0 / std::pow(2.0, 1.0 / Q);
  double sigma = (1.0 - factor) / (1.0 + factor) * xi / std::sqrt(2.0 * std::log(1.0 / r_psi));
  const double sigma_min = kSigma0 / std::pow(2.0, J);
  if (sigma <= sigma_min) {
    xi = sigma;
  } else {
    out.push_back({xi, sigma, 0});
    while (sigma > sigma_min * std::pow(2.0, 1.0 / Q)) {
      xi /= std::pow(2.0, 1.0 / Q);
      sigma /= std::pow(2.0, 1.0 / Q);
      out.push_back({xi, sigma, 0});
    }
  }
  const double elbow_xi = xi;
  for (int q = 0; q < Q - 1; ++q) {
    xi -= 1.0 / Q * elbow_xi;
    out.push_back({xi, sigma_min, 0});
  }
  return out;
}

int max_subsampling(double xi, double sigma) {
  const int j = static_cast<int>(std::floor(std::log2(0.5 / (xi + 3.0 * sigma))));
  return j < 0 ? 0 : j;
}

int ilog2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// Filter on an n-bin grid for the kernels (see FiltD).
FiltD make_filt(double xi, double sigma, int n, int k, int j, bool lowpass) {
  FiltD f{};
  const double c0 = xi * n;
  const double sn = sigma * n;
  f.c0 = static_cast<float>(c0);
  f.a = static_cast<float>(1.0 / (2.0 * sn * sn));
  double kappa = lowpass ? 0.0 : std::exp(-xi * xi / (2.0 * sigma * sigma));
  if (kappa < 1e-35) kappa = 0.0;
  f.kappa = static_cast<float>(kappa);
  const double w = kBandSigmas * sn;
  double lo = std::floor(c0 - w), hi = std::ceil(c0 + w);
  if (kappa > 0.0) {
    lo = std::min(lo, std::floor(-w));
    hi = std::max(hi, std::ceil(w));
  }
  lo = std::max(lo, -double(n / 2));
  hi = std::min(hi, double(n / 2 - 1));
  f.lo = static_cast<int>(lo);
  f.hi = static_cast<int>(hi);
  f.k = k;
  f.j = j;
  return f;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

int build_plan(Plan& p, int64_t N, int J, int Q, int Q2, int J_fr, int Q_fr,
               int64_t T, int F, int batch, uint32_t flags) {
  if (!is_pow2(N) || N < 16 || N > (int64_t(1) << 20)) return JTFS_ERR_SHAPE;
  if (!is_pow2(T) || T < 2 || T > N) return JTFS_ERR_SHAPE;
  if (F < 1 || batch < 1 || J < 1 || Q < 1 || Q2 < 1 || J_fr < 1 || Q_fr < 1) return JTFS_ERR_SHAPE;
  if (J > 24 || Q > 64 || Q2 > 64 || J_fr > 12 || Q_fr > 16) return JTFS_ERR_SHAPE;
  p.N = N; p.J = J; p.Q = Q; p.Q2 = Q2; p.J_fr = J_fr; p.Q_fr = Q_fr;
  p.T = T; p.F = F; p.batch = batch; p.flags = flags;
  p.unpooled_t = (flags & JTFS_PLAN_UNPOOLED_T) != 0;
  p.unpooled_f = (flags & JTFS_PLAN_UNPOOLED_F) != 0;
  p.logN = ilog2(N);
  p.lT = ilog2(T);
  p.lF = static_cast<int>(std::floor(std::log2(double(F))));

  p.psi1 = filterbank(J, Q);
  p.psi2 = filterbank(J, Q2);
  p.psifr = filterbank(J_fr, Q_fr);
  if (p.psi1.empty() || p.psi2.empty() || p.psifr.empty()) return JTFS_ERR_SHAPE;
  for (auto* fb : {&p.psi1, &p.psi2, &p.psifr})
    for (auto& f : *fb) f.j = max_subsampling(f.xi, f.sigma);
  p.phiT = {0.0, kSigma0 / double(T), 0};
  p.phiT.j = max_subsampling(0.0, p.phiT.sigma);
  p.phiF = {0.0, kSigma0 / double(F), 0};
  p.phiF.j = max_subsampling(0.0, p.phiF.sigma);

  p.N1 = static_cast<int>(p.psi1.size());
  p.N2 = static_cast<int>(p.psi2.size());
  p.K = static_cast<int>(p.psifr.size());
  p.N_fr = 1;
  while (p.N_fr < p.N1 + (1 << (J_fr + 1))) p.N_fr <<= 1;
  p.logNfr = ilog2(p.N_fr);
  if (p.lF > p.logNfr) return JTFS_ERR_SHAPE;
  if (p.N_fr > (1 << kSmallLogMax) || p.N_fr > 1024) return JTFS_ERR_SHAPE;
  p.R_out = p.N_fr >> p.lF;
  p.n_frames = static_cast<int>(N >> p.lT);
  p.log_frames = p.logN - p.lT;
  p.n_beta1 = 1 + p.K;
  p.n_beta2 = 1 + 2 * p.K;

  p.k1.resize(p.N1);
  for (int n1 = 0; n1 < p.N1; ++n1) p.k1[n1] = std::min(p.psi1[n1].j, p.lT);
  p.n1max.assign(p.N2, 0);
  for (int n2 = 0; n2 < p.N2; ++n2)
    for (int n1 = 0; n1 < p.N1; ++n1)
      if (p.psi1[n1].j < p.psi2[n2].j) p.n1max[n2]++;
  p.active.clear();
  p.s2.clear();
  for (int n2 = 0; n2 < p.N2; ++n2)
    if (p.n1max[n2] > 0) {
      p.active.push_back(n2);
      p.s2.push_back(p.unpooled_t ? p.psi2[n2].j : std::min(p.psi2[n2].j, p.lT));
    }
  p.n_active = static_cast<int>(p.active.size());
  // Unpooled in time: the rows feeding the second order are read at stride
  // j1; supported where that equals the first order's min(j1, log2 T).
  if (p.unpooled_t)
    for (int n1 = 0; n1 < p.N1; ++n1)
      if (p.psi1[n1].j > p.lT) return JTFS_ERR_SHAPE;
  // Rows with j1 < j2 are a prefix of n1 because j1 is non-decreasing in n1.
  for (int n1 = 1; n1 < p.N1; ++n1)
    if (p.psi1[n1].j < p.psi1[n1 - 1].j) return JTFS_ERR_SHAPE;

  // Frequential filters on the N_fr grid: phi_F, then +xi_n, then -xi_n.
  p.h_beta.clear();
  p.beta_k.clear();
  {
    // Frequential strides capped at floor(log2 F), or 2^j when unpooled along n1.
    const int kphi = p.unpooled_f ? p.phiF.j : std::min(p.phiF.j, p.lF);
    if (kphi > p.logNfr - 1) return JTFS_ERR_SHAPE;  // at least two rows per path
    p.h_beta.push_back(make_filt(0.0, p.phiF.sigma, p.N_fr, kphi, p.phiF.j, true));
    for (int s = 0; s < 2; ++s)
      for (auto& f : p.psifr) {
        const int k = p.unpooled_f ? f.j : std::min(f.j, p.lF);
        if (k > p.logNfr - 1) return JTFS_ERR_SHAPE;
        p.h_beta.push_back(make_filt(s == 0 ? f.xi : -f.xi, f.sigma, p.N_fr, k, f.j, false));
      }
    for (auto& f : p.h_beta) p.beta_k.push_back(f.k);
  }
  p.row_off.assign(p.n_beta2 + 1, 0);
  for (int b = 0; b < p.n_beta2; ++b)
    p.row_off[b + 1] = p.row_off[b] + (p.unpooled_f ? (p.N_fr >> p.beta_k[b]) : p.R_out);
  p.rows1 = p.row_off[p.n_beta1];
  p.rows2 = p.row_off[p.n_beta2];
  p.h_psi1.clear();
  for (int n1 = 0; n1 < p.N1; ++n1)
    p.h_psi1.push_back(make_filt(p.psi1[n1].xi, p.psi1[n1].sigma, int(N), p.k1[n1], p.psi1[n1].j, false));
  // Band gains of the coloured initialisation: mean over the N bins of
  // psi_hat^6, summed where it exceeds exp(-108) of its peak (6 sigma around
  // xi, and around 0 where the kappa term is not negligible).
  p.h_cinit.resize(p.N1);
  for (int n1 = 0; n1 < p.N1; ++n1) {
    const double xi = p.psi1[n1].xi, sg = p.psi1[n1].sigma;
    const double kappa = std::exp(-xi * xi / (2.0 * sg * sg));
    const int64_t half = N / 2;
    auto bin = [&](double w) { return std::max<int64_t>(-half, std::min<int64_t>(half - 1, int64_t(std::floor(w * N)))); };
    int64_t lo = bin(xi - 6.0 * sg), hi = bin(xi + 6.0 * sg) + 1;
    if (kappa > 1e-8) lo = std::min(lo, bin(-6.0 * sg));
    double s6 = 0.0;
    for (int64_t m = lo; m <= hi && m < half; ++m) {
      const double w = double(m) / double(N);
      const double v = std::exp(-(w - xi) * (w - xi) / (2.0 * sg * sg)) - kappa * std::exp(-w * w / (2.0 * sg * sg));
      const double v2 = v * v;
      s6 += v2 * v2 * v2;
    }
    p.h_cinit[n1] = static_cast<float>(std::ldexp(1.0, p.lT + 1) / std::sqrt(s6 / double(N)));
  }
  p.h_psi2.clear();
  for (int n2 = 0; n2 < p.N2; ++n2)
    p.h_psi2.push_back(make_filt(p.psi2[n2].xi, p.psi2[n2].sigma, int(N),
                                 std::min(p.psi2[n2].j, p.lT), p.psi2[n2].j, false));
  p.h_phiT = make_filt(0.0, p.phiT.sigma, int(N), p.lT, p.phiT.j, true);
  p.h_phiF = make_filt(0.0, p.phiF.sigma, p.N_fr, p.lF, p.phiF.j, true);

  // Per-clip layouts.
  p.u1_off.resize(p.N1);
  p.u1_tot = 0;
  for (int n1 = 0; n1 < p.N1; ++n1) {
    p.u1_off[n1] = p.u1_tot;
    p.u1_tot += N >> p.k1[n1];
  }
  p.y2_off.resize(p.n_active);
  p.v2_off.resize(p.n_active);
  p.phi2_off.resize(p.n_active);
  p.y2_tot = 0;
  p.v2_tot = 0;
  p.phi1_off = p.unpooled_t ? N : p.n_frames;
  p.phi2_base = p.phi1_off + int64_t(p.rows1) * p.n_frames;
  for (int a = 0; a < p.n_active; ++a) {
    const int64_t L2 = N >> p.s2[a];
    p.y2_off[a] = p.y2_tot;
    p.y2_tot += int64_t(p.n1max[p.active[a]]) * L2;
    p.v2_off[a] = p.v2_tot;
    p.v2_tot += int64_t(p.rows2) * L2;
    // Unpooled in time, the second-order blocks are V2 itself.
    p.phi2_off[a] = p.phi2_base + (p.unpooled_t ? p.v2_off[a] : int64_t(a) * p.rows2 * p.n_frames);
  }
  p.phi_size = p.phi2_base + (p.unpooled_t ? p.v2_tot : int64_t(p.n_active) * p.rows2 * p.n_frames);

  // Time-pooling taps g_s[t] = 2^s phi_T[2^s t] for every level s <= log2 T,
  // where phi_T[tau] = (1/N) sum_m phi_hat_T(m/N) e^{2 pi i m tau / N}
  // = sigma sqrt(2 pi) sum_p exp(-2 pi^2 sigma^2 (tau - p N)^2) (Poisson
  // summation; phi_hat_T(1/2) <= exp(-12.5 T^2) is negligible for T >= 2).
  p.tap_off.resize(p.lT + 1);
  p.tap_tot = 0;
  for (int s = 0; s <= p.lT; ++s) {
    p.tap_off[s] = p.tap_tot;
    p.tap_tot += N >> s;
  }
  p.h_taps.assign(p.tap_tot, 0.f);
  {
    const double sg = p.phiT.sigma;
    const double c = 2.0 * M_PI * M_PI * sg * sg;
    const double amp = sg * std::sqrt(2.0 * M_PI);
    const int P = static_cast<int>(std::ceil(std::sqrt(60.0 / c) / double(N))) + 1;
    // phi_T is even, so g_s[t] = g_s[L - t]: computed for t <= L / 2 and mirrored, which makes the table
    // exactly symmetric (the pooling kernels read g_s[(t - f D) mod L] for g_s[(f D - t) mod L]).
    for (int s = 0; s <= p.lT; ++s) {
      const int64_t L = N >> s;
      for (int64_t t = 0; t <= L / 2; ++t) {
        const int64_t tau = t << s;
        double acc = 0.0;
        for (int q = -P; q <= P; ++q) {
          const double d = double(tau) - double(q) * double(N);
          acc += std::exp(-c * d * d);
        }
        const float v = static_cast<float>(double(int64_t(1) << s) * amp * acc);
        p.h_taps[p.tap_off[s] + t] = v;
        p.h_taps[p.tap_off[s] + ((L - t) & (L - 1))] = v;
      }
    }
  }

  // Launch descriptions.
  p.jobs.clear();
  auto add = [&](std::vector<FftLaunch>& L, int logn, const std::vector<Job>& js) {
    if (js.empty()) return;
    L.push_back({logn, static_cast<int>(js.size()), static_cast<int>(p.jobs.size()), 0, 0});
    p.jobs.insert(p.jobs.end(), js.begin(), js.end());
  };
  const int B = batch;
  p.L_x.clear(); p.L_u1.clear(); p.L_s0.clear(); p.L_s1.clear(); p.L_y2.clear();
  p.L_u1inplace.clear(); p.L_y2inplace.clear(); p.L_ds1.clear(); p.L_ds0.clear();
  {
    std::vector<Job> js;
    for (int b = 0; b < B; ++b) js.push_back({int64_t(b) * N, int64_t(b) * N, -1, p.logN, b, 0});
    add(p.L_x, p.logN, js);
  }
  // Rows of U1 per level: all band jobs, then all row jobs, so that the row jobs of every level
  // are consecutive (the adjoint's k_dU1 covers them in one launch).
  for (int pass = 0; pass < 2; ++pass)
    for (int lev = 0; lev <= p.lT; ++lev) {
      std::vector<Job> js;
      for (int b = 0; b < B; ++b)
        for (int n1 = 0; n1 < p.N1; ++n1)
          if (p.k1[n1] == lev) {
            const int64_t o = int64_t(b) * p.u1_tot + p.u1_off[n1];
            if (pass == 0) js.push_back({int64_t(b) * N, o, n1, p.logN, b, 0});
            else js.push_back({o, o, n1, p.logN - lev, b, 0});
          }
      add(pass == 0 ? p.L_u1 : p.L_u1inplace, p.logN - lev, js);
    }
  {
    std::vector<Job> s0, ds0, s1, ds1;
    for (int b = 0; b < B; ++b) {
      s0.push_back({int64_t(b) * N, int64_t(b) * p.phi_size, -1, p.logN, b, 0});
      ds0.push_back({int64_t(b) * p.phi_size, int64_t(b) * p.n_frames, -1, p.log_frames, b, 0});
      for (int n1 = 0; n1 < p.N1; ++n1) {
        const int64_t row = (int64_t(b) * p.N1 + n1) * p.n_frames;
        s1.push_back({int64_t(b) * p.u1_tot + p.u1_off[n1], row, n1, p.logN - p.k1[n1], b, 0});
        ds1.push_back({row, row, n1, p.log_frames, b, 0});
      }
    }
    add(p.L_s0, p.log_frames, s0);
    add(p.L_ds0, p.log_frames, ds0);
    add(p.L_s1, p.log_frames, s1);
    add(p.L_ds1, p.log_frames, ds1);
  }
  int max_s2 = p.lT;
  for (int a = 0; a < p.n_active; ++a) max_s2 = std::max(max_s2, p.s2[a]);
  for (int lev = 0; lev <= max_s2; ++lev) {
    std::vector<Job> band, rows;
    for (int b = 0; b < B; ++b)
      for (int a = 0; a < p.n_active; ++a) {
        if (p.s2[a] != lev) continue;
        const int n2 = p.active[a];
        const int64_t L2 = N >> lev;
        for (int n1 = 0; n1 < p.n1max[n2]; ++n1) {
          const int64_t o = int64_t(b) * p.y2_tot + p.y2_off[a] + int64_t(n1) * L2;
          band.push_back({int64_t(b) * p.u1_tot + p.u1_off[n1], o, n2, p.logN - p.k1[n1], b, 0});
          rows.push_back({o, o, n2, p.logN - lev, b, 0});
        }
      }
    add(p.L_y2, p.logN - lev, band);
    add(p.L_y2inplace, p.logN - lev, rows);
  }

  // Items of the time-axis FFT engine's merged launches: for every stage, its launches of up to
  // 2^13 points get consecutive items (as many jobs per CTA as 2^13 points and 256 jobs allow), so
  // one launch over the stage's item range runs all of them.
  p.tf_items.clear();
  for (auto* L : {&p.L_x, &p.L_u1, &p.L_u1inplace, &p.L_s0, &p.L_s1, &p.L_y2, &p.L_y2inplace, &p.L_ds1,
                  &p.L_ds0})
    for (FftLaunch& l : *L) {
      l.item0 = static_cast<int>(p.tf_items.size());
      l.n_items = 0;
      if (l.logn > 13) continue;
      const int per = std::min(256, 1 << (13 - l.logn));
      for (int j = 0; j < l.njobs; j += per)
        p.tf_items.push_back(make_int4(l.job0 + j, std::min(per, l.njobs - j), l.logn, 0));
      l.n_items = static_cast<int>(p.tf_items.size()) - l.item0;
    }
  // Blocks of the U1-row gradient gather (k_dU1): (job relative to the first U1 job, block in the row)
  // for every row, so one launch covers every level without blocks past a row's end.
  p.du1_blocks.clear();
  for (const FftLaunch& l : p.L_u1inplace)
    for (int j = 0; j < l.njobs; ++j)
      for (int bx = 0; bx < std::max(1, (1 << l.logn) / kDU1Block); ++bx)
        p.du1_blocks.push_back(make_int2(l.job0 + j - p.L_u1inplace.front().job0, bx));

  // Frequential tiles.
  p.freq_cols = std::max(2, std::min(kFreqCols, 2048 / p.N_fr));  // >= 2: kernels pair columns
  p.tiles1.clear();
  p.tiles2.clear();
  for (int b = 0; b < B; ++b)
    for (int t0 = 0; t0 < p.n_frames; t0 += p.freq_cols)
      p.tiles1.push_back({b, -1, t0, std::min(p.freq_cols, p.n_frames - t0)});
  p.freq_cols_wide = std::min(kFreqCols, 2 * p.freq_cols);
  p.tiles2w.clear();
  for (int b = 0; b < B; ++b)
    for (int a = 0; a < p.n_active; ++a) {
      const int L2 = static_cast<int>(N >> p.s2[a]);
      for (int t0 = 0; t0 < L2; t0 += p.freq_cols)
        p.tiles2.push_back({b, a, t0, std::min(p.freq_cols, L2 - t0)});
      for (int t0 = 0; t0 < L2; t0 += p.freq_cols_wide)
        p.tiles2w.push_back({b, a, t0, std::min(p.freq_cols_wide, L2 - t0)});
    }

  // Frequential tables (double precision on the host, stored as float).
  {
    const int n = p.N_fr;
    p.n_ftab = p.n_beta2 + 1 + (p.lF + 1);
    p.h_ftab.assign(size_t(p.n_ftab) * n, 0.f);
    auto omega = [n](int m) { return double(m < n / 2 ? m : m - n) / double(n); };
    auto gauss = [](double w, double c, double sg) { return std::exp(-(w - c) * (w - c) / (2.0 * sg * sg)); };
    for (int b = 0; b < p.n_beta2; ++b) {
      const FilterH& f = b == 0 ? p.phiF : p.psifr[(b - 1) % p.K];
      const double xi = b == 0 ? 0.0 : (b <= p.K ? f.xi : -f.xi);
      const double kappa = b == 0 ? 0.0 : std::exp(-f.xi * f.xi / (2.0 * f.sigma * f.sigma));
      for (int m = 0; m < n; ++m)
        p.h_ftab[size_t(b) * n + m] =
            static_cast<float>(gauss(omega(m), xi, f.sigma) - kappa * gauss(omega(m), 0.0, f.sigma));
    }
    for (int m = 0; m < n; ++m)
      p.h_ftab[size_t(p.n_beta2) * n + m] = static_cast<float>(gauss(omega(m), 0.0, p.phiF.sigma));
    for (int k = 0; k <= p.lF; ++k) {
      const int R = n >> k;
      for (int m = 0; m < R; ++m) {
        double acc = 0.0;
        for (int r = 0; r < (1 << k); ++r) acc += gauss(omega(m + r * R), 0.0, p.phiF.sigma);
        p.h_ftab[size_t(p.n_beta2 + 1 + k) * n + m] = static_cast<float>(acc);
      }
    }
    p.h_ftabc.clear();
    p.h_ftabc_off.assign(p.n_beta2, 0);
    for (int b = 0; b < p.n_beta2; ++b) {
      p.h_ftabc_off[b] = static_cast<int>(p.h_ftabc.size());
      for (int sb = p.h_beta[b].lo; sb <= p.h_beta[b].hi; ++sb) p.h_ftabc.push_back(p.h_ftab[size_t(b) * n + (sb & (n - 1))]);
    }
    p.ftabc_phi = static_cast<int>(p.h_ftabc.size());
    for (int sb = p.h_phiF.lo; sb <= p.h_phiF.hi; ++sb)
      p.h_ftabc.push_back(p.h_ftab[size_t(p.n_beta2) * n + (sb & (n - 1))]);
    for (int k = 0; k <= p.lF && k < 16; ++k) {
      p.ftabc_lev[k] = static_cast<int>(p.h_ftabc.size());
      for (int m = 0; m < (n >> k); ++m) p.h_ftabc.push_back(p.h_ftab[size_t(p.n_beta2 + 1 + k) * n + m]);
    }
  }
  // Chunks of frequential filters with equal stride level.
  int kmax = p.lF;
  for (int b = 0; b < p.n_beta2; ++b) kmax = std::max(kmax, p.beta_k[b]);
  auto make_chunks = [&](int nb, std::vector<FreqChunk>& out) {
    out.clear();
    for (int k = 0; k <= kmax; ++k) {
      const int cap = std::min(16, 1 << k);
      FreqChunk c{};
      c.k = k;
      for (int b = 0; b < nb; ++b) {
        if (p.beta_k[b] != k) continue;
        c.beta[c.n++] = b;
        if (c.n == cap) {
          out.push_back(c);
          c.n = 0;
        }
      }
      if (c.n) out.push_back(c);
    }
  };
  make_chunks(p.n_beta1, p.chunks1);
  make_chunks(p.n_beta2, p.chunks2);
  // Tiles of the adjoint time pooling: 64 path-rows x 64 time samples.
  // Banded pooling where the taps' reach is small against the circle: g_s[d] /
  // g_s[0] = exp(-c (2^s d)^2) (c = 2 pi^2 sigma_T^2) is below 2^-40 once
  // 2^s |d| > sqrt(40 ln 2 / c), so a frame only sees W = floor(that / 2^s) + 1
  // level samples on either side.  Chosen when a 32-frame window (forward) and
  // the frames of a 64-sample tile (adjoint) stay within the circle.
  p.pool_w.assign(p.n_active, 0);
  if (!p.unpooled_t) {
    const double c = 2.0 * M_PI * M_PI * p.phiT.sigma * p.phiT.sigma;
    const double reach = std::sqrt(40.0 * std::log(2.0) / c);
    for (int a = 0; a < p.n_active; ++a) {
      const int s = p.s2[a];
      const int64_t L = N >> s, D = int64_t(1) << (p.lT - s);
      const int64_t W = static_cast<int64_t>(std::floor(reach / double(int64_t(1) << s))) + 1;
      if (2 * W + 32 * D <= L / 2 && (63 + 2 * W) / D + 2 <= p.n_frames) p.pool_w[a] = static_cast<int>(W);
    }
  }
  // Adjoint tiles: 64 rows x 64 samples for the banded groups, 64 rows x 512
  // samples (four 128-sample sub-tiles) for the dense ones.
  p.pool_tiles.clear();
  p.pool_tiles2.clear();
  if (!p.unpooled_t) {
    const int rows = p.rows2;
    for (int b = 0; b < B; ++b)
      for (int a = 0; a < p.n_active; ++a) {
        const int L = static_cast<int>(N >> p.s2[a]);
        for (int rt = 0; rt < (rows + 63) / 64; ++rt) {
          if (p.pool_w[a])
            for (int tt = 0; tt < (L + 63) / 64; ++tt) p.pool_tiles.push_back(make_int4(b, a, rt, tt));
          else
            for (int tt = 0; tt < (L + 511) / 512; ++tt) p.pool_tiles2.push_back(make_int4(b, a, rt, tt));
        }
      }
  }
  // Banded adjoint on the tensor cores: a CTA of 128 rows takes S samples and the kPoolBandAdjF frames from
  // floor((t0 - W) / D), which hold every frame within reach when floor((S - 1 + 2 W) / D) + 2 <= that
  // count; S is the largest multiple of 128 up to 1024 (and L) that satisfies it.
  p.pool_band_S.assign(p.n_active, 0);
  p.pool_tc_band_adj_tiles.clear();
  p.pool_tiles_rest.clear();
  if (!p.unpooled_t && p.n_frames >= kPoolBandAdjF) {
    for (int a = 0; a < p.n_active; ++a) {
      if (!p.pool_w[a]) continue;
      const int64_t L = N >> p.s2[a], D = int64_t(1) << (p.lT - p.s2[a]), W = p.pool_w[a];
      for (int64_t S = std::min<int64_t>(1024, L) / 128 * 128; S >= 128; S -= 128)
        if ((S - 1 + 2 * W) / D + 2 <= kPoolBandAdjF) {
          p.pool_band_S[a] = static_cast<int>(S);
          break;
        }
    }
  }
  if (!p.unpooled_t) {
    for (int b = 0; b < B; ++b)
      for (int a = 0; a < p.n_active; ++a) {
        if (!p.pool_w[a]) continue;
        const int L = static_cast<int>(N >> p.s2[a]), S = p.pool_band_S[a];
        for (int rt = 0; rt < (p.rows2 + 63) / 64; ++rt) {
          if (S) {
            if ((rt & 1) == 0)
              for (int t0 = 0; t0 < L; t0 += S) p.pool_tc_band_adj_tiles.push_back(make_int4(b, a, rt, t0));
          } else {
            for (int tt = 0; tt < (L + 63) / 64; ++tt) p.pool_tiles_rest.push_back(make_int4(b, a, rt, tt));
          }
        }
      }
  }
  // Tensor-core adjoint pooling of the dense groups: 128 rows x 1024 samples per CTA.
  p.pool_tc_adj_tiles.clear();
  if (!p.unpooled_t) {
    for (int b = 0; b < B; ++b)
      for (int a = 0; a < p.n_active; ++a) {
        if (p.pool_w[a]) continue;
        const int L = static_cast<int>(N >> p.s2[a]);
        for (int rt = 0; rt < (p.rows2 + 63) / 64; rt += 2)
          for (int tb = 0; tb < (L + 1023) / 1024; ++tb) p.pool_tc_adj_tiles.push_back(make_int4(b, a, rt, tb));
      }
  }
  p.pool_band_tiles.clear();
  p.pool_tc_band_tiles.clear();
  p.pool_tc_band_long = false;
  p.pool_band_rest.clear();
  if (!p.unpooled_t) {
    const int rows = p.rows2;
    for (int b = 0; b < B; ++b)
      for (int a = 0; a < p.n_active; ++a) {
        if (!p.pool_w[a]) continue;
        const int64_t L = N >> p.s2[a], D = int64_t(1) << (p.lT - p.s2[a]);
        // The widened range must fit the circle (long windows are summed in sub-windows of 4096 samples
        // inside the kernel, so the FP32 accumulation stays as short as a split of the dense path).
        const int64_t span = 31 * D + 2 * int64_t(p.pool_w[a]) + 128;
        const bool tc = p.n_frames % 32 == 0 && span <= L;
        if (tc && span > 4096 + 128) p.pool_tc_band_long = true;
        for (int rt = 0; rt < (rows + 63) / 64; ++rt)
          for (int fb = 0; fb < (p.n_frames + 31) / 32; ++fb) {
            p.pool_band_tiles.push_back(make_int4(b, a, rt, fb));
            if (!tc) p.pool_band_rest.push_back(make_int4(b, a, rt, fb));
            else if ((rt & 1) == 0) p.pool_tc_band_tiles.push_back(make_int4(b, a, rt, fb));  // rows rt, rt + 1
          }
      }
  }
  for (int si = 0; si < 3; ++si) {
    p.pool_fwd_tiles[si].clear();
    p.pool_tile0[si].clear();
    p.pool_tc_tiles[si].clear();
    if (p.unpooled_t) continue;
    const int rows = p.rows2;
    for (int b = 0; b < B; ++b)
      for (int a = 0; a < p.n_active; ++a) {
        const int L = static_cast<int>(N >> p.s2[a]);
        const int nsplit = (L + kPoolSplits[si] - 1) / kPoolSplits[si];
        p.pool_tile0[si].push_back(static_cast<int>(p.pool_fwd_tiles[si].size()));
        if (p.pool_w[a]) continue;
        for (int rt = 0; rt < (rows + 63) / 64; ++rt)
          for (int sp = 0; sp < nsplit; ++sp) {
            p.pool_fwd_tiles[si].push_back(make_int4(b, a, rt, sp));
            if ((rt & 1) == 0) p.pool_tc_tiles[si].push_back(make_int4(b, a, rt, sp));  // 128 rows: tiles rt, rt + 1
          }
      }
  }

  // Four-step scratch: the largest large-size launch.
  p.scr_elems = 0;
  for (auto* L : {&p.L_x, &p.L_u1, &p.L_u1inplace, &p.L_y2, &p.L_y2inplace})
    for (auto& l : *L)
      if (l.logn > kSmallLogMax) p.scr_elems = std::max(p.scr_elems, int64_t(l.njobs) << l.logn);

  // Workspace layout.
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t r = o; o = align256(o + bytes); return r; };
  const size_t c8 = sizeof(float2), f4 = sizeof(float);
  p.ws_Xh = take(size_t(B) * N * c8);
  p.ws_U1h = take(size_t(B) * p.u1_tot * c8);
  p.ws_Zs = take(size_t(B) * p.u1_tot * c8);
  p.ws_S1 = take(size_t(B) * p.N1 * p.n_frames * f4);
  p.ws_dS1h = take(size_t(B) * p.N1 * p.n_frames * c8);
  p.ws_Y2 = take(size_t(B) * p.y2_tot * c8);
  p.ws_dY2 = take(size_t(B) * p.y2_tot * c8);
  p.ws_V2 = take(size_t(B) * p.v2_tot * f4);
  p.ws_phi = take(size_t(B) * p.phi_size * f4);
  p.ws_dphi = take(size_t(B) * p.phi_size * f4);
  p.ws_dXh = take(size_t(B) * N * c8);
  p.ws_dS0h = take(size_t(B) * p.n_frames * c8);
  p.ws_dy = take(size_t(B) * N * f4);
  p.ws_scr = take(size_t(std::max<int64_t>(p.scr_elems, 1)) * c8);
  p.ws_part = take(std::max<size_t>(p.pool_fwd_tiles[0].size(), 1) * 64 * p.n_frames * f4);
  // Loss reduction: one CTA per clip up to 2^15 Phi entries, else one per 2^13 (at most 1024).
  p.loss_parts = p.phi_size <= (int64_t(1) << 15)
                     ? 1 : static_cast<int>(std::min<int64_t>(1024, (p.phi_size + (1 << 13) - 1) >> 13));
  p.ws_lossp = take(size_t(B) * p.loss_parts * sizeof(double));
  p.ws_bytes = o;
  tc_build(p);
  return JTFS_OK;
}

void release_streams(Plan& p) {
  for (int k = 0; k < 3; ++k) {
    if (p.aux[k]) cudaStreamDestroy(p.aux[k]);
    if (p.ev_join[k]) cudaEventDestroy(p.ev_join[k]);
    p.aux[k] = nullptr;
    p.ev_join[k] = nullptr;
  }
  if (p.ev_fork) cudaEventDestroy(p.ev_fork);
  p.ev_fork = nullptr;
  p.aux_mu.reset();
}

int upload_plan(Plan& p) {
  // Twiddles W^k = exp(-2 pi i k / TW) for the largest transform, in double.
  int64_t TW = std::max<int64_t>(p.N, p.N_fr);
  p.twlog = ilog2(TW);
  std::vector<float2> tw(TW);
  for (int64_t k = 0; k < TW; ++k) {
    const double ang = -2.0 * M_PI * double(k) / double(TW);
    tw[k] = make_float2(static_cast<float>(std::cos(ang)), static_cast<float>(std::sin(ang)));
  }
  std::vector<int> act_n2(p.active), n1max_act(p.n_active);
  for (int a = 0; a < p.n_active; ++a) n1max_act[a] = p.n1max[p.active[a]];

  struct Part { const void* src; size_t bytes; size_t off; };
  std::vector<Part> parts;
  size_t total = 0;
  auto put = [&](const void* src, size_t bytes) {
    const size_t off = total;
    parts.push_back({src, bytes, off});
    total = align256(total + std::max<size_t>(bytes, 1));
    return off;
  };
  const size_t o_tw = put(tw.data(), tw.size() * sizeof(float2));
  const size_t o_psi1 = put(p.h_psi1.data(), p.h_psi1.size() * sizeof(FiltD));
  const size_t o_psi2 = put(p.h_psi2.data(), p.h_psi2.size() * sizeof(FiltD));
  const size_t o_beta = put(p.h_beta.data(), p.h_beta.size() * sizeof(FiltD));
  const size_t o_taps = put(p.h_taps.data(), p.h_taps.size() * sizeof(float));
  const size_t o_jobs = put(p.jobs.data(), p.jobs.size() * sizeof(Job));
  const size_t o_tfi = put(p.tf_items.data(), p.tf_items.size() * sizeof(int4));
  const size_t o_du1 = put(p.du1_blocks.data(), p.du1_blocks.size() * sizeof(int2));
  const size_t o_t1 = put(p.tiles1.data(), p.tiles1.size() * sizeof(Tile));
  const size_t o_t2 = put(p.tiles2.data(), p.tiles2.size() * sizeof(Tile));
  const size_t o_t2w = put(p.tiles2w.data(), p.tiles2w.size() * sizeof(Tile));
  const size_t o_c1 = put(p.chunks1.data(), p.chunks1.size() * sizeof(FreqChunk));
  const size_t o_c2 = put(p.chunks2.data(), p.chunks2.size() * sizeof(FreqChunk));
  const size_t o_ftab = put(p.h_ftab.data(), p.h_ftab.size() * sizeof(float));
  const size_t o_ftabc = put(p.h_ftabc.data(), p.h_ftabc.size() * sizeof(float));
  const size_t o_ftabc_off = put(p.h_ftabc_off.data(), p.h_ftabc_off.size() * sizeof(int));
  const size_t o_pt = put(p.pool_tiles.data(), p.pool_tiles.size() * sizeof(int4));
  const size_t o_pt2 = put(p.pool_tiles2.data(), p.pool_tiles2.size() * sizeof(int4));
  size_t o_pft[3], o_pt0[3], o_ptc[3];
  for (int si = 0; si < 3; ++si) {
    o_pft[si] = put(p.pool_fwd_tiles[si].data(), p.pool_fwd_tiles[si].size() * sizeof(int4));
    o_pt0[si] = put(p.pool_tile0[si].data(), p.pool_tile0[si].size() * sizeof(int));
    o_ptc[si] = put(p.pool_tc_tiles[si].data(), p.pool_tc_tiles[si].size() * sizeof(int4));
  }
  const size_t o_pta = put(p.pool_tc_adj_tiles.data(), p.pool_tc_adj_tiles.size() * sizeof(int4));
  const size_t o_s2 = put(p.s2.data(), p.s2.size() * sizeof(int));
  const size_t o_pw = put(p.pool_w.data(), p.pool_w.size() * sizeof(int));
  const size_t o_pbt = put(p.pool_band_tiles.data(), p.pool_band_tiles.size() * sizeof(int4));
  const size_t o_ptcb = put(p.pool_tc_band_tiles.data(), p.pool_tc_band_tiles.size() * sizeof(int4));
  const size_t o_pbS = put(p.pool_band_S.data(), p.pool_band_S.size() * sizeof(int));
  const size_t o_pbat = put(p.pool_tc_band_adj_tiles.data(), p.pool_tc_band_adj_tiles.size() * sizeof(int4));
  const size_t o_ptr = put(p.pool_tiles_rest.data(), p.pool_tiles_rest.size() * sizeof(int4));
  const size_t o_pbr = put(p.pool_band_rest.data(), p.pool_band_rest.size() * sizeof(int4));
  const size_t o_n1m = put(n1max_act.data(), n1max_act.size() * sizeof(int));
  const size_t o_y2o = put(p.y2_off.data(), p.y2_off.size() * sizeof(int64_t));
  const size_t o_v2o = put(p.v2_off.data(), p.v2_off.size() * sizeof(int64_t));
  const size_t o_p2o = put(p.phi2_off.data(), p.phi2_off.size() * sizeof(int64_t));
  const size_t o_u1o = put(p.u1_off.data(), p.u1_off.size() * sizeof(int64_t));
  const size_t o_k1 = put(p.k1.data(), p.k1.size() * sizeof(int));
  const size_t o_act = put(act_n2.data(), act_n2.size() * sizeof(int));
  const size_t o_tapo = put(p.tap_off.data(), p.tap_off.size() * sizeof(int64_t));
  const size_t o_cin = put(p.h_cinit.data(), p.h_cinit.size() * sizeof(float));
  const size_t o_roff = put(p.row_off.data(), p.row_off.size() * sizeof(int));

  if (cudaGetDevice(&p.device) != cudaSuccess) return JTFS_ERR_CUDA;
  void* blob = nullptr;
  if (cudaMalloc(&blob, total) != cudaSuccess) return JTFS_ERR_NOMEM;
  std::vector<unsigned char> host(total, 0);
  for (auto& pt : parts)
    if (pt.bytes) std::memcpy(host.data() + pt.off, pt.src, pt.bytes);
  if (cudaMemcpy(blob, host.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(blob);
    return JTFS_ERR_CUDA;
  }
  auto at = [&](size_t off) { return static_cast<unsigned char*>(blob) + off; };
  p.d_blob = blob;
  p.d_tw = reinterpret_cast<const float2*>(at(o_tw));
  p.d_psi1 = reinterpret_cast<const FiltD*>(at(o_psi1));
  p.d_psi2 = reinterpret_cast<const FiltD*>(at(o_psi2));
  p.d_beta = reinterpret_cast<const FiltD*>(at(o_beta));
  p.d_taps = reinterpret_cast<const float*>(at(o_taps));
  p.d_jobs = reinterpret_cast<const Job*>(at(o_jobs));
  p.d_tf_items = reinterpret_cast<const int4*>(at(o_tfi));
  p.d_du1_blocks = reinterpret_cast<const int2*>(at(o_du1));
  p.d_tiles1 = reinterpret_cast<const Tile*>(at(o_t1));
  p.d_tiles2 = reinterpret_cast<const Tile*>(at(o_t2));
  p.d_tiles2w = reinterpret_cast<const Tile*>(at(o_t2w));
  p.d_chunks1 = reinterpret_cast<const FreqChunk*>(at(o_c1));
  p.d_chunks2 = reinterpret_cast<const FreqChunk*>(at(o_c2));
  p.d_ftab = reinterpret_cast<const float*>(at(o_ftab));
  p.d_ftabc = reinterpret_cast<const float*>(at(o_ftabc));
  p.d_ftabc_off = reinterpret_cast<const int*>(at(o_ftabc_off));
  p.d_pool_tiles = reinterpret_cast<const int4*>(at(o_pt));
  p.d_pool_tiles2 = reinterpret_cast<const int4*>(at(o_pt2));
  for (int si = 0; si < 3; ++si) {
    p.d_pool_fwd_tiles[si] = reinterpret_cast<const int4*>(at(o_pft[si]));
    p.d_pool_tile0[si] = reinterpret_cast<const int*>(at(o_pt0[si]));
    p.d_pool_tc_tiles[si] = reinterpret_cast<const int4*>(at(o_ptc[si]));
    if (si == 2) p.d_pool_tc_adj_tiles = reinterpret_cast<const int4*>(at(o_pta));
  }
  p.d_s2 = reinterpret_cast<const int*>(at(o_s2));
  p.d_pool_w = reinterpret_cast<const int*>(at(o_pw));
  p.d_pool_band_tiles = reinterpret_cast<const int4*>(at(o_pbt));
  p.d_pool_tc_band_tiles = reinterpret_cast<const int4*>(at(o_ptcb));
  p.d_pool_band_S = reinterpret_cast<const int*>(at(o_pbS));
  p.d_pool_tc_band_adj_tiles = reinterpret_cast<const int4*>(at(o_pbat));
  p.d_pool_tiles_rest = reinterpret_cast<const int4*>(at(o_ptr));
  p.d_pool_band_rest = reinterpret_cast<const int4*>(at(o_pbr));
  p.d_n1max_act = reinterpret_cast<const int*>(at(o_n1m));
  p.d_y2_off = reinterpret_cast<const int64_t*>(at(o_y2o));
  p.d_v2_off = reinterpret_cast<const int64_t*>(at(o_v2o));
  p.d_phi2_off = reinterpret_cast<const int64_t*>(at(o_p2o));
  p.d_u1_off = reinterpret_cast<const int64_t*>(at(o_u1o));
  p.d_k1 = reinterpret_cast<const int*>(at(o_k1));
  p.d_act_n2 = reinterpret_cast<const int*>(at(o_act));
  p.d_tap_off = reinterpret_cast<const int64_t*>(at(o_tapo));
  p.d_cinit = reinterpret_cast<const float*>(at(o_cin));
  p.d_row_off = reinterpret_cast<const int*>(at(o_roff));
  p.on_device = true;
  // Streams and events of the frequential stage's concurrent launches; without them the launches run
  // in order on the caller's stream.
  bool conc = true;
  for (int k = 0; k < 3; ++k) {
    conc = conc && cudaStreamCreateWithFlags(&p.aux[k], cudaStreamNonBlocking) == cudaSuccess;
    conc = conc && cudaEventCreateWithFlags(&p.ev_join[k], cudaEventDisableTiming) == cudaSuccess;
  }
  conc = conc && cudaEventCreateWithFlags(&p.ev_fork, cudaEventDisableTiming) == cudaSuccess;
  if (conc) {
    p.aux_mu = std::make_shared<std::mutex>();
  } else {
    release_streams(p);
    cudaGetLastError();
  }
  return tc_upload(p);
}

void release_plan(Plan& p) {
  if (p.d_blob) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (p.device >= 0 && cur != p.device) cudaSetDevice(p.device);
    cudaFree(p.d_blob);
    tc_release(p);
    release_streams(p);
    if (cur >= 0 && cur != p.device) cudaSetDevice(cur);
  }
  p.d_blob = nullptr;
  p.on_device = false;
}

}  // namespace jtfs

// ---------------------------------------------------------------------------
// C ABI: plan management and inspection.
// ---------------------------------------------------------------------------

extern "C" int jtfs_plan(jtfs_plan_t* out, int64_t N, int J, int Q, int Q2, int J_fr,
                         int Q_fr, int64_t T, int F, int batch, uint32_t flags) {
  if (!out) return JTFS_ERR_ARG;
  *out = nullptr;
  jtfs_plan_s* h = new (std::nothrow) jtfs_plan_s();
  if (!h) return JTFS_ERR_NOMEM;
  int rc;
  try {
    rc = jtfs::build_plan(h->p, N, J, Q, Q2, J_fr, Q_fr, T, F, batch, flags);
    if (rc == JTFS_OK && !(flags & JTFS_PLAN_HOST_ONLY)) rc = jtfs::upload_plan(h->p);
  } catch (...) {
    rc = JTFS_ERR_NOMEM;
  }
  if (rc != JTFS_OK) {
    jtfs::release_plan(h->p);
    delete h;
    return rc;
  }
  *out = h;
  return JTFS_OK;
}

extern "C" int jtfs_plan_destroy(jtfs_plan_t plan) {
  if (!plan) return JTFS_OK;
  jtfs::release_plan(plan->p);
  delete plan;
  return JTFS_OK;
}

extern "C" int64_t jtfs_phi_size(jtfs_plan_t plan) {
  return plan ? plan->p.phi_size : JTFS_ERR_ARG;
}

extern "C" size_t jtfs_workspace_bytes(jtfs_plan_t plan) {
  return plan ? plan->p.ws_bytes : 0;
}

extern "C" int jtfs_path_meta(jtfs_plan_t plan, int32_t* order, int32_t* n2, int32_t* beta_idx, int32_t* spin,
                              int64_t* offset) {
  if (!plan) return JTFS_ERR_ARG;
  const jtfs::Plan& p = plan->p;
  int k = 0;
  auto put = [&](int o, int nn, int bi, int sp, int64_t off) {
    if (order) order[k] = o;
    if (n2) n2[k] = nn;
    if (beta_idx) beta_idx[k] = bi;
    if (spin) spin[k] = sp;
    if (offset) offset[k] = off;
    ++k;
  };
  auto spin_of = [&](int b) { return b == 0 ? 0 : (b <= p.K ? 1 : -1); };
  put(0, -1, -1, 0, 0);  // zeroth order
  for (int b = 0; b < p.n_beta1; ++b) put(1, -1, b, spin_of(b), p.phi1_off + int64_t(p.row_off[b]) * p.n_frames);
  for (int a = 0; a < p.n_active; ++a) {
    const int64_t frames = p.unpooled_t ? (int64_t(p.N) >> p.s2[a]) : p.n_frames;
    for (int b = 0; b < p.n_beta2; ++b) put(2, p.active[a], b, spin_of(b), p.phi2_off[a] + p.row_off[b] * frames);
  }
  return k;
}

extern "C" int jtfs_plan_info(jtfs_plan_t plan, int64_t* info, int count) {
  if (!plan || (count > 0 && !info)) return JTFS_ERR_ARG;
  const jtfs::Plan& p = plan->p;
  const int64_t v[19] = {p.N, p.J, p.Q, p.Q2, p.J_fr, p.Q_fr, p.T, p.F, p.batch, p.N1,
                         p.N2, p.K, p.N_fr, p.lT, p.lF, p.R_out, p.n_frames, p.n_active,
                         p.phi_size};
  for (int i = 0; i < count && i < 19; ++i) info[i] = v[i];
  return 19;
}

extern "C" int64_t jtfs_plan_schedule(jtfs_plan_t plan, int which, int64_t* out, int64_t n) {
  if (!plan || n < 0 || (n > 0 && !out)) return JTFS_ERR_ARG;
  const jtfs::Plan& p = plan->p;
  std::vector<int64_t> v;
  switch (which) {
    case 0:  // U1-row gradient gather: (row, block, log2 row length) per block
      for (const int2& e : p.du1_blocks)
        v.insert(v.end(), {e.x, e.y, p.jobs[size_t(p.L_u1inplace.front().job0 + e.x)].lslog});
      break;
    case 1:  // banded phi_T adjoint on the tensor cores: (clip, group, first row, first sample) per CTA
      for (const int4& t : p.pool_tc_band_adj_tiles) v.insert(v.end(), {t.x, t.y, int64_t(t.z) * 64, t.w});
      break;
    case 2:  // per active group: s2, rows, n1max, reach W (0: dense pooling), band samples per CTA (0: FMA),
             // forward tensor-core K atoms (0: FFT kernels), adjoint tensor-core K atoms (0: FFT kernels)
      for (int a = 0; a < p.n_active; ++a) {
        int kf = 0, kb = 0;
        for (int k = 0; k < 5; ++k)
          for (const jtfs::Tile& t : p.tc_tiles[k])
            if (t.a == a) kf = k + 1;
        for (int k = 0; k < 2; ++k)
          for (const jtfs::Tile& t : p.tc_tiles[k])
            if (t.a == a) kb = k + 1;
        v.insert(v.end(), {p.s2[a], p.rows2, p.n1max[p.active[a]], p.pool_w[a], p.pool_band_S[a], kf, kb});
      }
      break;
    default:
      return JTFS_ERR_ARG;
  }
  for (int64_t i = 0; i < n && i < int64_t(v.size()); ++i) out[i] = v[size_t(i)];
  return static_cast<int64_t>(v.size());
}

extern "C" int jtfs_plan_filters(jtfs_plan_t plan, int which, double* xi, double* sigma,
                                 int32_t* j, int count) {
  if (!plan) return JTFS_ERR_ARG;
  const jtfs::Plan& p = plan->p;
  std::vector<jtfs::FilterH> fb;
  switch (which) {
    case 0: fb = p.psi1; break;
    case 1: fb = p.psi2; break;
    case 2: fb = p.psifr; break;
    case 3: fb = {p.phiT, p.phiF}; break;
    default: return JTFS_ERR_ARG;
  }
  const int n = static_cast<int>(fb.size());
  for (int i = 0; i < count && i < n; ++i) {
    if (xi) xi[i] = fb[i].xi;
    if (sigma) sigma[i] = fb[i].sigma;
    if (j) j[i] = fb[i].j;
  }
  return n;
}

extern "C" const char* jtfs_error_string(int code) {
  switch (code) {
    case JTFS_OK: return "success";
    case JTFS_ERR_ARG: return "invalid argument";
    case JTFS_ERR_SHAPE: return "unsupported sizes";
    case JTFS_ERR_WORKSPACE: return "workspace missing or misaligned";
    case JTFS_ERR_CUDA: return "CUDA runtime error";
    case JTFS_ERR_NOMEM: return "allocation failed";
    case JTFS_ERR_NODEVICE: return "plan has no device tables (host-only)";
    case JTFS_ERR_TOOBIG: return "plan needs more scratch than the fixed 32 MiB array of jtfs_forward_noalloc";
    case JTFS_ERR_NONFINITE: return "a loss was NaN or infinite (non-finite input or target)";
    case JTFS_ERR_TIMEOUT: return "a tensor-core kernel gave up waiting on a barrier; its outputs are invalid";
    default: return "unknown error";
  }
}
