// C ABI of libpspec: plan, workspace layout, argument validation and the launch sequence
// of the SH-FFT multipole estimator (declarations and conventions in include/pspec.h).
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>
#include "pspec.h"
#include "launch.h"

using namespace pspec;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kSmemBudget = 200 * 1024;   // one block
constexpr size_t kSmemMaxBlock = 227 * 1024; // per-block limit of the device
constexpr int kMaxElls = PSPEC_MAX_ELL / 2 + 1;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// N even, 2^a (N >= 16) or 3*2^a (N >= 48), N <= 1024: the register FFT holds 8 (24)
// elements per thread and needs N/2 >= 8 (24).
bool good_nmesh(int n) {
  if (n < 16 || n > 1024 || (n & 1)) return false;
  int x = n;
  while ((x & 1) == 0) x >>= 1;
  if (x == 1) return true;
  return x == 3 && n >= 48;
}

int pow2_floor(int v) {
  int p = 1;
  while (p * 2 <= v) p *= 2;
  return p;
}

struct Plan {
  Geo g;
  int E;
  int esz;  // sizeof(T)
  size_t csz;
  const PassTable<float>* tf;
  const PassTable<double>* td;
  int tw_y, tw_comb, tw_bin, rows_z;
  int group_max, ylm_rows_max;
  int ctas_comb, ctas_bin, ctas_bin_plain;  // plain: the binning kernel without the Y table
  int nblk_sum;
  bool roundtrip;
  int xp;  // FP32 harmonic and inverse transforms in exact-add stages
  size_t Sr, Sc;
  int n2max;
  // workspace offsets
  bool has_ytab = false, has_ctab = false, has_rtab = false;
  size_t ytab_bytes = 0, o_ytab = 0, ctab_bytes = 0, o_ctab = 0, rtab_bytes = 0, o_rtab = 0;
  size_t o_xtiles;  // x-pass tiles (j, kz-tile) of the binning pass that hold a binned mode, in order
  size_t o_twh12 = 0, o_twf12 = 0, o_twr12 = 0;  // twiddles of the exact-add stages (FP32)
  size_t o_mesh1, o_mesh2, o_f0, o_w, o_f, o_g, o_twh, o_twf, o_twr, o_axis, o_phase, o_invw, o_bin, o_kmag, o_cnt,
      o_lo, o_hi, o_nmodes, o_ksum, o_sums, o_derived, o_bins, o_out, o_tcnt, o_toff, o_tcur, o_prec, o_ptile,
      o_psort, total;
  int64_t max_particles;  // capacity of the tile-binned paint (0: direct painting only)
  int ntiles;
  bool cache_randoms;
  size_t o_rmesh1, o_rmesh2, o_rsums, o_desc, o_cur, o_bout;
};

pspec_status build_plan(const pspec_params* p, int max_kbins, int nsm, Plan* pl, std::string* why) {
  if (!p) { *why = "params is NULL"; return PSPEC_EINVAL; }
  if (!good_nmesh(p->nmesh)) { *why = "nmesh must be even, 16..1024 and 2^a, or 48..768 and 3*2^a"; return PSPEC_EUNSUPPORTED; }
  if (p->window != PSPEC_WINDOW_CIC && p->window != PSPEC_WINDOW_TSC) { *why = "window must be CIC or TSC"; return PSPEC_EINVAL; }
  if (p->compensate < 0 || p->compensate > 3) { *why = "compensate must be 0..3"; return PSPEC_EINVAL; }
  if (p->precision != PSPEC_FP32 && p->precision != PSPEC_FP64 && p->precision != PSPEC_FP32_PLAIN) { *why = "precision must be FP32, FP32_PLAIN or FP64"; return PSPEC_EINVAL; }
  if (p->ell_max < 0) { *why = "ell_max must be >= 0"; return PSPEC_EUNSUPPORTED; }
  if (p->ell_max > PSPEC_MAX_ELL) { *why = "ell_max > 16"; return PSPEC_EUNSUPPORTED; }
  if (!(std::isfinite(p->box_size) && p->box_size > 0)) { *why = "box_size must be finite and > 0"; return PSPEC_EINVAL; }
  for (int d = 0; d < 3; d++)
    if (!std::isfinite(p->box_corner[d]) || !std::isfinite(p->observer[d])) { *why = "corner/observer must be finite"; return PSPEC_EINVAL; }
  if (!(std::isfinite(p->P0) && p->P0 >= 0) || !(std::isfinite(p->nbar) && p->nbar >= 0)) { *why = "P0 and nbar must be finite and >= 0"; return PSPEC_EINVAL; }
  if (max_kbins < 1 || max_kbins > PSPEC_MAX_KBINS) { *why = "max_kbins out of range"; return PSPEC_EINVAL; }
  if (p->max_group_bytes < 0) { *why = "max_group_bytes < 0"; return PSPEC_EINVAL; }
  if (p->ylm_table != 0 && p->ylm_table != -1) { *why = "ylm_table must be 0 or -1"; return PSPEC_EINVAL; }
  if (p->cartesian != 0 && p->cartesian != 1) { *why = "cartesian must be 0 or 1"; return PSPEC_EINVAL; }
  if (p->cartesian && p->precision == PSPEC_FP64) { *why = "the Cartesian route is built for FP32 contexts"; return PSPEC_EUNSUPPORTED; }
  if (p->max_particles < 0 || p->max_particles > (int64_t)0xfffffff0) { *why = "max_particles out of range"; return PSPEC_EINVAL; }

  const bool f64 = p->precision == PSPEC_FP64;
  // FP32: the harmonic transforms and the inverse transform of the round trip in exact-add
  // stages (xp_engine.cuh); FP32_PLAIN: every transform a plain FP32 radix tree
  pl->xp = p->precision == PSPEC_FP32 ? 1 : 0;
  const int N = p->nmesh, NH = N / 2;
  pl->g.N = N;
  pl->g.NH = NH;
  pl->E = elems_per_thread(N);
  pl->esz = f64 ? 8 : 4;
  pl->csz = f64 ? 16 : 8;
  const size_t csz = pl->csz;
  pl->tf = pass_table<float>(N);
  pl->td = pass_table<double>(N);
  if (!pl->tf || !pl->td) { *why = "no compiled transform passes for this nmesh"; return PSPEC_EUNSUPPORTED; }
  // the inverse transform is needed for interlacing, and for compensation of the field; with
  // compensation per mode (3) the painted mesh itself is weighted
  pl->roundtrip = p->interlaced || p->compensate == 1 || p->compensate == 2;
  pl->Sr = (size_t)N * N * N * pl->esz;
  pl->Sc = (size_t)N * N * NH * csz;
  pl->n2max = 3 * NH * NH;

  pl->tw_y = pl->tw_comb = pl->tw_bin = pl->tf->tw;
  pl->rows_z = pl->tf->rows_z;

  // harmonics per group (spectra buffered between the z and x passes): bounded by memory
  const int nharm = 2 * p->ell_max + 1;
  int m_mem = p->max_group_bytes > 0 ? (int)(p->max_group_bytes / (int64_t)pl->Sc) : nharm;
  pl->group_max = p->ell_max == 0 ? 0 : std::max(1, std::min(nharm, m_mem));

  // Y_lm(khat) of every stored mode for the FP32 binning pass (even l = 2..l_max; odd l are
  // binned with Y_lm evaluated in the kernel)
  pl->ytab_bytes = (size_t)N * N * NH * sizeof(float) * (size_t)ytab_base((p->ell_max & ~1) + 2);
  pl->has_ytab = !f64 && p->ell_max >= 2 && p->ylm_table == 0 && pl->ytab_bytes <= (size_t)PSPEC_YLM_TABLE_AUTO_MAX;
  // Y_lm(rhat) of every node for the z pass (even l = 2..l_max), twice the k-space table's size
  pl->rtab_bytes = (size_t)N * N * N * sizeof(float) * (size_t)ytab_base((p->ell_max & ~1) + 2);
  pl->has_rtab = !f64 && p->ell_max >= 2 && p->ylm_table == 0 && pl->rtab_bytes <= (size_t)PSPEC_YLM_RTABLE_AUTO_MAX;
  {
    size_t need = f64 ? std::max(pl->td->smem_bin(max_kbins), pl->td->smem_combine(max_kbins))
                      : std::max(pl->tf->smem_bin(max_kbins), pl->tf->smem_combine(max_kbins));
    if (pl->has_ytab) need = std::max(need, pl->tf->smem_bin_pipe(max_kbins));
    if (need > kSmemMaxBlock) { *why = "max_kbins too large for this mesh (shared memory)"; return PSPEC_EINVAL; }
  }
  if (f64) {
    pl->ctas_comb = pl->td->ctas(0, max_kbins, nsm, 0);
    pl->ctas_bin = pl->ctas_bin_plain = pl->td->ctas(1, max_kbins, nsm, 0);
  } else {
    pl->ctas_comb = pl->tf->ctas(0, max_kbins, nsm, pl->xp);
    pl->ctas_bin = pl->tf->ctas(pl->has_ytab ? 2 : 1, max_kbins, nsm, pl->xp);
    pl->ctas_bin_plain = pl->tf->ctas(1, max_kbins, nsm, pl->xp);
  }
  pl->nblk_sum = 2 * nsm;

  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  pl->o_mesh1 = take(pl->Sr);
  pl->o_mesh2 = p->interlaced ? take(pl->Sr) : 0;
  pl->o_f0 = take(pl->Sc);
  pl->o_w = take(pl->Sc);
  pl->o_f = pl->roundtrip ? take(pl->Sr) : 0;
  pl->o_g = pl->group_max ? take(pl->Sc * pl->group_max) : 0;
  const size_t usz = 16;  // one table factor: float4 or double2
  pl->o_twh = take(NH * usz);
  pl->o_twf = take(N * usz);
  pl->o_twr = take(NH * usz);
  if (pl->xp) {
    pl->o_twh12 = take(NH * sizeof(float4));
    pl->o_twf12 = take(N * sizeof(float4));
    pl->o_twr12 = take(NH * sizeof(float4));
  }
  pl->o_axis = take(3 * (size_t)N * pl->esz);
  pl->o_phase = take(3 * (size_t)N * usz);
  pl->o_invw = take((N + NH) * csz);
  pl->o_ytab = pl->has_ytab ? take(pl->ytab_bytes) : 0;
  pl->o_rtab = pl->has_rtab ? take(pl->rtab_bytes) : 0;
  pl->has_ctab = !f64 && p->cartesian == 1;
  pl->ctab_bytes = pl->has_ctab ? (size_t)N * N * NH * sizeof(float) * kCartItems : 0;
  pl->o_ctab = pl->has_ctab ? take(pl->ctab_bytes) : 0;
  pl->o_bin = take((pl->n2max + 1) * sizeof(int32_t));
  pl->o_xtiles = take((size_t)N * (NH / pl->tf->tw) * sizeof(int32_t));
  pl->o_kmag = take((pl->n2max + 1) * sizeof(double));
  pl->o_cnt = take((pl->n2max + 1) * sizeof(uint32_t));
  pl->o_lo = take(max_kbins * sizeof(int32_t));
  pl->o_hi = take(max_kbins * sizeof(int32_t));
  pl->o_nmodes = take(max_kbins * sizeof(double));
  pl->o_ksum = take(max_kbins * sizeof(double));
  pl->o_sums = take(2 * (size_t)pl->nblk_sum * kSumVals * sizeof(double));
  pl->o_derived = take(D_COUNT * sizeof(double));
  pl->o_bins = take((size_t)(SLOT_ELL0 + kMaxElls) * max_kbins * sizeof(double));
  pl->o_out = take(((size_t)kMaxElls + 2) * max_kbins * sizeof(double));
  pl->max_particles = f64 ? 0 : p->max_particles;
  pl->ntiles = (N / kPaintTile) * (N / kPaintTile) * (N / kPaintTile);
  if (pl->max_particles > 0) {
    pl->o_tcnt = take((size_t)pl->ntiles * sizeof(unsigned));
    pl->o_toff = take((size_t)pl->ntiles * sizeof(unsigned));
    pl->o_tcur = take((size_t)pl->ntiles * sizeof(unsigned));
    pl->o_prec = take((size_t)pl->max_particles * 16);
    pl->o_ptile = take((size_t)pl->max_particles * sizeof(unsigned));
    pl->o_psort = take((size_t)pl->max_particles * kPaintRecordsMax * 16);
  }
  pl->cache_randoms = p->cache_randoms != 0;
  if (pl->cache_randoms) {
    pl->o_rmesh1 = take(pl->Sr);
    pl->o_rmesh2 = p->interlaced ? take(pl->Sr) : 0;
    pl->o_rsums = take(4 * sizeof(double));
    pl->o_desc = take((size_t)PSPEC_MAX_BATCH * sizeof(DevCat));
    pl->o_cur = take(sizeof(int));
    pl->o_bout = take(sizeof(BatchOut));
  }
  pl->total = o;
  return PSPEC_OK;
}

struct Ctx {
  pspec_params p;
  int device = 0;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  int64_t ws_bytes = 0;
  int max_kbins = 0;
  int nsm = 0;
  Plan pl;
  bool painted = false;
  bool randoms_set = false;
  std::vector<double> edges;
  // From the bins of `edges`: no |n|^2 >= n2_cut is binned, so x columns (ny, kz) with
  // ny^2 + kz^2 >= n2_cut are neither stored by the harmonics' y pass nor read by the binning
  // pass. Fractions of what remains, for the byte accounting: slabs read and outputs stored
  // by that y pass, tiles of the binning pass.
  int n2_cut = INT_MAX;
  int n_xtiles = 0;  // entries of the plan's x-tile list
  double frac_yr = 1.0, frac_yw = 1.0, frac_tile = 1.0;
  // captured per-mock graph and what it was captured for
  cudaGraphExec_t graph = nullptr;
  cudaStream_t cap_stream = nullptr;  // graphs are captured and replayed here (never the legacy stream)
  std::vector<int32_t> graph_ells;
  std::vector<double> graph_edges;
  int graph_binned = -1;
  int64_t graph_kernels = 0;
  std::vector<DevCat> desc_host;
  BatchOut bout_host{};  // this batch's output buffers, uploaded to o_bout
  pspec_catalog batch_proto{};  // dtype of the mocks' positions (pointers come from the table)
  pspec_tuning tune{1, 64, 0, 0};
  std::string err;
  int64_t launches = 0;
  int64_t transforms_last = 0;
  int64_t sh_last = 0;
  double bytes_paint = 0, bytes_mult = 0;
  // profiling
  bool prof = false;
  struct Rec {
    int k;
    cudaEvent_t a, b;
    double bytes;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  int64_t k_launch[PSPEC_K_COUNT] = {};
  double k_ms[PSPEC_K_COUNT] = {};
  double k_bytes[PSPEC_K_COUNT] = {};

  template <typename U> U* at(size_t off) { return reinterpret_cast<U*>(ws + off); }
};

cudaEvent_t take_event(Ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch wrapper: counts launches, brackets with events when profiling, checks errors.
template <typename F>
pspec_status run(Ctx* c, int kclass, double bytes, F&& launch) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (c->prof) {
    a = take_event(c);
    b = take_event(c);
    cudaEventRecord(a, c->stream);
  }
  launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    c->err = std::string("kernel launch failed: ") + cudaGetErrorString(e);
    return PSPEC_ECUDA;
  }
  c->launches++;
  if (c->prof) {
    cudaEventRecord(b, c->stream);
    c->recs.push_back({kclass, a, b, bytes});
  }
  return PSPEC_OK;
}

#define TRY(x)                     \
  do {                             \
    pspec_status _s = (x);         \
    if (_s != PSPEC_OK) return _s; \
  } while (0)

pspec_status cuda_fail(Ctx* c, cudaError_t e, const char* what) {
  c->err = std::string(what) + ": " + cudaGetErrorString(e);
  return PSPEC_ECUDA;
}

// exp(i a) as a table entry; in FP32 each component as hi + lo (lo = its rounding error).
template <typename T> ux<T> unit_factor(double a);
template <> ux<float> unit_factor<float>(double a) {
  const double c = std::cos(a), s = std::sin(a);
  const float ch = (float)c, sh = (float)s;
  return make_float4(ch, sh, (float)(c - (double)ch), (float)(s - (double)sh));
}
template <> ux<double> unit_factor<double>(double a) { return make_double2(std::cos(a), std::sin(a)); }
// The form the exact-add stages use: {c12, s12, c - c12, s - s12}, c12 and s12 multiples of 2^-12.
float4 unit_factor12(double a) {
  const double c = std::cos(a), s = std::sin(a);
  const double c12 = std::nearbyint(c * 4096.0) / 4096.0, s12 = std::nearbyint(s * 4096.0) / 4096.0;
  return make_float4((float)c12, (float)s12, (float)(c - c12), (float)(s - s12));
}

template <typename T>
pspec_status upload_tables(Ctx* c) {
  const Plan& pl = c->pl;
  const int N = pl.g.N, NH = pl.g.NH;
  using C = cx<T>;
  using U = ux<T>;
  std::vector<U> twh(NH), twf(N), twr(NH), phase(3 * N);
  std::vector<C> invw(N + NH);
  std::vector<T> axis(3 * N);
  for (int t = 0; t < NH; t++) {
    twh[t] = unit_factor<T>(-2.0 * M_PI * t / NH);
    twr[t] = unit_factor<T>(-2.0 * M_PI * t / N);
  }
  for (int t = 0; t < N; t++) twf[t] = unit_factor<T>(-2.0 * M_PI * t / N);
  const double H = c->p.box_size / N;
  for (int d = 0; d < 3; d++)
    for (int i = 0; i < N; i++) axis[d * N + i] = T(c->p.box_corner[d] + i * H - c->p.observer[d]);
  const int p = c->p.window;  // order of sinc^p
  // compensation divisor per axis: sinc^p(pi n/N), or (compensate = 2) the square root of its
  // alias sum sum_m sinc^{2p}(pi (n/N + m)) in closed form (Jing 2005): 1 - 2/3 s^2 (CIC),
  // 1 - s^2 + 2/15 s^4 (TSC), s = sin(pi n/N)
  auto sincp = [&](int n) {
    const double x = M_PI * n / N;
    if (c->p.compensate == 2) {
      const double s2 = std::sin(x) * std::sin(x);
      return std::sqrt(p == PSPEC_WINDOW_CIC ? 1.0 - 2.0 / 3.0 * s2 : 1.0 - s2 + 2.0 / 15.0 * s2 * s2);
    }
    if (n == 0) return 1.0;
    return std::pow(std::sin(x) / x, p);
  };
  // exp(-i pi s / N), s = nx + ny + nz in [-3N/2, 3N/2): the H/2 shift of the second mesh
  for (int i = 0; i < 3 * N; i++) phase[i] = unit_factor<T>(-M_PI * (i - 3 * N / 2) / N);
  for (int i = 0; i < N + NH; i++) {
    const int n = i < N ? (i < NH ? i : i - N) : (i - N);
    const double w = 1.0 / sincp(n);
    const T hi = T(w);
    invw[i] = mk(hi, T(w / (double)hi - 1.0));
  }
  cudaError_t e;
  e = cudaMemcpyAsync(c->at<U>(pl.o_twh), twh.data(), NH * sizeof(U), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->at<U>(pl.o_twf), twf.data(), N * sizeof(U), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->at<U>(pl.o_twr), twr.data(), NH * sizeof(U), cudaMemcpyHostToDevice, c->stream);
  std::vector<float4> twh12(NH), twf12(N), twr12(NH);
  if (pl.xp) {
    for (int t = 0; t < NH; t++) {
      twh12[t] = unit_factor12(-2.0 * M_PI * t / NH);
      twr12[t] = unit_factor12(-2.0 * M_PI * t / N);
    }
    for (int t = 0; t < N; t++) twf12[t] = unit_factor12(-2.0 * M_PI * t / N);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->at<float4>(pl.o_twh12), twh12.data(), NH * sizeof(float4), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->at<float4>(pl.o_twf12), twf12.data(), N * sizeof(float4), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->at<float4>(pl.o_twr12), twr12.data(), NH * sizeof(float4), cudaMemcpyHostToDevice, c->stream);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->at<T>(pl.o_axis), axis.data(), 3 * N * sizeof(T), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->at<U>(pl.o_phase), phase.data(), 3 * N * sizeof(U), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->at<C>(pl.o_invw), invw.data(), (N + NH) * sizeof(C), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->at<uint32_t>(pl.o_cnt), 0, (pl.n2max + 1) * sizeof(uint32_t), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "table upload");
  TRY(run(c, PSPEC_K_OTHER, 0.0, [&] { launch_mode_counts(pl.g, c->at<uint32_t>(pl.o_cnt), c->nsm, c->stream); }));
  if (pl.has_ytab)
    TRY(run(c, PSPEC_K_OTHER, 0.0, [&] { launch_ytab_build(c->at<float>(pl.o_ytab), N, pl.tf->tw, c->p.ell_max, c->nsm, c->stream); }));
  if (pl.has_rtab) {
    RGeo g;
    for (int d = 0; d < 3; d++) {
      g.corner[d] = c->p.box_corner[d];
      g.observer[d] = c->p.observer[d];
    }
    g.H = H;
    TRY(run(c, PSPEC_K_OTHER, 0.0, [&] { launch_rtab_build(c->at<float>(pl.o_rtab), N, c->p.ell_max, g, c->nsm, c->stream); }));
  }
  if (pl.has_ctab)
    TRY(run(c, PSPEC_K_OTHER, 0.0, [&] { launch_ctab_build(c->at<float>(pl.o_ctab), N, pl.tf->tw, c->nsm, c->stream); }));
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "table upload");
  return PSPEC_OK;
}

// Bin decision of every |n|^2 in FP64: b iff t_b <= n2 < t_{b+1}, t_b = (k_b L/(2 pi))^2.
// The |n|^2 values of a bin form one range [lo_b, hi_b); N_b and sum |k| follow on the
// device from the mode counts.
pspec_status upload_bins(Ctx* c, const double* edges, int nk) {
  std::vector<double> e(edges, edges + nk + 1);
  if (e == c->edges) return PSPEC_OK;
  const Plan& pl = c->pl;
  std::vector<double> t(nk + 1);
  for (int b = 0; b <= nk; b++) {
    const double x = e[b] * c->p.box_size / (2.0 * M_PI);
    t[b] = x * x;
  }
  std::vector<int32_t> bin(pl.n2max + 1), lo(nk, 0), hi(nk, 0);
  std::vector<double> kmag(pl.n2max + 1);
  const double kf = 2.0 * M_PI / c->p.box_size;
  int n2_cut = 0;
  for (int n2 = 0; n2 <= pl.n2max; n2++) {
    const double x = (double)n2;
    int b = -1;
    if (n2 > 0 && x >= t[0] && x < t[nk]) b = (int)(std::upper_bound(t.begin(), t.end(), x) - t.begin()) - 1;
    bin[n2] = b;
    kmag[n2] = kf * std::sqrt(x);
    if (b >= 0) {
      if (hi[b] == 0) lo[b] = n2;
      hi[b] = n2 + 1;
      n2_cut = n2 + 1;
    }
  }
  {
    const int N = pl.g.N, NH = pl.g.NH;
    const int tw = c->p.precision == PSPEC_FP64 ? pl.td->tw : pl.tf->tw;
    const int ntz = NH / tw;
    int64_t yr = 0, yw = 0;
    std::vector<int32_t> xt;
    xt.reserve((size_t)N * ntz);
    // x tiles in storage order, tile = kz tile * N + j; active when the (ky, kz) column's
    // smallest |n|^2 is below the last bin
    for (int kt = 0; kt < ntz; kt++)
      for (int j = 0; j < N; j++) {
        const int64_t ny2 = (int64_t)(j < NH ? j : j - N) * (j < NH ? j : j - N);
        if (ny2 + (int64_t)kt * tw * kt * tw < n2_cut) xt.push_back(kt * N + j);
        for (int kz = kt * tw; kz < (kt + 1) * tw; kz++) yw += ny2 + (int64_t)kz * kz < n2_cut;
      }
    for (int kz0 = 0; kz0 < NH; kz0 += tw) yr += (int64_t)kz0 * kz0 < n2_cut;
    c->frac_yw = (double)yw / ((double)N * NH);
    c->frac_tile = (double)xt.size() / ((double)N * ntz);
    c->frac_yr = (double)yr / (double)ntz;
    c->n_xtiles = (int)xt.size();
    if (!xt.empty()) {
      const cudaError_t ex = cudaMemcpyAsync(c->at<int32_t>(pl.o_xtiles), xt.data(), xt.size() * sizeof(int32_t),
                                             cudaMemcpyHostToDevice, c->stream);
      if (ex != cudaSuccess) return cuda_fail(c, ex, "tile list upload");
    }
  }
  cudaError_t er = cudaMemcpyAsync(c->at<int32_t>(pl.o_bin), bin.data(), bin.size() * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, c->stream);
  if (er == cudaSuccess)
    er = cudaMemcpyAsync(c->at<double>(pl.o_kmag), kmag.data(), kmag.size() * sizeof(double), cudaMemcpyHostToDevice,
                         c->stream);
  if (er == cudaSuccess)
    er = cudaMemcpyAsync(c->at<int32_t>(pl.o_lo), lo.data(), nk * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream);
  if (er == cudaSuccess)
    er = cudaMemcpyAsync(c->at<int32_t>(pl.o_hi), hi.data(), nk * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream);
  if (er != cudaSuccess) return cuda_fail(c, er, "bin table upload");
  TRY(run(c, PSPEC_K_OTHER, 0.0, [&] {
    launch_bin_counts(c->at<uint32_t>(pl.o_cnt), c->at<double>(pl.o_kmag), c->at<int32_t>(pl.o_lo),
                      c->at<int32_t>(pl.o_hi), nk, c->at<double>(pl.o_nmodes), c->at<double>(pl.o_ksum), c->stream);
  }));
  er = cudaStreamSynchronize(c->stream);
  if (er != cudaSuccess) return cuda_fail(c, er, "bin table upload");
  c->edges = e;
  c->n2_cut = n2_cut;
  return PSPEC_OK;
}

pspec_status check_catalog(Ctx* c, const pspec_catalog* cat, const char* name, bool need_points) {
  if (!cat) { c->err = std::string(name) + " catalog is NULL"; return PSPEC_EINVAL; }
  if (cat->count < 0) { c->err = std::string(name) + " count < 0"; return PSPEC_EINVAL; }
  if (need_points && cat->count == 0) { c->err = std::string(name) + " catalog is empty"; return PSPEC_EINVAL; }
  if (cat->count > 0 && !cat->pos) { c->err = std::string(name) + " positions are NULL"; return PSPEC_EINVAL; }
  if (cat->pos_dtype != PSPEC_POS_F64 && cat->pos_dtype != PSPEC_POS_F32) { c->err = "pos_dtype"; return PSPEC_EINVAL; }
  return PSPEC_OK;
}

double fkp(double nbar, double P0) { return P0 > 0 ? 1.0 / (1.0 + nbar * P0) : 1.0; }

PaintArgs paint_args(Ctx* c, const pspec_catalog* cat) {
  PaintArgs a;
  a.pos = cat->pos;
  a.pos_f32 = cat->pos_dtype == PSPEC_POS_F32;
  a.weight = cat->weight;
  a.nbar = cat->nbar;
  a.count = cat->count;
  for (int d = 0; d < 3; d++) a.corner[d] = c->p.box_corner[d];
  a.inv_cell = (double)c->p.nmesh / c->p.box_size;
  a.P0 = c->p.P0;
  a.nbar_default = c->p.nbar;
  a.wf_default = fkp(c->p.nbar, c->p.P0);
  a.dc = nullptr;
  a.cur = nullptr;
  return a;
}

double cat_bytes(const pspec_catalog* cat) {
  const double per = (cat->pos_dtype == PSPEC_POS_F32 ? 12.0 : 24.0) + (cat->weight ? 8.0 : 0.0) +
                     (cat->nbar ? 8.0 : 0.0);
  return per * (double)cat->count;
}

TileArgs tile_args(Ctx* c) {
  const Plan& pl = c->pl;
  TileArgs ta;
  ta.cnt = c->at<unsigned>(pl.o_tcnt);
  ta.off = c->at<unsigned>(pl.o_toff);
  ta.cursor = c->at<unsigned>(pl.o_tcur);
  ta.rec = c->at<uint4>(pl.o_prec);
  ta.tile_of = c->at<unsigned>(pl.o_ptile);
  ta.sorted = c->at<uint4>(pl.o_psort);
  return ta;
}

template <typename T>
pspec_status do_paint(Ctx* c, const pspec_catalog* d, const pspec_catalog* r) {
  const Plan& pl = c->pl;
  const int N = pl.g.N;
  T* m1 = c->at<T>(pl.o_mesh1);
  T* m2 = c->p.interlaced ? c->at<T>(pl.o_mesh2) : nullptr;
  cudaError_t e = cudaSuccess;
  double* der = c->at<double>(pl.o_derived);
  const PaintArgs ad = paint_args(c, d), ar = paint_args(c, r);
  const bool uniform = !d->weight && !d->nbar && !r->weight && !r->nbar;
  double bytes = 0;
  if (uniform) {
    TRY(run(c, PSPEC_K_SUMS, 0.0, [&] {
      launch_derive_uniform(d->count, r->count, ad.wf_default, c->p.nbar, der, c->stream);
    }));
  } else {
    double* sums = c->at<double>(pl.o_sums);
    double* part_d = sums;
    double* part_r = sums + (size_t)pl.nblk_sum * kSumVals;
    TRY(run(c, PSPEC_K_SUMS, cat_bytes(d), [&] { launch_catalog_partials(ad, part_d, pl.nblk_sum, c->stream); }));
    TRY(run(c, PSPEC_K_SUMS, cat_bytes(r), [&] { launch_catalog_partials(ar, part_r, pl.nblk_sum, c->stream); }));
    TRY(run(c, PSPEC_K_SUMS, 0.0, [&] {
      launch_catalog_final(part_d, pl.nblk_sum, part_r, pl.nblk_sum, der, c->stream, der + D_FIX);
    }));
    bytes += cat_bytes(d) + cat_bytes(r);
  }
  // algorithmic bytes of painting: the particles once and each mesh written once
  const int nb = 16 * c->nsm;
  const double nmesh = c->p.interlaced ? 2.0 : 1.0;
  const int64_t total = d->count + r->count;
  if (sizeof(T) == 4 && c->tune.paint_binned && pl.max_particles > 0 && total <= pl.max_particles) {
    // exact tile-binned paint: every cell of both meshes is stored, nothing to clear
    TileArgs ta = tile_args(c);
    e = cudaMemsetAsync(ta.cnt, 0, (size_t)pl.ntiles * sizeof(unsigned), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tile counts clear");
    float* f1 = reinterpret_cast<float*>(m1);
    float* f2 = reinterpret_cast<float*>(m2);
    TRY(run(c, PSPEC_K_PAINT, cat_bytes(d), [&] {
      launch_ptile_prep(ad, c->p.window, c->p.interlaced, 0, der, ta, 0, N, nb, c->stream);
    }));
    TRY(run(c, PSPEC_K_PAINT, cat_bytes(r), [&] {
      launch_ptile_prep(ar, c->p.window, c->p.interlaced, 1, der, ta, d->count, N, nb, c->stream);
    }));
    TRY(run(c, PSPEC_K_PAINT, 0.0, [&] { launch_ptile_scan(ta, pl.ntiles, c->stream); }));
    TRY(run(c, PSPEC_K_PAINT, 0.0, [&] { launch_ptile_scatter(ta, total, nullptr, nullptr, N, nb, c->stream); }));
    TRY(run(c, PSPEC_K_PAINT, nmesh * pl.Sr, [&] {
      launch_ptile_paint(ta, c->p.window, c->p.interlaced, f1, f2, N, der + D_FIX, c->stream);
    }));
    c->bytes_paint = bytes + cat_bytes(d) + cat_bytes(r) + nmesh * pl.Sr;
    return PSPEC_OK;
  }
  e = cudaMemsetAsync(m1, 0, pl.Sr, c->stream);
  if (e == cudaSuccess && m2) e = cudaMemsetAsync(m2, 0, pl.Sr, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "mesh clear");
  const double frac_d = (double)d->count / (double)(d->count + r->count);
  if (d->count > 0)
    TRY(run(c, PSPEC_K_PAINT, cat_bytes(d) + frac_d * nmesh * pl.Sr, [&] {
      launch_paint<T>(ad, c->p.window, c->p.interlaced, 0, der, m1, m2, N, nb, c->stream);
    }));
  TRY(run(c, PSPEC_K_PAINT, cat_bytes(r) + (1.0 - frac_d) * nmesh * pl.Sr, [&] {
    launch_paint<T>(ar, c->p.window, c->p.interlaced, 1, der, m1, m2, N, nb, c->stream);
  }));
  c->bytes_paint = bytes + cat_bytes(d) + cat_bytes(r) + nmesh * pl.Sr;
  return PSPEC_OK;
}

// Range of the flattened harmonic list (see pspec_multipoles_range) a multipoles call covers.
struct HRange {
  int q0 = 0;
  int q1 = 1 << 30;
  bool include_p0 = true;
  double* bins_out = nullptr;  // raw bins instead of finalized multipoles
  bool cartesian = false;      // Cartesian decomposition (monomials of degree 2 and 4)
};

template <typename T>
pspec_status do_multipoles(Ctx* c, const int32_t* ells, int n_ells, int nk, double* P, double* km, double* nm,
                           const HRange& hr = HRange()) {
  using C = cx<T>;
  const Plan& pl = c->pl;
  const Geo& g = pl.g;
  const int N = g.N;
  const PassTable<T>* PT = pass_table<T>(N);
  cudaStream_t s = c->stream;
  T* m1 = c->at<T>(pl.o_mesh1);
  T* m2 = c->at<T>(pl.o_mesh2);
  C* F0 = c->at<C>(pl.o_f0);
  C* W = c->at<C>(pl.o_w);
  T* f = pl.roundtrip ? c->at<T>(pl.o_f) : m1;
  C* G = c->at<C>(pl.o_g);
  using U = ux<T>;
  const U* twh = c->at<U>(pl.o_twh);
  const U* twf = c->at<U>(pl.o_twf);
  const U* twr = c->at<U>(pl.o_twr);
  // the exact-add launches take the twiddles in their 12-bit form (FP32 contexts with xp)
  const U* twh_x = pl.xp ? reinterpret_cast<const U*>(c->at<float4>(pl.o_twh12)) : twh;
  const U* twf_x = pl.xp ? reinterpret_cast<const U*>(c->at<float4>(pl.o_twf12)) : twf;
  const U* twr_x = pl.xp ? reinterpret_cast<const U*>(c->at<float4>(pl.o_twr12)) : twr;
  const T* axis = c->at<T>(pl.o_axis);
  const U* phase = c->at<U>(pl.o_phase);
  const C* invw = c->at<C>(pl.o_invw);
  const double Sr = (double)pl.Sr, Sc = (double)pl.Sc;
  BinArgs ba;
  ba.bin_of_n2 = c->at<int32_t>(pl.o_bin);
  ba.nk = nk;
  ba.bins = c->at<double>(pl.o_bins);
  ba.permode_w = c->p.compensate == 3 ? static_cast<const void*>(c->at<C>(pl.o_invw)) : nullptr;
  ba.odd = 0;
  ba.xtiles = c->at<int32_t>(pl.o_xtiles);
  ba.n_xtiles = c->n_xtiles;
  cudaError_t e = cudaMemsetAsync(ba.bins, 0, (size_t)(SLOT_ELL0 + std::max(n_ells, 2)) * nk * sizeof(double), s);
  if (e != cudaSuccess) return cuda_fail(c, e, "bins clear");
  int64_t transforms = 0;
  double bytes = 0;
  const int ntiles_x = N * (g.NH / PT->tw);
  const int ctas_comb = c->tune.bin_blocks_per_sm > 0 ? std::min(ntiles_x, c->tune.bin_blocks_per_sm * c->nsm)
                                                      : pl.ctas_comb;
  const int ctas_bin = c->tune.bin_blocks_per_sm > 0 ? std::min(ntiles_x, c->tune.bin_blocks_per_sm * c->nsm)
                                                     : pl.ctas_bin;
  const int ctas_bin_plain = c->tune.bin_blocks_per_sm > 0 ? ctas_bin : pl.ctas_bin_plain;
  auto acc = [&](double b) {
    bytes += b;
    return b;
  };

  // a3: F1 (and F2), combine + compensate -> F0 with the l = 0 sums; round trip -> f
  TRY(run(c, PSPEC_K_FFT_Z, acc(Sr + Sc), [&] { PT->r2c_z(m1, F0, twh, twr, s); }));
  TRY(run(c, PSPEC_K_FFT_Y, acc(2 * Sc), [&] { PT->fft_y(F0, 0, 1, twf, -1, c->tune.tile_y, INT_MAX, 0, s); }));
  transforms++;
  if (c->p.interlaced) {
    TRY(run(c, PSPEC_K_FFT_X, acc(2 * Sc), [&] { PT->fft_x(F0, F0, twf, -1, 0, s); }));
    TRY(run(c, PSPEC_K_FFT_Z, acc(Sr + Sc), [&] { PT->r2c_z(m2, W, twh, twr, s); }));
    TRY(run(c, PSPEC_K_FFT_Y, acc(2 * Sc), [&] { PT->fft_y(W, 0, 1, twf, -1, c->tune.tile_y, INT_MAX, 0, s); }));
    transforms++;
    TRY(run(c, PSPEC_K_COMBINE, acc(3 * Sc), [&] {
      PT->combine_x(W, F0, twf, 1, c->p.compensate, pl.roundtrip, phase, invw, ba, ctas_comb, s);
    }));
  } else {
    TRY(run(c, PSPEC_K_COMBINE, acc(2 * Sc), [&] {
      PT->combine_x(F0, F0, twf, 0, c->p.compensate, pl.roundtrip, phase, invw, ba, ctas_comb, s);
    }));
  }
  if (pl.roundtrip) {
    TRY(run(c, PSPEC_K_FFT_X, acc(2 * Sc), [&] { PT->fft_x(F0, W, twf_x, +1, pl.xp, s); }));
    TRY(run(c, PSPEC_K_FFT_Y, acc(2 * Sc), [&] { PT->fft_y(W, 0, 1, twf_x, +1, c->tune.tile_y, INT_MAX, pl.xp, s); }));
    const T scale = T(2.0 / ((double)N * N * N));
    TRY(run(c, PSPEC_K_C2R_Z, acc(Sc + Sr), [&] { PT->c2r_z(W, f, twh_x, twr_x, scale, pl.xp, s); }));
    transforms++;
  }

  // a4 + a5: per multipole l >= 2 (or per monomial degree of the Cartesian route), groups of
  // harmonics (those of [q0, q1) of the flat list)
  int64_t sh = 0;
  const int64_t stride = (int64_t)N * N * g.NH;
  struct Job {
    int zarg, nh, slot;
    const float* table;  // k-space factor slot of item 0, or nullptr
  };
  Job jobs[kMaxElls];
  int njobs = 0;
  if (!hr.cartesian) {
    int qbase = 0;
    for (int i = 0; i < n_ells; i++) {
      const int ell = ells[i];
      sh += 2 * ell + 1;
      if (ell == 0) continue;
      const int nh = 2 * ell + 1;
      const float* tb = pl.has_ytab && !(ell & 1) ? c->at<float>(pl.o_ytab) + (int64_t)ytab_base(ell) * stride : nullptr;
      jobs[njobs++] = {ell, nh, SLOT_ELL0 + i, tb};
      (void)qbase;
    }
  } else {
    int lmax = 0;
    for (int i = 0; i < n_ells; i++) lmax = std::max(lmax, (int)ells[i]);
    sh = 1 + (lmax >= 2 ? 6 : 0) + (lmax >= 4 ? 15 : 0);
    const float* ct = c->at<float>(pl.o_ctab);
    if (lmax >= 2) jobs[njobs++] = {-2, 6, SLOT_ELL0, ct};
    if (lmax >= 4) jobs[njobs++] = {-4, 15, SLOT_ELL0 + 1, ct + 6 * stride};
  }
  int qbase = 0;
  for (int jb = 0; jb < njobs; jb++) {
    const int ell = jobs[jb].zarg;
    const int nh = jobs[jb].nh;
    const int hlo = std::max(0, hr.q0 - qbase), hhi = std::min(nh, hr.q1 - qbase);
    qbase += nh;
    for (int h0 = hlo; h0 < hhi; h0 += pl.group_max) {
      const int M = std::min(pl.group_max, hhi - h0);
      // z pass with the Y_lm weights: one block holds Ms harmonics x rows rows, tz threads each
      const int tz = pl.xp ? PT->tz_xp : PT->tz;
      const int cap = ylm_thread_cap(ell);
      const int ms_max = std::max(1, std::min(c->tune.ylm_harmonics, cap / tz));
      for (int hs = 0; hs < M; hs += ms_max) {
        const int Ms = std::min(ms_max, M - hs);
        int rows = std::max(1, pow2_floor(std::max(1, cap / (Ms * tz))));
        while (rows > 1 && (((int64_t)N * N) % rows || PT->smem_ylm(Ms, rows) > kSmemBudget)) rows >>= 1;
        // even l of the SH route read their weights from the Y_lm(rhat) table when the plan holds it
        const float* rt = pl.has_rtab && ell > 0 && !(ell & 1)
                              ? c->at<float>(pl.o_rtab) + (int64_t)(ytab_base(ell) + h0 + hs) * N * N * N
                              : nullptr;
        TRY(run(c, PSPEC_K_YLM_Z, acc(Sr + Ms * Sc + (rt ? Ms * (double)N * N * N * sizeof(float) : 0.0)), [&] {
          PT->ylm_z(f, G + hs * stride, stride, ell, h0 + hs, Ms, twh_x, twr_x, axis, rows, rt, pl.xp, s);
        }));
      }
      TRY(run(c, PSPEC_K_FFT_Y, acc(M * Sc * (c->frac_yr + c->frac_yw)),
              [&] { PT->fft_y(G, stride, M, twf_x, -1, c->tune.tile_y, c->n2_cut, pl.xp, s); }));
      const float* ytab = jobs[jb].table ? jobs[jb].table + (int64_t)h0 * stride : nullptr;
      const double ybytes = ytab ? M * (double)N * N * g.NH * sizeof(float) : 0.0;
      BinArgs bj = ba;
      bj.odd = ell > 0 && (ell & 1);
      TRY(run(c, PSPEC_K_BIN_X, acc((Sc + M * Sc + ybytes) * c->frac_tile), [&] {
        PT->bin_x(G, stride, ell, h0, M, F0, twf_x, jobs[jb].slot, bj, ytab ? ctas_bin : ctas_bin_plain, ytab, pl.xp, s);
      }));
      transforms += M;
    }
  }
  if (hr.bins_out) {
    const size_t nb = (size_t)(SLOT_ELL0 + n_ells) * nk * sizeof(double);
    e = cudaMemcpyAsync(hr.bins_out, ba.bins, nb, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && !hr.include_p0) e = cudaMemsetAsync(hr.bins_out, 0, (size_t)nk * sizeof(double), s);
    if (e != cudaSuccess) return cuda_fail(c, e, "range bins");
    c->transforms_last = transforms;
    c->sh_last = sh;
    c->bytes_mult = bytes;
    return PSPEC_OK;
  }
  // a6
  TRY(run(c, PSPEC_K_FINAL, 0.0, [&] {
    launch_finalize(ba.bins, c->at<double>(pl.o_nmodes), c->at<double>(pl.o_ksum), nk, ells, n_ells,
                    c->at<double>(pl.o_derived), P, km, nm, s, hr.cartesian ? 1 : 0);
  }));
  c->transforms_last = transforms;
  c->sh_last = sh;
  c->bytes_mult = bytes;
  return PSPEC_OK;
}

// Paint `a` (a data catalog, or randoms with is_randoms = 2) into m1/m2 (zeroed here):
// tile-binned when `binned`, else direct atomics. `max_count` bounds the particles.
template <typename T>
pspec_status paint_one(Ctx* c, const PaintArgs& a, int is_randoms, bool binned, int64_t max_count, T* m1, T* m2,
                       const double* fix) {
  const Plan& pl = c->pl;
  const int N = pl.g.N;
  const int nb = 16 * c->nsm;
  double* der = c->at<double>(pl.o_derived);
  cudaError_t e = cudaSuccess;
  const double nmesh = c->p.interlaced ? 2.0 : 1.0;
  const double pbytes = (a.pos_f32 ? 12.0 : 24.0) * (double)max_count;
  if (binned && sizeof(T) == 4) {
    TileArgs ta = tile_args(c);
    e = cudaMemsetAsync(ta.cnt, 0, (size_t)pl.ntiles * sizeof(unsigned), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tile counts clear");
    TRY(run(c, PSPEC_K_PAINT, pbytes, [&] {
      launch_ptile_prep(a, c->p.window, c->p.interlaced, is_randoms, der, ta, 0, N, nb, c->stream);
    }));
    TRY(run(c, PSPEC_K_PAINT, 0.0, [&] { launch_ptile_scan(ta, pl.ntiles, c->stream); }));
    TRY(run(c, PSPEC_K_PAINT, 0.0, [&] { launch_ptile_scatter(ta, a.count, a.dc, a.cur, N, nb, c->stream); }));
    TRY(run(c, PSPEC_K_PAINT, nmesh * pl.Sr, [&] {
      launch_ptile_paint(ta, c->p.window, c->p.interlaced, reinterpret_cast<float*>(m1), reinterpret_cast<float*>(m2),
                         N, fix, c->stream);
    }));
  } else {
    e = cudaMemsetAsync(m1, 0, pl.Sr, c->stream);
    if (e == cudaSuccess && m2) e = cudaMemsetAsync(m2, 0, pl.Sr, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "mesh clear");
    TRY(run(c, PSPEC_K_PAINT, pbytes + nmesh * pl.Sr, [&] {
      launch_paint<T>(a, c->p.window, c->p.interlaced, is_randoms, der, m1, m2, N, nb, c->stream);
    }));
  }
  return PSPEC_OK;
}

template <typename T>
pspec_status do_set_randoms(Ctx* c, const pspec_catalog* r) {
  const Plan& pl = c->pl;
  PaintArgs ar = paint_args(c, r);
  double* part = c->at<double>(pl.o_sums) + (size_t)pl.nblk_sum * kSumVals;
  TRY(run(c, PSPEC_K_SUMS, cat_bytes(r), [&] { launch_catalog_partials(ar, part, pl.nblk_sum, c->stream); }));
  TRY(run(c, PSPEC_K_SUMS, 0.0, [&] { launch_randoms_sums(part, pl.nblk_sum, c->at<double>(pl.o_rsums), c->stream); }));
  T* r1 = c->at<T>(pl.o_rmesh1);
  T* r2 = c->p.interlaced ? c->at<T>(pl.o_rmesh2) : nullptr;
  const bool binned = c->tune.paint_binned && pl.max_particles >= r->count;
  TRY(paint_one<T>(c, ar, 2, binned, r->count, r1, r2, c->at<double>(pl.o_rsums) + 3));
  return PSPEC_OK;
}

// One mock of a batch: sums, paint, mesh -= alpha * randoms, multipoles, outputs, counter.
template <typename T>
pspec_status enqueue_mock(Ctx* c, bool binned, int64_t max_count, const int32_t* ells, int n_ells, int nk) {
  const Plan& pl = c->pl;
  PaintArgs a = paint_args(c, &c->batch_proto);
  a.dc = c->at<DevCat>(pl.o_desc);
  a.cur = c->at<int>(pl.o_cur);
  double* part = c->at<double>(pl.o_sums);
  double* der = c->at<double>(pl.o_derived);
  TRY(run(c, PSPEC_K_SUMS, 0.0, [&] { launch_catalog_partials(a, part, pl.nblk_sum, c->stream); }));
  TRY(run(c, PSPEC_K_SUMS, 0.0, [&] {
    launch_catalog_final_cached(part, pl.nblk_sum, c->at<double>(pl.o_rsums), der, c->stream);
  }));
  T* m1 = c->at<T>(pl.o_mesh1);
  T* m2 = c->p.interlaced ? c->at<T>(pl.o_mesh2) : nullptr;
  TRY(paint_one<T>(c, a, 0, binned, max_count, m1, m2, der + D_FIX));
  const int64_t n = (int64_t)pl.g.N * pl.g.N * pl.g.N;
  TRY(run(c, PSPEC_K_OTHER, 3.0 * pl.Sr, [&] { launch_axpy_randoms(m1, c->at<T>(pl.o_rmesh1), n, der, c->stream); }));
  if (m2)
    TRY(run(c, PSPEC_K_OTHER, 3.0 * pl.Sr, [&] { launch_axpy_randoms(m2, c->at<T>(pl.o_rmesh2), n, der, c->stream); }));
  double* out = c->at<double>(pl.o_out);
  TRY(do_multipoles<T>(c, ells, n_ells, nk, out + 2 * (size_t)nk, out, out + nk));
  TRY(run(c, PSPEC_K_OTHER, 0.0, [&] {
    launch_batch_outputs(out + 2 * (size_t)nk, n_ells, nk, der, a.cur, c->at<BatchOut>(pl.o_bout), c->stream);
  }));
  TRY(run(c, PSPEC_K_OTHER, 0.0, [&] { launch_advance(c->at<int>(pl.o_cur), c->stream); }));
  return PSPEC_OK;
}

pspec_status check_ells_edges(Ctx* c, const int32_t* ells, int n_ells, const double* k_edges, int nk) {
  if (!ells || n_ells < 1 || n_ells > kMaxElls) { c->err = "need 1..9 multipoles"; return PSPEC_EINVAL; }
  for (int i = 0; i < n_ells; i++) {
    if (ells[i] < 0) { c->err = "negative l"; return PSPEC_EINVAL; }
    if (ells[i] > c->p.ell_max) { c->err = "l above the context's ell_max"; return PSPEC_EUNSUPPORTED; }
    for (int j = 0; j < i; j++)
      if (ells[j] == ells[i]) { c->err = "repeated l"; return PSPEC_EINVAL; }
  }
  if (!k_edges || nk < 1 || nk > c->max_kbins) { c->err = "n_kbins out of range"; return PSPEC_EINVAL; }
  for (int b = 0; b <= nk; b++) {
    if (!std::isfinite(k_edges[b]) || k_edges[b] < 0) { c->err = "k edges must be finite and >= 0"; return PSPEC_EINVAL; }
    if (b && !(k_edges[b] > k_edges[b - 1])) { c->err = "k edges must increase strictly"; return PSPEC_EINVAL; }
  }
  if (!c->painted) { c->err = "multipoles before paint"; return PSPEC_ESTATE; }
  return PSPEC_OK;
}

pspec_status multipoles_common(Ctx* c, const int32_t* ells, int n_ells, const double* k_edges, int nk, double* P,
                               double* km, double* nm) {
  TRY(check_ells_edges(c, ells, n_ells, k_edges, nk));
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  TRY(upload_bins(c, k_edges, nk));
  if (c->p.precision == PSPEC_FP64) return do_multipoles<double>(c, ells, n_ells, nk, P, km, nm);
  return do_multipoles<float>(c, ells, n_ells, nk, P, km, nm);
}

}  // namespace

extern "C" {

pspec_status pspec_workspace_size(const pspec_params* p, int32_t max_kbins, int64_t* bytes) {
  if (!bytes) return PSPEC_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PSPEC_ECUDA;
  Plan pl;
  std::string why;
  pspec_status st = build_plan(p, max_kbins, nsm, &pl, &why);
  if (st != PSPEC_OK) return st;
  *bytes = (int64_t)pl.total;
  return PSPEC_OK;
}

pspec_status pspec_create(const pspec_params* p, int32_t device, void* stream, void* workspace, int64_t workspace_bytes,
                          int32_t max_kbins, void** out) {
  if (!out) return PSPEC_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return PSPEC_ECUDA;
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return PSPEC_ECUDA;
  Ctx* c = new Ctx();
  std::string why;
  pspec_status st = build_plan(p, max_kbins, nsm, &c->pl, &why);
  if (st != PSPEC_OK) {
    delete c;
    return st;
  }
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) || workspace_bytes < (int64_t)c->pl.total) {
    const bool small = workspace_bytes < (int64_t)c->pl.total;
    delete c;
    return small ? PSPEC_ENOMEM : PSPEC_EINVAL;
  }
  c->p = *p;
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  c->ws = static_cast<char*>(workspace);
  c->ws_bytes = workspace_bytes;
  c->max_kbins = max_kbins;
  c->nsm = nsm;
  st = c->p.precision == PSPEC_FP64 ? upload_tables<double>(c) : upload_tables<float>(c);
  if (st != PSPEC_OK) {
    delete c;
    return st;
  }
  *out = c;
  return PSPEC_OK;
}

pspec_status pspec_destroy(void* ctx) {
  if (!ctx) return PSPEC_EINVAL;
  Ctx* c = static_cast<Ctx*>(ctx);
  for (auto& r : c->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto ev : c->pool) cudaEventDestroy(ev);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
  return PSPEC_OK;
}

pspec_status pspec_paint(void* ctx, const pspec_catalog* data, const pspec_catalog* randoms, pspec_stats* stats) {
  if (!ctx) return PSPEC_EINVAL;
  Ctx* c = static_cast<Ctx*>(ctx);
  TRY(check_catalog(c, data, "data", false));
  TRY(check_catalog(c, randoms, "randoms", true));
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  pspec_status st = c->p.precision == PSPEC_FP64 ? do_paint<double>(c, data, randoms) : do_paint<float>(c, data, randoms);
  if (st != PSPEC_OK) return st;
  c->painted = true;
  if (stats) {
    double d[D_COUNT];
    e = cudaMemcpyAsync(d, c->at<double>(c->pl.o_derived), sizeof(d), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stats copy");
    stats->alpha = d[D_ALPHA];
    stats->I = d[D_I];
    stats->S = d[D_S];
    stats->W_d = d[D_WD];
    stats->W_r = d[D_WR];
    stats->n_nonfinite = (int64_t)d[D_NONFINITE];
    stats->n_wrapped = (int64_t)d[D_WRAPPED];
    if (stats->n_nonfinite > 0) {
      c->err = "invalid position, weight or nbar in the catalogs";
      c->painted = false;
      return PSPEC_EINVAL;
    }
    if (!(d[D_WR] > 0)) {
      c->err = "randoms completeness weights sum to zero";
      c->painted = false;
      return PSPEC_EINVAL;
    }
  }
  return PSPEC_OK;
}

pspec_status pspec_multipoles_cartesian(void* ctx, const int32_t* ells, int32_t n_ells, const double* k_edges,
                                        int32_t n_kbins, double* P, double* k_mean, double* n_modes) {
  if (!ctx) return PSPEC_EINVAL;
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!P || !k_mean || !n_modes) { c->err = "output pointers are NULL"; return PSPEC_EINVAL; }
  if (!c->pl.has_ctab) { c->err = "context created without cartesian = 1 (or not FP32)"; return PSPEC_EUNSUPPORTED; }
  TRY(check_ells_edges(c, ells, n_ells, k_edges, n_kbins));
  for (int i = 0; i < n_ells; i++)
    if (ells[i] > 4 || (ells[i] & 1)) { c->err = "the Cartesian route covers even l <= 4"; return PSPEC_EUNSUPPORTED; }
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  TRY(upload_bins(c, k_edges, n_kbins));
  double* out = c->at<double>(c->pl.o_out);
  const int nk = n_kbins;
  HRange hr;
  hr.cartesian = true;
  TRY(do_multipoles<float>(c, ells, n_ells, nk, out + 2 * (size_t)nk, out, out + nk, hr));
  std::vector<double> h((size_t)(n_ells + 2) * nk);
  e = cudaMemcpyAsync(h.data(), out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "multipoles");
  std::memcpy(k_mean, h.data(), nk * sizeof(double));
  std::memcpy(n_modes, h.data() + nk, nk * sizeof(double));
  std::memcpy(P, h.data() + 2 * (size_t)nk, (size_t)n_ells * nk * sizeof(double));
  return PSPEC_OK;
}

pspec_status pspec_multipoles(void* ctx, const int32_t* ells, int32_t n_ells, const double* k_edges, int32_t n_kbins,
                              double* P, double* k_mean, double* n_modes) {
  if (!ctx) return PSPEC_EINVAL;
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!P || !k_mean || !n_modes) { c->err = "output pointers are NULL"; return PSPEC_EINVAL; }
  double* out = c->at<double>(c->pl.o_out);
  const int nk = n_kbins;
  TRY(multipoles_common(c, ells, n_ells, k_edges, nk, out + 2 * (size_t)nk, out, out + nk));
  std::vector<double> h((size_t)(n_ells + 2) * nk);
  cudaError_t e = cudaMemcpyAsync(h.data(), out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "multipoles");
  std::memcpy(k_mean, h.data(), nk * sizeof(double));
  std::memcpy(n_modes, h.data() + nk, nk * sizeof(double));
  std::memcpy(P, h.data() + 2 * (size_t)nk, (size_t)n_ells * nk * sizeof(double));
  return PSPEC_OK;
}

pspec_status pspec_multipoles_device(void* ctx, const int32_t* ells, int32_t n_ells, const double* k_edges,
                                     int32_t n_kbins, double* P_dev, double* k_mean_dev, double* n_modes_dev) {
  if (!ctx) return PSPEC_EINVAL;
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!P_dev || !k_mean_dev || !n_modes_dev) { c->err = "output pointers are NULL"; return PSPEC_EINVAL; }
  return multipoles_common(c, ells, n_ells, k_edges, n_kbins, P_dev, k_mean_dev, n_modes_dev);
}

pspec_status pspec_multipoles_range(void* ctx, const int32_t* ells, int32_t n_ells, const double* k_edges,
                                    int32_t n_kbins, int32_t q0, int32_t q1, int32_t include_p0, double* bins) {
  if (!ctx) return PSPEC_EINVAL;
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!bins || q0 < 0 || q1 < q0) { c->err = "bad harmonic range or NULL bins"; return PSPEC_EINVAL; }
  TRY(check_ells_edges(c, ells, n_ells, k_edges, n_kbins));
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  TRY(upload_bins(c, k_edges, n_kbins));
  HRange hr;
  hr.q0 = q0;
  hr.q1 = q1;
  hr.include_p0 = include_p0 != 0;
  hr.bins_out = bins;
  double* out = c->at<double>(c->pl.o_out);
  const int nk = n_kbins;
  if (c->p.precision == PSPEC_FP64)
    return do_multipoles<double>(c, ells, n_ells, nk, out + 2 * (size_t)nk, out, out + nk, hr);
  return do_multipoles<float>(c, ells, n_ells, nk, out + 2 * (size_t)nk, out, out + nk, hr);
}

pspec_status pspec_finalize_bins(void* ctx, const double* bins, const int32_t* ells, int32_t n_ells,
                                 const double* k_edges, int32_t n_kbins, double* P_dev, double* k_mean_dev,
                                 double* n_modes_dev) {
  if (!ctx) return PSPEC_EINVAL;
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!bins || !P_dev || !k_mean_dev || !n_modes_dev) { c->err = "NULL pointer"; return PSPEC_EINVAL; }
  TRY(check_ells_edges(c, ells, n_ells, k_edges, n_kbins));
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  TRY(upload_bins(c, k_edges, n_kbins));
  const Plan& pl = c->pl;
  TRY(run(c, PSPEC_K_FINAL, 0.0, [&] {
    launch_finalize(bins, c->at<double>(pl.o_nmodes), c->at<double>(pl.o_ksum), n_kbins, ells, n_ells,
                    c->at<double>(pl.o_derived), P_dev, k_mean_dev, n_modes_dev, c->stream);
  }));
  return PSPEC_OK;
}

pspec_status pspec_set_randoms(void* ctx, const pspec_catalog* randoms) {
  if (!ctx) return PSPEC_EINVAL;
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c->pl.cache_randoms) { c->err = "context was created without cache_randoms"; return PSPEC_ESTATE; }
  TRY(check_catalog(c, randoms, "randoms", true));
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  pspec_status st = c->p.precision == PSPEC_FP64 ? do_set_randoms<double>(c, randoms) : do_set_randoms<float>(c, randoms);
  if (st != PSPEC_OK) return st;
  c->randoms_set = true;
  return PSPEC_OK;
}

pspec_status pspec_run_batch(void* ctx, const pspec_catalog* mocks, int32_t n_mocks, const int32_t* ells,
                             int32_t n_ells, const double* k_edges, int32_t n_kbins, double* P_all, double* sums_all,
                             double* k_mean, double* n_modes, int32_t use_graph) {
  if (!ctx) return PSPEC_EINVAL;
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c->pl.cache_randoms || !c->randoms_set) { c->err = "pspec_set_randoms must come first"; return PSPEC_ESTATE; }
  if (!mocks || n_mocks < 1 || n_mocks > PSPEC_MAX_BATCH) { c->err = "n_mocks out of range"; return PSPEC_EINVAL; }
  if (!P_all || !k_mean || !n_modes) { c->err = "output pointers are NULL"; return PSPEC_EINVAL; }
  int64_t max_count = 0;
  for (int i = 0; i < n_mocks; i++) {
    TRY(check_catalog(c, &mocks[i], "mock", false));
    if (mocks[i].pos_dtype != mocks[0].pos_dtype) { c->err = "mocks must share one position dtype"; return PSPEC_EINVAL; }
    max_count = std::max(max_count, mocks[i].count);
  }
  c->painted = true;  // the meshes are produced inside the batch sequence
  TRY(check_ells_edges(c, ells, n_ells, k_edges, n_kbins));
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  TRY(upload_bins(c, k_edges, n_kbins));  // synchronous, so before any capture
  const Plan& pl = c->pl;
  c->desc_host.resize(n_mocks);
  for (int i = 0; i < n_mocks; i++) {
    DevCat d;
    d.pos = mocks[i].pos;
    d.weight = mocks[i].weight;
    d.nbar = mocks[i].nbar;
    d.count = mocks[i].count;
    d.pos_f32 = mocks[i].pos_dtype == PSPEC_POS_F32;
    d.pad = 0;
    c->desc_host[i] = d;
  }
  c->batch_proto = mocks[0];
  e = cudaMemcpyAsync(c->at<DevCat>(pl.o_desc), c->desc_host.data(), n_mocks * sizeof(DevCat), cudaMemcpyHostToDevice,
                      c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->at<int>(pl.o_cur), 0, sizeof(int), c->stream);
  // the destinations go through device memory: a graph captured in an earlier call replays into
  // this call's buffers
  c->bout_host = BatchOut{P_all, sums_all};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->at<BatchOut>(pl.o_bout), &c->bout_host, sizeof(BatchOut), cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "batch table upload");
  const bool binned = c->tune.paint_binned && pl.max_particles >= max_count && c->p.precision != PSPEC_FP64;
  const bool f64 = c->p.precision == PSPEC_FP64;
  auto one = [&]() {
    return f64 ? enqueue_mock<double>(c, binned, max_count, ells, n_ells, n_kbins)
               : enqueue_mock<float>(c, binned, max_count, ells, n_ells, n_kbins);
  };
  if (!use_graph) {
    for (int i = 0; i < n_mocks; i++) TRY(one());
  } else {
    // capture and replay on a private stream ordered after, and before, the caller's stream
    if (!c->cap_stream) {
      e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(c, e, "capture stream");
    }
    cudaStream_t user = c->stream;
    cudaEvent_t ev_in = take_event(c), ev_out = take_event(c);
    e = cudaEventRecord(ev_in, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->cap_stream, ev_in, 0);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream ordering");
    c->stream = c->cap_stream;
    struct Restore {
      Ctx* c;
      cudaStream_t user;
      cudaEvent_t ev_in, ev_out;
      ~Restore() {
        cudaEventRecord(ev_out, c->stream);
        c->stream = user;
        cudaStreamWaitEvent(user, ev_out, 0);
        c->pool.push_back(ev_in);
        c->pool.push_back(ev_out);
      }
    } restore{c, user, ev_in, ev_out};
    std::vector<int32_t> ev(ells, ells + n_ells);
    std::vector<double> ed(k_edges, k_edges + n_kbins + 1);
    if (!c->graph || ev != c->graph_ells || ed != c->graph_edges || c->graph_binned != (int)binned) {
      if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
      }
      const bool prof = c->prof;
      c->prof = false;
      const int64_t l0 = c->launches;
      e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed);
      if (e != cudaSuccess) {
        c->prof = prof;
        return cuda_fail(c, e, "begin capture");
      }
      pspec_status st = one();
      cudaGraph_t g = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
      c->prof = prof;
      if (st != PSPEC_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e2 != cudaSuccess) return cuda_fail(c, e2, "end capture");
      e2 = cudaGraphInstantiate(&c->graph, g, 0);
      cudaGraphDestroy(g);
      if (e2 != cudaSuccess) {
        c->graph = nullptr;
        return cuda_fail(c, e2, "graph instantiate");
      }
      c->graph_kernels = c->launches - l0;
      c->launches = l0;
      c->graph_ells = ev;
      c->graph_edges = ed;
      c->graph_binned = (int)binned;
    }
    for (int i = 0; i < n_mocks; i++) {
      e = cudaGraphLaunch(c->graph, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
    }
    c->launches += c->graph_kernels * n_mocks;
  }
  double* out = c->at<double>(pl.o_out);
  e = cudaMemcpyAsync(k_mean, out, n_kbins * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(n_modes, out + n_kbins, n_kbins * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "batch outputs");
  return PSPEC_OK;
}

pspec_status pspec_wedges(const double* P, const int32_t* ells, int32_t n_ells, int32_t n_kbins, const double* mu_edges,
                          int32_t n_mu, double* out, void* stream) {
  if (!P || !ells || !mu_edges || !out) return PSPEC_EINVAL;
  if (n_ells < 1 || n_ells > kMaxElls || n_kbins < 1 || n_mu < 1 || n_mu > PSPEC_MAX_MU) return PSPEC_EINVAL;
  for (int w = 0; w <= n_mu; w++) {
    if (!std::isfinite(mu_edges[w]) || mu_edges[w] < 0.0 || mu_edges[w] > 1.0) return PSPEC_EINVAL;
    if (w && !(mu_edges[w] > mu_edges[w - 1])) return PSPEC_EINVAL;
  }
  for (int i = 0; i < n_ells; i++) {
    if (ells[i] < 0 || ells[i] > PSPEC_MAX_ELL) return PSPEC_EINVAL;
    if (ells[i] & 1) return PSPEC_EUNSUPPORTED;
  }
  // Lbar_l(a, b) = [L_{l+1} - L_{l-1}]_a^b / ((2l+1)(b - a)), Lbar_0 = 1 (Sec. 2.2 eq. Lbar)
  auto legendre = [](int l, double x) {
    if (l == 0) return 1.0;
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= l; k++) {
      const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    return p1;
  };
  WedgeTab t;
  for (int i = 0; i < n_ells; i++) {
    const int l = ells[i];
    for (int w = 0; w < n_mu; w++) {
      const double a = mu_edges[w], b = mu_edges[w + 1];
      double v = 1.0;
      if (l > 0)
        v = ((legendre(l + 1, b) - legendre(l - 1, b)) - (legendre(l + 1, a) - legendre(l - 1, a))) /
            ((2.0 * l + 1.0) * (b - a));
      t.lbar[i * n_mu + w] = v;
    }
  }
  launch_wedges(P, n_ells, n_kbins, n_mu, t, out, static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? PSPEC_OK : PSPEC_ECUDA;
}

pspec_status pspec_get_tuning(void* ctx, pspec_tuning* t) {
  if (!ctx || !t) return PSPEC_EINVAL;
  *t = static_cast<Ctx*>(ctx)->tune;
  return PSPEC_OK;
}

pspec_status pspec_set_tuning(void* ctx, const pspec_tuning* t) {
  if (!ctx || !t) return PSPEC_EINVAL;
  Ctx* c = static_cast<Ctx*>(ctx);
  if (t->paint_binned < 0 || t->paint_binned > 1 || t->ylm_harmonics < 1 || t->ylm_harmonics > 512 ||
      t->bin_blocks_per_sm < 0 || t->bin_blocks_per_sm > 16 || t->tile_y < 0 || t->tile_y > 1) {
    c->err = "tuning value out of range";
    return PSPEC_EINVAL;
  }
  c->tune = *t;
  return PSPEC_OK;
}

pspec_status pspec_autotune(void* ctx, const pspec_catalog* data, const pspec_catalog* randoms, const int32_t* ells,
                            int32_t n_ells, const double* k_edges, int32_t n_kbins, int32_t reps, pspec_tuning* best) {
  if (!ctx || !best) return PSPEC_EINVAL;
  Ctx* c = static_cast<Ctx*>(ctx);
  if (reps < 1) reps = 1;
  double* out = c->at<double>(c->pl.o_out);
  const int nk = n_kbins;
  cudaEvent_t e0 = take_event(c), e1 = take_event(c);
  const bool prof = c->prof;
  c->prof = false;
  // time one configuration: paint + multipoles, `reps` times after one warm-up
  auto measure = [&](const pspec_tuning& t, float* ms) -> pspec_status {
    c->tune = t;
    for (int r = -1; r < reps; r++) {
      if (r == 0) cudaEventRecord(e0, c->stream);
      TRY(pspec_paint(ctx, data, randoms, nullptr));
      TRY(pspec_multipoles_device(ctx, ells, n_ells, k_edges, nk, out + 2 * (size_t)nk, out, out + nk));
    }
    cudaEventRecord(e1, c->stream);
    cudaError_t er = cudaEventSynchronize(e1);
    if (er != cudaSuccess) return cuda_fail(c, er, "autotune");
    cudaEventElapsedTime(ms, e0, e1);
    return PSPEC_OK;
  };
  pspec_tuning cur = c->tune;
  float best_ms = 0.f;
  pspec_status st = measure(cur, &best_ms);
  // coordinate search over the knobs
  const int tz = c->pl.xp ? pass_table<float>(c->p.nmesh)->tz_xp : pass_table<float>(c->p.nmesh)->tz;
  const int hmax = std::max(1, 512 / tz);
  std::vector<std::vector<int>> cand = {
      {1, 0}, {hmax, std::max(1, hmax / 2), std::max(1, hmax / 4)}, {0, 1, 2}, {0, 1}};
  for (int knob = 0; knob < 4 && st == PSPEC_OK; knob++) {
    for (int v : cand[knob]) {
      pspec_tuning t = cur;
      int* f = knob == 0 ? &t.paint_binned : knob == 1 ? &t.ylm_harmonics : knob == 2 ? &t.bin_blocks_per_sm : &t.tile_y;
      if (*f == v) continue;
      *f = v;
      float ms = 0.f;
      st = measure(t, &ms);
      if (st != PSPEC_OK) break;
      if (ms < best_ms) {
        best_ms = ms;
        cur = t;
      }
    }
  }
  c->tune = cur;
  c->prof = prof;
  c->pool.push_back(e0);
  c->pool.push_back(e1);
  *best = cur;
  return st;
}

pspec_status pspec_get_plan_info(void* ctx, pspec_plan_info* info) {
  if (!ctx || !info) return PSPEC_EINVAL;
  Ctx* c = static_cast<Ctx*>(ctx);
  info->nmesh = c->p.nmesh;
  info->precision = c->p.precision;
  info->ell_max = c->p.ell_max;
  info->tile_y = c->pl.tw_y;
  info->tile_x = c->pl.tw_comb;
  info->tile_bin = c->pl.tw_bin;
  info->rows_z = c->pl.rows_z;
  info->group_max = c->pl.group_max;
  info->bin_ctas = c->pl.ctas_bin;
  info->sh_transforms = c->sh_last;
  info->transforms_executed = c->transforms_last;
  info->kernel_launches = c->launches;
  info->model_bytes_last = c->bytes_paint + c->bytes_mult;
  info->ylm_table_bytes = c->pl.has_ytab ? (int64_t)c->pl.ytab_bytes : 0;
  info->ylm_rtable_bytes = c->pl.has_rtab ? (int64_t)c->pl.rtab_bytes : 0;
  info->cartesian_table_bytes = (int64_t)c->pl.ctab_bytes;
  return PSPEC_OK;
}

pspec_status pspec_set_profiling(void* ctx, int32_t enable) {
  if (!ctx) return PSPEC_EINVAL;
  static_cast<Ctx*>(ctx)->prof = enable != 0;
  return PSPEC_OK;
}

pspec_status pspec_kernel_times(void* ctx, int64_t* launches, double* ms, double* bytes) {
  if (!ctx) return PSPEC_EINVAL;
  Ctx* c = static_cast<Ctx*>(ctx);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "kernel times");
  for (auto& r : c->recs) {
    float t = 0.f;
    cudaEventElapsedTime(&t, r.a, r.b);
    c->k_launch[r.k]++;
    c->k_ms[r.k] += t;
    c->k_bytes[r.k] += r.bytes;
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->recs.clear();
  for (int k = 0; k < PSPEC_K_COUNT; k++) {
    if (launches) launches[k] = c->k_launch[k];
    if (ms) ms[k] = c->k_ms[k];
    if (bytes) bytes[k] = c->k_bytes[k];
    c->k_launch[k] = 0;
    c->k_ms[k] = 0;
    c->k_bytes[k] = 0;
  }
  return PSPEC_OK;
}

const char* pspec_kernel_name(int32_t k) {
  static const char* names[PSPEC_K_COUNT] = {"catalog_sums", "paint", "r2c_z", "fft_y", "fft_x", "combine_x",
                                             "ylm_r2c_z", "bin_x", "c2r_z", "finalize", "other"};
  return (k >= 0 && k < PSPEC_K_COUNT) ? names[k] : "unknown";
}

const char* pspec_strerror(pspec_status s) {
  switch (s) {
    case PSPEC_OK: return "ok";
    case PSPEC_EINVAL: return "invalid argument";
    case PSPEC_ENOMEM: return "workspace too small";
    case PSPEC_ECUDA: return "CUDA error";
    case PSPEC_ETIMEOUT: return "device wait timed out";
    case PSPEC_ECANCELED: return "cancelled";
    case PSPEC_EUNSUPPORTED: return "unsupported";
    case PSPEC_ESTATE: return "call out of order";
    default: return "unknown status";
  }
}

const char* pspec_last_error(void* ctx) {
  if (!ctx) return "no context";
  return static_cast<Ctx*>(ctx)->err.c_str();
}

const char* pspec_version(void) { return "libpspec 0.2 sm_103a"; }

}  // extern "C"
