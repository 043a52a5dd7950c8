// Catalog sums, mass assignment, finalisation and wedges of the SH-FFT estimator.
//   a1 catalog sums: Sec. 2.1 eq. FKP-density (alpha, I) and the shot-noise term.
//   a2 painting:     Sec. 2.3 (CIC / TSC kernels, interlaced second mesh at u - 1/2).
//   a6 finalise:     Sec. 2.1 eq. Pell-ours (4 pi / (I N_b) for l >= 2; noise for l = 0).
//   a7 wedges:       Sec. 2.2 eqs. wedge-est and Lbar.
#include <cmath>
#include "launch.h"
#include "intconv.cuh"

namespace pspec {

constexpr int kSumThreads = 256;
// Positions further than this many cells from the corner are invalid (reported with the
// non-finite ones): beyond it the periodic reduction of the grid coordinate loses meaning.
constexpr int kMaxCellsLog2 = 38;  // |u| < 2^38 cells for a valid particle

// Grid coordinate of a position along one axis in units of 2^-24 cell, t = u 2^24 with
// u = (x - corner) N/L in FP64 (the power-of-two scaling is exact). A particle is valid when every
// |t| is below 2^62 (|u| < 2^kMaxCellsLog2 cells; NaN and infinities fail), tested on the exponent
// bits. The test and the conversions (intconv.cuh) use integer instructions: GB300's FP64 pipe is
// narrow, and FP64 compares and conversions between FP64 or FP32 and 64-bit integers all run on it. (One FMA,
// x K - corner K with K = 2^24 N/L, gives the same t but for rare last-bit ties; measured over 30
// axis-permutation draws of the 512^3 survey catalogs, the FP32 results then came out with higher
// median errors, so the two-operation form is kept.)
struct GridMap {
  double c[3], inv;
  __device__ __forceinline__ explicit GridMap(const PaintArgs& a) : inv(a.inv_cell) {
    c[0] = a.corner[0];
    c[1] = a.corner[1];
    c[2] = a.corner[2];
  }
  __device__ __forceinline__ double t(double x, int d) const { return ((x - c[d]) * inv) * 16777216.0; }
};
__device__ __forceinline__ bool grid_ok(double t) { return exp_below(t, kMaxCellsLog2 + 24); }

__device__ __forceinline__ void load_pos(const PaintArgs& a, int64_t p, double& x, double& y, double& z) {
  if (a.pos_f32) {
    const float* q = static_cast<const float*>(a.pos) + 3 * p;
    x = q[0];
    y = q[1];
    z = q[2];
  } else {
    const double* q = static_cast<const double*>(a.pos) + 3 * p;
    x = q[0];
    y = q[1];
    z = q[2];
  }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) r += red[i];
  return r;
}

__device__ __forceinline__ double fkp_w(const PaintArgs& a, double nb) {
  return a.nbar ? (a.P0 > 0.0 ? 1.0 / (1.0 + nb * a.P0) : 1.0) : a.wf_default;
}

// The FP32 mesh value of one particle: v rounded down or up to a neighbouring float, chosen
// by a hash of (particle, catalog) with the probabilities that make its expectation v. All
// particles of a catalog with constant weights share one v; rounded to nearest, its error
// would scale that catalog's whole field, survey window included, and at the lowest k the
// randoms' window exceeds the data-minus-randoms field by two orders of magnitude. Dithered,
// the rounding errors are independent across particles and only add white noise ~1e-7 of the
// shot noise. The hash is the 32-bit finaliser of MurmurHash3 (Appleby) applied to the
// particle index mixed with a per-catalog salt.
struct Dither {
  float lo, hi;    // the two floats around v (equal when v is a float)
  uint32_t thr;    // P(hi) * 2^32
};
__device__ __forceinline__ Dither dither_of(double v) {
  Dither d;
  d.lo = (float)v;
  const double r = v - (double)d.lo;
  d.hi = r == 0.0 ? d.lo : nextafterf(d.lo, r > 0.0 ? INFINITY : -INFINITY);
  const double p = r == 0.0 ? 0.0 : r / ((double)d.hi - (double)d.lo);  // in [0, 1/2]
  d.thr = (uint32_t)(p * 4294967296.0);
  return d;
}
__device__ __forceinline__ uint32_t mix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
__device__ __forceinline__ float dither_pick(const Dither& d, int64_t p, int is_randoms) {
  const uint32_t key = (uint32_t)p ^ ((uint32_t)(p >> 32) * 0x9e3779b9u) ^ (is_randoms ? 0x5bd1e995u : 0u);
  return mix32(key) < d.thr ? d.hi : d.lo;
}
// Catalog fields from the device descriptor of the current mock, when the arguments carry one.
__device__ __forceinline__ PaintArgs resolve(const PaintArgs& in) {
  PaintArgs a = in;
  if (a.dc) {
    const DevCat d = a.dc[*a.cur];
    a.pos = d.pos;
    a.weight = d.weight;
    a.nbar = d.nbar;
    a.count = d.count;
    a.pos_f32 = d.pos_f32;
  }
  return a;
}

// ------------------------------------------------------------------ a1: weighted catalogs
// Per-block partials: [0] sum w_c, [1] sum v^2 (v = w_c w_fkp), [2] sum nbar w_c w_fkp^2,
// [3] sum |v| (bounds every mesh value, for the fixed-point scale of the exact paint).
// Invalid particles are left out here and counted by the paint kernel.
__global__ void __launch_bounds__(kSumThreads) k_catalog_partials(PaintArgs a_in, double* out) {
  __shared__ double red[kSumThreads / 32];
  const PaintArgs a = resolve(a_in);
  const GridMap gm(a);
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.count;
       p += (int64_t)gridDim.x * blockDim.x) {
    double x, y, z;
    load_pos(a, p, x, y, z);
    const double wc = a.weight ? a.weight[p] : 1.0;
    const double nb = a.nbar ? a.nbar[p] : a.nbar_default;
    if (!(grid_ok(gm.t(x, 0)) && grid_ok(gm.t(y, 1)) && grid_ok(gm.t(z, 2)) && isfinite(wc) && isfinite(nb)))
      continue;
    const double wf = fkp_w(a, nb);
    const double v = wc * wf;
    s0 += wc;
    s1 += v * v;
    s2 += nb * wc * wf * wf;
    s3 += fabs(v);
  }
  const double r0 = block_sum(s0, red);
  const double r1 = block_sum(s1, red);
  const double r2 = block_sum(s2, red);
  const double r3 = block_sum(s3, red);
  if (threadIdx.x == 0) {
    double* o = out + (int64_t)blockIdx.x * kSumVals;
    o[0] = r0;
    o[1] = r1;
    o[2] = r2;
    o[3] = r3;
  }
}

// Neumaier-compensated FP64 accumulator (the block partials are few).
struct Neu {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    const double t = s + x;
    c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double val() const { return s + c; }
};

// The fixed-point scale 2^S of the exact paint for meshes whose values are all bounded by
// `bound` in magnitude: every cell sum then stays below 2^61 in units of 2^-S.
__device__ double fix_scale(double bound) {
  int e = 0;
  frexp(bound, &e);  // bound < 2^e
  int S = bound > 0.0 ? 61 - e : 61;
  S = S > 100 ? 100 : (S < -100 ? -100 : S);
  return ldexp(1.0, S);
}

// One thread adds the block partials in a fixed order: deterministic alpha, I, S. `fix`
// (nullable) receives the exact paint's fixed-point scale for data (+v) and randoms
// (-alpha v) painted together.
__global__ void k_catalog_final(const double* pd, int nbd, const double* pr, int nbr, double* d, double* fix) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Neu wd, sd, wr, sr, ir;
  double ad = 0.0, ar = 0.0;
  for (int b = 0; b < nbd; b++) {
    wd.add(pd[b * kSumVals + 0]);
    sd.add(pd[b * kSumVals + 1]);
    ad += pd[b * kSumVals + 3];
  }
  for (int b = 0; b < nbr; b++) {
    wr.add(pr[b * kSumVals + 0]);
    sr.add(pr[b * kSumVals + 1]);
    ir.add(pr[b * kSumVals + 2]);
    ar += pr[b * kSumVals + 3];
  }
  const double alpha = wd.val() / wr.val();
  d[D_WD] = wd.val();
  d[D_WR] = wr.val();
  d[D_ALPHA] = alpha;
  d[D_I] = alpha * ir.val();
  d[D_S] = sd.val() + alpha * alpha * sr.val();
  d[D_NONFINITE] = 0.0;
  d[D_WRAPPED] = 0.0;
  d[D_SD] = sd.val();
  d[D_SR] = sr.val();
  d[D_IR] = ir.val();
  if (fix) *fix = fix_scale(ad + fabs(alpha) * ar);
}

// Unit completeness weights and one n̄: W = counts, v = w_fkp for every particle.
__global__ void k_derive_uniform(int64_t nd, int64_t nr, double wf, double nbar, double* d) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double Wd = (double)nd, Wr = (double)nr;
  const double alpha = Wd / Wr;
  const double sd = Wd * wf * wf, sr = Wr * wf * wf, ir = Wr * nbar * wf * wf;
  d[D_WD] = Wd;
  d[D_WR] = Wr;
  d[D_ALPHA] = alpha;
  d[D_I] = alpha * ir;
  d[D_S] = sd + alpha * alpha * sr;
  d[D_NONFINITE] = 0.0;
  d[D_WRAPPED] = 0.0;
  d[D_SD] = sd;
  d[D_SR] = sr;
  d[D_IR] = ir;
  d[D_FIX] = fix_scale(fabs(wf) * (Wd + alpha * Wr));
}

void launch_catalog_partials(const PaintArgs& a, double* partials, int nblocks, cudaStream_t s) {
  k_catalog_partials<<<nblocks, kSumThreads, 0, s>>>(a, partials);
}

void launch_catalog_final(const double* part_d, int nb_d, const double* part_r, int nb_r, double* derived,
                          cudaStream_t s, double* fix) {
  k_catalog_final<<<1, 32, 0, s>>>(part_d, nb_d, part_r, nb_r, derived, fix);
}

void launch_derive_uniform(int64_t n_d, int64_t n_r, double wf, double nbar, double* derived, cudaStream_t s) {
  k_derive_uniform<<<1, 32, 0, s>>>(n_d, n_r, wf, nbar, derived);
}

// ------------------------------------------------------------------ a2: painting
__device__ __forceinline__ int wrap(int64_t i, int N) {
  if (i >= 0 && i < N) return (int)i;
  const int r = (int)(i % N);
  return r < 0 ? r + N : r;
}

// One axis of the assignment kernel. FP32 meshes use a 24-bit fixed-point grid coordinate
// U = round(u 2^24) (u computed in FP64), so the cell index is U >> 24 and the fraction is
// exact in FP32; FP64 meshes keep u in FP64. Fills the node indices (wrapped into [0, N))
// and the weights.
template <typename T, int WIN> struct Axis;

template <int WIN> struct Axis<float, WIN> {
  static __device__ __forceinline__ void nodes(int64_t U, int N, int* idx, float* w) {
    if (WIN == PSPEC_WINDOW_CIC) {
      const int64_t c = U >> 24;
      const float d = (float)(U - c * 16777216ll) * 5.9604644775390625e-8f;  // 2^-24
      w[0] = 1.f - d;
      w[1] = d;
      idx[0] = wrap(c, N);
      idx[1] = wrap(c + 1, N);
    } else {
      const int64_t c = (U + (1ll << 23)) >> 24;  // floor(u + 1/2)
      const float d = (float)(U - c * 16777216ll) * 5.9604644775390625e-8f;  // in [-1/2, 1/2)
      w[0] = 0.5f * (0.5f - d) * (0.5f - d);
      w[1] = 0.75f - d * d;
      w[2] = 0.5f * (0.5f + d) * (0.5f + d);
      idx[0] = wrap(c - 1, N);
      idx[1] = wrap(c, N);
      idx[2] = wrap(c + 1, N);
    }
  }
};

template <int WIN> struct Axis<double, WIN> {
  static __device__ __forceinline__ void nodes(double u, int N, int* idx, double* w) {
    if (WIN == PSPEC_WINDOW_CIC) {
      const double f = floor(u);
      const double d = u - f;
      const int64_t c = (int64_t)f;
      w[0] = 1.0 - d;
      w[1] = d;
      idx[0] = wrap(c, N);
      idx[1] = wrap(c + 1, N);
    } else {
      const double f = floor(u + 0.5);
      const double d = u - f;
      const int64_t c = (int64_t)f;
      w[0] = 0.5 * (0.5 - d) * (0.5 - d);
      w[1] = 0.75 - d * d;
      w[2] = 0.5 * (0.5 + d) * (0.5 + d);
      idx[0] = wrap(c - 1, N);
      idx[1] = wrap(c, N);
      idx[2] = wrap(c + 1, N);
    }
  }
};

template <typename T, int WIN>
__device__ __forceinline__ void scatter(T* __restrict__ m, int N, const int (&ix)[3], const int (&iy)[3],
                                        const int (&iz)[3], const T (&wx)[3], const T (&wy)[3], const T (&wz)[3],
                                        T v) {
  constexpr int K = WIN == PSPEC_WINDOW_CIC ? 2 : 3;
#pragma unroll
  for (int a = 0; a < K; a++) {
    const T va = v * wx[a];
#pragma unroll
    for (int b = 0; b < K; b++) {
      const T vb = va * wy[b];
      T* row = m + ((int64_t)ix[a] * N + iy[b]) * N;
#pragma unroll
      for (int c = 0; c < K; c++) atomicAdd(row + iz[c], vb * wz[c]);
    }
  }
}

template <typename T, int WIN, bool INTER>
__global__ void __launch_bounds__(256) k_paint(PaintArgs a_in, int is_randoms, double* __restrict__ derived,
                                               T* __restrict__ m1, T* __restrict__ m2, int N) {
  const PaintArgs a = resolve(a_in);
  const double sign = is_randoms == 1 ? -derived[D_ALPHA] : 1.0;
  const bool uniform = (a.weight == nullptr) && (a.nbar == nullptr);
  const double v_uniform = sign * a.wf_default;
  const Dither d_uniform = dither_of(v_uniform);
  const GridMap gm(a);
  const int64_t lim24 = (int64_t)N << 24;
  unsigned bad = 0, out = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.count;
       p += (int64_t)gridDim.x * blockDim.x) {
    double x, y, z;
    load_pos(a, p, x, y, z);
    double wc = 1.0, nb = a.nbar_default;
    if (!uniform) {
      wc = a.weight ? a.weight[p] : 1.0;
      nb = a.nbar ? a.nbar[p] : a.nbar_default;
    }
    const double tx = gm.t(x, 0), ty = gm.t(y, 1), tz = gm.t(z, 2);
    if (!(grid_ok(tx) && grid_ok(ty) && grid_ok(tz) && (uniform || (isfinite(wc) && isfinite(nb))))) {
      bad++;
      continue;
    }
    T v;
    if constexpr (sizeof(T) == 4)
      v = dither_pick(uniform ? d_uniform : dither_of(sign * wc * fkp_w(a, nb)), p, is_randoms);
    else
      v = sign * wc * fkp_w(a, nb);
    int ix[3], iy[3], iz[3];
    T wx[3], wy[3], wz[3];
    if constexpr (sizeof(T) == 4) {
      const int64_t Ux = d2ll_rn_int(tx), Uy = d2ll_rn_int(ty), Uz = d2ll_rn_int(tz);
      if (Ux < 0 || Ux >= lim24 || Uy < 0 || Uy >= lim24 || Uz < 0 || Uz >= lim24) out++;
      Axis<float, WIN>::nodes(Ux, N, ix, wx);
      Axis<float, WIN>::nodes(Uy, N, iy, wy);
      Axis<float, WIN>::nodes(Uz, N, iz, wz);
      scatter<T, WIN>(m1, N, ix, iy, iz, wx, wy, wz, v);
      if (INTER) {
        const int64_t h = 1ll << 23;  // half a cell
        Axis<float, WIN>::nodes(Ux - h, N, ix, wx);
        Axis<float, WIN>::nodes(Uy - h, N, iy, wy);
        Axis<float, WIN>::nodes(Uz - h, N, iz, wz);
        scatter<T, WIN>(m2, N, ix, iy, iz, wx, wy, wz, v);
      }
    } else {
      const double ux = tx * 5.9604644775390625e-8, uy = ty * 5.9604644775390625e-8,
                   uz = tz * 5.9604644775390625e-8;  // 2^-24: exact
      const double lim = (double)N;
      if (ux < 0.0 || ux >= lim || uy < 0.0 || uy >= lim || uz < 0.0 || uz >= lim) out++;
      Axis<double, WIN>::nodes(ux, N, ix, wx);
      Axis<double, WIN>::nodes(uy, N, iy, wy);
      Axis<double, WIN>::nodes(uz, N, iz, wz);
      scatter<T, WIN>(m1, N, ix, iy, iz, wx, wy, wz, v);
      if (INTER) {
        Axis<double, WIN>::nodes(ux - 0.5, N, ix, wx);
        Axis<double, WIN>::nodes(uy - 0.5, N, iy, wy);
        Axis<double, WIN>::nodes(uz - 0.5, N, iz, wz);
        scatter<T, WIN>(m2, N, ix, iy, iz, wx, wy, wz, v);
      }
    }
  }
  // rare events: one atomic per warp that saw any
  const unsigned nb_w = __reduce_add_sync(0xffffffffu, bad);
  const unsigned no_w = __reduce_add_sync(0xffffffffu, out);
  if ((threadIdx.x & 31) == 0) {
    if (nb_w) atomicAdd(&derived[D_NONFINITE], (double)nb_w);
    if (no_w) atomicAdd(&derived[D_WRAPPED], (double)no_w);
  }
}

template <typename T>
void launch_paint(const PaintArgs& a, int window, int interlaced, int is_randoms, double* derived, T* mesh1, T* mesh2,
                  int N, int nblocks, cudaStream_t s) {
  if (!a.dc && a.count <= 0) return;
  const int64_t need = a.dc ? nblocks : (a.count + 255) / 256;
  const int nb = (int)(need < nblocks ? need : nblocks);
  if (window == PSPEC_WINDOW_CIC) {
    if (interlaced)
      k_paint<T, PSPEC_WINDOW_CIC, true><<<nb, 256, 0, s>>>(a, is_randoms, derived, mesh1, mesh2, N);
    else
      k_paint<T, PSPEC_WINDOW_CIC, false><<<nb, 256, 0, s>>>(a, is_randoms, derived, mesh1, mesh2, N);
  } else {
    if (interlaced)
      k_paint<T, PSPEC_WINDOW_TSC, true><<<nb, 256, 0, s>>>(a, is_randoms, derived, mesh1, mesh2, N);
    else
      k_paint<T, PSPEC_WINDOW_TSC, false><<<nb, 256, 0, s>>>(a, is_randoms, derived, mesh1, mesh2, N);
  }
}
template void launch_paint<float>(const PaintArgs&, int, int, int, double*, float*, float*, int, int, cudaStream_t);
template void launch_paint<double>(const PaintArgs&, int, int, int, double*, double*, double*, int, int,
                                   cudaStream_t);

// ------------------------------------------------------------------ a2: tile-binned painting
// FP32 meshes, accumulated exactly. One block per 16^3-cell tile owns its cells: it sums every
// contribution that lands in them as a 64-bit fixed-point integer (units 2^-S, S from the
// catalogs' sum of |v| so that no sum can overflow) and stores each cell once, rounded to FP32.
// Integer sums do not depend on the order of the additions, so the meshes are the exact sums of
// the particles' FP32 contributions, rounded once, identical from run to run. With FP32 atomics
// instead, each run adds in another order, and the rounding of the many small randoms
// contributions left an order-dependent error on the survey window's largest-scale modes large
// enough to move a 3%-of-P_0 quadrupole in the first k bin by ~1e-5.
//
// A particle whose footprint (both interlaced meshes) crosses a tile face is listed for every
// tile it touches: per axis the footprint spans at most 4 cells, so at most 2 tiles per axis.
// Record: per axis the grid coordinate relative to the origin of the particle's first tile,
// in 2^-24 cells (29 bits), with bit 31 set when the footprint reaches the next tile; in the
// tile-sorted copy bit 29 says the record sits in that next tile (coordinate 16 cells less).
constexpr int kPT = 16;  // tile side (cells)
constexpr int kPT3 = kPT * kPT * kPT;
constexpr unsigned kNoTile = 0xffffffffu;
constexpr unsigned kCoordMask = (1u << 29) - 1u;
constexpr unsigned kSpan2 = 1u << 31;
constexpr unsigned kNextTile = 1u << 29;

// Lowest and highest footprint cell along one axis (unwrapped), both meshes.
template <int WIN, bool INTER>
__device__ __forceinline__ void footprint(int64_t U, int64_t& lo, int64_t& hi) {
  if (WIN == PSPEC_WINDOW_CIC) {
    const int64_t c1 = U >> 24;
    lo = INTER ? ((U - (1ll << 23)) >> 24) : c1;
    hi = c1 + 1;
  } else {
    const int64_t c1 = (U + (1ll << 23)) >> 24;  // floor(u + 1/2)
    const int64_t c2 = U >> 24;                   // centre of the mesh painted at u - 1/2
    lo = (INTER ? (c1 < c2 ? c1 : c2) : c1) - 1;
    hi = (INTER ? (c1 > c2 ? c1 : c2) : c1) + 1;
  }
}

template <int WIN, bool INTER>
__global__ void __launch_bounds__(256) k_ptile_prep(PaintArgs a_in, int is_randoms, double* __restrict__ derived,
                                                    TileArgs ta, int64_t offset, int N) {
  const PaintArgs a = resolve(a_in);
  const double sign = is_randoms == 1 ? -derived[D_ALPHA] : 1.0;
  const bool uniform = (a.weight == nullptr) && (a.nbar == nullptr);
  const double v_uniform = sign * a.wf_default;
  const Dither d_uniform = dither_of(v_uniform);
  const GridMap gm(a);
  const int64_t lim24 = (int64_t)N << 24;
  const int nts = N / kPT;
  unsigned bad = 0, out = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.count;
       p += (int64_t)gridDim.x * blockDim.x) {
    double x, y, z;
    load_pos(a, p, x, y, z);
    double wc = 1.0, nb = a.nbar_default;
    if (!uniform) {
      wc = a.weight ? a.weight[p] : 1.0;
      nb = a.nbar ? a.nbar[p] : a.nbar_default;
    }
    const double tt[3] = {gm.t(x, 0), gm.t(y, 1), gm.t(z, 2)};
    if (!(grid_ok(tt[0]) && grid_ok(tt[1]) && grid_ok(tt[2]) && (uniform || (isfinite(wc) && isfinite(nb))))) {
      bad++;
      ta.tile_of[offset + p] = kNoTile;
      continue;
    }
    const int64_t Ud[3] = {d2ll_rn_int(tt[0]), d2ll_rn_int(tt[1]), d2ll_rn_int(tt[2])};
    if (Ud[0] < 0 || Ud[0] >= lim24 || Ud[1] < 0 || Ud[1] >= lim24 || Ud[2] < 0 || Ud[2] >= lim24) out++;
    const float v = dither_pick(uniform ? d_uniform : dither_of(sign * wc * fkp_w(a, nb)), p, is_randoms);
    unsigned packed[3];
    int tb[3], span[3];
    for (int d = 0; d < 3; d++) {
      const int64_t U = Ud[d];
      int64_t lo, hi;
      footprint<WIN, INTER>(U, lo, hi);
      const int low = wrap(lo, N);  // the footprint's first cell, wrapped; U shifted by the same period
      tb[d] = low / kPT;
      const int64_t rel = U - (lo - low + (int64_t)tb[d] * kPT) * 16777216ll;  // in [0, 19 cells)
      span[d] = (low - tb[d] * kPT) + (int)(hi - lo) >= kPT ? 2 : 1;
      packed[d] = (unsigned)rel | (span[d] == 2 ? kSpan2 : 0u);
    }
    const unsigned tile = (unsigned)((tb[0] * nts + tb[1]) * nts + tb[2]);
    ta.rec[offset + p] = make_uint4(packed[0], packed[1], packed[2], __float_as_uint(v));
    ta.tile_of[offset + p] = tile;
    for (int dx = 0; dx < span[0]; dx++)
      for (int dy = 0; dy < span[1]; dy++)
        for (int dz = 0; dz < span[2]; dz++) {
          const int t = ((((tb[0] + dx) % nts) * nts + (tb[1] + dy) % nts) * nts) + (tb[2] + dz) % nts;
          atomicAdd(&ta.cnt[t], 1u);
        }
  }
  const unsigned nb_w = __reduce_add_sync(0xffffffffu, bad);
  const unsigned no_w = __reduce_add_sync(0xffffffffu, out);
  if ((threadIdx.x & 31) == 0) {
    if (nb_w) atomicAdd(&derived[D_NONFINITE], (double)nb_w);
    if (no_w) atomicAdd(&derived[D_WRAPPED], (double)no_w);
  }
}

// Exclusive prefix sum of the tile counts (one block): off[] and cursor[].
__global__ void __launch_bounds__(1024) k_ptile_scan(TileArgs ta, int ntiles) {
  __shared__ unsigned part[1024];
  const int per = (ntiles + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per;
  unsigned s = 0;
  for (int i = b0; i < b0 + per && i < ntiles; i++) s += ta.cnt[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    const unsigned add = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += add;
    __syncthreads();
  }
  unsigned run = part[threadIdx.x] - s;
  for (int i = b0; i < b0 + per && i < ntiles; i++) {
    ta.off[i] = run;
    ta.cursor[i] = run;
    run += ta.cnt[i];
  }
}

// Each record goes to every tile its footprint touches (the order within a tile is free: the
// tile's sums are exact).
__global__ void __launch_bounds__(256) k_ptile_scatter(TileArgs ta, int64_t total, const DevCat* dc, const int* cur,
                                                       int N) {
  if (dc) total = dc[*cur].count;
  const int nts = N / kPT;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
    const unsigned t = ta.tile_of[p];
    if (t == kNoTile) continue;
    const uint4 r = ta.rec[p];
    const int tb[3] = {(int)(t / (nts * nts)), (int)((t / nts) % nts), (int)(t % nts)};
    const int sx = (r.x & kSpan2) ? 2 : 1, sy = (r.y & kSpan2) ? 2 : 1, sz = (r.z & kSpan2) ? 2 : 1;
    for (int dx = 0; dx < sx; dx++)
      for (int dy = 0; dy < sy; dy++)
        for (int dz = 0; dz < sz; dz++) {
          const int tt = ((((tb[0] + dx) % nts) * nts + (tb[1] + dy) % nts) * nts) + (tb[2] + dz) % nts;
          const unsigned pos = atomicAdd(&ta.cursor[tt], 1u);
          ta.sorted[pos] = make_uint4((r.x & kCoordMask) | (dx ? kNextTile : 0u),
                                      (r.y & kCoordMask) | (dy ? kNextTile : 0u),
                                      (r.z & kCoordMask) | (dz ? kNextTile : 0u), r.w);
        }
  }
}

// Tile-local node indices (may fall outside [0, kPT): not this tile's) and weights along one
// axis from the tile-local grid coordinate V (2^24 per cell).
template <int WIN>
__device__ __forceinline__ void tile_nodes(int V, int* idx, float* w) {
  if (WIN == PSPEC_WINDOW_CIC) {
    const int c = V >> 24;
    const float d = (float)(V - c * 16777216) * 5.9604644775390625e-8f;
    w[0] = 1.f - d;
    w[1] = d;
    idx[0] = c;
    idx[1] = c + 1;
  } else {
    const int c = (V + (1 << 23)) >> 24;
    const float d = (float)(V - c * 16777216) * 5.9604644775390625e-8f;
    w[0] = 0.5f * (0.5f - d) * (0.5f - d);
    w[1] = 0.75f - d * d;
    w[2] = 0.5f * (0.5f + d) * (0.5f + d);
    idx[0] = c - 1;
    idx[1] = c;
    idx[2] = c + 1;
  }
}

__device__ __forceinline__ bool in_tile(int i) { return (unsigned)i < (unsigned)kPT; }

// Adds the 64-bit integer q into the cell's sum held as two 32-bit words (lo at acc[c], hi at
// acc[c + hi_off]) with 32-bit shared atomics: lo wraps modulo 2^32, and each add that wraps it
// (the returned old value shows it) carries 1 into hi, so hi:lo is the exact sum modulo 2^64 in
// any order. The hi add is skipped when it adds 0 (small q, or a small negative q that carried).
__device__ __forceinline__ void add64(unsigned* acc, int c, int hi_off, long long q) {
  const unsigned long long u = (unsigned long long)q;
  const unsigned lo = (unsigned)u, hi = (unsigned)(u >> 32);
  const unsigned old = atomicAdd(acc + c, lo);
  const unsigned h = hi + (old + lo < old ? 1u : 0u);
  if (h) atomicAdd(acc + c + hi_off, h);
}

// The contribution v wx wy wz (FP32, rounded as the direct paint rounds it) in units of 2^-S.
template <int WIN>
__device__ __forceinline__ void tile_scatter(unsigned* acc, int hi_off, const int (&ix)[3], const int (&iy)[3],
                                             const int (&iz)[3], const float (&wx)[3], const float (&wy)[3],
                                             const float (&wz)[3], float v, float scale) {
  constexpr int K = WIN == PSPEC_WINDOW_CIC ? 2 : 3;
#pragma unroll
  for (int a = 0; a < K; a++) {
    if (!in_tile(ix[a])) continue;
    const float va = v * wx[a];
#pragma unroll
    for (int b = 0; b < K; b++) {
      if (!in_tile(iy[b])) continue;
      const float vb = va * wy[b];
      const int row = (ix[a] * kPT + iy[b]) * kPT;
#pragma unroll
      for (int c = 0; c < K; c++) {
        if (!in_tile(iz[c])) continue;
        add64(acc, row + iz[c], hi_off, f2ll_rn_int((vb * wz[c]) * scale));
      }
    }
  }
}

// One block per tile (every tile, so that empty tiles store their zeros): sums its records into
// shared 64-bit accumulators (lo words of both meshes, then hi words), then stores each cell of
// the tile once, four cells along z per 16-byte store. A tile without records stores zeros and
// skips the accumulators.
template <int WIN, bool INTER>
__global__ void __launch_bounds__(256) k_ptile_paint(TileArgs ta, float* __restrict__ m1, float* __restrict__ m2,
                                                     int N, const double* __restrict__ fix) {
  extern __shared__ __align__(16) unsigned acc[];  // lo [NM][kPT^3], then hi [NM][kPT^3]
  constexpr int NM = INTER ? 2 : 1;
  constexpr int HI = NM * kPT3;
  const int tile = blockIdx.x;
  const unsigned n = ta.cnt[tile];
  const unsigned o = ta.off[tile];
  const int nts = N / kPT;
  const int tz = tile % nts, ty = (tile / nts) % nts, tx = tile / (nts * nts);
  // 16-byte group i of the tile: mesh, then cells (lx, ly, lz..lz+3); its mesh address
  auto group = [&](int i, int& mesh) {
    mesh = i / (kPT3 / 4);
    const int cell = (i - mesh * (kPT3 / 4)) * 4;
    const int lx = cell / (kPT * kPT), ly = (cell / kPT) % kPT, lz = cell % kPT;
    return ((int64_t)(tx * kPT + lx) * N + (ty * kPT + ly)) * N + tz * kPT + lz;
  };
  if (n == 0) {
    for (int i = threadIdx.x; i < NM * kPT3 / 4; i += blockDim.x) {
      int mesh;
      const int64_t g = group(i, mesh);
      *reinterpret_cast<float4*>((mesh ? m2 : m1) + g) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    return;  // uniform over the block: no barrier is left behind
  }
  const double sc = *fix;
  const float scale = (float)sc, inv = (float)(1.0 / sc);  // powers of two: exact
  for (int i = threadIdx.x; i < 2 * NM * kPT3 / 4; i += blockDim.x) reinterpret_cast<uint4*>(acc)[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  for (unsigned q = threadIdx.x; q < n; q += blockDim.x) {
    const uint4 r = ta.sorted[o + q];
    const float v = __uint_as_float(r.w);
    const int V[3] = {(int)(r.x & kCoordMask) - ((r.x & kNextTile) ? (kPT << 24) : 0),
                      (int)(r.y & kCoordMask) - ((r.y & kNextTile) ? (kPT << 24) : 0),
                      (int)(r.z & kCoordMask) - ((r.z & kNextTile) ? (kPT << 24) : 0)};
    int ix[3], iy[3], iz[3];
    float wx[3], wy[3], wz[3];
    tile_nodes<WIN>(V[0], ix, wx);
    tile_nodes<WIN>(V[1], iy, wy);
    tile_nodes<WIN>(V[2], iz, wz);
    tile_scatter<WIN>(acc, HI, ix, iy, iz, wx, wy, wz, v, scale);
    if (INTER) {
      const int h = 1 << 23;  // half a cell
      tile_nodes<WIN>(V[0] - h, ix, wx);
      tile_nodes<WIN>(V[1] - h, iy, wy);
      tile_nodes<WIN>(V[2] - h, iz, wz);
      tile_scatter<WIN>(acc + kPT3, HI, ix, iy, iz, wx, wy, wz, v, scale);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NM * kPT3 / 4; i += blockDim.x) {
    int mesh;
    const int64_t g = group(i, mesh);
    const uint4 lo = reinterpret_cast<const uint4*>(acc)[i], hi = reinterpret_cast<const uint4*>(acc + HI)[i];
    auto cell = [&](unsigned l, unsigned h) {
      return ll2f_rn_int((long long)(((unsigned long long)h << 32) | l)) * inv;
    };
    *reinterpret_cast<float4*>((mesh ? m2 : m1) + g) =
        make_float4(cell(lo.x, hi.x), cell(lo.y, hi.y), cell(lo.z, hi.z), cell(lo.w, hi.w));
  }
}

void launch_ptile_prep(const PaintArgs& a, int window, int interlaced, int is_randoms, double* derived,
                       const TileArgs& ta, int64_t offset, int N, int nblocks, cudaStream_t s) {
  if (!a.dc && a.count <= 0) return;
  const int64_t need = a.dc ? nblocks : (a.count + 255) / 256;
  const int nb = (int)(need < nblocks ? need : nblocks);
  if (window == PSPEC_WINDOW_CIC) {
    if (interlaced)
      k_ptile_prep<PSPEC_WINDOW_CIC, true><<<nb, 256, 0, s>>>(a, is_randoms, derived, ta, offset, N);
    else
      k_ptile_prep<PSPEC_WINDOW_CIC, false><<<nb, 256, 0, s>>>(a, is_randoms, derived, ta, offset, N);
  } else {
    if (interlaced)
      k_ptile_prep<PSPEC_WINDOW_TSC, true><<<nb, 256, 0, s>>>(a, is_randoms, derived, ta, offset, N);
    else
      k_ptile_prep<PSPEC_WINDOW_TSC, false><<<nb, 256, 0, s>>>(a, is_randoms, derived, ta, offset, N);
  }
}

void launch_ptile_scan(const TileArgs& ta, int ntiles, cudaStream_t s) { k_ptile_scan<<<1, 1024, 0, s>>>(ta, ntiles); }

void launch_ptile_scatter(const TileArgs& ta, int64_t total, const DevCat* dc, const int* cur, int N, int nblocks,
                          cudaStream_t s) {
  if (!dc && total <= 0) return;
  const int64_t need = dc ? nblocks : (total + 255) / 256;
  const int nb = (int)(need < nblocks ? need : nblocks);
  k_ptile_scatter<<<nb, 256, 0, s>>>(ta, total, dc, cur, N);
}

template <typename K> static void set_smem_attr(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

void launch_ptile_paint(const TileArgs& ta, int window, int interlaced, float* m1, float* m2, int N,
                        const double* fix, cudaStream_t s) {
  const int ntiles = (N / kPT) * (N / kPT) * (N / kPT);
  const size_t smem = (size_t)(interlaced ? 2 : 1) * kPT3 * sizeof(unsigned long long);
  if (window == PSPEC_WINDOW_CIC) {
    if (interlaced) {
      set_smem_attr(k_ptile_paint<PSPEC_WINDOW_CIC, true>, smem);
      k_ptile_paint<PSPEC_WINDOW_CIC, true><<<ntiles, 256, smem, s>>>(ta, m1, m2, N, fix);
    } else {
      k_ptile_paint<PSPEC_WINDOW_CIC, false><<<ntiles, 256, smem, s>>>(ta, m1, m2, N, fix);
    }
  } else {
    if (interlaced) {
      set_smem_attr(k_ptile_paint<PSPEC_WINDOW_TSC, true>, smem);
      k_ptile_paint<PSPEC_WINDOW_TSC, true><<<ntiles, 256, smem, s>>>(ta, m1, m2, N, fix);
    } else {
      k_ptile_paint<PSPEC_WINDOW_TSC, false><<<ntiles, 256, smem, s>>>(ta, m1, m2, N, fix);
    }
  }
}

// ------------------------------------------------------------------ batched mocks
// rsums = (W_r, S_r, I_r, fixed-point scale of the randoms mesh painted alone) of the cached randoms.
__global__ void k_randoms_sums(const double* pr, int nbr, double* rsums) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Neu wr, sr, ir;
  double ar = 0.0;
  for (int b = 0; b < nbr; b++) {
    wr.add(pr[b * kSumVals + 0]);
    sr.add(pr[b * kSumVals + 1]);
    ir.add(pr[b * kSumVals + 2]);
    ar += pr[b * kSumVals + 3];
  }
  rsums[0] = wr.val();
  rsums[1] = sr.val();
  rsums[2] = ir.val();
  rsums[3] = fix_scale(ar);
}

__global__ void k_catalog_final_cached(const double* pd, int nbd, const double* rsums, double* d) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Neu wd, sd;
  double ad = 0.0;
  for (int b = 0; b < nbd; b++) {
    wd.add(pd[b * kSumVals + 0]);
    sd.add(pd[b * kSumVals + 1]);
    ad += pd[b * kSumVals + 3];
  }
  const double Wr = rsums[0], Sr = rsums[1], Ir = rsums[2];
  const double alpha = wd.val() / Wr;
  d[D_WD] = wd.val();
  d[D_WR] = Wr;
  d[D_ALPHA] = alpha;
  d[D_I] = alpha * Ir;
  d[D_S] = sd.val() + alpha * alpha * Sr;
  d[D_NONFINITE] = 0.0;
  d[D_WRAPPED] = 0.0;
  d[D_SD] = sd.val();
  d[D_SR] = Sr;
  d[D_IR] = Ir;
  d[D_FIX] = fix_scale(ad);  // the mock's data mesh is painted alone
}

template <typename T>
__global__ void k_axpy_randoms(T* __restrict__ m, const T* __restrict__ r, int64_t n, const double* __restrict__ d) {
  const T a = (T)d[D_ALPHA];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m[i] -= a * r[i];
}

__global__ void k_batch_outputs(const double* __restrict__ P, int n, const double* __restrict__ d,
                                const int* __restrict__ cur, const BatchOut* __restrict__ bo) {
  const int c = *cur;
  double* P_all = bo->P_all;
  double* sums_all = bo->sums_all;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    P_all[(int64_t)c * n + i] = P[i];
  if (blockIdx.x == 0 && threadIdx.x == 0 && sums_all) {
    sums_all[4 * c + 0] = d[D_ALPHA];
    sums_all[4 * c + 1] = d[D_I];
    sums_all[4 * c + 2] = d[D_S];
    sums_all[4 * c + 3] = d[D_WD];
  }
}

__global__ void k_advance(int* cur) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *cur += 1;
}

void launch_randoms_sums(const double* part_r, int nb_r, double* rsums, cudaStream_t s) {
  k_randoms_sums<<<1, 32, 0, s>>>(part_r, nb_r, rsums);
}
void launch_catalog_final_cached(const double* part_d, int nb_d, const double* rsums, double* derived,
                                 cudaStream_t s) {
  k_catalog_final_cached<<<1, 32, 0, s>>>(part_d, nb_d, rsums, derived);
}
void launch_axpy_randoms(float* mesh, const float* rmesh, int64_t n, const double* derived, cudaStream_t s) {
  k_axpy_randoms<float><<<2048, 256, 0, s>>>(mesh, rmesh, n, derived);
}
void launch_axpy_randoms(double* mesh, const double* rmesh, int64_t n, const double* derived, cudaStream_t s) {
  k_axpy_randoms<double><<<2048, 256, 0, s>>>(mesh, rmesh, n, derived);
}
void launch_batch_outputs(const double* P, int n_ells, int nk, const double* derived, const int* cur,
                          const BatchOut* out, cudaStream_t s) {
  k_batch_outputs<<<(n_ells * nk + 127) / 128, 128, 0, s>>>(P, n_ells * nk, derived, cur, out);
}
void launch_advance(int* cur, cudaStream_t s) { k_advance<<<1, 32, 0, s>>>(cur); }

// ------------------------------------------------------------------ a6: finalise
struct EllList {
  int n;
  int ell[PSPEC_MAX_ELL / 2 + 1];
};

__global__ void k_finalize(const double* __restrict__ bins, const double* __restrict__ nmodes_in,
                           const double* __restrict__ ksum, int nk, EllList el, const double* __restrict__ derived,
                           double* P, double* kmean, double* nmodes, int cart) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nk) return;
  const double n = nmodes_in[b];
  const double I = derived[D_I], S = derived[D_S];
  const double nan = __longlong_as_double(0x7ff8000000000000ULL);
  nmodes[b] = n;
  kmean[b] = n > 0.0 ? ksum[b] / n : nan;
  for (int i = 0; i < el.n; i++) {
    const int ell = el.ell[i];
    double v;
    const double B0 = bins[SLOT_P0 * nk + b];
    if (ell == 0)
      v = (B0 / n - S) / I;
    else if (!cart)
      v = 4.0 * M_PI * bins[(SLOT_ELL0 + i) * nk + b] / (I * n);
    else {
      // Cartesian: A2, A4 = sum mult (khat . rhat)^2, ^4 terms; L_2 = (3mu^2-1)/2, L_4 = (35mu^4-30mu^2+3)/8
      const double A2 = bins[SLOT_ELL0 * nk + b], A4 = bins[(SLOT_ELL0 + 1) * nk + b];
      v = ell == 2 ? 2.5 * (3.0 * A2 - B0) / (I * n) : 1.125 * (35.0 * A4 - 30.0 * A2 + 3.0 * B0) / (I * n);
    }
    P[(int64_t)i * nk + b] = n > 0.0 ? v : nan;
  }
}

void launch_finalize(const double* bins, const double* nmodes_in, const double* ksum, int nk, const int32_t* ells,
                     int n_ells, const double* derived, double* P, double* k_mean, double* n_modes, cudaStream_t s,
                     int cartesian) {
  EllList el;
  el.n = n_ells;
  for (int i = 0; i < n_ells; i++) el.ell[i] = ells[i];
  k_finalize<<<(nk + 127) / 128, 128, 0, s>>>(bins, nmodes_in, ksum, nk, el, derived, P, k_mean, n_modes, cartesian);
}

// ------------------------------------------------------------------ a7: wedges
__global__ void k_wedges(const double* __restrict__ P, int n_ells, int nk, int n_mu, WedgeTab t, double* out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_mu * nk) return;
  const int w = idx / nk, b = idx - w * nk;
  double s = 0.0;
  for (int i = 0; i < n_ells; i++) s += P[(int64_t)i * nk + b] * t.lbar[i * n_mu + w];
  out[idx] = s;
}

void launch_wedges(const double* P, int n_ells, int nk, int n_mu, const WedgeTab& t, double* out, cudaStream_t s) {
  const int n = n_mu * nk;
  if (n <= 0) return;
  k_wedges<<<(n + 127) / 128, 128, 0, s>>>(P, n_ells, nk, n_mu, t, out);
}

}  // namespace pspec
