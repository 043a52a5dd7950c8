// Catalog sums, mass assignment, finalisation and wedges of the SH-FFT estimator.
//   a1 catalog sums: Sec. 2.1 eq. FKP-density (alpha, I) and the shot-noise term.
//   a2 painting:     Sec. 2.3 (CIC / TSC kernels, interlaced second mesh at u - 1/2).
//   a6 finalise:     Sec. 2.1 eq. Pell-ours (4 pi / (I N_b) for l >= 2; noise for l = 0).
//   a7 wedges:       Sec. 2.2 eqs. wedge-est and Lbar.
#include <cmath>
#include "launch.h"

namespace pspec {

constexpr int kSumThreads = 256;
// Positions further than this many cells from the corner are rejected as invalid (with the
// non-finite ones): beyond it the periodic reduction of the grid coordinate loses meaning.
constexpr double kMaxCells = 1099511627776.0;  // 2^40

__device__ __forceinline__ bool usable(double ux, double uy, double uz, double wc, double nb) {
  return fabs(ux) < kMaxCells && fabs(uy) < kMaxCells && fabs(uz) < kMaxCells && isfinite(wc) && isfinite(nb);
}

// Neumaier-compensated FP64 accumulator.
struct Neu {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    const double t = s + x;
    c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double val() const { return s + c; }
};

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

// Per-block partials: [0] sum w_c, [1] sum v^2, [2] sum nbar w_c w_fkp^2, [3] non-finite,
// [4] outside the box.
__global__ void __launch_bounds__(kSumThreads) k_catalog_partials(PaintArgs a, int nmesh, double* out) {
  __shared__ double red[kSumThreads / 32];
  Neu s0, s1, s2;
  double nonfin = 0.0, wrapped = 0.0;
  const double lim = (double)nmesh;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.count;
       p += (int64_t)gridDim.x * blockDim.x) {
    double x, y, z;
    load_pos(a, p, x, y, z);
    const double wc = a.weight ? a.weight[p] : 1.0;
    const double nb = a.nbar ? a.nbar[p] : a.nbar_default;
    const double ux = (x - a.corner[0]) / a.cell, uy = (y - a.corner[1]) / a.cell,
                 uz = (z - a.corner[2]) / a.cell;
    if (!usable(ux, uy, uz, wc, nb)) {
      nonfin += 1.0;
      continue;
    }
    const double wf = a.P0 > 0.0 ? 1.0 / (1.0 + nb * a.P0) : 1.0;
    const double v = wc * wf;
    s0.add(wc);
    s1.add(v * v);
    s2.add(nb * wc * wf * wf);
    if (ux < 0.0 || ux >= lim || uy < 0.0 || uy >= lim || uz < 0.0 || uz >= lim) wrapped += 1.0;
  }
  const double r0 = block_sum(s0.val(), red);
  const double r1 = block_sum(s1.val(), red);
  const double r2 = block_sum(s2.val(), red);
  const double r3 = block_sum(nonfin, red);
  const double r4 = block_sum(wrapped, red);
  if (threadIdx.x == 0) {
    double* o = out + (int64_t)blockIdx.x * kSumVals;
    o[0] = r0;
    o[1] = r1;
    o[2] = r2;
    o[3] = r3;
    o[4] = r4;
    o[5] = 0.0;
  }
}

// One thread adds the block partials in a fixed order: deterministic alpha, I, S.
__global__ void k_catalog_final(const double* pd, int nbd, const double* pr, int nbr, double* d) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Neu wd, sd, wr, sr, ir;
  double nf = 0.0, wp = 0.0;
  for (int b = 0; b < nbd; b++) {
    wd.add(pd[b * kSumVals + 0]);
    sd.add(pd[b * kSumVals + 1]);
    nf += pd[b * kSumVals + 3];
    wp += pd[b * kSumVals + 4];
  }
  for (int b = 0; b < nbr; b++) {
    wr.add(pr[b * kSumVals + 0]);
    sr.add(pr[b * kSumVals + 1]);
    ir.add(pr[b * kSumVals + 2]);
    nf += pr[b * kSumVals + 3];
    wp += pr[b * kSumVals + 4];
  }
  const double alpha = wd.val() / wr.val();
  d[D_WD] = wd.val();
  d[D_WR] = wr.val();
  d[D_ALPHA] = alpha;
  d[D_I] = alpha * ir.val();
  d[D_S] = sd.val() + alpha * alpha * sr.val();
  d[D_NONFINITE] = nf;
  d[D_WRAPPED] = wp;
  d[D_SD] = sd.val();
  d[D_SR] = sr.val();
  d[D_IR] = ir.val();
}

void launch_catalog_partials(const PaintArgs& a, int nmesh, double* partials, int nblocks, cudaStream_t s) {
  k_catalog_partials<<<nblocks, kSumThreads, 0, s>>>(a, nmesh, partials);
}

void launch_catalog_final(const double* part_d, int nb_d, const double* part_r, int nb_r, double* derived,
                          cudaStream_t s) {
  k_catalog_final<<<1, 32, 0, s>>>(part_d, nb_d, part_r, nb_r, derived);
}

// ------------------------------------------------------------------ painting
// Node weights along one axis at grid coordinate u, |u| < kMaxCells: u is first reduced
// to about [0, N) and every node index is then wrapped into [0, N) on both sides, so a
// rounding at the ends of the reduction cannot leave the mesh.
template <int WIN>
__device__ __forceinline__ void axis_weights(double u, int N, int* idx, double* w) {
  u = u - (double)N * floor(u / (double)N);
  if (WIN == PSPEC_WINDOW_CIC) {
    const double f = floor(u);
    const double d = u - f;
    const int b = (int)f;
    w[0] = 1.0 - d;
    w[1] = d;
    for (int k = 0; k < 2; k++) {
      int i = (b + k) % N;
      idx[k] = i < 0 ? i + N : i;
    }
  } else {
    const double c = floor(u + 0.5);
    const double d = u - c;
    const int b = (int)c - 1;
    w[0] = 0.5 * (0.5 - d) * (0.5 - d);
    w[1] = 0.75 - d * d;
    w[2] = 0.5 * (0.5 + d) * (0.5 + d);
    for (int k = 0; k < 3; k++) {
      int i = (b + k) % N;
      idx[k] = i < 0 ? i + N : i;
    }
  }
}

template <typename T, int WIN>
__device__ __forceinline__ void paint_one(T* __restrict__ m, int N, double ux, double uy, double uz, double v) {
  constexpr int K = WIN == PSPEC_WINDOW_CIC ? 2 : 3;
  int ix[3], iy[3], iz[3];
  double wx[3], wy[3], wz[3];
  axis_weights<WIN>(ux, N, ix, wx);
  axis_weights<WIN>(uy, N, iy, wy);
  axis_weights<WIN>(uz, N, iz, wz);
#pragma unroll
  for (int a = 0; a < K; a++) {
    const double va = v * wx[a];
#pragma unroll
    for (int b = 0; b < K; b++) {
      const double vb = va * wy[b];
      T* row = m + ((int64_t)ix[a] * N + iy[b]) * N;
#pragma unroll
      for (int c = 0; c < K; c++) atomicAdd(row + iz[c], (T)(vb * wz[c]));
    }
  }
}

template <typename T, int WIN, bool INTER>
__global__ void __launch_bounds__(256) k_paint(PaintArgs a, int is_randoms, const double* __restrict__ derived,
                                               T* __restrict__ m1, T* __restrict__ m2, int N) {
  const double sign = is_randoms ? -derived[D_ALPHA] : 1.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.count;
       p += (int64_t)gridDim.x * blockDim.x) {
    double x, y, z;
    load_pos(a, p, x, y, z);
    const double wc = a.weight ? a.weight[p] : 1.0;
    const double nb = a.nbar ? a.nbar[p] : a.nbar_default;
    const double ux = (x - a.corner[0]) / a.cell, uy = (y - a.corner[1]) / a.cell,
                 uz = (z - a.corner[2]) / a.cell;
    if (!usable(ux, uy, uz, wc, nb)) continue;
    const double wf = a.P0 > 0.0 ? 1.0 / (1.0 + nb * a.P0) : 1.0;
    const double v = sign * wc * wf;
    paint_one<T, WIN>(m1, N, ux, uy, uz, v);
    if (INTER) paint_one<T, WIN>(m2, N, ux - 0.5, uy - 0.5, uz - 0.5, v);
  }
}

template <typename T>
void launch_paint(const PaintArgs& a, int window, int interlaced, int is_randoms, const double* derived,
                  T* mesh1, T* mesh2, int N, int nblocks, cudaStream_t s) {
  if (a.count <= 0) return;
  int64_t need = (a.count + 255) / 256;
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
template void launch_paint<float>(const PaintArgs&, int, int, int, const double*, float*, float*, int, int,
                                  cudaStream_t);
template void launch_paint<double>(const PaintArgs&, int, int, int, const double*, double*, double*, int, int,
                                   cudaStream_t);

// ------------------------------------------------------------------ finalise
struct EllList {
  int n;
  int ell[PSPEC_MAX_ELL / 2 + 1];
};

__global__ void k_finalize(const double* __restrict__ part, int ctas, int nslots, int nk, EllList el,
                           const double* __restrict__ derived, double* P, double* kmean, double* nmodes) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nk) return;
  Neu nm, ks, p0;
  for (int c = 0; c < ctas; c++) {
    const double* pc = part + (int64_t)c * nslots * nk;
    nm.add(pc[SLOT_NMODES * nk + b]);
    ks.add(pc[SLOT_KSUM * nk + b]);
    p0.add(pc[SLOT_P0 * nk + b]);
  }
  const double n = nm.val();
  const double I = derived[D_I], S = derived[D_S];
  const double nan = __longlong_as_double(0x7ff8000000000000ULL);
  nmodes[b] = n;
  kmean[b] = n > 0.0 ? ks.val() / n : nan;
  for (int i = 0; i < el.n; i++) {
    const int ell = el.ell[i];
    double v;
    if (ell == 0) {
      v = (p0.val() / n - S) / I;
    } else {
      Neu acc;
      for (int c = 0; c < ctas; c++) acc.add(part[((int64_t)c * nslots + SLOT_ELL0 + i) * nk + b]);
      v = 4.0 * M_PI * acc.val() / (I * n);
    }
    P[(int64_t)i * nk + b] = n > 0.0 ? v : nan;
  }
}

void launch_finalize(const double* partials, int ctas, int nslots, int nk, const int32_t* ells, int n_ells,
                     const double* derived, double* P, double* k_mean, double* n_modes, cudaStream_t s) {
  EllList el;
  el.n = n_ells;
  for (int i = 0; i < n_ells; i++) el.ell[i] = ells[i];
  k_finalize<<<(nk + 127) / 128, 128, 0, s>>>(partials, ctas, nslots, nk, el, derived, P, k_mean, n_modes);
}

// ------------------------------------------------------------------ wedges
__global__ void k_wedges(const double* __restrict__ P, int n_ells, int nk, int n_mu, WedgeTab t, double* out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_mu * nk) return;
  const int w = idx / nk, b = idx - w * nk;
  double s = 0.0;
  for (int i = 0; i < n_ells; i++) s += P[(int64_t)i * nk + b] * t.lbar[i * n_mu + w];
  out[idx] = s;
}

void launch_wedges(const double* P, int n_ells, int nk, int n_mu, const WedgeTab& t, double* out,
                   cudaStream_t s) {
  const int n = n_mu * nk;
  if (n <= 0) return;
  k_wedges<<<(n + 127) / 128, 128, 0, s>>>(P, n_ells, nk, n_mu, t, out);
}

}  // namespace pspec
