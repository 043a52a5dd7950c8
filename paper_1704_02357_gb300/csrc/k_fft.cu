// Shared pieces of the transform passes: the mode counts behind N_b and k_mean, the Y_lm
// recurrence tables, and the dispatch from a mesh side N to its compiled passes.
#include <cmath>
#include "launch.h"

namespace pspec {

__device__ __forceinline__ int signed_freq(int i, int N) { return i < N / 2 ? i : i - N; }

// cnt[|n|^2] += multiplicity over every stored mode that can be binned (no n_d = -N/2).
__global__ void k_mode_counts(Geo g, unsigned int* cnt) {
  const int N = g.N, NH = g.NH;
  const int64_t total = (int64_t)N * N * NH;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int kz = (int)(idx % NH);
    const int64_t ij = idx / NH;
    const int j = (int)(ij % N), i = (int)(ij / N);
    if (i == N / 2 || j == N / 2) continue;
    const int nx = signed_freq(i, N), ny = signed_freq(j, N);
    atomicAdd(&cnt[nx * nx + ny * ny + kz * kz], kz ? 2u : 1u);
  }
}

// N_b and sum |k| per bin from the counts of the |n|^2 values in [lo_b, hi_b).
__global__ void k_bin_counts(const unsigned int* __restrict__ cnt, const double* __restrict__ kmag,
                             const int* __restrict__ lo, const int* __restrict__ hi, int nk, double* nmodes,
                             double* ksum) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nk) return;
  double n = 0.0, k = 0.0;
  for (int q = lo[b]; q < hi[b]; q++) {
    if (q == 0) continue;
    const double m = (double)cnt[q];
    n += m;
    k += m * kmag[q];
  }
  nmodes[b] = n;
  ksum[b] = k;
}

void launch_mode_counts(const Geo& g, unsigned int* cnt, int nsm, cudaStream_t s) {
  k_mode_counts<<<8 * nsm, 256, 0, s>>>(g, cnt);
}

void launch_bin_counts(const unsigned int* cnt, const double* kmag, const int* lo, const int* hi, int nk,
                       double* nmodes, double* ksum, cudaStream_t s) {
  k_bin_counts<<<(nk + 127) / 128, 128, 0, s>>>(cnt, kmag, lo, hi, nk, nmodes, ksum);
}

// ------------------------------------------------------------------ Y tables
template <typename T> static YTab<T> build_ytab() {
  YTab<T> t;
  double c[kLdim];
  c[0] = 1.0 / std::sqrt(4.0 * M_PI);
  for (int a = 1; a < kLdim; a++) c[a] = -std::sqrt((2.0 * a + 1.0) / (2.0 * a)) * c[a - 1];
  for (int i = 0; i < kLdim * kLdim; i++) {
    t.A[i] = T(0);
    t.B[i] = T(0);
    t.Al[i] = T(0);
    t.Bl[i] = T(0);
  }
  for (int a = 0; a < kLdim; a++) {
    const double n = a == 0 ? c[0] : std::sqrt(2.0) * c[a];
    t.n[a] = T(n);
    t.nl[a] = sizeof(T) == 4 ? T(n - (double)T(n)) : T(0);
  }
  for (int l = 1; l < kLdim; l++) {
    for (int a = 0; a < l; a++) {
      const double A = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)a * a));
      const double num = (double)(l - 1) * (l - 1) - (double)a * a;
      const double B = num > 0 ? std::sqrt(num / (4.0 * (l - 1) * (l - 1) - 1.0)) : 0.0;
      t.A[l * kLdim + a] = T(A);
      t.B[l * kLdim + a] = T(B);
      if (sizeof(T) == 4) {
        t.Al[l * kLdim + a] = T(A - (double)T(A));
        t.Bl[l * kLdim + a] = T(B - (double)T(B));
      }
    }
  }
  return t;
}

template <> const YTab<float>& host_ytab<float>() {
  static const YTab<float> t = build_ytab<float>();
  return t;
}
template <> const YTab<double>& host_ytab<double>() {
  static const YTab<double> t = build_ytab<double>();
  return t;
}

// ------------------------------------------------------------------ Y_lm(khat) table
// Position m of a k-space table of the binning pass -> its mode (i, j, kz): one block of N x tw
// values per x tile (j, kz tile), rows i, m = ((kz / tw * N + j) * N + i) * tw + kz % tw.
__device__ __forceinline__ void table_mode(int64_t m, int N, int tw, int& i, int& j, int& kz) {
  const int c = (int)(m % tw);
  int64_t r = m / tw;
  i = (int)(r % N);
  r /= N;
  j = (int)(r % N);
  kz = (int)(r / N) * tw + c;
}

// One thread per stored mode (i, j, kz): khat in FP64, then for a = 0..l_max the recurrence in
// l (FP64 coefficients) and (x + i y)^a; each Y_{l,m} of an even l >= 2 is stored rounded to
// FP32 at ytab[(ytab_base(l) + h) * modes + m] (h = 0, 2a-1, 2a for m = 0, +a, -a; m the
// table position of the mode). The mode k = 0 gets 0.
__global__ void __launch_bounds__(256) k_ytab_build(float* __restrict__ ytab, int N, int tw, int ell_max,
                                                    const __grid_constant__ YTab<double> yt) {
  const int NH = N / 2;
  const int64_t modes = (int64_t)N * N * NH;
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < modes; m += (int64_t)gridDim.x * blockDim.x) {
    int i, j, kz;
    table_mode(m, N, tw, i, j, kz);
    const double fx = i < NH ? i : i - N, fy = j < NH ? j : j - N, fz = kz;
    const double r2 = fx * fx + fy * fy + fz * fz;
    const double inv = r2 > 0.0 ? 1.0 / sqrt(r2) : 0.0;
    const double x = fx * inv, y = fy * inv, z = fz * inv;
    double pr = 1.0, pi = 0.0;  // (x + i y)^a
    for (int a = 0; a <= ell_max; a++) {
      double qm1 = 0.0, qm2 = 0.0;
      for (int l = a; l <= ell_max; l++) {
        double q;
        if (l == a)
          q = 1.0;
        else if (l == a + 1)
          q = yt.A[l * kLdim + a] * z * qm1;
        else
          q = yt.A[l * kLdim + a] * (z * qm1 - yt.B[l * kLdim + a] * qm2);
        qm2 = qm1;
        qm1 = q;
        if (l < 2 || (l & 1)) continue;
        float* base = ytab + (int64_t)ytab_base(l) * modes + m;
        if (r2 == 0.0) {
          if (a == 0) base[0] = 0.f;
          else base[(int64_t)(2 * a - 1) * modes] = base[(int64_t)(2 * a) * modes] = 0.f;
        } else if (a == 0) {
          base[0] = (float)(yt.n[0] * q);
        } else {
          base[(int64_t)(2 * a - 1) * modes] = (float)(yt.n[a] * q * pr);
          base[(int64_t)(2 * a) * modes] = (float)(yt.n[a] * q * pi);
        }
      }
      const double nr = pr * x - pi * y;
      pi = pr * y + pi * x;
      pr = nr;
    }
  }
}

// ------------------------------------------------------------------ Y_lm(rhat) table
// One thread per mesh node (i, j, k): rhat = (corner + (i, j, k) H - observer)/|.| in FP64,
// the recurrence in l (FP64 coefficients) and (x + i y)^a, each Y_{l,m} of an even l >= 2
// stored rounded once to FP32 at rtab[(ytab_base(l) + h) * N^3 + (i N + j) N + k]. The node at
// the observer gets 0.
__global__ void __launch_bounds__(256) k_rtab_build(float* __restrict__ rtab, int N, int ell_max, RGeo g,
                                                    const __grid_constant__ YTab<double> yt) {
  const int64_t pts = (int64_t)N * N * N;
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < pts; m += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(m % N);
    const int64_t ij = m / N;
    const int j = (int)(ij % N), i = (int)(ij / N);
    const double vx = g.corner[0] + i * g.H - g.observer[0], vy = g.corner[1] + j * g.H - g.observer[1],
                 vz = g.corner[2] + k * g.H - g.observer[2];
    const double r2 = vx * vx + vy * vy + vz * vz;
    const double inv = r2 > 0.0 ? 1.0 / sqrt(r2) : 0.0;
    const double x = vx * inv, y = vy * inv, z = vz * inv;
    double pr = 1.0, pi = 0.0;  // (x + i y)^a
    for (int a = 0; a <= ell_max; a++) {
      double qm1 = 0.0, qm2 = 0.0;
      for (int l = a; l <= ell_max; l++) {
        double q;
        if (l == a)
          q = 1.0;
        else if (l == a + 1)
          q = yt.A[l * kLdim + a] * z * qm1;
        else
          q = yt.A[l * kLdim + a] * (z * qm1 - yt.B[l * kLdim + a] * qm2);
        qm2 = qm1;
        qm1 = q;
        if (l < 2 || (l & 1)) continue;
        float* base = rtab + (int64_t)ytab_base(l) * pts + m;
        if (r2 == 0.0) {
          if (a == 0) base[0] = 0.f;
          else base[(int64_t)(2 * a - 1) * pts] = base[(int64_t)(2 * a) * pts] = 0.f;
        } else if (a == 0) {
          base[0] = (float)(yt.n[0] * q);
        } else {
          base[(int64_t)(2 * a - 1) * pts] = (float)(yt.n[a] * q * pr);
          base[(int64_t)(2 * a) * pts] = (float)(yt.n[a] * q * pi);
        }
      }
      const double nr = pr * x - pi * y;
      pi = pr * y + pi * x;
      pr = nr;
    }
  }
}

void launch_rtab_build(float* rtab, int N, int ell_max, const RGeo& g, int nsm, cudaStream_t s) {
  k_rtab_build<<<8 * nsm, 256, 0, s>>>(rtab, N, ell_max, g, host_ytab<double>());
}

void launch_ytab_build(float* ytab, int N, int tw, int ell_max, int nsm, cudaStream_t s) {
  k_ytab_build<<<8 * nsm, 256, 0, s>>>(ytab, N, tw, ell_max, host_ytab<double>());
}

// Cartesian k-space factors: ctab[q * modes + m] = mult_q khat^q in FP64, rounded once to FP32
// (0 for k = 0), m the table position of the mode.
__global__ void __launch_bounds__(256) k_ctab_build(float* __restrict__ ctab, int N, int tw) {
  const int NH = N / 2;
  const int64_t modes = (int64_t)N * N * NH;
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < modes; m += (int64_t)gridDim.x * blockDim.x) {
    int i, j, kz;
    table_mode(m, N, tw, i, j, kz);
    const double fx = i < NH ? i : i - N, fy = j < NH ? j : j - N, fz = kz;
    const double r2 = fx * fx + fy * fy + fz * fz;
    const double inv = r2 > 0.0 ? 1.0 / sqrt(r2) : 0.0;
    const double x = fx * inv, y = fy * inv, z = fz * inv;
    for (int q = 0; q < kCartItems; q++) {
      int a, b, c;
      cart_exp(q, a, b, c);
      ctab[(int64_t)q * modes + m] = (float)(cart_mult(q) * ipow(x, a) * ipow(y, b) * ipow(z, c));
    }
  }
}

void launch_ctab_build(float* ctab, int N, int tw, int nsm, cudaStream_t s) {
  k_ctab_build<<<8 * nsm, 256, 0, s>>>(ctab, N, tw);
}

// ------------------------------------------------------------------ dispatch
template <typename T> const PassTable<T>* pass_table(int N) {
  switch (N) {
    case 16: return pass_table_n<T, 16>();
    case 32: return pass_table_n<T, 32>();
    case 64: return pass_table_n<T, 64>();
    case 128: return pass_table_n<T, 128>();
    case 256: return pass_table_n<T, 256>();
    case 512: return pass_table_n<T, 512>();
    case 1024: return pass_table_n<T, 1024>();
    case 48: return pass_table_n<T, 48>();
    case 96: return pass_table_n<T, 96>();
    case 192: return pass_table_n<T, 192>();
    case 384: return pass_table_n<T, 384>();
    case 768: return pass_table_n<T, 768>();
    default: return nullptr;
  }
}
template const PassTable<float>* pass_table<float>(int);
template const PassTable<double>* pass_table<double>(int);

}  // namespace pspec
