// Transform passes of the SH-FFT multipole estimator (Sec. 2.1 eqs. Pell-ours, Fell;
// Sec. 2.3 interlacing, compensation and the inverse transform before the Y_lm weights).
//
// Storage: real mesh r[(i*N + j)*N + k]; half spectrum s[(i*N + j)*NH + kz], NH = N/2.
// The kz = N/2 plane is never stored: its modes are zeroed before the inverse transform
// and never binned, so nothing downstream reads it.
//
// A 3-D forward transform is three passes, each one HBM round trip:
//   z: rows of N reals -> N/2-point complex FFT of packed pairs -> unpack to N/2 modes
//   y: columns along j of an (i, kz-tile) slab, in place
//   x: columns along i of a (j, kz-tile) slab; fused with the interlace/compensate
//      combine (F0 and the l = 0 sums) or with the Y_lm(khat) accumulate-and-bin.
// Every pass keeps its elements in registers (fft_engine.cuh); kz tiles of TW columns give
// TW*8-byte contiguous segments per row.
#include <cstdio>
#include <cmath>
#include "launch.h"
#include "fft_engine.cuh"

namespace pspec {

__constant__ YTab<float> c_ytab_f;
__constant__ YTab<double> c_ytab_d;
template <typename T> __device__ __forceinline__ const YTab<T>& ytab();
template <> __device__ __forceinline__ const YTab<float>& ytab<float>() { return c_ytab_f; }
template <> __device__ __forceinline__ const YTab<double>& ytab<double>() { return c_ytab_d; }

__device__ __forceinline__ int signed_freq(int i, int N) { return i < N / 2 ? i : i - N; }

// r2c unpack: X[k] = (Z[k] + Z*[L-k])/2 - i/2 w^k (Z[k] - Z*[L-k]), w = exp(-2 pi i/N)
template <typename C, typename T>
__device__ __forceinline__ C r2c_unpack(C zk, C zm, C w) {
  const C zc = cconj(zm);
  const C e = cscale(cadd(zk, zc), T(0.5));
  const C d = csub(zk, zc);
  const C o = mk(T(0.5) * d.y, T(-0.5) * d.x);
  return cadd(e, cmul(w, o));
}

// ------------------------------------------------------------------ pass z: r2c of plain rows
// Block: `rows` rows x Tc threads (t fastest). Each row of N reals is read as L = N/2
// complex pairs.
template <typename T, int E>
__global__ void __launch_bounds__(512) k_r2c_z(const T* __restrict__ in, cx<T>* __restrict__ out, Geo g,
                                               FftPlan pz, const cx<T>* __restrict__ twh,
                                               const cx<T>* __restrict__ twr, int rows) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int L = g.NH, Tc = L / E, Lp = padded_len(L);
  const int r = threadIdx.x / Tc, t = threadIdx.x - r * Tc;
  const int64_t row = (int64_t)blockIdx.x * rows + r;
  const C* src = reinterpret_cast<const C*>(in + row * g.N);
  C v[E];
#pragma unroll
  for (int e = 0; e < E; e++) v[e] = src[t + Tc * e];
  fft_regs<C, E, kPaddedRows, -1>(v, sm, pz, t, r, rows, twh);
#pragma unroll
  for (int e = 0; e < E; e++) sm[sidx<kPaddedRows>(r, t + Tc * e, rows, Lp)] = v[e];
  __syncthreads();
  C* dst = out + row * L;
#pragma unroll
  for (int e = 0; e < E; e++) {
    const int k = t + Tc * e;
    const C zm = sm[sidx<kPaddedRows>(r, k ? L - k : 0, rows, Lp)];
    dst[k] = r2c_unpack<C, T>(v[e], zm, ldg_c(twr + k));
  }
}

// ------------------------------------------------------------------ pass z: c2r
// Rows of L stored modes (the kz = N/2 mode taken as 0) -> N reals, times `scale`.
template <typename T, int E>
__global__ void __launch_bounds__(512) k_c2r_z(const cx<T>* __restrict__ in, T* __restrict__ out, Geo g,
                                               FftPlan pz, const cx<T>* __restrict__ twh,
                                               const cx<T>* __restrict__ twr, int rows, T scale) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int L = g.NH, Tc = L / E;
  const int r = threadIdx.x / Tc, t = threadIdx.x - r * Tc;
  const int64_t row = (int64_t)blockIdx.x * rows + r;
  const C* src = in + row * L;
  C v[E];
#pragma unroll
  for (int e = 0; e < E; e++) {
    const int k = t + Tc * e;
    const C xk = src[k];
    const C xm = k ? cconj(src[L - k]) : mk(T(0), T(0));
    const C ev = cscale(cadd(xk, xm), T(0.5));
    const C od = cmul(cscale(csub(xk, xm), T(0.5)), cconj(ldg_c(twr + k)));
    v[e] = mk(ev.x - od.y, ev.y + od.x);  // E + i O
  }
  fft_regs<C, E, kPaddedRows, +1>(v, sm, pz, t, r, rows, twh);
  C* dst = reinterpret_cast<C*>(out + row * g.N);
#pragma unroll
  for (int e = 0; e < E; e++) dst[t + Tc * e] = cscale(v[e], scale);
}

// ------------------------------------------------------------------ pass z: Y_lm-weighted r2c
// For `rows` rows of f and the M harmonics h0..h0+M-1 of multipole l. Every point sweeps
// its harmonics once ((x+iy)^a carried from one |m| to the next) into a shared staging
// area of nseq = M*rows real rows; then each of the nseq*Tc threads loads its slots, the
// sequences are transformed (the staging area is reused as the exchange buffer) and
// unpacked into the M spectra.
template <typename T, int E>
__global__ void __launch_bounds__(512) k_ylm_r2c_z(const T* __restrict__ f, cx<T>* __restrict__ out,
                                                  int64_t spec_stride, int ell, int h0, int M, Geo g, FftPlan pz,
                                                  const cx<T>* __restrict__ twh, const cx<T>* __restrict__ twr,
                                                  const T* __restrict__ axis, int rows) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = g.N, L = g.NH, Tc = L / E, Lp = padded_len(L);
  const int nseq = M * rows;
  T* stage = reinterpret_cast<T*>(smraw);  // [nseq][N] reals, then the exchange buffer
  C* xb = reinterpret_cast<C*>(smraw);
  const YTab<T>& yt = ytab<T>();
  const int64_t row0 = (int64_t)blockIdx.x * rows;
  const int a_lo = harm_a(h0), a_hi = harm_a(h0 + M - 1);
  const T sq2 = T(1.41421356237309504880);
  for (int p = threadIdx.x; p < rows * N; p += blockDim.x) {
    const int r = p / N, kk = p - r * N;
    const int64_t grow = row0 + r;
    const int i = (int)(grow / N), j = (int)(grow - (int64_t)i * N);
    const T fv = f[grow * N + kk];
    const T vx = axis[i], vy = axis[N + j], vz = axis[2 * N + kk];
    const T r2 = vx * vx + vy * vy + vz * vz;
    if (r2 == T(0)) {
      for (int s = 0; s < M; s++) stage[(s * rows + r) * N + kk] = T(0);
      continue;
    }
    const T inv = rsqrt_t<T>(r2);
    const T x = vx * inv, y = vy * inv, z = vz * inv;
    T pr = T(1), pi = T(0);
    for (int s = 0; s < a_lo; s++) {
      const T nr = pr * x - pi * y;
      pi = pr * y + pi * x;
      pr = nr;
    }
    for (int a = a_lo; a <= a_hi; a++) {
      const T q = fv * ylm_q<T>(yt, ell, a, z);
      if (a == 0) {
        stage[r * N + kk] = q;
      } else {
        const int hp = 2 * a - 1, hm = 2 * a;
        if (hp >= h0 && hp < h0 + M) stage[((hp - h0) * rows + r) * N + kk] = sq2 * q * pr;
        if (hm >= h0 && hm < h0 + M) stage[((hm - h0) * rows + r) * N + kk] = sq2 * q * pi;
      }
      const T nr = pr * x - pi * y;
      pi = pr * y + pi * x;
      pr = nr;
    }
  }
  __syncthreads();
  const C* stc = reinterpret_cast<const C*>(stage);
  const int sq = threadIdx.x / Tc, t = threadIdx.x - sq * Tc;
  C v[E];
#pragma unroll
  for (int e = 0; e < E; e++) v[e] = stc[sq * L + t + Tc * e];
  __syncthreads();
  fft_regs<C, E, kPaddedRows, -1>(v, xb, pz, t, sq, nseq, twh);
#pragma unroll
  for (int e = 0; e < E; e++) xb[sidx<kPaddedRows>(sq, t + Tc * e, nseq, Lp)] = v[e];
  __syncthreads();
  const int s = sq / rows, r = sq - s * rows;
  C* dst = out + s * spec_stride + (row0 + r) * L;
#pragma unroll
  for (int e = 0; e < E; e++) {
    const int k = t + Tc * e;
    const C zm = xb[sidx<kPaddedRows>(sq, k ? L - k : 0, nseq, Lp)];
    dst[k] = r2c_unpack<C, T>(v[e], zm, ldg_c(twr + k));
  }
}

// ------------------------------------------------------------------ pass y (in place)
// Block: one (i, kz-tile) slab, TW columns x Tc threads (column fastest).
template <typename T, int E, int DIR>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) k_fft_y(cx<T>* __restrict__ data, int64_t spec_stride, Geo g, FftPlan pf,
                                                  const cx<T>* __restrict__ twf, int TW) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int N = g.N, NH = g.NH, Tc = N / E;
  const int c = threadIdx.x % TW, t = threadIdx.x / TW;
  const int ntz = NH / TW;
  const int i = blockIdx.x / ntz, kz0 = (blockIdx.x - i * ntz) * TW;
  C* base = data + (int64_t)blockIdx.y * spec_stride + (int64_t)i * N * NH + kz0 + c;
  C v[E];
#pragma unroll
  for (int e = 0; e < E; e++) v[e] = base[(int64_t)(t + Tc * e) * NH];
  fft_regs<C, E, kInterleaved, DIR>(v, sm, pf, t, c, TW, twf);
#pragma unroll
  for (int e = 0; e < E; e++) base[(int64_t)(t + Tc * e) * NH] = v[e];
}

// ------------------------------------------------------------------ pass x (plain)
template <typename T, int E, int DIR>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) k_fft_x(const cx<T>* in, cx<T>* out, Geo g, FftPlan pf,
                                                  const cx<T>* __restrict__ twf, int TW) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int N = g.N, NH = g.NH, Tc = N / E;
  const int c = threadIdx.x % TW, t = threadIdx.x / TW;
  const int ntz = NH / TW;
  const int j = blockIdx.x / ntz, kz0 = (blockIdx.x - j * ntz) * TW;
  const int64_t si = (int64_t)N * NH;
  const int64_t off = (int64_t)j * NH + kz0 + c;
  C v[E];
#pragma unroll
  for (int e = 0; e < E; e++) v[e] = in[off + (t + Tc * e) * si];
  fft_regs<C, E, kInterleaved, DIR>(v, sm, pf, t, c, TW, twf);
#pragma unroll
  for (int e = 0; e < E; e++) out[off + (t + Tc * e) * si] = v[e];
}

// ------------------------------------------------------------------ pass x + combine (F0) + l = 0 sums
// X = (F1 + exp(-i k.s) F2)/2 (interlaced) or F1; divided by W(k) when compensating; zeroed
// where some n_d = -N/2 when the inverse transform follows; stored as F0.
// Binned: sum over modes of mult |X|^2 (slot SLOT_P0). Persistent over tiles.
template <typename T, int E>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) k_combine_x(const cx<T>* B, cx<T>* F0, Geo g, FftPlan pf,
                                                   const cx<T>* __restrict__ twf, int TW, int interlaced,
                                                   int compensate, int roundtrip, const cx<T>* __restrict__ phase,
                                                   const T* __restrict__ invw, BinArgs ba) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = g.N, NH = g.NH, Tc = N / E;
  C* sm = reinterpret_cast<C*>(smraw);
  WarpBins<T> wb;
  wb.nk = ba.nk;
  wb.nwarps = (blockDim.x + 31) >> 5;
  wb.b = reinterpret_cast<double*>(sm + N * TW);
  wb.w = reinterpret_cast<T*>(wb.b + ba.nk);
  wb.init();
  const int c = threadIdx.x % TW, t = threadIdx.x / TW;
  const int ntz = NH / TW, ntiles = N * ntz;
  const int64_t si = (int64_t)N * NH;
  __syncthreads();
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int j = tile / ntz, kz0 = (tile - j * ntz) * TW;
    const int kz = kz0 + c;
    const int64_t off = (int64_t)j * NH + kz;
    C v[E];
#pragma unroll
    for (int e = 0; e < E; e++) v[e] = B[off + (t + Tc * e) * si];
    fft_regs<C, E, kInterleaved, -1>(v, sm, pf, t, c, TW, twf);
    const int ny = signed_freq(j, N);
    const C phy = ldg_c(phase + j), phz = ldg_c(phase + N + kz);
    const T wyz = invw[j] * invw[N + kz];
    const T mult = kz ? T(2) : T(1);
#pragma unroll
    for (int e = 0; e < E; e++) {
      const int ii = t + Tc * e;
      const int64_t addr = off + ii * si;
      C X = v[e];
      if (interlaced) {
        const C A = F0[addr];
        const C ph = cmul(cmul(ldg_c(phase + ii), phy), phz);
        X = cscale(cadd(A, cmul(ph, X)), T(0.5));
      }
      if (compensate) X = cscale(X, invw[ii] * wyz);
      const bool nyq = (ii == N / 2) || (j == N / 2);
      if (roundtrip && nyq) X = mk(T(0), T(0));
      F0[addr] = X;
      if (!nyq) {
        const int nx = signed_freq(ii, N);
        const int n2 = nx * nx + ny * ny + kz * kz;
        const int b = ba.bin_of_n2[n2];
        if (b >= 0 && n2 > 0) wb.add(b, mult * (X.x * X.x + X.y * X.y));
      }
    }
    __syncthreads();
    wb.fold();
    __syncthreads();
  }
  for (int b = threadIdx.x; b < ba.nk; b += blockDim.x) atomicAdd(&ba.bins[SLOT_P0 * ba.nk + b], wb.b[b]);
}

// ------------------------------------------------------------------ pass x + accumulate-and-bin
// Per tile: F0 once (kept in shared memory, each thread its own modes); for each harmonic h
// of the group, the x-pass of G_h and acc += Y_{l,m(h)}(khat) Re[G_h conj(F0)] per mode;
// then mult * acc into the bins of `slot`.
template <typename T, int E>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) k_bin_x(const cx<T>* G, int64_t spec_stride, int ell, int h0, int M,
                                                  const cx<T>* __restrict__ F0, Geo g, FftPlan pf,
                                                  const cx<T>* __restrict__ twf, int TW, int slot, BinArgs ba) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = g.N, NH = g.NH, Tc = N / E;
  C* sm = reinterpret_cast<C*>(smraw);
  C* sF0 = sm + N * TW;
  WarpBins<T> wb;
  wb.nk = ba.nk;
  wb.nwarps = (blockDim.x + 31) >> 5;
  wb.b = reinterpret_cast<double*>(sF0 + N * TW);
  wb.w = reinterpret_cast<T*>(wb.b + ba.nk);
  wb.init();
  const YTab<T>& yt = ytab<T>();
  const T sq2 = T(1.41421356237309504880);
  const int c = threadIdx.x % TW, t = threadIdx.x / TW;
  const int ntz = NH / TW, ntiles = N * ntz;
  const int64_t si = (int64_t)N * NH;
  __syncthreads();
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int j = tile / ntz, kz0 = (tile - j * ntz) * TW;
    const int kz = kz0 + c;
    const int64_t off = (int64_t)j * NH + kz;
    const T fy = T(signed_freq(j, N)), fz = T(kz);
    const T r2yz = fy * fy + fz * fz;
    T acc[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
      sF0[(t + Tc * e) * TW + c] = F0[off + (t + Tc * e) * si];
      acc[e] = T(0);
    }
    for (int s = 0; s < M; s++) {
      const int h = h0 + s;
      const int a = harm_a(h), sg = harm_sign(h);
      const C* Gs = G + (int64_t)s * spec_stride;
      C v[E];
#pragma unroll
      for (int e = 0; e < E; e++) v[e] = Gs[off + (t + Tc * e) * si];
      fft_regs<C, E, kInterleaved, -1>(v, sm, pf, t, c, TW, twf);
#pragma unroll
      for (int e = 0; e < E; e++) {
        const T fx = T(signed_freq(t + Tc * e, N));
        const T r2 = fx * fx + r2yz;
        if (r2 == T(0)) continue;
        const T inv = rsqrt_t<T>(r2);
        const T x = fx * inv, y = fy * inv;
        T Y = ylm_q<T>(yt, ell, a, fz * inv);
        if (a > 0) {
          T pr = x, pi = y;
          for (int u = 1; u < a; u++) {
            const T nr = pr * x - pi * y;
            pi = pr * y + pi * x;
            pr = nr;
          }
          Y = sq2 * Y * (sg > 0 ? pr : pi);
        }
        const C fv = sF0[(t + Tc * e) * TW + c];
        acc[e] += Y * (v[e].x * fv.x + v[e].y * fv.y);
      }
    }
    if (j != N / 2) {
      const T mult = kz ? T(2) : T(1);
      const int ny = signed_freq(j, N);
#pragma unroll
      for (int e = 0; e < E; e++) {
        const int ii = t + Tc * e;
        if (ii == N / 2) continue;
        const int nx = signed_freq(ii, N);
        const int n2 = nx * nx + ny * ny + kz * kz;
        const int b = ba.bin_of_n2[n2];
        if (b >= 0 && n2 > 0) wb.add(b, mult * acc[e]);
      }
    }
    __syncthreads();
    wb.fold();
    __syncthreads();
  }
  for (int b = threadIdx.x; b < ba.nk; b += blockDim.x) atomicAdd(&ba.bins[slot * ba.nk + b], wb.b[b]);
}

// ------------------------------------------------------------------ mode counts
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

// ------------------------------------------------------------------ launch helpers
template <typename K> static void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define PSPEC_DISPATCH_E(E_, ...)      \
  do {                                 \
    if ((E_) == 24) {                  \
      constexpr int EE = 24;           \
      __VA_ARGS__;                     \
    } else {                           \
      constexpr int EE = 8;            \
      __VA_ARGS__;                     \
    }                                  \
  } while (0)

size_t smem_rows(int L, int rows, size_t csz) { return (size_t)rows * padded_len(L) * csz; }

template <typename T>
void launch_r2c_z(const T* in, cx<T>* out, const Geo& g, const FftPlan& pz, int E, const cx<T>* tw_half,
                  const cx<T>* twr, int rows, cudaStream_t s) {
  const size_t smem = smem_rows(g.NH, rows, sizeof(cx<T>));
  const int threads = rows * (g.NH / E);
  const unsigned grid = (unsigned)((int64_t)g.N * g.N / rows);
  PSPEC_DISPATCH_E(E, {
    set_smem(k_r2c_z<T, EE>, smem);
    k_r2c_z<T, EE><<<grid, threads, smem, s>>>(in, out, g, pz, tw_half, twr, rows);
  });
}

template <typename T>
void launch_c2r_z(const cx<T>* in, T* out, const Geo& g, const FftPlan& pz, int E, const cx<T>* tw_half,
                  const cx<T>* twr, int rows, T scale, cudaStream_t s) {
  const size_t smem = smem_rows(g.NH, rows, sizeof(cx<T>));
  const int threads = rows * (g.NH / E);
  const unsigned grid = (unsigned)((int64_t)g.N * g.N / rows);
  PSPEC_DISPATCH_E(E, {
    set_smem(k_c2r_z<T, EE>, smem);
    k_c2r_z<T, EE><<<grid, threads, smem, s>>>(in, out, g, pz, tw_half, twr, rows, scale);
  });
}

template <typename T> size_t smem_ylm_z(const Geo& g, int E, int M, int rows, int threads) {
  (void)E;
  (void)threads;
  const size_t stage = (size_t)M * rows * g.N * sizeof(T);
  const size_t xb = smem_rows(g.NH, M * rows, sizeof(cx<T>));
  return stage > xb ? stage : xb;
}

template <typename T>
void launch_ylm_r2c_z(const T* f, cx<T>* out, int64_t spec_stride, int ell, int h0, int M, const Geo& g,
                      const FftPlan& pz, int E, const cx<T>* tw_half, const cx<T>* twr, const T* axis_pos, int rows,
                      int threads, cudaStream_t s) {
  (void)threads;
  const size_t smem = smem_ylm_z<T>(g, E, M, rows, 0);
  const int nthreads = M * rows * (g.NH / E);
  const unsigned grid = (unsigned)((int64_t)g.N * g.N / rows);
  PSPEC_DISPATCH_E(E, {
    set_smem(k_ylm_r2c_z<T, EE>, smem);
    k_ylm_r2c_z<T, EE><<<grid, nthreads, smem, s>>>(f, out, spec_stride, ell, h0, M, g, pz, tw_half, twr, axis_pos,
                                                    rows);
  });
}

template <typename T> size_t smem_cols(const Geo& g, int tw) { return (size_t)g.N * tw * sizeof(cx<T>); }

template <typename T>
void launch_fft_y(cx<T>* data, int64_t spec_stride, int nspec, const Geo& g, const FftPlan& pf, int E,
                  const cx<T>* tw_full, int tw, int dir, cudaStream_t s) {
  const size_t smem = smem_cols<T>(g, tw);
  dim3 grid((unsigned)(g.N * (g.NH / tw)), (unsigned)nspec);
  const int threads = tw * (g.N / E);
  PSPEC_DISPATCH_E(E, {
    if (dir < 0) {
      set_smem(k_fft_y<T, EE, -1>, smem);
      k_fft_y<T, EE, -1><<<grid, threads, smem, s>>>(data, spec_stride, g, pf, tw_full, tw);
    } else {
      set_smem(k_fft_y<T, EE, 1>, smem);
      k_fft_y<T, EE, 1><<<grid, threads, smem, s>>>(data, spec_stride, g, pf, tw_full, tw);
    }
  });
}

template <typename T>
void launch_fft_x(const cx<T>* in, cx<T>* out, const Geo& g, const FftPlan& pf, int E, const cx<T>* tw_full, int tw,
                  int dir, cudaStream_t s) {
  const size_t smem = smem_cols<T>(g, tw);
  const int threads = tw * (g.N / E);
  const unsigned grid = (unsigned)(g.N * (g.NH / tw));
  PSPEC_DISPATCH_E(E, {
    if (dir < 0) {
      set_smem(k_fft_x<T, EE, -1>, smem);
      k_fft_x<T, EE, -1><<<grid, threads, smem, s>>>(in, out, g, pf, tw_full, tw);
    } else {
      set_smem(k_fft_x<T, EE, 1>, smem);
      k_fft_x<T, EE, 1><<<grid, threads, smem, s>>>(in, out, g, pf, tw_full, tw);
    }
  });
}

template <typename T> size_t smem_combine(const Geo& g, int E, int tw, int nk) {
  const int nw = (tw * (g.N / E) + 31) / 32;
  return smem_cols<T>(g, tw) + (size_t)nk * sizeof(double) + (size_t)nw * nk * sizeof(T);
}

template <typename T> size_t smem_bin_x(const Geo& g, int E, int tw, int nk) {
  const int nw = (tw * (g.N / E) + 31) / 32;
  return 2 * smem_cols<T>(g, tw) + (size_t)nk * sizeof(double) + (size_t)nw * nk * sizeof(T);
}

template <typename T>
void launch_combine_x(const cx<T>* B, cx<T>* F0, const Geo& g, const FftPlan& pf, int E, const cx<T>* tw_full, int tw,
                      int interlaced, int compensate, int roundtrip, const cx<T>* phase_axis, const T* invw_axis,
                      const BinArgs& ba, int ctas, cudaStream_t s) {
  const size_t smem = smem_combine<T>(g, E, tw, ba.nk);
  const int threads = tw * (g.N / E);
  PSPEC_DISPATCH_E(E, {
    set_smem(k_combine_x<T, EE>, smem);
    k_combine_x<T, EE><<<ctas, threads, smem, s>>>(B, F0, g, pf, tw_full, tw, interlaced, compensate, roundtrip,
                                                   phase_axis, invw_axis, ba);
  });
}

template <typename T>
void launch_bin_x(const cx<T>* G, int64_t spec_stride, int ell, int h0, int M, const cx<T>* F0, const Geo& g,
                  const FftPlan& pf, int E, const cx<T>* tw_full, int tw, int slot, const BinArgs& ba, int ctas,
                  cudaStream_t s) {
  const size_t smem = smem_bin_x<T>(g, E, tw, ba.nk);
  const int threads = tw * (g.N / E);
  PSPEC_DISPATCH_E(E, {
    set_smem(k_bin_x<T, EE>, smem);
    k_bin_x<T, EE><<<ctas, threads, smem, s>>>(G, spec_stride, ell, h0, M, F0, g, pf, tw_full, tw, slot, ba);
  });
}

void launch_mode_counts(const Geo& g, unsigned int* cnt, int nsm, cudaStream_t s) {
  k_mode_counts<<<8 * nsm, 256, 0, s>>>(g, cnt);
}

void launch_bin_counts(const unsigned int* cnt, const double* kmag, const int* lo, const int* hi, int nk,
                       double* nmodes, double* ksum, cudaStream_t s) {
  k_bin_counts<<<(nk + 127) / 128, 128, 0, s>>>(cnt, kmag, lo, hi, nk, nmodes, ksum);
}

// Persistent CTA counts from the occupancy of the binning passes.
template <typename T> int persistent_ctas(int which, const Geo& g, int E, int tw, int nk, int nsm) {
  const int threads = tw * (g.N / E);
  int per = 0;
  size_t smem;
  if (which == 0) {
    smem = smem_combine<T>(g, E, tw, nk);
    PSPEC_DISPATCH_E(E, {
      set_smem(k_combine_x<T, EE>, smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_combine_x<T, EE>, threads, smem);
    });
  } else {
    smem = smem_bin_x<T>(g, E, tw, nk);
    PSPEC_DISPATCH_E(E, {
      set_smem(k_bin_x<T, EE>, smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bin_x<T, EE>, threads, smem);
    });
  }
  if (per < 1) per = 1;
  const int ntiles = g.N * (g.NH / tw);
  return per * nsm < ntiles ? per * nsm : ntiles;
}

// ------------------------------------------------------------------ Y tables
template <typename T> static void build_ytab(YTab<T>& t) {
  double c[kLdim];
  c[0] = 1.0 / std::sqrt(4.0 * M_PI);
  for (int a = 1; a < kLdim; a++) c[a] = -std::sqrt((2.0 * a + 1.0) / (2.0 * a)) * c[a - 1];
  for (int i = 0; i < kLdim * kLdim; i++) {
    t.A[i] = T(0);
    t.B[i] = T(0);
  }
  for (int a = 0; a < kLdim; a++) t.c[a] = T(c[a]);
  for (int l = 1; l < kLdim; l++) {
    for (int a = 0; a < l; a++) {
      const double A = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)a * a));
      const double num = (double)(l - 1) * (l - 1) - (double)a * a;
      const double B = num > 0 ? std::sqrt(num / (4.0 * (l - 1) * (l - 1) - 1.0)) : 0.0;
      t.A[l * kLdim + a] = T(A);
      t.B[l * kLdim + a] = T(B);
    }
  }
}

cudaError_t upload_ylm_tables(cudaStream_t s) {
  static YTab<float> tf;
  static YTab<double> td;
  static bool built = false;
  if (!built) {
    build_ytab(tf);
    build_ytab(td);
    built = true;
  }
  cudaError_t e = cudaMemcpyToSymbolAsync(c_ytab_f, &tf, sizeof(tf), 0, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbolAsync(c_ytab_d, &td, sizeof(td), 0, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

// ------------------------------------------------------------------ instantiations
#define PSPEC_INST(T)                                                                                          \
  template void launch_r2c_z<T>(const T*, cx<T>*, const Geo&, const FftPlan&, int, const cx<T>*, const cx<T>*, \
                                int, cudaStream_t);                                                            \
  template void launch_c2r_z<T>(const cx<T>*, T*, const Geo&, const FftPlan&, int, const cx<T>*, const cx<T>*, \
                                int, T, cudaStream_t);                                                         \
  template void launch_ylm_r2c_z<T>(const T*, cx<T>*, int64_t, int, int, int, const Geo&, const FftPlan&, int,  \
                                    const cx<T>*, const cx<T>*, const T*, int, int, cudaStream_t);             \
  template void launch_fft_y<T>(cx<T>*, int64_t, int, const Geo&, const FftPlan&, int, const cx<T>*, int, int, \
                                cudaStream_t);                                                                 \
  template void launch_fft_x<T>(const cx<T>*, cx<T>*, const Geo&, const FftPlan&, int, const cx<T>*, int, int,  \
                                cudaStream_t);                                                                 \
  template void launch_combine_x<T>(const cx<T>*, cx<T>*, const Geo&, const FftPlan&, int, const cx<T>*, int,  \
                                    int, int, int, const cx<T>*, const T*, const BinArgs&, int, cudaStream_t); \
  template void launch_bin_x<T>(const cx<T>*, int64_t, int, int, int, const cx<T>*, const Geo&, const FftPlan&, \
                                int, const cx<T>*, int, int, const BinArgs&, int, cudaStream_t);               \
  template size_t smem_ylm_z<T>(const Geo&, int, int, int, int);                                                \
  template size_t smem_cols<T>(const Geo&, int);                                                               \
  template size_t smem_combine<T>(const Geo&, int, int, int);                                                  \
  template size_t smem_bin_x<T>(const Geo&, int, int, int);                                                    \
  template int persistent_ctas<T>(int, const Geo&, int, int, int, int);

PSPEC_INST(float)
PSPEC_INST(double)

}  // namespace pspec
