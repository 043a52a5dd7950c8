// Transform passes of the SH-FFT multipole estimator (Sec. 2.1 eqs. Pell-ours, Fell;
// Sec. 2.3 interlacing, compensation and the inverse transform before the Y_lm weights).
//
// Storage: real mesh r[(i*N + j)*N + k]; half spectrum s[(i*N + j)*NH + kz], NH = N/2.
// The kz = N/2 plane is never stored: its modes are zeroed before the inverse transform
// and never binned, so nothing downstream reads it.
//
// A 3-D forward transform is three passes, each one HBM round trip:
//   z: rows of N reals -> N/2-point complex FFT of packed pairs -> unpack to N/2 modes
//   y: columns along j of a (i, kz-tile) slab, in place
//   x: columns along i of a (j, kz-tile) slab; fused with the interlace/compensate
//      combine (F0) or with the Y_lm(khat) accumulate-and-bin reduction.
#include <cstdio>
#include <cmath>
#include "launch.h"

namespace pspec {

__constant__ YTab<float> c_ytab_f;
__constant__ YTab<double> c_ytab_d;
template <typename T> __device__ __forceinline__ const YTab<T>& ytab();
template <> __device__ __forceinline__ const YTab<float>& ytab<float>() { return c_ytab_f; }
template <> __device__ __forceinline__ const YTab<double>& ytab<double>() { return c_ytab_d; }

constexpr int kThreads = 256;

// ------------------------------------------------------------------ pass z: r2c of plain rows
template <typename T>
__global__ void __launch_bounds__(kThreads) k_r2c_z(const T* __restrict__ in, cx<T>* __restrict__ out,
                                                   Geo g, FftPlan pz, const cx<T>* __restrict__ twh,
                                                   const cx<T>* __restrict__ twr_g, int rows) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char sm[];
  const int L = g.NH;
  C* bufA = reinterpret_cast<C*>(sm);
  C* bufB = bufA + rows * L;
  C* tw = bufB + rows * L;
  C* twr = tw + L;
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    tw[t] = twh[t];
    twr[t] = twr_g[t];
  }
  const int64_t row0 = (int64_t)blockIdx.x * rows;
  const C* src = reinterpret_cast<const C*>(in + row0 * g.N);
  for (int t = threadIdx.x; t < rows * L; t += blockDim.x) bufA[t] = src[t];
  __syncthreads();
  C* res = fft_smem<C>(bufA, bufB, pz, rows, L, 1, false, tw, -1);
  C* dst = out + row0 * L;
  for (int t = threadIdx.x; t < rows * L; t += blockDim.x) {
    const int r = t / L, k = t - r * L;
    const C zk = res[r * L + k];
    const C zc = cconj(res[r * L + ((L - k) % L)]);
    const C e = cscale(cadd(zk, zc), T(0.5));
    const C d = csub(zk, zc);
    const C o = mk(T(0.5) * d.y, T(-0.5) * d.x);  // (zk - zc) * (-i/2)
    dst[t] = cadd(e, cmul(twr[k], o));
  }
}

// ------------------------------------------------------------------ pass z: Y_lm-weighted r2c
// For the rows of this CTA, writes DFT_z[f(x) Y_{l,m(h)}(rhat_x)] for the M harmonics
// h0..h0+M-1 of multipole l into M spectra. Each point sweeps its harmonics once:
// (x+iy)^a is carried from one |m| to the next.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_ylm_r2c_z(const T* __restrict__ f, cx<T>* __restrict__ out,
                                                       int64_t spec_stride, int ell, int h0, int M, Geo g,
                                                       FftPlan pz, const cx<T>* __restrict__ twh,
                                                       const cx<T>* __restrict__ twr_g,
                                                       const T* __restrict__ axis, int rows) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char sm[];
  const int N = g.N, L = g.NH;
  const int nseq = M * rows;
  C* bufA = reinterpret_cast<C*>(sm);
  C* bufB = bufA + nseq * L;
  C* tw = bufB + nseq * L;
  C* twr = tw + L;
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    tw[t] = twh[t];
    twr[t] = twr_g[t];
  }
  const YTab<T>& yt = ytab<T>();
  const int64_t row0 = (int64_t)blockIdx.x * rows;
  T* bufR = reinterpret_cast<T*>(bufA);
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
      for (int s = 0; s < M; s++) bufR[s * rows * N + p] = (ell == 0) ? fv * yt.c[0] : T(0);
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
      const T q = ylm_q<T>(yt, ell, a, z);
      if (a == 0) {
        if (h0 == 0) bufR[p] = fv * q;
      } else {
        const int hp = 2 * a - 1, hm = 2 * a;
        if (hp >= h0 && hp < h0 + M) bufR[(hp - h0) * rows * N + p] = fv * sq2 * q * pr;
        if (hm >= h0 && hm < h0 + M) bufR[(hm - h0) * rows * N + p] = fv * sq2 * q * pi;
      }
      const T nr = pr * x - pi * y;
      pi = pr * y + pi * x;
      pr = nr;
    }
  }
  __syncthreads();
  C* res = fft_smem<C>(bufA, bufB, pz, nseq, L, 1, false, tw, -1);
  for (int t = threadIdx.x; t < nseq * L; t += blockDim.x) {
    const int sq = t / L, k = t - sq * L;
    const int s = sq / rows, r = sq - s * rows;
    const C zk = res[sq * L + k];
    const C zc = cconj(res[sq * L + ((L - k) % L)]);
    const C e = cscale(cadd(zk, zc), T(0.5));
    const C d = csub(zk, zc);
    const C o = mk(T(0.5) * d.y, T(-0.5) * d.x);
    out[s * spec_stride + (row0 + r) * L + k] = cadd(e, cmul(twr[k], o));
  }
}

// ------------------------------------------------------------------ pass y (in place)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fft_y(cx<T>* __restrict__ data, int64_t spec_stride, Geo g,
                                                   FftPlan pf, const cx<T>* __restrict__ twf, int TW,
                                                   int dir) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char sm[];
  const int N = g.N, NH = g.NH;
  C* bufA = reinterpret_cast<C*>(sm);
  C* bufB = bufA + N * TW;
  C* tw = bufB + N * TW;
  for (int t = threadIdx.x; t < N; t += blockDim.x) tw[t] = twf[t];
  const int ntz = NH / TW;
  const int i = blockIdx.x / ntz, kz0 = (blockIdx.x - i * ntz) * TW;
  C* base = data + (int64_t)blockIdx.y * spec_stride + (int64_t)i * N * NH + kz0;
  for (int t = threadIdx.x; t < N * TW; t += blockDim.x) {
    const int jj = t / TW, c = t - jj * TW;
    bufA[t] = base[(int64_t)jj * NH + c];
  }
  __syncthreads();
  C* res = fft_smem<C>(bufA, bufB, pf, TW, 1, TW, true, tw, dir);
  for (int t = threadIdx.x; t < N * TW; t += blockDim.x) {
    const int jj = t / TW, c = t - jj * TW;
    base[(int64_t)jj * NH + c] = res[t];
  }
}

// ------------------------------------------------------------------ pass x (plain)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fft_x(const cx<T>* in, cx<T>* out, Geo g, FftPlan pf,
                                                   const cx<T>* __restrict__ twf, int TW, int dir) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char sm[];
  const int N = g.N, NH = g.NH;
  C* bufA = reinterpret_cast<C*>(sm);
  C* bufB = bufA + N * TW;
  C* tw = bufB + N * TW;
  for (int t = threadIdx.x; t < N; t += blockDim.x) tw[t] = twf[t];
  const int ntz = NH / TW;
  const int j = blockIdx.x / ntz, kz0 = (blockIdx.x - j * ntz) * TW;
  const int64_t stride_i = (int64_t)N * NH;
  const int64_t off = (int64_t)j * NH + kz0;
  for (int t = threadIdx.x; t < N * TW; t += blockDim.x) {
    const int ii = t / TW, c = t - ii * TW;
    bufA[t] = in[off + ii * stride_i + c];
  }
  __syncthreads();
  C* res = fft_smem<C>(bufA, bufB, pf, TW, 1, TW, true, tw, dir);
  for (int t = threadIdx.x; t < N * TW; t += blockDim.x) {
    const int ii = t / TW, c = t - ii * TW;
    out[off + ii * stride_i + c] = res[t];
  }
}

__device__ __forceinline__ int signed_freq(int i, int N) { return i < N / 2 ? i : i - N; }

// ------------------------------------------------------------------ pass x + combine (F0) + l=0 bins
// X = (F1 + exp(-i k.s) F2)/2 (interlaced) or F1, divided by W(k) when compensating,
// zeroed where some n_d = -N/2 when a round trip follows; stored as F0. Binned: N_b,
// sum |k|, sum |X|^2 with the half-spectrum multiplicity.
template <typename T, bool INTER, bool COMP, bool RT>
__global__ void __launch_bounds__(kThreads) k_combine_x(const cx<T>* B, cx<T>* F0, Geo g, FftPlan pf,
                                                       const cx<T>* __restrict__ twf, int TW,
                                                       const cx<T>* __restrict__ phase,
                                                       const T* __restrict__ invw, BinTabs bt) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char sm[];
  const int N = g.N, NH = g.NH;
  C* bufA = reinterpret_cast<C*>(sm);
  C* bufB = bufA + N * TW;
  C* tw = bufB + N * TW;
  double* sb = reinterpret_cast<double*>(tw + N);
  for (int t = threadIdx.x; t < N; t += blockDim.x) tw[t] = twf[t];
  for (int t = threadIdx.x; t < 3 * bt.nk; t += blockDim.x) sb[t] = 0.0;
  const int ntz = NH / TW;
  const int ntiles = N * ntz;
  const int64_t stride_i = (int64_t)N * NH;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int j = tile / ntz, kz0 = (tile - j * ntz) * TW;
    const int64_t off = (int64_t)j * NH + kz0;
    __syncthreads();
    for (int t = threadIdx.x; t < N * TW; t += blockDim.x) {
      const int ii = t / TW, c = t - ii * TW;
      bufA[t] = B[off + ii * stride_i + c];
    }
    __syncthreads();
    C* res = fft_smem<C>(bufA, bufB, pf, TW, 1, TW, true, tw, -1);
    const int ny = signed_freq(j, N);
    for (int t = threadIdx.x; t < N * TW; t += blockDim.x) {
      const int ii = t / TW, c = t - ii * TW;
      const int kz = kz0 + c;
      const int64_t addr = off + ii * stride_i + c;
      C X = res[t];
      if (INTER) {
        const C A = F0[addr];
        const C ph = cmul(cmul(phase[ii], phase[j]), phase[N + kz]);
        X = cscale(cadd(A, cmul(ph, X)), T(0.5));
      }
      if (COMP) X = cscale(X, invw[ii] * invw[j] * invw[N + kz]);
      const bool nyq = (ii == N / 2) || (j == N / 2);
      if (RT && nyq) X = mk(T(0), T(0));
      F0[addr] = X;
      if (!nyq) {
        const int nx = signed_freq(ii, N);
        const int n2 = nx * nx + ny * ny + kz * kz;
        const int b = bt.bin_of_n2[n2];
        if (b >= 0 && n2 > 0) {
          const double mult = kz ? 2.0 : 1.0;
          const double p2 = (double)X.x * (double)X.x + (double)X.y * (double)X.y;
          atomicAdd(&sb[b], mult);
          atomicAdd(&sb[bt.nk + b], mult * bt.kmag_of_n2[n2]);
          atomicAdd(&sb[2 * bt.nk + b], mult * p2);
        }
      }
    }
  }
  __syncthreads();
  double* part = bt.partials + (int64_t)blockIdx.x * bt.nslots * bt.nk;
  for (int t = threadIdx.x; t < bt.nk; t += blockDim.x) {
    part[SLOT_NMODES * bt.nk + t] += sb[t];
    part[SLOT_KSUM * bt.nk + t] += sb[bt.nk + t];
    part[SLOT_P0 * bt.nk + t] += sb[2 * bt.nk + t];
  }
}

// ------------------------------------------------------------------ pass x + accumulate-and-bin
// For each tile: F0 loaded once; for each harmonic h of the group, the x-pass of G_h and
// acc += Y_{l,m(h)}(khat) Re[G_h conj(F0)] per mode (FP32 or FP64, per mode); then
// acc x multiplicity is added to FP64 bins of slot `slot`.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_bin_x(const cx<T>* G, int64_t spec_stride, int ell, int h0,
                                                   int M, const cx<T>* __restrict__ F0, Geo g, FftPlan pf,
                                                   const cx<T>* __restrict__ twf, int TW, int slot,
                                                   BinTabs bt) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char sm[];
  const int N = g.N, NH = g.NH;
  C* bufA = reinterpret_cast<C*>(sm);
  C* bufB = bufA + N * TW;
  C* sF0 = bufB + N * TW;
  C* tw = sF0 + N * TW;
  T* acc = reinterpret_cast<T*>(tw + N);
  double* sb = reinterpret_cast<double*>(acc + N * TW);
  for (int t = threadIdx.x; t < N; t += blockDim.x) tw[t] = twf[t];
  for (int t = threadIdx.x; t < bt.nk; t += blockDim.x) sb[t] = 0.0;
  const YTab<T>& yt = ytab<T>();
  const int ntz = NH / TW;
  const int ntiles = N * ntz;
  const int64_t stride_i = (int64_t)N * NH;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int j = tile / ntz, kz0 = (tile - j * ntz) * TW;
    const int64_t off = (int64_t)j * NH + kz0;
    const int ny = signed_freq(j, N);
    __syncthreads();
    for (int t = threadIdx.x; t < N * TW; t += blockDim.x) {
      const int ii = t / TW, c = t - ii * TW;
      sF0[t] = F0[off + ii * stride_i + c];
      acc[t] = T(0);
    }
    for (int s = 0; s < M; s++) {
      const int h = h0 + s;
      const C* Gs = G + (int64_t)s * spec_stride;
      __syncthreads();
      for (int t = threadIdx.x; t < N * TW; t += blockDim.x) {
        const int ii = t / TW, c = t - ii * TW;
        bufA[t] = Gs[off + ii * stride_i + c];
      }
      __syncthreads();
      C* res = fft_smem<C>(bufA, bufB, pf, TW, 1, TW, true, tw, -1);
      for (int t = threadIdx.x; t < N * TW; t += blockDim.x) {
        const int ii = t / TW, c = t - ii * TW;
        const int nx = signed_freq(ii, N), kz = kz0 + c;
        const int n2 = nx * nx + ny * ny + kz * kz;
        if (n2 == 0) continue;
        const T Y = ylm_dir<T>(yt, ell, h, T(nx), T(ny), T(kz), T(n2));
        const C gv = res[t], fv = sF0[t];
        acc[t] += Y * (gv.x * fv.x + gv.y * fv.y);
      }
    }
    __syncthreads();
    if (j != N / 2) {
      for (int t = threadIdx.x; t < N * TW; t += blockDim.x) {
        const int ii = t / TW, c = t - ii * TW;
        if (ii == N / 2) continue;
        const int nx = signed_freq(ii, N), kz = kz0 + c;
        const int n2 = nx * nx + ny * ny + kz * kz;
        const int b = bt.bin_of_n2[n2];
        if (b >= 0 && n2 > 0) atomicAdd(&sb[b], (kz ? 2.0 : 1.0) * (double)acc[t]);
      }
    }
  }
  __syncthreads();
  double* part = bt.partials + ((int64_t)blockIdx.x * bt.nslots + slot) * bt.nk;
  for (int t = threadIdx.x; t < bt.nk; t += blockDim.x) part[t] += sb[t];
}

// ------------------------------------------------------------------ pass z: c2r
// Rows of N/2 stored modes (kz = N/2 taken as 0) -> N reals, times `scale`.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_c2r_z(const cx<T>* __restrict__ in, T* __restrict__ out, Geo g,
                                                   FftPlan pz, const cx<T>* __restrict__ twh,
                                                   const cx<T>* __restrict__ twr_g, int rows, T scale) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char sm[];
  const int L = g.NH;
  C* bufA = reinterpret_cast<C*>(sm);
  C* bufB = bufA + rows * L;
  C* tw = bufB + rows * L;
  C* twr = tw + L;
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    tw[t] = twh[t];
    twr[t] = twr_g[t];
  }
  const int64_t row0 = (int64_t)blockIdx.x * rows;
  const C* src = in + row0 * L;
  __syncthreads();
  for (int t = threadIdx.x; t < rows * L; t += blockDim.x) {
    const int r = t / L, k = t - r * L;
    const C xk = src[t];
    const C xm = k ? cconj(src[r * L + (L - k)]) : mk(T(0), T(0));
    const C e = cscale(cadd(xk, xm), T(0.5));
    const C o = cmul(cscale(csub(xk, xm), T(0.5)), cconj(twr[k]));
    bufA[t] = mk(e.x - o.y, e.y + o.x);  // e + i o
  }
  __syncthreads();
  C* res = fft_smem<C>(bufA, bufB, pz, rows, L, 1, false, tw, +1);
  C* dst = reinterpret_cast<C*>(out + row0 * g.N);
  for (int t = threadIdx.x; t < rows * L; t += blockDim.x) dst[t] = cscale(res[t], scale);
}

// ------------------------------------------------------------------ launch helpers
template <typename K>
static void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T>
void launch_r2c_z(const T* in, cx<T>* out, const Geo& g, const FftPlan& pz, const cx<T>* tw_half,
                  const cx<T>* twr, int rows, cudaStream_t s) {
  const size_t smem = (size_t)(2 * rows * g.NH + 2 * g.NH) * sizeof(cx<T>);
  set_smem(k_r2c_z<T>, smem);
  const int64_t nrows = (int64_t)g.N * g.N;
  k_r2c_z<T><<<(unsigned)(nrows / rows), kThreads, smem, s>>>(in, out, g, pz, tw_half, twr, rows);
}

template <typename T> size_t smem_ylm_z(const Geo& g, int M, int rows) {
  return (size_t)(2 * M * rows * g.NH + 2 * g.NH) * sizeof(cx<T>);
}

template <typename T>
void launch_ylm_r2c_z(const T* f, cx<T>* out, int64_t spec_stride, int ell, int h0, int M, const Geo& g,
                      const FftPlan& pz, const cx<T>* tw_half, const cx<T>* twr, const T* axis_pos,
                      int rows, cudaStream_t s) {
  const size_t smem = smem_ylm_z<T>(g, M, rows);
  set_smem(k_ylm_r2c_z<T>, smem);
  const int64_t nrows = (int64_t)g.N * g.N;
  k_ylm_r2c_z<T><<<(unsigned)(nrows / rows), kThreads, smem, s>>>(f, out, spec_stride, ell, h0, M, g, pz,
                                                                  tw_half, twr, axis_pos, rows);
}

template <typename T> size_t smem_fft_y(const Geo& g, int tw) {
  return (size_t)(2 * g.N * tw + g.N) * sizeof(cx<T>);
}

template <typename T>
void launch_fft_y(cx<T>* data, int64_t spec_stride, int nspec, const Geo& g, const FftPlan& pf,
                  const cx<T>* tw_full, int tw, int dir, cudaStream_t s) {
  const size_t smem = smem_fft_y<T>(g, tw);
  set_smem(k_fft_y<T>, smem);
  dim3 grid((unsigned)(g.N * (g.NH / tw)), (unsigned)nspec);
  k_fft_y<T><<<grid, kThreads, smem, s>>>(data, spec_stride, g, pf, tw_full, tw, dir);
}

template <typename T>
void launch_fft_x(const cx<T>* in, cx<T>* out, const Geo& g, const FftPlan& pf, const cx<T>* tw_full,
                  int tw, int dir, cudaStream_t s) {
  const size_t smem = smem_fft_y<T>(g, tw);
  set_smem(k_fft_x<T>, smem);
  k_fft_x<T><<<(unsigned)(g.N * (g.NH / tw)), kThreads, smem, s>>>(in, out, g, pf, tw_full, tw, dir);
}

template <typename T> size_t smem_combine(const Geo& g, int tw, int nk) {
  return (size_t)3 * nk * sizeof(double) + (size_t)(2 * g.N * tw + g.N) * sizeof(cx<T>);
}

template <typename T>
void launch_combine_x(const cx<T>* B, cx<T>* F0, const Geo& g, const FftPlan& pf, const cx<T>* tw_full,
                      int tw, int interlaced, int compensate, int roundtrip, const cx<T>* phase_axis,
                      const T* invw_axis, const BinTabs& bt, cudaStream_t s) {
  const size_t smem = smem_combine<T>(g, tw, bt.nk);
  auto pick = [&](auto kern) {
    set_smem(kern, smem);
    kern<<<bt.ctas, kThreads, smem, s>>>(B, F0, g, pf, tw_full, tw, phase_axis, invw_axis, bt);
  };
  const int key = (interlaced ? 4 : 0) | (compensate ? 2 : 0) | (roundtrip ? 1 : 0);
  switch (key) {
    case 0: pick(k_combine_x<T, false, false, false>); break;
    case 1: pick(k_combine_x<T, false, false, true>); break;
    case 2: pick(k_combine_x<T, false, true, false>); break;
    case 3: pick(k_combine_x<T, false, true, true>); break;
    case 4: pick(k_combine_x<T, true, false, false>); break;
    case 5: pick(k_combine_x<T, true, false, true>); break;
    case 6: pick(k_combine_x<T, true, true, false>); break;
    default: pick(k_combine_x<T, true, true, true>); break;
  }
}

template <typename T> size_t smem_bin_x(const Geo& g, int tw) {
  // bins are added separately (nk doubles)
  return (size_t)(3 * g.N * tw + g.N) * sizeof(cx<T>) + (size_t)g.N * tw * sizeof(T);
}

template <typename T>
void launch_bin_x(const cx<T>* G, int64_t spec_stride, int ell, int h0, int M, const cx<T>* F0,
                  const Geo& g, const FftPlan& pf, const cx<T>* tw_full, int tw, int slot,
                  const BinTabs& bt, cudaStream_t s) {
  const size_t smem = smem_bin_x<T>(g, tw) + (size_t)bt.nk * sizeof(double);
  set_smem(k_bin_x<T>, smem);
  k_bin_x<T><<<bt.ctas, kThreads, smem, s>>>(G, spec_stride, ell, h0, M, F0, g, pf, tw_full, tw, slot, bt);
}

template <typename T>
void launch_c2r_z(const cx<T>* in, T* out, const Geo& g, const FftPlan& pz, const cx<T>* tw_half,
                  const cx<T>* twr, int rows, T scale, cudaStream_t s) {
  const size_t smem = (size_t)(2 * rows * g.NH + 2 * g.NH) * sizeof(cx<T>);
  set_smem(k_c2r_z<T>, smem);
  const int64_t nrows = (int64_t)g.N * g.N;
  k_c2r_z<T><<<(unsigned)(nrows / rows), kThreads, smem, s>>>(in, out, g, pz, tw_half, twr, rows, scale);
}

template <typename T> int bin_x_ctas(const Geo& g, int tw, int nsm, int nk_max) {
  const size_t smem = smem_bin_x<T>(g, tw) + (size_t)nk_max * sizeof(double);
  set_smem(k_bin_x<T>, smem);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bin_x<T>, kThreads, smem);
  if (per < 1) per = 1;
  const int ntiles = g.N * (g.NH / tw);
  return per * nsm < ntiles ? per * nsm : ntiles;
}

template <typename T> int combine_x_ctas(const Geo& g, int tw, int nsm, int nk_max) {
  const size_t smem = smem_combine<T>(g, tw, nk_max);
  auto kern = k_combine_x<T, true, true, true>;
  set_smem(kern, smem);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, smem);
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
#define PSPEC_INST(T)                                                                                     \
  template void launch_r2c_z<T>(const T*, cx<T>*, const Geo&, const FftPlan&, const cx<T>*, const cx<T>*, \
                                int, cudaStream_t);                                                       \
  template void launch_ylm_r2c_z<T>(const T*, cx<T>*, int64_t, int, int, int, const Geo&, const FftPlan&, \
                                    const cx<T>*, const cx<T>*, const T*, int, cudaStream_t);             \
  template void launch_fft_y<T>(cx<T>*, int64_t, int, const Geo&, const FftPlan&, const cx<T>*, int, int, \
                                cudaStream_t);                                                            \
  template void launch_fft_x<T>(const cx<T>*, cx<T>*, const Geo&, const FftPlan&, const cx<T>*, int, int, \
                                cudaStream_t);                                                            \
  template void launch_combine_x<T>(const cx<T>*, cx<T>*, const Geo&, const FftPlan&, const cx<T>*, int, \
                                    int, int, int, const cx<T>*, const T*, const BinTabs&, cudaStream_t); \
  template void launch_bin_x<T>(const cx<T>*, int64_t, int, int, int, const cx<T>*, const Geo&,           \
                                const FftPlan&, const cx<T>*, int, int, const BinTabs&, cudaStream_t);    \
  template void launch_c2r_z<T>(const cx<T>*, T*, const Geo&, const FftPlan&, const cx<T>*, const cx<T>*, \
                                int, T, cudaStream_t);                                                    \
  template int bin_x_ctas<T>(const Geo&, int, int, int);                                                  \
  template int combine_x_ctas<T>(const Geo&, int, int, int);                                              \
  template size_t smem_combine<T>(const Geo&, int, int);                                                  \
  template size_t smem_fft_y<T>(const Geo&, int);                                                         \
  template size_t smem_bin_x<T>(const Geo&, int);                                                         \
  template size_t smem_ylm_z<T>(const Geo&, int, int);

PSPEC_INST(float)
PSPEC_INST(double)

}  // namespace pspec
