// Transform passes of the SH-FFT multipole estimator (Sec. 2.1 eqs. Pell-ours, Fell;
// Sec. 2.3 interlacing, compensation and the inverse transform before the Y_lm weights),
// as templates on the mesh side N; each supported N is instantiated in its own translation
// unit (pass_<N>.cu) and reached through a PassTable.
//
// Storage: real mesh r[(i*N + j)*N + k]; half spectrum (NH = N/2 stored kz) in kz tiles of TW
// modes, each tile an (i, j) plane of TW-mode rows (Lay below). The kz = N/2 plane is never
// stored: its modes are zeroed before the inverse transform and never binned, so nothing
// downstream reads it.
//
// A 3-D forward transform is three passes, each one HBM round trip:
//   z: rows of N reals -> N/2-point complex FFT of packed pairs -> unpack to N/2 modes
//   y: columns along j of an (i, kz-tile) slab, in place
//   x: columns along i of a (j, kz-tile) slab; fused with the interlace/compensate
//      combine (F0 and the l = 0 sums) or with the Y_lm(khat) accumulate-and-bin.
// Every pass keeps its elements in registers (fft_engine.cuh).
#pragma once
#include <cmath>
#include "launch.h"
#include "fft_engine.cuh"
#include "xp_engine.cuh"

namespace pspec {

// ------------------------------------------------------------------ compile-time shapes
template <int N> struct Shape {
  static constexpr int NH = N / 2;
  static constexpr int E = elems_for(N);
  static constexpr int EY = (N == 512) ? 32 : E;  // elements per thread in the y pass (512 = 32 x 16)
  static constexpr int TcY = N / EY;               // threads per column in the y pass
  static constexpr int EX = EY;                    // ... in the plain x pass
  static constexpr int TcX = N / EX;
  // Exact-add y and plain x passes (FP32): no radix-32 stage (its 32 pairs h + l would not fit
  // in registers), 512 = 16 x 16 x 2 with 16 elements per thread.
  static constexpr int EYX = (N == 512) ? 16 : E;
  static constexpr int TcYX = N / EYX;
  static constexpr int EZ = z_elems(N);  // elements per thread in the z passes
  static constexpr int Tz = NH / EZ;     // threads per row in the z passes
  static constexpr bool ZW = Tz <= 32;   // a z row within one warp: warp-level barriers suffice
  static constexpr int Tc = N / E;       // threads per column in the y / x passes
  static constexpr int TW = col_tile(N); // kz columns per tile
  static constexpr int ROWS = z_rows(N); // rows per block in the plain z passes
  static constexpr int CT = TW * Tc;     // threads of a column block
  static constexpr int CTX = TW * TcX;   // threads of a plain x-pass block
  static constexpr int ZT = ROWS * Tz;   // threads of a row block
};

// Row shapes of the z passes: the plain ones (Shape), or for exact-add stages (XP) at most 8
// elements per thread (16 pairs h + l would not fit in registers at the occupancy these passes
// need), the same threads per block.
template <int N, bool XP> struct ZShape {
  using S = Shape<N>;
  static constexpr int E = (XP && S::EZ == 16) ? 8 : S::EZ;
  static constexpr int Tz = S::NH / E;
  static constexpr bool ZW = Tz <= 32;
  static constexpr int ROWS = (S::ROWS * S::Tz / Tz) > 0 ? (S::ROWS * S::Tz / Tz) : 1;
  static constexpr int ZT = ROWS * Tz;
};

// ------------------------------------------------------------------ spectrum storage order
// s[((kz / TW * N + i) * N + j) * TW + kz % TW]: a y-pass slab (i, kz tile) is one contiguous
// block, an x-pass tile (j, kz tile) is N rows of TW modes N*TW modes apart, and a z-pass block
// of consecutive rows writes a run of rows*TW modes into each kz tile. (With rows of TW modes
// N*N/2 modes apart, the order of rows along kz, the x passes ran at about 3/4 of this order's
// bandwidth: the requests of the concurrent tiles fell into too few DRAM channels.)
template <int N> struct Lay {
  static constexpr int TW = Shape<N>::TW;
  static constexpr int64_t KT = (int64_t)N * N * TW;  // between kz tiles
  static constexpr int64_t XI = (int64_t)N * TW;      // between i: the x passes' element stride
  static constexpr int64_t YJ = TW;                   // between j: the y pass's element stride
  // mode kz of z-pass row r = i N + j
  __device__ static __forceinline__ int64_t row(int64_t r, int kz) { return (int64_t)(kz / TW) * KT + r * TW + kz % TW; }
  __device__ static __forceinline__ int64_t at(int i, int j, int kz) { return row((int64_t)i * N + j, kz); }
  // first mode of the k-space table block of x tile (j, kz tile kt); element (i, c) at + i TW + c
  __device__ static __forceinline__ int64_t table_tile(int kt, int j) { return ((int64_t)kt * N + j) * N * TW; }
};

// Resident blocks per SM the register allocation must allow. Threads holding 24 complex
// elements (3 * 2^a meshes) get at least 128 registers in FP32; 8 elements fit in 64.
template <typename T, int E> constexpr int min_blocks(int threads) {
  if constexpr (sizeof(T) != 4) return 1;
  if constexpr (E > 8) return threads >= 512 ? 1 : 65536 / (((threads + 31) / 32) * 32 * 128);
  return threads >= 512 ? 2 : (threads >= 256 ? 3 : 4);
}

template <int N> __device__ __forceinline__ int sfreq(int i) { return i < N / 2 ? i : i - N; }

// r2c unpack: X[k] = (Z[k] + Z*[L-k])/2 - i/2 w^k (Z[k] - Z*[L-k]), w = exp(-2 pi i/N)
template <typename C, typename T>
__device__ __forceinline__ C r2c_unpack(C zk, C zm, ux<T> w) {
  const C zc = cconj(zm);
  const C e = cscale(cadd(zk, zc), T(0.5));
  const C d = csub(zk, zc);
  const C o = mk(T(0.5) * d.y, T(-0.5) * d.x);
  return cadd(e, umul(o, w));
}

// X[L - k] for each output k = t + Tc e this thread holds after a row transform, fetched with
// shuffles from the thread holding it (lane Tc - t of the row, element E - 1 - e); thread 0
// holds its own mirrors (k = Tc e -> Tc (E - e), and X[0] for k = 0). Rows within one warp.
template <typename C, int E, int Tc>
__device__ __forceinline__ void row_mirrors(const C (&v)[E], C (&zm)[E], int t) {
  static_assert(Tc <= 32 && (Tc & (Tc - 1)) == 0, "row within a warp");
  const int src = (Tc - t) & (Tc - 1);
#pragma unroll
  for (int e = 0; e < E; e++) {
    C w;
    w.x = __shfl_sync(0xffffffffu, v[E - 1 - e].x, src, Tc);
    w.y = __shfl_sync(0xffffffffu, v[E - 1 - e].y, src, Tc);
    zm[e] = t ? w : v[(E - e) % E];
  }
}

// v / W(k)^2 for the mode (ii, j, kz), 1/W = prod_d hi_d (1 + lo_d) from the per-axis table: the
// relative errors lo_d enter the rounding of the exact product v * p^2 (compensation per mode).
template <typename T, int N>
__device__ __forceinline__ T per_mode_w2(T v, const cx<T>* __restrict__ iw, int ii, int j, int kz) {
  const cx<T> a = iw[ii], b = iw[j], c = iw[N + kz];
  const T p = a.x * b.x * c.x, p2 = p * p, l2 = T(2) * (a.y + b.y + c.y);
  return fma_t(v, p2, v * p2 * l2);
}

// ------------------------------------------------------------------ pass z: r2c of plain rows
template <typename T, int N>
__global__ void __launch_bounds__(Shape<N>::ZT, min_blocks<T, Shape<N>::EZ>(Shape<N>::ZT))
    k_r2c_z(const T* __restrict__ in, cx<T>* __restrict__ out, const ux<T>* __restrict__ twh,
            const ux<T>* __restrict__ twr) {
  using C = cx<T>;
  using S = Shape<N>;
  constexpr int L = S::NH, E = S::EZ, Tc = S::Tz;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int r = threadIdx.x / Tc, t = threadIdx.x - r * Tc;
  const int row = blockIdx.x * S::ROWS + r;
  const C* src = reinterpret_cast<const C*>(in + (int64_t)row * N);
  C v[E];
#pragma unroll
  for (int e = 0; e < E; e++) v[e] = src[t + Tc * e];
  fft_ct<C, E, L, kPaddedRows, 1, -1, S::ZW>(v, sm, t, r, twh);
  C zm[E];
  if constexpr (S::ZW) {
    row_mirrors<C, E, Tc>(v, zm, t);
  } else {
#pragma unroll
    for (int e = 0; e < E; e++) sm[sidx<kPaddedRows, L, 1>(r, t + Tc * e)] = v[e];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; e++) {
      const int k = t + Tc * e;
      zm[e] = sm[sidx<kPaddedRows, L, 1>(r, k ? L - k : 0)];
    }
  }
#pragma unroll
  for (int e = 0; e < E; e++) {
    const int k = t + Tc * e;
    out[Lay<N>::row(row, k)] = r2c_unpack<C, T>(v[e], zm[e], ldg_u(twr + k));
  }
}

// ------------------------------------------------------------------ pass z: c2r
// Rows of L stored modes (the kz = N/2 mode taken as 0) -> N reals, times `scale`.
// XP: exact-add pack and stages (FP32 only).
template <typename T, int N, bool XP>
__global__ void __launch_bounds__(ZShape<N, XP>::ZT, min_blocks<T, ZShape<N, XP>::E>(ZShape<N, XP>::ZT))
    k_c2r_z(const cx<T>* __restrict__ in, T* __restrict__ out, const ux<T>* __restrict__ twh,
            const ux<T>* __restrict__ twr, T scale) {
  using C = cx<T>;
  using S = ZShape<N, XP>;
  constexpr int L = N / 2, E = S::E, Tc = S::Tz;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int r = threadIdx.x / Tc, t = threadIdx.x - r * Tc;
  const int row = blockIdx.x * S::ROWS + r;
  C v[E];
#pragma unroll
  for (int e = 0; e < E; e++) {
    const int k = t + Tc * e;
    const C xk = in[Lay<N>::row(row, k)];
    if constexpr (XP) {
      v[e] = c2r_pack_xp(xk, k ? in[Lay<N>::row(row, L - k)] : mk(T(0), T(0)), uconj(ldg_u(twr + k)));
    } else {
      const C xm = k ? cconj(in[Lay<N>::row(row, L - k)]) : mk(T(0), T(0));
      const C ev = cscale(cadd(xk, xm), T(0.5));
      const C od = umul(cscale(csub(xk, xm), T(0.5)), uconj(ldg_u(twr + k)));
      v[e] = mk(ev.x - od.y, ev.y + od.x);  // E + i O
    }
  }
  fft_any<XP, C, E, L, kPaddedRows, 1, +1, S::ZW>(v, sm, t, r, twh);
  C* dst = reinterpret_cast<C*>(out + (int64_t)row * N);
#pragma unroll
  for (int e = 0; e < E; e++) dst[t + Tc * e] = cscale(v[e], scale);
}

// ------------------------------------------------------------------ pass z: Y_lm-weighted r2c
// For `rows` rows of f and the M harmonics h0..h0+M-1 of multipole l. Every point sweeps
// its harmonics once ((x+iy)^a carried from one |m| to the next) into a shared staging
// area of nseq = M*rows real rows; then each of the nseq*Tz threads loads its slots, the
// sequences are transformed (the staging area is reused as the exchange buffer) and unpacked
// into the M spectra. With the Y_lm(rhat) table and sequences within one warp, each thread loads
// its own slots of f and of the table and multiplies them in registers: no staging, and no block
// barrier.
template <typename T, int N, int LT, bool XP>
__global__ void __launch_bounds__(ylm_thread_cap(LT), sizeof(T) == 4 ? ylm_min_blocks(LT, XP) : 0) k_ylm_r2c_z(const T* __restrict__ f, cx<T>* __restrict__ out,
                                                  int64_t spec_stride, int ell, int h0, int M,
                                                  const ux<T>* __restrict__ twh, const ux<T>* __restrict__ twr,
                                                  const T* __restrict__ axis, int rows,
                                                  const float* __restrict__ rtab,
                                                  const __grid_constant__ YTab<T> yt) {
  using C = cx<T>;
  using S = ZShape<N, XP>;
  constexpr int L = N / 2, E = S::E, Tc = S::Tz;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* stage = reinterpret_cast<T*>(smraw);  // [nseq][N] reals, then the exchange buffer
  C* xb = reinterpret_cast<C*>(smraw);
  const int row0 = blockIdx.x * rows;
  const int a_lo = LT < 0 ? 0 : harm_a(h0), a_hi = LT < 0 ? 0 : harm_a(h0 + M - 1);
  const int sq = threadIdx.x / Tc, t = threadIdx.x - sq * Tc;
  C v[E];
  constexpr bool kWarpTable = sizeof(T) == 4 && LT >= 0 && S::ZW;
  const bool warp_local = kWarpTable && rtab != nullptr;  // uniform over the block
  if constexpr (kWarpTable) {
    if (rtab) {
      // the Tc threads of sequence (s, r) load their own slots: complex slot k of the row packs
      // f Y_lm(rhat) of nodes 2k and 2k + 1
      constexpr int64_t pts = (int64_t)N * N * N;
      const int s = sq / rows, r = sq - s * rows;
      const int64_t at0 = (int64_t)(row0 + r) * N;
      const float2* fr = reinterpret_cast<const float2*>(f + at0);
      const float2* yr = reinterpret_cast<const float2*>(rtab + (int64_t)s * pts + at0);
#pragma unroll
      for (int e = 0; e < E; e++) {
        const float2 a = __ldg(fr + t + Tc * e), b = __ldg(yr + t + Tc * e);
        v[e] = mk(a.x * b.x, a.y * b.y);
      }
    }
  } else if constexpr (sizeof(T) == 4 && LT >= 0) {
    if (rtab) {
      // Y_lm(rhat) from the table (harmonics h0.., one slot of N^3 nodes each): each thread takes
      // one 4-node vector of one row, loads f once and the M table vectors back to back
      constexpr int64_t pts = (int64_t)N * N * N;
      constexpr int NV = N / 4;
      for (int q = threadIdx.x; q < rows * NV; q += blockDim.x) {
        const int r = q / NV, kv = q - r * NV;
        const int64_t at = (int64_t)(row0 + r) * N + 4 * kv;
        const float4 fv = __ldg(reinterpret_cast<const float4*>(f + at));
        const float* trow = rtab + at;
#pragma unroll 4
        for (int s = 0; s < M; s++) {
          const float4 y = __ldg(reinterpret_cast<const float4*>(trow + s * pts));
          *reinterpret_cast<float4*>(stage + (s * rows + r) * N + 4 * kv) =
              make_float4(fv.x * y.x, fv.y * y.y, fv.z * y.z, fv.w * y.w);
        }
      }
    }
  }
  for (int r = 0; r < rows; r++) {
    const int grow = row0 + r;
    if constexpr (sizeof(T) == 4 && LT >= 0) {
      if (rtab) continue;
    }
    const int i = grow / N, j = grow - i * N;
    const T vx = axis[i], vy = axis[N + j];
    const T* frow = f + (int64_t)grow * N;
    for (int kk = threadIdx.x; kk < N; kk += blockDim.x) {
      const T fv = frow[kk];
      const T vz = axis[2 * N + kk];
      const T r2 = vx * vx + vy * vy + vz * vz;
      if (r2 == T(0)) {
        for (int s = 0; s < M; s++) stage[(s * rows + r) * N + kk] = T(0);
        continue;
      }
      if constexpr (LT < 0) {
        // Cartesian decomposition: weights rhat^q of the monomials h0..h0+M-1 of degree -LT
        // (refined 1/|r|: the shot noise cancels only in the final combination of degrees)
        const T inv = rsqrt_t<T>(r2);
        const T x = vx * inv, y = vy * inv, z = vz * inv;
        for (int s = 0; s < M; s++) {
          int ea, eb, ec;
          cart_exp((LT == -4 ? 6 : 0) + h0 + s, ea, eb, ec);
          stage[(s * rows + r) * N + kk] = fv * (ipow(x, ea) * ipow(y, eb) * ipow(z, ec));
        }
        continue;
      }
      const T inv = rsqrt_t<T>(r2);
      const T x = vx * inv, y = vy * inv, z = vz * inv;
      T pr = T(1), pi = T(0);
      if constexpr (LT > 0) {
        // l known at compile time: every recurrence unrolled with constant coefficient offsets
#pragma unroll
        for (int a = 0; a <= LT; a++) {
          if (a >= a_lo && a <= a_hi) {
            const T q = ylm_qt<T, true>(yt, LT, a, z);
            if (a == 0) {
              stage[r * N + kk] = fv * ylm_norm(yt, 0, q);
            } else {
              const int hp = 2 * a - 1, hm = 2 * a;
              if (hp >= h0 && hp < h0 + M) stage[((hp - h0) * rows + r) * N + kk] = fv * ylm_norm(yt, a, q * pr);
              if (hm >= h0 && hm < h0 + M) stage[((hm - h0) * rows + r) * N + kk] = fv * ylm_norm(yt, a, q * pi);
            }
          }
          const T nr = pr * x - pi * y;
          pi = pr * y + pi * x;
          pr = nr;
        }
      } else {
        for (int s = 0; s < a_lo; s++) {
          const T nr = pr * x - pi * y;
          pi = pr * y + pi * x;
          pr = nr;
        }
        for (int a = a_lo; a <= a_hi; a++) {
          const T q = ylm_qt<T, true>(yt, ell, a, z);
          if (a == 0) {
            stage[r * N + kk] = fv * ylm_norm(yt, 0, q);
          } else {
            const int hp = 2 * a - 1, hm = 2 * a;
            if (hp >= h0 && hp < h0 + M) stage[((hp - h0) * rows + r) * N + kk] = fv * ylm_norm(yt, a, q * pr);
            if (hm >= h0 && hm < h0 + M) stage[((hm - h0) * rows + r) * N + kk] = fv * ylm_norm(yt, a, q * pi);
          }
          const T nr = pr * x - pi * y;
          pi = pr * y + pi * x;
          pr = nr;
        }
      }
    }
  }
  if (!warp_local) {
    __syncthreads();
    const C* stc = reinterpret_cast<const C*>(stage);
#pragma unroll
    for (int e = 0; e < E; e++) v[e] = stc[sq * L + t + Tc * e];
    __syncthreads();  // the staging area becomes the exchange buffer
  }
  fft_any<XP, C, E, L, kPaddedRows, 1, -1, S::ZW>(v, xb, t, sq, twh);
  // mirrors through shared memory (shuffles would raise this kernel's register count, measured slower)
#pragma unroll
  for (int e = 0; e < E; e++) xb[sidx<kPaddedRows, L, 1>(sq, t + Tc * e)] = v[e];
  fft_sync<S::ZW>();
  const int s = sq / rows, r = sq - s * rows;
  C* dst = out + s * spec_stride;
  const int64_t grow = row0 + r;
#pragma unroll
  for (int e = 0; e < E; e++) {
    const int k = t + Tc * e;
    const C zm = xb[sidx<kPaddedRows, L, 1>(sq, k ? L - k : 0)];
    if constexpr (XP)
      dst[Lay<N>::row(grow, k)] = r2c_unpack_xp(v[e], zm, ldg_u(twr + k));
    else
      dst[Lay<N>::row(grow, k)] = r2c_unpack<C, T>(v[e], zm, ldg_u(twr + k));
  }
}

// ------------------------------------------------------------------ pass y (in place)
// Block: one (i, kz-tile) slab, TW columns x Tc threads (column fastest); blocks in storage
// order (kz tile, i, part of the tile when TW is a fraction of the storage tile). Outputs (ky, kz)
// with ky^2 + kz^2 >= n2_cut are not stored: every mode of their x column lies beyond the
// last bin, and the binning pass skips those columns (INT_MAX stores everything).
// XP: exact-add stages (FP32 only).
template <int N, bool XP> constexpr int col_elems() { return XP ? Shape<N>::EYX : Shape<N>::EY; }

// Exact-add blocks of 256 threads: three per SM (80 registers) beat two (104), measured.
template <int N, bool XP> constexpr int y_min_blocks(int threads) {
  return XP && threads == 256 ? 3 : min_blocks<float, col_elems<N, XP>()>(threads);
}
template <typename T, int N, int DIR, int TW, bool XP>
__global__ void __launch_bounds__(TW * (N / col_elems<N, XP>()),
                                  sizeof(T) == 4 ? y_min_blocks<N, XP>(TW * (N / col_elems<N, XP>()))
                                                 : min_blocks<T, col_elems<N, XP>()>(TW * (N / col_elems<N, XP>())))
    k_fft_y(cx<T>* __restrict__ data, int64_t spec_stride, const ux<T>* __restrict__ twf, int n2_cut) {
  using C = cx<T>;
  using S = Shape<N>;
  constexpr int NH = S::NH, E = col_elems<N, XP>(), Tc = N / E;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  static_assert(Lay<N>::TW % TW == 0, "a y tile lies within one storage tile");
  constexpr int SUB = Lay<N>::TW / TW;
  const int c = threadIdx.x % TW, t = threadIdx.x / TW;
  const int part = blockIdx.x % SUB, slab = blockIdx.x / SUB, kt = slab / N, i = slab - kt * N;
  const int kz0 = kt * Lay<N>::TW + part * TW;
  if (kz0 * kz0 >= n2_cut) return;  // the whole slab is beyond the last bin (uniform per block)
  const int kz = kz0 + c;
  C* base = data + (int64_t)blockIdx.y * spec_stride + Lay<N>::at(i, 0, kz);
  C v[E];
#pragma unroll
  for (int e = 0; e < E; e++) v[e] = base[(int64_t)(t + Tc * e) * Lay<N>::YJ];
  fft_any<XP, C, E, N, kInterleaved, TW, DIR>(v, sm, t, c, twf);
#pragma unroll
  for (int e = 0; e < E; e++) {
    const int ny = sfreq<N>(t + Tc * e);
    if (ny * ny + kz * kz < n2_cut) base[(int64_t)(t + Tc * e) * Lay<N>::YJ] = v[e];
  }
}

// ------------------------------------------------------------------ pass x (plain)
template <typename T, int N, int DIR, bool XP>
__global__ void __launch_bounds__(Shape<N>::TW * (N / col_elems<N, XP>()),
                                  min_blocks<T, col_elems<N, XP>()>(Shape<N>::TW * (N / col_elems<N, XP>())))
    k_fft_x(const cx<T>* in, cx<T>* out, const ux<T>* __restrict__ twf) {
  using C = cx<T>;
  using S = Shape<N>;
  constexpr int NH = S::NH, E = col_elems<N, XP>(), Tc = N / E, TW = S::TW;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int c = threadIdx.x % TW, t = threadIdx.x / TW;
  const int kt = blockIdx.x / N, j = blockIdx.x - kt * N;  // tiles in storage order
  constexpr int64_t si = Lay<N>::XI;
  const int64_t off = Lay<N>::at(0, j, kt * TW + c);
  C v[E];
#pragma unroll
  for (int e = 0; e < E; e++) v[e] = in[off + (t + Tc * e) * si];
  fft_any<XP, C, E, N, kInterleaved, TW, DIR>(v, sm, t, c, twf);
#pragma unroll
  for (int e = 0; e < E; e++) out[off + (t + Tc * e) * si] = v[e];
}

// ------------------------------------------------------------------ pass x + combine (F0) + l = 0 sums
// X = (F1 + exp(-i k.s) F2)/2 (interlaced) or F1; divided by W(k) when compensating; zeroed
// where some n_d = -N/2 when the inverse transform follows; stored as F0.
// Binned: sum over modes of mult |X|^2 (slot SLOT_P0). Persistent over tiles.
template <typename T, int N>
__global__ void __launch_bounds__(Shape<N>::CT, min_blocks<T, Shape<N>::E>(Shape<N>::CT))
    k_combine_x(const cx<T>* B, cx<T>* F0, const ux<T>* __restrict__ twf, int interlaced, int compensate,
                int roundtrip, const ux<T>* __restrict__ phase, const cx<T>* __restrict__ invw, BinArgs ba) {
  using C = cx<T>;
  using S = Shape<N>;
  constexpr int NH = S::NH, E = S::E, Tc = S::Tc, TW = S::TW;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  WarpBins<T> wb;
  wb.nk = ba.nk;
  wb.nwarps = (S::CT + 31) >> 5;
  wb.b = reinterpret_cast<double*>(sm + N * TW);
  wb.w = reinterpret_cast<T*>(wb.b + ba.nk);
  wb.init();
  const int c = threadIdx.x % TW, t = threadIdx.x / TW;
  constexpr int ntiles = N * (NH / TW);
  constexpr int64_t si = Lay<N>::XI;
  __syncthreads();
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int kt = tile / N, j = tile - kt * N;  // tiles in storage order
    const int kz = kt * TW + c;
    const int64_t off = Lay<N>::at(0, j, kz);
    C v[E];
#pragma unroll
    for (int e = 0; e < E; e++) v[e] = B[off + (t + Tc * e) * si];
    fft_ct<C, E, N, kInterleaved, TW, -1>(v, sm, t, c, twf);
    const int ny = sfreq<N>(j);
    const C iwy = ldg_c(invw + j), iwz = ldg_c(invw + N + kz);
    const T wyz = iwy.x * iwz.x, lyz = iwy.y + iwz.y;
    const int syz = sfreq<N>(j) + kz + 3 * N / 2;  // index of exp(-i pi (nx + ny + nz) / N) less nx
    const T mult = kz ? T(2) : T(1);
#pragma unroll
    for (int e = 0; e < E; e++) {
      const int ii = t + Tc * e;
      const int64_t addr = off + ii * si;
      C X = v[e];
      if (interlaced) {
        const C A = F0[addr];
        X = cscale(cadd(A, umul(X, ldg_u(phase + syz + sfreq<N>(ii)))), T(0.5));
      }
      if (compensate == 1 || compensate == 2) {
        // 1/W = prod_d hi_d (1 + lo_d): the relative rounding errors lo_d of the per-axis
        // factors enter the roundings of the products X * w3, so that no per-axis
        // deterministic error is left on the modes
        const C iwx = ldg_c(invw + ii);
        const T w3 = iwx.x * wyz, l3 = iwx.y + lyz;
        X = mk(fma_t(X.x, w3, X.x * w3 * l3), fma_t(X.y, w3, X.y * w3 * l3));
      }
      const bool nyq = (ii == N / 2) || (j == N / 2);
      if (roundtrip && nyq) X = mk(T(0), T(0));
      F0[addr] = X;
      if (!nyq) {
        const int nx = sfreq<N>(ii);
        const int n2 = nx * nx + ny * ny + kz * kz;
        const int b = ba.bin_of_n2[n2];
        if (b >= 0 && n2 > 0) {
          T x2 = X.x * X.x + X.y * X.y;
          if (compensate == 3) x2 = per_mode_w2<T, N>(x2, invw, ii, j, kz);  // compensation per mode
          wb.add(b, mult * x2);
        }
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
// then mult * acc into the bins of `slot`. For odd l, F0 is stored times i, so the same
// product gives Re[G conj(i F0)] = Im[G conj(F0)].
template <typename C> __device__ __forceinline__ C f0_for(C f, int odd) { return odd ? mk(-f.y, f.x) : f; }

template <typename T, int N, bool YT, bool XP>
__global__ void __launch_bounds__(Shape<N>::CT, min_blocks<T, Shape<N>::E>(Shape<N>::CT))
    k_bin_x(const cx<T>* G, int64_t spec_stride, int ell, int h0, int M, const cx<T>* __restrict__ F0,
            const ux<T>* __restrict__ twf, int slot, BinArgs ba, const float* __restrict__ ytab,
            const __grid_constant__ YTab<T> yt) {
  using C = cx<T>;
  using S = Shape<N>;
  constexpr int NH = S::NH, E = S::E, Tc = S::Tc, TW = S::TW;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  C* sF0 = sm + N * TW;
  WarpBins<T> wb;
  wb.nk = ba.nk;
  wb.nwarps = (S::CT + 31) >> 5;
  wb.b = reinterpret_cast<double*>(sF0 + N * TW);
  wb.w = reinterpret_cast<T*>(wb.b + ba.nk);
  wb.init();
  const int c = threadIdx.x % TW, t = threadIdx.x / TW;
  constexpr int64_t si = Lay<N>::XI, modes = (int64_t)N * N * NH;
  __syncthreads();
  for (int q = blockIdx.x; q < ba.n_xtiles; q += gridDim.x) {
    const int tile = ba.xtiles[q];
    const int kt = tile / N, j = tile - kt * N;  // x tiles in storage order
    const int kz = kt * TW + c;
    const int64_t off = Lay<N>::at(0, j, kz);
    const T fy = T(sfreq<N>(j)), fz = T(kz);
    const T r2yz = fy * fy + fz * fz;
    T acc[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
      sF0[(t + Tc * e) * TW + c] = f0_for(F0[off + (t + Tc * e) * si], ba.odd);
      acc[e] = T(0);
    }
    for (int s = 0; s < M; s++) {
      const int h = h0 + s;
      const int a = harm_a(h), sg = harm_sign(h);
      const C* Gs = G + (int64_t)s * spec_stride;
      // FP32 with a table: Y_lm(khat) of this harmonic, one contiguous block per x tile
      const float* Ys = YT ? ytab + (int64_t)s * modes + Lay<N>::table_tile(kt, j) + c : nullptr;
      C v[E];
      float yv[YT ? E : 1];  // table values, loaded with the spectrum so that the FFT hides their latency
#pragma unroll
      for (int e = 0; e < E; e++) {
        v[e] = Gs[off + (t + Tc * e) * si];
        if constexpr (YT) yv[e] = __ldg(Ys + (t + Tc * e) * TW);
      }
      fft_any<XP, C, E, N, kInterleaved, TW, -1>(v, sm, t, c, twf);
#pragma unroll
      for (int e = 0; e < E; e++) {
        const T fx = T(sfreq<N>(t + Tc * e));
        const T r2 = fx * fx + r2yz;
        if (r2 == T(0)) continue;
        T Y;
        if constexpr (YT) {
          Y = (T)yv[e];
        } else {
          const T inv = rsqrt_t<T>(r2);
          const T x = fx * inv, y = fy * inv;
          Y = ylm_qt<T>(yt, ell, a, fz * inv);
          if (a == 0) Y = ylm_norm(yt, 0, Y);
          if (a > 0) {
            T pr = x, pi = y;
            for (int u = 1; u < a; u++) {
              const T nr = pr * x - pi * y;
              pi = pr * y + pi * x;
              pr = nr;
            }
            Y = ylm_norm(yt, a, Y * (sg > 0 ? pr : pi));
          }
        }
        const C fv = sF0[(t + Tc * e) * TW + c];
        acc[e] += Y * (v[e].x * fv.x + v[e].y * fv.y);
      }
    }
    if (j != N / 2) {
      const T mult = kz ? T(2) : T(1);
      const int ny = sfreq<N>(j);
#pragma unroll
      for (int e = 0; e < E; e++) {
        const int ii = t + Tc * e;
        if (ii == N / 2) continue;
        const int nx = sfreq<N>(ii);
        const int n2 = nx * nx + ny * ny + kz * kz;
        const int b = ba.bin_of_n2[n2];
        if (b >= 0 && n2 > 0) {
          auto a = acc[e];
          using V = decltype(a);
          if (ba.permode_w) a = per_mode_w2<V, N>(a, static_cast<const cx<V>*>(ba.permode_w), ii, j, kz);
          wb.add(b, mult * a);
        }
      }
    }
    __syncthreads();
    wb.fold();
    __syncthreads();
  }
  for (int b = threadIdx.x; b < ba.nk; b += blockDim.x) atomicAdd(&ba.bins[slot * ba.nk + b], wb.b[b]);
}

// ------------------------------------------------------------------ pass x + bin, pipelined (FP32, Y table)
// Asynchronous global -> shared copies (cp.async): 16 bytes each, tracked per thread in
// commit groups; a group's data is visible to the block after wait + __syncthreads.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NPEND> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND) : "memory");
}

// The binning pass of the FP32 path with the Y_lm(khat) table, as one stream of copy stages
// per block: for each of its x tiles the F0 tile, then the M harmonic stages (the G tile and the
// Y_lm(khat) tile of harmonic h0 + k - 1). While one stage is used, the next one (of the same
// tile, or the first of the block's next tile) is copied asynchronously into the other half of
// a double buffer, so neither the x pass nor a new tile waits on global loads. A landed G tile
// serves as its transform's exchange buffer; F0 stays in registers over the tile's harmonics.
// (Summing S = sum_h Y_h Ghat_h and multiplying by F0 once per tile saves 8 registers, but it
// rounds differently and gave higher median errors over 30 axis-permutation draws of the 512^3
// survey catalogs.)
template <int N, bool XP>
__global__ void __launch_bounds__(Shape<N>::CT, min_blocks<float, Shape<N>::E>(Shape<N>::CT))
    k_bin_x_pipe(const float2* G, int64_t spec_stride, int ell, int h0, int M, const float2* __restrict__ F0,
                 const float4* __restrict__ twf, int slot, BinArgs ba, const float* __restrict__ ytab) {
  using C = float2;
  using S = Shape<N>;
  constexpr int NH = S::NH, E = S::E, Tc = S::Tc, TW = S::TW, CT = S::CT;
  static_assert(TW >= 4, "a tile row must hold whole 16-byte chunks");
  constexpr int GCH = TW * 8 / 16, YCH = TW * 4 / 16;  // 16-byte chunks per tile row
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sG = reinterpret_cast<C*>(smraw);                  // [2][N * TW]
  float* sY = reinterpret_cast<float*>(sG + 2 * N * TW);  // [2][N * TW]
  WarpBins<float> wb;
  wb.nk = ba.nk;
  wb.nwarps = (CT + 31) >> 5;
  wb.b = reinterpret_cast<double*>(sY + 2 * N * TW);
  wb.w = reinterpret_cast<float*>(wb.b + ba.nk);
  wb.init();
  const int c = threadIdx.x % TW, t = threadIdx.x / TW;
  constexpr int64_t si = Lay<N>::XI, modes = (int64_t)N * N * NH;
  // stage k of the block's tile q into half `buf`: k = 0 the F0 tile, k > 0 harmonic h0 + k - 1
  auto issue = [&](int q, int k, int buf) {
    const int tile = ba.xtiles[q];
    const int kt = tile / N, j = tile - kt * N;  // x tiles in storage order
    const C* Gs = (k > 0 ? G + (int64_t)(k - 1) * spec_stride : F0) + Lay<N>::at(0, j, kt * TW);
    C* dG = sG + buf * N * TW;
    for (int u = threadIdx.x; u < N * GCH; u += CT) {
      const int i = u / GCH, part = u - i * GCH;
      cp_async16(dG + i * TW + part * 2, Gs + i * si + part * 2);
    }
    if (k > 0) {
      // the table block of a tile is contiguous, in the tile's own [i][c] order
      const float* Ys = ytab + (int64_t)(k - 1) * modes + Lay<N>::table_tile(kt, j);
      float* dY = sY + buf * N * TW;
      for (int u = threadIdx.x; u < N * YCH; u += CT) cp_async16(dY + u * 4, Ys + u * 4);
    }
    cp_async_commit();
  };
  __syncthreads();
  int buf = 0;
  if ((int)blockIdx.x < ba.n_xtiles) issue(blockIdx.x, 0, 0);
  for (int q = blockIdx.x; q < ba.n_xtiles; q += gridDim.x) {
    const int tile = ba.xtiles[q];
    const int kt = tile / N, j = tile - kt * N;
    const int kz = kt * TW + c;
    C f0[E];
    float acc[E];
    for (int k = 0; k <= M; k++, buf ^= 1) {
      const int nq = k < M ? q : q + (int)gridDim.x, nk = k < M ? k + 1 : 0;
      if (nq < ba.n_xtiles) {
        // that half was last read before a barrier every thread has passed: the end of a
        // transform, or the one after an F0 stage
        issue(nq, nk, buf ^ 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();  // stage k landed for the whole block
      C* tg = sG + buf * N * TW;
      if (k == 0) {
#pragma unroll
        for (int e = 0; e < E; e++) {
          f0[e] = f0_for(tg[(t + Tc * e) * TW + c], ba.odd);
          acc[e] = 0.f;
        }
        __syncthreads();  // the F0 half is refilled by the next stage's copy
      } else {
        const float* ty = sY + buf * N * TW;
        C v[E];
        float yv[E];
#pragma unroll
        for (int e = 0; e < E; e++) {
          v[e] = tg[(t + Tc * e) * TW + c];
          yv[e] = ty[(t + Tc * e) * TW + c];
        }
        __syncthreads();  // the tile becomes the transform's exchange buffer
        fft_any<XP, C, E, N, kInterleaved, TW, -1>(v, tg, t, c, twf);
#pragma unroll
        for (int e = 0; e < E; e++) acc[e] += yv[e] * (v[e].x * f0[e].x + v[e].y * f0[e].y);  // Y(k=0) = 0
      }
    }
    if (j != N / 2) {
      const float mult = kz ? 2.f : 1.f;
      const int ny = sfreq<N>(j);
#pragma unroll
      for (int e = 0; e < E; e++) {
        const int ii = t + Tc * e;
        if (ii == N / 2) continue;
        const int nx = sfreq<N>(ii);
        const int n2 = nx * nx + ny * ny + kz * kz;
        const int b = ba.bin_of_n2[n2];
        if (b >= 0 && n2 > 0) {
          float a = acc[e];
          if (ba.permode_w) a = per_mode_w2<float, N>(a, static_cast<const cx<float>*>(ba.permode_w), ii, j, kz);
          wb.add(b, mult * a);
        }
      }
    }
    __syncthreads();
    wb.fold();
    __syncthreads();
  }
  for (int b = threadIdx.x; b < ba.nk; b += blockDim.x) atomicAdd(&ba.bins[slot * ba.nk + b], wb.b[b]);
}

// ------------------------------------------------------------------ launchers of one size
template <typename K> static void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int N> struct Passes {
  using C = cx<T>;
  using U = ux<T>;
  using S = Shape<N>;
  static size_t smem_col() { return (size_t)N * S::TW * sizeof(C); }
  static size_t smem_bins(int nk, int threads = S::CT) {
    return (size_t)nk * sizeof(double) + (size_t)((threads + 31) / 32) * nk * sizeof(T);
  }
  static size_t smem_combine(int nk) { return smem_col() + smem_bins(nk); }
  static size_t smem_bin(int nk) { return 2 * smem_col() + smem_bins(nk); }
  // pipelined FP32 pass: two G tiles and two Y tiles (float), then the bins
  static size_t smem_bin_pipe(int nk) {
    return 2 * (size_t)N * S::TW * (sizeof(float2) + sizeof(float)) + (size_t)nk * sizeof(double) +
           (size_t)((S::CT + 31) / 32) * nk * sizeof(float);
  }

  static void r2c_z(const T* in, C* out, const U* twh, const U* twr, cudaStream_t s) {
    const size_t smem = (size_t)S::ROWS * padded_len(S::NH) * sizeof(C);
    set_smem(k_r2c_z<T, N>, smem);
    k_r2c_z<T, N><<<N * N / S::ROWS, S::ZT, smem, s>>>(in, out, twh, twr);
  }
  // Launchers taking `xp` run the exact-add variant of their kernel when it is set (FP32 only).
  template <bool XP> static void c2r_z_v(const C* in, T* out, const U* twh, const U* twr, T scale, cudaStream_t s) {
    using Z = ZShape<N, XP>;
    const size_t smem = (size_t)Z::ROWS * padded_len(S::NH) * sizeof(C);
    set_smem(k_c2r_z<T, N, XP>, smem);
    k_c2r_z<T, N, XP><<<N * N / Z::ROWS, Z::ZT, smem, s>>>(in, out, twh, twr, scale);
  }
  static void c2r_z(const C* in, T* out, const U* twh, const U* twr, T scale, int xp, cudaStream_t s) {
    if (sizeof(T) == 4 && xp)
      c2r_z_v<sizeof(T) == 4>(in, out, twh, twr, scale, s);
    else
      c2r_z_v<false>(in, out, twh, twr, scale, s);
  }
  static size_t smem_ylm(int M, int rows) {
    const size_t stage = (size_t)M * rows * N * sizeof(T);
    const size_t xb = (size_t)M * rows * padded_len(S::NH) * sizeof(C);
    return stage > xb ? stage : xb;
  }
  template <int LT, bool XP>
  static void ylm_z_v(const T* f, C* out, int64_t stride, int ell, int h0, int M, const U* twh, const U* twr,
                      const T* axis, int rows, const float* rtab, cudaStream_t s) {
    const size_t smem = smem_ylm(M, rows);
    const dim3 grid(N * N / rows), block(M * rows * ZShape<N, XP>::Tz);
    set_smem(k_ylm_r2c_z<T, N, LT, XP>, smem);
    k_ylm_r2c_z<T, N, LT, XP><<<grid, block, smem, s>>>(f, out, stride, ell, h0, M, twh, twr, axis, rows, rtab,
                                                         host_ytab<T>());
  }
  template <bool XP>
  static void ylm_z_x(const T* f, C* out, int64_t stride, int ell, int h0, int M, const U* twh, const U* twr,
                      const T* axis, int rows, const float* rtab, cudaStream_t s) {
    if (rtab && ell >= 0) {  // weights from the table: no recurrence to specialise
      ylm_z_v<0, XP>(f, out, stride, ell, h0, M, twh, twr, axis, rows, rtab, s);
      return;
    }
    switch (ell) {  // the headline multipoles get unrolled recurrences
      case 2: ylm_z_v<2, XP>(f, out, stride, ell, h0, M, twh, twr, axis, rows, nullptr, s); break;
      case 4: ylm_z_v<4, XP>(f, out, stride, ell, h0, M, twh, twr, axis, rows, nullptr, s); break;
      // Cartesian monomials of degree 2 and 4 (h = monomial index)
      case -2: ylm_z_v<-2, XP>(f, out, stride, ell, h0, M, twh, twr, axis, rows, nullptr, s); break;
      case -4: ylm_z_v<-4, XP>(f, out, stride, ell, h0, M, twh, twr, axis, rows, nullptr, s); break;
      default: ylm_z_v<0, XP>(f, out, stride, ell, h0, M, twh, twr, axis, rows, nullptr, s);
    }
  }
  static void ylm_z(const T* f, C* out, int64_t stride, int ell, int h0, int M, const U* twh, const U* twr,
                    const T* axis, int rows, const float* rtab, int xp, cudaStream_t s) {
    if (sizeof(T) == 4 && xp)
      ylm_z_x<sizeof(T) == 4>(f, out, stride, ell, h0, M, twh, twr, axis, rows, rtab, s);
    else
      ylm_z_x<false>(f, out, stride, ell, h0, M, twh, twr, axis, rows, sizeof(T) == 4 ? rtab : nullptr, s);
  }
  // variant 0: TW columns per block; variant 1: TW/2 (half the threads and shared memory)
  template <int TWV, bool XP>
  static void fft_y_tw(C* data, int64_t stride, int nspec, const U* twf, int dir, int n2_cut, cudaStream_t s) {
    const size_t smem = (size_t)N * TWV * sizeof(C);
    const int threads = TWV * (N / col_elems<N, XP>());
    dim3 grid(N * (S::NH / TWV), nspec);
    if (dir < 0) {
      set_smem(k_fft_y<T, N, -1, TWV, XP>, smem);
      k_fft_y<T, N, -1, TWV, XP><<<grid, threads, smem, s>>>(data, stride, twf, n2_cut);
    } else {
      set_smem(k_fft_y<T, N, 1, TWV, XP>, smem);
      k_fft_y<T, N, 1, TWV, XP><<<grid, threads, smem, s>>>(data, stride, twf, n2_cut);
    }
  }
  template <bool XP>
  static void fft_y_x(C* data, int64_t stride, int nspec, const U* twf, int dir, int variant, int n2_cut,
                      cudaStream_t s) {
    constexpr int TW2 = S::TW > 1 ? S::TW / 2 : 1;
    if (variant == 1 && S::TW > 1)
      fft_y_tw<TW2, XP>(data, stride, nspec, twf, dir, n2_cut, s);
    else
      fft_y_tw<S::TW, XP>(data, stride, nspec, twf, dir, n2_cut, s);
  }
  static void fft_y(C* data, int64_t stride, int nspec, const U* twf, int dir, int variant, int n2_cut, int xp,
                    cudaStream_t s) {
    if (sizeof(T) == 4 && xp)
      fft_y_x<sizeof(T) == 4>(data, stride, nspec, twf, dir, variant, n2_cut, s);
    else
      fft_y_x<false>(data, stride, nspec, twf, dir, variant, n2_cut, s);
  }
  template <bool XP> static void fft_x_v(const C* in, C* out, const U* twf, int dir, cudaStream_t s) {
    const size_t smem = smem_col();
    const unsigned grid = N * (S::NH / S::TW);
    const int threads = S::TW * (N / col_elems<N, XP>());
    if (dir < 0) {
      set_smem(k_fft_x<T, N, -1, XP>, smem);
      k_fft_x<T, N, -1, XP><<<grid, threads, smem, s>>>(in, out, twf);
    } else {
      set_smem(k_fft_x<T, N, 1, XP>, smem);
      k_fft_x<T, N, 1, XP><<<grid, threads, smem, s>>>(in, out, twf);
    }
  }
  static void fft_x(const C* in, C* out, const U* twf, int dir, int xp, cudaStream_t s) {
    if (sizeof(T) == 4 && xp)
      fft_x_v<sizeof(T) == 4>(in, out, twf, dir, s);
    else
      fft_x_v<false>(in, out, twf, dir, s);
  }
  static void combine_x(const C* B, C* F0, const U* twf, int interlaced, int compensate, int roundtrip,
                        const U* phase, const C* invw, const BinArgs& ba, int ctas, cudaStream_t s) {
    const size_t smem = smem_combine(ba.nk);
    set_smem(k_combine_x<T, N>, smem);
    k_combine_x<T, N><<<ctas, S::CT, smem, s>>>(B, F0, twf, interlaced, compensate, roundtrip, phase, invw, ba);
  }
  template <bool XP>
  static void bin_x_v(const C* G, int64_t stride, int ell, int h0, int M, const C* F0, const U* twf, int slot,
                      const BinArgs& ba, int ctas, const float* ytab, cudaStream_t s) {
    const size_t smem = smem_bin(ba.nk);
    if constexpr (sizeof(T) == 4 && S::E == 8) {
      if (ytab) {
        const size_t sp = smem_bin_pipe(ba.nk);
        set_smem(k_bin_x_pipe<N, XP>, sp);
        k_bin_x_pipe<N, XP><<<ctas, S::CT, sp, s>>>(G, stride, ell, h0, M, F0, twf, slot, ba, ytab);
        return;
      }
    }
    if (ytab && sizeof(T) == 4) {
      set_smem(k_bin_x<T, N, true, XP>, smem);
      k_bin_x<T, N, true, XP><<<ctas, S::CT, smem, s>>>(G, stride, ell, h0, M, F0, twf, slot, ba, ytab, host_ytab<T>());
    } else {
      set_smem(k_bin_x<T, N, false, XP>, smem);
      k_bin_x<T, N, false, XP><<<ctas, S::CT, smem, s>>>(G, stride, ell, h0, M, F0, twf, slot, ba, ytab, host_ytab<T>());
    }
  }
  static void bin_x(const C* G, int64_t stride, int ell, int h0, int M, const C* F0, const U* twf, int slot,
                    const BinArgs& ba, int ctas, const float* ytab, int xp, cudaStream_t s) {
    if (sizeof(T) == 4 && xp)
      bin_x_v<sizeof(T) == 4>(G, stride, ell, h0, M, F0, twf, slot, ba, ctas, ytab, s);
    else
      bin_x_v<false>(G, stride, ell, h0, M, F0, twf, slot, ba, ctas, ytab, s);
  }
  template <bool XP> static int ctas_v(int which, int nk, int nsm) {
    int per = 0;
    if (which == 0) {
      const size_t smem = smem_combine(nk);
      set_smem(k_combine_x<T, N>, smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_combine_x<T, N>, S::CT, smem);
    } else if (which == 2 && sizeof(T) == 4 && S::E == 8) {
      if constexpr (sizeof(T) == 4 && S::E == 8) {
        const size_t smem = smem_bin_pipe(nk);
        set_smem(k_bin_x_pipe<N, XP>, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bin_x_pipe<N, XP>, S::CT, smem);
      }
    } else if (which == 2) {
      const size_t smem = smem_bin(nk);
      set_smem(k_bin_x<T, N, true, XP>, smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bin_x<T, N, true, XP>, S::CT, smem);
    } else {
      const size_t smem = smem_bin(nk);
      set_smem(k_bin_x<T, N, false, XP>, smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bin_x<T, N, false, XP>, S::CT, smem);
    }
    if (per < 1) per = 1;
    const int ntiles = N * (S::NH / S::TW);
    return per * nsm < ntiles ? per * nsm : ntiles;
  }
  static int ctas(int which, int nk, int nsm, int xp) {
    if (sizeof(T) == 4 && xp) return ctas_v<sizeof(T) == 4>(which, nk, nsm);
    return ctas_v<false>(which, nk, nsm);
  }
  static PassTable<T> table() {
    PassTable<T> t;
    t.N = N;
    t.E = S::E;
    t.tw = S::TW;
    t.rows_z = S::ROWS;
    t.tz = S::Tz;
    t.tz_xp = ZShape<N, sizeof(T) == 4>::Tz;
    t.r2c_z = &r2c_z;
    t.c2r_z = &c2r_z;
    t.ylm_z = &ylm_z;
    t.smem_ylm = &smem_ylm;
    t.fft_y = &fft_y;
    t.fft_x = &fft_x;
    t.combine_x = &combine_x;
    t.bin_x = &bin_x;
    t.ctas = &ctas;
    t.smem_combine = &smem_combine;
    t.smem_bin = &smem_bin;
    t.smem_bin_pipe = &smem_bin_pipe;
    return t;
  }
};

#define PSPEC_DEFINE_PASSES(N_)                                                     \
  template <> const PassTable<float>* pass_table_n<float, N_>() {                   \
    static const PassTable<float> t = Passes<float, N_>::table();                   \
    return &t;                                                                      \
  }                                                                                 \
  template <> const PassTable<double>* pass_table_n<double, N_>() {                 \
    static const PassTable<double> t = Passes<double, N_>::table();                 \
    return &t;                                                                      \
  }

}  // namespace pspec
