// Register-resident Stockham FFT engine for the transform passes, with the transform length
// and the tile shape fixed at compile time.
//
// A sequence of length L is spread over Tc = L/E threads; thread t of a sequence holds the
// E elements t + Tc*e (e = 0..E-1) in registers. Every stage reads exactly that set (a
// radix-R butterfly q uses slots q + r*E/R), so the first stage is fed straight from
// global memory and the last stage's outputs land back in the same slots in natural
// order, ready to be stored. Between stages the butterfly outputs go through shared
// memory: an S-stage transform costs S - 1 shared-memory exchanges.
//
// Stage with radix R after Ns = product of earlier radices: butterfly j (k = j mod Ns)
// twiddles input r by w_L^{r k L/(Ns R)}, takes an R-point DFT and writes output r to
// position (j - k) R + k + r Ns. Radices are 8, 4, 2 (largest first) and a factor 3 last,
// so every Ns before the last stage is a power of two and k = j mod Ns is a mask; in the
// last stage k = j.
#pragma once
#include <type_traits>
#include "common.cuh"

namespace pspec {

// ------------------------------------------------------------------ compile-time plans
constexpr int elems_for(int N) { return N % 3 == 0 ? 24 : 8; }

struct CtPlan {
  int nst;
  int rad[12];
  int ns[12];
};

// Radices in order 16 (only when a thread holds a multiple of 16 elements), 8, 4, 2, then 3.
__host__ __device__ constexpr CtPlan ct_plan(int L, int E = 8) {
  CtPlan p{0, {0}, {0}};
  int x = L, ns = 1, three = 0;
  while (x % 3 == 0) {
    x /= 3;
    three++;
  }
  if (E % 32 == 0 && x % 32 == 0 && x != 32 * 32) {  // one radix-32 stage, then radix 16 (512 = 32 x 16)
    p.rad[p.nst] = 32;
    p.ns[p.nst] = ns;
    ns *= 32;
    x /= 32;
    p.nst++;
  }
  while (E % 16 == 0 && x % 16 == 0) {
    p.rad[p.nst] = 16;
    p.ns[p.nst] = ns;
    ns *= 16;
    x /= 16;
    p.nst++;
  }
  while (x % 8 == 0) {
    p.rad[p.nst] = 8;
    p.ns[p.nst] = ns;
    ns *= 8;
    x /= 8;
    p.nst++;
  }
  while (x % 4 == 0) {
    p.rad[p.nst] = 4;
    p.ns[p.nst] = ns;
    ns *= 4;
    x /= 4;
    p.nst++;
  }
  while (x % 2 == 0) {
    p.rad[p.nst] = 2;
    p.ns[p.nst] = ns;
    ns *= 2;
    x /= 2;
    p.nst++;
  }
  for (int i = 0; i < three; i++) {
    p.rad[p.nst] = 3;
    p.ns[p.nst] = ns;
    ns *= 3;
    p.nst++;
  }
  return p;
}

template <int B, int E, typename F> __device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// Shared-memory layouts of the exchange buffer.
//   kInterleaved: [pos][NSEQ], sequence fastest (columns of a tile; lanes run across seqs)
//   kPaddedRows:  [seq][L + L/16], position fastest with one pad slot per 16 (rows)
enum { kInterleaved = 0, kPaddedRows = 1 };

__host__ __device__ constexpr int padded_len(int L) { return L + (L >> 4); }

template <int LAYOUT, int L, int NSEQ>
__device__ __forceinline__ int sidx(int seq, int pos) {
  if constexpr (LAYOUT == kInterleaved)
    return pos * NSEQ + seq;
  else
    return seq * padded_len(L) + pos + (pos >> 4);
}

template <typename C> __device__ __forceinline__ C ldg_c(const C* p) { return __ldg(p); }

template <typename C, int E, int L, int R, int NS, bool LAST, int LAYOUT, int NSEQ, int DIR>
__device__ __forceinline__ void stage_ct(C (&v)[E], C* sm, int t, int seq, const ux_of<C>* __restrict__ tw) {
  using U = ux_of<C>;
  constexpr int Q = E / R;
  constexpr int Tc = L / E;
  constexpr int TSTEP = L / (NS * R);
  // With NS | Tc every butterfly of this thread has k = t mod NS: load its twiddles once.
  constexpr bool kShared = (Q > 1) && (NS > 1) && !LAST && (NS <= Tc);
  U ws[kShared ? R : 1];
  if constexpr (kShared) {
    const int k = t & (NS - 1);
#pragma unroll
    for (int r = 1; r < R; r++) {
      ws[r] = ldg_u(tw + r * k * TSTEP);
      if (DIR > 0) ws[r] = uconj(ws[r]);
    }
  }
#pragma unroll
  for (int q = 0; q < Q; q++) {
    const int j = t + Tc * q;
    const int k = LAST ? j : (j & (NS - 1));
    C u[R];
#pragma unroll
    for (int r = 0; r < R; r++) u[r] = v[q + r * Q];
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; r++) {
        U w;
        if constexpr (kShared) {
          w = ws[r];
        } else {
          w = ldg_u(tw + r * k * TSTEP);
          if (DIR > 0) w = uconj(w);
        }
        u[r] = umul(u[r], w);
      }
    }
    Dft<C, R>::run(u, DIR);
    if constexpr (LAST) {
#pragma unroll
      for (int r = 0; r < R; r++) v[q + r * Q] = u[r];
    } else {
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; r++) sm[sidx<LAYOUT, L, NSEQ>(seq, base + r * NS)] = u[r];
    }
  }
}

// Barrier between exchange steps: the whole block, or (WARP) only the warp, when every
// sequence's threads lie in one warp and its shared rows are its own.
template <bool WARP> __device__ __forceinline__ void fft_sync() {
  if constexpr (WARP)
    __syncwarp();
  else
    __syncthreads();
}

// Transforms the length-L sequence whose slots this thread holds (DIR = -1 forward, +1
// inverse). All threads of the block (WARP: of the warp) must call it; the shared buffer of
// the sequence is free again when it returns. NSEQ is the number of interleaved sequences
// (kInterleaved only).
template <typename C, int E, int L, int LAYOUT, int NSEQ, int DIR, bool WARP = false>
__device__ __forceinline__ void fft_ct(C (&v)[E], C* sm, int t, int seq, const ux_of<C>* __restrict__ tw) {
  constexpr CtPlan P = ct_plan(L, E);
  constexpr int Tc = L / E;
  static_assert(!WARP || (LAYOUT == kPaddedRows && Tc <= 32 && 32 % Tc == 0), "warp-synchronous rows only");
  static_for<0, P.nst>([&](auto s_) {
    constexpr int s = decltype(s_)::value;
    constexpr bool last = (s == P.nst - 1);
    stage_ct<C, E, L, P.rad[s], P.ns[s], last, LAYOUT, NSEQ, DIR>(v, sm, t, seq, tw);
    if constexpr (!last) {
      fft_sync<WARP>();
#pragma unroll
      for (int e = 0; e < E; e++) v[e] = sm[sidx<LAYOUT, L, NSEQ>(seq, t + Tc * e)];
      fft_sync<WARP>();
    }
  });
}

// Per-warp histograms flushed into per-block FP64 bins. On the FP32 path the warp partials
// are FP32: one warp's partial over one tile holds at most a few hundred terms, and the FP64
// adds then happen once per bin per tile instead of once per mode. The FP64 path keeps
// FP64 partials.
template <typename W> struct WarpBins {
  W* w;          // [nwarps][nk]
  double* b;     // [nk]
  int nk;
  int nwarps;
  __device__ __forceinline__ void add(int bin, W v) const { atomicAdd(&w[(threadIdx.x >> 5) * nk + bin], v); }
  // All threads: zero the warp and block bins (call once before the first tile).
  __device__ __forceinline__ void init() const {
    for (int i = threadIdx.x; i < nwarps * nk; i += blockDim.x) w[i] = W(0);
    for (int i = threadIdx.x; i < nk; i += blockDim.x) b[i] = 0.0;
  }
  // All threads, between __syncthreads: fold the warp partials into the FP64 bins.
  __device__ __forceinline__ void fold() const {
    for (int i = threadIdx.x; i < nk; i += blockDim.x) {
      double s = 0.0;
      for (int q = 0; q < nwarps; q++) {
        s += (double)w[q * nk + i];
        w[q * nk + i] = W(0);
      }
      b[i] += s;
    }
  }
};

}  // namespace pspec
