// Register-resident Stockham FFT engine for the transform passes.
//
// A sequence of length L is spread over Tc = L/E threads; thread t of a sequence holds the
// E elements t + Tc*e (e = 0..E-1) in registers. Every stage reads exactly that set (a
// radix-R butterfly q uses slots q + r*E/R), so the first stage is fed straight from
// global memory and the last stage's outputs land back in the same slots in natural
// order, ready to be stored. Between stages the butterfly outputs go through shared
// memory: L/E-stage transforms cost (stages - 1) shared-memory exchanges.
//
// Stage with radix R after Ns = product of earlier radices: butterfly j (k = j mod Ns)
// twiddles input r by w_L^{r k L/(Ns R)}, takes an R-point DFT and writes output r to
// position (j - k) R + k + r Ns. Radix 3, when present, is the last stage, so every Ns
// before it is a power of two and k = j mod Ns is a mask; in the last stage k = j.
#pragma once
#include "common.cuh"

namespace pspec {

// Shared-memory layouts of the exchange buffer.
//   kInterleaved: [pos][nseq], sequence fastest (columns of a tile; lanes run across seqs)
//   kPaddedRows:  [seq][L + L/16], position fastest with one pad slot per 16 (rows)
enum { kInterleaved = 0, kPaddedRows = 1 };

template <int LAYOUT>
__device__ __forceinline__ int sidx(int seq, int pos, int nseq, int Lp) {
  return LAYOUT == kInterleaved ? pos * nseq + seq : seq * Lp + pos + (pos >> 4);
}

__host__ __device__ __forceinline__ int padded_len(int L) { return L + (L >> 4); }

template <typename C> __device__ __forceinline__ C ldg_c(const C* p) { return __ldg(p); }

template <typename C, int E, int R, int LAYOUT, int DIR>
__device__ __forceinline__ void stage_regs(C (&v)[E], C* sm, int t, int Tc, int L, int Ns, bool last, int seq,
                                           int nseq, int Lp, const C* __restrict__ tw) {
  constexpr int Q = E / R;
  const int tstep = L / (Ns * R);
  // When Ns divides Tc (both powers of two) every butterfly of this thread has the same
  // k = t mod Ns, so with several butterflies (Q > 1) its R - 1 twiddles are loaded once.
  const bool shared_k = (Q > 1) && (Ns > 1) && !last && (Ns <= Tc);
  C ws[R > 1 && Q > 1 ? R : 1];
  if constexpr (Q > 1) if (shared_k) {
    const int k = t & (Ns - 1);
#pragma unroll
    for (int r = 1; r < R; r++) {
      ws[r] = ldg_c(tw + r * k * tstep);
      if (DIR > 0) ws[r].y = -ws[r].y;
    }
  }
#pragma unroll
  for (int q = 0; q < Q; q++) {
    const int j = t + Tc * q;
    const int k = last ? j : (j & (Ns - 1));
    C u[R];
#pragma unroll
    for (int r = 0; r < R; r++) u[r] = v[q + r * Q];
    if constexpr (Q > 1) {
      if (shared_k) {
#pragma unroll
        for (int r = 1; r < R; r++) u[r] = cmul(u[r], ws[r]);
      }
    }
    if (!shared_k && Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; r++) {
        C w = ldg_c(tw + r * k * tstep);
        if (DIR > 0) w.y = -w.y;
        u[r] = cmul(u[r], w);
      }
    }
    Dft<C, R>::run(u, DIR);
    if (last) {
#pragma unroll
      for (int r = 0; r < R; r++) v[q + r * Q] = u[r];
    } else {
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; r++) sm[sidx<LAYOUT>(seq, base + r * Ns, nseq, Lp)] = u[r];
    }
  }
}

// Transforms the sequence whose slots this thread holds (DIR = -1 forward, +1 inverse).
// All threads of the block must call it (it contains __syncthreads); the shared buffer is
// free again when it returns.
template <typename C, int E, int LAYOUT, int DIR>
__device__ __forceinline__ void fft_regs(C (&v)[E], C* sm, const FftPlan& p, int t, int seq, int nseq,
                                         const C* __restrict__ tw) {
  const int L = p.L;
  const int Tc = L / E;
  const int Lp = padded_len(L);
  for (int s = 0; s < p.nst; s++) {
    const bool last = (s == p.nst - 1);
    const int Ns = p.ns[s];
    switch (p.rad[s]) {
      case 8:
        if constexpr (E % 8 == 0) stage_regs<C, E, 8, LAYOUT, DIR>(v, sm, t, Tc, L, Ns, last, seq, nseq, Lp, tw);
        break;
      case 4:
        if constexpr (E % 4 == 0) stage_regs<C, E, 4, LAYOUT, DIR>(v, sm, t, Tc, L, Ns, last, seq, nseq, Lp, tw);
        break;
      case 3:
        if constexpr (E % 3 == 0) stage_regs<C, E, 3, LAYOUT, DIR>(v, sm, t, Tc, L, Ns, last, seq, nseq, Lp, tw);
        break;
      default:
        if constexpr (E % 2 == 0) stage_regs<C, E, 2, LAYOUT, DIR>(v, sm, t, Tc, L, Ns, last, seq, nseq, Lp, tw);
        break;
    }
    if (!last) {
      __syncthreads();
#pragma unroll
      for (int e = 0; e < E; e++) v[e] = sm[sidx<LAYOUT>(seq, t + Tc * e, nseq, Lp)];
      __syncthreads();
    }
  }
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
