// Device-side building blocks shared by the libpspec kernels: complex arithmetic,
// the shared-memory Stockham FFT stage, and the real spherical-harmonic recurrence.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pspec {

// ------------------------------------------------------------------ complex helpers
template <typename T> struct CxOf;
template <> struct CxOf<float> { using type = float2; };
template <> struct CxOf<double> { using type = double2; };
template <typename T> using cx = typename CxOf<T>::type;

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return mk(a.x * s, a.y * s); }
// a * (i * sgn): sgn = +1 multiplies by i, -1 by -i
template <typename C> __device__ __forceinline__ C cmul_i(C a, int sgn) {
  return sgn > 0 ? mk(-a.y, a.x) : mk(a.y, -a.x);
}

// ------------------------------------------------------------------ FFT plan
// A length-L transform as a product of radices (2, 3, 4, 8), applied as Stockham
// auto-sort stages. ns[s] is the product of the radices before stage s.
constexpr int kMaxStages = 16;
struct FftPlan {
  int L;
  int nst;
  int rad[kMaxStages];
  int ns[kMaxStages];
};

// Small DFTs in registers. dir = -1: exp(-2 pi i jk/R) (forward); +1: inverse.
template <typename C, int R> struct Dft;

template <typename C> struct Dft<C, 2> {
  static __device__ __forceinline__ void run(C* v, int) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <typename C> struct Dft<C, 4> {
  static __device__ __forceinline__ void run(C* v, int dir) {
    C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    C t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
    // forward: y1 = t1 - i t3, y3 = t1 + i t3; inverse swaps the sign
    C it3 = cmul_i(t3, dir);
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, it3);
    v[3] = csub(t1, it3);
  }
};

template <typename C> struct Dft<C, 8> {
  static __device__ __forceinline__ void run(C* v, int dir) {
    using T = decltype(v[0].x);
    const T h = T(0.70710678118654752440);
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    Dft<C, 4>::run(e, dir);
    Dft<C, 4>::run(o, dir);
    // twiddles w8^k = exp(dir * 2 pi i k / 8), k = 0..3
    C o1 = mk(h * (o[1].x - dir * o[1].y), h * (o[1].y + dir * o[1].x));  // o1 * (1 + dir i)/sqrt2
    C o2 = cmul_i(o[2], dir);                                               // o2 * (dir i)
    C o3 = mk(h * (-o[3].x - dir * o[3].y), h * (-o[3].y + dir * o[3].x)); // o3 * (-1 + dir i)/sqrt2
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
};

template <typename C> struct Dft<C, 3> {
  static __device__ __forceinline__ void run(C* v, int dir) {
    using T = decltype(v[0].x);
    const T s = T(0.86602540378443864676) * T(dir);  // sin(2 pi/3) with the direction's sign
    C t = cadd(v[1], v[2]);
    C u = csub(v[1], v[2]);
    C m = mk(v[0].x - T(0.5) * t.x, v[0].y - T(0.5) * t.y);
    C isu = mk(-s * u.y, s * u.x);  // i s u
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, isu);
    v[2] = csub(m, isu);
  }
};

// One Stockham stage over `nseq` sequences of length L, from `in` to `out` (both shared).
// Element e of sequence q sits at q*seq_stride + e*el_stride. Butterfly bf handles
// inputs j + r L/R and writes outputs (j - k) R + k + r Ns, k = j mod Ns, after the
// twiddles w_L^{r k L/(Ns R)} from `tw` (tw[t] = exp(-2 pi i t / L)).
template <typename C, int R>
__device__ __forceinline__ void stockham_stage(const C* in, C* out, int nseq, int L, int Ns,
                                               int seq_stride, int el_stride, bool seq_fast,
                                               const C* tw, int dir) {
  const int LR = L / R;
  const int total = nseq * LR;
  const int tstep = L / (Ns * R);
  for (int bf = threadIdx.x; bf < total; bf += blockDim.x) {
    int q, j;
    if (seq_fast) {
      q = bf % nseq;
      j = bf / nseq;
    } else {
      j = bf % LR;
      q = bf / LR;
    }
    const int k = j % Ns;
    C v[R];
    const C* ip = in + q * seq_stride;
#pragma unroll
    for (int r = 0; r < R; r++) v[r] = ip[(j + r * LR) * el_stride];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; r++) {
        C w = tw[r * k * tstep];
        if (dir > 0) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    Dft<C, R>::run(v, dir);
    const int base = (j - k) * R + k;
    C* op = out + q * seq_stride;
#pragma unroll
    for (int r = 0; r < R; r++) op[(base + r * Ns) * el_stride] = v[r];
  }
}

// Full transform of every sequence in shared memory, ping-ponging between a and b.
// Returns the buffer holding the result (natural order). Ends with __syncthreads().
template <typename C>
__device__ C* fft_smem(C* a, C* b, const FftPlan& p, int nseq, int seq_stride, int el_stride,
                       bool seq_fast, const C* tw, int dir) {
  C* in = a;
  C* out = b;
  for (int s = 0; s < p.nst; s++) {
    switch (p.rad[s]) {
      case 8: stockham_stage<C, 8>(in, out, nseq, p.L, p.ns[s], seq_stride, el_stride, seq_fast, tw, dir); break;
      case 4: stockham_stage<C, 4>(in, out, nseq, p.L, p.ns[s], seq_stride, el_stride, seq_fast, tw, dir); break;
      case 3: stockham_stage<C, 3>(in, out, nseq, p.L, p.ns[s], seq_stride, el_stride, seq_fast, tw, dir); break;
      default: stockham_stage<C, 2>(in, out, nseq, p.L, p.ns[s], seq_stride, el_stride, seq_fast, tw, dir); break;
    }
    __syncthreads();
    C* t = in;
    in = out;
    out = t;
  }
  return in;
}

// ------------------------------------------------------------------ real Y_lm recurrence
// Reduced, normalised associated Legendre functions q_l^a(z) (the sin^a(theta) factor is
// carried by Re/Im (x + i y)^a on the unit sphere):
//   q_a^a = c_a,  q_{a+1}^a = A(a+1,a) z c_a,
//   q_l^a = A(l,a) (z q_{l-1}^a - B(l,a) q_{l-2}^a),
//   A(l,a) = sqrt((4l^2-1)/(l^2-a^2)), B(l,a) = sqrt(((l-1)^2-a^2)/(4(l-1)^2-1)),
//   c_0 = 1/sqrt(4 pi), c_a = -sqrt((2a+1)/(2a)) c_{a-1}.
// Real harmonics (eq. real-Ylm): Y_l0 = q_l^0(z), Y_{l,+a} = sqrt2 q_l^a Re(x+iy)^a,
// Y_{l,-a} = sqrt2 q_l^a Im(x+iy)^a. Tables are computed in FP64 on the host.
constexpr int kLmax = 16;
constexpr int kLdim = kLmax + 1;
template <typename T> struct YTab {
  T c[kLdim];
  T A[kLdim * kLdim];  // [l * kLdim + a]
  T B[kLdim * kLdim];
};

template <typename T>
__device__ __forceinline__ T ylm_q(const YTab<T>& t, int ell, int a, T z) {
  T q2 = t.c[a];
  if (ell == a) return q2;
  T q1 = t.A[(a + 1) * kLdim + a] * z * q2;
  for (int l = a + 2; l <= ell; l++) {
    T q = t.A[l * kLdim + a] * (z * q1 - t.B[l * kLdim + a] * q2);
    q2 = q1;
    q1 = q;
  }
  return q1;
}

// Harmonic index h within multipole l: h = 0 -> m = 0; h = 2a-1 -> m = +a; h = 2a -> m = -a.
__host__ __device__ __forceinline__ int harm_a(int h) { return (h + 1) >> 1; }
__host__ __device__ __forceinline__ int harm_sign(int h) { return h == 0 ? 0 : ((h & 1) ? 1 : -1); }

template <typename T> __device__ __forceinline__ T rsqrt_t(T x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }

// Y_{l,m(h)} at the direction of (vx, vy, vz) with squared length r2 > 0.
template <typename T>
__device__ __forceinline__ T ylm_dir(const YTab<T>& t, int ell, int h, T vx, T vy, T vz, T r2) {
  const T inv = rsqrt_t<T>(r2);
  const T x = vx * inv, y = vy * inv, z = vz * inv;
  const int a = harm_a(h);
  T q = ylm_q<T>(t, ell, a, z);
  if (a == 0) return q;
  T pr = x, pi = y;  // (x + i y)^a
  for (int s = 1; s < a; s++) {
    T nr = pr * x - pi * y;
    pi = pr * y + pi * x;
    pr = nr;
  }
  const T sq2 = T(1.41421356237309504880);
  return sq2 * q * (harm_sign(h) > 0 ? pr : pi);
}

}  // namespace pspec
