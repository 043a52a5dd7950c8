// Device-side building blocks shared by the libpspec kernels: complex arithmetic,
// unit-modulus table factors, the small in-register DFTs, and the real spherical-harmonic
// recurrence.
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

// ------------------------------------------------------------------ unit-modulus factors
// Twiddles and phase factors as the tables hold them. Rounded to FP32, (cos, sin) lies off the
// unit circle by up to ~6e-8 with a negative mean over small tables; applied in every stage
// of every axis that becomes a gain bias of ~1e-7 on |F|^2 that also depends on the mode's
// index digits (the shot noise then leaks into P_0 and P_4 at high k). The FP32 entry is
// therefore a pair hi + lo per component ({c_hi, s_hi, c_lo, s_lo}, lo = the rounding error
// of hi) and a product folds a*lo into the roundings of the exact products a*hi. A correction
// added after rounding would be lost: it is below half an ulp of an already rounded value.
template <typename T> struct UnitOf;
template <> struct UnitOf<float> { using type = float4; };   // {c_hi, s_hi, c_lo, s_lo}
template <> struct UnitOf<double> { using type = double2; };  // {cos, sin}
template <typename T> using ux = typename UnitOf<T>::type;
template <typename C> struct BaseOf;
template <> struct BaseOf<float2> { using type = float; };
template <> struct BaseOf<double2> { using type = double; };
template <typename C> using ux_of = ux<typename BaseOf<C>::type>;

__device__ __forceinline__ float4 ldg_u(const float4* p) { return __ldg(p); }
__device__ __forceinline__ double2 ldg_u(const double2* p) { return __ldg(p); }
__device__ __forceinline__ float4 uconj(float4 w) { return make_float4(w.x, -w.y, w.z, -w.w); }
__device__ __forceinline__ double2 uconj(double2 w) { return make_double2(w.x, -w.y); }
// a * w
__device__ __forceinline__ float2 umul(float2 a, float4 w) {
  const float lx = fmaf(a.x, w.z, -a.y * w.w), ly = fmaf(a.x, w.w, a.y * w.z);
  return make_float2(fmaf(a.x, w.x, fmaf(-a.y, w.y, lx)), fmaf(a.x, w.y, fmaf(a.y, w.x, ly)));
}
__device__ __forceinline__ double2 umul(double2 a, double2 w) {
  return make_double2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
// x * K for an irrational constant K: in FP32 as x*K_hi + x*K_lo (K_lo = K - K_hi), so that
// the product carries no systematic rounding of K (a rounded K = sqrt(1/2) alone scales a
// quarter of every radix-8 stage's output power by 1 - 3.4e-8).
template <typename T> struct ConstMul;
template <> struct ConstMul<float> {
  float hi, lo;
  __device__ __forceinline__ constexpr ConstMul(double k) : hi((float)k), lo((float)(k - (double)(float)k)) {}
  __device__ __forceinline__ float operator()(float x) const { return fmaf(x, hi, x * lo); }
};
template <> struct ConstMul<double> {
  double k;
  __device__ __forceinline__ constexpr ConstMul(double k_) : k(k_) {}
  __device__ __forceinline__ double operator()(double x) const { return x * k; }
};

// ------------------------------------------------------------------ butterflies
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
    using T = typename BaseOf<C>::type;
    const ConstMul<T> h(0.70710678118654752440);
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    Dft<C, 4>::run(e, dir);
    Dft<C, 4>::run(o, dir);
    // twiddles w8^k = exp(dir * 2 pi i k / 8), k = 0..3
    C o1 = mk(h(o[1].x - dir * o[1].y), h(o[1].y + dir * o[1].x));   // o1 * (1 + dir i)/sqrt2
    C o2 = cmul_i(o[2], dir);                                          // o2 * (dir i)
    C o3 = mk(h(-o[3].x - dir * o[3].y), h(-o[3].y + dir * o[3].x));  // o3 * (-1 + dir i)/sqrt2
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

// 16 = 4 x 4: four DFT4 over n1 (inputs n2 + 4 n1), twiddles W16^(n2 k1), four DFT4 over n2;
// output k1 + 4 k2. Irrational constants as hi + lo (ConstMul), as in the radix-8 butterfly.
template <typename C> struct Dft<C, 16> {
  static __device__ __forceinline__ void run(C* v, int dir) {
    using T = typename BaseOf<C>::type;
    const ConstMul<T> h(0.70710678118654752440), c1(0.92387953251128675613), s1(0.38268343236508977173);
    C a[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; n2++) {
      C t[4] = {v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]};
      Dft<C, 4>::run(t, dir);
#pragma unroll
      for (int k1 = 0; k1 < 4; k1++) a[n2][k1] = t[k1];
    }
    // W16^m = cos(2 pi m/16) + i dir sin(2 pi m/16) for m = n2 k1
    const T d = T(dir);
    auto rot = [&](C z, const ConstMul<T>& cr, const ConstMul<T>& ci, T sr, T si) {  // z * (sr cr + i si ci)
      const T re = sr * cr(z.x) - si * ci(z.y), im = sr * cr(z.y) + si * ci(z.x);
      return mk(re, im);
    };
    a[1][1] = rot(a[1][1], c1, s1, T(1), d);                                       // m = 1
    a[1][2] = mk(h(a[1][2].x - d * a[1][2].y), h(a[1][2].y + d * a[1][2].x));      // m = 2
    a[1][3] = rot(a[1][3], s1, c1, T(1), d);                                       // m = 3
    a[2][1] = mk(h(a[2][1].x - d * a[2][1].y), h(a[2][1].y + d * a[2][1].x));      // m = 2
    a[2][2] = cmul_i(a[2][2], dir);                                                // m = 4
    a[2][3] = mk(h(-a[2][3].x - d * a[2][3].y), h(-a[2][3].y + d * a[2][3].x));    // m = 6
    a[3][1] = rot(a[3][1], s1, c1, T(1), d);                                       // m = 3
    a[3][2] = mk(h(-a[3][2].x - d * a[3][2].y), h(-a[3][2].y + d * a[3][2].x));    // m = 6
    a[3][3] = rot(a[3][3], c1, s1, T(-1), -d);                                     // m = 9
#pragma unroll
    for (int k1 = 0; k1 < 4; k1++) {
      C t[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
      Dft<C, 4>::run(t, dir);
#pragma unroll
      for (int k2 = 0; k2 < 4; k2++) v[k1 + 4 * k2] = t[k2];
    }
  }
};

// 32 = 2 x 16: two DFT16 over the even and odd inputs, twiddles W32^k1 on the odd half (hi/lo
// constants), one DFT2 per k1; output k1 + 16 k2.
template <typename C> struct Dft<C, 32> {
  static __device__ __forceinline__ void run(C* v, int dir) {
    using T = typename BaseOf<C>::type;
    C e[16], o[16];
#pragma unroll
    for (int i = 0; i < 16; i++) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    Dft<C, 16>::run(e, dir);
    Dft<C, 16>::run(o, dir);
    // cos(2 pi k/32), k = 0..8 (sin(2 pi k/32) = cos(2 pi (8-k)/32))
    constexpr double kc[9] = {1.0, 0.98078528040323044913, 0.92387953251128675613, 0.83146961230254523708,
                              0.70710678118654752440, 0.55557023301960222474, 0.38268343236508977173,
                              0.19509032201612826785, 0.0};
    const T d = T(dir);
#pragma unroll
    for (int k = 0; k < 16; k++) {
      C w = o[k];
      if (k > 0) {
        // W32^k = cos + i dir sin; for k > 8: cos(2 pi k/32) = -cos(2 pi (16-k)/32), sin = sin(2 pi (16-k)/32)
        const int kk = k <= 8 ? k : 16 - k;
        const ConstMul<T> cr(kc[kk]), ci(kc[8 - kk]);
        const T sr = k <= 8 ? T(1) : T(-1);
        const T re = sr * cr(w.x) - d * ci(w.y), im = sr * cr(w.y) + d * ci(w.x);
        w = mk(re, im);
      }
      v[k] = cadd(e[k], w);
      v[k + 16] = csub(e[k], w);
    }
  }
};

template <typename C> struct Dft<C, 3> {
  static __device__ __forceinline__ void run(C* v, int dir) {
    using T = typename BaseOf<C>::type;
    const ConstMul<T> s3(0.86602540378443864676);  // sin(2 pi/3)
    C t = cadd(v[1], v[2]);
    C u = csub(v[1], v[2]);
    C m = mk(v[0].x - T(0.5) * t.x, v[0].y - T(0.5) * t.y);
    const T su_x = s3(u.x) * T(dir), su_y = s3(u.y) * T(dir);
    C isu = mk(-su_y, su_x);  // i s u, s = dir sin(2 pi/3)
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, isu);
    v[2] = csub(m, isu);
  }
};

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
// The recurrence runs on q_l^a / c_a (seed 1) and the constant factor n_a (c_0 for a = 0,
// sqrt2 c_a for a > 0) is applied last. In FP32 the coefficients A, B and n_a are split into
// hi + lo (lo = the rounding error of hi) and lo enters the roundings of the exact products:
// rounded coefficients alone would change the shape of q_l^a(z) by ~1e-7, an error smooth over
// the sphere whose shell averages are not zero, and a rounded n_a would scale a whole harmonic
// by up to 3e-8; through either, the k-independent shot-noise term leaks into P_l (l >= 2).
template <typename T> struct YTab {
  T n[kLdim];          // n_a
  T nl[kLdim];         // lo part of n_a (FP32 only; zero in FP64)
  T A[kLdim * kLdim];  // [l * kLdim + a]
  T B[kLdim * kLdim];
  T Al[kLdim * kLdim];  // lo parts (FP32 only; zero in FP64)
  T Bl[kLdim * kLdim];
};

// q_l^a(z) / c_a. HILO = false: coefficients rounded to T only. Both spaces use HILO = true:
// a coherent error in the real-space weights Y_lm(rhat) leaks part of the shot noise into P_l
// through shell sums of Y_lm(khat) that the mesh's cubic symmetry leaves nonzero, and it grows
// with l.
template <typename T, bool HILO = true>
__device__ __forceinline__ T ylm_qt(const YTab<T>& t, int ell, int a, T z) {
  T q2 = T(1);
  if (ell == a) return q2;
  const int i1 = (a + 1) * kLdim + a;
  T q1;
  if constexpr (sizeof(T) == 4 && HILO) {
    q1 = fmaf(t.A[i1], z, t.Al[i1] * z);
  } else {
    q1 = t.A[i1] * z;
  }
  for (int l = a + 2; l <= ell; l++) {
    const int i = l * kLdim + a;
    T q;
    if constexpr (sizeof(T) == 4 && HILO) {
      const T u = fmaf(z, q1, -(t.Bl[i] * q2));  // z q1 - B_lo q2
      const T s = fmaf(-t.B[i], q2, u);          // - B_hi q2 + u
      q = fmaf(t.A[i], s, t.Al[i] * s);           // (A_hi + A_lo) s
    } else {
      q = t.A[i] * (z * q1 - t.B[i] * q2);
    }
    q2 = q1;
    q1 = q;
  }
  return q1;
}

// x n_a: Y_l0 = n_0 qt; Y_{l,+a} = n_a qt Re(x+iy)^a, Y_{l,-a} = n_a qt Im(x+iy)^a.
template <typename T> __device__ __forceinline__ T ylm_norm(const YTab<T>& t, int a, T x) {
  if constexpr (sizeof(T) == 4)
    return fmaf(x, t.n[a], x * t.nl[a]);
  else
    return x * t.n[a];
}

// Cartesian decomposition (the route the paper compares against, Sec. 2.1): monomials
// xhat^a yhat^b zhat^c of degree 2 (q = 0..5) and 4 (q = 6..20), and their multinomial
// coefficients deg! / (a! b! c!), so that sum_q mult_q khat^q rhat^q = (khat . rhat)^deg.
constexpr int kCartItems = 21;
__host__ __device__ __forceinline__ void cart_exp(int q, int& a, int& b, int& c) {
  if (q < 6) {  // (2,0,0) (0,2,0) (0,0,2) (1,1,0) (1,0,1) (0,1,1)
    a = q == 0 ? 2 : (q == 3 || q == 4 ? 1 : 0);
    b = q == 1 ? 2 : (q == 3 || q == 5 ? 1 : 0);
    c = 2 - a - b;
    return;
  }
  int r = q - 6;  // a from 4 down to 0, then b from 4 - a down to 0
  for (a = 4; a >= 0; a--) {
    const int nb = 5 - a;
    if (r < nb) {
      b = 4 - a - r;
      c = 4 - a - b;
      return;
    }
    r -= nb;
  }
  a = b = c = 0;
}
__host__ __device__ __forceinline__ int cart_mult(int q) {
  int a, b, c;
  cart_exp(q, a, b, c);
  const int f[5] = {1, 1, 2, 6, 24};
  return f[a + b + c] / (f[a] * f[b] * f[c]);
}
template <typename T> __device__ __forceinline__ T ipow(T x, int n) {
  T r = T(1);
  for (int i = 0; i < n; i++) r *= x;
  return r;
}

// Harmonic index h within multipole l: h = 0 -> m = 0; h = 2a-1 -> m = +a; h = 2a -> m = -a.
__host__ __device__ __forceinline__ int harm_a(int h) { return (h + 1) >> 1; }
__host__ __device__ __forceinline__ int harm_sign(int h) { return h == 0 ? 0 : ((h & 1) ? 1 : -1); }

// 1/sqrt(x) to within about half an ulp. In FP32 the hardware approximation is refined by one
// Newton step: its error is the same for every mode of a shell (same |n|^2), and as the
// reduced q_l^a(z) are not homogeneous in the direction's length, an unrefined error would
// change the shape of Y_lm over the shell (leaking the shot noise into P_l, l >= 2).
template <typename T> __device__ __forceinline__ T rsqrt_t(T x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) {
  const float y = rsqrtf(x);
  const float e = fmaf(-(x * y), y, 1.0f);  // 1 - x y^2
  return fmaf(0.5f * y, e, y);
}
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }


}  // namespace pspec
