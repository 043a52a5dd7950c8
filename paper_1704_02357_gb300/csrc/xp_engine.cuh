// Exact-add FP32 transform stages.
//
// The rounding error of an FP32 radix tree sits in its additions: every add level rounds its
// result (about 0.42 u rms of the output, u = 2^-24), nine levels per 512-point pass. In the
// harmonic transforms of the estimator (Sec. 2.1 eq. Fell) that noise is what limits how
// closely a multipole of a few percent of P_0 can be recovered against a shot noise of ~80 P_0.
//
// Here a stage keeps every value as a pair h + l of floats:
//   * h is a multiple of a power-of-two quantum q chosen per thread and stage from the thread's
//     inputs, so that every value of the stage's butterflies stays below 2^11 q: h has at most
//     12 significant bits above q. Sums and differences of such multiples are exact in FP32.
//   * Constants and twiddles are split the same way, K = K12 + Kr with K12 a multiple of 2^-12
//     (|K| <= 1) and Kr the remainder (held to 24 bits of its own). h * K12 then has at most 23
//     significant bits and is exact in FP32, and so are sums of such products; h * Kr and
//     l * K go to l, rounded at ~2^-24 q.
//   * A product lies on the finer quantum q/4096, so before a value is multiplied again it is
//     put back on q (re-split): g = (h + M) - M with M = 1.5 * 2^23 q rounds to q exactly and
//     h - g is exact.
// Values cross the shared-memory exchanges and leave the transform as h + l rounded to one
// float, so a pass rounds each value once per exchange and once at the end, instead of once per
// add level. Every operation whose exactness the scheme relies on uses the _rn intrinsics or an
// FMA whose result is exact, and the compiler never contracts the intrinsics into a multiply-add.
#pragma once
#include "fft_engine.cuh"

namespace pspec {

struct xf {
  float h, l;
};
struct xc {
  xf x, y;
};

__device__ __forceinline__ float xadd_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float xsub_(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float xmul_(float a, float b) { return __fmul_rn(a, b); }

// M = 1.5 * 2^23 * q for the smallest power-of-two q with `bound` <= 2^11 q.
__device__ __forceinline__ float xmagic(float bound) {
  int eb = (__float_as_int(bound) >> 23) & 0xff;  // bound < 2^(eb - 126)
  eb = eb > 240 ? 240 : eb;
  return __int_as_float(((eb + 13) << 23) | 0x400000);  // q = 2^(eb - 137), M = 1.5 * 2^(eb - 114)
}
__device__ __forceinline__ float xgrid(float p, float M) { return xsub_(xadd_(p, M), M); }

__device__ __forceinline__ xf xsplit(float v, float M) {
  const float g = xgrid(v, M);
  return {g, xsub_(v, g)};
}
__device__ __forceinline__ xc xsplit(float2 v, float M) { return {xsplit(v.x, M), xsplit(v.y, M)}; }
// back onto the quantum q before another multiplication
__device__ __forceinline__ xf xresplit(xf a, float M) {
  const float g = xgrid(a.h, M);
  return {g, xadd_(a.l, xsub_(a.h, g))};
}
__device__ __forceinline__ xc xresplit(xc a, float M) { return {xresplit(a.x, M), xresplit(a.y, M)}; }
__device__ __forceinline__ float xround(xf a) { return xadd_(a.h, a.l); }
__device__ __forceinline__ float2 xround(xc a) { return make_float2(xround(a.x), xround(a.y)); }

__device__ __forceinline__ xf operator+(xf a, xf b) { return {xadd_(a.h, b.h), xadd_(a.l, b.l)}; }
__device__ __forceinline__ xf operator-(xf a, xf b) { return {xsub_(a.h, b.h), xsub_(a.l, b.l)}; }
__device__ __forceinline__ xf operator-(xf a) { return {-a.h, -a.l}; }
__device__ __forceinline__ xc operator+(xc a, xc b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ xc operator-(xc a, xc b) { return {a.x - b.x, a.y - b.y}; }
// a * (i * sgn)
__device__ __forceinline__ xc xmul_i(xc a, int sgn) { return sgn > 0 ? xc{-a.y, a.x} : xc{a.y, -a.x}; }
__device__ __forceinline__ xc xconj(xc a) { return {a.x, -a.y}; }
__device__ __forceinline__ xf xhalf(xf a) { return {0.5f * a.h, 0.5f * a.l}; }  // exact

// A constant |K| <= 1 as K12 (a multiple of 2^-12) + Kr, with kf = K rounded to FP32.
struct K12 {
  float k12, kr, kf;
  __device__ __forceinline__ constexpr K12(double k)
      : k12((float)((double)(long long)(k * 4096.0 + (k >= 0 ? 0.5 : -0.5)) / 4096.0)),
        kr((float)(k - (double)(long long)(k * 4096.0 + (k >= 0 ? 0.5 : -0.5)) / 4096.0)),
        kf((float)k) {}
};
// a * K; a.h on the quantum q (at most 12 significant bits): a.h * K12 is exact.
__device__ __forceinline__ xf xcm(xf a, const K12& k) {
  return {xmul_(a.h, k.k12), fmaf(a.l, k.kf, a.h * k.kr)};
}

// a * w for a twiddle in the 12-bit form {c12, s12, cr, sr} (tables built on the host); a on the
// quantum q. The h parts are exact: each product has at most 23 significant bits and the FMA's
// exact result is representable.
__device__ __forceinline__ xc xtw(xc a, float4 w) {
  const float cf = xadd_(w.x, w.z), sf = xadd_(w.y, w.w);
  xc r;
  r.x.h = fmaf(a.x.h, w.x, -xmul_(a.y.h, w.y));
  r.y.h = fmaf(a.x.h, w.y, xmul_(a.y.h, w.x));
  r.x.l = fmaf(a.x.l, cf, fmaf(-a.y.l, sf, fmaf(a.x.h, w.z, -(a.y.h * w.w))));
  r.y.l = fmaf(a.x.l, sf, fmaf(a.y.l, cf, fmaf(a.x.h, w.w, a.y.h * w.z)));
  return r;
}
__device__ __forceinline__ xc xtw(float2 a, float4 w, float M) { return xtw(xsplit(a, M), w); }
// conjugate twiddle (inverse transforms)
__device__ __forceinline__ float4 xconj_w(float4 w) { return make_float4(w.x, -w.y, w.z, -w.w); }

// ------------------------------------------------------------------ butterflies
// The radix-R DFTs of common.cuh (same decompositions and constants) on exact-add values. The
// inputs may lie on the finer quantum (twiddled): a value is re-split before each internal
// multiplication.
template <int R> struct XDft;

template <> struct XDft<2> {
  static __device__ __forceinline__ void run(xc* v, int, float) {
    const xc a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  }
};

template <> struct XDft<4> {
  static __device__ __forceinline__ void run(xc* v, int dir, float) {
    const xc t0 = v[0] + v[2], t1 = v[0] - v[2];
    const xc t2 = v[1] + v[3], t3 = v[1] - v[3];
    const xc it3 = xmul_i(t3, dir);
    v[0] = t0 + t2;
    v[2] = t0 - t2;
    v[1] = t1 + it3;
    v[3] = t1 - it3;
  }
};

// z * (sr cr + i si ci) with sr, si = +-1
__device__ __forceinline__ xc xrot(xc z, const K12& cr, const K12& ci, int sr, int si, float M) {
  z = xresplit(z, M);
  const xf ax = xcm(z.x, cr), ay = xcm(z.y, ci);  // cr z.x, ci z.y
  const xf bx = xcm(z.y, cr), by = xcm(z.x, ci);  // cr z.y, ci z.x
  const xf p = sr > 0 ? ax : -ax, q = si > 0 ? ay : -ay;
  const xf s = sr > 0 ? bx : -bx, u = si > 0 ? by : -by;
  return {p - q, s + u};
}
// z * (sgn + dir i) / sqrt2 (sgn = +-1)
__device__ __forceinline__ xc xdiag(xc z, int sgn, int dir, const K12& h, float M) {
  const xf zx = sgn > 0 ? z.x : -z.x, zy = sgn > 0 ? z.y : -z.y;
  const xf re = dir > 0 ? zx - z.y : zx + z.y;  // sgn z.x - dir z.y
  const xf im = dir > 0 ? zy + z.x : zy - z.x;  // sgn z.y + dir z.x
  return {xcm(xresplit(re, M), h), xcm(xresplit(im, M), h)};
}

template <> struct XDft<8> {
  static __device__ __forceinline__ void run(xc* v, int dir, float M) {
    const K12 h(0.70710678118654752440);
    xc e[4] = {v[0], v[2], v[4], v[6]};
    xc o[4] = {v[1], v[3], v[5], v[7]};
    XDft<4>::run(e, dir, M);
    XDft<4>::run(o, dir, M);
    const xc o1 = xdiag(o[1], 1, dir, h, M);
    const xc o2 = xmul_i(o[2], dir);
    const xc o3 = xdiag(o[3], -1, dir, h, M);
    v[0] = e[0] + o[0];
    v[4] = e[0] - o[0];
    v[1] = e[1] + o1;
    v[5] = e[1] - o1;
    v[2] = e[2] + o2;
    v[6] = e[2] - o2;
    v[3] = e[3] + o3;
    v[7] = e[3] - o3;
  }
};

template <> struct XDft<16> {
  static __device__ __forceinline__ void run(xc* v, int dir, float M) {
    const K12 h(0.70710678118654752440), c1(0.92387953251128675613), s1(0.38268343236508977173);
    xc a[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; n2++) {
      xc t[4] = {v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]};
      XDft<4>::run(t, dir, M);
#pragma unroll
      for (int k1 = 0; k1 < 4; k1++) a[n2][k1] = t[k1];
    }
    const int d = dir;
    a[1][1] = xrot(a[1][1], c1, s1, 1, d, M);    // m = 1
    a[1][2] = xdiag(a[1][2], 1, d, h, M);        // m = 2
    a[1][3] = xrot(a[1][3], s1, c1, 1, d, M);    // m = 3
    a[2][1] = xdiag(a[2][1], 1, d, h, M);        // m = 2
    a[2][2] = xmul_i(a[2][2], d);                // m = 4
    a[2][3] = xdiag(a[2][3], -1, d, h, M);       // m = 6
    a[3][1] = xrot(a[3][1], s1, c1, 1, d, M);    // m = 3
    a[3][2] = xdiag(a[3][2], -1, d, h, M);       // m = 6
    a[3][3] = xrot(a[3][3], c1, s1, -1, -d, M);  // m = 9
#pragma unroll
    for (int k1 = 0; k1 < 4; k1++) {
      xc t[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
      XDft<4>::run(t, dir, M);
#pragma unroll
      for (int k2 = 0; k2 < 4; k2++) v[k1 + 4 * k2] = t[k2];
    }
  }
};

template <> struct XDft<3> {
  static __device__ __forceinline__ void run(xc* v, int dir, float M) {
    const K12 s3(0.86602540378443864676);
    const xc t = v[1] + v[2];
    const xc u = xresplit(v[1] - v[2], M);
    const xc m = v[0] - xc{xhalf(t.x), xhalf(t.y)};
    const xf sx = xcm(u.x, s3), sy = xcm(u.y, s3);
    const xc isu = dir > 0 ? xc{-sy, sx} : xc{sy, -sx};  // i dir sin(2 pi/3) u
    v[0] = v[0] + t;
    v[1] = m + isu;
    v[2] = m - isu;
  }
};

// ------------------------------------------------------------------ stages
// One Stockham stage as stage_ct (fft_engine.cuh) on float2 values held per thread, computed in
// exact-add arithmetic. The quantum is chosen from the thread's E inputs: every intermediate of
// a butterfly is a sum of its inputs times factors of modulus <= 1, so each component stays below
// sqrt(2) times the sum of the inputs' |re| + |im|; the bound passed is twice that sum.
template <int E, int L, int R, int NS, bool LAST, int LAYOUT, int NSEQ, int DIR>
__device__ __forceinline__ void stage_xp(float2 (&v)[E], float2* sm, int t, int seq, const float4* __restrict__ tw) {
  constexpr int Q = E / R;
  constexpr int Tc = L / E;
  constexpr int TSTEP = L / (NS * R);
  constexpr bool kShared = (Q > 1) && (NS > 1) && !LAST && (NS <= Tc);
  float4 ws[kShared ? R : 1];
  if constexpr (kShared) {
    const int k = t & (NS - 1);
#pragma unroll
    for (int r = 1; r < R; r++) {
      ws[r] = ldg_u(tw + r * k * TSTEP);
      if (DIR > 0) ws[r] = uconj(ws[r]);
    }
  }
  float bound = 0.f;
#pragma unroll
  for (int e = 0; e < E; e++) bound += fabsf(v[e].x) + fabsf(v[e].y);
  const float M = xmagic(2.f * bound);  // twice: a rotated component reaches sqrt2 |x|
#pragma unroll
  for (int q = 0; q < Q; q++) {
    const int j = t + Tc * q;
    const int k = LAST ? j : (j & (NS - 1));
    xc u[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
      if (NS > 1 && r > 0) {
        float4 w;
        if constexpr (kShared) {
          w = ws[r];
        } else {
          w = ldg_u(tw + r * k * TSTEP);
          if (DIR > 0) w = uconj(w);
        }
        u[r] = xtw(v[q + r * Q], w, M);  // the 12-bit twiddle table
      } else {
        u[r] = xsplit(v[q + r * Q], M);
      }
    }
    XDft<R>::run(u, DIR, M);
    if constexpr (LAST) {
#pragma unroll
      for (int r = 0; r < R; r++) v[q + r * Q] = xround(u[r]);
    } else {
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; r++) sm[sidx<LAYOUT, L, NSEQ>(seq, base + r * NS)] = xround(u[r]);
    }
  }
}

// fft_ct in exact-add arithmetic (same plan, layouts and synchronisation).
template <int E, int L, int LAYOUT, int NSEQ, int DIR, bool WARP = false>
__device__ __forceinline__ void fft_xp(float2 (&v)[E], float2* sm, int t, int seq, const float4* __restrict__ tw) {
  constexpr CtPlan P = ct_plan(L, E);
  constexpr int Tc = L / E;
  static_assert(!WARP || (LAYOUT == kPaddedRows && Tc <= 32 && 32 % Tc == 0), "warp-synchronous rows only");
  static_for<0, P.nst>([&](auto s_) {
    constexpr int s = decltype(s_)::value;
    constexpr bool last = (s == P.nst - 1);
    stage_xp<E, L, P.rad[s], P.ns[s], last, LAYOUT, NSEQ, DIR>(v, sm, t, seq, tw);
    if constexpr (!last) {
      fft_sync<WARP>();
#pragma unroll
      for (int e = 0; e < E; e++) v[e] = sm[sidx<LAYOUT, L, NSEQ>(seq, t + Tc * e)];
      fft_sync<WARP>();
    }
  });
}

// The transform the kernels call: exact-add stages when XP, else the plain engine.
template <bool XP, typename C, int E, int L, int LAYOUT, int NSEQ, int DIR, bool WARP = false>
__device__ __forceinline__ void fft_any(C (&v)[E], C* sm, int t, int seq, const ux_of<C>* __restrict__ tw) {
  if constexpr (XP)
    fft_xp<E, L, LAYOUT, NSEQ, DIR, WARP>(v, sm, t, seq, tw);
  else
    fft_ct<C, E, L, LAYOUT, NSEQ, DIR, WARP>(v, sm, t, seq, tw);
}

// r2c unpack (k_r2c_z) in exact-add arithmetic: 2X[k] = (Z[k] + Z*[L-k]) - i w^k (Z[k] - Z*[L-k]),
// halved once at the end (exact); w in the 12-bit form.
__device__ __forceinline__ float2 r2c_unpack_xp(float2 zk, float2 zm, float4 w) {
  const float bound = fabsf(zk.x) + fabsf(zk.y) + fabsf(zm.x) + fabsf(zm.y);
  const float M = xmagic(4.f * bound);
  const xc a = xsplit(zk, M), b = xconj(xsplit(zm, M));
  const xc s = a + b, d = a - b;
  const xc o = xtw(xc{d.y, -d.x}, w);  // -i d w
  const float2 r = xround(s + o);
  return make_float2(0.5f * r.x, 0.5f * r.y);
}

// c2r pack (k_c2r_z) in exact-add arithmetic: with A = X[k] and B = conj(X[L-k]) (0 for k = 0),
// 2Z = (A + B) + i (A - B) conj(w^k), halved once at the end; wc = conj(w^k) in the 12-bit form.
__device__ __forceinline__ float2 c2r_pack_xp(float2 xk, float2 xm, float4 wc) {
  const float bound = fabsf(xk.x) + fabsf(xk.y) + fabsf(xm.x) + fabsf(xm.y);
  const float M = xmagic(4.f * bound);
  const xc a = xsplit(xk, M), b = xconj(xsplit(xm, M));
  const xc ev = a + b, od = xtw(a - b, wc);
  const float2 r = xround(xc{ev.x - od.y, ev.y + od.x});  // 2E + i 2O'
  return make_float2(0.5f * r.x, 0.5f * r.y);
}

}  // namespace pspec
