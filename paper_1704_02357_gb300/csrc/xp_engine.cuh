// Exact-add FP32 transform stages.
//
// The rounding error of an FP32 radix tree sits in its additions: every add level rounds its
// result (about 0.42 u rms of the output, u = 2^-24), nine levels per 512-point pass. In the
// harmonic transforms of the estimator (Sec. 2.1 eq. Fell) that noise is what limits how
// closely a multipole of a few percent of P_0 can be recovered against a shot noise of ~80 P_0.
//
// Here a stage keeps every value as a pair h + l of floats:
//   * h is a multiple of a power-of-two quantum q chosen per thread and stage, large enough
//     that every partial sum of the stage's butterflies stays below 2^22 q. Sums and
//     differences of such multiples are exact in FP32, so the butterfly additions of h never
//     round.
//   * l carries what h cannot hold: the part of a product below q and the product's own
//     rounding error (an FMA gives it exactly). l stays within a few q, so its own roundings are
//     ~2^-24 q, far below the rounding of the stored result.
// A product p is put on the grid with the magic-number rounding g = (p + M) - M,
// M = 1.5 * 2^23 q (exact for |p| < 2^22 q); p - g is then exact as well.
//
// Values cross the shared-memory exchanges and leave the transform as h + l rounded to one
// float, so a pass rounds each value once per exchange and once at the end, instead of once per
// add level. Every operation whose exactness the scheme relies on uses the _rn intrinsics,
// which the compiler never contracts into a multiply-add.
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

// M = 1.5 * 2^23 * q for the smallest power-of-two q with `bound` < 2^22 q.
__device__ __forceinline__ float xmagic(float bound) {
  int eb = (__float_as_int(bound) >> 23) & 0xff;  // bound < 2^(eb - 126)
  eb = eb > 250 ? 250 : eb;
  return __int_as_float(((eb + 2) << 23) | 0x400000);  // 1.5 * 2^(eb - 125)
}
__device__ __forceinline__ float xgrid(float p, float M) { return xsub_(xadd_(p, M), M); }

__device__ __forceinline__ xf xsplit(float v, float M) {
  const float g = xgrid(v, M);
  return {g, xsub_(v, g)};
}
__device__ __forceinline__ xc xsplit(float2 v, float M) { return {xsplit(v.x, M), xsplit(v.y, M)}; }
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

// a * K for a constant K = hi + lo (ConstMul<float>): the exact product a.h * hi goes to the
// grid, its remainder and rounding error, a.h * lo and a.l * K to l.
__device__ __forceinline__ xf xcmul(xf a, const ConstMul<float>& k, float M) {
  const float p = xmul_(a.h, k.hi);
  const float e = fmaf(a.h, k.hi, -p);
  const float t = fmaf(a.h, k.lo, fmaf(a.l, k.hi, e));
  const float g = xgrid(p, M);
  return {g, xadd_(xsub_(p, g), t)};
}

// a * w for a unit twiddle w = {c_hi, s_hi, c_lo, s_lo} (tables as the plain stages use them).
__device__ __forceinline__ xc xtw(float2 a, float4 w, float M) {
  const float p1 = xmul_(a.x, w.x), e1 = fmaf(a.x, w.x, -p1);
  const float p2 = xmul_(a.y, w.y), e2 = fmaf(a.y, w.y, -p2);
  const float p3 = xmul_(a.x, w.y), e3 = fmaf(a.x, w.y, -p3);
  const float p4 = xmul_(a.y, w.x), e4 = fmaf(a.y, w.x, -p4);
  const float g1 = xgrid(p1, M), g2 = xgrid(p2, M), g3 = xgrid(p3, M), g4 = xgrid(p4, M);
  const float lre = fmaf(a.x, w.z, fmaf(-a.y, w.w, xsub_(e1, e2)));
  const float lim = fmaf(a.x, w.w, fmaf(a.y, w.z, xadd_(e3, e4)));
  xc r;
  r.x = {xsub_(g1, g2), xadd_(xsub_(xsub_(p1, g1), xsub_(p2, g2)), lre)};
  r.y = {xadd_(g3, g4), xadd_(xadd_(xsub_(p3, g3), xsub_(p4, g4)), lim)};
  return r;
}
__device__ __forceinline__ xc xtw(xc a, float4 w, float M) {
  xc r = xtw(make_float2(a.x.h, a.y.h), w, M);
  r.x.l = fmaf(a.x.l, w.x, fmaf(-a.y.l, w.y, r.x.l));
  r.y.l = fmaf(a.x.l, w.y, fmaf(a.y.l, w.x, r.y.l));
  return r;
}

// ------------------------------------------------------------------ butterflies
// The radix-R DFTs of common.cuh (same decompositions and constants) on exact-add values.
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
__device__ __forceinline__ xc xrot(xc z, const ConstMul<float>& cr, const ConstMul<float>& ci, int sr, int si,
                                   float M) {
  const xf ax = xcmul(z.x, cr, M), ay = xcmul(z.y, ci, M);  // cr z.x, ci z.y
  const xf bx = xcmul(z.y, cr, M), by = xcmul(z.x, ci, M);  // cr z.y, ci z.x
  const xf p = sr > 0 ? ax : -ax, q = si > 0 ? ay : -ay;
  const xf s = sr > 0 ? bx : -bx, u = si > 0 ? by : -by;
  return {p - q, s + u};
}
// z * (sgn + dir i) / sqrt2 (sgn = +-1)
__device__ __forceinline__ xc xdiag(xc z, int sgn, int dir, const ConstMul<float>& h, float M) {
  const xf zx = sgn > 0 ? z.x : -z.x, zy = sgn > 0 ? z.y : -z.y;
  const xf re = dir > 0 ? zx - z.y : zx + z.y;  // sgn z.x - dir z.y
  const xf im = dir > 0 ? zy + z.x : zy - z.x;  // sgn z.y + dir z.x
  return {xcmul(re, h, M), xcmul(im, h, M)};
}

template <> struct XDft<8> {
  static __device__ __forceinline__ void run(xc* v, int dir, float M) {
    const ConstMul<float> h(0.70710678118654752440);
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
    const ConstMul<float> h(0.70710678118654752440), c1(0.92387953251128675613), s1(0.38268343236508977173);
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

template <> struct XDft<32> {
  static __device__ __forceinline__ void run(xc* v, int dir, float M) {
    xc e[16], o[16];
#pragma unroll
    for (int i = 0; i < 16; i++) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    XDft<16>::run(e, dir, M);
    XDft<16>::run(o, dir, M);
    constexpr double kc[9] = {1.0, 0.98078528040323044913, 0.92387953251128675613, 0.83146961230254523708,
                              0.70710678118654752440, 0.55557023301960222474, 0.38268343236508977173,
                              0.19509032201612826785, 0.0};
#pragma unroll
    for (int k = 0; k < 16; k++) {
      xc w = o[k];
      if (k > 0) {
        const int kk = k <= 8 ? k : 16 - k;
        const ConstMul<float> cr(kc[kk]), ci(kc[8 - kk]);
        w = xrot(w, cr, ci, k <= 8 ? 1 : -1, dir, M);
      }
      v[k] = e[k] + w;
      v[k + 16] = e[k] - w;
    }
  }
};

template <> struct XDft<3> {
  static __device__ __forceinline__ void run(xc* v, int dir, float M) {
    const ConstMul<float> s3(0.86602540378443864676), half(0.5);
    const xc t = v[1] + v[2];
    const xc u = v[1] - v[2];
    const xc m = v[0] - xc{xcmul(t.x, half, M), xcmul(t.y, half, M)};
    const xf sx = xcmul(u.x, s3, M), sy = xcmul(u.y, s3, M);
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
  const float M = xmagic(2.f * bound);
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
        u[r] = xtw(v[q + r * Q], w, M);
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
// halved once at the end (exact).
__device__ __forceinline__ float2 r2c_unpack_xp(float2 zk, float2 zm, float4 w) {
  const float bound = fabsf(zk.x) + fabsf(zk.y) + fabsf(zm.x) + fabsf(zm.y);
  const float M = xmagic(4.f * bound);
  const xc a = xsplit(zk, M), b = xconj(xsplit(zm, M));
  const xc s = a + b, d = a - b;
  const xc o = xtw(xc{d.y, -d.x}, w, M);  // -i d w
  const float2 r = xround(s + o);
  return make_float2(0.5f * r.x, 0.5f * r.y);
}

// c2r pack (k_c2r_z) in exact-add arithmetic: Z = E + i O with 2E = X[k] + X*[L-k] and
// 2O = i conj(w^k) (X[k] - X*[L-k]) -> 2Z = (X[k] + X*[L-k]) - conj(w^k) (X[k] - X*[L-k]) ... halved at the end.
__device__ __forceinline__ float2 c2r_pack_xp(float2 xk, float2 xm, float4 wc) {
  const float bound = fabsf(xk.x) + fabsf(xk.y) + fabsf(xm.x) + fabsf(xm.y);
  const float M = xmagic(4.f * bound);
  const xc a = xsplit(xk, M), b = xconj(xsplit(xm, M));
  const xc ev = a + b, od = xtw(a - b, wc, M);  // 2E, 2O' = (X - X*) conj(w)
  const float2 r = xround(xc{ev.x - od.y, ev.y + od.x});  // 2E + i 2O'
  return make_float2(0.5f * r.x, 0.5f * r.y);
}

}  // namespace pspec
