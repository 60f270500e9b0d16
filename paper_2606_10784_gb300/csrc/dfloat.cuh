// Double-float complex arithmetic: FP64-class accuracy on the FP32 pipe.
//
// GB300's FP64 rate is about 1/64 of its FP32 rate, so the FP64-accurate grid product runs its
// FFTs in "double-float" arithmetic: every real value is an unevaluated sum hi + lo of two
// floats (T. J. Dekker, "A floating-point technique for extending the available precision",
// 1971); inputs are split with |lo| <= ulp(hi)/2, results are left unnormalised (see df_add). Sums use Knuth's error-free TwoSum, products the FMA-based
// exact product a*b = p + fma(a, b, -p). The relative error of one operation is about 2^-47
// (sums are accurate relative to |a|+|b|, which is what the normwise error bound of an FFT
// needs). Every operation is written with explicit round-to-nearest intrinsics so that the
// compiler cannot contract or reassociate the error-free transformations.
#pragma once

#include <cuda_runtime.h>

namespace aim {

// Laid out as (xh, yh, xl, yl): the high parts and the low parts of re and im are register pairs,
// so the complex sums and products below run the real and imaginary parts' identical operation
// sequences as paired FP32 instructions (__fadd2_rn, __fmul2_rn, __ffma2_rn: one instruction for
// two lanes of the same operation, each component rounded exactly as its scalar form).
struct __align__(16) dfc {
  float xh, yh, xl, yl;   // re = xh + xl, im = yh + yl
};

__device__ __forceinline__ void ef_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (ah + al) + (bh + bl). Results are left unnormalised: rl may exceed half an ulp of rh. Every
// consumer (another of these operations, the hi + lo conversion to binary64, storage) is exact
// for such pairs, and skipping the renormalising FastTwoSum saves 3 of 11 instructions. The
// normwise error of a 2048-point convolution round trip goes from ~9e-15 to ~2e-14.
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& rh, float& rl) {
  float s, e;
  ef_two_sum(ah, bh, s, e);
  rh = s;
  rl = __fadd_rn(e, __fadd_rn(al, bl));
}

// (ah + al)(bh + bl) - (ch + cl)(dh + dl)  (sign = -1)  or  ... + ...  (sign = +1)
template <int SIGN>
__device__ __forceinline__ void df_dot2(float ah, float al, float bh, float bl, float ch, float cl, float dh,
                                        float dl, float& rh, float& rl) {
  const float p1 = __fmul_rn(ah, bh);
  const float e1 = __fmaf_rn(ah, bh, -p1);
  const float cs = SIGN > 0 ? ch : -ch;
  const float cls = SIGN > 0 ? cl : -cl;
  const float p2 = __fmul_rn(cs, dh);
  const float e2 = __fmaf_rn(cs, dh, -p2);
  float s, es;
  ef_two_sum(p1, p2, s, es);
  float err = __fadd_rn(es, __fadd_rn(e1, e2));
  err = __fmaf_rn(ah, bl, err);
  err = __fmaf_rn(al, bh, err);
  err = __fmaf_rn(cs, dl, err);
  err = __fmaf_rn(cls, dh, err);
  rh = s;   // unnormalised, as in df_add
  rl = err;
}

// ---- paired forms: lane 0 carries the real part's operation, lane 1 the imaginary part's
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __fadd2_rn(a, f2neg(b)); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// df_add on both lanes: (ah + al) + (bh + bl), TwoSum of the high parts, unnormalised
__device__ __forceinline__ void df_add2(float2 ah, float2 al, float2 bh, float2 bl, float2& rh, float2& rl) {
  const float2 s = f2add(ah, bh);
  const float2 bb = f2sub(s, ah);
  const float2 e = f2add(f2sub(ah, f2sub(s, bb)), f2sub(bh, bb));
  rh = s;
  rl = f2add(e, f2add(al, bl));
}

// df_dot2 on both lanes: (ah + al)(bh + bl) + (ch + cl)(dh + dl), the signs folded into c by the
// caller (lane by lane the same operations as df_dot2)
__device__ __forceinline__ void df_dot2_2(float2 ah, float2 al, float2 bh, float2 bl, float2 ch, float2 cl, float2 dh,
                                          float2 dl, float2& rh, float2& rl) {
  const float2 p1 = f2mul(ah, bh);
  const float2 e1 = f2fma(ah, bh, f2neg(p1));
  const float2 p2 = f2mul(ch, dh);
  const float2 e2 = f2fma(ch, dh, f2neg(p2));
  const float2 s = f2add(p1, p2);
  const float2 bb = f2sub(s, p1);
  const float2 es = f2add(f2sub(p1, f2sub(s, bb)), f2sub(p2, bb));
  float2 err = f2add(es, f2add(e1, e2));
  err = f2fma(ah, bl, err);
  err = f2fma(al, bh, err);
  err = f2fma(ch, dl, err);
  err = f2fma(cl, dh, err);
  rh = s;
  rl = err;
}

__device__ __forceinline__ dfc cadd(dfc a, dfc b) {
  float2 rh, rl;
  df_add2(f2(a.xh, a.yh), f2(a.xl, a.yl), f2(b.xh, b.yh), f2(b.xl, b.yl), rh, rl);
  return dfc{rh.x, rh.y, rl.x, rl.y};
}

__device__ __forceinline__ dfc csub(dfc a, dfc b) {
  float2 rh, rl;
  df_add2(f2(a.xh, a.yh), f2(a.xl, a.yl), f2(-b.xh, -b.yh), f2(-b.xl, -b.yl), rh, rl);
  return dfc{rh.x, rh.y, rl.x, rl.y};
}

// (x + iy)(u + iv) = (xu - yv) + i(xv + yu): lane 0 x u + (-y) v, lane 1 x v + y u
__device__ __forceinline__ dfc cmul(dfc a, dfc b) {
  float2 rh, rl;
  df_dot2_2(f2(a.xh, a.xh), f2(a.xl, a.xl), f2(b.xh, b.yh), f2(b.xl, b.yl), f2(-a.yh, a.yh), f2(-a.yl, a.yl),
            f2(b.yh, b.xh), f2(b.yl, b.xl), rh, rl);
  return dfc{rh.x, rh.y, rl.x, rl.y};
}

// a * conj(b) = (xu + yv) + i(yu - xv): lane 0 x u + y v, lane 1 y u + (-x) v
__device__ __forceinline__ dfc cmulc(dfc a, dfc b) {
  float2 rh, rl;
  df_dot2_2(f2(a.xh, a.yh), f2(a.xl, a.yl), f2(b.xh, b.xh), f2(b.xl, b.xl), f2(a.yh, -a.xh), f2(a.yl, -a.xl),
            f2(b.yh, b.yh), f2(b.yl, b.yl), rh, rl);
  return dfc{rh.x, rh.y, rl.x, rl.y};
}

// conj(a) * b = (ax bx + ay by) + i(ax by - ay bx): lane 0 ax bx + ay by, lane 1 ax by + (-ay) bx
__device__ __forceinline__ dfc cconjmul(dfc a, dfc b) {
  float2 rh, rl;
  df_dot2_2(f2(a.xh, a.xh), f2(a.xl, a.xl), f2(b.xh, b.yh), f2(b.xl, b.yl), f2(a.yh, -a.yh), f2(a.yl, -a.yl),
            f2(b.yh, b.xh), f2(b.yl, b.xl), rh, rl);
  return dfc{rh.x, rh.y, rl.x, rl.y};
}

__device__ __forceinline__ dfc mul_minus_i(dfc a) {
  dfc r;
  r.xh = a.yh; r.xl = a.yl; r.yh = -a.xh; r.yl = -a.xl;
  return r;
}
__device__ __forceinline__ dfc mul_plus_i(dfc a) {
  dfc r;
  r.xh = -a.yh; r.xl = -a.yl; r.yh = a.xh; r.yl = a.xl;
  return r;
}

// split of a double into hi + lo floats (round to nearest each)
__device__ __forceinline__ void df_split(double d, float& h, float& l) {
  h = __double2float_rn(d);
  l = __double2float_rn(d - (double)h);
}

__host__ __device__ constexpr float df_hi(double d) { return (float)d; }
__host__ __device__ constexpr float df_lo(double d) { return (float)(d - (double)(float)d); }

// (ah + al) * c for a double-float constant c = ch + cl (exact product of the high parts by FMA,
// cross terms added to the low part; unnormalised like df_add)
__device__ __forceinline__ void df_scale(float ah, float al, float ch, float cl, float& rh, float& rl) {
  const float p = __fmul_rn(ah, ch);
  float e = __fmaf_rn(ah, ch, -p);
  e = __fmaf_rn(ah, cl, e);
  e = __fmaf_rn(al, ch, e);
  rh = p;
  rl = e;
}

// d * W16^e with double-float constants (forward W16 = exp(-2 pi i/16); inverse conjugate)
template <bool INV>
__device__ __forceinline__ dfc rot16(dfc d, int e) {
  constexpr double C1 = 0.92387953251128675613, S1 = 0.38268343236508977173, C2 = 0.70710678118654752440;
  switch (e) {
    case 0: return d;
    case 4: return INV ? mul_plus_i(d) : mul_minus_i(d);
    case 2:
    case 6: {
      // W8 and W8^3 have |re| = |im| = 1/sqrt2: one paired sum and one paired scaling (the two
      // lanes are the result's re and im) instead of a full complex product. With x + iy = d:
      //   forward e = 2: c (x + y) + i c (y - x)      inverse e = 2: c (x - y) + i c (x + y)
      //   forward e = 6: c (y - x) - i c (x + y)      inverse e = 6: -c (x + y) + i c (x - y)
      // (a sum of negated parts is the negated sum, bit for bit, as is its scaling)
      constexpr float ch = df_hi(C2), cl = df_lo(C2);
      float2 ah, al, bh, bl;
      if (e == 2) {
        if (INV) { ah = f2(d.xh, d.xh); al = f2(d.xl, d.xl); bh = f2(-d.yh, d.yh); bl = f2(-d.yl, d.yl); }
        else { ah = f2(d.xh, d.yh); al = f2(d.xl, d.yl); bh = f2(d.yh, -d.xh); bl = f2(d.yl, -d.xl); }
      } else {
        if (INV) { ah = f2(-d.xh, d.xh); al = f2(-d.xl, d.xl); bh = f2(-d.yh, -d.yh); bl = f2(-d.yl, -d.yl); }
        else { ah = f2(d.yh, -d.xh); al = f2(d.yl, -d.xl); bh = f2(-d.xh, -d.yh); bl = f2(-d.xl, -d.yl); }
      }
      float2 sh, sl;
      df_add2(ah, al, bh, bl, sh, sl);
      // df_scale on both lanes by (ch + cl)
      const float2 c2 = f2(ch, ch), c2l = f2(cl, cl);
      const float2 p = f2mul(sh, c2);
      float2 er = f2fma(sh, c2, f2neg(p));
      er = f2fma(sh, c2l, er);
      er = f2fma(sl, c2, er);
      return dfc{p.x, p.y, er.x, er.y};
    }
    default: {
      double c, s;
      switch (e) {
        case 1: c = C1; s = S1; break;
        case 2: c = C2; s = C2; break;
        case 3: c = S1; s = C1; break;
        case 5: c = -S1; s = C1; break;
        case 6: c = -C2; s = C2; break;
        default: c = -C1; s = S1; break;
      }
      // multiply by (c - i s) forward, (c + i s) inverse
      dfc w;
      w.xh = df_hi(c);
      w.xl = df_lo(c);
      w.yh = INV ? df_hi(s) : df_hi(-s);
      w.yl = INV ? df_lo(s) : df_lo(-s);
      return cmul(d, w);
    }
  }
}

}  // namespace aim
