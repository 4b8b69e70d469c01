// Double-float arithmetic: every value an unevaluated sum of two floats
// (hi + lo, about 44-48 significant bits) on the FP32 units. Products use the
// exact FMA product error, sums use TwoSum; accumulators keep a compensated
// (hi, lo) pair. Complex values are float4 (re.hi, re.lo, im.hi, im.lo).
#pragma once

#include "pinv_internal.h"

namespace pinv {

// ------------------------------------------------------------------ double-float arithmetic
__device__ inline float4 to_df(double2 v) {
    const float rh = (float)v.x, ih = (float)v.y;
    return make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
}
__device__ inline double2 from_df(float4 a) {
    return make_double2((double)a.x + (double)a.y, (double)a.z + (double)a.w);
}
__device__ inline void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ inline void fast_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    e = b - (s - a);
}
// The same conversions without the FP64 pipe (integer and FP32 instructions only),
// for kernels that convert many values on one SM.
// (float)x, round to nearest even, on the integer pipe (the FP64 conversion for
// zero, results outside the normal float range, infinity and NaN)
__device__ inline float f64_to_f32_rn(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ffu);
    const int fe = ex - 1023 + 127;
    if (ex == 0 || ex == 0x7ff || fe <= 0 || fe >= 255) return (float)x;
    const unsigned m = (unsigned)((b >> 29) & 0x7fffffu), rem = (unsigned)(b & 0x1fffffffu);
    unsigned u = ((unsigned)(b >> 32) & 0x80000000u) | ((unsigned)fe << 23) | m;
    if (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ++u;  // a carry moves into the exponent
    return __uint_as_float(u);
}
// to_df on the integer pipe, bit for bit: hi = (float)x, lo = (float)(x - hi)
// (the FP64 conversion where lo or hi would leave the normal float range)
__device__ inline float2 f64_to_df_rn(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ffu);
    const int fe = ex - 1023 + 127;
    if (ex == 0 || ex == 0x7ff || fe <= 52 || fe >= 254) {
        const float h = (float)x;
        return make_float2(h, (float)(x - (double)h));
    }
    const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
    const unsigned m = (unsigned)((b >> 29) & 0x7fffffu), rem = (unsigned)(b & 0x1fffffffu);
    const bool up = rem > 0x10000000u || (rem == 0x10000000u && (m & 1u));
    const unsigned u = (sgn | ((unsigned)fe << 23) | m) + (up ? 1u : 0u);
    const int d = up ? (int)rem - (1 << 29) : (int)rem;  // |x| - |hi| in units of 2^(E - 52)
    const float l = (float)(sgn ? -d : d) * __uint_as_float((unsigned)(fe - 52) << 23);
    return make_float2(__uint_as_float(u), l);
}
__device__ inline float4 to_df_i(double2 v) {
    const float2 r = f64_to_df_rn(v.x), i = f64_to_df_rn(v.y);
    return make_float4(r.x, r.y, i.x, i.y);
}
// (hi, lo) -> double within one unit in the last place: hi exactly, plus lo
// rounded to hi's grid (units of 2^-52 |hi|, twice as fine below a power of two).
__device__ inline double join_f64(float h, float l) {
    const unsigned hb = __float_as_uint(h), lb = __float_as_uint(l);
    const int eh = (int)((hb >> 23) & 0xffu), el = (int)((lb >> 23) & 0xffu);
    if (eh == 0 || eh == 0xff || el == 0xff) return (double)h + (double)l;
    const unsigned mh = hb & 0x7fffffu;
    unsigned long long bits = ((unsigned long long)(hb & 0x80000000u) << 32) |
                              ((unsigned long long)(eh - 127 + 1023) << 52) | ((unsigned long long)mh << 29);
    if (el == 0) return __longlong_as_double((long long)bits);  // lo zero or below the float range
    // lo in units of hi's last place: (2^23 + ml) * 2^(el - eh + 29)
    const unsigned ml = (lb & 0x7fffffu) | 0x800000u;
    const int sh = el - eh + 29;
    unsigned long long d;
    if (sh >= 0)
        d = sh < 40 ? (unsigned long long)ml << sh : 0ull;  // |lo| <= ulp(hi) keeps sh <= 6
    else
        d = -sh < 26 ? ((unsigned long long)ml + (1ull << (-sh - 1))) >> -sh : 0ull;
    if ((hb ^ lb) & 0x80000000u)
        bits -= mh == 0 ? 2 * d : d;  // below a power of two the grid is twice as fine
    else
        bits += d;
    return __longlong_as_double((long long)bits);
}
// (xh + xl)(yh + yl) as a normalised pair
__device__ inline void df_mul(float xh, float xl, float yh, float yl, float& rh, float& rl) {
    const float p = xh * yh;
    float e = fmaf(xh, yh, -p);
    e = fmaf(xh, yl, e);
    e = fmaf(xl, yh, e);
    fast_two_sum(p, e, rh, rl);
}
__device__ inline void df_add(float ah, float al, float bh, float bl, float& rh, float& rl) {
    float s, e;
    two_sum(ah, bh, s, e);
    e += al + bl;
    fast_two_sum(s, e, rh, rl);
}
// complex double-float product, layout (re.hi, re.lo, im.hi, im.lo)
__device__ inline float4 cdf_mul(float4 a, float4 b) {
    float p1h, p1l, p2h, p2l, p3h, p3l, p4h, p4l, rh, rl, ih, il;
    df_mul(a.x, a.y, b.x, b.y, p1h, p1l);
    df_mul(a.z, a.w, b.z, b.w, p2h, p2l);
    df_mul(a.x, a.y, b.z, b.w, p3h, p3l);
    df_mul(a.z, a.w, b.x, b.y, p4h, p4l);
    df_add(p1h, p1l, -p2h, -p2l, rh, rl);
    df_add(p3h, p3l, p4h, p4l, ih, il);
    return make_float4(rh, rl, ih, il);
}
__device__ inline float4 cdf_conj(float4 a) { return make_float4(a.x, a.y, -a.z, -a.w); }
// H + L += x * y (x, y double-float reals)
__device__ inline void acc_prod(float& H, float& L, float xh, float xl, float yh, float yl) {
    const float p = xh * yh;
    float e = fmaf(xh, yh, -p);
    e = fmaf(xh, yl, e);
    e = fmaf(xl, yh, e);
    float s, t;
    two_sum(H, p, s, t);
    H = s;
    L += t + e;
}
// complex accumulate acc += a * b, acc = (re.H, re.L, im.H, im.L)
__device__ inline void cacc(float4& acc, float4 a, float4 b) {
    acc_prod(acc.x, acc.y, a.x, a.y, b.x, b.y);
    acc_prod(acc.x, acc.y, -a.z, -a.w, b.z, b.w);
    acc_prod(acc.z, acc.w, a.x, a.y, b.z, b.w);
    acc_prod(acc.z, acc.w, a.z, a.w, b.x, b.y);
}

// ------------------------------------------------------------------ double-float matrix storage
// Mixed plans hold G (then L) and W = L^-1 in double-float form while they are
// factored and inverted: a complex entry is the float4 (re.hi, re.lo, im.hi, im.lo)
// in the 16 bytes of a complex double, so every update runs on the FP32 pipe (GB300
// issues about one FP64 add per clock per SM). Zero has the same bits in both forms.
__device__ inline float4 df_of_f32(float2 v) { return make_float4(v.x, 0.f, v.y, 0.f); }
// a - v for an FP32 v: TwoSum of the leading parts, the error added to the trailing
// part, renormalised. Where the leading parts cancel their difference is exact and
// at least the trailing part, so the final fast TwoSum is exact too.
__device__ inline float4 df_sub_f32(float4 a, float2 v) {
    float s, e, rh, rl, ih, il;
    two_sum(a.x, -v.x, s, e);
    fast_two_sum(s, a.y + e, rh, rl);
    two_sum(a.z, -v.y, s, e);
    fast_two_sum(s, a.w + e, ih, il);
    return make_float4(rh, rl, ih, il);
}
// the FP32 rounding of a double-float complex value
__device__ inline float2 df_to_f32(float4 a) { return make_float2(a.x + a.y, a.z + a.w); }
// FP64 from double-float on the integer pipe (join_f64)
__device__ inline double2 df_to_f64(float4 a) { return make_double2(join_f64(a.x, a.y), join_f64(a.z, a.w)); }

// encoding element A[m][n] and E[(c,m)][n] from the double-float tables
__device__ inline float4 gen_a_df(const EncodeDev& e, int64_t m, int64_t n) {
    const int* g = e.vox_ijk + 3 * n;
    float4 v = e.exdf[m * e.nx + g[0]];
    if (e.ny > 1) v = cdf_mul(v, e.eydf[m * e.ny + g[1]]);
    if (e.nz > 1) v = cdf_mul(v, e.ezdf[m * e.nz + g[2]]);
    if (e.b0df) v = cdf_mul(v, e.b0df[(int64_t)e.tidx[m] * e.N + n]);
    return v;
}
__device__ inline float4 gen_e_df(const EncodeDev& e, int c, int64_t m, int64_t n) {
    float4 v = gen_a_df(e, m, n);
    if (e.coilsdf) v = cdf_mul(v, e.coilsdf[(int64_t)c * e.N + n]);
    return v;
}

}  // namespace pinv
