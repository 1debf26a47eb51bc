// Device helpers of the FP64-accurate tensor-core forms (exact digit
// slicing, the Ozaki scheme): TMA bulk copies and mbarrier waits, balanced
// base-1024 digits (exact in FP16) of FP64 and double-float values, the
// double-float combination of the level sums, the bit-level split of FP64
// into hi + lo floats, and the double-float 3-term dot product of the
// geometric factor.
#pragma once

#include <algorithm>
#include <climits>

#include "ax_f64x.cuh"
#include "mma_sync.cuh"

namespace semax {
namespace oz {

using dfx::acc2;
using dfx::acc2x2;
using dfx::df;
using dfx::df2;
using dfx::dot2_step2;
using dfx::dot3_2;
using dfx::f2;
using dfx::pack_df2;
using dfx::prod2;
using dfx::sub2;
using dfx::two_sum2;
using mma::smem_u32;

constexpr int kBadExp = 1 << 20;             // marks a non-finite input in the exponent reductions

// Status word of a CTA whose staging wait gave up (NULL: not reported).  The
// CTA then marks every output it has not written NaN, waits once more (with
// the default poll limit) for its copies in flight, and leaves.
__device__ __forceinline__ void report_timeout(int *status) {
    if (status) atomicExch(status, (int)SEMAX_ETIMEOUT);
}

// TMA bulk copy global -> shared, completing on an mbarrier transaction
// count; the CTA is its own cluster, so its shared::cta address is valid.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, unsigned bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Wait for phase `parity` of the mbarrier, giving up after `polls` polls
// (each try_wait may itself suspend briefly): false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, unsigned parity, int polls = kDefaultWaitPolls) {
    for (int it = 0; it < polls; ++it) {
        unsigned done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ int bexp(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }
// |x|'s high word: the biased exponent in bits 20-30 above the top significand
// bits, so the largest such word of a group carries the group's largest
// exponent, and word >= (e << 20) tests exponent >= e
__device__ __forceinline__ unsigned habs(double x) { return (unsigned)__double2hiint(x) & 0x7fffffffu; }

// The integer v (|v| < 2^22) as a float, by the 1.5 * 2^23 bias.
__device__ __forceinline__ float int_to_float(int v) { return __fsub_rn(__int_as_float(0x4B400000 + v), 12582912.0f); }

// 2^k as a float for k in [-126, 127]; 0 below
__device__ __forceinline__ float pow2f_or_zero(int k) {
    return k < -126 ? 0.0f : __uint_as_float((unsigned)(min(k, 127) + 127) << 23);
}

// m 2^20 for a digit scale m = 2^k from pow2f_or_zero, clamped like it
__device__ __forceinline__ float times2p20(float m) { return fminf(__fmul_rn(m, 0x1p20f), 0x1p127f); }

// A Dot2 result s + c renormalised for digit extraction.  The fast two-sum
// is exact when |s| >= |c|, the usual case (c collects rounding errors);
// when a sum cancels below its own error terms it errs by at most ulp(c)/2,
// under the Dot2 sum's own error bound.
__device__ __forceinline__ acc2 renorm(acc2 y) {
    const df n = dfx::fast_two_sum(y.s, y.c);
    return acc2{n.hi, n.lo};
}

// ---- base-1024 digits in FP16 (five per operand)
//
// Balanced base-1024 digits are integers of magnitude <= 528 here, exact in
// FP16 (11 significant bits).  With K = 16 terms per product, the level sums
// of levels 0..2 stay below 2^24 and are exact in FP32; levels 3 and 4 may
// exceed it by a few per cent and round by a unit or two, at weights 2^-30
// and 2^-40 of level 0, which is far below the 2^-48 the five digits keep.

constexpr int kS10 = 5;

// Two integer-valued floats (|v| <= 2048) as an FP16 pair, a in the low half
// (exact: such a float has at most 11 significant bits).
__device__ __forceinline__ uint32_t pack_f16(float a, float b) {
    uint32_t d;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    return d;
}

// Balanced base-1024 digits of x * 2^-(E - 1022), E >= the biased exponent
// of x (at least 1): M = round(x * 2^(49 - (E - 1022))) = sum_q d[q]
// 2^(10 (4 - q)), |M| <= 2^49, d[1..4] in [-512, 511], |d[0]| <= 512.
// Integer arithmetic only.
__device__ __forceinline__ void digits10_fp64(double x, int E, float (&d)[kS10]) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int eb = (int)((b >> 52) & 0x7ffu);
    const unsigned long long m = (b & 0xfffffffffffffull) | (eb ? (1ull << 52) : 0ull);
    const int s = min(E + 4 - max(eb, 1), 63);   // >= 4
    long long M = (long long)((m + (1ull << (s - 1))) >> s);
    if (b >> 63) M = -M;
    int lo = (int)(M & 0x3fffffff);   // M = hi 2^30 + lo, lo in [0, 2^30)
    int hi = (int)(M >> 30);
    int q[kS10];
#pragma unroll
    for (int i = kS10 - 1; i >= 2; --i) {
        q[i] = ((lo + 512) & 1023) - 512;
        lo = (lo - q[i]) >> 10;
    }
    hi += lo;                         // carry (0 or 1)
    q[1] = ((hi + 512) & 1023) - 512;
    q[0] = (hi - q[1]) >> 10;
#pragma unroll
    for (int i = 0; i < kS10; ++i) d[i] = int_to_float(q[i]);
}

// Balanced base-1024 digits of the double-float value (hi + lo) m, m a
// power of two, |hi m| < 512 and |lo| <= ulp(hi) / 2 (normalised):
// (hi + lo) m = sum_q d[q] 2^(-10q) + (error <= 2^-41 + 2^-45), |d[2]| <= 528,
// the others <= 512.  Digits 0-2 come from hi alone, each step exact.  Then
// lo joins the remainder r2 of digit 2 (units of 2^-20): S = r2 + lo m 2^20
// (m20 = m 2^20) is exact when |lo m 2^20| >= 1/2, because hi then has no
// bits below 2^-20 and r2 = 0, and rounds by at most 2^-25 otherwise; S's
// integer part goes into digit 2 and its fraction, |f| <= 1/2 exactly, gives
// digits 3 and 4.
__device__ __forceinline__ void digits10_df(float hi, float lo, float m, float m20, float (&d)[kS10]) {
    constexpr float C = 12582912.0f;
    float q = __fsub_rn(__fmaf_rn(hi, m, C), C);
    float r = __fmaf_rn(hi, m, -q);
    d[0] = q;
    q = __fsub_rn(__fmaf_rn(r, 1024.0f, C), C);
    r = __fmaf_rn(r, 1024.0f, -q);
    d[1] = q;
    q = __fsub_rn(__fmaf_rn(r, 1024.0f, C), C);
    r = __fmaf_rn(r, 1024.0f, -q);
    const float S = __fmaf_rn(lo, m20, r);
    const float li = __fsub_rn(__fadd_rn(S, C), C);
    d[2] = __fadd_rn(q, li);
    r = __fsub_rn(S, li);
    q = __fsub_rn(__fmaf_rn(r, 1024.0f, C), C);
    r = __fmaf_rn(r, 1024.0f, -q);
    d[3] = q;
    d[4] = __fsub_rn(__fmaf_rn(r, 1024.0f, C), C);
}

// ---- the same on pairs of values with the packed FP32 instructions
// (fma/add/mul.rn.f32x2: two results per instruction slot).  A - B is
// formed as fma(B, -1, A), exact wherever the scalar form's subtraction is.



// digits10_df of two values at once, the digits NEGATED: every step is the
// scalar form's with -q = C - (t + C) computed as fma(t + C, -1, C) (exact),
// so nd0[q] = -d0[q] bit for bit.  Negated digits of both operands of a
// product leave the tensor-core sums unchanged.
__device__ __forceinline__ void digits10_df2_neg(float2 hi, float2 lo, float2 m, float2 m20, float (&nd0)[kS10],
                                                 float (&nd1)[kS10]) {
    const float2 C = f2(12582912.0f), M1 = f2(-1.0f), K = f2(1024.0f);
    float2 a = __ffma2_rn(hi, m, C);
    float2 nq = __ffma2_rn(a, M1, C);
    float2 r = __ffma2_rn(hi, m, nq);
    nd0[0] = nq.x, nd1[0] = nq.y;
    a = __ffma2_rn(r, K, C);
    nq = __ffma2_rn(a, M1, C);
    r = __ffma2_rn(r, K, nq);
    nd0[1] = nq.x, nd1[1] = nq.y;
    a = __ffma2_rn(r, K, C);
    nq = __ffma2_rn(a, M1, C);
    r = __ffma2_rn(r, K, nq);
    const float2 S = __ffma2_rn(lo, m20, r);
    const float2 nli = __ffma2_rn(__fadd2_rn(S, C), M1, C);
    const float2 nd2 = __fadd2_rn(nq, nli);
    nd0[2] = nd2.x, nd1[2] = nd2.y;
    r = __fadd2_rn(S, nli);
    a = __ffma2_rn(r, K, C);
    nq = __ffma2_rn(a, M1, C);
    r = __ffma2_rn(r, K, nq);
    nd0[3] = nq.x, nd1[3] = nq.y;
    nq = __ffma2_rn(__ffma2_rn(r, K, C), M1, C);
    nd0[4] = nq.x, nd1[4] = nq.y;
}

// combine5_k8 of the outputs e and e + 1 (bit for bit the scalar form)
__device__ __forceinline__ void combine5_k8x2(const float (&x)[kS10][4], int e, df &v0, df &v1) {
    auto P = [&](int L) { return make_float2(x[L][e], x[L][e + 1]); };
    const float2 M1 = f2(-1.0f);
    const float2 s1 = __ffma2_rn(P(1), f2(0x1p-10f), P(0));
    const float2 e1 = __ffma2_rn(P(1), f2(0x1p-10f), __ffma2_rn(s1, M1, P(0)));
    const float2 s2 = __ffma2_rn(P(2), f2(0x1p-20f), s1);
    const float2 e2 = __ffma2_rn(P(2), f2(0x1p-20f), __ffma2_rn(s2, M1, s1));
    const float2 r = __ffma2_rn(P(3), f2(0x1p-30f), __ffma2_rn(P(4), f2(0x1p-40f), e1));
    const float2 lo = __fadd2_rn(r, e2);
    v0 = df{s2.x, lo.x};
    v1 = df{s2.y, lo.y};
}

// split_g of two values (x.x with hw0, K0, mw0; x.y with hw1, K1, mw1)
__device__ __forceinline__ df2 split_g2(double2 x, unsigned hw0, unsigned hw1, unsigned K0, unsigned K1, unsigned mw0,
                                        unsigned mw1) {
    const unsigned h0 = (unsigned)__double2hiint(x.x), l0 = (unsigned)__double2loint(x.x);
    const unsigned h1 = (unsigned)__double2hiint(x.y), l1 = (unsigned)__double2loint(x.y);
    const float hi0 = hw0 >= mw0 ? __uint_as_float((__funnelshift_l(l0, h0, 3) - K0) | (h0 & 0x80000000u)) : 0.0f;
    const float hi1 = hw1 >= mw1 ? __uint_as_float((__funnelshift_l(l1, h1, 3) - K1) | (h1 & 0x80000000u)) : 0.0f;
    const float2 r = __fadd2_rn(make_float2(__uint_as_float(0x4B000000u | ((l0 >> 6) & 0x7fffffu)),
                                            __uint_as_float(0x4B000000u | ((l1 >> 6) & 0x7fffffu))),
                                f2(-8388608.0f));
    const float2 sc = __fmul2_rn(make_float2(__uint_as_float(__float_as_uint(hi0) & 0xff800000u),
                                             __uint_as_float(__float_as_uint(hi1) & 0xff800000u)),
                                 f2(0x1p-46f));   // signed, as in split_g
    return {make_float2(hi0, hi1), __fmul2_rn(r, sc)};
}

// combine5 of the outputs e and e + 1 (bit for bit the scalar form)
__device__ __forceinline__ void combine5x2(const float (&x)[kS10][4], int e, df &v0, df &v1) {
    auto P = [&](int L) { return make_float2(x[L][e], x[L][e + 1]); };
    const float2 s1 = __ffma2_rn(P(1), f2(0x1p-10f), P(0));
    const float2 e1 = __ffma2_rn(P(1), f2(0x1p-10f), sub2(P(0), s1));
    const df2 s2 = two_sum2(s1, __fmul2_rn(P(2), f2(0x1p-20f)));
    const float2 r = __ffma2_rn(P(3), f2(0x1p-30f), __ffma2_rn(P(4), f2(0x1p-40f), e1));
    const float2 lo = __fadd2_rn(r, s2.lo);
    v0 = df{s2.hi.x, lo.x};
    v1 = df{s2.hi.y, lo.y};
}

// V = x0 + x1 2^-10 + x2 2^-20 + x3 2^-30 + x4 2^-40 (x_L the level sums,
// x0..x2 exact, |x_L| < 2^25) as an unevaluated sum hi + lo.  The first
// addition is error-free with the fast two-sum (the larger magnitude comes
// first, or the sum fits 24 bits since |x0| < 2^13 then); the second uses
// the full two-sum; the rest err by < 2^-47 of |V|'s bound.
__device__ __forceinline__ df combine5(const float (&x)[kS10][4], int e) {
    const float s1 = __fmaf_rn(x[1][e], 0x1p-10f, x[0][e]);
    const float e1 = __fmaf_rn(x[1][e], 0x1p-10f, -__fsub_rn(s1, x[0][e]));
    const float b = __fmul_rn(x[2][e], 0x1p-20f);
    const df s2 = dfx::two_sum(s1, b);
    const float r = __fmaf_rn(x[3][e], 0x1p-30f, __fmaf_rn(x[4][e], 0x1p-40f, e1));
    return {s2.hi, __fadd_rn(r, s2.lo)};
}

// combine5 for K = 8 terms per product: the level sums then stay below 2^23
// (levels 0..2) and both leading additions are error-free with the fast
// two-sum (when |s1| < |x2| 2^-20 < 2^3, the sum needs at most 24 bits).
__device__ __forceinline__ df combine5_k8(const float (&x)[kS10][4], int e) {
    const float s1 = __fmaf_rn(x[1][e], 0x1p-10f, x[0][e]);
    const float e1 = __fmaf_rn(x[1][e], 0x1p-10f, -__fsub_rn(s1, x[0][e]));
    const float s2 = __fmaf_rn(x[2][e], 0x1p-20f, s1);
    const float e2 = __fmaf_rn(x[2][e], 0x1p-20f, -__fsub_rn(s2, s1));
    const float r = __fmaf_rn(x[3][e], 0x1p-30f, __fmaf_rn(x[4][e], 0x1p-40f, e1));
    return {s2, __fadd_rn(r, e2)};
}

// x 2^-sh as hi + lo by bit operations: hi = the top 24 bits of x's
// significand, lo = the next 23.  K = (896 + sh) << 23 turns the double's
// exponent field (its low 9 bits, shifted into place with the significand)
// into the float's.  hw = habs(x); entries whose biased exponent is below
// max(897 + sh, 1) (min_word = that << 20: zeros, subnormals, and values below
// 2^-126 of the scale) become zero.  lo = r23 2^-46 2^(ef - 127), formed as a
// product so that small exponents underflow gracefully.
__device__ __forceinline__ df split_g(double x, unsigned hw, unsigned K, unsigned min_word) {
    const unsigned h32 = (unsigned)__double2hiint(x), l32 = (unsigned)__double2loint(x);
    const unsigned f = __funnelshift_l(l32, h32, 3);
    const float hi = hw >= min_word ? __uint_as_float((f - K) | (h32 & 0x80000000u)) : 0.0f;
    const float r = __fsub_rn(__uint_as_float(0x4B000000u | ((l32 >> 6) & 0x7fffffu)), 8388608.0f);
    // 2^(ef - 127 - 46) with hi's sign (so lo takes x's sign), 0 with hi
    const float sc = __fmul_rn(__uint_as_float(__float_as_uint(hi) & 0xff800000u), 0x1p-46f);
    return {hi, __fmul_rn(r, sc)};
}

// y = sum_b Gh[b] V[b] (double-float products, Dot2-style accumulation)
__device__ __forceinline__ acc2 dot3(df g0, df g1, df g2, df v0, df v1, df v2) {
    const float m = __fmul_rn(g0.hi, v0.hi);
    float r = __fmaf_rn(g0.hi, v0.hi, -m);
    r = __fmaf_rn(g0.hi, v0.lo, r);
    r = __fmaf_rn(g0.lo, v0.hi, r);
    acc2 a{m, r};
    dfx::dot2_step(a, g1, v1);
    dfx::dot2_step(a, g2, v2);
    return a;
}

// x * 2^s for a double x, exact unless the result leaves the double range
__device__ __forceinline__ double scale2(double x, int s) {
    const int s1 = max(min(s / 2, 1023), -1022), s2 = max(min(s - s1, 1023), -1022);
    return x * __longlong_as_double((long long)(s1 + 1023) << 52) * __longlong_as_double((long long)(s2 + 1023) << 52);
}

}  // namespace oz
}  // namespace semax
