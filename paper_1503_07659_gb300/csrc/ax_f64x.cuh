// FP64-accurate Ax with the six contractions in double-float arithmetic.
//
// GB300 issues FP32 62.5 times faster than FP64 (2 DFMA/clk/SM), so the FP64
// form of Ax is bound by the FP64 pipe at 1.73 flop/B.  This kernel keeps
// FP64 inputs, outputs and geometric-factor multiply, but runs the
// contractions on the FP32 pipe with each value held as an unevaluated sum
// hi + lo of two floats (double-float, ~47 significant bits):
//   * per element, u is scaled by a power of two so that its largest entry
//     lies in [1, 2) (exact), and split hi + lo by integer bit operations
//     (hi = the top 24 significant bits, lo = the next 23);
//   * products use the exact FMA residual (p = a*b, fma(a, b, -p)) and sums
//     the error-free two-sum, so each operation errs by ~2^-46 of its
//     operands' magnitude;
//   * the gradient (even/odd lines, as MAP_EO) is converted to FP64 for the
//     G multiply, the result is scaled per element by a power of two again,
//     split, and the transposed contractions run in double-float;
//   * the final sum is converted to FP64 and the two scales are undone.
// The error against the FP64 definition stays near 1e-14 of ||w||_inf,
// inside the 1e-12 that FP64 Ax is held to.  Intended for even n with a
// centro-antisymmetric D (the GLL derivative); anything else takes the FP64
// tile.  The published double-word algorithms (Dekker 1971; Joldes, Muller
// & Popescu, ACM TOMS 2017) are the basis of the arithmetic.
#pragma once

#include "ax_tile.cuh"

namespace semax {
namespace dfx {

struct __align__(8) df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df add(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(__fadd_rn(a.lo, b.lo), s.lo));
}

__device__ __forceinline__ df sub(df a, df b) { return add(a, df{-b.hi, -b.lo}); }

// acc + p * x
__device__ __forceinline__ df fma_df(df p, df x, df acc) {
    const float m = __fmul_rn(p.hi, x.hi);
    float r = __fmaf_rn(p.hi, x.hi, -m);
    r = __fmaf_rn(p.hi, x.lo, r);
    r = __fmaf_rn(p.lo, x.hi, r);
    const df s = two_sum(acc.hi, m);
    return fast_two_sum(s.hi, __fadd_rn(__fadd_rn(acc.lo, r), s.lo));
}

// Dot-product accumulator in the manner of Ogita, Rump & Oishi's Dot2: s
// carries the running float sum, c the sum of every rounding error (exact
// product residuals, cross terms, two-sum errors); s + c is the result.
struct acc2 {
    float s, c;
};

// a += p * x  (p, x double-float)
__device__ __forceinline__ void dot2_step(acc2 &a, df p, df x) {
    const float m = __fmul_rn(p.hi, x.hi);
    float r = __fmaf_rn(p.hi, x.hi, -m);
    r = __fmaf_rn(p.hi, x.lo, r);
    r = __fmaf_rn(p.lo, x.hi, r);
    const df t = two_sum(a.s, m);
    a.s = t.hi;
    a.c = __fadd_rn(a.c, __fadd_rn(r, t.lo));
}

// (a.s + a.c) +/- (b.s + b.c) as a normalised double-float
__device__ __forceinline__ df acc_add(acc2 a, acc2 b) {
    const df t = two_sum(a.s, b.s);
    return fast_two_sum(t.hi, __fadd_rn(__fadd_rn(a.c, b.c), t.lo));
}
__device__ __forceinline__ df acc_sub(acc2 a, acc2 b) { return acc_add(a, acc2{-b.s, -b.c}); }

// ---- two lanes at once with the packed FP32 instructions (fma/add/mul.rn.f32x2:
// two results per issue slot).  Each lane takes the scalar form's steps in
// the same order, so the results are bit-identical; a - b is formed as
// fma(b, -1, a), exact like the subtraction.

__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }

// Double-float values of two nodes, lane-wise.
struct df2 {
    float2 hi, lo;
};
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }   // a - b

__device__ __forceinline__ df2 two_sum2(float2 a, float2 b) {
    const float2 s = __fadd2_rn(a, b);
    const float2 bb = sub2(s, a);
    return {s, __fadd2_rn(sub2(a, sub2(s, bb)), sub2(b, bb))};
}

// fast_two_sum lane-wise (|a| >= |b| in each lane)
__device__ __forceinline__ df2 fast_two_sum2(float2 a, float2 b) {
    const float2 s = __fadd2_rn(a, b);
    return {s, sub2(b, sub2(s, a))};
}

// add(a, b) lane-wise
__device__ __forceinline__ df2 add2(const df2 &a, const df2 &b) {
    const df2 s = two_sum2(a.hi, b.hi);
    return fast_two_sum2(s.hi, __fadd2_rn(__fadd2_rn(a.lo, b.lo), s.lo));
}

// Dot2 accumulators of two lanes
struct acc2x2 {
    float2 s, c;
};
__device__ __forceinline__ df2 pack_df2(df a, df b) { return {make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)}; }

// a * x lane-wise (the exact product of the high parts plus the cross terms)
__device__ __forceinline__ acc2x2 prod2(const df2 &a, const df2 &x) {
    const float2 m = __fmul2_rn(a.hi, x.hi);
    float2 r = __ffma2_rn(a.hi, x.hi, make_float2(-m.x, -m.y));
    r = __ffma2_rn(a.hi, x.lo, r);
    r = __ffma2_rn(a.lo, x.hi, r);
    return {m, r};
}

// a += p * x lane-wise (dot2_step)
__device__ __forceinline__ void dot2_step2(acc2x2 &a, const df2 &p, const df2 &x) {
    const acc2x2 q = prod2(p, x);
    const df2 t = two_sum2(a.s, q.s);
    a.s = t.hi;
    a.c = __fadd2_rn(a.c, __fadd2_rn(q.c, t.lo));
}

// dot3 lane-wise
__device__ __forceinline__ acc2x2 dot3_2(const df2 &g0, const df2 &g1, const df2 &g2, const df2 &v0, const df2 &v1,
                                         const df2 &v2) {
    acc2x2 a = prod2(g0, v0);
    dot2_step2(a, g1, v1);
    dot2_step2(a, g2, v2);
    return a;
}

// x * 2^-sh split into hi + lo by bit operations (no FP64 instruction).
// Values whose scaled magnitude is below the float range flush to zero.
// Inf and NaN are not representable here (they come out finite): the tile
// recognises their element by its exponent maximum (0x7ff) and writes NaN.
__device__ __forceinline__ df split_double(double x, int sh) {
    // A funnel shift puts the double's exponent (its low 9 bits) next to the
    // top 23 significand bits; subtracting (896 + sh) << 23 rebiases it to
    // the float's.  Zeros, subnormals and entries below the float range
    // (biased exponent < 897 + sh) give hi = 0, hence lo = 0 through sc.
    const unsigned h32 = (unsigned)__double2hiint(x), l32 = (unsigned)__double2loint(x);
    const unsigned sign = h32 & 0x80000000u;
    const unsigned min_word = (unsigned)(897 + sh > 1 ? 897 + sh : 1) << 20;
    const unsigned f = __funnelshift_l(l32, h32, 3);
    const float hi = (h32 & 0x7fffffffu) >= min_word ? __uint_as_float((f - ((unsigned)(896 + sh) << 23)) | sign) : 0.f;
    const float r = __fsub_rn(__uint_as_float(0x4B000000u | ((l32 >> 6) & 0x7fffffu)), 8388608.0f);   // r23
    const float sc = __fmul_rn(__uint_as_float(__float_as_uint(hi) & 0xff800000u), 0x1p-46f);   // +-2^(ef-127-46)
    return {hi, __fmul_rn(r, sc)};   // lo takes hi's sign through sc
}

// a float (normal or zero) as a double, exactly, by bit operations
__device__ __forceinline__ double f2d(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    if (e == 0) return 0.0;
    const unsigned long long d = ((unsigned long long)(b & 0x80000000u) << 32) |
                                 ((unsigned long long)(e + 896u) << 52) |
                                 ((unsigned long long)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}

__device__ __forceinline__ double to_double(df a) { return f2d(a.hi) + f2d(a.lo); }

// f * 2^sh as a double by adding sh to the exponent field; false when the
// result would leave the normal double range (the caller then multiplies).
__device__ __forceinline__ bool f2d_scaled(float f, int sh, double &out) {
    const unsigned b = __float_as_uint(f);
    const int e = (int)((b >> 23) & 0xffu);
    if (e == 0) { out = 0.0; return true; }
    const int ed = e + 896 + sh;
    if (ed < 1 || ed > 2046) return false;
    out = __longlong_as_double((long long)(((unsigned long long)(b & 0x80000000u) << 32) |
                                           ((unsigned long long)ed << 52) |
                                           ((unsigned long long)(b & 0x7fffffu) << 29)));
    return true;
}

// f * 2^SH as a double when SH is in [-896, 896], where every normal float's
// exponent plus 896 + SH stays in the double's normal range: exponent-field
// arithmetic only, csh = (896 + SH) << 20 computed once per element; the same
// bits as f2d_scaled; 0 for zero and subnormal f.
__device__ __forceinline__ double f2d_shift(float f, unsigned csh) {
    const unsigned b = __float_as_uint(f);
    const unsigned hw = (((b >> 3) & 0x0fffffffu) + csh) | (b & 0x80000000u);
    return (b & 0x7f800000u) ? __hiloint2double((int)hw, (int)(b << 29)) : 0.0;
}

__device__ __forceinline__ int biased_exponent(double x) {
    return (int)((((unsigned long long)__double_as_longlong(x)) >> 52) & 0x7ffu);
}

// y = M x by the even/odd split, the even and the odd sums as the two lanes
// of one packed Dot2 chain; each output pair is written to shared memory as
// soon as it is formed (y[l * stride]), so no output array stays live.  PQ[i * h + l] holds (P.hi, Q.hi, P.lo, Q.lo) of entry (i, l),
// one 16-byte load; lane 0 forms e = x_l + x_{n-1-l} and pe, lane 1
// o = x_l - x_{n-1-l} and qo, and the output pair (qo + pe, qo - pe) is
// formed the same way.  Bit for bit the scalar form.
template <int n>
__device__ __forceinline__ void eo_apply_st2(const df (&x)[n], const float4 *PQ, df *y, int stride) {
    constexpr int h = n / 2;
    df2 eo[h];
#pragma unroll
    for (int l = 0; l < h; ++l) {
        const df xr = x[n - 1 - l];
        eo[l] = add2(df2{f2(x[l].hi), f2(x[l].lo)}, df2{make_float2(xr.hi, -xr.hi), make_float2(xr.lo, -xr.lo)});
    }
    const unsigned base = (unsigned)__cvta_generic_to_shared(PQ);
#pragma unroll 1
    for (int i = 0; i < h; ++i) {
        acc2x2 a{f2(0.f), f2(0.f)};
#pragma unroll
        for (int l = 0; l < h; ++l) {
            df2 c;   // volatile: the coefficients are not hoisted out of the i loop
            asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                         : "=f"(c.hi.x), "=f"(c.hi.y), "=f"(c.lo.x), "=f"(c.lo.y)
                         : "r"(base + 16u * (unsigned)(i * h + l)));
            dot2_step2(a, c, eo[l]);
        }
        // lane 0: qo + pe, lane 1: qo - pe
        const df2 t = two_sum2(f2(a.s.y), make_float2(a.s.x, -a.s.x));
        const df2 r = fast_two_sum2(t.hi, __fadd2_rn(__fadd2_rn(f2(a.c.y), make_float2(a.c.x, -a.c.x)), t.lo));
        y[i * stride] = df{r.hi.x, r.lo.x};
        y[(n - 1 - i) * stride] = df{r.hi.y, r.lo.y};
    }
}

template <int n>
__device__ __forceinline__ void ld_line(const df *p, int stride, df (&x)[n]) {
    if (stride == 1) {
#pragma unroll
        for (int q = 0; q < n / 2; ++q) {
            const float4 v = reinterpret_cast<const float4 *>(p)[q];
            x[2 * q] = df{v.x, v.y};
            x[2 * q + 1] = df{v.z, v.w};
        }
    } else {
#pragma unroll
        for (int l = 0; l < n; ++l) x[l] = p[l * stride];
    }
}

// raw FP64 line -> df with shift sh
template <int n>
__device__ __forceinline__ void ld_line_split(const df *p, int stride, int sh, df (&x)[n]) {
    const double *d = reinterpret_cast<const double *>(p);
    if (stride == 1) {
#pragma unroll
        for (int q = 0; q < n / 2; ++q) {
            const double2 v = reinterpret_cast<const double2 *>(d)[q];
            x[2 * q] = split_double(v.x, sh);
            x[2 * q + 1] = split_double(v.y, sh);
        }
    } else {
#pragma unroll
        for (int l = 0; l < n; ++l) x[l] = split_double(d[l * stride], sh);
    }
}

// Per-element maximum of biased exponents: lanes of a warp that work on the
// same element combine first, then one shared atomic per group.
__device__ __forceinline__ void exp_max(int *slot_base, int e, int ex) {
    const unsigned grp = __match_any_sync(__activemask(), e);
    const int m = __reduce_max_sync(grp, ex);
    if ((__ffs(grp) - 1) == (int)(threadIdx.x & 31)) atomicMax(slot_base + e, m);
}

constexpr int kThreads = 256;

template <int n>
__host__ __device__ constexpr int elems_per_tile() { return kThreads / (n * n) > 0 ? kThreads / (n * n) : 1; }

template <int n>
__host__ __device__ constexpr size_t smem_bytes(int epb) {
    return sizeof(double) * (size_t)round_up(n * n, 2) + sizeof(df) * 4 * (n / 2) * (n / 2) +
           sizeof(int) * (size_t)round_up(2 * epb, 4) + sizeof(df) * 3 * (size_t)epb * eo_elem_pitch<double>(n);
}

// One tile of cnt (<= epb) consecutive elements; ue, Ge, we point at its
// first element; smem_raw holds smem_bytes<n>(epb) bytes.  All threads of the
// block take part (blockDim.x = kThreads).
template <int n>
__device__ __forceinline__ void f64x_tile(int cnt, int epb, const double *__restrict__ ue,
                                          const double *__restrict__ Ge, const double *__restrict__ D,
                                          double *__restrict__ we, unsigned char *smem_raw) {
    constexpr int n2 = n * n, n3 = n * n * n, h = n / 2;
    constexpr int RP = eo_row_pitch<double>(n), PP = eo_plane_pitch<double>(n), EP = eo_elem_pitch<double>(n);
    double *sD = reinterpret_cast<double *>(smem_raw);
    float4 *coef = reinterpret_cast<float4 *>(sD + round_up(n2, 2));   // [2][h * h]: (P, Q), (Pt, Qt) interleaved
    int *sexp = reinterpret_cast<int *>(coef + 2 * h * h);      // [0, epb): u, [epb, 2 epb): w
    df *su = reinterpret_cast<df *>(sexp + round_up(2 * epb, 4));
    df *sr = su + cnt * EP, *ss = sr + cnt * EP;   // the t-direction reuses su

    for (int q = threadIdx.x; q < n2; q += blockDim.x) sD[q] = D[q];
    if (threadIdx.x < 2 * epb) sexp[threadIdx.x] = 0;
    // stage u (raw FP64) in the padded layout, tracking each element's largest exponent
    for (int q = threadIdx.x; q < cnt * n3 / 2; q += blockDim.x) {
        const int f = 2 * q, e = f / n3, r = f - e * n3;
        const int k = r / n2, j = (r / n) % n, i = r % n;
        double2 v;
        asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(ue + f));
        *reinterpret_cast<double2 *>(su + e * EP + k * PP + j * RP + i) = v;
    }
    __syncthreads();
    int ok = 1;
    for (int q = threadIdx.x; q < n2; q += blockDim.x) {
        const int i = q / n, l = q - (q / n) * n;
        if (sD[q] != -sD[(n - 1 - i) * n + (n - 1 - l)] || biased_exponent(sD[q]) == 0x7ff) ok = 0;
    }
    if (!__syncthreads_and(ok)) {
        // D is not centro-antisymmetric: the FP64 node phases on a dense copy
        double *du = reinterpret_cast<double *>(su);   // 4 dense blocks fit in 3 padded ones
        double *dr = du + cnt * n3, *ds = dr + cnt * n3, *dt = ds + cnt * n3;
        copy_to_smem(du, ue, cnt * n3);
        __syncthreads();
        tile_node_phases<double, n>(cnt, Ge, we, nullptr, Helm<double>{nullptr, 1.0, 0.0}, sD, du, dr, ds, dt);
        return;
    }
    for (int q = threadIdx.x; q < h * h; q += blockDim.x) {
        const int i = q / h, l = q - (q / h) * h;
        const double a = sD[i * n + l], b = sD[i * n + (n - 1 - l)];
        const double at = sD[l * n + i], bt = sD[(n - 1 - l) * n + i];
        const df P = split_double(0.5 * (a + b), 0), Q = split_double(0.5 * (a - b), 0);
        const df Pt = split_double(0.5 * (at + bt), 0), Qt = split_double(0.5 * (at - bt), 0);
        coef[q] = make_float4(P.hi, Q.hi, P.lo, Q.lo);
        coef[h * h + q] = make_float4(Pt.hi, Qt.hi, Pt.lo, Qt.lo);
    }
    for (int f = threadIdx.x; f < cnt * n3; f += blockDim.x) {
        const int e = f / n3, r = f - e * n3;
        const int k = r / n2, j = (r / n) % n, i = r % n;
        exp_max(sexp, e, biased_exponent(reinterpret_cast<const double *>(su)[e * EP + k * PP + j * RP + i]));
    }
    __syncthreads();
    // u -> double-float, scaled so that each element's largest entry is in [1, 2)
    for (int f = threadIdx.x; f < cnt * n3; f += blockDim.x) {
        const int e = f / n3, r = f - e * n3;
        const int k = r / n2, j = (r / n) % n, i = r % n;
        const int s = e * EP + k * PP + j * RP + i;
        su[s] = split_double(reinterpret_cast<const double *>(su)[s], sexp[e] - 1023);
    }
    __syncthreads();

    const float4 *PQ = coef, *PQt = coef + h * h;
    const int lines = cnt * n2;
    // gradient, r- and s-lines
#pragma unroll 1
    for (int dir = 0; dir < 2; ++dir) {
        df *out = dir == 0 ? sr : ss;
        for (int t = threadIdx.x; t < lines; t += blockDim.x) {
            const int e = t / n2, ab = t - e * n2, a = ab / n, b = ab - a * n;
            const int off = e * EP + a * PP + (dir == 0 ? b * RP : b);
            const int stride = dir == 0 ? 1 : RP;
            df x[n];
            ld_line<n>(su + off, stride, x);
            eo_apply_st2<n>(x, PQ, out + off, stride);
        }
    }
    __syncthreads();
    // columns: t-line of u into the column's own slots of su, then the FP64
    // geometric factor per node; raw FP64 results wr -> sr, ws -> ss, wt -> su
    for (int t = threadIdx.x; t < lines; t += blockDim.x) {
        const int e = t / n2, ji = t - e * n2, j = ji / n, i = ji - j * n;
        const int off = e * EP + j * RP + i;
        df x[n];
        ld_line<n>(su + off, PP, x);
        eo_apply_st2<n>(x, PQ, su + off, PP);
        const double *Gq = Ge + (size_t)e * 6 * n3 + ji;
        int mx = 0;
#pragma unroll 2
        for (int k = 0; k < n; ++k) {
            const int s = off + k * PP;
            double wr, ws, wt;
            geo_multiply(Gq + k * n2, n3, to_double(sr[s]), to_double(ss[s]), to_double(su[s]), wr, ws, wt);
            reinterpret_cast<double *>(sr)[s] = wr;
            reinterpret_cast<double *>(ss)[s] = ws;
            reinterpret_cast<double *>(su)[s] = wt;
            mx = max(mx, (int)(max(__double2hiint(wr) & 0x7fffffff,
                                   max(__double2hiint(ws) & 0x7fffffff, __double2hiint(wt) & 0x7fffffff)) >> 20));
        }
        exp_max(sexp + epb, e, mx);
    }
    __syncthreads();
    // transposed contractions, all three directions, split on load, in place
#pragma unroll 1
    for (int dir = 0; dir < 3; ++dir) {
        df *io = dir == 0 ? sr : (dir == 1 ? ss : su);
        for (int t = threadIdx.x; t < lines; t += blockDim.x) {
            const int e = t / n2, ab = t - e * n2, a = ab / n, b = ab - a * n;
            const int off = e * EP + (dir == 0 ? a * PP + b * RP : (dir == 1 ? a * PP + b : a * RP + b));
            const int stride = dir == 0 ? 1 : (dir == 1 ? RP : PP);
            df x[n];
            ld_line_split<n>(io + off, stride, sexp[epb + e] - 1023, x);
            eo_apply_st2<n>(x, PQt, io + off, stride);
        }
    }
    __syncthreads();
    // sum, back to FP64, undo both scales, one coalesced store
    for (int f = threadIdx.x; f < cnt * n3; f += blockDim.x) {
        const int e = f / n3, r = f - e * n3;
        const int k = r / n2, j = (r / n) % n, i = r % n;
        const int s = e * EP + k * PP + j * RP + i;
        if (sexp[e] == 0x7ff || sexp[epb + e] == 0x7ff) {   // Inf or NaN in u or in G: the element is NaN
            we[f] = __longlong_as_double(0x7ff8000000000000ll);
            continue;
        }
        const df acc = add(add(sr[s], ss[s]), su[s]);
        const int su_e = sexp[e] > 0 ? sexp[e] : 1, sw_e = sexp[epb + e] > 0 ? sexp[epb + e] : 1;
        const int SH = su_e + sw_e - 2046;
        double dh, dl;
        if (SH >= -896 && SH <= 896) {
            const unsigned cSH = (unsigned)(896 + SH) << 20;
            we[f] = f2d_shift(acc.hi, cSH) + f2d_shift(acc.lo, cSH);
        } else if (f2d_scaled(acc.hi, SH, dh) && f2d_scaled(acc.lo, SH, dl)) {
            we[f] = dh + dl;                       // exact scaling, one FP64 add
        } else {
            const double su_scale = __longlong_as_double((long long)su_e << 52);
            const double sw_scale = __longlong_as_double((long long)sw_e << 52);
            we[f] = (to_double(acc) * su_scale) * sw_scale;
        }
    }
}


template <int n>
__global__ void __launch_bounds__(kThreads, (n <= 8 ? 3 : (n == 12 ? 4 : 1)))
ax_f64x_kernel(int64_t E, const double *__restrict__ u, const double *__restrict__ G,
               const double *__restrict__ D, double *__restrict__ w) {
    constexpr int n3 = n * n * n, epb = elems_per_tile<n>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t e0 = (int64_t)blockIdx.x * epb;
    const int cnt = (int)(E - e0 < epb ? E - e0 : epb);
    f64x_tile<n>(cnt, epb, u + e0 * n3, G + e0 * 6 * n3, D, w + e0 * n3, smem_raw);
}

}  // namespace dfx
}  // namespace semax
