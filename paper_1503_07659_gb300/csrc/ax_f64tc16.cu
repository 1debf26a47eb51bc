// FP64-accurate Ax for order N = 15 (n = 16) on FP16 tensor cores by exact
// digit slicing (the Ozaki scheme, as in the order-7 form): each operand as
// five balanced base-1024 digits (integers of magnitude <= 528, exact in
// FP16) against a power-of-two scale, the 15 digit pairs of levels 0..4
// summed in FP32 accumulators (one pair per m16n8k16 product, K = 16 terms;
// levels 0..2 stay below 2^24 and are exact, levels 3 and 4 weigh 2^-30 and
// 2^-40), the level sums combined in double-float.  Against six base-256
// digits in BF16 (21 pairs) this takes 29 % fewer tensor-core products at
// the same digit-extraction cost; at n = 16 the products are a third of the
// kernel's time.
//
// One CTA of 16 warps per element, persistent over elements.  Warp w owns
// plane k = w for every pointwise step, in the accumulator layout of an
// m16n8 tile pair (rows j, columns i = 0..7 and 8..15).  With n = 16 = M,
// the r- and s-contractions of a plane both land in that layout:
//   r: C[j][i] = sum_l U_k[j][l] D^T[l][i]   (A: u digits, B: D digits)
//   s: C[j][i] = sum_l D[j][l] U_k[l][i]     (A: D digits, B: u digits)
// so the gradient's r and s parts never leave their warp; the t-part is
// formed per row j (warp w owns j = w there: C[k][i] = sum_l D[k][l] U_j[l][i])
// and crosses through a shared double-float buffer.  The transposed side
// mirrors this: the digits of y_r = (G grad)_r pack from the accumulator
// layout straight into A fragments, those of y_s are transposed into B
// fragments by movmatrix, and only y_t's digits go through shared memory.
// y_r, y_s and y_t take separate per-element scales.
//
// G is staged in two halves by TMA bulk copies: (rr, rs, rt) while the
// gradient runs (y_r complete, the r-parts of y_s and y_t formed), then
// (ss, st, tt) while the transposed r-contraction runs.  The next element's
// u is loaded into registers during the last phases.
#include "ax_f64tc.cuh"

namespace semax {
namespace oz16 {

using namespace oz;

constexpr int kThreads = 512;
constexpr int kN3 = 4096;
constexpr int kPlaneB = 512;                 // one 16 x 16 BF16 plane
constexpr int kDigitB = 16 * kPlaneB;        // one digit of a 16^3 operand
constexpr int kUD = kS10 * kDigitB;            // digits of u, later of y_t (40 KB)
constexpr int kDD = kS10 * kPlaneB;            // digits of D (2.5 KB)
constexpr int kTB = kN3 * 8;                 // double-float per node: t-direction (32 KB)
constexpr int kSB = kN3 * 8;                 // double-float per node: the s-gradient, parked (32 KB)
constexpr int kGS = 3 * kN3 * 8;             // half of an element's G (96 KB)
constexpr int kRed = 64 * 4;                 // reduction slots
constexpr int kTail = 16;                    // prepared form: the element's largest G exponent, before its halves
constexpr int kPreElem = kTail + 2 * kGS;    // prepared form: one element (192 KB + 16 B)
template <bool PRE>
constexpr size_t smem_bytes() { return kUD + kDD + kTB + kSB + kTail + kGS + kRed + 16; }   // + two mbarriers

// Byte offset of (row r, 16-byte chunk c) of the 16 x 16 BF16 plane p: the
// 32 chunks of a plane are permuted by p and by bit 2 of r, so that ldmatrix
// over 8 rows of a plane (r = 0..7 or 8..15) and over 8 planes of a row both
// touch 8 distinct bank groups.
__device__ __forceinline__ int pch(int p, int r, int c) {
    return p * kPlaneB + ((((2 * r + c) ^ ((p & 7) ^ ((r >> 2) & 1)))) << 4);
}

// Node-pair slot (16 bytes: two double-floats) of (k, j, i = 2 ip) in the
// t-direction buffer; bit 2 flipped by (j ^ k) & 1, so that the row owners'
// writes and the plane owners' reads are both conflict-free.
__device__ __forceinline__ int tslot(int k, int j, int ip) { return (k * 128 + j * 8 + ip) ^ (((j ^ k) & 1) << 2); }

// acc[L] += A_a B_b over the 15 digit pairs a + b = L <= 4, issued round-robin
// over the levels so that consecutive products update different accumulators
__device__ __forceinline__ void pairs15(float (&acc)[kS10][4], const uint32_t (&A)[kS10][4], const uint32_t (&B)[kS10][2]) {
#pragma unroll
    for (int L = 0; L < kS10; ++L) acc[L][0] = acc[L][1] = acc[L][2] = acc[L][3] = 0.0f;
#pragma unroll
    for (int a = 0; a < kS10; ++a)
#pragma unroll
        for (int L = a; L < kS10; ++L)
            mma::f16_16816(acc[L], A[a][0], A[a][1], A[a][2], A[a][3], B[L - a][0], B[L - a][1]);
}

// (hi + lo) 2^SH as a double with integer operations only, for SH in
// [-896, 896] with csh = (896 + SH) << 20 as in f2d_shift: the pair is
// renormalised by a two-sum (|lo| <= ulp(hi) / 2), so the double of hi has
// its low 29 significand bits clear and lo, counted in units of that
// double's ulp and rounded to the nearest integer (ties to even), is an
// integer k with |k| <= 2^28; adding k to the bit pattern adds k ulps to the
// magnitude.  Where hi is a power of two and lo pulls its magnitude down, the
// result lies in the binade below, whose ulp is half as large, and k is
// counted in those units.  The result is the correctly rounded (hi + lo)
// 2^SH, bit for bit the FP64 add of the two f2d_shift values.  The prepared
// instance's output phase converts one node of each pair this way and the
// other with that add, so that the ALU and the FP64 pipe share the work.
__device__ __forceinline__ double df_to_double_int(float hi, float lo, unsigned csh) {
    const df n = dfx::two_sum(hi, lo);
    const unsigned bs = __float_as_uint(n.hi), bl = __float_as_uint(n.lo);
    const int es = (int)((bs >> 23) & 0xffu), el = (int)((bl >> 23) & 0xffu);
    if (es == 0) return dfx::f2d_shift(n.lo, csh);
    const unsigned hw = (((bs >> 3) & 0x0fffffffu) + csh) | (bs & 0x80000000u);
    int k = 0;
    if (el != 0) {
        const unsigned m = (bl & 0x7fffffu) | 0x800000u;
        const bool opp = ((bs ^ bl) & 0x80000000u) != 0;
        const int sh = el - es + 29 + ((opp && !(bs & 0x7fffffu)) ? 1 : 0);   // <= 6
        unsigned mag = 0u;
        if (sh >= 0) {
            mag = m << sh;
        } else if (sh > -25) {
            const int r = -sh;
            const unsigned q = m >> r, rem = m & ((1u << r) - 1u), half = 1u << (r - 1);
            mag = q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u);
        }
        k = opp ? -(int)mag : (int)mag;
    }
    const unsigned long long bits = ((unsigned long long)hw << 32 | (unsigned long long)(bs << 29)) +
                                    (unsigned long long)(long long)k;
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ int max16(const int *p) {
    const int4 a = reinterpret_cast<const int4 *>(p)[0], b = reinterpret_cast<const int4 *>(p)[1];
    const int4 c = reinterpret_cast<const int4 *>(p)[2], d = reinterpret_cast<const int4 *>(p)[3];
    return max(max(max(max(a.x, a.y), max(a.z, a.w)), max(max(b.x, b.y), max(b.z, b.w))),
               max(max(max(c.x, c.y), max(c.z, c.w)), max(max(d.x, d.y), max(d.z, d.w))));
}

// PRE = false: G is FP64 [E][6][4096]; PRE = true: G points at the prepared
// form, per element a 16-byte tail whose first int is the element's largest
// biased exponent of G, then the halves (rr, rs, rt) and (ss, st, tt), each
// 3 x 4096 (hi, lo) float pairs split against that one scale (so the halves
// need no alignment; FP64 G is split per node and half, below).
// The Helmholtz form's mass term: w = h1 (A u) + h2 B u, B [E][4096].
struct HelmArgs16 {
    const double *B;
    double h1, h2;
};

// HELM: w = h1 (A u) + h2 B u, the mass term added in FP64 to the FP64
// output of A u; u and B of the element are read again in the output phase
// (u's digits are gone by then), 16 B per node more than A u alone.
template <bool PRE, bool HELM = false>
__global__ void __launch_bounds__(kThreads, 1)
ax_f64tc16_kernel(int64_t E, const double *__restrict__ u, const double *__restrict__ G,
                  const double *__restrict__ D, double *__restrict__ w, int *__restrict__ status, int polls,
                  HelmArgs16 hm) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *ud = smem;
    unsigned char *dd = ud + kUD;
    float4 *tb = reinterpret_cast<float4 *>(dd + kDD);                 // [2048] node pairs
    float2 *sb = reinterpret_cast<float2 *>(dd + kDD + kTB);           // [8][512] per-thread slots
    const int *tail = reinterpret_cast<const int *>(dd + kDD + kTB + kSB);            // prepared: the element's exponent
    const double2 *gs = reinterpret_cast<const double2 *>(dd + kDD + kTB + kSB + kTail);   // [3][2048]
    const float4 *gsp = reinterpret_cast<const float4 *>(gs);                       // prepared: [3][2048] pairs x 2
    int *sred = reinterpret_cast<int *>(dd + kDD + kTB + kSB + kTail + kGS);         // 4 x 16 slots
    const uint32_t ud_s = smem_u32(ud), dd_s = smem_u32(dd), gs_s = smem_u32(gs);
    const uint32_t barA = smem_u32(sred + 64), barB = barA + 8;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const int mi = lane >> 3, rr = lane & 7;
    const int k = warp;   // the plane this warp owns in the pointwise phases (and the row j in the t-phases)

    if (tid == 0) {
        mbar_init(barA, 1);
        mbar_init(barB, 1);
    }
    __syncthreads();
    // half h (0: rr, rs, rt; 1: ss, st, tt) of element ep into the staging buffer
    auto stage = [&](uint32_t bar, int64_t ep, int h) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (PRE) {   // the first half with the element's tail in front of it
            const unsigned char *src = reinterpret_cast<const unsigned char *>(G) + ep * (int64_t)kPreElem;
            if (h == 0) {
                mbar_expect_tx(bar, kTail + kGS);
                bulk_g2s(gs_s - kTail, src, kTail + kGS, bar);
            } else {
                mbar_expect_tx(bar, kGS);
                bulk_g2s(gs_s, src + kTail + kGS, kGS, bar);
            }
        } else {
            mbar_expect_tx(bar, kGS);
            bulk_g2s(gs_s, G + (2 * ep + h) * 3 * kN3, kGS, bar);
        }
    };
    if (tid == 0) stage(barA, blockIdx.x, 0);

    // ---- D digits, once per CTA: [p][16 x 16] in the plane layout
    int eD = 1;
    if (tid < 256) eD = max((int)(habs(D[tid]) >> 20), 1);
    eD = __reduce_max_sync(0xffffffffu, eD);
    if (lane == 0) sred[warp] = eD;
    __syncthreads();
    eD = max16(sred);
    if (tid < 256) {
        float d[kS10];
        digits10_fp64(D[tid], eD, d);
        const int a = tid >> 4, b = tid & 15;
#pragma unroll
        for (int p = 0; p < kS10; ++p)
            *reinterpret_cast<unsigned short *>(dd + p * kPlaneB + pch(0, a, b >> 3) + 2 * (b & 7)) =
                (unsigned short)(pack_f16(-d[p], 0.0f) & 0xffffu);   // negated, like u's and y's
    }
    __syncthreads();

    // lane addresses of the two ldmatrix x4 arrangements (row, 16-byte chunk)
    const int r1 = rr + 8 * (mi & 1), c1 = mi >> 1;   // a0..a3 = (0-7,0) (8-15,0) (0-7,1) (8-15,1)
    const int r2 = rr + 8 * (mi >> 1), c2 = mi & 1;   // (0-7,0) (0-7,1) (8-15,0) (8-15,1)
    const int rx = rr + 8 * (mi & 1);                 // x2: rows 0-7, 8-15 of one chunk (lanes 0-15)

    // thread's nodes: q = 4 nt + e -> (j, i) = (g + 8 (e >> 1), 8 nt + 2 t + (e & 1)) in plane k
    double2 uv[2][2];   // [nt][row half]
    auto load_u = [&](int64_t ep) {
        const double *ue = u + ep * kN3 + k * 256;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                double2 v;
                asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];"
                             : "=d"(v.x), "=d"(v.y) : "l"(ue + (g + 8 * h) * 16 + 8 * nt + 2 * t));
                uv[nt][h] = v;
            }
    };
    load_u(blockIdx.x);

    unsigned pA = 0, pB = 0;
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x, pA ^= 1u, pB ^= 1u) {
        double *we = w + e * kN3;

        // ---- A: u -> digits
        const bool toA = !mbar_wait(barA, pA, polls);   // G's first half (staged during the previous element)
        int ex = 1;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) ex = max(ex, (int)(max(habs(uv[nt][h].x), habs(uv[nt][h].y)) >> 20));
        ex = __reduce_max_sync(0xffffffffu, ex);
        if (lane == 0) sred[warp] = ex;
        if (__syncthreads_or(toA)) {   // the staged data never arrived: report, mark NaN, leave
            if (tid == 0) report_timeout(status);
            for (int64_t r = e; r < E; r += gridDim.x)
                for (int q = tid; q < kN3; q += kThreads) w[r * kN3 + q] = __longlong_as_double(0x7ff8000000000000ll);
            mbar_wait(barA, pA);
            return;
        }
        const int eU = max16(sred);
        const int egE = PRE ? tail[0] : 0;   // prepared: the element's largest biased G exponent
        {
            const unsigned Ku = (unsigned)(eU - 127) << 23, mw = (unsigned)max(eU - 126, 1) << 20;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float d0[kS10], d1[kS10];
                    const df a0 = split_g(uv[nt][h].x, habs(uv[nt][h].x), Ku, mw);
                    const df a1 = split_g(uv[nt][h].y, habs(uv[nt][h].y), Ku, mw);
                    const df n0 = dfx::fast_two_sum(a0.hi, a0.lo), n1 = dfx::fast_two_sum(a1.hi, a1.lo);
                    digits10_df2_neg(make_float2(n0.hi, n1.hi), make_float2(n0.lo, n1.lo), f2(256.0f), f2(268435456.0f),
                                     d0, d1);
                    unsigned char *p = ud + pch(k, g + 8 * h, nt) + 4 * t;
#pragma unroll
                    for (int q = 0; q < kS10; ++q) *reinterpret_cast<uint32_t *>(p + q * kDigitB) = pack_f16(d0[q], d1[q]);
                }
        }
        __syncthreads();

        // ---- B: gradient on tensor cores
        df vr[8];   // r-gradient of the thread's nodes
        {
            uint32_t fa[kS10][4];   // D as A (rows j or k, K = l)
#pragma unroll
            for (int p = 0; p < kS10; ++p)
                mma::ldsm_x4(dd_s + p * kPlaneB + pch(0, r1, c1), fa[p][0], fa[p][1], fa[p][2], fa[p][3]);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                // s: B = U_k (rows l, columns i), transposed load
                uint32_t bu[kS10][2];
#pragma unroll
                for (int q = 0; q < kS10; ++q) {
                    mma::ldsm_x2_t(ud_s + q * kDigitB + pch(k, rx, nt), bu[q][0], bu[q][1]);
                }
                float acc[kS10][4];
                pairs15(acc, fa, bu);
#pragma unroll
                for (int c = 0; c < 4; c += 2) {
                    df v0, v1;
                    combine5x2(acc, c, v0, v1);
                    sb[(4 * nt + c) * kThreads + tid] = make_float2(v0.hi, v0.lo);
                    sb[(4 * nt + c + 1) * kThreads + tid] = make_float2(v1.hi, v1.lo);
                }
            }
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                // t (row j = k): B = U at row j (rows = planes l, columns i)
                uint32_t bu[kS10][2];
#pragma unroll
                for (int q = 0; q < kS10; ++q) {
                    mma::ldsm_x2_t(ud_s + q * kDigitB + pch(rx, k, nt), bu[q][0], bu[q][1]);
                }
                float acc[kS10][4];
                pairs15(acc, fa, bu);
#pragma unroll
                for (int h = 0; h < 2; ++h) {   // rows kk = g + 8 h, columns i = 8 nt + 2 t, +1
                    df v0, v1;
                    combine5x2(acc, 2 * h, v0, v1);
                    tb[tslot(g + 8 * h, k, 4 * nt + t)] = make_float4(v0.hi, v0.lo, v1.hi, v1.lo);
                }
            }
        }
        {
            // r: A = U_k (rows j, K = l), B = D^T from D stored (rows i, columns l)
            uint32_t au[kS10][4];
#pragma unroll
            for (int q = 0; q < kS10; ++q)
                mma::ldsm_x4(ud_s + q * kDigitB + pch(k, r1, c1), au[q][0], au[q][1], au[q][2], au[q][3]);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                uint32_t bd[kS10][2];
#pragma unroll
                for (int p = 0; p < kS10; ++p) {
                    mma::ldsm_x2(dd_s + p * kPlaneB + pch(0, 8 * nt + rr, mi & 1), bd[p][0], bd[p][1]);
                }
                float acc[kS10][4];
                pairs15(acc, au, bd);
#pragma unroll
                for (int c = 0; c < 4; c += 2) combine5x2(acc, c, vr[4 * nt + c], vr[4 * nt + c + 1]);
            }
        }
        __syncthreads();

        // ---- C1: G's first half (rr, rs, rt): y_r, and the r-parts of y_s, y_t,
        // on the node pairs c = 0, 1 (p = 2 nt + h) lane-wise in packed FP32
        acc2x2 YR[4], YSP[4], YTP[4];
        int shA[8];
        int tmax = INT_MIN;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = g + 8 * h, nd2 = (k * 256 + j * 16 + 8 * nt + 2 * t) >> 1, p = 2 * nt + h, q0 = 2 * p;
                const float4 tv = tb[tslot(k, j, 4 * nt + t)];
                double2 gv[3];
                float4 gp[3];
                if (PRE) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) gp[a] = gsp[a * 2048 + nd2];
                } else {
#pragma unroll
                    for (int a = 0; a < 3; ++a) gv[a] = gs[a * 2048 + nd2];
                }
                const float2 s0 = sb[q0 * kThreads + tid], s1 = sb[(q0 + 1) * kThreads + tid];
                const df2 Vr = pack_df2(vr[q0], vr[q0 + 1]);
                const df2 Vs{make_float2(s0.x, s1.x), make_float2(s0.y, s1.y)};
                const df2 Vt{make_float2(tv.x, tv.z), make_float2(tv.y, tv.w)};
                df2 Gh[3];
                int eg0, eg1;
                if (PRE) {
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        Gh[a] = df2{make_float2(gp[a].x, gp[a].z), make_float2(gp[a].y, gp[a].w)};
                    eg0 = eg1 = egE;
                } else {
                    unsigned hw0[3], hw1[3], hm0 = 0, hm1 = 0;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        hw0[a] = habs(gv[a].x);
                        hw1[a] = habs(gv[a].y);
                        hm0 = max(hm0, hw0[a]);
                        hm1 = max(hm1, hw1[a]);
                    }
                    eg0 = (int)(hm0 >> 20);
                    eg1 = (int)(hm1 >> 20);
                    const int s0 = max(eg0, 1) - 1023, s1 = max(eg1, 1) - 1023;
                    const unsigned K0 = (unsigned)(896 + s0) << 23, mw0 = (unsigned)max(897 + s0, 1) << 20;
                    const unsigned K1 = (unsigned)(896 + s1) << 23, mw1 = (unsigned)max(897 + s1, 1) << 20;
#pragma unroll
                    for (int a = 0; a < 3; ++a) Gh[a] = split_g2(gv[a], hw0[a], hw1[a], K0, K1, mw0, mw1);
                }
                const int sh0 = max(eg0, 1) - 1023, sh1 = max(eg1, 1) - 1023;
                const acc2x2 y = dot3_2(Gh[0], Gh[1], Gh[2], Vr, Vs, Vt);
                const df2 yn = two_sum2(y.s, y.c);
                YR[p] = acc2x2{yn.hi, yn.lo};
                YSP[p] = prod2(Gh[1], Vr);
                YTP[p] = prod2(Gh[2], Vr);
                shA[q0] = sh0;
                shA[q0 + 1] = sh1;
                const int ev0 = (int)(__float_as_uint(fabsf(yn.hi.x)) >> 23);
                const int ev1 = (int)(__float_as_uint(fabsf(yn.hi.y)) >> 23);
                if (ev0) tmax = max(tmax, ev0 + sh0);
                if (ev1) tmax = max(tmax, ev1 + sh1);
                if (eg0 == 0x7ff || eg1 == 0x7ff) tmax = kBadExp;
            }
        tmax = __reduce_max_sync(0xffffffffu, tmax);
        if (lane == 0) sred[16 + warp] = tmax;
        __syncthreads();
        if (tid == 0) stage(barB, e, 1);   // every thread has read G's first half
        const int eRraw = max16(sred + 16);
        const int eR = eRraw == INT_MIN ? 0 : min(eRraw, kBadExp);

        // y_r digits, packed from the accumulator layout into A fragments
        uint32_t ya[kS10][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q0 = 4 * nt + 2 * h;
                float d0[kS10], d1[kS10];
                digits10_df2_neg(YR[2 * nt + h].s, YR[2 * nt + h].c,
                                 make_float2(pow2f_or_zero(shA[q0] - eR + 135), pow2f_or_zero(shA[q0 + 1] - eR + 135)),
                                 make_float2(pow2f_or_zero(shA[q0] - eR + 155), pow2f_or_zero(shA[q0 + 1] - eR + 155)), d0, d1);
#pragma unroll
                for (int d = 0; d < kS10; ++d) ya[d][2 * nt + h] = pack_f16(d0[d], d1[d]);
            }

        // ---- D_r: w_r = y_r D on tensor cores (B = D, rows l, columns i)
        df wr_[8];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            uint32_t bd[kS10][2];
#pragma unroll
            for (int p = 0; p < kS10; ++p) {
                mma::ldsm_x2_t(dd_s + p * kPlaneB + pch(0, rx, nt), bd[p][0], bd[p][1]);
            }
            float acc[kS10][4];
            pairs15(acc, ya, bd);
#pragma unroll
            for (int c = 0; c < 4; c += 2) combine5x2(acc, c, wr_[4 * nt + c], wr_[4 * nt + c + 1]);
        }

        // ---- C2: G's second half (ss, st, tt): finish y_s, y_t
        const bool toB = !mbar_wait(barB, pB, polls);
        acc2x2 YS[4], YT[4];
        int shS[8];
        int smax = INT_MIN, tmx = INT_MIN;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = g + 8 * h, nd2 = (k * 256 + j * 16 + 8 * nt + 2 * t) >> 1, p = 2 * nt + h, q0 = 2 * p;
                const float4 tv = tb[tslot(k, j, 4 * nt + t)];
                double2 gv[3];
                float4 gp[3];
                if (PRE) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) gp[a] = gsp[a * 2048 + nd2];
                } else {
#pragma unroll
                    for (int a = 0; a < 3; ++a) gv[a] = gs[a * 2048 + nd2];
                }
                const float2 s0 = sb[q0 * kThreads + tid], s1 = sb[(q0 + 1) * kThreads + tid];
                const df2 Vs{make_float2(s0.x, s1.x), make_float2(s0.y, s1.y)};
                const df2 Vt{make_float2(tv.x, tv.z), make_float2(tv.y, tv.w)};
                df2 Gh[3];
                int eg0, eg1;
                if (PRE) {
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        Gh[a] = df2{make_float2(gp[a].x, gp[a].z), make_float2(gp[a].y, gp[a].w)};
                    eg0 = eg1 = egE;
                } else {
                    unsigned hw0[3], hw1[3], hm0 = 0, hm1 = 0;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        hw0[a] = habs(gv[a].x);
                        hw1[a] = habs(gv[a].y);
                        hm0 = max(hm0, hw0[a]);
                        hm1 = max(hm1, hw1[a]);
                    }
                    eg0 = (int)(hm0 >> 20);
                    eg1 = (int)(hm1 >> 20);
                    const int s0 = max(eg0, 1) - 1023, s1 = max(eg1, 1) - 1023;
                    const unsigned K0 = (unsigned)(896 + s0) << 23, mw0 = (unsigned)max(897 + s0, 1) << 20;
                    const unsigned K1 = (unsigned)(896 + s1) << 23, mw1 = (unsigned)max(897 + s1, 1) << 20;
#pragma unroll
                    for (int a = 0; a < 3; ++a) Gh[a] = split_g2(gv[a], hw0[a], hw1[a], K0, K1, mw0, mw1);
                }
                const int sh0 = max(eg0, 1) - 1023, sh1 = max(eg1, 1) - 1023;
                // Gh: ss, st, tt.  y_s = Grs r + Gss s + Gst t,  y_t = Grt r + Gst s + Gtt t
                acc2x2 bs = prod2(Gh[0], Vs);
                dot2_step2(bs, Gh[1], Vt);
                acc2x2 bt = prod2(Gh[1], Vs);
                dot2_step2(bt, Gh[2], Vt);
                // align the two halves' sums to the larger of their scales (the
                // prepared form has one scale per element: nothing to align)
                const int sm0 = max(shA[q0], sh0), sm1 = max(shA[q0 + 1], sh1);
                df2 xs, zs, xt, zt;
                if (PRE) {
                    xs = df2{YSP[p].s, YSP[p].c}, zs = df2{bs.s, bs.c};
                    xt = df2{YTP[p].s, YTP[p].c}, zt = df2{bt.s, bt.c};
                } else {
                    const float2 fa = make_float2(pow2f_or_zero(shA[q0] - sm0), pow2f_or_zero(shA[q0 + 1] - sm1));
                    const float2 fb = make_float2(pow2f_or_zero(sh0 - sm0), pow2f_or_zero(sh1 - sm1));
                    xs = df2{__fmul2_rn(YSP[p].s, fa), __fmul2_rn(YSP[p].c, fa)}, zs = df2{__fmul2_rn(bs.s, fb), __fmul2_rn(bs.c, fb)};
                    xt = df2{__fmul2_rn(YTP[p].s, fa), __fmul2_rn(YTP[p].c, fa)}, zt = df2{__fmul2_rn(bt.s, fb), __fmul2_rn(bt.c, fb)};
                }
                const df2 ts = two_sum2(xs.hi, zs.hi), tt = two_sum2(xt.hi, zt.hi);
                const df2 sn = two_sum2(ts.hi, __fadd2_rn(__fadd2_rn(xs.lo, zs.lo), ts.lo));
                const df2 tn = two_sum2(tt.hi, __fadd2_rn(__fadd2_rn(xt.lo, zt.lo), tt.lo));
                YS[p] = acc2x2{sn.hi, sn.lo};
                YT[p] = acc2x2{tn.hi, tn.lo};
                shS[q0] = sm0;
                shS[q0 + 1] = sm1;
                const int es0 = (int)(__float_as_uint(fabsf(sn.hi.x)) >> 23), es1 = (int)(__float_as_uint(fabsf(sn.hi.y)) >> 23);
                const int et0 = (int)(__float_as_uint(fabsf(tn.hi.x)) >> 23), et1 = (int)(__float_as_uint(fabsf(tn.hi.y)) >> 23);
                if (es0) smax = max(smax, es0 + sm0);
                if (es1) smax = max(smax, es1 + sm1);
                if (et0) tmx = max(tmx, et0 + sm0);
                if (et1) tmx = max(tmx, et1 + sm1);
                if (eg0 == 0x7ff || eg1 == 0x7ff) smax = tmx = kBadExp;
            }
        smax = __reduce_max_sync(0xffffffffu, smax);
        tmx = __reduce_max_sync(0xffffffffu, tmx);
        if (lane == 0) {
            sred[32 + warp] = smax;
            sred[48 + warp] = tmx;
        }
        if (__syncthreads_or(toB)) {
            if (tid == 0) report_timeout(status);
            for (int64_t r = e; r < E; r += gridDim.x)
                for (int q = tid; q < kN3; q += kThreads) w[r * kN3 + q] = __longlong_as_double(0x7ff8000000000000ll);
            mbar_wait(barB, pB);
            return;
        }
        if (tid == 0 && e + gridDim.x < E) stage(barA, e + gridDim.x, 0);   // next element's first half
        const int eSraw = max16(sred + 32), eTraw = max16(sred + 48);
        const int eS = eSraw == INT_MIN ? 0 : min(eSraw, kBadExp), eT = eTraw == INT_MIN ? 0 : min(eTraw, kBadExp);
        const bool bad = eU == 0x7ff || eD == 0x7ff || eRraw >= kBadExp || eSraw >= kBadExp || eTraw >= kBadExp;

        // y_s digits -> B fragments (movmatrix transposes each 8 x 8 block);
        // y_t digits -> shared memory (plane k)
        uint32_t yb[kS10][4];   // [digit][b0(nt0), b1(nt0), b0(nt1), b1(nt1)]
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q0 = 4 * nt + 2 * h;
                float d0[kS10], d1[kS10];
                digits10_df2_neg(YS[2 * nt + h].s, YS[2 * nt + h].c,
                                 make_float2(pow2f_or_zero(shS[q0] - eS + 135), pow2f_or_zero(shS[q0 + 1] - eS + 135)),
                                 make_float2(pow2f_or_zero(shS[q0] - eS + 155), pow2f_or_zero(shS[q0 + 1] - eS + 155)), d0, d1);
                // block (rows j = 8h.., columns i = 8nt..) transposed: the B fragment of
                // K rows l = 8h.. (b0 for h = 0, b1 for h = 1) of n-tile nt
#pragma unroll
                for (int d = 0; d < kS10; ++d) yb[d][2 * nt + h] = mma::movm_t(pack_f16(d0[d], d1[d]));
                digits10_df2_neg(YT[2 * nt + h].s, YT[2 * nt + h].c,
                                 make_float2(pow2f_or_zero(shS[q0] - eT + 135), pow2f_or_zero(shS[q0 + 1] - eT + 135)),
                                 make_float2(pow2f_or_zero(shS[q0] - eT + 155), pow2f_or_zero(shS[q0 + 1] - eT + 155)), d0, d1);
                unsigned char *p = ud + pch(k, g + 8 * h, nt) + 4 * t;
#pragma unroll
                for (int d = 0; d < kS10; ++d) *reinterpret_cast<uint32_t *>(p + d * kDigitB) = pack_f16(d0[d], d1[d]);
            }
        __syncthreads();

        // ---- D_s, D_t: A = D^T (from D stored rows l, columns j: transposed load)
        df ws_[8];
        {
            uint32_t fat[kS10][4];
#pragma unroll
            for (int p = 0; p < kS10; ++p)
                mma::ldsm_x4_t(dd_s + p * kPlaneB + pch(0, r2, c2), fat[p][0], fat[p][1], fat[p][2], fat[p][3]);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                uint32_t bb[kS10][2];
#pragma unroll
                for (int d = 0; d < kS10; ++d) {
                    bb[d][0] = yb[d][2 * nt];
                    bb[d][1] = yb[d][2 * nt + 1];
                }
                float acc[kS10][4];
                pairs15(acc, fat, bb);
#pragma unroll
                for (int c = 0; c < 4; c += 2) combine5x2(acc, c, ws_[4 * nt + c], ws_[4 * nt + c + 1]);
            }
            if (e + gridDim.x < E) load_u(e + gridDim.x);   // next element's u, in flight through D_t and E
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                // row j = k: B = y_t digits at row j (rows = planes l, columns i)
                uint32_t bt[kS10][2];
#pragma unroll
                for (int q = 0; q < kS10; ++q) {
                    mma::ldsm_x2_t(ud_s + q * kDigitB + pch(rx, k, nt), bt[q][0], bt[q][1]);
                }
                float acc[kS10][4];
                pairs15(acc, fat, bt);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    df v0, v1;
                    combine5x2(acc, 2 * h, v0, v1);
                    tb[tslot(g + 8 * h, k, 4 * nt + t)] = make_float4(v0.hi, v0.lo, v1.hi, v1.lo);
                }
            }
        }
        __syncthreads();

        // ---- E: w = 2^SH_r V_r + 2^SH_s V_s + 2^SH_t V_t, stored
        const int base = (eU - 1022) + 2 * (eD - 1022) - 126 - 36;
        const int SHr = base + eR, SHs = base + eS, SHt = base + eT;
        const int SHm = max(SHr, max(SHs, SHt));
        const bool fastSH = SHm >= -896 && SHm <= 896;   // the same for the whole element
        const unsigned cSH = (unsigned)(896 + SHm) << 20;
        const float2 fr = f2(pow2f_or_zero(SHr - SHm)), fs = f2(pow2f_or_zero(SHs - SHm)), ft = f2(pow2f_or_zero(SHt - SHm));
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = g + 8 * h;
                const float4 tv = tb[tslot(k, j, 4 * nt + t)];
                const int q0 = 4 * nt + 2 * h;
                // the node pair lane-wise: the three parts aligned to 2^SHm, summed in double-float
                const df2 wa = pack_df2(wr_[q0], wr_[q0 + 1]), wb = pack_df2(ws_[q0], ws_[q0 + 1]);
                const df2 a{__fmul2_rn(wa.hi, fr), __fmul2_rn(wa.lo, fr)}, b{__fmul2_rn(wb.hi, fs), __fmul2_rn(wb.lo, fs)};
                const df2 cc{__fmul2_rn(make_float2(tv.x, tv.z), ft), __fmul2_rn(make_float2(tv.y, tv.w), ft)};
                const df2 s1 = two_sum2(a.hi, b.hi);
                const df2 s2 = two_sum2(s1.hi, cc.hi);
                const float2 lo = __fadd2_rn(__fadd2_rn(__fadd2_rn(a.lo, b.lo), cc.lo), __fadd2_rn(s1.lo, s2.lo));
                double o[2];
                const int64_t nd = e * 4096 + k * 256 + j * 16 + 8 * nt + 2 * t;   // this node pair
                double2 uv2 = make_double2(0.0, 0.0), bv2 = make_double2(0.0, 0.0);
                if (HELM) {
                    asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];"
                                 : "=d"(uv2.x), "=d"(uv2.y) : "l"(u + nd));
                    asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];"
                                 : "=d"(bv2.x), "=d"(bv2.y) : "l"(hm.B + nd));
                }
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const float vh = c ? s2.hi.y : s2.hi.x, vl = c ? lo.y : lo.x;
                    // bit-level conversions and scaling, one FP64 add per node; the whole CTA
                    // runs this phase at once, so the prepared instance gives the second node
                    // of each pair to the integer form (the same bits) and the ALU, and the
                    // Helmholtz instance, whose mass term needs the FP64 pipe, both nodes
                    double dh, dl;
                    if (fastSH)
                        o[c] = ((PRE && c) || HELM) ? df_to_double_int(vh, vl, cSH)
                                                    : dfx::f2d_shift(vh, cSH) + dfx::f2d_shift(vl, cSH);
                    else if (dfx::f2d_scaled(vh, SHm, dh) && dfx::f2d_scaled(vl, SHm, dl))
                        o[c] = dh + dl;
                    else
                        o[c] = scale2(dfx::f2d(vh) + dfx::f2d(vl), SHm);
                    if (HELM) {   // the Helmholtz instance leaves the FP64 pipe to the mass term
                        const double mb = hm.h2 * (c ? bv2.y : bv2.x), mu = c ? uv2.y : uv2.x;
                        o[c] = hm.h1 == 1.0 ? __fma_rn(mb, mu, o[c]) : __fma_rn(mb, mu, hm.h1 * o[c]);
                    }
                    if (bad) o[c] = __longlong_as_double(0x7ff8000000000000ll);
                }
                *reinterpret_cast<double2 *>(we + k * 256 + j * 16 + 8 * nt + 2 * t) = make_double2(o[0], o[1]);
            }
    }
    __syncthreads();
    if (tid == 0) {
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(barA) : "memory");
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(barB) : "memory");
    }
}

}  // namespace oz16

template <bool PRE, bool HELM = false>
static int launch16(int64_t E, const double *u, const double *G, const double *D, double *w, int *status,
                    cudaStream_t s, oz16::HelmArgs16 hm = oz16::HelmArgs16{nullptr, 1.0, 0.0}) {
    auto kern = oz16::ax_f64tc16_kernel<PRE, HELM>;
    constexpr size_t kSmem = oz16::smem_bytes<PRE>();
    int st = cuda_status(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
    if (st != SEMAX_OK) return st;
    const int64_t grid = std::min<int64_t>(E, (int64_t)device_sm_count());
    kern<<<(unsigned)grid, oz16::kThreads, kSmem, s>>>(E, u, G, D, w, status, first_wait_polls(), hm);
    return launch_status();
}

int launch_f64tc16(int64_t E, const double *u, const double *G, const double *D, double *w, int *status,
                   cudaStream_t s) {
    return launch16<false>(E, u, G, D, w, status, s);
}

int launch_f64tc16_prepared(int64_t E, const double *u, const void *Gp, const double *D, double *w, int *status,
                            cudaStream_t s) {
    return launch16<true>(E, u, reinterpret_cast<const double *>(Gp), D, w, status, s);
}

int launch_f64tc16_helmholtz(int64_t E, const double *u, const double *G, const double *B, const double *D,
                             double h1, double h2, double *w, cudaStream_t s) {
    return launch16<false, true>(E, u, G, D, w, nullptr, s, oz16::HelmArgs16{B, h1, h2});
}

size_t f64tc16_prepared_bytes_per_element() { return (size_t)oz16::kPreElem; }

namespace oz16 {
// The prepared geometric factor of order 15: the element's 6 x 4096 entries
// split hi + lo against one power-of-two scale, from the element's largest
// biased exponent (stored in the 16-byte tail in front of the halves).  One
// block per element: a pass for the exponent, a pass for the split.
__global__ void __launch_bounds__(256) prepare16_kernel(int64_t E, const double *__restrict__ G,
                                                        unsigned char *__restrict__ Gp) {
    __shared__ unsigned wmax[8];
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        const double *Ge = G + e * 6 * kN3;
        unsigned hmax = 0;
        for (int q = threadIdx.x; q < 6 * kN3; q += blockDim.x) hmax = max(hmax, habs(ld_stream(Ge + q)));
        hmax = __reduce_max_sync(0xffffffffu, hmax);
        if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = hmax;
        __syncthreads();
        hmax = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) hmax = max(hmax, wmax[q]);
        const int eg = (int)(hmax >> 20), sh = max(eg, 1) - 1023;
        const unsigned K = (unsigned)(896 + sh) << 23, mw = (unsigned)max(897 + sh, 1) << 20;
        unsigned char *pe = Gp + e * (int64_t)kPreElem;
        float2 *out = reinterpret_cast<float2 *>(pe + kTail);   // [6][4096]: the two halves in order
        for (int q = threadIdx.x; q < 6 * kN3; q += blockDim.x) {
            const double x = ld_stream(Ge + q);
            const df d = split_g(x, habs(x), K, mw);
            out[q] = make_float2(d.hi, d.lo);
        }
        if (threadIdx.x == 0) *reinterpret_cast<int4 *>(pe) = make_int4(eg, 0, 0, 0);
        __syncthreads();   // wmax is reused by the next element
    }
}
}  // namespace oz16

int prepare_f64tc16(int64_t E, const double *G, void *Gp, cudaStream_t s) {
    const int64_t blocks = std::min<int64_t>(E, (int64_t)device_sm_count() * 8);
    oz16::prepare16_kernel<<<(unsigned)blocks, 256, 0, s>>>(E, G, (unsigned char *)Gp);
    return launch_status();
}

}  // namespace semax
