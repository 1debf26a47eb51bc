// FP64-accurate Ax with the six contractions on FP16 tensor cores by exact
// slicing (the Ozaki scheme: Ozaki, Ogita, Oishi & Rump, Numer. Algorithms
// 59, 2012; its tensor-core forms: Mukunoki, Ozaki, Ogita & Imamura, ICCS
// 2020; Ootomo, Ozaki & Yokota, IJHPCA 2024).  Order n = 8 (N = 7).
//
// Slicing.  An operand x with one power-of-two scale 2^s per element is
// written in balanced base-1024 digits, the leading one taking nine bits,
//     x = 2^s sum_{q=0..4} d_q 2^(-10q - 9) + (error <= 2^(s-50)),
// with every d_q an integer of magnitude <= 528, which FP16 holds exactly.
// A digit of D times a digit of u is an integer of magnitude below 2^18.1;
// one m16n8k16 product sums 16 of them (two digit pairs of the same level,
// 8 terms each), and one level L = p + q collects at most five pairs, so
// every FP32 accumulator holds an integer below 2^24: the tensor-core sums
// are exact.  Levels L = 0..4 are kept (15 digit pairs per contraction, 7
// m16n8k16 + 3 m16n8k8 products per 16 x 8 output tile); the dropped levels
// weigh less than 2^-48 of the element's scale.  The five level sums of an
// output are combined in double-float (an unevaluated sum of two floats).
//
// Per element (one CTA of 4 warps, five CTAs per SM with G prepared and four
// with FP64 G; warp w owns the planes k = 2w, 2w+1 for every pointwise step,
// in the layout of the m16n8 accumulator of the r-direction tile; u and G of
// the CTA's next element are fetched by TMA bulk copies into shared memory
// while the current one finishes):
//   A  u (FP64) -> per-element scale -> 5 FP16 digit planes in shared memory;
//   B  ur, us, ut on tensor cores (B operand: the digits of D^T, held in
//      registers for the CTA's lifetime); ur stays in registers, us and ut
//      go through two swizzled double-float buffers (the r- and
//      s-contractions read only the warp's own planes and start before the
//      CTA barrier that the t-contraction needs);
//   C  y = G [ur us ut] in double-float, G split hi + lo by bit operations
//      after a power-of-two scale (per node from FP64 G, per element in the
//      prepared form); per-element scale of y; 5 digits of each component:
//      those of y_r stay in registers as A fragments, those of y_s too after
//      a movmatrix transpose, those of y_t go to shared memory;
//   D  w_r + w_s on tensor cores into one set of level accumulators (the
//      s-part through a block-diagonal A, below), w_t from the shared digits;
//   E  w = (w_rs + w_t) * 2^(scales) in FP64, stored.
// The only FP64 instruction is the final add of each node.
// Inputs with Inf or NaN make their element's output NaN.
#include "ax_f64tc.cuh"

namespace semax {
namespace oz {

constexpr int kThreads = 128;                // one element per CTA pass
constexpr int kPlane = 128;                  // bytes per 8 x 8 FP16 plane (rows XOR-swizzled)
constexpr int kSlice = 8 * kPlane;           // one digit of an 8^3 operand
constexpr int kDigBytes = kS10 * kSlice;     // digits of u, later of wt (wr and ws stay in registers)
constexpr int kBufBytes = 512 * 8;           // one double-float per node
constexpr int kGBytes = 6 * 512 * 8;         // one element's G (FP64), staged
constexpr int kUBytes = 512 * 8;             // one element's u (FP64), staged
constexpr int kTailBytes = 16;               // prepared form: the element's largest G exponent (and padding)
constexpr int kPreBytes = kGBytes + kTailBytes;   // one element of the prepared geometric factor
// + mbarrier in the last 8 of the reduction slots
template <bool PRE>
constexpr size_t smem_bytes() { return kDigBytes + 2 * kBufBytes + (PRE ? kPreBytes : kGBytes) + kUBytes + 16 * sizeof(int); }

// Byte offset of row j of plane p inside a digit slice: the 16-byte rows of
// a plane are permuted by p, so that ldmatrix over the 8 rows of a plane
// and over the 8 planes of a row both touch 8 distinct bank groups.
__device__ __forceinline__ int prow(int p, int j) { return p * kPlane + ((j ^ p) << 4); }

// One 16 x 8 output tile of a contraction along direction DIR (0: r / i,
// 1: s / j, 2: t / k) for warp w, all 15 digit pairs of levels 0..4.
// base: shared address of digit 0 of the operand; Bf[p]: the B fragment of
// digit p of D^T (gradient) or D (transposed).  Accumulator rows:
//   DIR 0: (k, j) = (2w + m / 8, m % 8), columns i;
//   DIR 1: (k, i) = (2w + m / 8, m % 8), columns j;
//   DIR 2: (j, i) = (2w + m / 8, m % 8), columns k.
template <int DIR>
__device__ __forceinline__ void contract(uint32_t base, int warp, int lane, const uint32_t (&Bf)[kS10],
                                         float (&acc)[kS10][4]) {
    const int mi = lane >> 3, rr = lane & 7;
    const int blk = 2 * warp + (mi & 1);
    // x4: digits q, q + 1 (lanes 16-31 address the second); x2: digit 4 (lanes 0-15)
    const uint32_t addr = base + (mi >> 1) * kSlice + (DIR == 2 ? prow(rr, blk) : prow(blk, rr));
    uint32_t a[kS10][2];
#pragma unroll
    for (int q = 0; q < 4; q += 2) {
        if (DIR == 0)
            mma::ldsm_x4(addr + q * kSlice, a[q][0], a[q][1], a[q + 1][0], a[q + 1][1]);
        else
            mma::ldsm_x4_t(addr + q * kSlice, a[q][0], a[q][1], a[q + 1][0], a[q + 1][1]);
    }
    if (DIR == 0)
        mma::ldsm_x2(addr + 4 * kSlice, a[4][0], a[4][1]);
    else
        mma::ldsm_x2_t(addr + 4 * kSlice, a[4][0], a[4][1]);
#pragma unroll
    for (int l = 0; l < kS10; ++l) acc[l][0] = acc[l][1] = acc[l][2] = acc[l][3] = 0.0f;
    // level L = p + q for D digit p and operand digit q (0-based)
#define OZ_K8(L, p, q) mma::f16_1688(acc[L], a[q][0], a[q][1], Bf[p])
#define OZ_K16(L, p1, q1, p2, q2) mma::f16_16816(acc[L], a[q1][0], a[q1][1], a[q2][0], a[q2][1], Bf[p1], Bf[p2])
    // round-robin over the levels: consecutive products update different accumulators
    OZ_K8(0, 0, 0);
    OZ_K16(1, 0, 1, 1, 0);
    OZ_K16(2, 0, 2, 1, 1);
    OZ_K16(3, 0, 3, 1, 2);
    OZ_K16(4, 0, 4, 1, 3);
    OZ_K8(2, 2, 0);
    OZ_K16(3, 2, 1, 3, 0);
    OZ_K16(4, 2, 2, 3, 1);
    OZ_K8(4, 4, 0);
#undef OZ_K8
#undef OZ_K16
}

// The same with the A fragments in registers: a[q][h] holds digit q of the
// rows of plane 2w + h (DIR 0: rows j, columns i; DIR 1: rows i, columns j).
__device__ __forceinline__ void contract_regs(const uint32_t (&a)[kS10][2], const uint32_t (&Bf)[kS10],
                                              float (&acc)[kS10][4]) {
#pragma unroll
    for (int l = 0; l < kS10; ++l) acc[l][0] = acc[l][1] = acc[l][2] = acc[l][3] = 0.0f;
#define OZ_K8(L, p, q) mma::f16_1688(acc[L], a[q][0], a[q][1], Bf[p])
#define OZ_K16(L, p1, q1, p2, q2) mma::f16_16816(acc[L], a[q1][0], a[q1][1], a[q2][0], a[q2][1], Bf[p1], Bf[p2])
    OZ_K8(0, 0, 0);
    OZ_K16(1, 0, 1, 1, 0);
    OZ_K16(2, 0, 2, 1, 1);
    OZ_K16(3, 0, 3, 1, 2);
    OZ_K16(4, 0, 4, 1, 3);
    OZ_K8(2, 2, 0);
    OZ_K16(3, 2, 1, 3, 0);
    OZ_K16(4, 2, 2, 3, 1);
    OZ_K8(4, 4, 0);
#undef OZ_K8
#undef OZ_K16
}

// Double-float buffers of the s- and t-direction results (one float2 per
// node), XOR-swizzled so that the accumulator-layout writes and the
// pointwise reads are both free of bank conflicts:
//   s: [k][i][j], t: [j][k][i], bits 2-3 of the flat index flipped by a key
//   that does not depend on them.
__device__ __forceinline__ int sidx(int k, int j, int i) { return (64 * k + 8 * i + j) ^ (((i >> 1) & 3) << 2); }
__device__ __forceinline__ int tidx(int k, int j, int i) {
    return (64 * j + 8 * k + i) ^ ((((k >> 1) & 3) ^ ((j & 1) << 1)) << 2);
}

// Write the s- or t-direction tile of warp w (levels combined) to its buffer.
template <int DIR>
__device__ __forceinline__ void store_tile(float2 *buf, const float (&acc)[kS10][4], int warp, int g, int t) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        df v0, v1;
        combine5_k8x2(acc, 2 * h, v0, v1);
        if (DIR == 1) {   // rows (k = 2w + h, i = g), columns j = 2t, 2t + 1: adjacent in [k][i][j]
            *reinterpret_cast<float4 *>(buf + sidx(2 * warp + h, 2 * t, g)) = make_float4(v0.hi, v0.lo, v1.hi, v1.lo);
        } else {          // rows (j = 2w + h, i = g), columns k = 2t, 2t + 1
            buf[tidx(2 * t, 2 * warp + h, g)] = make_float2(v0.hi, v0.lo);
            buf[tidx(2 * t + 1, 2 * warp + h, g)] = make_float2(v1.hi, v1.lo);
        }
    }
}

__device__ __forceinline__ int max4(const int *p) { return max(max(p[0], p[1]), max(p[2], p[3])); }

// The Helmholtz form's mass term: w = h1 (A u) + h2 B u, B [E][512].
struct HelmArgs {
    const double *B;
    double h1, h2;
};

// PRE = false: G is FP64 [E][6][512]; PRE = true: G points at the prepared
// form, per element 6 x 512 (hi, lo) float pairs (G split against the
// element's scale) and a 16-byte tail whose first int is the element's
// largest biased exponent of G.  HELM: w = h1 (A u) + h2 B u, the mass term
// added in FP64 to the FP64 output of A u (three FP64 operations per node).
template <bool PRE, bool HELM = false>
__global__ void __launch_bounds__(kThreads, PRE ? 5 : 4)
ax_f64tc_kernel(int64_t E, const double *__restrict__ u, const double *__restrict__ G,
                const double *__restrict__ D, double *__restrict__ w, int *__restrict__ status, int polls,
                HelmArgs hm) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *dig = smem;
    float2 *bs = reinterpret_cast<float2 *>(smem + kDigBytes);   // s-direction results
    float2 *bt = bs + 512;                                         // t-direction results
    const double2 *gst = reinterpret_cast<const double2 *>(bt + 512);   // staged G [6][256 node pairs]
    const float4 *gpre = reinterpret_cast<const float4 *>(gst);         // prepared: [6][256 node pairs] (hi, lo) x 2
    const int *egst = reinterpret_cast<const int *>(reinterpret_cast<const unsigned char *>(gst) + kGBytes);
    const double2 *ust = reinterpret_cast<const double2 *>(reinterpret_cast<const unsigned char *>(gst) +
                                                           (PRE ? kPreBytes : kGBytes));   // staged u [256 node pairs]
    int *sred = reinterpret_cast<int *>(smem + kDigBytes + 2 * kBufBytes + (PRE ? kPreBytes : kGBytes) + kUBytes);   // [0, 4) u, [4, 8) y exponents
    const uint32_t bar = smem_u32(sred + 8);                      // mbarrier of the staged u and G (8-byte aligned)
    const uint32_t dig_s = smem_u32(dig), gst_s = smem_u32(gst), ust_s = smem_u32(ust);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;

    // u_e and G_e are contiguous (4 KB, 24 KB) and staged in their global
    // layout by two TMA bulk copies, issued by one thread for element
    // e + gridDim.x once every thread has read element e's G; each element
    // completes one phase of the mbarrier.
    auto prefetch = [&](int64_t ep) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic reads before async writes
        mbar_expect_tx(bar, kUBytes + (PRE ? kPreBytes : kGBytes));
        bulk_g2s(ust_s, u + ep * 512, kUBytes, bar);
        if (PRE)
            bulk_g2s(gst_s, reinterpret_cast<const unsigned char *>(G) + ep * kPreBytes, kPreBytes, bar);
        else
            bulk_g2s(gst_s, G + ep * 3072, kGBytes, bar);
    };
    if (tid == 0) mbar_init(bar, 1);
    __syncthreads();
    // launched as a programmatic dependent of the previous kernel in the
    // stream: this CTA may already be resident while that kernel finishes;
    // no global memory is read before it has completed
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (tid == 0) prefetch(blockIdx.x);

    // D digits, once per CTA: B fragments of D^T (gradient) and D (transposed)
    int eD = 1;
    for (int q = lane; q < 64; q += 32) eD = max(eD, max(bexp(D[q]), 1));
    eD = __reduce_max_sync(0xffffffffu, eD);
    uint32_t fg[kS10], ft[kS10];
    {
        float x0[kS10], x1[kS10];
        digits10_fp64(D[g * 8 + 2 * t], eD, x0);
        digits10_fp64(D[g * 8 + 2 * t + 1], eD, x1);
#pragma unroll
        for (int p = 0; p < kS10; ++p) fg[p] = pack_f16(-x0[p], -x1[p]);   // negated, like u's and y's
        digits10_fp64(D[(2 * t) * 8 + g], eD, x0);
        digits10_fp64(D[(2 * t + 1) * 8 + g], eD, x1);
#pragma unroll
        for (int p = 0; p < kS10; ++p) ft[p] = pack_f16(-x0[p], -x1[p]);
    }

    unsigned parity = 0;
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x, parity ^= 1u) {
        double *we = w + e * 512;
        // the CTA's last element: a dependent launch may start taking SMs
        if (e + gridDim.x >= E) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

        // ---- A: u -> digits (thread's nodes: k = 2w + h, j = g, i = 2t + c)
        const bool timed_out = !mbar_wait(bar, parity, polls);
        double2 uv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) uv[h] = ust[(2 * warp + h) * 32 + g * 4 + t];
        int ex = 1;
#pragma unroll
        for (int h = 0; h < 2; ++h) ex = max(ex, (int)(max(habs(uv[h].x), habs(uv[h].y)) >> 20));
        ex = __reduce_max_sync(0xffffffffu, ex);
        if (lane == 0) sred[warp] = ex;
        if (__syncthreads_or(timed_out)) {
            // the staged data never arrived: report it, mark this CTA's remaining
            // outputs NaN and leave (the decision is the same in every thread)
            if (tid == 0) report_timeout(status);
            for (int64_t r = e; r < E; r += gridDim.x)
                for (int q = tid; q < 512; q += kThreads) w[r * 512 + q] = __longlong_as_double(0x7ff8000000000000ll);
            mbar_wait(bar, parity);   // one more bounded wait for the copies in flight
            return;
        }
        const int eU = max4(sred);
        // u 2^-(eU - 1023) in (-2, 2) split hi + lo (47 bits), normalised; its
        // digits at t = 256 u 2^-(eU - 1023) = 512 u 2^-(eU - 1022)
        const unsigned Ku = (unsigned)(eU - 127) << 23;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float d0[kS10], d1[kS10];
            const unsigned mw = (unsigned)max(eU - 126, 1) << 20;
            const df a0 = split_g(uv[h].x, habs(uv[h].x), Ku, mw);
            const df a1 = split_g(uv[h].y, habs(uv[h].y), Ku, mw);
            const df n0 = dfx::fast_two_sum(a0.hi, a0.lo), n1 = dfx::fast_two_sum(a1.hi, a1.lo);
            digits10_df2_neg(make_float2(n0.hi, n1.hi), make_float2(n0.lo, n1.lo), f2(256.0f), f2(268435456.0f), d0, d1);
            unsigned char *p = dig + prow(2 * warp + h, g) + 4 * t;
#pragma unroll
            for (int q = 0; q < kS10; ++q) *reinterpret_cast<uint32_t *>(p + q * kSlice) = pack_f16(d0[q], d1[q]);
        }
        __syncwarp();   // the r- and s-contractions read only this warp's planes

        // ---- B: gradient on tensor cores
        df vr[4];
        {
            float acc[kS10][4];
            contract<0>(dig_s, warp, lane, fg, acc);
#pragma unroll
            for (int q = 0; q < 4; q += 2) combine5_k8x2(acc, q, vr[q], vr[q + 1]);
        }
        {
            float acc[kS10][4];
            contract<1>(dig_s, warp, lane, fg, acc);
            store_tile<1>(bs, acc, warp, g, t);
        }
        __syncthreads();   // the t-contraction reads every warp's planes
        {
            float acc[kS10][4];
            contract<2>(dig_s, warp, lane, fg, acc);
            store_tile<2>(bt, acc, warp, g, t);
        }
        __syncthreads();

        // ---- C: y = G grad in double-float; per-element scale; digits
        // G is split against a power-of-two scale 2^sh: per node for FP64 G,
        // per element in the prepared form (the same digits unless the
        // element's G entries span more than ~2^100)
        acc2 y[4][3];
        int shn[4];
        int tmax = INT_MIN;
        const int egE = PRE ? egst[0] : 0;   // prepared: the element's largest biased G exponent
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 2 * warp + h, nb = k * 64 + g * 8 + 2 * t;
            double2 gv[6];
            float4 gp[6];
            if (PRE) {
#pragma unroll
                for (int a = 0; a < 6; ++a) gp[a] = gpre[a * 256 + (nb >> 1)];
            } else {
#pragma unroll
                for (int a = 0; a < 6; ++a) gv[a] = gst[a * 256 + (nb >> 1)];
            }
            const float4 tv = *reinterpret_cast<const float4 *>(bt + tidx(k, g, 2 * t));
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int q = 2 * h + c;
                const float2 sv = bs[sidx(k, g, 2 * t + c)];
                const df Vs{sv.x, sv.y};
                const df Vt = c ? df{tv.z, tv.w} : df{tv.x, tv.y};
                df Gh[6];
                int sh = 0;
                if (PRE) {
#pragma unroll
                    for (int a = 0; a < 6; ++a) Gh[a] = c ? df{gp[a].z, gp[a].w} : df{gp[a].x, gp[a].y};
                } else {
                    double Gc[6];
                    unsigned hws[6], hmax = 0;
#pragma unroll
                    for (int a = 0; a < 6; ++a) {
                        Gc[a] = c ? gv[a].y : gv[a].x;
                        hws[a] = habs(Gc[a]);
                        hmax = max(hmax, hws[a]);
                    }
                    const int eg = (int)(hmax >> 20);   // largest biased exponent of the node's G
                    sh = max(eg, 1) - 1023;             // G * 2^-sh has magnitude < 2
                    const unsigned K = (unsigned)(896 + sh) << 23;
#pragma unroll
                    for (int a = 0; a < 6; ++a) Gh[a] = split_g(Gc[a], hws[a], K, (unsigned)max(897 + sh, 1) << 20);
                    if (eg == 0x7ff) tmax = kBadExp;
                }
                y[q][0] = dot3(Gh[0], Gh[1], Gh[2], vr[q], Vs, Vt);
                y[q][1] = dot3(Gh[1], Gh[3], Gh[4], vr[q], Vs, Vt);
                y[q][2] = dot3(Gh[2], Gh[4], Gh[5], vr[q], Vs, Vt);
                // renormalise: when the leading level sums of a gradient cancel
                // exactly, its value sits in the low part, and so can y's
#pragma unroll
                for (int a = 0; a < 3; ++a) y[q][a] = renorm(y[q][a]);
                shn[q] = sh;
                const float ym = fmaxf(fabsf(y[q][0].s), fmaxf(fabsf(y[q][1].s), fabsf(y[q][2].s)));
                const int ev = (int)(__float_as_uint(ym) >> 23);
                if (ev) tmax = max(tmax, ev + sh);
            }
        }
        tmax = __reduce_max_sync(0xffffffffu, tmax);
        if (lane == 0) sred[4 + warp] = tmax;
        __syncthreads();
        if (tid == 0 && e + gridDim.x < E) prefetch(e + gridDim.x);   // every thread has read this element's G
        const int eWraw = max4(sred + 4);
        const bool bad = eU == 0x7ff || eD == 0x7ff || eWraw >= kBadExp || egE == 0x7ff;
        const int eW = eWraw == INT_MIN ? 0 : min(eWraw, kBadExp);   // y == 0 everywhere: any scale
        const int shE = PRE ? max(egE, 1) - 1023 : 0;                 // prepared: the element's G scale
        // digits of y_r and y_s stay in registers as A fragments (y_s transposed
        // by movmatrix); those of y_t, which the t-contraction reads across
        // warps, go to shared memory
        uint32_t yr[kS10][2], ys[kS10][2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            unsigned char *p = dig + prow(2 * warp + h, g) + 4 * t;
            const float m0 = pow2f_or_zero(shn[2 * h] - eW + 135);       // |y 2^(sh - eW + 126)| < 1
            const float m1 = pow2f_or_zero(shn[2 * h + 1] - eW + 135);
            const float m0s = times2p20(m0), m1s = times2p20(m1);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float d0[kS10], d1[kS10];
                digits10_df2_neg(make_float2(y[2 * h][a].s, y[2 * h + 1][a].s), make_float2(y[2 * h][a].c, y[2 * h + 1][a].c),
                                 make_float2(m0, m1), make_float2(m0s, m1s), d0, d1);
#pragma unroll
                for (int q = 0; q < kS10; ++q) {
                    const uint32_t v = pack_f16(d0[q], d1[q]);
                    if (a == 0)
                        yr[q][h] = v;
                    else if (a == 1)
                        ys[q][h] = mma::movm_t(v);
                    else
                        *reinterpret_cast<uint32_t *>(p + q * kSlice) = v;
                }
            }
        }

        // ---- D: transposed contractions on tensor cores.  The s-part lands in
        // the r-part's accumulators: with K = (plane, l) and the block-diagonal
        // A = diag(D^T, D^T) over the warp's two planes, the product of A with
        // the B fragments of y_s (planes 2w, 2w + 1) has rows (k, j) and
        // columns i, the layout of the r-part.  The level sums then collect
        // twice the products (levels 0..2 stay below 2^24 and exact; levels 3
        // and 4 may round by a unit at weights 2^-30 and 2^-40).
        df vo[4];
        {
            float acc[kS10][4];
            contract_regs(yr, ft, acc);
#pragma unroll
            for (int a = 0; a < kS10; ++a)
#pragma unroll
                for (int L = a; L < kS10; ++L) mma::f16_16816(acc[L], ft[a], 0u, 0u, ft[a], ys[L - a][0], ys[L - a][1]);
#pragma unroll
            for (int q = 0; q < 4; q += 2) combine5x2(acc, q, vo[q], vo[q + 1]);
        }
        __syncthreads();   // y_t's digits of every warp
        {
            float acc[kS10][4];
            contract<2>(dig_s, warp, lane, ft, acc);
            store_tile<2>(bt, acc, warp, g, t);
        }
        __syncthreads();

        // ---- E: sum, undo the scales, store
        // w = 2^((eU - 1022) + 2 (eD - 1022) + (eW - 126) - 36) V_out
        const int SH = (eU - 1022) + 2 * (eD - 1022) + (eW + shE - 126) - 36;
        const bool fastSH = SH >= -896 && SH <= 896;   // the same for the whole element
        const unsigned cSH = (unsigned)(896 + SH) << 20;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 2 * warp + h, nb = k * 64 + g * 8 + 2 * t;
            const float4 tv = *reinterpret_cast<const float4 *>(bt + tidx(k, g, 2 * t));
            double o[2];
            double2 bv = make_double2(0.0, 0.0);
            if (HELM)
                asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];"
                             : "=d"(bv.x), "=d"(bv.y) : "l"(hm.B + e * 512 + nb));
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const float th = c ? tv.z : tv.x, tl = c ? tv.w : tv.y;
                const df b = dfx::two_sum(vo[2 * h + c].hi, th);
                const float lo = __fadd_rn(__fadd_rn(vo[2 * h + c].lo, tl), b.lo);
                // bit-level conversions with the scale in the exponent field: one FP64 add
                double dh, dl;
                if (fastSH)
                    o[c] = dfx::f2d_shift(b.hi, cSH) + dfx::f2d_shift(lo, cSH);
                else if (dfx::f2d_scaled(b.hi, SH, dh) && dfx::f2d_scaled(lo, SH, dl))
                    o[c] = dh + dl;
                else
                    o[c] = scale2(dfx::f2d(b.hi) + dfx::f2d(lo), SH);
                if (HELM) {   // u of this node is still in uv from phase A
                    const double uu = c ? uv[h].y : uv[h].x, bb = c ? bv.y : bv.x;
                    o[c] = hm.h1 == 1.0 ? __fma_rn(hm.h2 * bb, uu, o[c]) : __fma_rn(hm.h2 * bb, uu, hm.h1 * o[c]);
                }
                if (bad) o[c] = __longlong_as_double(0x7ff8000000000000ll);
            }
            *reinterpret_cast<double2 *>(we + nb) = make_double2(o[0], o[1]);
        }
    }
    __syncthreads();   // no thread polls the mbarrier any more, and no copy is in flight
    if (tid == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

template <bool PRE, bool HELM = false>
static int launch(int64_t E, const double *u, const double *G, const double *D, double *w, int *status,
                  cudaStream_t s, HelmArgs hm = HelmArgs{nullptr, 1.0, 0.0}) {
    auto kern = ax_f64tc_kernel<PRE, HELM>;
    constexpr size_t kSmem = smem_bytes<PRE>();
    int st = cuda_status(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
    if (st != SEMAX_OK) return st;
    st = cuda_status(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          (int)cudaSharedmemCarveoutMaxShared));
    if (st != SEMAX_OK) return st;
    int per_sm = 0;
    st = cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, kSmem));
    if (st != SEMAX_OK) return st;
    const int64_t grid = std::min<int64_t>(E, (int64_t)device_sm_count() * std::max(per_sm, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    st = cuda_status(cudaLaunchKernelEx(&cfg, kern, E, u, G, D, w, status, first_wait_polls(), hm));
    if (st != SEMAX_OK) return st;
    return launch_status();
}

// The prepared geometric factor: G's entries split hi + lo against one
// power-of-two scale per element (from the element's largest biased exponent,
// stored after the 6 x 512 float pairs).  One block of 256 threads per
// element, two nodes per thread.
__global__ void __launch_bounds__(256) prepare_kernel(int64_t E, const double *__restrict__ G,
                                                      unsigned char *__restrict__ Gp) {
    __shared__ unsigned wmax[8];
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        const double *Ge = G + e * 3072;
        double Gc[2][6];
        unsigned hws[2][6], hmax = 0;
#pragma unroll
        for (int x = 0; x < 2; ++x)
#pragma unroll
            for (int a = 0; a < 6; ++a) {
                Gc[x][a] = ld_stream(Ge + a * 512 + threadIdx.x + 256 * x);
                hws[x][a] = habs(Gc[x][a]);
                hmax = max(hmax, hws[x][a]);
            }
        hmax = __reduce_max_sync(0xffffffffu, hmax);
        if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = hmax;
        __syncthreads();
        hmax = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) hmax = max(hmax, wmax[q]);
        const int eg = (int)(hmax >> 20), sh = max(eg, 1) - 1023;
        const unsigned K = (unsigned)(896 + sh) << 23, mw = (unsigned)max(897 + sh, 1) << 20;
        float2 *out = reinterpret_cast<float2 *>(Gp + e * kPreBytes);
#pragma unroll
        for (int x = 0; x < 2; ++x)
#pragma unroll
            for (int a = 0; a < 6; ++a) {
                const df d = split_g(Gc[x][a], hws[x][a], K, mw);
                out[a * 512 + threadIdx.x + 256 * x] = make_float2(d.hi, d.lo);
            }
        if (threadIdx.x == 0) *reinterpret_cast<int4 *>(Gp + e * kPreBytes + kGBytes) = make_int4(eg, 0, 0, 0);
        __syncthreads();   // wmax is reused by the next element
    }
}

}  // namespace oz
}  // namespace semax

namespace semax {
int launch_f64tc16(int64_t E, const double *u, const double *G, const double *D, double *w, int *status,
                   cudaStream_t s);
int launch_f64tc16_prepared(int64_t E, const double *u, const void *Gp, const double *D, double *w, int *status,
                            cudaStream_t s);
int prepare_f64tc16(int64_t E, const double *G, void *Gp, cudaStream_t s);
int launch_f64tc16_helmholtz(int64_t E, const double *u, const double *G, const double *B, const double *D,
                             double h1, double h2, double *w, cudaStream_t s);
size_t f64tc16_prepared_bytes_per_element();
}

using namespace semax;

extern "C" int sem_ax_f64tc_status(int64_t E, int N, const double *u, const double *G, const double *D, double *w,
                                   int *status, void *stream) {
    int st = check_args(E, N, u, G, D, w);
    if (st != SEMAX_OK || E == 0) return st;
    if (status && ((uintptr_t)status % alignof(int)) != 0) return SEMAX_EALIGN;
    if (N == 7) return oz::launch<false>(E, u, G, D, w, status, (cudaStream_t)stream);
    if (N == 15) return launch_f64tc16(E, u, G, D, w, status, (cudaStream_t)stream);
    return sem_ax_f64x(E, N, u, G, D, w, stream);   // other orders: the double-float tile (no waits)
}

extern "C" int sem_ax_helmholtz_f64tc(int64_t E, int N, const double *u, const double *G, const double *B,
                                      const double *D, double h1, double h2, double *w, void *stream) {
    if (N != 7 && N != 15) return sem_ax_helmholtz(E, N, u, G, B, D, h1, h2, w, stream);
    int st = check_args(E, N, u, G, D, w);
    if (st != SEMAX_OK || E == 0) return st;
    if (!B) return SEMAX_EINVAL;
    if (!aligned16(B)) return SEMAX_EALIGN;
    const size_t bytes = (size_t)E * (N + 1) * (N + 1) * (N + 1) * sizeof(double);
    if (overlaps(w, bytes, B, bytes)) return SEMAX_EALIAS;
    if (N == 15) return launch_f64tc16_helmholtz(E, u, G, B, D, h1, h2, w, (cudaStream_t)stream);
    return oz::launch<false, true>(E, u, G, D, w, nullptr, (cudaStream_t)stream, oz::HelmArgs{B, h1, h2});
}

extern "C" int sem_ax_f64tc(int64_t E, int N, const double *u, const double *G, const double *D, double *w,
                            void *stream) {
    return sem_ax_f64tc_status(E, N, u, G, D, w, nullptr, stream);
}

// bytes of one element of the prepared geometric factor, 0 if N has none
static size_t prepared_bytes(int N) {
    return N == 7 ? (size_t)oz::kPreBytes : (N == 15 ? f64tc16_prepared_bytes_per_element() : 0);
}

extern "C" int sem_ax_f64tc_prepare_size(int64_t E, int N, size_t *bytes) {
    if (!bytes || E < 0) return SEMAX_EINVAL;
    if (!prepared_bytes(N)) return SEMAX_EUNSUPPORTED_N;
    *bytes = (size_t)E * prepared_bytes(N);
    return SEMAX_OK;
}

extern "C" int sem_ax_f64tc_prepare(int64_t E, int N, const double *G, void *Gp, void *stream) {
    if (E < 0) return SEMAX_EINVAL;
    if (!prepared_bytes(N)) return SEMAX_EUNSUPPORTED_N;
    if (E == 0) return SEMAX_OK;
    if (!G || !Gp) return SEMAX_EINVAL;
    if (!aligned16(G) || !aligned16(Gp)) return SEMAX_EALIGN;
    const size_t n3 = (size_t)(N + 1) * (N + 1) * (N + 1);
    if (overlaps(G, (size_t)E * 6 * n3 * sizeof(double), Gp, (size_t)E * prepared_bytes(N))) return SEMAX_EALIAS;
    if (N == 15) return prepare_f64tc16(E, G, Gp, (cudaStream_t)stream);
    const int64_t blocks = std::min<int64_t>(E, (int64_t)device_sm_count() * 8);
    oz::prepare_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(E, G, (unsigned char *)Gp);
    return launch_status();
}

extern "C" int sem_ax_f64tc_prepared_status(int64_t E, int N, const double *u, const void *Gp, const double *D,
                                            double *w, int *status, void *stream) {
    if (E < 0) return SEMAX_EINVAL;
    if (!prepared_bytes(N)) return SEMAX_EUNSUPPORTED_N;
    if (E == 0) return SEMAX_OK;
    if (!u || !Gp || !D || !w) return SEMAX_EINVAL;
    if (!aligned16(u) || !aligned16(Gp) || !aligned16(w) || ((uintptr_t)D % alignof(double)) != 0)
        return SEMAX_EALIGN;
    if (status && ((uintptr_t)status % alignof(int)) != 0) return SEMAX_EALIGN;
    const size_t n = (size_t)N + 1, ub = (size_t)E * n * n * n * sizeof(double);
    if (overlaps(w, ub, u, ub) || overlaps(w, ub, Gp, (size_t)E * prepared_bytes(N)) ||
        overlaps(w, ub, D, n * n * sizeof(double)))
        return SEMAX_EALIAS;
    if (N == 15) return launch_f64tc16_prepared(E, u, Gp, D, w, status, (cudaStream_t)stream);
    return oz::launch<true>(E, u, reinterpret_cast<const double *>(Gp), D, w, status, (cudaStream_t)stream);
}

extern "C" int sem_ax_f64tc_prepared(int64_t E, int N, const double *u, const void *Gp, const double *D, double *w,
                                     void *stream) {
    return sem_ax_f64tc_prepared_status(E, N, u, Gp, D, w, nullptr, stream);
}
