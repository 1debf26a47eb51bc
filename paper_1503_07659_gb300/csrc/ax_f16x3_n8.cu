// FP16 split with three products (sem_ax_f16x3) for order N = 7 (n = 8):
// FP32 u, G, D, w; each contraction operand x, scaled by a power of two s so
// that its group's largest magnitude lies in [1, 2), is split into FP16
// pieces x s = x0 + x1, and the products x0 y0 + x0 y1 + x1 y0 are summed in
// FP32 on the tensor cores (mma.m16n8k8 / m16n8k16).  Scales: u per element,
// D once per CTA, wr and ws per warp (their contractions stay inside the
// warp's two planes), wt per element (its contraction crosses planes); all
// are undone on the output.  The geometric-factor multiply is FP32.
//
// Per element, one CTA of 4 warps; warp w owns the planes k = 2w, 2w + 1 in
// the layout of the m16n8 accumulator of the r-direction tile (rows (k, j),
// columns i), thread (g, t) the nodes (k, j = g, i = 2t + c):
//   A  u (staged by cp.async with the element's G while the previous element
//      finishes) -> scale -> two FP16 piece planes in shared memory;
//   B  ur (registers), us (warp-private buffer), ut (shared buffer) on
//      tensor cores, B operand the pieces of D^T held in registers;
//   C  [wr ws wt] = G [ur us ut] in FP32; pieces of wr stay in registers as
//      A fragments, of ws too after a movmatrix transpose; pieces of wt go
//      to shared memory;
//   D  w_r + w_s into one accumulator (the s-part through the block-diagonal
//      A = diag(D^T, D^T) over the warp's two planes, K = (plane, l)), w_t
//      from the shared pieces;
//   E  w = (w_rs / s_rs + w_t / s_t) / (s_u s_D^2) (times the element's G
//      scale), stored.
#include <cuda_fp16.h>

#include "common.cuh"
#include "mma_sync.cuh"

namespace semax {
namespace f16n8 {

constexpr int kThreads = 128;
constexpr int kN3 = 512;
constexpr int kPlane = 128;                  // bytes per 8 x 8 FP16 plane (rows XOR-swizzled)
constexpr int kSlice = 8 * kPlane;           // one piece of an 8^3 operand
constexpr int kPieces = 2 * kSlice;          // u's pieces, later wt's
constexpr int kStage = kN3 * 4 + 6 * kN3 * 4;   // u and G of one element (FP32, 14 KB)
constexpr int kSPitchI = 8, kSPlane = 64;    // us buffer [k][i][j]
constexpr int kTPlane = 68;                  // ut / w_t buffer [k][j][i], planes padded by 4 words
constexpr size_t kSmem = kStage + kPieces + (8 * kSPlane + 8 * kTPlane) * 4 + 16 * 4;

// Byte offset of row j of plane p inside a piece slice: the 16-byte rows of
// a plane are permuted by p, so that ldmatrix over the 8 rows of a plane and
// over the 8 planes of a row both touch 8 distinct bank groups.
__device__ __forceinline__ int prow(int p, int j) { return p * kPlane + ((j ^ p) << 4); }

__device__ __forceinline__ int sidx(int k, int j, int i) { return k * kSPlane + i * kSPitchI + j; }
__device__ __forceinline__ int tidx(int k, int j, int i) { return k * kTPlane + j * 8 + i; }

// 2^-e for a group whose largest magnitude has float bits mbits (e its
// exponent): the scaled group lies below 2; clamped to [2^-126, 2^127].
__device__ __forceinline__ float inv_pow2_of(unsigned mbits) {
    const int eb = (int)((mbits >> 23) & 0xffu);
    return __uint_as_float((unsigned)min(max(254 - eb, 1), 254) << 23);
}

// The pair (x, y) as two FP16 pieces: p0 = fp16(x, y), p1 = fp16 of the
// remainders (x in the low halves).
__device__ __forceinline__ void pieces(float x, float y, uint32_t &p0, uint32_t &p1) {
    const __half2 h = __floats2half2_rn(x, y);
    const __half2 l = __floats2half2_rn(x - __low2float(h), y - __high2float(h));
    p0 = *reinterpret_cast<const uint32_t *>(&h);
    p1 = *reinterpret_cast<const uint32_t *>(&l);
}

__device__ __forceinline__ unsigned absbits(float x) { return __float_as_uint(x) & 0x7fffffffu; }

// acc = A B over the piece pairs (0, 0), (0, 1), (1, 0): A fragments a[p][h]
// (piece p, rows of plane 2w + h), B fragments b[p].
__device__ __forceinline__ void mma3(float (&acc)[4], const uint32_t (&a)[2][2], const uint32_t (&b)[2]) {
    acc[0] = acc[1] = acc[2] = acc[3] = 0.0f;
    mma::f16_1688(acc, a[0][0], a[0][1], b[0]);
    mma::f16_16816(acc, a[0][0], a[0][1], a[1][0], a[1][1], b[1], b[0]);
}

// The A fragments of both pieces of the 16 x 8 tile along direction DIR
// (0: r, rows (k, j) of planes 2w, 2w + 1, columns l = i; 1: s, rows (k, i),
// columns l = j; 2: t, rows (j, i) of rows j = 2w, 2w + 1, columns l = k)
// from the piece planes at `base`.
template <int DIR>
__device__ __forceinline__ void load_a(uint32_t base, int warp, int lane, uint32_t (&a)[2][2]) {
    const int mi = lane >> 3, rr = lane & 7;
    const int blk = 2 * warp + (mi & 1);
    const uint32_t addr = base + (mi >> 1) * kSlice + (DIR == 2 ? prow(rr, blk) : prow(blk, rr));
    if (DIR == 0)
        mma::ldsm_x4(addr, a[0][0], a[0][1], a[1][0], a[1][1]);
    else
        mma::ldsm_x4_t(addr, a[0][0], a[0][1], a[1][0], a[1][1]);
}

__global__ void __launch_bounds__(kThreads, 8)
ax_f16x3_n8_kernel(int64_t E, const float *__restrict__ u, const float *__restrict__ G, const float *__restrict__ D,
                   float *__restrict__ w, const float *__restrict__ scale) {
    extern __shared__ __align__(16) unsigned char smem[];
    const float *su = reinterpret_cast<const float *>(smem);        // staged u [512]
    const float *sG = su + kN3;                                     // staged G [6][512]
    unsigned char *pc = smem + kStage;                              // pieces: u's, later wt's
    float *bs = reinterpret_cast<float *>(pc + kPieces);            // us [k][i][j]
    float *bt = bs + 8 * kSPlane;                                   // ut, later w_t [k][j][i]
    unsigned *sred = reinterpret_cast<unsigned *>(bt + 8 * kTPlane);   // [0, 4) |u|, [4, 8) |wt| maxima
    const uint32_t pc_s = mma::smem_u32(pc), stage_s = mma::smem_u32(smem);
    // launched as a programmatic dependent of the previous kernel in the
    // stream: no global memory is read before that kernel has completed
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;

    // u and G of element ep into the staging buffer: 896 16-byte chunks
    auto prefetch = [&](int64_t ep) {
        const char *gu = reinterpret_cast<const char *>(u + ep * kN3);
        const char *gg = reinterpret_cast<const char *>(G + ep * 6 * kN3);
        for (int q = tid; q < kStage / 16; q += kThreads) {
            const char *src = q < kN3 / 4 ? gu + 16 * q : gg + 16 * (q - kN3 / 4);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(stage_s + 16 * q), "l"(src) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (blockIdx.x < E) prefetch(blockIdx.x);

    // pieces of D sD as B fragments: fg (gradient, B[l][i] = D[i][l]) and ft
    // (transposed, B[l][i] = D[l][i]); the same values as the A fragment of
    // the block-diagonal D^T in the transposed s-part
    unsigned dm = max(absbits(D[lane]), absbits(D[lane + 32]));
    const float sD = inv_pow2_of(__reduce_max_sync(0xffffffffu, dm));
    uint32_t fg[2], ft[2];
    pieces(D[g * 8 + 2 * t] * sD, D[g * 8 + 2 * t + 1] * sD, fg[0], fg[1]);
    pieces(D[(2 * t) * 8 + g] * sD, D[(2 * t + 1) * 8 + g] * sD, ft[0], ft[1]);

    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        // the CTA's last element: a dependent launch may start taking SMs
        if (e + gridDim.x >= E) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();   // every thread's chunks of this element have landed

        // ---- A: u -> scale -> pieces (nodes k = 2w + h, j = g, i = 2t, 2t + 1)
        float2 uv[2];
        unsigned m = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uv[h] = *reinterpret_cast<const float2 *>(su + (2 * warp + h) * 64 + g * 8 + 2 * t);
            m = max(m, max(absbits(uv[h].x), absbits(uv[h].y)));
        }
        m = __reduce_max_sync(0xffffffffu, m);
        if (lane == 0) sred[warp] = m;
        __syncthreads();
        const float sU = inv_pow2_of(max(max(sred[0], sred[1]), max(sred[2], sred[3])));
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t p0, p1;
            pieces(uv[h].x * sU, uv[h].y * sU, p0, p1);
            unsigned char *p = pc + prow(2 * warp + h, g) + 4 * t;
            *reinterpret_cast<uint32_t *>(p) = p0;
            *reinterpret_cast<uint32_t *>(p + kSlice) = p1;
        }
        __syncwarp();   // the r- and s-contractions read only this warp's planes

        // ---- B: gradient on tensor cores
        float ur[4];
        {
            uint32_t a[2][2];
            load_a<0>(pc_s, warp, lane, a);
            mma3(ur, a, fg);
        }
        {
            uint32_t a[2][2];
            float acc[4];
            load_a<1>(pc_s, warp, lane, a);
            mma3(acc, a, fg);
            // rows (k = 2w + h, i = g), columns j = 2t, 2t + 1
#pragma unroll
            for (int h = 0; h < 2; ++h)
                *reinterpret_cast<float2 *>(bs + sidx(2 * warp + h, 2 * t, g)) = make_float2(acc[2 * h], acc[2 * h + 1]);
        }
        __syncthreads();   // the t-contraction reads every warp's planes
        {
            uint32_t a[2][2];
            float acc[4];
            load_a<2>(pc_s, warp, lane, a);
            mma3(acc, a, fg);
            // rows (j = 2w + h, i = g), columns k = 2t, 2t + 1
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int c = 0; c < 2; ++c) bt[tidx(2 * t + c, 2 * warp + h, g)] = acc[2 * h + c];
        }
        __syncthreads();

        // ---- C: [wr ws wt] = G [ur us ut] in FP32
        float wr[4], ws[4], wt[4];
        unsigned mrs = 0, mt = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 2 * warp + h, nb = k * 64 + g * 8 + 2 * t;
            float2 gv[6];
#pragma unroll
            for (int a = 0; a < 6; ++a) gv[a] = *reinterpret_cast<const float2 *>(sG + a * kN3 + nb);
            const float2 tv = *reinterpret_cast<const float2 *>(bt + tidx(k, g, 2 * t));
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int q = 2 * h + c;
                const float r = ur[q], s = bs[sidx(k, g, 2 * t + c)], tt = c ? tv.y : tv.x;
                const float grr = c ? gv[0].y : gv[0].x, grs = c ? gv[1].y : gv[1].x, grt = c ? gv[2].y : gv[2].x;
                const float gss = c ? gv[3].y : gv[3].x, gst = c ? gv[4].y : gv[4].x, gtt = c ? gv[5].y : gv[5].x;
                wr[q] = __fmaf_rn(grt, tt, __fmaf_rn(grs, s, grr * r));
                ws[q] = __fmaf_rn(gst, tt, __fmaf_rn(gss, s, grs * r));
                wt[q] = __fmaf_rn(gtt, tt, __fmaf_rn(gst, s, grt * r));
                mrs = max(mrs, max(absbits(wr[q]), absbits(ws[q])));
                mt = max(mt, absbits(wt[q]));
            }
        }
        mrs = __reduce_max_sync(0xffffffffu, mrs);
        mt = __reduce_max_sync(0xffffffffu, mt);
        if (lane == 0) sred[4 + warp] = mt;
        __syncthreads();   // every thread has read this element's u and G, and ut
        if (e + gridDim.x < E) prefetch(e + gridDim.x);
        const float sRS = inv_pow2_of(mrs);   // the warp's scale of wr and ws
        const float sT = inv_pow2_of(max(max(sred[4], sred[5]), max(sred[6], sred[7])));   // the element's, of wt
        // pieces of wr (A fragments) and ws (B fragments, transposed by movmatrix)
        // in registers; of wt in the piece planes
        uint32_t yr[2][2], ys[2][2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            pieces(wr[2 * h] * sRS, wr[2 * h + 1] * sRS, yr[0][h], yr[1][h]);
            uint32_t s0, s1, t0, t1;
            pieces(ws[2 * h] * sRS, ws[2 * h + 1] * sRS, s0, s1);
            ys[0][h] = mma::movm_t(s0);
            ys[1][h] = mma::movm_t(s1);
            pieces(wt[2 * h] * sT, wt[2 * h + 1] * sT, t0, t1);
            unsigned char *p = pc + prow(2 * warp + h, g) + 4 * t;
            *reinterpret_cast<uint32_t *>(p) = t0;
            *reinterpret_cast<uint32_t *>(p + kSlice) = t1;
        }

        // ---- D: w_r + w_s in one accumulator; the s-part through the
        // block-diagonal A = diag(D^T, D^T) (K = (plane, l)) and the B fragments
        // of y_s's two planes: rows (k, j), columns i, the r-part's layout
        float acc[4];
        mma3(acc, yr, ft);
        mma::f16_16816(acc, ft[0], 0u, 0u, ft[0], ys[0][0], ys[0][1]);
        mma::f16_16816(acc, ft[0], 0u, 0u, ft[0], ys[1][0], ys[1][1]);
        mma::f16_16816(acc, ft[1], 0u, 0u, ft[1], ys[0][0], ys[0][1]);
        __syncthreads();   // wt's pieces of every warp
        {
            uint32_t a[2][2];
            float acct[4];
            load_a<2>(pc_s, warp, lane, a);
            mma3(acct, a, ft);
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int c = 0; c < 2; ++c) bt[tidx(2 * t + c, 2 * warp + h, g)] = acct[2 * h + c];
        }
        __syncthreads();

        // ---- E: w = (w_rs / sRS + w_t / sT) / (sU sD^2), times the element's G scale
        const float invRS = __frcp_rn(sRS), invT = __frcp_rn(sT);
        const float outsc = (scale ? scale[e] : 1.0f) * __frcp_rn(sU * sD * sD);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 2 * warp + h, nb = k * 64 + g * 8 + 2 * t;
            const float2 tw = *reinterpret_cast<const float2 *>(bt + tidx(k, g, 2 * t));
            float2 o;
            o.x = __fmaf_rn(tw.x, invT, acc[2 * h] * invRS) * outsc;
            o.y = __fmaf_rn(tw.y, invT, acc[2 * h + 1] * invRS) * outsc;
            *reinterpret_cast<float2 *>(w + e * kN3 + nb) = o;
        }
    }
}

}  // namespace f16n8

int launch_f16x3_n8(int64_t E, const float *u, const float *G, const float *D, float *w, const float *scale,
                    cudaStream_t s) {
    auto kern = f16n8::ax_f16x3_n8_kernel;
    int st = cuda_status(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f16n8::kSmem));
    if (st != SEMAX_OK) return st;
    st = cuda_status(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          (int)cudaSharedmemCarveoutMaxShared));
    if (st != SEMAX_OK) return st;
    int per_sm = 0;
    st = cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, f16n8::kThreads, f16n8::kSmem));
    if (st != SEMAX_OK) return st;
    const int64_t grid = std::min<int64_t>(E, (int64_t)device_sm_count() * std::max(per_sm, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(f16n8::kThreads);
    cfg.dynamicSmemBytes = f16n8::kSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];   // a programmatic dependent of the previous kernel in the stream
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    st = cuda_status(cudaLaunchKernelEx(&cfg, kern, E, u, G, D, w, scale));
    if (st != SEMAX_OK) return st;
    return launch_status();
}

}  // namespace semax
