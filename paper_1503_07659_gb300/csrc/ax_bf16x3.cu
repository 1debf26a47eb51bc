// Ax with FP32 storage and the six derivative contractions on tensor cores:
// every FP32 operand x is split into BF16 pieces x0 = bf16(x),
// x1 = bf16(x - x0) (, x2 = bf16(x - x0 - x1)), and a product x*y is formed
// from the piece products with index sum <= NP-1 (3 products for NP = 2,
// 6 for NP = 3), accumulated in FP32 by mma.m16n8k16.  The geometric-factor
// multiply runs in FP32.  Order n = 16 (N = 15).
//
// Each contraction is a dense (16 x 16) x (16 x 16) product per plane of the
// element (the (n x n) x (n x n^2) form); the paper's Section 5.2 blocks a
// matrix-matrix product with on-chip prefetch of both operand tiles, which is
// the prior art for staging u_e and the intermediates here.
//
// Per element, one CTA of 8 warps:
//   load   u (FP32, prefetched with cp.async into the piece region while the
//          previous element's pass T' runs) -> BF16 pieces in shared memory (XOR
//          swizzled so that every ldmatrix and fragment store is free of bank
//          conflicts along both the j and the k axis);
//   pass T ut = D (x) I (x) I u: warp w owns rows j = 2w, 2w+1, output
//          tile (k x i); ut -> FP32 shared buffer W;
//   pass P warp w owns planes k = 2w, 2w+1, output tile (j x i):
//          ur = u_k D^T and us = D u_k on tensor cores, ut read from W, G
//          loaded from global memory, [wr ws wt] = G [ur us ut] in FP32;
//          wt -> BF16 pieces in shared memory; wr re-enters as an A operand
//          directly from the accumulator registers; ws as a B operand after a
//          movmatrix transpose; w_rs = wr D + D^T ws -> W (same plane);
//   pass T' warp w owns rows j again: w_t = D^T (x) I (x) I wt on tensor cores,
//          w = (w_rs + w_t) * s_e, stored to global memory.
//
// FP16 pieces (F16 = true, 3 products): FP16 keeps 11 significant bits per
// piece against BF16's 8, so two pieces hold ~22 bits, but its exponent range
// is narrow.  Every operand is therefore scaled by a power of two first (an
// exact operation): u and wt per element, D once, and wr, ws per plane (their
// contractions stay inside the plane), each so that its largest magnitude
// lies in [1, 2); the scales are undone on the outputs.  Values more than
// 2^-24 below their scale's maximum keep an absolute accuracy of 2^-25 of
// it (FP16 subnormals).  wt is kept raw in FP32 until every plane's maximum
// is known and split when pass T' loads it.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "mma_sync.cuh"

namespace semax {
namespace tc {

constexpr int kN = 16;
constexpr int kThreads = 256;
constexpr int kPieceBytes = 4096 * 2;      // one BF16 copy of an element
constexpr int kWRow = 24, kWPlane = 392;   // padded FP32 plane (words)
constexpr int kWBytes = kN * kWPlane * 4;
constexpr int kRawPlane = 260;             // FP16 pieces: raw FP32 wt [l][j][i], padded plane (words)
// bytes of the wt region: its pieces, or raw FP32 wt for the FP16 pieces
template <int NP, bool F16>
constexpr int wt_bytes() { return F16 ? kN * kRawPlane * 4 : NP * kPieceBytes; }

// byte offset of BF16 element (k, j, i) inside one piece buffer
__device__ __forceinline__ uint32_t swz(int k, int j, int i) {
    const int c = i >> 3;
    const int line = (k << 2) | (j >> 2);
    const int local = ((j & 3) << 1) | c;
    const int s = (k & 7) ^ ((j >> 2) & 1);
    return (uint32_t)((((line << 3) | (local ^ s)) << 4) + ((i & 7) << 1));
}

__device__ __forceinline__ int widx(int k, int j, int i) { return k * kWPlane + j * kWRow + i; }

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return mma::smem_u32(p); }
__device__ __forceinline__ void ldsm_x4(uint32_t a, uint32_t (&r)[4]) { mma::ldsm_x4(a, r[0], r[1], r[2], r[3]); }
__device__ __forceinline__ void ldsm_x4_t(uint32_t a, uint32_t (&r)[4]) { mma::ldsm_x4_t(a, r[0], r[1], r[2], r[3]); }
using mma::movm_t;
template <bool F16>
__device__ __forceinline__ void mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    if (F16)
        mma::f16_16816(c, a[0], a[1], a[2], a[3], b0, b1);
    else
        mma::bf16_16816(c, a[0], a[1], a[2], a[3], b0, b1);
}

__device__ __forceinline__ uint32_t pack(__nv_bfloat162 h) { return *reinterpret_cast<uint32_t *>(&h); }
__device__ __forceinline__ uint32_t pack(__half2 h) { return *reinterpret_cast<uint32_t *>(&h); }

// Split the pair (x, y) into NP BF16 (F16: FP16) pieces, packed (x in the low half).
template <int NP, bool F16 = false>
__device__ __forceinline__ void split2(float x, float y, uint32_t (&out)[NP]) {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        if (F16) {
            const __half2 h = __floats2half2_rn(x, y);
            out[p] = pack(h);
            x -= __low2float(h);
            y -= __high2float(h);
        } else {
            const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
            out[p] = pack(h);
            x -= __low2float(h);
            y -= __high2float(h);
        }
    }
}

// 2^-e for the largest magnitude m of a group (as float bits), e its
// exponent, so that the group scaled by it lies below 2 in magnitude:
// clamped to [2^-126, 2^127] (a zero group keeps any scale).
__device__ __forceinline__ float inv_pow2_of(unsigned mbits) {
    const int eb = (int)((mbits >> 23) & 0xffu);
    return __uint_as_float((unsigned)min(max(254 - eb, 1), 254) << 23);
}

// piece p of a scalar (for the constant D fragments)
template <int NP, bool F16 = false>
__device__ __forceinline__ uint32_t piece_pair(float x, float y, int p) {
    uint32_t o[NP];
    split2<NP, F16>(x, y, o);
    uint32_t r = o[0];
#pragma unroll
    for (int q = 1; q < NP; ++q)
        if (q == p) r = o[q];
    return r;
}

// acc += sum over piece pairs (pa, pb), pa + pb <= NP - 1, smallest first
template <int NP, bool F16>
__device__ __forceinline__ void mma_split(float (&c)[4], const uint32_t (&a)[NP][4],
                                          const uint32_t (&b)[NP][2]) {
#pragma unroll
    for (int s = NP - 1; s >= 0; --s)
#pragma unroll
        for (int pa = s; pa >= 0; --pa) {
            const int pb = s - pa;
            mma<F16>(c, a[pa], b[pb][0], b[pb][1]);
        }
}

template <int NP>
struct DFrag {
    uint32_t AD[NP][4];      // A(r, c) = D[r][c]
    uint32_t ADt[NP][4];     // A(r, c) = D[c][r]
    uint32_t BD[NP][2][2];   // B(l, i) = D[i][l], per n-tile
    uint32_t BDt[NP][2][2];  // B(l, i) = D[l][i], per n-tile
};

// The D fragments, of D * sD (sD = 1 for BF16; for FP16 the power of two
// that puts max |D sD| in [1, 2), returned).
template <int NP, bool F16>
__device__ __forceinline__ float load_dfrag(const float *__restrict__ D, DFrag<NP> &f) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float sD = 1.0f;
    if (F16) {
        unsigned m = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) m = max(m, __float_as_uint(D[lane + 32 * q]) & 0x7fffffffu);
        sD = inv_pow2_of(__reduce_max_sync(0xffffffffu, m));
    }
    auto d = [&](int r, int c) { return D[r * kN + c] * sD; };
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        f.AD[p][0] = piece_pair<NP, F16>(d(g, 2 * t), d(g, 2 * t + 1), p);
        f.AD[p][1] = piece_pair<NP, F16>(d(g + 8, 2 * t), d(g + 8, 2 * t + 1), p);
        f.AD[p][2] = piece_pair<NP, F16>(d(g, 2 * t + 8), d(g, 2 * t + 9), p);
        f.AD[p][3] = piece_pair<NP, F16>(d(g + 8, 2 * t + 8), d(g + 8, 2 * t + 9), p);
        f.ADt[p][0] = piece_pair<NP, F16>(d(2 * t, g), d(2 * t + 1, g), p);
        f.ADt[p][1] = piece_pair<NP, F16>(d(2 * t, g + 8), d(2 * t + 1, g + 8), p);
        f.ADt[p][2] = piece_pair<NP, F16>(d(2 * t + 8, g), d(2 * t + 9, g), p);
        f.ADt[p][3] = piece_pair<NP, F16>(d(2 * t + 8, g + 8), d(2 * t + 9, g + 8), p);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int i = g + 8 * nt;
            f.BD[p][nt][0] = piece_pair<NP, F16>(d(i, 2 * t), d(i, 2 * t + 1), p);
            f.BD[p][nt][1] = piece_pair<NP, F16>(d(i, 2 * t + 8), d(i, 2 * t + 9), p);
            f.BDt[p][nt][0] = piece_pair<NP, F16>(d(2 * t, i), d(2 * t + 1, i), p);
            f.BDt[p][nt][1] = piece_pair<NP, F16>(d(2 * t + 8, i), d(2 * t + 9, i), p);
        }
    }
    return sD;
}

// G = wq adj(J) adj(J)^T / det(J), components (rr, rs, rt, ss, st, tt), for
// the Jacobian J[c][d] = dx_c / dxi_d of an element's trilinear map at one
// node (the map x_c = sum_m a[c][m] mono_m(r, s, t) over the monomials
// (1, r, s, t, rs, rt, st, rst) is evaluated by the caller).  FP32.
__device__ __forceinline__ void geo_from_jacobian(const float (&J)[3][3], float wq, float (&G6)[6]) {
    const float A = J[0][0], B = J[0][1], C = J[0][2];
    const float Dd = J[1][0], Ee = J[1][1], F = J[1][2];
    const float Gg = J[2][0], H = J[2][1], I = J[2][2];
    const float adj[3][3] = {{Ee * I - F * H, C * H - B * I, B * F - C * Ee},
                             {F * Gg - Dd * I, A * I - C * Gg, C * Dd - A * F},
                             {Dd * H - Ee * Gg, B * Gg - A * H, A * Ee - B * Dd}};
    const float det = A * adj[0][0] + B * adj[1][0] + C * adj[2][0];
    const float sc = wq * __frcp_rn(det);
    int m = 0;
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = p; q < 3; ++q)
            G6[m++] = sc * (adj[p][0] * adj[q][0] + adj[p][1] * adj[q][1] + adj[p][2] * adj[q][2]);
}

// GEO = false: G is the stored [E][6][16][16][16] factor.
// GEO = true:  G is the element vertices [E][8][3] (FP32) and xq = (GLL nodes
// [16], GLL weights [16]); the factor is recomputed at every node from the
// trilinear map (96 bytes per element read instead of 96 KB).
template <int NP, bool GEO, bool F16>
__global__ void __launch_bounds__(kThreads, 2)
ax_bf16_kernel(int64_t E, const float *__restrict__ u, const float *__restrict__ G,
               const float *__restrict__ D, float *__restrict__ w, const float *__restrict__ scale,
               const float *__restrict__ xq) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *upc = smem;                                // NP pieces of u
    unsigned char *wpc = smem + NP * kPieceBytes;             // NP pieces of wt (F16: raw FP32 wt)
    float *wraw = reinterpret_cast<float *>(wpc);
    float *W = reinterpret_cast<float *>(smem + NP * kPieceBytes + wt_bytes<NP, F16>());
    float *sgeo = W + kWBytes / 4;                            // GEO: map coefficients [3][8], xi [16], wq [16]
    unsigned *smax = reinterpret_cast<unsigned *>(W + kWBytes / 4);   // F16: per-warp maxima of |u| and |wt|
    const uint32_t upc_s = smem_addr(upc), wpc_s = smem_addr(wpc);
    // launched as a programmatic dependent of the previous kernel in the
    // stream: no global memory is read before that kernel has completed
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (GEO && threadIdx.x < 32) sgeo[24 + threadIdx.x] = xq[threadIdx.x];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int lm = lane >> 3, lr = lane & 7;  // ldmatrix: matrix id, row id

    DFrag<NP> f;
    const float sD = load_dfrag<NP, F16>(D, f);

    // u of the CTA's first element, raw FP32, into the u-piece region: each
    // thread copies (and later reads back) its own four 16-byte chunks
    const unsigned raw_s = smem_addr(upc);
    auto prefetch_u = [&](int64_t ep) {
        const char *src = reinterpret_cast<const char *>(u + ep * 4096);
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            const int q = tid + it * kThreads;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(raw_s + 16 * q), "l"(src + 16 * q));
        }
        asm volatile("cp.async.commit_group;" ::);
    };
    if (blockIdx.x < E) prefetch_u(blockIdx.x);

    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        const float *Ge = G + e * (GEO ? 24 : 6 * 4096);
        // the CTA's last element: a dependent launch may start taking SMs
        if (e + gridDim.x >= E) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        // the element's stored G into L2 ahead of pass P (three 128-byte lines
        // per thread); two-piece forms only, the three-piece form measured slower
        if (!GEO && NP == 2) {
            const char *src = reinterpret_cast<const char *>(Ge);
#pragma unroll
            for (int it = 0; it < 3; ++it)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(src + 128 * (tid + it * kThreads)));
        }
        float *we = w + e * 4096;
        if (GEO && tid < 24) {   // trilinear map coefficients of this element
            const int c = tid >> 3, m = tid & 7;
            float acc = 0.f;
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const float sr = (v & 1) ? 1.f : -1.f, ss = (v & 2) ? 1.f : -1.f, st = (v & 4) ? 1.f : -1.f;
                const float b = m == 0 ? 1.f : m == 1 ? sr : m == 2 ? ss : m == 3 ? st
                              : m == 4 ? sr * ss : m == 5 ? sr * st : m == 6 ? ss * st : sr * ss * st;
                acc = __fmaf_rn(b, Ge[3 * v + c], acc);
            }
            sgeo[8 * c + m] = 0.125f * acc;
        }

        // ---- u (prefetched raw into the piece region), split into pieces
        asm volatile("cp.async.wait_all;" ::: "memory");
        float4 vr[4];
#pragma unroll
        for (int it = 0; it < 4; ++it) vr[it] = reinterpret_cast<const float4 *>(upc)[tid + it * kThreads];
        if (F16) {   // the element's largest |u|, per warp
            unsigned m = 0;
#pragma unroll
            for (int it = 0; it < 4; ++it)
                m = max(max(m, max(__float_as_uint(vr[it].x), __float_as_uint(vr[it].y)) & 0x7fffffffu),
                        max(__float_as_uint(vr[it].z), __float_as_uint(vr[it].w)) & 0x7fffffffu);
            m = __reduce_max_sync(0xffffffffu, m);
            if (lane == 0) smax[warp] = m;
        }
        __syncthreads();   // every thread has its raw values before pieces overwrite the region
        float su = 1.0f;   // F16: u's power-of-two scale
        if (F16) {
            unsigned m = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) m = max(m, smax[q]);
            su = inv_pow2_of(m);
        }
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            const int q = tid + it * kThreads;  // float4 index, 0..1023
            const float4 v = vr[it];
            const int k = q >> 6, j = (q >> 2) & 15, i = (q & 3) << 2;
            uint32_t lo[NP], hi[NP];
            split2<NP, F16>(v.x * su, v.y * su, lo);
            split2<NP, F16>(v.z * su, v.w * su, hi);
            const uint32_t off = swz(k, j, i);
#pragma unroll
            for (int p = 0; p < NP; ++p)
                *reinterpret_cast<uint2 *>(upc + p * kPieceBytes + off) = make_uint2(lo[p], hi[p]);
        }
        __syncthreads();

        // ---- pass T: ut[k][j][i] = sum_l D[k][l] u[l][j][i]
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
            const int j = 2 * warp + jj;
            uint32_t b[NP][4];
            const uint32_t a_off = swz(lr + 8 * (lm & 1), j, 8 * (lm >> 1));
#pragma unroll
            for (int p = 0; p < NP; ++p) ldsm_x4_t(upc_s + p * kPieceBytes + a_off, b[p]);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                uint32_t bb[NP][2];
#pragma unroll
                for (int p = 0; p < NP; ++p) { bb[p][0] = b[p][2 * nt]; bb[p][1] = b[p][2 * nt + 1]; }
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                mma_split<NP, F16>(c, f.AD, bb);
                const int i = 8 * nt + 2 * t;
                *reinterpret_cast<float2 *>(W + widx(g, j, i)) = make_float2(c[0], c[1]);
                *reinterpret_cast<float2 *>(W + widx(g + 8, j, i)) = make_float2(c[2], c[3]);
            }
        }
        __syncthreads();

        // ---- pass P: planes k = 2*warp, 2*warp+1
        unsigned tmax = 0;   // F16: the warp's largest |wt| (float bits)
#pragma unroll 1
        for (int kk = 0; kk < 2; ++kk) {
            const int k = 2 * warp + kk;
            // geometric factors of this thread's 8 nodes (2 n-tiles x 2 row halves)
            float2 gv[6][2][2];
            if constexpr (GEO) {
                // Along a line of fixed (s, t) = (xi_j, xi_k), dx/dr is constant and
                // dx/ds, dx/dt are linear in r: 15 line constants serve 4 nodes.
                const float tk = sgeo[24 + k], wk = sgeo[40 + k];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = g + 8 * h;
                    const float sj = sgeo[24 + j], wjk = sgeo[40 + j] * wk;
                    float j0[3], j1a[3], j1b[3], j2a[3], j2b[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float *ac = sgeo + 8 * c;
                        j0[c] = __fmaf_rn(ac[7], sj * tk, __fmaf_rn(ac[5], tk, __fmaf_rn(ac[4], sj, ac[1])));
                        j1a[c] = __fmaf_rn(ac[6], tk, ac[2]);
                        j1b[c] = __fmaf_rn(ac[7], tk, ac[4]);
                        j2a[c] = __fmaf_rn(ac[6], sj, ac[3]);
                        j2b[c] = __fmaf_rn(ac[7], sj, ac[5]);
                    }
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) {
                        float gg[2][6];
#pragma unroll
                        for (int x = 0; x < 2; ++x) {
                            const int i = 8 * nt + 2 * t + x;
                            const float r = sgeo[24 + i];
                            float J[3][3];
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                J[c][0] = j0[c];
                                J[c][1] = __fmaf_rn(j1b[c], r, j1a[c]);
                                J[c][2] = __fmaf_rn(j2b[c], r, j2a[c]);
                            }
                            geo_from_jacobian(J, sgeo[40 + i] * wjk, gg[x]);
                        }
#pragma unroll
                        for (int comp = 0; comp < 6; ++comp) gv[comp][nt][h] = make_float2(gg[0][comp], gg[1][comp]);
                    }
                }
            } else {
#pragma unroll
                for (int comp = 0; comp < 6; ++comp)
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float *p = Ge + comp * 4096 + k * 256 + (g + 8 * h) * 16 + 8 * nt + 2 * t;
                            float2 v;
                            asm volatile("ld.global.nc.L1::no_allocate.v2.f32 {%0,%1}, [%2];"
                                         : "=f"(v.x), "=f"(v.y) : "l"(p));
                            gv[comp][nt][h] = v;
                        }
            }
            uint32_t au[NP][4], bu[NP][4];
            const uint32_t off = swz(k, lr + 8 * (lm & 1), 8 * (lm >> 1));
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                ldsm_x4(upc_s + p * kPieceBytes + off, au[p]);
                ldsm_x4_t(upc_s + p * kPieceBytes + off, bu[p]);
            }
            float wacc[2][4];
            uint32_t awr[NP][4];   // wr as A operand (C -> A reuse)
            uint32_t bws[NP][2][2];
            float wrv[2][4], wsv[2][4];   // F16: wr, ws of the plane until its scale is known
            unsigned pmax = 0;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                float ur[4] = {0.f, 0.f, 0.f, 0.f}, us[4] = {0.f, 0.f, 0.f, 0.f};
                uint32_t bd[NP][2], bb[NP][2];
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    bd[p][0] = f.BD[p][nt][0];
                    bd[p][1] = f.BD[p][nt][1];
                    bb[p][0] = bu[p][2 * nt];
                    bb[p][1] = bu[p][2 * nt + 1];
                }
                // ur: A = u_k (rows j, cols l), B = D^T; us: A = D, B = u_k (rows l, cols i)
#pragma unroll
                for (int s = NP - 1; s >= 0; --s)
#pragma unroll
                    for (int pa = s; pa >= 0; --pa) mma<F16>(ur, au[s - pa], bd[pa][0], bd[pa][1]);
                mma_split<NP, F16>(us, f.AD, bb);
                const int i = 8 * nt + 2 * t;
                float wr[4], ws[4], wt[4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 ut2 = *reinterpret_cast<const float2 *>(W + widx(k, g + 8 * h, i));
                    const float utv[2] = {ut2.x, ut2.y};
#pragma unroll
                    for (int x = 0; x < 2; ++x) {
                        const int q = 2 * h + x;
                        const float grr = x ? gv[0][nt][h].y : gv[0][nt][h].x;
                        const float grs = x ? gv[1][nt][h].y : gv[1][nt][h].x;
                        const float grt = x ? gv[2][nt][h].y : gv[2][nt][h].x;
                        const float gss = x ? gv[3][nt][h].y : gv[3][nt][h].x;
                        const float gst = x ? gv[4][nt][h].y : gv[4][nt][h].x;
                        const float gtt = x ? gv[5][nt][h].y : gv[5][nt][h].x;
                        const float r = ur[q], s = us[q], tt = utv[x];
                        wr[q] = __fmaf_rn(grt, tt, __fmaf_rn(grs, s, grr * r));
                        ws[q] = __fmaf_rn(gst, tt, __fmaf_rn(gss, s, grs * r));
                        wt[q] = __fmaf_rn(gtt, tt, __fmaf_rn(gst, s, grt * r));
                    }
                }
                if (F16) {
                    // wt raw (FP32) -> shared, split in pass T' once every plane's
                    // maximum is known; wr and ws wait for the plane's scale
                    *reinterpret_cast<float2 *>(wraw + k * kRawPlane + g * kN + i) = make_float2(wt[0], wt[1]);
                    *reinterpret_cast<float2 *>(wraw + k * kRawPlane + (g + 8) * kN + i) = make_float2(wt[2], wt[3]);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        tmax = max(tmax, __float_as_uint(wt[q]) & 0x7fffffffu);
                        pmax = max(pmax, max(__float_as_uint(wr[q]), __float_as_uint(ws[q])) & 0x7fffffffu);
                        wrv[nt][q] = wr[q];
                        wsv[nt][q] = ws[q];
                    }
                    continue;
                }
                // wt pieces -> shared (for pass T')
                uint32_t p0[NP], p1[NP];
                split2<NP>(wt[0], wt[1], p0);
                split2<NP>(wt[2], wt[3], p1);
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    *reinterpret_cast<uint32_t *>(wpc + p * kPieceBytes + swz(k, g, i)) = p0[p];
                    *reinterpret_cast<uint32_t *>(wpc + p * kPieceBytes + swz(k, g + 8, i)) = p1[p];
                }
                // wr pieces as A fragment columns 8*nt..8*nt+7
                split2<NP>(wr[0], wr[1], p0);
                split2<NP>(wr[2], wr[3], p1);
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    awr[p][2 * nt] = p0[p];
                    awr[p][2 * nt + 1] = p1[p];
                }
                // ws pieces, transposed 8x8 blocks -> B fragment of n-tile nt
                split2<NP>(ws[0], ws[1], p0);
                split2<NP>(ws[2], ws[3], p1);
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    bws[p][nt][0] = movm_t(p0[p]);
                    bws[p][nt][1] = movm_t(p1[p]);
                }
            }
            float inv_sk = 1.0f;   // F16: undoes the plane's scale on w_rs
            if (F16) {
                const float sk = inv_pow2_of(__reduce_max_sync(0xffffffffu, pmax));
                inv_sk = __frcp_rn(sk);
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    uint32_t p0[NP], p1[NP];
                    split2<NP, true>(wrv[nt][0] * sk, wrv[nt][1] * sk, p0);
                    split2<NP, true>(wrv[nt][2] * sk, wrv[nt][3] * sk, p1);
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        awr[p][2 * nt] = p0[p];
                        awr[p][2 * nt + 1] = p1[p];
                    }
                    split2<NP, true>(wsv[nt][0] * sk, wsv[nt][1] * sk, p0);
                    split2<NP, true>(wsv[nt][2] * sk, wsv[nt][3] * sk, p1);
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        bws[p][nt][0] = movm_t(p0[p]);
                        bws[p][nt][1] = movm_t(p1[p]);
                    }
                }
            }
            // w_rs = wr D + D^T ws
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                wacc[nt][0] = wacc[nt][1] = wacc[nt][2] = wacc[nt][3] = 0.f;
                uint32_t bdt[NP][2], bw[NP][2];
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    bdt[p][0] = f.BDt[p][nt][0];
                    bdt[p][1] = f.BDt[p][nt][1];
                    bw[p][0] = bws[p][nt][0];
                    bw[p][1] = bws[p][nt][1];
                }
                mma_split<NP, F16>(wacc[nt], awr, bdt);
                mma_split<NP, F16>(wacc[nt], f.ADt, bw);
                const int i = 8 * nt + 2 * t;
                *reinterpret_cast<float2 *>(W + widx(k, g, i)) = make_float2(wacc[nt][0] * inv_sk, wacc[nt][1] * inv_sk);
                *reinterpret_cast<float2 *>(W + widx(k, g + 8, i)) = make_float2(wacc[nt][2] * inv_sk, wacc[nt][3] * inv_sk);
            }
        }
        if (F16) {
            tmax = __reduce_max_sync(0xffffffffu, tmax);
            if (lane == 0) smax[8 + warp] = tmax;
        }
        __syncthreads();
        if (e + gridDim.x < E) prefetch_u(e + gridDim.x);   // the u pieces are dead from here on

        // ---- pass T': w += sum_l D[l][k] wt[l][j][i]; store
        float sc = scale ? scale[e] : 1.f;
        float st = 1.0f, inv_st = 1.0f;   // F16: wt's scale, and its inverse
        if (F16) {
            unsigned m = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) m = max(m, smax[8 + q]);
            st = inv_pow2_of(m);
            inv_st = __frcp_rn(st);
            sc = sc * __frcp_rn(su * sD * sD);   // W and the t-part are in units of su sD^2
        }
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
            const int j = 2 * warp + jj;
            uint32_t b[NP][4];
            if (F16) {   // B fragments (rows l = 2t, 2t+1 (+8), column i = g (+8)) split from the raw wt
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int kh = 0; kh < 2; ++kh) {
                        const int l = 2 * t + 8 * kh, i = 8 * nt + g;
                        uint32_t pc[NP];
                        split2<NP, true>(wraw[l * kRawPlane + j * kN + i] * st, wraw[(l + 1) * kRawPlane + j * kN + i] * st,
                                         pc);
#pragma unroll
                        for (int p = 0; p < NP; ++p) b[p][2 * nt + kh] = pc[p];
                    }
            } else {
                const uint32_t a_off = swz(lr + 8 * (lm & 1), j, 8 * (lm >> 1));
#pragma unroll
                for (int p = 0; p < NP; ++p) ldsm_x4_t(wpc_s + p * kPieceBytes + a_off, b[p]);
            }
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                uint32_t bb[NP][2];
#pragma unroll
                for (int p = 0; p < NP; ++p) { bb[p][0] = b[p][2 * nt]; bb[p][1] = b[p][2 * nt + 1]; }
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                mma_split<NP, F16>(c, f.ADt, bb);
                const int i = 8 * nt + 2 * t;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = g + 8 * h;
                    const float2 prev = *reinterpret_cast<const float2 *>(W + widx(k, j, i));
                    float2 out = F16 ? make_float2(__fmaf_rn(c[2 * h], inv_st, prev.x) * sc,
                                                   __fmaf_rn(c[2 * h + 1], inv_st, prev.y) * sc)
                                     : make_float2((prev.x + c[2 * h]) * sc, (prev.y + c[2 * h + 1]) * sc);
                    *reinterpret_cast<float2 *>(we + k * 256 + j * 16 + i) = out;
                }
            }
        }
        __syncthreads();
    }
}

template <int NP, bool GEO, bool F16 = false>
static int launch(int64_t E, const float *u, const float *G, const float *D, float *w, const float *scale,
                  const float *xq, cudaStream_t s) {
    const size_t smem = NP * kPieceBytes + wt_bytes<NP, F16>() + kWBytes + (GEO ? 64 * sizeof(float) : 0) +
                        (F16 ? 16 * sizeof(unsigned) : 0);
    auto kern = ax_bf16_kernel<NP, GEO, F16>;
    int st = cuda_status(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (st != SEMAX_OK) return st;
    int per_sm = 0;
    st = cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    if (st != SEMAX_OK) return st;
    if (per_sm < 1) return SEMAX_EINVAL;
    int64_t grid = (int64_t)per_sm * device_sm_count();
    if (grid > E) grid = E;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];   // a programmatic dependent of the previous kernel in the stream
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    st = cuda_status(cudaLaunchKernelEx(&cfg, kern, E, u, G, D, w, scale, xq));
    if (st != SEMAX_OK) return st;
    return launch_status();
}

}  // namespace tc
}  // namespace semax

using namespace semax;

extern "C" int sem_ax_bf16x3(int64_t E, int N, const float *u, const float *G, const float *D, float *w,
                             const float *G_scale, int terms, void *stream) {
    if (terms != 3 && terms != 6) return SEMAX_EINVAL;
    int st = check_args(E, N, u, G, D, w);
    if (st != SEMAX_OK || E == 0) return st;
    if (N != 15) return SEMAX_EUNSUPPORTED_N;
    if (G_scale && overlaps(w, (size_t)E * 4096 * sizeof(float), G_scale, (size_t)E * sizeof(float)))
        return SEMAX_EALIAS;
    if (terms == 3) return tc::launch<2, false>(E, u, G, D, w, G_scale, nullptr, (cudaStream_t)stream);
    return tc::launch<3, false>(E, u, G, D, w, G_scale, nullptr, (cudaStream_t)stream);
}

namespace semax {
int launch_f16x3_n8(int64_t E, const float *u, const float *G, const float *D, float *w, const float *scale,
                    cudaStream_t s);
}

extern "C" int sem_ax_f16x3(int64_t E, int N, const float *u, const float *G, const float *D, float *w,
                            const float *G_scale, void *stream) {
    int st = check_args(E, N, u, G, D, w);
    if (st != SEMAX_OK || E == 0) return st;
    if (N != 7 && N != 15) return SEMAX_EUNSUPPORTED_N;
    if (N == 7) {
        if (G_scale && overlaps(w, (size_t)E * 512 * sizeof(float), G_scale, (size_t)E * sizeof(float)))
            return SEMAX_EALIAS;
        return launch_f16x3_n8(E, u, G, D, w, G_scale, (cudaStream_t)stream);
    }
    if (G_scale && overlaps(w, (size_t)E * 4096 * sizeof(float), G_scale, (size_t)E * sizeof(float)))
        return SEMAX_EALIAS;
    return tc::launch<2, false, true>(E, u, G, D, w, G_scale, nullptr, (cudaStream_t)stream);
}

extern "C" int sem_ax_bf16x3_geo(int64_t E, int N, const float *u, const float *X, const float *xi_wq,
                                 const float *D, float *w, int terms, void *stream) {
    if (terms != 3 && terms != 6) return SEMAX_EINVAL;
    if (E < 0) return SEMAX_EINVAL;
    if (N < 1 || N > kMaxN) return SEMAX_EUNSUPPORTED_N;
    if (E == 0) return SEMAX_OK;
    if (!u || !X || !xi_wq || !D || !w) return SEMAX_EINVAL;
    if (N != 15) return SEMAX_EUNSUPPORTED_N;
    if (!aligned16(u) || !aligned16(w) || ((uintptr_t)X & 3u) || ((uintptr_t)xi_wq & 3u) || ((uintptr_t)D & 3u))
        return SEMAX_EALIGN;
    const size_t ub = (size_t)E * 4096 * sizeof(float);
    if (overlaps(w, ub, u, ub) || overlaps(w, ub, X, (size_t)E * 24 * sizeof(float)) ||
        overlaps(w, ub, D, 256 * sizeof(float)) || overlaps(w, ub, xi_wq, 32 * sizeof(float)))
        return SEMAX_EALIAS;
    if (terms == 3) return tc::launch<2, true>(E, u, X, D, w, nullptr, xi_wq, (cudaStream_t)stream);
    return tc::launch<3, true>(E, u, X, D, w, nullptr, xi_wq, (cudaStream_t)stream);
}
