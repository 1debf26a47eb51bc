// Element-tile device routines of the spectral-element Ax operator
// (FP64 and FP32 CUDA-core forms).
//
// One CTA processes a tile of `cnt` consecutive elements of order n-1:
//   phase 1  stage u_e (n^3 per element) in shared memory;
//   phase 2  reference gradient ur, us, ut (three length-n contractions with
//            D) and the symmetric 3x3 geometric-factor multiply, G streamed
//            from global memory once;
//   phase 3  transposed contractions with D^T, summed over r, s, t, and one
//            store of w.
// This is the sum-factorised form of w_e = sum_ab D_a^T diag(G_ab) D_b u_e
// (Deville, Fischer & Mund 2002, Sec. 4.4); the paper's Section 4.3
// `precompute` (stage an array's footprint on chip before the loops that
// reuse it) is the prior art for staging u_e and the intermediates.
//
// Three thread mappings.  MAP_NODE and MAP_COLUMN are bit-identical in their
// results (same products, same fma order per output):
//   MAP_NODE    one thread per node, grid-stride over the tile; every operand
//               from shared memory; any block size;
//   MAP_COLUMN  one thread per (i,j) column of a tile element, the column of u
//               held in registers for the t-direction; needs
//               cnt * n^2 <= blockDim.x.
//   MAP_EO      even n only: one thread per line (n nodes along one direction)
//               and the even/odd split of a centro-antisymmetric matrix M
//               (M[n-1-i][n-1-l] = -M[i][l], true of the GLL derivative and of
//               its transpose): with e_l = x_l + x_{n-1-l}, o_l = x_l - x_{n-1-l}
//               (l < n/2), P = (M[i][l] + M[i][n-1-l]) / 2 and
//               Q = (M[i][l] - M[i][n-1-l]) / 2,
//                   y_i = (Pe)_i + (Qo)_i,  y_{n-1-i} = (Qo)_i - (Pe)_i,
//               so a line costs n^2/2 + 2n operations instead of n^2.  At
//               n = 8 a node takes 47 arithmetic instructions instead of 57.
//               The tile checks D's antisymmetry bit for bit on its shared
//               copy and takes the MAP_NODE phases when it does not hold.
#pragma once

#include "common.cuh"

namespace semax {

enum { MAP_NODE = 0, MAP_COLUMN = 1, MAP_EO = 2 };

__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Slots reserved at the start of the shared buffer for D and the even/odd
// blocks P, Q of D and of D^T (4 (n/2)^2 <= n^2); keeps the tile buffers
// behind it 16-byte aligned.
template <typename T>
__host__ __device__ constexpr int d_slots(int n) { return round_up(2 * n * n, 16 / (int)sizeof(T)); }

template <typename T>
__host__ __device__ constexpr int eo_elem_pitch(int n);

// Shared-memory footprint (bytes) of D plus one tile of `epb` elements: four
// dense element buffers (u and the three directions), or for MAP_EO three
// padded ones (the t-direction reuses u's slots), at least as large as the
// four dense buffers of its fallback path.
template <typename T>
__host__ __device__ constexpr size_t tile_smem_bytes(int n, int epb, int map) {
    return sizeof(T) * ((size_t)d_slots<T>(n) +
                        (size_t)epb * (map == 2 && n % 2 == 0
                                           ? (3 * eo_elem_pitch<T>(n) > 4 * n * n * n ? 3 * eo_elem_pitch<T>(n)
                                                                                     : 4 * n * n * n)
                                           : 4 * n * n * n));
}

template <typename T>
__device__ __forceinline__ T fma_(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
template <>
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Helmholtz extension w = h1 A u + h2 B u (B the diagonal mass matrix, one
// value per node, pointing at the tile's first element); used when the tile
// routines are instantiated with HELM = true.
template <typename T>
struct Helm {
    const T *B;
    T h1, h2;
};

// Multiply by the symmetric factor: G components (rr, rs, rt, ss, st, tt).
template <typename T>
__device__ __forceinline__ void geo_multiply(const T *__restrict__ Gq, int n3, T ur, T us, T ut,
                                             T &wr, T &ws, T &wt) {
    const T grr = ld_stream(Gq), grs = ld_stream(Gq + n3), grt = ld_stream(Gq + 2 * n3);
    const T gss = ld_stream(Gq + 3 * n3), gst = ld_stream(Gq + 4 * n3), gtt = ld_stream(Gq + 5 * n3);
    wr = fma_(grt, ut, fma_(grs, us, grr * ur));
    ws = fma_(gst, ut, fma_(gss, us, grs * ur));
    wt = fma_(gtt, ut, fma_(gst, us, grt * ur));
}

// Phases 2-3 with one thread per node (MAP_NODE).
template <typename T, int n, bool HELM = false>
__device__ __forceinline__ void tile_node_phases(int cnt, const T *__restrict__ G, T *__restrict__ w,
                                                 const T *__restrict__ scale, Helm<T> helm,
                                                 const T *__restrict__ sD, const T *su, T *sr, T *ss, T *st) {
    constexpr int n2 = n * n, n3 = n * n * n;
    const int nodes = cnt * n3;
    for (int p = threadIdx.x; p < nodes; p += blockDim.x) {
        const int e = p / n3, q = p - e * n3;
        const int k = q / n2, j = (q - k * n2) / n, i = q - k * n2 - j * n;
        const T *ue = su + e * n3;
        T ur = T(0), us = T(0), ut = T(0);
#pragma unroll
        for (int l = 0; l < n; ++l) {
            ur = fma_(sD[i * n + l], ue[k * n2 + j * n + l], ur);
            us = fma_(sD[j * n + l], ue[k * n2 + l * n + i], us);
            ut = fma_(sD[k * n + l], ue[l * n2 + j * n + i], ut);
        }
        T wr, ws, wt;
        geo_multiply(G + (size_t)e * 6 * n3 + q, n3, ur, us, ut, wr, ws, wt);
        sr[p] = wr;
        ss[p] = ws;
        st[p] = wt;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < nodes; p += blockDim.x) {
        const int e = p / n3, q = p - e * n3;
        const int k = q / n2, j = (q - k * n2) / n, i = q - k * n2 - j * n;
        const T *re = sr + e * n3, *se = ss + e * n3, *te = st + e * n3;
        T acc = T(0);
#pragma unroll
        for (int l = 0; l < n; ++l) acc = fma_(sD[l * n + i], re[k * n2 + j * n + l], acc);
#pragma unroll
        for (int l = 0; l < n; ++l) acc = fma_(sD[l * n + j], se[k * n2 + l * n + i], acc);
#pragma unroll
        for (int l = 0; l < n; ++l) acc = fma_(sD[l * n + k], te[l * n2 + j * n + i], acc);
        if constexpr (HELM) acc = fma_(helm.h2 * helm.B[p], su[p], helm.h1 * acc);
        if (scale) acc *= scale[e];
        w[p] = acc;
    }
}

}  // namespace semax

#include "ax_eo.cuh"

namespace semax {

// Tile routine.  sD holds D (n x n) already, with d_slots(n) slots reserved;
// `buf` is the tile's shared scratch (tile_smem_bytes minus the D part).
// u, G and w point at element e0.
template <typename T, int n, int MAP, bool HELM = false>
__device__ __forceinline__ void ax_tile(int cnt, const T *__restrict__ u, const T *__restrict__ G,
                                        T *__restrict__ w, const T *__restrict__ scale, Helm<T> helm,
                                        T *__restrict__ sD, T *__restrict__ buf) {
    constexpr int n2 = n * n, n3 = n * n * n;
    const int nodes = cnt * n3;
    if constexpr (MAP == MAP_EO && n % 2 == 0) {
        constexpr int h = n / 2, EP = eo_elem_pitch<T>(n);
        T *su = buf;
        T *sr = su + cnt * EP;
        T *ss = sr + cnt * EP;
        eo_stage<T, n>(su, u, cnt);
        __syncthreads();   // D (loaded by the caller) and the staged u are visible
        int ok = 1;
        for (int q = threadIdx.x; q < n2; q += blockDim.x) {
            const int i = q / n, l = q - (q / n) * n;
            if (sD[q] != -sD[(n - 1 - i) * n + (n - 1 - l)]) ok = 0;
        }
        if (__syncthreads_and(ok)) {
            T *sPQ = sD + n2;
            for (int q = threadIdx.x; q < h * h; q += blockDim.x) {
                const int i = q / h, l = q - (q / h) * h;
                const T a = sD[i * n + l], b = sD[i * n + (n - 1 - l)];          // D
                const T at = sD[l * n + i], bt = sD[(n - 1 - l) * n + i];        // D^T
                sPQ[q] = T(0.5) * (a + b);
                sPQ[h * h + q] = T(0.5) * (a - b);
                sPQ[2 * h * h + q] = T(0.5) * (at + bt);
                sPQ[3 * h * h + q] = T(0.5) * (at - bt);
            }
            __syncthreads();
            tile_eo_phases<T, n, HELM>(cnt, G, w, scale, helm, sPQ, su, sr, ss);
            return;
        }
        // D is not centro-antisymmetric: dense staging and the node phases
        su = buf;
        sr = su + nodes;
        ss = sr + nodes;
        T *st = ss + nodes;
        copy_to_smem(su, u, nodes);
        __syncthreads();
        tile_node_phases<T, n, HELM>(cnt, G, w, scale, helm, sD, su, sr, ss, st);
        return;
    }
    T *su = buf;
    T *sr = su + nodes;
    T *ss = sr + nodes;
    T *st = ss + nodes;
    copy_to_smem(su, u, nodes);
    __syncthreads();

    if constexpr (MAP == MAP_COLUMN) {
        const int c = threadIdx.x;  // column id within the tile
        const bool active = c < cnt * n2;
        const int e = active ? c / n2 : 0, ji = c - e * n2;
        const int j = ji / n, i = ji - j * n;
        const T *ue = su + e * n3;
        if (active) {
            T uc[n];
#pragma unroll
            for (int l = 0; l < n; ++l) uc[l] = ue[l * n2 + ji];
#pragma unroll 1
            for (int k = 0; k < n; ++k) {
                T ur = T(0), us = T(0), ut = T(0);
#pragma unroll
                for (int l = 0; l < n; ++l) {
                    ur = fma_(sD[i * n + l], ue[k * n2 + j * n + l], ur);
                    us = fma_(sD[j * n + l], ue[k * n2 + l * n + i], us);
                    ut = fma_(sD[k * n + l], uc[l], ut);
                }
                T wr, ws, wt;
                geo_multiply(G + (size_t)e * 6 * n3 + k * n2 + ji, n3, ur, us, ut, wr, ws, wt);
                sr[e * n3 + k * n2 + ji] = wr;
                ss[e * n3 + k * n2 + ji] = ws;
                st[e * n3 + k * n2 + ji] = wt;
            }
        }
        __syncthreads();
        if (active) {
            const T *re = sr + e * n3, *se = ss + e * n3, *te = st + e * n3;
            const T sc = scale ? scale[e] : T(1);
#pragma unroll 1
            for (int k = 0; k < n; ++k) {
                T acc = T(0);
#pragma unroll
                for (int l = 0; l < n; ++l) acc = fma_(sD[l * n + i], re[k * n2 + j * n + l], acc);
#pragma unroll
                for (int l = 0; l < n; ++l) acc = fma_(sD[l * n + j], se[k * n2 + l * n + i], acc);
#pragma unroll
                for (int l = 0; l < n; ++l) acc = fma_(sD[l * n + k], te[l * n2 + ji], acc);
                if constexpr (HELM) {
                    const int q = e * n3 + k * n2 + ji;
                    acc = fma_(helm.h2 * helm.B[q], su[q], helm.h1 * acc);
                }
                if (scale) acc *= sc;
                w[(size_t)e * n3 + k * n2 + ji] = acc;
            }
        }
    } else {
        tile_node_phases<T, n, HELM>(cnt, G, w, scale, helm, sD, su, sr, ss, st);
    }
}

template <typename T, int n>
__device__ __forceinline__ void load_D(const T *__restrict__ D, T *sD) {
    for (int q = threadIdx.x; q < n * n; q += blockDim.x) sD[q] = D[q];
}

}  // namespace semax
