// MAP_EO tile phases: one thread per line, even/odd split of the
// centro-antisymmetric D (see ax_tile.cuh), on a padded shared-memory layout.
//
// Layout of one element's block in shared memory: node (k, j, i) at
// k*PP + j*RP + i.  The row pitch RP keeps rows 16-byte aligned and makes the
// 128-bit row loads of 8 consecutive lines hit 8 different 16-byte bank
// groups; the plane pitch PP shifts consecutive planes by one line width so
// that the lanes of a warp walking a column line (i fastest, then k) cover
// distinct banks.  Rows are read and written with 128-bit vectors when n is
// a multiple of the vector width, and the coefficient rows of P and Q are
// read as 128-bit broadcasts.
#pragma once

namespace semax {

template <typename T>
__host__ __device__ constexpr int eo_row_pitch(int n) {
    const int V = 16 / (int)sizeof(T);
    int rp = (n + V - 1) / V * V + V;
    const int words = rp * (int)sizeof(T) / 4;
    if (words % 32 == 0 || words % 32 == 16) rp += V;
    return rp;
}

template <typename T>
__host__ __device__ constexpr int eo_plane_pitch(int n) {
    const int V = 16 / (int)sizeof(T), W = 128 / (int)sizeof(T);
    const int base = n * eo_row_pitch<T>(n);
    for (int pad = 0; pad < W; pad += V)
        if ((base + pad) % W == n % W) return base + pad;
    return base;
}

template <typename T>
__host__ __device__ constexpr int eo_elem_pitch(int n) { return n * eo_plane_pitch<T>(n); }

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

// m consecutive values at p (16-byte aligned when m is a multiple of the
// vector width) into registers, and back.
template <typename T, int m>
__device__ __forceinline__ void ld_run(const T *p, T (&x)[m]) {
    constexpr int V = 16 / (int)sizeof(T);
    if constexpr (m % V == 0) {
        using VT = typename Vec16<T>::type;
#pragma unroll
        for (int q = 0; q < m / V; ++q) {
            const VT v = reinterpret_cast<const VT *>(p)[q];
            const T *s = reinterpret_cast<const T *>(&v);
#pragma unroll
            for (int c = 0; c < V; ++c) x[q * V + c] = s[c];
        }
    } else {
#pragma unroll
        for (int q = 0; q < m; ++q) x[q] = p[q];
    }
}

template <typename T, int m>
__device__ __forceinline__ void st_run(T *p, const T (&x)[m]) {
    constexpr int V = 16 / (int)sizeof(T);
    if constexpr (m % V == 0) {
        using VT = typename Vec16<T>::type;
#pragma unroll
        for (int q = 0; q < m / V; ++q) {
            VT v;
            T *d = reinterpret_cast<T *>(&v);
#pragma unroll
            for (int c = 0; c < V; ++c) d[c] = x[q * V + c];
            reinterpret_cast<VT *>(p)[q] = v;
        }
    } else {
#pragma unroll
        for (int q = 0; q < m; ++q) p[q] = x[q];
    }
}

// A row of m coefficients from shared memory with volatile vector loads: the
// compiler may neither hoist these loop-invariant loads out of the line loop
// (which would hold all 4 (n/2)^2 coefficients in registers) nor merge them.
__device__ __forceinline__ void lds_vec(const float *p, float (&v)[4]) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "r"(a));
}
__device__ __forceinline__ void lds_vec(const double *p, double (&v)[2]) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v2.f64 {%0,%1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "r"(a));
}
__device__ __forceinline__ float lds_one(const float *p) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"((unsigned)__cvta_generic_to_shared(p)));
    return v;
}
__device__ __forceinline__ double lds_one(const double *p) {
    double v;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"((unsigned)__cvta_generic_to_shared(p)));
    return v;
}

template <typename T, int m>
__device__ __forceinline__ void ld_coef(const T *p, T (&x)[m]) {
    constexpr int V = 16 / (int)sizeof(T);
    if constexpr (m % V == 0) {
#pragma unroll
        for (int q = 0; q < m / V; ++q) {
            T v[V];
            lds_vec(p + q * V, v);
#pragma unroll
            for (int c = 0; c < V; ++c) x[q * V + c] = v[c];
        }
    } else {
#pragma unroll
        for (int q = 0; q < m; ++q) x[q] = lds_one(p + q);
    }
}

// y = M x on registers by the even/odd split; P, Q are h x h row-major.
template <typename T, int n>
__device__ __forceinline__ void eo_apply(const T (&x)[n], const T *__restrict__ P, const T *__restrict__ Q,
                                         T (&y)[n]) {
    constexpr int h = n / 2;
    T e[h], o[h];
#pragma unroll
    for (int l = 0; l < h; ++l) {
        e[l] = x[l] + x[n - 1 - l];
        o[l] = x[l] - x[n - 1 - l];
    }
#pragma unroll
    for (int i = 0; i < h; ++i) {
        T p[h], q[h];
        ld_coef<T, h>(P + i * h, p);
        ld_coef<T, h>(Q + i * h, q);
        T pe = T(0), qo = T(0);
#pragma unroll
        for (int l = 0; l < h; ++l) {
            pe = fma_(p[l], e[l], pe);
            qo = fma_(q[l], o[l], qo);
        }
        y[i] = qo + pe;
        y[n - 1 - i] = qo - pe;
    }
}

template <typename T, int n>
__device__ __forceinline__ void ld_line(const T *p, int stride, T (&x)[n]) {
    if (stride == 1) {
        ld_run<T, n>(p, x);
    } else {
#pragma unroll
        for (int l = 0; l < n; ++l) x[l] = p[l * stride];
    }
}

template <typename T, int n>
__device__ __forceinline__ void st_line(T *p, int stride, const T (&y)[n]) {
    if (stride == 1) {
        st_run<T, n>(p, y);
    } else {
#pragma unroll
        for (int l = 0; l < n; ++l) p[l * stride] = y[l];
    }
}

// Stage cnt elements of u (dense [e][k][j][i] in global memory) into the
// padded layout.
template <typename T, int n>
__device__ __forceinline__ void eo_stage(T *su, const T *__restrict__ u, int cnt) {
    constexpr int V = 16 / (int)sizeof(T), RP = eo_row_pitch<T>(n), PP = eo_plane_pitch<T>(n);
    constexpr int EP = eo_elem_pitch<T>(n), n3 = n * n * n;
    if constexpr (n % V == 0) {
        using VT = typename Vec16<T>::type;
        const int nv = cnt * n3 / V;
        const VT *src = reinterpret_cast<const VT *>(u);
        for (int q = threadIdx.x; q < nv; q += blockDim.x) {
            const int f = q * V;
            const int e = f / n3, r = f - e * n3;
            const int k = r / (n * n), j = (r / n) % n, i = r % n;
            VT v;
            if constexpr (sizeof(T) == 4) v = ld_stream4(reinterpret_cast<const float4 *>(src + q));
            else v = src[q];
            *reinterpret_cast<VT *>(su + e * EP + k * PP + j * RP + i) = v;
        }
    } else {
        for (int f = threadIdx.x; f < cnt * n3; f += blockDim.x) {
            const int e = f / n3, r = f - e * n3;
            const int k = r / (n * n), j = (r / n) % n, i = r % n;
            su[e * EP + k * PP + j * RP + i] = ld_stream(u + f);
        }
    }
}

// y = M x for one line x (registers) by the even/odd split, each output
// pair stored as soon as it is formed (y[l * stride] in shared memory).
template <typename T, int n>
__device__ __forceinline__ void eo_apply_st(const T (&x)[n], const T *__restrict__ P,
                                            const T *__restrict__ Q, T *y, int stride) {
    constexpr int h = n / 2;
    T e[h], o[h];
#pragma unroll
    for (int l = 0; l < h; ++l) {
        e[l] = x[l] + x[n - 1 - l];
        o[l] = x[l] - x[n - 1 - l];
    }
#pragma unroll
    for (int i = 0; i < h; ++i) {
        T p[h], q[h];
        ld_coef<T, h>(P + i * h, p);
        ld_coef<T, h>(Q + i * h, q);
        T pe = T(0), qo = T(0);
#pragma unroll
        for (int l = 0; l < h; ++l) {
            pe = fma_(p[l], e[l], pe);
            qo = fma_(q[l], o[l], qo);
        }
        y[i * stride] = qo + pe;
        y[(n - 1 - i) * stride] = qo - pe;
    }
}

// Phases after staging (the caller has synchronised):
//   1  r- and s-lines of the gradient -> sr, ss
//   2  one thread per (i,j) column: the t-line of u; the geometric factor at
//      each node of the column (G from global memory; wr, ws in place, wt in
//      registers); the transposed t-line of wt written back over the column
//      of u (only this thread touches it in this phase).  Fusing the G loads
//      into this pass spreads them among other warps' arithmetic.
//   3  transposed r- and s-lines in place
//   4  w = r + s + t, one coalesced store
template <typename T, int n, bool HELM>
__device__ __forceinline__ void tile_eo_phases(int cnt, const T *__restrict__ G, T *__restrict__ w,
                                               const T *__restrict__ scale, Helm<T> helm,
                                               const T *__restrict__ sPQ, T *su, T *sr, T *ss) {
    constexpr int n2 = n * n, n3 = n * n * n, h = n / 2;
    constexpr int RP = eo_row_pitch<T>(n), PP = eo_plane_pitch<T>(n), EP = eo_elem_pitch<T>(n);
    const T *P = sPQ, *Q = sPQ + h * h, *Pt = sPQ + 2 * h * h, *Qt = sPQ + 3 * h * h;
    const int lines = cnt * n2;

    // 1: r-lines (k, j), then s-lines (k, i)
#pragma unroll 1
    for (int dir = 0; dir < 2; ++dir) {
        T *out = dir == 0 ? sr : ss;
        for (int t = threadIdx.x; t < lines; t += blockDim.x) {
            const int e = t / n2, ab = t - e * n2, a = ab / n, b = ab - a * n;
            const int off = e * EP + a * PP + (dir == 0 ? b * RP : b);
            const int stride = dir == 0 ? 1 : RP;
            T x[n];
            ld_line<T, n>(su + off, stride, x);
            eo_apply_st<T, n>(x, P, Q, out + off, stride);
        }
    }
    __syncthreads();

    // 2: columns (j, i)
    for (int t = threadIdx.x; t < lines; t += blockDim.x) {
        const int e = t / n2, ji = t - e * n2, j = ji / n, i = ji - j * n;
        const int off = e * EP + j * RP + i;
        T x[n], y[n];
        ld_line<T, n>(su + off, PP, x);
        eo_apply<T, n>(x, P, Q, y);                         // ut
        T m[HELM ? n : 1];                                  // h2 B u on this column
        if constexpr (HELM) {
#pragma unroll
            for (int k = 0; k < n; ++k) m[k] = helm.h2 * helm.B[e * n3 + k * n2 + ji] * x[k];
        }
        const T *Ge = G + (size_t)e * 6 * n3 + ji;
#pragma unroll
        for (int k = 0; k < n; ++k) {
            const int q = off + k * PP;
            T wr, ws;
            geo_multiply(Ge + k * n2, n3, sr[q], ss[q], y[k], wr, ws, x[k]);
            if constexpr (HELM) {
                wr *= helm.h1;
                ws *= helm.h1;
                x[k] *= helm.h1;
            }
            sr[q] = wr;
            ss[q] = ws;
        }
        if constexpr (HELM) {                               // transposed t plus the mass term
            eo_apply<T, n>(x, Pt, Qt, y);
#pragma unroll
            for (int k = 0; k < n; ++k) su[off + k * PP] = y[k] + m[k];
        } else {
            eo_apply_st<T, n>(x, Pt, Qt, su + off, PP);      // transposed t, over u's column
        }
    }
    __syncthreads();

    // 3: transposed r- and s-lines, in place
#pragma unroll 1
    for (int dir = 0; dir < 2; ++dir) {
        T *io = dir == 0 ? sr : ss;
        for (int t = threadIdx.x; t < lines; t += blockDim.x) {
            const int e = t / n2, ab = t - e * n2, a = ab / n, b = ab - a * n;
            const int off = e * EP + a * PP + (dir == 0 ? b * RP : b);
            const int stride = dir == 0 ? 1 : RP;
            T x[n];
            ld_line<T, n>(io + off, stride, x);
            eo_apply_st<T, n>(x, Pt, Qt, io + off, stride);
        }
    }
    __syncthreads();

    // 4: sum and store, dense global order
    for (int p = threadIdx.x; p < cnt * n3; p += blockDim.x) {
        const int e = p / n3, r = p - e * n3;
        const int k = r / n2, j = (r / n) % n, i = r % n;
        const int q = e * EP + k * PP + j * RP + i;
        T acc = (sr[q] + ss[q]) + su[q];
        if (scale) acc *= scale[e];
        w[p] = acc;
    }
}

}  // namespace semax
