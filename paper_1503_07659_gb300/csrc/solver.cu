// A conjugate-gradient solver around Ax: direct stiffness summation
// (gather-scatter), the operator's diagonal (Jacobi preconditioner), and a
// Jacobi-PCG whose iteration is captured once in a CUDA graph and replayed,
// with every scalar (alpha, beta, residual) kept in device memory so that no
// host round trip sits inside an iteration.  This is the PDE-solver setting
// the paper's Section 1 names as Loo.py's first use case.
//
// Vectors are kept in local (element) form, E n^3 values; a continuous vector
// has equal copies at nodes shared by elements.  Direct stiffness summation
// replaces every local value by the sum of the copies of its global node
// (Q Q^T); global inner products weight each local product by 1 / (number of
// copies).  Homogeneous Dirichlet nodes are held at zero by the
// gather-scatter's mask.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ax_plain.cuh"

namespace semax {

constexpr int kSolverThreads = 256;
constexpr int kSolverMaxBlocks = 1024;

static int solver_blocks(int64_t count) {
    int64_t b = (count + kSolverThreads * 4 - 1) / (kSolverThreads * 4);
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, kSolverMaxBlocks));
}

// ---------------------------------------------------------------- gather-scatter

__global__ void __launch_bounds__(kSolverThreads)
gs_kernel(int64_t nglobal, const int64_t *__restrict__ offsets, const int64_t *__restrict__ locals,
          const unsigned char *__restrict__ dirichlet, double *__restrict__ v) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nglobal; g += stride) {
        const int64_t q0 = offsets[g], q1 = offsets[g + 1];
        double s = 0.0;
        for (int64_t q = q0; q < q1; ++q) s += v[locals[q]];
        if (dirichlet && dirichlet[g]) s = 0.0;
        for (int64_t q = q0; q < q1; ++q) v[locals[q]] = s;
    }
}

// ---------------------------------------------------------------- operator diagonal

// diag(A_e) at node (k, j, i):
//   sum_l D[l][i]^2 Grr[k][j][l] + sum_l D[l][j]^2 Gss[k][l][i] + sum_l D[l][k]^2 Gtt[l][j][i]
//   + 2 (D[i][i] D[j][j] Grs + D[i][i] D[k][k] Grt + D[j][j] D[k][k] Gst)[k][j][i]
// (the cross terms D_a^T G_ab D_b touch the diagonal only through q = p).
template <int n>
__global__ void __launch_bounds__(kSolverThreads)
diag_kernel(int64_t E, const double *__restrict__ G, const double *__restrict__ D, double *__restrict__ d) {
    constexpr int n2 = n * n, n3 = n * n * n;
    __shared__ double sD[n2];
    for (int q = threadIdx.x; q < n2; q += blockDim.x) sD[q] = D[q];
    __syncthreads();
    const int64_t total = E * n3, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += stride) {
        const int64_t e = p / n3;
        const int q = (int)(p - e * n3), k = q / n2, j = (q / n) % n, i = q % n;
        const double *Ge = G + e * 6 * n3;
        double s = 0.0;
#pragma unroll
        for (int l = 0; l < n; ++l) {
            s = __fma_rn(sD[l * n + i] * sD[l * n + i], Ge[0 * n3 + k * n2 + j * n + l], s);
            s = __fma_rn(sD[l * n + j] * sD[l * n + j], Ge[3 * n3 + k * n2 + l * n + i], s);
            s = __fma_rn(sD[l * n + k] * sD[l * n + k], Ge[5 * n3 + l * n2 + j * n + i], s);
        }
        const double di = sD[i * n + i], dj = sD[j * n + j], dk = sD[k * n + k];
        s += 2.0 * (di * dj * Ge[1 * n3 + q] + di * dk * Ge[2 * n3 + q] + dj * dk * Ge[4 * n3 + q]);
        d[p] = s;
    }
}

// ---------------------------------------------------------------- PCG kernels

enum { S_RZ = 0, S_PAP, S_RR, S_RR0, S_ALPHA, S_BETA, S_COUNT };

__device__ __forceinline__ void block_sum2(double &a, double &b, double *out2) {
    __shared__ double sh[2][kSolverThreads / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[0][warp] = a; sh[1][warp] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < kSolverThreads / 32; ++q) { a += sh[0][q]; b += sh[1][q]; }
        out2[0] = a;
        out2[1] = b;
    }
}

// partials of sum a b wt and sum c c wt
__global__ void __launch_bounds__(kSolverThreads)
dot_kernel(int64_t count, const double *__restrict__ a, const double *__restrict__ b,
           const double *__restrict__ c, const double *__restrict__ wt, double *__restrict__ part) {
    double s0 = 0.0, s1 = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += stride) {
        s0 = __fma_rn(a[q] * b[q], wt[q], s0);
        if (c) s1 = __fma_rn(c[q] * c[q], wt[q], s1);
    }
    block_sum2(s0, s1, part + 2 * blockIdx.x);
}

// What to do with the two sums of the partials.
enum { FIN_PAP = 0, FIN_RZ_RR = 1, FIN_INIT = 2, FIN_REPLACE = 3 };

// The scalars that a mode derives from the two global sums a, b.
__device__ __forceinline__ void apply_final(double *scal, int mode, double a, double b) {
        if (mode == FIN_PAP) {
            scal[S_PAP] = a;
            scal[S_ALPHA] = a != 0.0 ? scal[S_RZ] / a : 0.0;
        } else if (mode == FIN_RZ_RR) {
            scal[S_BETA] = scal[S_RZ] != 0.0 ? a / scal[S_RZ] : 0.0;
            scal[S_RZ] = a;
            scal[S_RR] = b;
        } else if (mode == FIN_REPLACE) {   // residual replacement: r.z and r.r of the true residual
            scal[S_RZ] = a;
            scal[S_RR] = b;
        } else {
            scal[S_RZ] = a;
            scal[S_RR] = b;
            scal[S_RR0] = b;
            scal[S_BETA] = 0.0;
        }
}

__global__ void __launch_bounds__(kSolverThreads)
final_kernel(int nparts, const double *__restrict__ part, double *__restrict__ scal, int mode) {
    double s0 = 0.0, s1 = 0.0;
    for (int q = threadIdx.x; q < nparts; q += blockDim.x) {
        s0 += part[2 * q];
        s1 += part[2 * q + 1];
    }
    __shared__ double out[2];
    block_sum2(s0, s1, out);
    if (threadIdx.x == 0) apply_final(scal, mode, out[0], out[1]);
}

// The last block of a grid to finish (counted on `counter`) sums every
// block's partials, in index order like final_kernel, applies `mode` and
// resets the counter; each block must have written its partials before.
__device__ __forceinline__ void finish_in_last_block(const double *part, double *scal, int mode,
                                                     unsigned *counter) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s0 = 0.0, s1 = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) {
        s0 += __ldcg(part + 2 * q);
        s1 += __ldcg(part + 2 * q + 1);
    }
    __shared__ double out[2];
    block_sum2(s0, s1, out);
    if (threadIdx.x == 0) {
        apply_final(scal, mode, out[0], out[1]);
        *counter = 0;
    }
}

// x += alpha p; r -= alpha w; z = invdiag r; partials of r.z and (RR) r.r
// (weighted).  r.r only serves the host's convergence test, read after the
// last iteration of each launched block of iterations; the others skip it
// (and leave 0 in its scalar).
template <bool RR>
__global__ void __launch_bounds__(kSolverThreads)
update_kernel(int64_t count, double *__restrict__ x, double *__restrict__ r, double *__restrict__ z,
              const double *__restrict__ p, const double *__restrict__ w, const double *__restrict__ invdiag,
              const double *__restrict__ wt, double *__restrict__ scal, double *__restrict__ part,
              unsigned *__restrict__ counter) {
    const double alpha = scal[S_ALPHA];
    double s0 = 0.0, s1 = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += stride) {
        x[q] = __fma_rn(alpha, p[q], x[q]);
        const double rq = __fma_rn(-alpha, w[q], r[q]);
        r[q] = rq;
        const double zq = invdiag[q] * rq;
        z[q] = zq;
        const double tq = rq * wt[q];   // shared by both weighted partials
        s0 = __fma_rn(tq, zq, s0);
        if (RR) s1 = __fma_rn(tq, rq, s1);
    }
    block_sum2(s0, s1, part + 2 * blockIdx.x);
    finish_in_last_block(part, scal, FIN_RZ_RR, counter);
}

// p = z + beta p  (use_beta = 0: p = z)
__global__ void __launch_bounds__(kSolverThreads)
pupdate_kernel(int64_t count, double *__restrict__ p, const double *__restrict__ z,
               const double *__restrict__ scal, int use_beta) {
    const double beta = use_beta ? scal[S_BETA] : 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += stride)
        p[q] = use_beta ? __fma_rn(beta, p[q], z[q]) : z[q];
}

// r = b - w; z = invdiag r
__global__ void __launch_bounds__(kSolverThreads)
residual_kernel(int64_t count, const double *__restrict__ b, const double *__restrict__ w,
                const double *__restrict__ invdiag, double *__restrict__ r, double *__restrict__ z) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += stride) {
        const double rq = b[q] - w[q];
        r[q] = rq;
        z[q] = invdiag[q] * rq;
    }
}

// Gather-scatter of w fused with the partials of (p, w): p and w are
// continuous after the sum (equal copies), so the weighted local sum
// sum_l p_l w_l / mult_l is the sum over global nodes of p_g w_g.
__global__ void __launch_bounds__(kSolverThreads)
gs_dot_kernel(int64_t nglobal, const int64_t *__restrict__ offsets, const int64_t *__restrict__ locals,
              const unsigned char *__restrict__ dirichlet, double *__restrict__ w, const double *__restrict__ p,
              double *__restrict__ part, double *__restrict__ scal, unsigned *__restrict__ counter) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double acc = 0.0, unused = 0.0;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nglobal; g += stride) {
        const int64_t q0 = offsets[g], q1 = offsets[g + 1];
        double sum = 0.0;
        for (int64_t q = q0; q < q1; ++q) sum += w[locals[q]];
        if (dirichlet && dirichlet[g]) sum = 0.0;
        for (int64_t q = q0; q < q1; ++q) w[locals[q]] = sum;
        if (q1 > q0) acc = __fma_rn(p[locals[q0]], sum, acc);
    }
    block_sum2(acc, unused, part + 2 * blockIdx.x);
    finish_in_last_block(part, scal, FIN_PAP, counter);
}

// The same on the handle's split index: index t < nwork walks the global
// nodes that need work (Dirichlet nodes first, their copies set to zero,
// then the shared nodes, summed and written back, in the CSR's order);
// t >= nwork takes a local node that is its global node's only copy and not
// Dirichlet, which gather-scatter leaves as it is, so it only adds p_l w_l.
__global__ void __launch_bounds__(kSolverThreads)
gs_dot_split_kernel(int64_t nwork, int64_t ndir, int64_t nalone, const int *__restrict__ offsets,
                    const int *__restrict__ locals, const int *__restrict__ alone, double *__restrict__ w,
                    const double *__restrict__ p, double *__restrict__ part, double *__restrict__ scal,
                    unsigned *__restrict__ counter) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x, total = nwork + nalone;
    double acc = 0.0, unused = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        if (t < nwork) {
            const int q0 = offsets[t], q1 = offsets[t + 1];
            double sum = 0.0;
            if (t >= ndir)
                for (int q = q0; q < q1; ++q) sum += w[locals[q]];
            for (int q = q0; q < q1; ++q) w[locals[q]] = sum;
            acc = __fma_rn(p[locals[q0]], sum, acc);
        } else {
            const int l = alone[t - nwork];
            acc = __fma_rn(p[l], w[l], acc);
        }
    }
    block_sum2(acc, unused, part + 2 * blockIdx.x);
    finish_in_last_block(part, scal, FIN_PAP, counter);
}

// p = z + beta p (beta from the previous iteration, 0 after a restart) and
// its FP32 copy, for the mixed-precision operator
__global__ void __launch_bounds__(kSolverThreads)
pupdate_f32_kernel(int64_t count, double *__restrict__ p, const double *__restrict__ z, float *__restrict__ p32,
                   const double *__restrict__ scal) {
    const double beta = scal[S_BETA];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += stride) {
        const double v = __fma_rn(beta, p[q], z[q]);
        p[q] = v;
        p32[q] = (float)v;
    }
}

// precision conversions of the mixed-precision operator
__global__ void __launch_bounds__(kSolverThreads)
to_f32_kernel(int64_t count, const double *__restrict__ a, float *__restrict__ b) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += stride) b[q] = (float)a[q];
}
__global__ void __launch_bounds__(kSolverThreads)
to_f64_kernel(int64_t count, const float *__restrict__ a, double *__restrict__ b) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += stride) b[q] = (double)a[q];
}

// x += d
__global__ void __launch_bounds__(kSolverThreads)
axpy1_kernel(int64_t count, double *__restrict__ x, const double *__restrict__ d) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += stride) x[q] += d[q];
}

// invdiag = free ? 1 / d : 0 (d already summed; Dirichlet nodes were zeroed)
__global__ void __launch_bounds__(kSolverThreads)
invert_kernel(int64_t count, double *__restrict__ d) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += stride)
        d[q] = d[q] != 0.0 ? 1.0 / d[q] : 0.0;
}

template <int n>
static int launch_diag(int64_t E, const double *G, const double *D, double *d, cudaStream_t s) {
    const int64_t total = E * n * n * n;
    const int64_t blocks = std::min<int64_t>((total + kSolverThreads - 1) / kSolverThreads, 65535LL * 16);
    diag_kernel<n><<<(unsigned)blocks, kSolverThreads, 0, s>>>(E, G, D, d);
    return launch_status();
}

static int launch_diag_N(int64_t E, int N, const double *G, const double *D, double *d, cudaStream_t s) {
    switch (N + 1) {
#define SEMAX_CASE(nn) \
    case nn: return launch_diag<nn>(E, G, D, d, s);
        SEMAX_CASE(2) SEMAX_CASE(3) SEMAX_CASE(4) SEMAX_CASE(5) SEMAX_CASE(6) SEMAX_CASE(7)
        SEMAX_CASE(8) SEMAX_CASE(9) SEMAX_CASE(10) SEMAX_CASE(11) SEMAX_CASE(12) SEMAX_CASE(13)
        SEMAX_CASE(14) SEMAX_CASE(15) SEMAX_CASE(16)
#undef SEMAX_CASE
        default: return SEMAX_EUNSUPPORTED_N;
    }
}

}  // namespace semax

using namespace semax;

// ---------------------------------------------------------------- gather-scatter handle

struct semax_gs {
    int64_t nlocal = 0, nglobal = 0;
    int64_t *offsets = nullptr;        // [nglobal + 1]
    int64_t *locals = nullptr;         // [nlocal], grouped by global node
    unsigned char *dirichlet = nullptr;
    double *inv_mult = nullptr;        // [nlocal]
    // split index (32-bit, when nlocal < 2^31): the global nodes that need
    // work, Dirichlet first (ndir of them), then shared (nwork in all), as a
    // CSR; and the local nodes that are alone on a non-Dirichlet global node
    int64_t nwork = 0, ndir = 0, nalone = 0;
    int *work_off = nullptr, *work_loc = nullptr, *alone = nullptr;
    unsigned magic = 0x95u;
};

static void gs_free(semax_gs *g) {
    if (!g) return;
    cudaFree(g->offsets);
    cudaFree(g->locals);
    cudaFree(g->dirichlet);
    cudaFree(g->inv_mult);
    cudaFree(g->work_off);
    cudaFree(g->work_loc);
    cudaFree(g->alone);
    g->magic = 0;
    delete g;
}

extern "C" int semax_gs_create(semax_gs **gs, int64_t nlocal, const int64_t *l2g, int64_t nglobal,
                               const unsigned char *dirichlet) {
    if (!gs) return SEMAX_EINVAL;
    *gs = nullptr;
    if (nlocal <= 0 || nglobal <= 0 || !l2g) return SEMAX_EINVAL;
    std::vector<int64_t> off(nglobal + 1, 0);
    for (int64_t l = 0; l < nlocal; ++l) {
        if (l2g[l] < 0 || l2g[l] >= nglobal) return SEMAX_EINVAL;
        ++off[l2g[l] + 1];
    }
    for (int64_t g = 0; g < nglobal; ++g) off[g + 1] += off[g];
    std::vector<int64_t> loc(nlocal), fill(off.begin(), off.end() - 1);
    for (int64_t l = 0; l < nlocal; ++l) loc[fill[l2g[l]]++] = l;
    std::vector<double> im(nlocal);
    for (int64_t l = 0; l < nlocal; ++l) im[l] = 1.0 / (double)(off[l2g[l] + 1] - off[l2g[l]]);
    semax_gs *g = new semax_gs();
    g->nlocal = nlocal;
    g->nglobal = nglobal;
    int st = cuda_status(cudaMalloc(&g->offsets, sizeof(int64_t) * (nglobal + 1)));
    if (st == SEMAX_OK) st = cuda_status(cudaMalloc(&g->locals, sizeof(int64_t) * nlocal));
    if (st == SEMAX_OK) st = cuda_status(cudaMalloc(&g->inv_mult, sizeof(double) * nlocal));
    if (st == SEMAX_OK) st = cuda_status(cudaMemcpy(g->offsets, off.data(), sizeof(int64_t) * (nglobal + 1), cudaMemcpyHostToDevice));
    if (st == SEMAX_OK) st = cuda_status(cudaMemcpy(g->locals, loc.data(), sizeof(int64_t) * nlocal, cudaMemcpyHostToDevice));
    if (st == SEMAX_OK) st = cuda_status(cudaMemcpy(g->inv_mult, im.data(), sizeof(double) * nlocal, cudaMemcpyHostToDevice));
    if (st == SEMAX_OK && dirichlet) {
        st = cuda_status(cudaMalloc(&g->dirichlet, nglobal));
        if (st == SEMAX_OK) st = cuda_status(cudaMemcpy(g->dirichlet, dirichlet, nglobal, cudaMemcpyHostToDevice));
    }
    if (st == SEMAX_OK && nlocal < (int64_t)INT32_MAX) {
        std::vector<int> woff(1, 0), wloc, al;
        auto add = [&](int64_t gn) {
            for (int64_t q = off[gn]; q < off[gn + 1]; ++q) wloc.push_back((int)loc[q]);
            woff.push_back((int)wloc.size());
        };
        for (int64_t gn = 0; gn < nglobal; ++gn)
            if (dirichlet && dirichlet[gn] && off[gn + 1] > off[gn]) add(gn);
        g->ndir = (int64_t)woff.size() - 1;
        for (int64_t gn = 0; gn < nglobal; ++gn) {
            const int64_t m = off[gn + 1] - off[gn];
            if (dirichlet && dirichlet[gn]) continue;
            if (m > 1) add(gn);
            else if (m == 1) al.push_back((int)loc[off[gn]]);
        }
        g->nwork = (int64_t)woff.size() - 1;
        g->nalone = (int64_t)al.size();
        st = cuda_status(cudaMalloc(&g->work_off, sizeof(int) * woff.size()));
        if (st == SEMAX_OK && !wloc.empty()) st = cuda_status(cudaMalloc(&g->work_loc, sizeof(int) * wloc.size()));
        if (st == SEMAX_OK && !al.empty()) st = cuda_status(cudaMalloc(&g->alone, sizeof(int) * al.size()));
        if (st == SEMAX_OK) st = cuda_status(cudaMemcpy(g->work_off, woff.data(), sizeof(int) * woff.size(), cudaMemcpyHostToDevice));
        if (st == SEMAX_OK && !wloc.empty())
            st = cuda_status(cudaMemcpy(g->work_loc, wloc.data(), sizeof(int) * wloc.size(), cudaMemcpyHostToDevice));
        if (st == SEMAX_OK && !al.empty())
            st = cuda_status(cudaMemcpy(g->alone, al.data(), sizeof(int) * al.size(), cudaMemcpyHostToDevice));
    }
    if (st != SEMAX_OK) {
        gs_free(g);
        return st;
    }
    *gs = g;
    return SEMAX_OK;
}

static int gs_enqueue(const semax_gs *gs, double *v, int apply_mask, cudaStream_t s) {
    const int blocks = solver_blocks(gs->nglobal);
    gs_kernel<<<blocks, kSolverThreads, 0, s>>>(gs->nglobal, gs->offsets, gs->locals,
                                                 apply_mask ? gs->dirichlet : nullptr, v);
    return launch_status();
}

extern "C" int semax_gs_apply(const semax_gs *gs, double *v, int apply_mask, void *stream) {
    if (!gs || gs->magic != 0x95u) return SEMAX_ENOPLAN;
    if (!v) return SEMAX_EINVAL;
    return gs_enqueue(gs, v, apply_mask, (cudaStream_t)stream);
}

extern "C" int semax_gs_destroy(semax_gs *gs) {
    if (!gs || gs->magic != 0x95u) return SEMAX_ENOPLAN;
    gs_free(gs);
    return SEMAX_OK;
}

extern "C" int sem_ax_diag(int64_t E, int N, const double *G, const double *D, double *diag, void *stream) {
    if (E < 0) return SEMAX_EINVAL;
    if (N < 1 || N > kMaxN) return SEMAX_EUNSUPPORTED_N;
    if (E == 0) return SEMAX_OK;
    if (!G || !D || !diag) return SEMAX_EINVAL;
    return launch_diag_N(E, N, G, D, diag, (cudaStream_t)stream);
}

// ---------------------------------------------------------------- PCG

struct semax_pcg {
    int64_t E = 0;
    int N = 0;
    int64_t count = 0;
    const double *G = nullptr, *D = nullptr;
    const semax_gs *gs = nullptr;
    double *r = nullptr, *z = nullptr, *p = nullptr, *w = nullptr, *invdiag = nullptr;
    double *part = nullptr, *scal = nullptr;
    float *G32 = nullptr, *D32 = nullptr, *p32 = nullptr, *w32 = nullptr;   // SEMAX_PCG_MIXED
    double *d = nullptr;                                                   // its correction vector
    void *Gp = nullptr;                 // SEMAX_PCG_F64TC at N = 7: the prepared geometric factor
    unsigned *counters = nullptr;   // last-block reductions (2), then the tensor-core operator's status word
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double *x_bound = nullptr;          // the x the graph was captured with
    int flags = 0;
    unsigned magic = 0x9c9u;
};


// w = A_L v, FP64-accurate, with the operator the solver was created with
static int pcg_apply_a64(semax_pcg *s, const double *v, double *w, cudaStream_t cs) {
    if (s->flags & SEMAX_PCG_F64X) return sem_ax_f64x(s->E, s->N, v, s->G, s->D, w, cs);
    int *status = reinterpret_cast<int *>(s->counters + 2);
    if (s->Gp) return sem_ax_f64tc_prepared_status(s->E, s->N, v, s->Gp, s->D, w, status, cs);   // bit for bit sem_ax_f64tc
    if (s->flags & SEMAX_PCG_F64TC) return sem_ax_f64tc_status(s->E, s->N, v, s->G, s->D, w, status, cs);
    return launch_plain<double>(s->E, s->N, default_tile<double>(s->N + 1), v, s->G, s->D, w, nullptr,
                                Helm<double>{nullptr, 1.0, 0.0}, cs);
}

static const int kItersPerGraph = 10;

static void pcg_free(semax_pcg *s) {
    if (!s) return;
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    if (s->cs) cudaStreamDestroy(s->cs);
    cudaFree(s->r);
    cudaFree(s->z);
    cudaFree(s->p);
    cudaFree(s->w);
    cudaFree(s->invdiag);
    cudaFree(s->part);
    cudaFree(s->scal);
    cudaFree(s->G32);
    cudaFree(s->D32);
    cudaFree(s->p32);
    cudaFree(s->w32);
    cudaFree(s->d);
    cudaFree(s->Gp);
    cudaFree(s->counters);
    s->magic = 0;
    delete s;
}

// One PCG iteration on stream cs (x is the caller's solution vector).
// With SEMAX_PCG_MIXED the direction update p = z + beta p is deferred to
// the start of the next iteration, fused with its FP32 conversion.
static int pcg_iteration(semax_pcg *s, double *x, cudaStream_t cs, bool rr) {
    const int blocks = solver_blocks(s->count);
    const bool mixed = (s->flags & SEMAX_PCG_MIXED) != 0;
    int st = SEMAX_OK;
    if (mixed) {
        pupdate_f32_kernel<<<blocks, kSolverThreads, 0, cs>>>(s->count, s->p, s->z, s->p32, s->scal);
        st = launch_status();
        if (st == SEMAX_OK)
            st = launch_plain<float>(s->E, s->N, default_tile<float>(s->N + 1), s->p32, s->G32, s->D32, s->w32,
                                     nullptr, Helm<float>{nullptr, 1.0f, 0.0f}, cs);
        if (st == SEMAX_OK) {
            to_f64_kernel<<<blocks, kSolverThreads, 0, cs>>>(s->count, s->w32, s->w);
            st = launch_status();
        }
    } else {
        st = pcg_apply_a64(s, s->p, s->w, cs);
    }
    if (st != SEMAX_OK) return st;
    const semax_gs *gs = s->gs;
    if (gs->work_off)   // the split index: only the nodes that need work walk the CSR
        gs_dot_split_kernel<<<solver_blocks(gs->nwork + gs->nalone), kSolverThreads, 0, cs>>>(
            gs->nwork, gs->ndir, gs->nalone, gs->work_off, gs->work_loc, gs->alone, s->w, s->p, s->part, s->scal,
            s->counters);
    else
        gs_dot_kernel<<<solver_blocks(gs->nglobal), kSolverThreads, 0, cs>>>(gs->nglobal, gs->offsets, gs->locals,
                                                                              gs->dirichlet, s->w, s->p, s->part,
                                                                              s->scal, s->counters);
    if (rr)
        update_kernel<true><<<blocks, kSolverThreads, 0, cs>>>(s->count, x, s->r, s->z, s->p, s->w, s->invdiag,
                                                               s->gs->inv_mult, s->scal, s->part, s->counters + 1);
    else
        update_kernel<false><<<blocks, kSolverThreads, 0, cs>>>(s->count, x, s->r, s->z, s->p, s->w, s->invdiag,
                                                                s->gs->inv_mult, s->scal, s->part, s->counters + 1);
    if (!mixed) pupdate_kernel<<<blocks, kSolverThreads, 0, cs>>>(s->count, s->p, s->z, s->scal, 1);
    return launch_status();
}

extern "C" int sem_pcg_create(semax_pcg **pcg, int64_t E, int N, const double *G, const double *D,
                              const semax_gs *gs, int flags) {
    if (!pcg) return SEMAX_EINVAL;
    *pcg = nullptr;
    if (E <= 0 || !G || !D || !gs || gs->magic != 0x95u ||
        (flags & ~(SEMAX_PCG_F64X | SEMAX_PCG_F64TC | SEMAX_PCG_MIXED)) ||
        (flags & (SEMAX_PCG_F64X | SEMAX_PCG_F64TC)) == (SEMAX_PCG_F64X | SEMAX_PCG_F64TC))
        return SEMAX_EINVAL;
    if (N < 1 || N > kMaxN) return SEMAX_EUNSUPPORTED_N;
    const int64_t count = E * (N + 1) * (N + 1) * (N + 1);
    if (gs->nlocal != count) return SEMAX_EINVAL;
    semax_pcg *s = new semax_pcg();
    s->E = E;
    s->N = N;
    s->count = count;
    s->G = G;
    s->D = D;
    s->gs = gs;
    s->flags = flags;
    const size_t vb = sizeof(double) * (size_t)count;
    int st = SEMAX_OK;
    for (double **v : {&s->r, &s->z, &s->p, &s->w, &s->invdiag})
        if (st == SEMAX_OK) st = cuda_status(cudaMalloc(v, vb));
    if (st == SEMAX_OK) st = cuda_status(cudaMalloc(&s->part, sizeof(double) * 2 * kSolverMaxBlocks));
    if (st == SEMAX_OK) st = cuda_status(cudaMalloc(&s->scal, sizeof(double) * S_COUNT));
    if (st == SEMAX_OK) st = cuda_status(cudaMalloc(&s->counters, 4 * sizeof(unsigned)));
    if (st == SEMAX_OK) st = cuda_status(cudaMemset(s->counters, 0, 4 * sizeof(unsigned)));
    if (st == SEMAX_OK) st = cuda_status(cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking));
    if (st == SEMAX_OK && (flags & SEMAX_PCG_MIXED)) {
        const int64_t nn = (int64_t)(N + 1) * (N + 1);
        for (float **v : {&s->p32, &s->w32})
            if (st == SEMAX_OK) st = cuda_status(cudaMalloc(v, sizeof(float) * (size_t)count));
        if (st == SEMAX_OK) st = cuda_status(cudaMalloc(&s->G32, sizeof(float) * 6 * (size_t)count));
        if (st == SEMAX_OK) st = cuda_status(cudaMalloc(&s->D32, sizeof(float) * (size_t)nn));
        if (st == SEMAX_OK) st = cuda_status(cudaMalloc(&s->d, sizeof(double) * (size_t)count));
        if (st == SEMAX_OK) {
            to_f32_kernel<<<solver_blocks(6 * count), kSolverThreads, 0, s->cs>>>(6 * count, G, s->G32);
            to_f32_kernel<<<1, kSolverThreads, 0, s->cs>>>(nn, D, s->D32);
            st = launch_status();
        }
    }
    // the tensor-core operator at order 7 reads G prepared once (split into float pairs)
    if (st == SEMAX_OK && (flags & SEMAX_PCG_F64TC) && N == 7) {
        size_t bytes = 0;
        st = sem_ax_f64tc_prepare_size(E, N, &bytes);
        if (st == SEMAX_OK) st = cuda_status(cudaMalloc(&s->Gp, bytes));
        if (st == SEMAX_OK) st = sem_ax_f64tc_prepare(E, N, G, s->Gp, s->cs);
    }
    // Jacobi: invdiag = 1 / (Q Q^T diag(A_L)) at free nodes, 0 at Dirichlet nodes
    if (st == SEMAX_OK) st = launch_diag_N(E, N, G, D, s->invdiag, s->cs);
    if (st == SEMAX_OK) st = gs_enqueue(gs, s->invdiag, 1, s->cs);
    if (st == SEMAX_OK) {
        invert_kernel<<<solver_blocks(count), kSolverThreads, 0, s->cs>>>(count, s->invdiag);
        st = launch_status();
    }
    if (st == SEMAX_OK) st = cuda_status(cudaStreamSynchronize(s->cs));
    if (st != SEMAX_OK) {
        pcg_free(s);
        return st;
    }
    *pcg = s;
    return SEMAX_OK;
}

extern "C" int sem_pcg_solve(semax_pcg *s, const double *b, double *x, int max_iter, double rtol, int *iters,
                             double *rel_res, void *stream) {
    if (!s || s->magic != 0x9c9u) return SEMAX_ENOPLAN;
    if (!b || !x || max_iter < 0 || !(rtol >= 0.0)) return SEMAX_EINVAL;
    if (overlaps(x, sizeof(double) * s->count, b, sizeof(double) * s->count)) return SEMAX_EALIAS;
    cudaStream_t us = (cudaStream_t)stream;
    cudaStream_t cs = s->cs;
    // order the solver's stream after the caller's work
    cudaEvent_t ev;
    int st = cuda_status(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    if (st != SEMAX_OK) return st;
    st = cuda_status(cudaEventRecord(ev, us));
    if (st == SEMAX_OK) st = cuda_status(cudaStreamWaitEvent(cs, ev, 0));
    const int blocks = solver_blocks(s->count);
    const bool mixed = (s->flags & SEMAX_PCG_MIXED) != 0;
    double *xi = mixed ? s->d : x;   // the vector the iterations update (the graph is bound to it)
    // r = b - A v (FP64-accurate operator), z = M r, p = z, and the scalars of a fresh start
    auto restart = [&](const double *v) {
        int rs = pcg_apply_a64(s, v, s->w, cs);
        if (rs == SEMAX_OK) rs = gs_enqueue(s->gs, s->w, 1, cs);
        if (rs == SEMAX_OK) {
            residual_kernel<<<blocks, kSolverThreads, 0, cs>>>(s->count, b, s->w, s->invdiag, s->r, s->z);
            dot_kernel<<<blocks, kSolverThreads, 0, cs>>>(s->count, s->r, s->z, s->r, s->gs->inv_mult, s->part);
            final_kernel<<<1, kSolverThreads, 0, cs>>>(blocks, s->part, s->scal, FIN_INIT);
            pupdate_kernel<<<blocks, kSolverThreads, 0, cs>>>(s->count, s->p, s->z, s->scal, 0);
            rs = launch_status();
        }
        return rs;
    };
    // (re)capture a block of iterations bound to xi
    if (st == SEMAX_OK && s->x_bound != xi) {
        if (s->exec) { cudaGraphExecDestroy(s->exec); s->exec = nullptr; }
        if (s->graph) { cudaGraphDestroy(s->graph); s->graph = nullptr; }
        cudaStream_t cap = nullptr;
        st = cuda_status(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        if (st == SEMAX_OK) st = cuda_status(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        if (st == SEMAX_OK) {
            int lst = SEMAX_OK;
            for (int it = 0; it < kItersPerGraph && lst == SEMAX_OK; ++it)
                lst = pcg_iteration(s, xi, cap, it == kItersPerGraph - 1);
            int est = cuda_status(cudaStreamEndCapture(cap, &s->graph));
            st = lst != SEMAX_OK ? lst : est;
        }
        if (st == SEMAX_OK) st = cuda_status(cudaGraphInstantiate(&s->exec, s->graph, 0));
        if (cap) cudaStreamDestroy(cap);
        s->x_bound = st == SEMAX_OK ? xi : nullptr;
    }
    double h[S_COUNT] = {0};
    int dev_status = SEMAX_OK;
    // the scalars, and the status word of the tensor-core operator: a staging
    // wait that gave up ends the solve with SEMAX_ETIMEOUT
    auto read_scalars = [&]() {
        int rs = cuda_status(cudaMemcpyAsync(h, s->scal, sizeof h, cudaMemcpyDeviceToHost, cs));
        if (rs == SEMAX_OK)
            rs = cuda_status(cudaMemcpyAsync(&dev_status, s->counters + 2, sizeof dev_status, cudaMemcpyDeviceToHost, cs));
        if (rs == SEMAX_OK) rs = cuda_status(cudaStreamSynchronize(cs));
        return rs == SEMAX_OK && dev_status == SEMAX_ETIMEOUT ? SEMAX_ETIMEOUT : rs;
    };
    // iterate on xi until its recurrence residual falls to `target` of its start
    int done = 0;
    bool broke_down = false;   // the recurrence produced NaN
    auto iterate = [&](double target) {
        int rs = SEMAX_OK;
        double r = 1.0;
        while (rs == SEMAX_OK && done < max_iter && r > target) {
            const int left = max_iter - done;
            if (left >= kItersPerGraph) {
                rs = cuda_status(cudaGraphLaunch(s->exec, cs));
                done += kItersPerGraph;
            } else {
                for (int it = 0; it < left && rs == SEMAX_OK; ++it) rs = pcg_iteration(s, xi, cs, it == left - 1);
                done += left;
            }
            if (rs == SEMAX_OK) rs = read_scalars();
            r = h[S_RR0] > 0.0 ? std::sqrt(std::max(h[S_RR], 0.0) / h[S_RR0]) : 0.0;
            if (!(r == r)) {   // NaN: stop
                broke_down = true;
                break;
            }
        }
        return rs;
    };
    double rel = 1.0;
    if (st == SEMAX_OK) st = cuda_status(cudaMemsetAsync(s->counters + 2, 0, sizeof(int), cs));
    if (st == SEMAX_OK) st = restart(x);
    if (st == SEMAX_OK) st = read_scalars();
    const double rr0 = h[S_RR0];
    if (!mixed) {
        rel = rr0 > 0.0 ? 1.0 : 0.0;
        if (st == SEMAX_OK && rel > rtol) st = iterate(rtol);
        if (rel > 0.0) rel = std::sqrt(std::max(h[S_RR], 0.0) / rr0);
    } else {
        // Mixed-precision iterative refinement: each outer step takes the true
        // residual with the FP64-accurate operator, solves A d = r from d = 0
        // with the FP32 operator inside the FP64 iteration to a relative
        // reduction eta, and adds d to x.  Restarting keeps the FP32
        // operator's error relative to the current residual.
        // Stops when an outer step fails to halve the true residual: the
        // FP64-accurate operator's own error then sets the floor.
        const int64_t vbytes = (int64_t)sizeof(double) * s->count;
        double prev = 2.0;
        for (;;) {
            rel = rr0 > 0.0 ? std::sqrt(std::max(h[S_RR0], 0.0) / rr0) : 0.0;
            if (st != SEMAX_OK || !(rel > rtol) || done >= max_iter || rel > 0.5 * prev) break;
            prev = rel;
            const double eta = std::min(0.5, std::max(1e-5, 0.5 * rtol / rel));
            st = cuda_status(cudaMemsetAsync(s->d, 0, (size_t)vbytes, cs));
            if (st == SEMAX_OK) st = iterate(eta);
            if (broke_down) break;   // x keeps the last refined iterate
            if (st == SEMAX_OK) {
                axpy1_kernel<<<blocks, kSolverThreads, 0, cs>>>(s->count, x, s->d);
                st = launch_status();
            }
            if (st == SEMAX_OK) st = restart(x);
            if (st == SEMAX_OK) st = read_scalars();
        }
    }
    // the caller's stream continues after the solve
    if (st == SEMAX_OK) st = cuda_status(cudaEventRecord(ev, cs));
    if (st == SEMAX_OK) st = cuda_status(cudaStreamWaitEvent(us, ev, 0));
    cudaEventDestroy(ev);
    if (iters) *iters = done;
    if (rel_res) *rel_res = rel;
    return st;
}

extern "C" int sem_pcg_destroy(semax_pcg *s) {
    if (!s || s->magic != 0x9c9u) return SEMAX_ENOPLAN;
    pcg_free(s);
    return SEMAX_OK;
}
