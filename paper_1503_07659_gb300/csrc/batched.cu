// Batched Ax over groups of uneven polynomial order in ONE persistent launch,
// plus plans (captured CUDA graph) and the autotuner that picks the tile
// shape per order.
//
// Work decomposition: group g of E_g elements is cut into tiles of epb_g
// elements; groups are ordered by cost per element (n^4) descending, so the
// tile index space runs longest-first.  The table of groups and the prefix
// sums of their tile counts travel in the kernel parameters; each CTA takes
// the next tile index from one device counter (atomicAdd) and finds its group
// by a scan of the prefix array.  No CTA ever waits on another.
//
// The tuning knobs mirror the transformation search space the paper's
// Section 1 assigns to an autotuner and its Section 3 `split_iname`/tag
// transforms (how many elements one work-group handles, and how loop indices
// map to threads): elements per tile and thread mapping (one thread per node
// or one thread per (i,j) column).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ax_f64x.cuh"

namespace semax {

constexpr int kMaxGroups = 32;
constexpr int MAP_F64X = 3;   // the double-float FP64-accurate tile (even n)
constexpr int MAP_F64TC = 4;  // orders 7 and 15 under SEMAX_PLAN_F64TC: the tensor-core form, own launch
constexpr int kBatchThreads = 256;

struct GroupDev {
    const double *u;
    const double *G;
    const double *D;
    double *w;
    int64_t E;
    int n;
    int epb;
    int map;
};

struct BatchParams {
    int ngroups;
    int64_t ntiles;
    int64_t tile_start[kMaxGroups + 1];
    GroupDev g[kMaxGroups];
};

template <int n, int MAP>
__device__ __forceinline__ void run_tile(const GroupDev &g, int64_t e0, int cnt, double *sD,
                                         double *buf) {
    constexpr int n3 = n * n * n;
    ax_tile<double, n, MAP>(cnt, g.u + e0 * n3, g.G + e0 * 6 * n3, g.w + e0 * n3, nullptr,
                            Helm<double>{nullptr, 1.0, 0.0}, sD, buf);
}

__global__ void __launch_bounds__(kBatchThreads)
ax_batched_kernel(const __grid_constant__ BatchParams P, unsigned long long *counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long s_tile;
    double *sD = reinterpret_cast<double *>(smem_raw);
    double *buf = sD + d_slots<double>(16);
    for (;;) {
        if (threadIdx.x == 0) s_tile = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const int64_t t = s_tile;
        if (t >= P.ntiles) break;
        int gi = 0;
        while (gi + 1 < P.ngroups && P.tile_start[gi + 1] <= t) ++gi;
        const GroupDev &g = P.g[gi];
        const int64_t e0 = (t - P.tile_start[gi]) * g.epb;
        const int cnt = (int)(g.E - e0 < g.epb ? g.E - e0 : g.epb);
        if (g.map != MAP_F64X)   // the double-float tile stages D itself
            for (int q = threadIdx.x; q < g.n * g.n; q += blockDim.x) sD[q] = g.D[q];
        switch (g.n * 4 + g.map) {
#define SEMAX_CASE(nn)                                                                \
    case nn * 4 + MAP_NODE: run_tile<nn, MAP_NODE>(g, e0, cnt, sD, buf); break;       \
    case nn * 4 + MAP_COLUMN: run_tile<nn, MAP_COLUMN>(g, e0, cnt, sD, buf); break;
#define SEMAX_CASE_EVEN(nn) SEMAX_CASE(nn) \
    case nn * 4 + MAP_EO: run_tile<nn, MAP_EO>(g, e0, cnt, sD, buf); break; \
    case nn * 4 + MAP_F64X: \
        dfx::f64x_tile<nn>(cnt, g.epb, g.u + e0 * nn * nn * nn, g.G + e0 * 6 * nn * nn * nn, g.D, \
                           g.w + e0 * nn * nn * nn, smem_raw); \
        break;
            SEMAX_CASE_EVEN(2) SEMAX_CASE(3) SEMAX_CASE_EVEN(4) SEMAX_CASE(5) SEMAX_CASE_EVEN(6)
            SEMAX_CASE(7) SEMAX_CASE_EVEN(8) SEMAX_CASE(9) SEMAX_CASE_EVEN(10) SEMAX_CASE(11)
            SEMAX_CASE_EVEN(12) SEMAX_CASE(13) SEMAX_CASE_EVEN(14) SEMAX_CASE(15) SEMAX_CASE_EVEN(16)
#undef SEMAX_CASE_EVEN
#undef SEMAX_CASE
            default: break;
        }
        __syncthreads();  // sD, the tile buffers and s_tile are reused next round
    }
}

// ---------------------------------------------------------------- host side

struct TileChoice {
    int epb;
    int map;
};

// Elements per tile and shared bytes of the double-float tile for order n.
static int f64x_epb(int n) { return std::max(1, dfx::kThreads / (n * n)); }
static size_t f64x_smem(int n, int epb) {
    switch (n) {
        case 2: return dfx::smem_bytes<2>(epb);
        case 4: return dfx::smem_bytes<4>(epb);
        case 6: return dfx::smem_bytes<6>(epb);
        case 8: return dfx::smem_bytes<8>(epb);
        case 10: return dfx::smem_bytes<10>(epb);
        case 12: return dfx::smem_bytes<12>(epb);
        case 14: return dfx::smem_bytes<14>(epb);
        case 16: return dfx::smem_bytes<16>(epb);
        default: return 0;
    }
}

static size_t batch_smem(const BatchParams &P) {
    size_t m = 0;
    for (int q = 0; q < P.ngroups; ++q) {
        const GroupDev &g = P.g[q];
        if (g.map == MAP_F64X)
            m = std::max(m, f64x_smem(g.n, g.epb));
        else
            m = std::max(m, tile_smem_bytes<double>(g.n, g.epb, g.map) - sizeof(double) * d_slots<double>(g.n) +
                                sizeof(double) * d_slots<double>(16));
    }
    return m;
}

static bool choice_valid(int n, TileChoice c) {
    if (c.map == MAP_F64X) return n % 2 == 0 && c.epb == f64x_epb(n);
    if (c.epb < 1) return false;
    if (c.map == MAP_COLUMN && c.epb * n * n > kBatchThreads) return false;
    if (c.map == MAP_EO && n % 2 != 0) return false;
    if (c.map != MAP_COLUMN && c.map != MAP_NODE && c.map != MAP_EO) return false;
    return tile_smem_bytes<double>(n, c.epb, c.map) + sizeof(double) * 256 <= 200 * 1024;
}

// Same mapping and elements per tile as the plain FP64 launch's default (so
// the two agree bit for bit).
static TileChoice default_choice(int n) {
    TileChoice c{std::max(1, kBatchThreads / (n * n)), n % 2 == 0 ? MAP_EO : MAP_COLUMN};
    return c;
}

static int check_groups(const semax_group *groups, int ngroups) {
    if (ngroups < 0 || ngroups > kMaxGroups || (ngroups > 0 && !groups)) return SEMAX_EINVAL;
    for (int q = 0; q < ngroups; ++q) {
        const semax_group &g = groups[q];
        int st = check_args(g.E, g.N, g.u, g.G, g.D, g.w);
        if (st != SEMAX_OK) return st;
    }
    // outputs must not overlap any input or each other
    for (int a = 0; a < ngroups; ++a) {
        const semax_group &ga = groups[a];
        const size_t na = (size_t)ga.N + 1, wa = (size_t)ga.E * na * na * na * 8;
        for (int b = 0; b < ngroups; ++b) {
            if (a == b) continue;
            const semax_group &gb = groups[b];
            const size_t nb = (size_t)gb.N + 1, ub = (size_t)gb.E * nb * nb * nb * 8;
            if (overlaps(ga.w, wa, gb.u, ub) || overlaps(ga.w, wa, gb.G, 6 * ub) ||
                overlaps(ga.w, wa, gb.w, ub) || overlaps(ga.w, wa, gb.D, nb * nb * 8))
                return SEMAX_EALIAS;
        }
    }
    return SEMAX_OK;
}

// Fill P from groups with per-order choices; groups sorted by n descending.
static void build_params(BatchParams &P, const semax_group *groups, int ngroups,
                         const std::vector<TileChoice> &choice_by_n) {
    std::vector<int> order;
    for (int q = 0; q < ngroups; ++q)
        if (groups[q].E > 0) order.push_back(q);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return groups[a].N > groups[b].N; });
    std::memset(&P, 0, sizeof(P));
    P.ngroups = (int)order.size();
    int64_t t = 0;
    for (int q = 0; q < P.ngroups; ++q) {
        const semax_group &g = groups[order[q]];
        const int n = g.N + 1;
        TileChoice c = choice_by_n[n];
        P.g[q] = GroupDev{g.u, g.G, g.D, g.w, g.E, n, c.epb, c.map};
        P.tile_start[q] = t;
        t += (g.E + c.epb - 1) / c.epb;
    }
    P.tile_start[P.ngroups] = t;
    P.ntiles = t;
}

struct LaunchShape {
    unsigned grid;
    size_t smem;
};

// Kernel attributes and grid size; not a stream operation, so it is done
// before any graph capture starts.
static int prepare_batched(const BatchParams &P, LaunchShape *ls) {
    ls->grid = 0;
    ls->smem = batch_smem(P);
    if (P.ntiles == 0) return SEMAX_OK;
    int st = cuda_status(cudaFuncSetAttribute(ax_batched_kernel,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ls->smem));
    if (st != SEMAX_OK) return st;
    int per_sm = 0;
    st = cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ax_batched_kernel,
                                                                   kBatchThreads, ls->smem));
    if (st != SEMAX_OK) return st;
    if (per_sm < 1) return SEMAX_EINVAL;
    int64_t grid = (int64_t)per_sm * device_sm_count();
    if (grid > P.ntiles) grid = P.ntiles;
    ls->grid = (unsigned)grid;
    return SEMAX_OK;
}

// Queue the counter reset and the persistent kernel on s.
static int enqueue_batched(const BatchParams &P, const LaunchShape &ls, unsigned long long *counter,
                           cudaStream_t s) {
    if (ls.grid == 0) return SEMAX_OK;
    int st = cuda_status(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
    if (st != SEMAX_OK) return st;
    ax_batched_kernel<<<ls.grid, kBatchThreads, ls.smem, s>>>(P, counter);
    return launch_status();
}

static int launch_batched(const BatchParams &P, unsigned long long *counter, cudaStream_t s) {
    LaunchShape ls;
    int st = prepare_batched(P, &ls);
    return st != SEMAX_OK ? st : enqueue_batched(P, ls, counter, s);
}

}  // namespace semax

using namespace semax;

// ---------------------------------------------------------------- one-shot batched call

extern "C" int sem_ax_batched_workspace_size(const semax_group *groups, int ngroups, size_t *bytes) {
    if (!bytes) return SEMAX_EINVAL;
    int st = check_groups(groups, ngroups);
    if (st != SEMAX_OK) return st;
    *bytes = 256;  // the work counter (kept on its own 256-byte line)
    return SEMAX_OK;
}

extern "C" int sem_ax_batched(const semax_group *groups, int ngroups, void *workspace,
                              size_t ws_bytes, void *stream) {
    int st = check_groups(groups, ngroups);
    if (st != SEMAX_OK) return st;
    if (!workspace || ws_bytes < 256) return SEMAX_EWORKSPACE;
    if (!aligned16(workspace)) return SEMAX_EALIGN;
    std::vector<TileChoice> ch(17);
    for (int n = 2; n <= 16; ++n) ch[n] = default_choice(n);
    BatchParams P;
    build_params(P, groups, ngroups, ch);
    return launch_batched(P, (unsigned long long *)workspace, (cudaStream_t)stream);
}

// ---------------------------------------------------------------- plans and tuning

struct semax_plan {
    BatchParams P;                    // the groups of the persistent launch
    std::vector<semax_group> tc;      // SEMAX_PLAN_F64TC: the groups launched apart (own graph branches)
    std::vector<void *> prep;         // SEMAX_PLAN_F64TC_PREPARED: each tc group's prepared G, or NULL
    std::vector<TileChoice> choice;   // by n
    unsigned long long *counter = nullptr;   // 256 bytes: the work counter, and at byte 128 the status word
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned magic = 0x5e3a9u;
};

static std::string device_name() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return "unknown";
    return std::string(prop.name);
}

// Tuning cache: {"device": "...", "entries": [{"N": 7, "prec": "f64", "epb": 4, "map": 1, "us": 1.0}, ...]}
static bool read_cache(const char *path, const std::string &dev, std::vector<TileChoice> &ch,
                       std::vector<bool> &have) {
    FILE *f = std::fopen(path, "rb");
    if (!f) return false;
    std::string text;
    char tmp[4096];
    size_t got;
    while ((got = std::fread(tmp, 1, sizeof tmp, f)) > 0) text.append(tmp, got);
    std::fclose(f);
    const std::string key = "\"device\": \"" + dev + "\"";
    if (text.find(key) == std::string::npos) return false;
    size_t pos = 0;
    while ((pos = text.find("{\"N\":", pos)) != std::string::npos) {
        int N = 0, epb = 0, map = 0;
        if (std::sscanf(text.c_str() + pos, "{\"N\": %d, \"prec\": \"f64\", \"epb\": %d, \"map\": %d", &N, &epb,
                        &map) == 3 &&
            N >= 1 && N <= kMaxN && choice_valid(N + 1, TileChoice{epb, map})) {
            ch[N + 1] = TileChoice{epb, map};
            have[N + 1] = true;
        }
        pos += 5;
    }
    return true;
}

static bool write_cache(const char *path, const std::string &dev, const std::vector<TileChoice> &ch,
                        const std::vector<bool> &have, const std::vector<float> &us) {
    std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return false;
    std::fprintf(f, "{\"device\": \"%s\", \"entries\": [", dev.c_str());
    bool first = true;
    for (int n = 2; n <= 16; ++n) {
        if (!have[n]) continue;
        std::fprintf(f, "%s\n  {\"N\": %d, \"prec\": \"f64\", \"epb\": %d, \"map\": %d, \"us\": %.3f}",
                     first ? "" : ",", n - 1, ch[n].epb, ch[n].map, us[n]);
        first = false;
    }
    std::fprintf(f, "\n]}\n");
    const bool ok = std::fclose(f) == 0;
    return ok && std::rename(tmp.c_str(), path) == 0;
}

// Time one order's group alone with a candidate choice (median of reps).
static int time_candidate(const semax_group &g, TileChoice c, unsigned long long *counter,
                          cudaStream_t s, float *us_out) {
    std::vector<TileChoice> ch(17, c);
    BatchParams P;
    build_params(P, &g, 1, ch);
    cudaEvent_t a, b;
    int st = cuda_status(cudaEventCreate(&a));
    if (st != SEMAX_OK) return st;
    st = cuda_status(cudaEventCreate(&b));
    if (st != SEMAX_OK) { cudaEventDestroy(a); return st; }
    std::vector<float> t;
    for (int r = 0; r < 8 && st == SEMAX_OK; ++r) {
        st = cuda_status(cudaEventRecord(a, s));
        if (st == SEMAX_OK) st = launch_batched(P, counter, s);
        if (st == SEMAX_OK) st = cuda_status(cudaEventRecord(b, s));
        if (st == SEMAX_OK) st = cuda_status(cudaEventSynchronize(b));
        float ms = 0.f;
        if (st == SEMAX_OK) st = cuda_status(cudaEventElapsedTime(&ms, a, b));
        if (r >= 2) t.push_back(ms * 1000.f);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != SEMAX_OK) return st;
    std::sort(t.begin(), t.end());
    *us_out = t[t.size() / 2];
    return SEMAX_OK;
}

static std::vector<TileChoice> candidates(int n) {
    std::vector<TileChoice> out;
    const int cols = n * n;
    for (int epb = 1; epb * cols <= kBatchThreads; epb *= 2) out.push_back({epb, MAP_COLUMN});
    if (kBatchThreads / cols >= 1 && (kBatchThreads / cols) & (kBatchThreads / cols - 1))
        out.push_back({kBatchThreads / cols, MAP_COLUMN});
    for (int epb = 1; epb <= 16; epb *= 2) out.push_back({epb, MAP_NODE});
    if (n % 2 == 0)
        for (int epb = 1; epb <= 16; epb *= 2) out.push_back({epb, MAP_EO});
    std::vector<TileChoice> ok;
    for (auto c : out)
        if (choice_valid(n, c)) ok.push_back(c);
    return ok;
}

static int *plan_status(semax_plan *p) { return reinterpret_cast<int *>(reinterpret_cast<char *>(p->counter) + 128); }

static void destroy_plan(semax_plan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->counter) cudaFree(p->counter);
    for (void *b : p->prep)
        if (b) cudaFree(b);
    p->magic = 0;
    delete p;
}

extern "C" int sem_ax_plan_create(semax_plan **plan, const semax_group *groups, int ngroups, int tune,
                                  const char *cache_path, int flags) {
    if (!plan) return SEMAX_EINVAL;
    *plan = nullptr;
    if (flags & ~(SEMAX_PLAN_F64X | SEMAX_PLAN_F64TC | SEMAX_PLAN_F64TC_PREPARED)) return SEMAX_EINVAL;
    if ((flags & SEMAX_PLAN_F64TC_PREPARED) && !(flags & SEMAX_PLAN_F64TC)) return SEMAX_EINVAL;
    int st = check_groups(groups, ngroups);
    if (st != SEMAX_OK) return st;
    semax_plan *p = new semax_plan();
    // SEMAX_PLAN_F64TC: orders 7 and 15 leave the persistent launch for the
    // tensor-core FP64-accurate kernels; with SEMAX_PLAN_F64X as well, every
    // group of even n does (orders other than 7 and 15 then run sem_ax_f64x's
    // kernel).  Each such launch is captured on a branch of its own beside the
    // persistent launch, so that groups too small to fill the GPU alone share it.
    const bool all_even_apart = (flags & SEMAX_PLAN_F64TC) && (flags & SEMAX_PLAN_F64X);
    std::vector<semax_group> rest;
    for (int q = 0; q < ngroups; ++q) {
        const int N = groups[q].N;
        if ((flags & SEMAX_PLAN_F64TC) && (N == 7 || N == 15 || (all_even_apart && (N + 1) % 2 == 0)))
            p->tc.push_back(groups[q]);
        else
            rest.push_back(groups[q]);
    }
    // longest first: nodes, the double-float kernel counted at twice the
    // tensor-core one's cost per node
    std::stable_sort(p->tc.begin(), p->tc.end(), [](const semax_group &a, const semax_group &b) {
        auto cost = [](const semax_group &g) {
            const double n3 = (double)(g.N + 1) * (g.N + 1) * (g.N + 1);
            return (double)g.E * n3 * ((g.N == 7 || g.N == 15) ? 1.0 : 2.0);
        };
        return cost(a) > cost(b);
    });
    p->choice.assign(17, TileChoice{1, MAP_COLUMN});
    for (int n = 2; n <= 16; ++n) p->choice[n] = default_choice(n);
    std::vector<bool> have(17, false);
    std::vector<float> us(17, 0.f);
    const std::string dev = device_name();
    if (cache_path && !tune) read_cache(cache_path, dev, p->choice, have);

    st = cuda_status(cudaMalloc(&p->counter, 256));
    if (st == SEMAX_OK) st = cuda_status(cudaMemset(p->counter, 0, 256));
    cudaStream_t cs = nullptr;
    if (st == SEMAX_OK) st = cuda_status(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));

    if (st == SEMAX_OK && tune) {
        // the largest group of each order stands for that order
        for (int n = 2; n <= 16 && st == SEMAX_OK; ++n) {
            if ((flags & SEMAX_PLAN_F64X) && n % 2 == 0) continue;   // fixed double-float tile
            int best_g = -1;
            for (int q = 0; q < (int)rest.size(); ++q)
                if (rest[q].N + 1 == n && rest[q].E > 0 && (best_g < 0 || rest[q].E > rest[best_g].E))
                    best_g = q;
            if (best_g < 0) continue;
            float best = 1e30f;
            for (TileChoice c : candidates(n)) {
                float t = 0.f;
                st = time_candidate(rest[best_g], c, p->counter, cs, &t);
                if (st != SEMAX_OK) break;
                if (t < best) { best = t; p->choice[n] = c; }
            }
            have[n] = true;
            us[n] = best;
        }
        if (st == SEMAX_OK && cache_path && !write_cache(cache_path, dev, p->choice, have, us)) st = SEMAX_EIO;
    }

    if (st == SEMAX_OK && (flags & SEMAX_PLAN_F64X))
        for (int n = 2; n <= 16; n += 2) p->choice[n] = TileChoice{f64x_epb(n), MAP_F64X};
    // SEMAX_PLAN_F64TC_PREPARED: the geometric factor of the groups of order
    // 7 and 15 split once, now, into buffers the plan owns
    p->prep.assign(p->tc.size(), nullptr);
    if (st == SEMAX_OK && (flags & SEMAX_PLAN_F64TC_PREPARED)) {
        for (size_t q = 0; q < p->tc.size() && st == SEMAX_OK; ++q) {
            const semax_group &g = p->tc[q];
            if (g.E <= 0 || (g.N != 7 && g.N != 15)) continue;
            size_t bytes = 0;
            st = sem_ax_f64tc_prepare_size(g.E, g.N, &bytes);
            if (st == SEMAX_OK) st = cuda_status(cudaMalloc(&p->prep[q], bytes));
            if (st == SEMAX_OK) st = sem_ax_f64tc_prepare(g.E, g.N, g.G, p->prep[q], cs);
        }
        if (st == SEMAX_OK) st = cuda_status(cudaStreamSynchronize(cs));
    }
    // up to kBranches forked streams, the groups launched apart dealt to them in turn
    constexpr int kBranches = 8;
    const int nb = std::min<int>((int)p->tc.size(), kBranches);
    cudaStream_t cs2[kBranches] = {};
    cudaEvent_t fork = nullptr, join[kBranches] = {};
    if (st == SEMAX_OK && nb > 0) {
        st = cuda_status(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        for (int b = 0; b < nb && st == SEMAX_OK; ++b) {
            st = cuda_status(cudaStreamCreateWithFlags(&cs2[b], cudaStreamNonBlocking));
            if (st == SEMAX_OK) st = cuda_status(cudaEventCreateWithFlags(&join[b], cudaEventDisableTiming));
        }
    }
    if (st == SEMAX_OK) {
        build_params(p->P, rest.data(), (int)rest.size(), p->choice);
        LaunchShape ls;
        if (!rest.empty()) st = prepare_batched(p->P, &ls);
        if (st == SEMAX_OK) st = cuda_status(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        if (st == SEMAX_OK) {
            int lst = SEMAX_OK;
            if (nb > 0) {   // fork: the groups launched apart on their branches, joined back before the end
                lst = cuda_status(cudaEventRecord(fork, cs));
                for (int b = 0; b < nb && lst == SEMAX_OK; ++b) lst = cuda_status(cudaStreamWaitEvent(cs2[b], fork, 0));
                for (size_t q = 0; q < p->tc.size() && lst == SEMAX_OK; ++q) {
                    const semax_group &g = p->tc[q];   // sem_ax_f64tc_status runs sem_ax_f64x's kernel for other orders
                    if (g.E > 0 && p->prep[q])
                        lst = sem_ax_f64tc_prepared_status(g.E, g.N, g.u, p->prep[q], g.D, g.w, plan_status(p),
                                                           cs2[q % nb]);
                    else if (g.E > 0)
                        lst = sem_ax_f64tc_status(g.E, g.N, g.u, g.G, g.D, g.w, plan_status(p), cs2[q % nb]);
                }
                for (int b = 0; b < nb && lst == SEMAX_OK; ++b) lst = cuda_status(cudaEventRecord(join[b], cs2[b]));
            }
            if (lst == SEMAX_OK && !rest.empty()) lst = enqueue_batched(p->P, ls, p->counter, cs);
            for (int b = 0; b < nb; ++b) {
                const int jst = cuda_status(cudaStreamWaitEvent(cs, join[b], 0));
                if (lst == SEMAX_OK) lst = jst;
            }
            int est = cuda_status(cudaStreamEndCapture(cs, &p->graph));
            st = lst != SEMAX_OK ? lst : est;
        }
        if (st == SEMAX_OK) st = cuda_status(cudaGraphInstantiate(&p->exec, p->graph, 0));
    }
    if (fork) cudaEventDestroy(fork);
    for (int b = 0; b < nb; ++b) {
        if (join[b]) cudaEventDestroy(join[b]);
        if (cs2[b]) cudaStreamDestroy(cs2[b]);
    }
    if (cs) cudaStreamDestroy(cs);
    if (st != SEMAX_OK) {
        destroy_plan(p);
        return st;
    }
    *plan = p;
    return SEMAX_OK;
}

extern "C" int sem_ax_plan_exec(semax_plan *plan, void *stream) {
    if (!plan || plan->magic != 0x5e3a9u) return SEMAX_ENOPLAN;
    return cuda_status(cudaGraphLaunch(plan->exec, (cudaStream_t)stream));
}

extern "C" int sem_ax_plan_status(semax_plan *plan, void *stream) {
    if (!plan || plan->magic != 0x5e3a9u) return SEMAX_ENOPLAN;
    cudaStream_t s = (cudaStream_t)stream;
    int h = SEMAX_OK;
    int st = cuda_status(cudaMemcpyAsync(&h, plan_status(plan), sizeof h, cudaMemcpyDeviceToHost, s));
    if (st == SEMAX_OK) st = cuda_status(cudaMemsetAsync(plan_status(plan), 0, sizeof h, s));
    if (st == SEMAX_OK) st = cuda_status(cudaStreamSynchronize(s));
    if (st != SEMAX_OK) return st;
    return h == SEMAX_ETIMEOUT ? SEMAX_ETIMEOUT : SEMAX_OK;
}

extern "C" int sem_ax_plan_destroy(semax_plan *plan) {
    if (!plan || plan->magic != 0x5e3a9u) return SEMAX_ENOPLAN;
    destroy_plan(plan);
    return SEMAX_OK;
}

extern "C" int sem_ax_plan_config(const semax_plan *plan, int N, int *elems_per_tile, int *mapping) {
    if (!plan || plan->magic != 0x5e3a9u) return SEMAX_ENOPLAN;
    for (const semax_group &g : plan->tc) {
        if (g.N == N) {   // launched apart: the tensor-core kernel (one element per CTA pass) or sem_ax_f64x's
            const bool tcn = N == 7 || N == 15;
            if (elems_per_tile) *elems_per_tile = tcn ? 1 : f64x_epb(N + 1);
            if (mapping) *mapping = tcn ? MAP_F64TC : MAP_F64X;
            return SEMAX_OK;
        }
    }
    for (int q = 0; q < plan->P.ngroups; ++q) {
        if (plan->P.g[q].n == N + 1) {
            if (elems_per_tile) *elems_per_tile = plan->P.g[q].epb;
            if (mapping) *mapping = plan->P.g[q].map;
            return SEMAX_OK;
        }
    }
    return SEMAX_EINVAL;
}
