// C ABI of libsemax: the plain FP64 / FP32 entry points, status strings and
// device queries.  Argument checks happen here, before anything is queued.
#include <atomic>

#include "ax_plain.cuh"

namespace semax {

int &last_cuda_error() {
    static thread_local int err = 0;
    return err;
}

static std::atomic<int> g_wait_polls{kDefaultWaitPolls};
int first_wait_polls() { return g_wait_polls.load(std::memory_order_relaxed); }

int device_sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return kNumSMsHint;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return kNumSMsHint;
    return sms;
}

}  // namespace semax

using namespace semax;

extern "C" int sem_ax(int64_t E, int N, const double *u, const double *G, const double *D,
                      double *w, void *stream) {
    int st = check_args(E, N, u, G, D, w);
    if (st != SEMAX_OK || E == 0) return st;
    return launch_plain<double>(E, N, default_tile<double>(N + 1), u, G, D, w, nullptr,
                                Helm<double>{nullptr, 1.0, 0.0}, (cudaStream_t)stream);
}

extern "C" int sem_ax_f32(int64_t E, int N, const float *u, const float *G, const float *D,
                          float *w, const float *G_scale, void *stream) {
    int st = check_args(E, N, u, G, D, w);
    if (st != SEMAX_OK || E == 0) return st;
    if (G_scale && overlaps(w, (size_t)E * (N + 1) * (N + 1) * (N + 1) * sizeof(float), G_scale,
                            (size_t)E * sizeof(float)))
        return SEMAX_EALIAS;
    return launch_plain<float>(E, N, default_tile<float>(N + 1), u, G, D, w, G_scale,
                               Helm<float>{nullptr, 1.0f, 0.0f}, (cudaStream_t)stream);
}

extern "C" int sem_ax_helmholtz(int64_t E, int N, const double *u, const double *G, const double *B,
                                const double *D, double h1, double h2, double *w, void *stream) {
    int st = check_args(E, N, u, G, D, w);
    if (st != SEMAX_OK || E == 0) return st;
    if (!B) return SEMAX_EINVAL;
    if (!aligned16(B)) return SEMAX_EALIGN;
    const size_t ub = (size_t)E * (N + 1) * (N + 1) * (N + 1) * sizeof(double);
    if (overlaps(w, ub, B, ub)) return SEMAX_EALIAS;
    return launch_plain<double, true>(E, N, default_tile<double>(N + 1), u, G, D, w, nullptr,
                                      Helm<double>{B, h1, h2}, (cudaStream_t)stream);
}

extern "C" const char *semax_strerror(int status) {
    switch (status) {
        case SEMAX_OK: return "ok";
        case SEMAX_EINVAL: return "invalid argument (count, NULL pointer or option)";
        case SEMAX_EUNSUPPORTED_N: return "unsupported polynomial order (need 1 <= N <= 15)";
        case SEMAX_EALIGN: return "array not 16-byte aligned";
        case SEMAX_EALIAS: return "output overlaps an input";
        case SEMAX_ECUDA: return "CUDA runtime error (see semax_last_cuda_error)";
        case SEMAX_ETIMEOUT: return "device-side wait timed out";
        case SEMAX_ENOPLAN: return "no plan";
        case SEMAX_EWORKSPACE: return "workspace missing or too small";
        case SEMAX_EIO: return "tuning cache I/O error";
        default: return "unknown status";
    }
}

extern "C" int semax_last_cuda_error(void) { return last_cuda_error(); }

extern "C" int semax_set_wait_polls(int polls) {
    g_wait_polls.store(polls < 0 ? kDefaultWaitPolls : polls, std::memory_order_relaxed);
    return SEMAX_OK;
}
