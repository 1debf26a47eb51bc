// FP64 Helmholtz instantiation of the plain kernels: w = h1 A u + h2 B u.
#include "ax_plain.cuh"

namespace semax {
template int launch_plain<double, true>(int64_t, int, const TileConfig &, const double *, const double *,
                                        const double *, double *, const double *, Helm<double>, cudaStream_t);
}  // namespace semax
