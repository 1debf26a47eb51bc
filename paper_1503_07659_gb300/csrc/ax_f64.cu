// FP64 instantiation of the plain Ax kernels.
#include "ax_plain.cuh"

namespace semax {
template int launch_plain<double, false>(int64_t, int, const TileConfig &, const double *, const double *,
                                         const double *, double *, const double *, Helm<double>, cudaStream_t);
}  // namespace semax
