// Instantiations of the matrix-free slab operator (stencil_impl.cuh) for FP64
// and FP32 data in their own arithmetic.
#include "stencil_impl.cuh"

namespace st {

template cudaError_t launch_stencil<double, double>(const double *, const double *, double *,
                                                    const Bands<double> &, const Grid &,
                                                    const TimeCoefs<double> &, int, int, int,
                                                    cudaStream_t, int);
template cudaError_t launch_stencil<float, float>(const float *, const float *, float *,
                                                  const Bands<float> &, const Grid &,
                                                  const TimeCoefs<float> &, int, int, int,
                                                  cudaStream_t, int);

}  // namespace st
