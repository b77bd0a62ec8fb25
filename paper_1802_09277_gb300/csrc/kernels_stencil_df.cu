// Instantiation of the matrix-free slab operator (stencil_impl.cuh) on FP64
// data in double-float arithmetic: the residual of the mixed-precision
// refinement.  N_t = 3 .. 6 get kernels with N_t fixed at compile time.
#include "stencil_impl.cuh"

namespace st {

template cudaError_t launch_stencil<double, dfloat>(const double *, const double *, double *,
                                                    const Bands<double> &, const Grid &,
                                                    const TimeCoefs<dfloat> &, int, int, int,
                                                    cudaStream_t, int);

}  // namespace st
