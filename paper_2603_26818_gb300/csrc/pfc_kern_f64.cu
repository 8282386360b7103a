// FP64 instantiation of the pass and reduction kernels, and the precision-free finish kernel.
#include "pfc_kern.cuh"

namespace pfc {
PFC_INSTANTIATE_LAUNCH(double)

void launch_finish(cudaStream_t s, const double *partials, int nb, double scale, double *out,
                   bool accumulate) {
    k_finish<<<1, RED_THREADS, 0, s>>>(partials, nb, scale, out, accumulate ? 1 : 0);
}
}  // namespace pfc
