// De-dispersion kernel instantiations for FP16 input.
#include "dd_kernel.cuh"

namespace dd {

cudaError_t launch_kernel_f16(const KArgs &a, unsigned grid, int threads, int smem,
                             cudaStream_t s, int dthr, int nw) {
    return launch_elem<2>(a, grid, threads, smem, s, dthr, nw);
}

}  // namespace dd
