// De-dispersion kernel instantiations for FP32 input.
#include "dd_kernel.cuh"

namespace dd {

cudaError_t launch_kernel_f32(const KArgs &a, unsigned grid, int threads, int smem,
                             cudaStream_t s, int dthr, int nw) {
    return launch_elem<4>(a, grid, threads, smem, s, dthr, nw);
}

}  // namespace dd
