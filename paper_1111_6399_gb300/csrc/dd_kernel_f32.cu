// De-dispersion kernel instantiations for FP32 input.
#include "dd_kernel_tm.cuh"

namespace dd {

cudaError_t launch_kernel_f32(const KArgs &a, unsigned grid, int threads, int smem,
                             cudaStream_t s, int dthr, int nw) {
    if (nw == 17)  // the TMEM-window kernel (dd_kernel_tm.cuh)
        return launch_tm<4>(a, grid, threads, smem, s);
    return launch_elem<4>(a, grid, threads, smem, s, dthr, nw);
}

}  // namespace dd
