// De-dispersion kernel instantiations for uint8 input.
#include "dd_kernel.cuh"

namespace dd {

cudaError_t launch_kernel_u8(const KArgs &a, unsigned grid, int threads, int smem,
                             cudaStream_t s, int dthr, int nw) {
    return launch_elem<1>(a, grid, threads, smem, s, dthr, nw);
}

cudaError_t launch_planes_u8(const uint8_t *in, int64_t pitch_b, int nchan, int64_t nsamp_in,
                             uint8_t *planes, int64_t plane_stride, cudaStream_t s) {
    return launch_planes_elem<1>(in, pitch_b, nchan, nsamp_in, planes, plane_stride, s);
}

}  // namespace dd
