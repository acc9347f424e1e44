// Spectral path of the hop-size CWT: the 1024-thread kernels (one CTA per
// SM, for segments whose inverse FFT does not fit beside the spectrum in the
// paired shape).  The device code is in spectral_kernel.cuh.
#include "spectral_kernel.cuh"

namespace cwth {

cudaError_t spectral_prepare_solo() {
    cudaError_t e = cudaSuccess;
    for (const void* f : {(const void*)spectral_segment_kernel<kSpecThreadsSolo, false>,
                          (const void*)spectral_segment_kernel<kSpecThreadsSolo, true>})
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     227 * 1024 - 1024);
    return e;
}

cudaError_t spectral_launch_solo(const SpecLaunch& L, bool prune, dim3 grid, size_t smem,
                                 cudaStream_t st, bool dependent) {
    if (dependent)
        return spectral_launch_dependent(
            prune ? spectral_segment_kernel<kSpecThreadsSolo, true>
                  : spectral_segment_kernel<kSpecThreadsSolo, false>,
            L, grid, kSpecThreadsSolo, smem, st);
    if (prune)
        spectral_segment_kernel<kSpecThreadsSolo, true><<<grid, kSpecThreadsSolo, smem, st>>>(L);
    else
        spectral_segment_kernel<kSpecThreadsSolo, false><<<grid, kSpecThreadsSolo, smem, st>>>(L);
    return cudaGetLastError();
}

}  // namespace cwth
