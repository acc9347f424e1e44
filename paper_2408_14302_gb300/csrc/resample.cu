// Resample-first reading of the hop (paper Sec. III.B, Fig. 2): the signal is
// re-sampled at the hop spacing, y[m] = x[m H], and the CWT is evaluated at
// every sample of y with scales a / H.  This kernel forms y (and the clip
// lengths of y) on the device; the transform of y is the ordinary hop-1 path.
#include "cwth_internal.h"

namespace cwth {
namespace {

// y[b][m] = x[b][m H] for m < ceil(len_b / H), else 0, m < ld_y; len_y[b] =
// ceil(len_b / H) when len_y is given.
__global__ void resample_kernel(const float* __restrict__ x, int64_t ld_x,
                                const int64_t* __restrict__ lengths, int64_t in_len, int32_t H,
                                float* __restrict__ y, int64_t ld_y, int64_t* __restrict__ len_y) {
    const int b = blockIdx.y;
    int64_t len = lengths ? lengths[b] : in_len;
    len = len < 0 ? 0 : (len > in_len ? in_len : len);
    const int64_t ly = (len + H - 1) / H;
    const float* xr = x + (int64_t)b * ld_x;
    float* yr = y + (int64_t)b * ld_y;
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < ld_y;
         m += (int64_t)gridDim.x * blockDim.x)
        yr[m] = m < ly ? __ldg(xr + m * H) : 0.f;
    if (len_y && blockIdx.x == 0 && threadIdx.x == 0) len_y[b] = ly;
}

}  // namespace

cudaError_t resample_launch(const float* x, int64_t ld_x, const int64_t* lengths, int64_t in_len,
                            int32_t H, float* y, int64_t ld_y, int64_t* len_y, int batch,
                            cudaStream_t st) {
    const unsigned bx = (unsigned)std::min<int64_t>((ld_y + 255) / 256, 4096);
    dim3 grid(bx > 0 ? bx : 1, (unsigned)batch);
    resample_kernel<<<grid, 256, 0, st>>>(x, ld_x, lengths, in_len, H, y, ld_y, len_y);
    return cudaGetLastError();
}

}  // namespace cwth
