// Spectral path of the hop-size CWT: the 512-thread kernels, the batch work
// list, the tables and the launches.  The device code is in
// spectral_kernel.cuh; the 1024-thread kernels compile in spectral_solo.cu.
#include "spectral_kernel.cuh"

namespace cwth {
namespace {

// Two-level table: entries i < M/128 hold exp(-2 pi i 128 i / M), the next
// 128 hold exp(-2 pi i j / M); float64, rounded once to float32.
__global__ void twiddle_kernel(float2* tw, int M) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n1 = M >> 7;
    if (i < n1 + 128) {
        const double m = i < n1 ? 128.0 * i : (double)(i - n1);
        double s, c;
        sincospi(2.0 * m / (double)M, &s, &c);
        tw[i] = make_float2((float)c, (float)-s);
    }
}

// Tap tables of the fused time-domain scales, float64 then rounded once:
// table g, row tau, column j holds g_j[t] = a^{-1/2} conj(psi(t / a)) =
// a^{-1/2} (pi B)^{-1/2} exp(-(t/a)^2 / B) exp(-2 pi i C t / a) at
// t = tau - hg for |t| <= h_j, zero elsewhere and in padding columns.
// gidx[g * kFdMaxG + j] is the fused-scale index of column j.
__global__ void fd_taps_kernel(const double* __restrict__ scales, const int32_t* __restrict__ h_of,
                               const int32_t* __restrict__ gidx, const FdGroup* __restrict__ grp,
                               double B, double C, float2* __restrict__ taps) {
    const FdGroup g = grp[blockIdx.x];
    const int n = (2 * g.hg + 1) * g.gp;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int tau = i / g.gp, j = i - tau * g.gp;
        const int t = tau - g.hg;
        float2 v = make_float2(0.f, 0.f);
        if (j < g.n) {
            const int s = gidx[blockIdx.x * kFdMaxG + j];
            if (t >= -h_of[s] && t <= h_of[s]) {
                const double a = scales[s];
                const double u = (double)t / a;
                const double env = exp(-(u * u) / B) / sqrt(a * M_PI * B);
                double sn, cs;
                sincospi(2.0 * C * u, &sn, &cs);
                v = make_float2((float)(env * cs), (float)(-env * sn));
            }
        }
        taps[g.off + i] = v;
    }
}

}  // namespace

size_t spectral_smem_bytes(int M, int P, int nconc, size_t fd_bytes) {
    const size_t z = std::max((size_t)nconc * P * sizeof(float2), fd_bytes);
    return (size_t)(spectral_twiddle_entries(M) + M / 2 + 2) * sizeof(float2) + z;
}

size_t spectral_fd_bytes(int taps_n, int hw, int fst, int n_groups) {
    if (taps_n <= 0) return 0;
    return (size_t)taps_n * sizeof(float2) + (size_t)n_groups * sizeof(FdGroup) +
           (((size_t)(2 * hw + 1) * fst + 4) * sizeof(float) + 15) / 16 * 16;
}

cudaError_t spectral_make_fd_taps(const double* d_scales, const int32_t* d_h, const int32_t* d_gidx,
                                  const FdGroup* d_grp, int n_groups, int taps_n, double B,
                                  double C, float2* d_taps, cudaStream_t st) {
    if (n_groups <= 0) return cudaSuccess;
    (void)taps_n;
    fd_taps_kernel<<<n_groups, 256, 0, st>>>(d_scales, d_h, d_gidx, d_grp, B, C, d_taps);
    return cudaGetLastError();
}

int spectral_twiddle_entries(int M) { return (M >> 7) + 128; }

cudaError_t spectral_prepare_device() {
    cudaError_t e = cudaSuccess;
    for (const void* f : {(const void*)spectral_worklist_kernel<kSpecThreadsPair>,
                          (const void*)spectral_segment_kernel<kSpecThreadsPair, false>,
                          (const void*)spectral_segment_kernel<kSpecThreadsPair, true>})
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     227 * 1024 - 1024);
    if (e == cudaSuccess) e = spectral_prepare_solo();
    return e;
}

cudaError_t spectral_worklist_launch(const SpecWorkList& wl, size_t smem, cudaStream_t st) {
    if (wl.n_items <= 0) return cudaSuccess;
    spectral_worklist_kernel<kSpecThreadsPair><<<wl.n_items, kSpecThreadsPair, smem, st>>>(wl);
    return cudaGetLastError();
}

cudaError_t spectral_make_twiddles(float2* d_tw, int M, cudaStream_t st) {
    twiddle_kernel<<<(spectral_twiddle_entries(M) + 255) / 256, 256, 0, st>>>(d_tw, M);
    return cudaGetLastError();
}

cudaError_t spectral_launch(const SpecLaunch& L, int threads, bool prune, int n_seg, int batch,
                            int n_groups, size_t smem, cudaStream_t st, bool dependent) {
    dim3 grid(n_seg, batch, n_groups);
    if (threads == kSpecThreadsSolo)
        return spectral_launch_solo(L, prune, grid, smem, st, dependent);
    if (dependent)
        return spectral_launch_dependent(
            prune ? spectral_segment_kernel<kSpecThreadsPair, true>
                  : spectral_segment_kernel<kSpecThreadsPair, false>,
            L, grid, kSpecThreadsPair, smem, st);
    if (prune)
        spectral_segment_kernel<kSpecThreadsPair, true><<<grid, kSpecThreadsPair, smem, st>>>(L);
    else
        spectral_segment_kernel<kSpecThreadsPair, false><<<grid, kSpecThreadsPair, smem, st>>>(L);
    return cudaGetLastError();
}

}  // namespace cwth
