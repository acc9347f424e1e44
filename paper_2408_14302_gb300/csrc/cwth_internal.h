// Internal declarations shared by the translation units of libcwth.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "cwth.h"

namespace cwth {

constexpr uint32_t kPlanMagic = 0xC0A7B17Eu;
constexpr int kSpecThreads = 512;
// Largest batched shared-memory FFT (complex points) one CTA performs: at
// most 16 points per thread per pass.
constexpr int kMaxFftPoints = 16 * kSpecThreads;

// Per-scale parameters of the spectral path (one entry per spectral scale).
// The multiplier at unwrapped bin q_u is
//     gscale * exp2(kexp * (q_u * a_over_m - C)^2)
// i.e. sqrt(a)/M * Psi(a q_u / M) with Psi(f) = exp(-pi^2 B (f - C)^2); the
// band [q_lo, q_hi] holds every q_u where Psi exceeds the band threshold.
// Iterating over unwrapped q_u and reducing it mod M sums the Poisson
// aliases of the sampled wavelet's spectrum.
struct SpecScale {
    float a_over_m;
    float gscale;
    int32_t q_lo;
    int32_t q_hi;
    int32_t row;     // output row (index into the caller's scale list)
    int32_t pad_[3];
};

struct SpecLaunch {
    const float* x;
    int64_t ld_x;
    const int64_t* lengths;
    int64_t max_len;
    float* out;
    int64_t frames_max;
    int32_t S_total;
    int32_t hop;
    int32_t M;         // segment length
    int32_t P;         // M / hop
    int32_t halo;      // left context, a multiple of hop
    int32_t kp0;       // halo / hop: first valid local frame
    int32_t seg_frames;
    int32_t n_sp;      // spectral scales
    int32_t group_size;
    int32_t nconc;     // scales folded and inverted together
    float center;
    float kexp;        // -pi^2 B log2(e)
    const float2* tw;  // exp(-2 pi i m / M), m < M
    const SpecScale* sc;
};

size_t spectral_smem_bytes(int M, int P, int nconc);
cudaError_t spectral_prepare_device();
cudaError_t spectral_make_twiddles(float2* d_tw, int M, cudaStream_t st);
cudaError_t spectral_launch(const SpecLaunch& L, int n_seg, int batch, int n_groups,
                            size_t smem, cudaStream_t st);

}  // namespace cwth

struct cwth_plan_s {
    uint32_t magic = 0;
    int device = 0;
    double B = 0, C = 0, fs = 0;
    int32_t S = 0, hop = 0, precision = 0, path = 0;
    int64_t max_len = 0, frames_max = 0;
    std::vector<double> scales;
    std::vector<int32_t> scale_path;

    // spectral path
    int32_t n_sp = 0;
    int32_t M = 0, P = 0, halo = 0, kp0 = 0, seg_frames = 0, n_seg = 0;
    float2* d_tw = nullptr;
    cwth::SpecScale* d_sp = nullptr;

    // direct path
    int32_t n_dir = 0;
    int32_t dir_taps = 0;

    int64_t table_bytes = 0;

    // host-API staging (grown on demand)
    float* d_stage_x = nullptr;
    size_t stage_x_elems = 0;
    float* d_stage_out = nullptr;
    size_t stage_out_elems = 0;
    int64_t* d_stage_len = nullptr;
    size_t stage_len_elems = 0;
};
