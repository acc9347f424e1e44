// C ABI of libcwth.so: argument checking, planning, launches (include/cwth.h).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "cwth_internal.h"

using cwth::SpecLaunch;
using cwth::SpecScale;

namespace {

// Wavelet tail left outside a segment: taps below this fraction of the peak
// may wrap around the segment (the segment halo covers everything above it).
constexpr double kEpsWrap = 1e-10;
// Morlet band threshold: spectrum bins where Psi(a nu) < kEpsBand are skipped.
constexpr double kEpsBand = 1e-9;
// Shared memory a spectral CTA may use.
constexpr size_t kSmemCap = 227 * 1024;
// Preferred ceiling, so that two CTAs fit on one SM.
constexpr size_t kSmemTwoPerSm = 112 * 1024;
constexpr int kNumSms = 152;

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int64_t v) {
    int e = 0;
    while ((int64_t(1) << e) < v) ++e;
    return e;
}

bool valid_plan(const cwth_plan_s* p) { return p && p->magic == cwth::kPlanMagic; }

cwth_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return CWTH_OK;
    if (e == cudaErrorMemoryAllocation) return CWTH_ERR_OOM;
    return CWTH_ERR_CUDA;
}

// Band of scale a in unwrapped bins of an M-point spectrum: Psi(a q/M) >= eps
// <=> |a q/M - C| <= delta, delta = sqrt(ln(1/eps) / (pi^2 B)).
void band_limits(double a, double B, double C, int M, int64_t* q_lo, int64_t* q_hi) {
    const double delta = sqrt(log(1.0 / kEpsBand) / (M_PI * M_PI * B));
    *q_lo = (int64_t)floor((double)M * (C - delta) / a);
    *q_hi = (int64_t)ceil((double)M * (C + delta) / a);
}

struct SegChoice {
    int M = 0, P = 0, halo = 0, kp0 = 0, seg_frames = 0, n_seg = 0;
    double cost = 0;
};

// Segment length for the spectral path: the power of two M (P = M/H >= 8,
// shared memory within bounds) minimising a lane-operation cost model of
// FFT + fold + inverse FFTs + stores per clip.
bool choose_segment(const cwth_plan_s& p, const std::vector<double>& sp_scales, SegChoice* out) {
    double a_max = 0;
    for (double a : sp_scales) a_max = std::max(a_max, a);
    const int hop = p.hop;
    const int64_t h = (int64_t)ceil(a_max * sqrt(p.B * log(1.0 / kEpsWrap)));
    const int64_t halo = ((h + hop - 1) / hop) * hop;
    const int64_t kp0 = halo / hop;
    bool found = false;
    for (int lg = 9; lg <= 15; ++lg) {
        const int64_t M = int64_t(1) << lg;
        if (M < 8 * (int64_t)hop) continue;
        const int64_t P = M / hop;
        if (M - 1 - h < 0) continue;
        const int64_t last = (M - 1 - h) / hop;
        const int64_t Fseg = last - kp0 + 1;
        if (Fseg < 1) continue;
        if (cwth::spectral_smem_bytes((int)M, (int)P, 1) > kSmemCap) continue;
        if (M / 2 > cwth::kMaxFftPoints || P > cwth::kMaxFftPoints) continue;
        const int64_t n_seg = (p.frames_max + Fseg - 1) / Fseg;
        double fold = 0;
        for (double a : sp_scales) {
            int64_t lo, hi;
            band_limits(a, p.B, p.C, (int)M, &lo, &hi);
            fold += 12.0 * (double)(hi - lo + 1) + 4.0 * (double)P;
        }
        const double fft = 2.5 * (double)(M / 2) * (lg - 1) + 8.0 * (double)M;
        const double ifft = 2.5 * (double)P * ilog2(P) * (double)sp_scales.size();
        const double store = 2.0 * (double)Fseg * (double)sp_scales.size();
        const double cost = (double)n_seg * (fft + fold + ifft + store);
        if (!found || cost < out->cost) {
            found = true;
            out->M = (int)M;
            out->P = (int)P;
            out->halo = (int)halo;
            out->kp0 = (int)kp0;
            out->seg_frames = (int)Fseg;
            out->n_seg = (int)n_seg;
            out->cost = cost;
        }
    }
    return found;
}

void free_plan_memory(cwth_plan_s* p) {
    cudaFree(p->d_tw);
    cudaFree(p->d_sp);
    cudaFree(p->d_stage_x);
    cudaFree(p->d_stage_out);
    cudaFree(p->d_stage_len);
    p->d_tw = nullptr;
    p->d_sp = nullptr;
    p->d_stage_x = nullptr;
    p->d_stage_out = nullptr;
    p->d_stage_len = nullptr;
}

cwth_status build_spectral(cwth_plan_s* p) {
    std::vector<double> sp;
    std::vector<int32_t> rows;
    for (int s = 0; s < p->S; ++s)
        if (p->scale_path[s] == CWTH_PATH_SPECTRAL) {
            sp.push_back(p->scales[s]);
            rows.push_back(s);
        }
    p->n_sp = (int32_t)sp.size();
    if (p->n_sp == 0) return CWTH_OK;
    if (!is_pow2(p->hop)) return CWTH_ERR_UNSUPPORTED;
    SegChoice ch;
    if (!choose_segment(*p, sp, &ch)) return CWTH_ERR_UNSUPPORTED;
    p->M = ch.M;
    p->P = ch.P;
    p->halo = ch.halo;
    p->kp0 = ch.kp0;
    p->seg_frames = ch.seg_frames;
    p->n_seg = ch.n_seg;

    std::vector<SpecScale> host(sp.size());
    for (size_t i = 0; i < sp.size(); ++i) {
        int64_t lo, hi;
        band_limits(sp[i], p->B, p->C, p->M, &lo, &hi);
        SpecScale& s = host[i];
        memset(&s, 0, sizeof(s));
        s.a_over_m = (float)(sp[i] / (double)p->M);
        s.gscale = (float)(sqrt(sp[i]) / (double)p->M);
        s.q_lo = (int32_t)lo;
        s.q_hi = (int32_t)hi;
        s.row = rows[i];
    }
    cudaError_t e = cudaMalloc(&p->d_tw, sizeof(float2) * (size_t)p->M);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaMalloc(&p->d_sp, sizeof(SpecScale) * host.size());
    if (e != cudaSuccess) return cuda_status(e);
    p->table_bytes += (int64_t)(sizeof(float2) * (size_t)p->M + sizeof(SpecScale) * host.size());
    e = cudaMemcpy(p->d_sp, host.data(), sizeof(SpecScale) * host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_status(e);
    e = cwth::spectral_make_twiddles(p->d_tw, p->M, 0);
    if (e != cudaSuccess) return cuda_status(e);
    e = cwth::spectral_prepare_device();
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaDeviceSynchronize();
    return cuda_status(e);
}

cwth_status launch_spectral(const cwth_plan_s* p, const float* d_x, int64_t ld_x,
                            const int64_t* d_len, int32_t batch, float* d_out, cudaStream_t st) {
    if (p->n_sp == 0 || batch == 0) return CWTH_OK;
    // Scale groups: enough CTAs for two waves, each group at least 8 scales.
    const int64_t base = (int64_t)p->n_seg * batch;
    int n_groups = (int)std::min<int64_t>((2 * kNumSms + base - 1) / base,
                                          std::max(1, p->n_sp / 8));
    n_groups = std::max(1, n_groups);
    const int gs = (p->n_sp + n_groups - 1) / n_groups;
    n_groups = (p->n_sp + gs - 1) / gs;
    int nconc = gs;
    const size_t cap = std::max(kSmemTwoPerSm, cwth::spectral_smem_bytes(p->M, p->P, 1));
    while (nconc > 1 && cwth::spectral_smem_bytes(p->M, p->P, nconc) > cap) --nconc;
    while (nconc > 1 && (int64_t)nconc * p->P > cwth::kMaxFftPoints) --nconc;
    if (batch > 65535 || p->n_seg > 0x7fffffff) return CWTH_ERR_UNSUPPORTED;

    SpecLaunch L;
    L.x = d_x;
    L.ld_x = ld_x;
    L.lengths = d_len;
    L.max_len = p->max_len;
    L.out = d_out;
    L.frames_max = p->frames_max;
    L.S_total = p->S;
    L.hop = p->hop;
    L.M = p->M;
    L.P = p->P;
    L.halo = p->halo;
    L.kp0 = p->kp0;
    L.seg_frames = p->seg_frames;
    L.n_sp = p->n_sp;
    L.group_size = gs;
    L.nconc = nconc;
    L.center = (float)p->C;
    L.kexp = (float)(-M_PI * M_PI * p->B / M_LN2);
    L.tw = p->d_tw;
    L.sc = p->d_sp;
    const size_t smem = cwth::spectral_smem_bytes(p->M, p->P, nconc);
    return cuda_status(cwth::spectral_launch(L, p->n_seg, batch, n_groups, smem, st));
}

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <class T>
cwth_status grow(T** ptr, size_t* have, size_t need) {
    if (*have >= need) return CWTH_OK;
    cudaFree(*ptr);
    *ptr = nullptr;
    *have = 0;
    cudaError_t e = cudaMalloc((void**)ptr, need * sizeof(T));
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return cuda_status(e);
    }
    *have = need;
    return CWTH_OK;
}

}  // namespace

extern "C" {

int64_t cwth_num_frames(int64_t n, int32_t hop) {
    if (n <= 0 || hop <= 0) return 0;
    return (n + hop - 1) / hop;
}

const char* cwth_status_string(cwth_status s) {
    switch (s) {
        case CWTH_OK: return "CWTH_OK";
        case CWTH_ERR_INVALID_ARG: return "CWTH_ERR_INVALID_ARG";
        case CWTH_ERR_OOM: return "CWTH_ERR_OOM";
        case CWTH_ERR_CUDA: return "CWTH_ERR_CUDA";
        case CWTH_ERR_UNSUPPORTED: return "CWTH_ERR_UNSUPPORTED";
        case CWTH_ERR_TIMEOUT: return "CWTH_ERR_TIMEOUT";
        case CWTH_ERR_BAD_PLAN: return "CWTH_ERR_BAD_PLAN";
    }
    return "CWTH_ERR_UNKNOWN";
}

cwth_status cwth_plan(const cwth_morlet* w, const double* scales, int32_t S, int32_t hop,
                      double sample_rate, int64_t max_len, int32_t precision, int32_t path,
                      cwth_plan_t* out) {
    if (out) *out = nullptr;
    if (!w || !scales || !out) return CWTH_ERR_INVALID_ARG;
    if (S < 1 || hop < 1 || max_len < 1) return CWTH_ERR_INVALID_ARG;
    if (!(isfinite(w->bandwidth) && w->bandwidth > 0)) return CWTH_ERR_INVALID_ARG;
    if (!(isfinite(w->center_freq) && w->center_freq > 0)) return CWTH_ERR_INVALID_ARG;
    if (!(isfinite(sample_rate) && sample_rate > 0)) return CWTH_ERR_INVALID_ARG;
    if (precision < CWTH_PREC_FP32 || precision > CWTH_PREC_BF16X2) return CWTH_ERR_INVALID_ARG;
    if (path < CWTH_PATH_AUTO || path > CWTH_PATH_DIRECT) return CWTH_ERR_INVALID_ARG;
    for (int32_t s = 0; s < S; ++s)
        if (!(isfinite(scales[s]) && scales[s] > 0)) return CWTH_ERR_INVALID_ARG;
    if (max_len > (int64_t(1) << 40)) return CWTH_ERR_UNSUPPORTED;

    cwth_plan_s* p = new (std::nothrow) cwth_plan_s();
    if (!p) return CWTH_ERR_OOM;
    cwth_status st = CWTH_OK;
    try {
        if (cudaGetDevice(&p->device) != cudaSuccess) {
            delete p;
            return CWTH_ERR_CUDA;
        }
        p->B = w->bandwidth;
        p->C = w->center_freq;
        p->fs = sample_rate;
        p->S = S;
        p->hop = hop;
        p->precision = precision;
        p->path = path;
        p->max_len = max_len;
        p->frames_max = cwth_num_frames(max_len, hop);
        p->scales.assign(scales, scales + S);
        p->scale_path.assign(S, CWTH_PATH_SPECTRAL);
        if (path == CWTH_PATH_DIRECT) st = CWTH_ERR_UNSUPPORTED;
        if (st == CWTH_OK) st = build_spectral(p);
    } catch (...) {
        st = CWTH_ERR_OOM;
    }
    if (st != CWTH_OK) {
        free_plan_memory(p);
        delete p;
        return st;
    }
    p->magic = cwth::kPlanMagic;
    *out = p;
    return CWTH_OK;
}

cwth_status cwth_execute(cwth_plan_t p, const float* d_x, int64_t ld_x, const int64_t* d_lengths,
                         int32_t batch, float* d_out, void* stream) {
    if (!valid_plan(p)) return CWTH_ERR_BAD_PLAN;
    if (batch < 0) return CWTH_ERR_INVALID_ARG;
    if (batch == 0) return CWTH_OK;
    if (!d_x || !d_out || ld_x < p->max_len) return CWTH_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    if (!g.ok) return CWTH_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    return launch_spectral(p, d_x, ld_x, d_lengths, batch, d_out, st);
}

cwth_status cwth_execute_host(cwth_plan_t p, const float* h_x, int64_t ld_x,
                              const int64_t* h_lengths, int32_t batch, float* h_out,
                              void* stream) {
    if (!valid_plan(p)) return CWTH_ERR_BAD_PLAN;
    if (batch < 0) return CWTH_ERR_INVALID_ARG;
    if (batch == 0) return CWTH_OK;
    if (!h_x || !h_out || ld_x < p->max_len) return CWTH_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    if (!g.ok) return CWTH_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nx = (size_t)batch * (size_t)ld_x;
    const size_t no = (size_t)batch * (size_t)p->S * (size_t)p->frames_max;
    cwth_status s = grow(&p->d_stage_x, &p->stage_x_elems, nx);
    if (s == CWTH_OK) s = grow(&p->d_stage_out, &p->stage_out_elems, no);
    if (s == CWTH_OK && h_lengths) s = grow(&p->d_stage_len, &p->stage_len_elems, (size_t)batch);
    if (s != CWTH_OK) return s;
    cudaError_t e = cudaMemcpyAsync(p->d_stage_x, h_x, nx * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && h_lengths)
        e = cudaMemcpyAsync(p->d_stage_len, h_lengths, (size_t)batch * sizeof(int64_t),
                            cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_status(e);
    s = launch_spectral(p, p->d_stage_x, ld_x, h_lengths ? p->d_stage_len : nullptr, batch,
                        p->d_stage_out, st);
    if (s != CWTH_OK) return s;
    if (!h_lengths) {
        e = cudaMemcpyAsync(h_out, p->d_stage_out, no * sizeof(float), cudaMemcpyDeviceToHost, st);
    } else {
        // Rows of short clips keep their trailing frames untouched in h_out:
        // copy only the written prefix of each row.
        std::vector<int64_t> F(batch);
        for (int32_t i = 0; i < batch; ++i) {
            int64_t len = std::min<int64_t>(std::max<int64_t>(h_lengths[i], 0), p->max_len);
            F[i] = cwth_num_frames(len, p->hop);
        }
        e = cudaSuccess;
        for (int32_t i = 0; i < batch && e == cudaSuccess; ++i) {
            if (F[i] == 0) continue;
            e = cudaMemcpy2DAsync(h_out + (size_t)i * p->S * p->frames_max,
                                  (size_t)p->frames_max * sizeof(float),
                                  p->d_stage_out + (size_t)i * p->S * p->frames_max,
                                  (size_t)p->frames_max * sizeof(float), (size_t)F[i] * sizeof(float),
                                  (size_t)p->S, cudaMemcpyDeviceToHost, st);
        }
    }
    if (e != cudaSuccess) return cuda_status(e);
    return cuda_status(cudaStreamSynchronize(st));
}

cwth_status cwth_destroy(cwth_plan_t p) {
    if (!p) return CWTH_OK;
    if (!valid_plan(p)) return CWTH_ERR_BAD_PLAN;
    DeviceGuard g(p->device);
    p->magic = 0;
    free_plan_memory(p);
    delete p;
    return CWTH_OK;
}

cwth_status cwth_plan_query(cwth_plan_t p, cwth_plan_info* info) {
    if (!valid_plan(p)) return CWTH_ERR_BAD_PLAN;
    if (!info) return CWTH_ERR_INVALID_ARG;
    memset(info, 0, sizeof(*info));
    info->num_scales = p->S;
    info->hop = p->hop;
    info->max_len = p->max_len;
    info->frames_max = p->frames_max;
    info->num_spectral = p->n_sp;
    info->num_direct = p->n_dir;
    info->seg_len = p->M;
    info->seg_frames = p->seg_frames;
    info->seg_halo = p->halo;
    info->fold_len = p->P;
    info->num_segments = p->n_seg;
    info->direct_taps = p->dir_taps;
    info->table_bytes = p->table_bytes;
    info->sample_rate = p->fs;
    return CWTH_OK;
}

cwth_status cwth_plan_scale_paths(cwth_plan_t p, int32_t* paths) {
    if (!valid_plan(p)) return CWTH_ERR_BAD_PLAN;
    if (!paths) return CWTH_ERR_INVALID_ARG;
    for (int s = 0; s < p->S; ++s) paths[s] = p->scale_path[s];
    return CWTH_OK;
}

}  // extern "C"
