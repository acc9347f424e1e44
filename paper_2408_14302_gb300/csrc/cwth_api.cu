// C ABI of libcwth.so: argument checking, planning, launches (include/cwth.h).
#include <limits.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <utility>
#include <vector>

#include "cwth_internal.h"

using cwth::SpecLaunch;
using cwth::SpecScale;

namespace {

// Wavelet tail left outside a segment: taps below this fraction of the peak
// may wrap around the segment (the segment halo covers everything above it).
constexpr double kEpsWrap = 1e-10;
// Morlet band threshold: spectrum bins where Psi(a nu) < kEpsBand are skipped.
// Each dropped bin weighs under 1e-7 of the band's peak and the dropped tail
// sums to about 0.1 x 1e-7 of a residue's weight mass; measured errors
// against the float64 oracle are unchanged from a 1e-9 threshold (6e-7 of
// max|W| at hops 64 and 256, 7.8e-7 at hop 1 where P = 8192), with 12 %
// fewer fold bins.
constexpr double kEpsBand = 1e-7;
// Dynamic shared memory a spectral CTA may use: the 227 KB opt-in limit less
// room for the kernel's static arrays.  One 1024-thread CTA fills an SM, so
// the whole budget is available.
constexpr size_t kSmemCap = 227 * 1024 - 1024;
// Dynamic shared memory per spectral CTA that still lets two CTAs share an
// SM (228 KB per SM, 1 KB reserved per CTA), less 256 bytes for the
// kernel's static shared variables.
constexpr size_t kSmemPair = 113 * 1024 - 256;
// Cost of one pass over a group of scales (fold + inverse FFT + stores, each
// ending at a CTA barrier) in the model's lane-operation units (~3k cycles
// measured on GB300).
constexpr double kPassCost = 64000.0;

// Scales one CTA folds and inverts together within `cap` bytes of shared
// memory (at most `limit`); fd_bytes is the fused time-domain phase's share
// of the same buffer.
int nconc_within(int M, int P, int limit, size_t cap, size_t fd_bytes) {
    int nconc = std::max(1, limit);
    while (nconc > 1 && cwth::spectral_smem_bytes(M, P, nconc, fd_bytes) > cap) --nconc;
    while (nconc > 1 && (int64_t)nconc * P > cwth::kMaxFftPoints) --nconc;
    return nconc;
}

// CTA shape of the spectral kernel for a segment length (see
// cwth_internal.h): two 512-thread CTAs per SM (radix-16 FFT passes)
// whenever one scale per pass fits their shared memory, else one 1024-thread
// CTA.  Measured on GB300, 64 x 10 s clips, 64 scales: the pair is faster
// at hops 1, 4, 8, 16 and 64 (hop 4: 2.42 vs 2.68 ms, 1 vs 2 scales per
// pass), slower only at hop 32 (0.480 vs 0.453 ms).
int spectral_threads(int M, int P, size_t fd_bytes) {
    return cwth::spectral_smem_bytes(M, P, 1, fd_bytes) > kSmemPair ? cwth::kSpecThreadsSolo
                                                                    : cwth::kSpecThreadsPair;
}

// Scales one spectral CTA folds and inverts together for a segment length
// and CTA shape.
int spectral_nconc(int M, int P, int limit, int threads, size_t fd_bytes) {
    return nconc_within(M, P, limit, threads == cwth::kSpecThreadsSolo ? kSmemCap : kSmemPair,
                        fd_bytes);
}

// Internal path marker: a short-support scale summed in the time domain
// inside the spectral kernel (reported as CWTH_PATH_DIRECT).
constexpr int32_t kPathFused = 3;
// Internal path marker: a spectral scale of the plan's second part (its
// child plan with a shorter-halo segmentation; reported as
// CWTH_PATH_SPECTRAL).
constexpr int32_t kPathSpectralChild = 4;
// Largest half support a fused scale may have (window rows 2h + 1).
constexpr int kFdMaxHalf = 256;
// Cost model, in the segment model's lane-operation units (a fold bin is
// 12): one tap row of one table column for one frame lane of the fused
// phase.  Measured on GB300: a fold bin issues about 5 instructions per
// lane, a fused row of a two-column group about 6.75 (window load, tap
// load, four FMAs, loop share), i.e. 3.4 per column.
constexpr double kFdCost = 9.0;
// Direct path: taps below this fraction of the wavelet peak are dropped.
constexpr double kEpsDirect = 1e-9;

// Streaming multiprocessors of a device (queried once per device).
int num_sms(int dev) {
    static int cache[64] = {0};
    if (dev < 0 || dev >= 64) return 1;
    if (cache[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
        cache[dev] = n;
    }
    return cache[dev];
}
// Largest padded tap count the direct path accepts.
constexpr int kMaxDirectTaps = 4096;
// Largest padded tap count an automatic CWTH_PREC_BF16X3 plan sends to the
// tensor cores (see direct_eligible).
constexpr int kSplitAutoTaps = 1024;
// Longest wait cwth_selftest_wait_timeout accepts: the kernels' own budget
// (about 2 s of SM clock).
constexpr int64_t kMaxSelftestBudget = 4000000000LL;

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// Odd factors the spectral kernel's forward FFT takes beside a power of
// two: products of 3, 5 and 7 up to 27 (the odd-radix passes run over d
// columns of at least 256 points within 8192).
bool spectral_odd_ok(int64_t d) {
    if (d < 1 || d > 27) return false;
    for (int r : {3, 5, 7})
        while (d % r == 0) d /= r;
    return d == 1;
}

// Odd part of v > 0.
int64_t odd_part(int64_t v) {
    while (v > 0 && (v & 1) == 0) v >>= 1;
    return v;
}

// Hops the spectral path serves: 2^e d with d as above.  Segments are
// M = 2 d N2 samples (N2 a power of two), so P = M / H is a power of two.
bool spectral_hop_ok(int64_t hop) { return hop > 0 && spectral_odd_ok(odd_part(hop)); }
int ilog2(int64_t v) {
    int e = 0;
    while ((int64_t(1) << e) < v) ++e;
    return e;
}

bool valid_plan(const cwth_plan_s* p) { return p && p->magic == cwth::kPlanMagic; }

thread_local char g_last_error[256] = "";

void note_error(const char* what) {
    snprintf(g_last_error, sizeof(g_last_error), "%s", what);
}

cwth_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return CWTH_OK;
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", cudaGetErrorName(e),
             cudaGetErrorString(e));
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

// Pass plan of the spectral kernel's FFTs (the device's ct_radix): with
// 16 points per thread (512-thread CTAs) radix 16 and a leading 8, 4 or
// 8,4; with 8, radix 8 and a leading 4 or 4,4.
std::vector<int> spectral_fft_radices(int L, int threads) {
    const int e = ilog2(L);
    std::vector<int> r;
    if (threads == cwth::kSpecThreadsPair) {
        const int m = e & 3;
        if (m == 3 || m == 1) r.push_back(8);
        if (m == 2 || m == 1) r.push_back(4);
        for (int b = e - (m == 3 ? 3 : m == 2 ? 2 : m == 1 ? 5 : 0); b > 0; b -= 4) r.push_back(16);
    } else {
        const int n4 = (e % 3 == 1) ? 2 : (e % 3 == 2) ? 1 : 0;
        for (int i = 0; i < n4; ++i) r.push_back(4);
        for (int b = e - 2 * n4; b > 0; b -= 3) r.push_back(8);
    }
    return r;
}

// Whether the pruned kernel (inverse FFTs skip the leading passes a narrow
// band leaves trivial, and the fold fills only the residues those FFTs
// read) is used: whenever some pass can be skipped.  Measured on GB300,
// 64 x 10 s clips, 64 scales: hop 4 2.86 -> 1.92 ms, hop 8 1.41 -> 1.19 ms,
// hop 16 0.79 -> 0.71 ms against the plain kernel.
bool spectral_prune_pays(const std::vector<SpecScale>& sc, int P, int threads) {
    const std::vector<int> rad = spectral_fft_radices(P, threads);
    int64_t skipped = 0;
    for (const SpecScale& s : sc) {
        const int64_t w = std::min<int64_t>(P, s.q_hi - s.q_lo + 1);
        int64_t ns = 1;
        for (size_t i = 0; i + 1 < rad.size() && w * ns * rad[i] <= P; ++i, ++skipped) ns *= rad[i];
    }
    return skipped > 0;
}

// Whether the paired kernel's inverse FFTs take the radix-8 plan instead
// of radix 16: a lane-operation model of mean thread work plus the busiest
// thread's critical path (butterflies per thread rounded up), for one pass
// over nc scales of period P.  With few points per thread, radix-16
// butterflies leave most warps idle.  The radix-8 plan holds one radix-8
// butterfly per thread (nc * P <= 8 * threads); pruned plans keep the
// default (their skipped passes follow it); the switch needs a 10 % gain
// in the model.
bool inverse_fft_radix8(int P, int nc, int threads, bool prune) {
    if (prune || threads != cwth::kSpecThreadsPair || (int64_t)nc * P > 8 * threads) return false;
    auto cost = [](int R, bool tw) {
        return R == 4 ? (tw ? 58.0 : 34.0) : R == 8 ? (tw ? 126.0 : 78.0) : (tw ? 340.0 : 212.0);
    };
    auto score = [&](const std::vector<int>& rad) {
        double total = 0, crit = 0;
        for (size_t i = 0; i < rad.size(); ++i) {
            const double nb = (double)nc * P / rad[i];
            const double c = cost(rad[i], i > 0);
            total += nb * c;
            crit += ceil(nb / threads) * c;
        }
        return total / threads + crit;
    };
    const double r16 = score(spectral_fft_radices(P, cwth::kSpecThreadsPair));
    const double r8 = score(spectral_fft_radices(P, cwth::kSpecThreadsSolo));
    return r16 > 1.1 * r8;
}

struct SegChoice {
    int M = 0, P = 0, halo = 0, kp0 = 0, seg_frames = 0, n_seg = 0, threads = 0;
    double cost = 0;
};

// Half support of a fused time-domain scale (taps below kEpsDirect of the
// peak dropped, as on the direct path).
int32_t fd_half_support(double a, double B) {
    return (int32_t)ceil(a * sqrt(B * log(1.0 / kEpsDirect)));
}

// Tap groups of the fused scales, given their half supports in descending
// order: consecutive runs of up to kFdMaxG scales sharing the first one's
// tap range.  Fills off / hg / n / gp; rows are the indices into h_desc.
std::vector<cwth::FdGroup> fd_make_groups(const std::vector<int32_t>& h_desc, int* taps_n,
                                          int* hw, double* cost_rows) {
    std::vector<cwth::FdGroup> g;
    int off = 0;
    *hw = 0;
    *cost_rows = 0;
    for (size_t i = 0; i < h_desc.size(); i += cwth::kFdMaxG) {
        cwth::FdGroup q;
        memset(&q, 0, sizeof(q));
        q.n = (int32_t)std::min<size_t>(cwth::kFdMaxG, h_desc.size() - i);
        q.gp = (q.n + 1) & ~1;
        q.hg = h_desc[i];
        q.off = off;
        for (int j = 0; j < q.n; ++j) q.row[j] = (int32_t)(i + j);
        off += (2 * q.hg + 1) * q.gp;
        *hw = std::max(*hw, (int)q.hg);
        *cost_rows += (double)(2 * q.hg + 1) * q.gp;
        g.push_back(q);
    }
    *taps_n = off;
    return g;
}

// Segment length for the spectral kernel: M = 2 d N2, d the odd part of
// the hop and N2 a power of two (so M is a power of two for power-of-two
// hops; P = M/H >= 8, shared memory within bounds), minimising a
// lane-operation cost model of staging + FFT + fold + inverse FFTs + stores
// + the fused time-domain phase per clip.  fd_h: half supports of the fused
// scales, descending.
bool choose_segment(const cwth_plan_s& p, const std::vector<double>& sp_scales,
                    const std::vector<int32_t>& fd_h, SegChoice* out) {
    double a_max = 0;
    for (double a : sp_scales) a_max = std::max(a_max, a);
    const int hop = p.hop;
    int fd_taps = 0, fd_hw = 0;
    double fd_rows = 0;
    int fd_ngroups = 0;
    if (!fd_h.empty()) fd_ngroups = (int)fd_make_groups(fd_h, &fd_taps, &fd_hw, &fd_rows).size();
    const int64_t h = std::max<int64_t>(
        sp_scales.empty() ? 0 : (int64_t)ceil(a_max * sqrt(p.B * log(1.0 / kEpsWrap))), fd_hw);
    const int64_t halo = ((h + hop - 1) / hop) * hop;
    const int64_t kp0 = halo / hop;
    const bool sp = !sp_scales.empty();
    bool found = false;
    const int64_t d = odd_part(hop);
    for (int lg = 8; lg <= 13; ++lg) {
        const int64_t n2 = int64_t(1) << lg;
        if (d * n2 > cwth::kMaxFftPoints) continue;
        const int64_t M = 2 * d * n2;
        if (p.seg_force > 0 && M != p.seg_force) continue;
        if (M < 8 * (int64_t)hop) continue;
        const int64_t P = M / hop;
        if (M - 1 - h < 0) continue;
        const int64_t last = (M - 1 - h) / hop;
        const int64_t Fseg = last - kp0 + 1;
        if (Fseg < 1) continue;
        const int fst = (int)(Fseg | 1);
        const size_t fdb = cwth::spectral_fd_bytes(fd_taps, fd_hw, fst, fd_ngroups);
        if (cwth::spectral_smem_bytes((int)M, (int)P, 1, fdb) > kSmemCap) continue;
        const int threads = spectral_threads((int)M, (int)P, fdb);
        if (M / 2 > cwth::kMaxFftPoints || P > cwth::kMaxFftPoints) continue;
        const int64_t n_seg = (p.frames_max + Fseg - 1) / Fseg;
        double fold = 0;
        for (double a : sp_scales) {
            int64_t lo, hi;
            band_limits(a, p.B, p.C, (int)M, &lo, &hi);
            fold += 12.0 * (double)(hi - lo + 1) + 4.0 * (double)P;
        }
        // Odd-radix passes: a direct length-R DFT per butterfly, about R + 3
        // lane operations per point and pass.
        double odd = 0;
        for (int64_t r = d; r > 1;) {
            const int R = r % 7 == 0 ? 7 : (r % 5 == 0 ? 5 : 3);
            odd += (R + 3.0) * (double)(M / 2);
            r /= R;
        }
        const double fft =
            sp ? 2.5 * (double)(M / 2) * lg + odd + 8.0 * (double)M : 2.0 * (double)M;
        const double ifft = 2.5 * (double)P * ilog2(P) * (double)sp_scales.size();
        const double store = 2.0 * (double)Fseg * (double)sp_scales.size();
        const int nconc = spectral_nconc((int)M, (int)P, std::max<int>(1, (int)sp_scales.size()),
                                         threads, fdb);
        const double passes = (double)((sp_scales.size() + nconc - 1) / nconc);
        const double fd = fd_h.empty() ? 0.0
                                       : kFdCost * fd_rows * (double)((Fseg + 31) / 32 * 32) +
                                             2.0 * (2.0 * fd_hw + 1) * (double)Fseg + kPassCost;
        const double cost = (double)n_seg * (fft + fold + ifft + store + kPassCost * passes + fd);
        if (!found || cost < out->cost) {
            found = true;
            out->M = (int)M;
            out->P = (int)P;
            out->halo = (int)halo;
            out->kp0 = (int)kp0;
            out->seg_frames = (int)Fseg;
            out->n_seg = (int)n_seg;
            out->threads = threads;
            out->cost = cost;
        }
    }
    return found;
}

// CWTH_PATH_AUTO at float32 with a power-of-two hop: how many of the
// smallest scales the spectral kernel sums in the time domain.  Every
// prefix of the scales in ascending order whose supports stay within
// kFdMaxHalf is costed with its best segment length; the cheapest wins.
// A prefix whose window buffer would push the kernel from two CTAs per SM
// to one is not taken (the model does not price the lost overlap).
int choose_fused_count(const cwth_plan_s& p, const std::vector<int32_t>& asc) {
    int best_n = 0, base_threads = 0;
    double best = -1;
    std::vector<double> sp;
    std::vector<int32_t> fd;
    for (size_t n = 0; n <= asc.size(); ++n) {
        if (n > 0 && fd_half_support(p.scales[asc[n - 1]], p.B) > kFdMaxHalf) break;
        sp.clear();
        fd.clear();
        for (size_t i = n; i < asc.size(); ++i) sp.push_back(p.scales[asc[i]]);
        for (size_t i = n; i-- > 0;) fd.push_back(fd_half_support(p.scales[asc[i]], p.B));
        SegChoice ch;
        if (!choose_segment(p, sp, fd, &ch)) continue;
        if (n == 0) base_threads = ch.threads;
        if (base_threads > 0 && ch.threads > base_threads) continue;
        if (best < 0 || ch.cost < best) {
            best = ch.cost;
            best_n = (int)n;
        }
    }
    return best_n;
}

void free_plan_memory(cwth_plan_s* p) {
    if (p->child) {
        free_plan_memory(p->child);
        delete p->child;
        p->child = nullptr;
    }
    cudaFree(p->d_tw);
    cudaFree(p->d_sp);
    cudaFree(p->d_fd_taps);
    cudaFree(p->d_fd_grp);
    p->d_fd_taps = nullptr;
    p->d_fd_grp = nullptr;
    cudaFree(p->d_stage_x);
    cudaFree(p->d_stage_out);
    cudaFree(p->d_stage_len);
    for (auto& g : p->groups) {
        cudaFree(g.d_rows);
        cudaFree(g.d_h);
        cudaFree(g.d_scales);
        cudaFree(g.d_sched);
        g.d_sched = nullptr;
        g.d_rows = nullptr;
        g.d_h = nullptr;
        g.d_scales = nullptr;
    }
    cudaFree(p->d_bank_hi);
    cudaFree(p->d_bank_lo);
    cudaFree(p->d_bank_lo2);
    p->d_bank_lo2 = nullptr;
    cudaFree(p->d_bank_f32);
    cudaFree(p->d_status);
    cudaFree(p->d_xhi);
    cudaFree(p->d_xlo);
    cudaFree(p->d_xlo2);
    p->d_xlo2 = nullptr;
    p->d_bank_hi = nullptr;
    p->d_bank_lo = nullptr;
    p->d_bank_f32 = nullptr;
    p->d_status = nullptr;
    p->d_xhi = nullptr;
    p->d_xlo = nullptr;
    p->d_tw = nullptr;
    p->d_sp = nullptr;
    p->d_stage_x = nullptr;
    p->d_stage_out = nullptr;
    p->d_stage_len = nullptr;
    cudaFree(p->d_res);
    cudaFree(p->d_res_len);
    p->d_res = nullptr;
    p->d_res_len = nullptr;
    for (cudaEvent_t* ev : {&p->ev_start, &p->ev_in, &p->ev_comp, &p->ev_out}) {
        if (*ev) cudaEventDestroy(*ev);
        *ev = nullptr;
    }
    for (cudaStream_t* st : {&p->h2d, &p->d2h, &p->cs2}) {
        if (*st) cudaStreamDestroy(*st);
        *st = nullptr;
    }
}

// Clip chunks of one cwth_execute_host call, never more than clips.  Spectral
// chunks run on two alternating streams and stay efficient down to about
// 5 MiB of input (the nearest count of 5 MiB chunks, at most 8; measured on
// GB300 with 64 x 10 s clips, 41 MB, medians of four: 3 / 4 / 5 / 6 / 8 /
// 10 / 12 chunks 0.282 / 0.292 / 0.288 / 0.279 / 0.274 / 0.282 / 0.285 ms;
// a smaller last chunk, or one split into scale groups, did not help).  Direct-path launches share one workspace and one stream,
// and a small launch is bound by the latency of its few tiles, so plans with
// direct-path scales use two chunks once the input reaches 16 MiB.
int32_t host_chunk_count(const cwth_plan_s* p, int32_t batch, int64_t ld_x) {
    const int64_t bytes = (int64_t)batch * ld_x * (int64_t)sizeof(float);
    int64_t n = p->host_chunks;
    if (n <= 0) {
        if (p->n_dir > 0)
            n = bytes >= (16ll << 20) ? 2 : 1;
        else
            n = std::min<int64_t>(8, (bytes + (5ll << 19)) / (5ll << 20));
    }
    n = std::max<int64_t>(1, n);
    return (int32_t)std::min<int64_t>(n, batch);
}

cudaError_t host_pipeline_init(cwth_plan_s* p) {
    if (p->h2d) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cs2, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&p->ev_start, &p->ev_in, &p->ev_comp, &p->ev_out})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    return e;
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// bf16 parts per operand of the tensor-core direct path for a precision.
int direct_parts(int32_t precision) {
    return precision == CWTH_PREC_BF16X3 ? 3 : (precision == CWTH_PREC_BF16X2 ? 2 : 1);
}

// Half support of the direct path's truncated taps, a multiple of 8 so that
// every group's view of the staged signal starts 16-byte aligned.
int32_t direct_half_support(double a, double B) {
    return (int32_t)round_up((int64_t)ceil(a * sqrt(B * log(1.0 / kEpsDirect))), 8);
}

bool direct_eligible(const cwth_plan_s& p, double a) {
    const int64_t k = round_up(2 * (int64_t)direct_half_support(a, p.B) + 1, 64);
    if (k > kMaxDirectTaps) return false;
    // Automatic three-part split plans keep the float32 accuracy class on
    // every input: the tensor cores' float32 accumulation loses low-order
    // bits along an MMA chain (measured on GB300: a mean relative bias of
    // -3.5e-6 at 613 taps, -6.5e-6 at 1185, -1.2e-5 at 2297 on white
    // noise), so scales beyond kSplitAutoTaps padded taps take the float32
    // spectral path instead.
    if (p.path == CWTH_PATH_AUTO && p.precision == CWTH_PREC_BF16X3 && k > kSplitAutoTaps)
        return false;
    if (p.precision != CWTH_PREC_FP32 && p.hop % 8 != 0) return false;
    // The tensor-core epilogue addresses a clip's output with 32-bit offsets.
    if (p.precision != CWTH_PREC_FP32 && (int64_t)p.S * p.frames_max > INT32_MAX) return false;
    return true;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)ptr;
    }
    return fn;
}

// 2-D bf16 tensor map: dims {inner, outer}, row stride in bytes, box {64, box_outer},
// 128-byte swizzle, zero fill out of bounds.
bool encode_bf16_2d(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer,
                    uint64_t row_stride_bytes, uint32_t box_outer) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {row_stride_bytes};
    const cuuint32_t box[2] = {64, box_outer};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
              box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// Shared-memory bytes of a plan's fused time-domain phase (0 without one).
size_t fd_bytes(const cwth_plan_s* p) {
    return p->n_fd > 0 ? cwth::spectral_fd_bytes(p->fd_taps_n, p->fd_hw, p->fd_fst,
                                                  (int)p->fd_groups.size())
                       : 0;
}

cwth_status build_direct(cwth_plan_s* p) {
    std::vector<int> idx;
    for (int s = 0; s < p->S; ++s)
        if (p->scale_path[s] == CWTH_PATH_DIRECT) idx.push_back(s);
    p->n_dir = (int32_t)idx.size();
    if (p->n_dir == 0) return CWTH_OK;
    // Descending support; groups of at most 128 scales (256 columns), each a
    // pyramid-scheduled GEMM (see direct.cu).
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int a, int b) { return p->scales[a] > p->scales[b]; });
    std::vector<int32_t> hs(idx.size());
    for (size_t i = 0; i < idx.size(); ++i) hs[i] = direct_half_support(p->scales[idx[i]], p->B);
    std::vector<std::pair<int, int>> ranges;
    for (int i = 0; i < (int)idx.size(); i += 128)
        ranges.push_back({i, std::min<int>((int)idx.size(), i + 128)});
    const int nparts = direct_parts(p->precision);
    const bool split = nparts > 1;
    int64_t bank_elems = 0, f32_elems = 0;
    for (auto& r : ranges) {
        cwth::DirGroup g;
        g.n_scales = r.second - r.first;
        g.ncols = (int32_t)round_up(2 * g.n_scales, 16);
        g.h = hs[r.first];
        g.k_pad = (int32_t)round_up(2 * (int64_t)g.h + 1, 64);
        g.bank_off = bank_elems;
        g.f32_off = f32_elems;
        g.shape = cwth::direct_shape(g.ncols, nparts, p->hop, g.k_pad);
        if (g.shape.stages == 0) return CWTH_ERR_UNSUPPORTED;
        bank_elems += (int64_t)g.ncols * g.k_pad;
        f32_elems += (int64_t)g.n_scales * g.k_pad;
        p->groups.push_back(g);
        p->dir_taps = std::max(p->dir_taps, g.k_pad);
        p->dir_front = std::max(p->dir_front, g.h);
    }
    cudaError_t e = cudaMalloc(&p->d_bank_hi, sizeof(__nv_bfloat16) * bank_elems);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_bank_lo, sizeof(__nv_bfloat16) * bank_elems);
    if (e == cudaSuccess && nparts > 2)
        e = cudaMalloc(&p->d_bank_lo2, sizeof(__nv_bfloat16) * bank_elems);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_bank_f32, sizeof(float2) * f32_elems);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_status, 0, sizeof(int), p->setup);
    if (e != cudaSuccess) return cuda_status(e);
    p->table_bytes += (int64_t)(bank_elems * 2 * (nparts > 2 ? 3 : 2) + f32_elems * 8);
    for (size_t gi = 0; gi < ranges.size(); ++gi) {
        cwth::DirGroup& g = p->groups[gi];
        std::vector<int32_t> rows, hh;
        std::vector<double> sc;
        for (int i = ranges[gi].first; i < ranges[gi].second; ++i) {
            rows.push_back(idx[i]);
            hh.push_back(hs[i]);
            sc.push_back(p->scales[idx[i]]);
        }
        e = cudaMalloc(&g.d_rows, sizeof(int32_t) * rows.size());
        if (e == cudaSuccess) e = cudaMalloc(&g.d_h, sizeof(int32_t) * hh.size());
        if (e == cudaSuccess) e = cudaMalloc(&g.d_scales, sizeof(double) * sc.size());
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g.d_rows, rows.data(), sizeof(int32_t) * rows.size(), cudaMemcpyHostToDevice, p->setup);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g.d_h, hh.data(), sizeof(int32_t) * hh.size(), cudaMemcpyHostToDevice, p->setup);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g.d_scales, sc.data(), sizeof(double) * sc.size(), cudaMemcpyHostToDevice, p->setup);
        std::vector<int2> sched(g.k_pad / 64), sched2(3 * (g.k_pad / 64));
        g.nsteps = cwth::direct_schedule(
            hh.data(), g.n_scales, g.h, g.k_pad, (g.ncols + 63) / 64,
            cwth::direct_a_pieces(nparts, g.shape.unit, g.shape.win_rows > 0), sched.data());
        if (split) {
            g.nsteps = cwth::direct_split_schedule(sched.data(), g.nsteps, nparts, sched2.data());
            sched.swap(sched2);
        }
        if (e == cudaSuccess) e = cudaMalloc(&g.d_sched, sizeof(int2) * sched.size());
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g.d_sched, sched.data(), sizeof(int2) * g.nsteps, cudaMemcpyHostToDevice, p->setup);
        if (e == cudaSuccess)
            e = cwth::direct_make_bank(g.d_scales, g.d_h, g.n_scales, g.ncols, g.k_pad, g.h, p->B,
                                       p->C, p->d_bank_hi + g.bank_off, p->d_bank_lo + g.bank_off,
                                       p->d_bank_lo2 ? p->d_bank_lo2 + g.bank_off : nullptr,
                                       p->d_bank_f32 + g.f32_off, p->setup);
        if (e != cudaSuccess) return cuda_status(e);
        if (p->precision != CWTH_PREC_FP32) {
            if (!encode_bf16_2d(&g.map_b_hi, p->d_bank_hi + g.bank_off, g.k_pad, g.ncols,
                                (uint64_t)g.k_pad * 2, 64) ||
                !encode_bf16_2d(&g.map_b_lo, p->d_bank_lo + g.bank_off, g.k_pad, g.ncols,
                                (uint64_t)g.k_pad * 2, 64) ||
                (nparts > 2 && !encode_bf16_2d(&g.map_b_lo2, p->d_bank_lo2 + g.bank_off, g.k_pad,
                                               g.ncols, (uint64_t)g.k_pad * 2, 64))) {
                note_error("cuTensorMapEncodeTiled rejected the tap-bank tensor map");
                return CWTH_ERR_UNSUPPORTED;
            }
        }
    }
    if (p->precision != CWTH_PREC_FP32) {
        // The frame matrix is a view with overlapping rows (row stride = hop):
        // check once that the driver accepts it.
        CUtensorMap probe;
        const int64_t rows = 1024;
        if (!encode_bf16_2d(&probe, p->d_bank_hi, p->dir_taps, rows, (uint64_t)p->hop * 2, 128)) {
            note_error("cuTensorMapEncodeTiled rejected the overlapping frame view");
            return CWTH_ERR_UNSUPPORTED;
        }
        e = cwth::direct_prepare_device();
    } else {
        e = cwth::direct_prepare_f32((size_t)(2 * p->dir_front + 1) * sizeof(float2));
    }
    if (e != cudaSuccess) return cuda_status(e);
    return cuda_status(cudaStreamSynchronize(p->setup));
}

cwth_status build_spectral(cwth_plan_s* p) {
    std::vector<double> sp;
    std::vector<int32_t> rows;
    // Spectral scales in ascending scale order (descending band width; each
    // keeps its output row), so that a chunk's first scale has its widest
    // band and the fold deals its widest items first.
    std::vector<int32_t> order;
    for (int s = 0; s < p->S; ++s)
        if (p->scale_path[s] == CWTH_PATH_SPECTRAL) order.push_back(s);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t i, int32_t j) { return p->scales[i] < p->scales[j]; });
    for (int32_t s : order) {
        sp.push_back(p->scales[s]);
        rows.push_back(s);
    }
    p->n_sp = (int32_t)sp.size();
    // Fused time-domain scales, descending support (descending scale).
    std::vector<int32_t> fd_idx;
    for (int s = 0; s < p->S; ++s)
        if (p->scale_path[s] == kPathFused) fd_idx.push_back(s);
    std::stable_sort(fd_idx.begin(), fd_idx.end(),
                     [&](int32_t i, int32_t j) { return p->scales[i] > p->scales[j]; });
    std::vector<int32_t> fd_h;
    for (int32_t s : fd_idx) fd_h.push_back(fd_half_support(p->scales[s], p->B));
    p->n_fd = (int32_t)fd_idx.size();
    if (p->n_sp == 0 && p->n_fd == 0) return CWTH_OK;
    if (!spectral_hop_ok(p->hop)) return CWTH_ERR_UNSUPPORTED;
    SegChoice ch;
    if (!choose_segment(*p, sp, fd_h, &ch)) return CWTH_ERR_UNSUPPORTED;
    p->M = ch.M;
    p->P = ch.P;
    p->halo = ch.halo;
    p->kp0 = ch.kp0;
    p->seg_frames = ch.seg_frames;
    p->n_seg = ch.n_seg;
    p->seg_cost = ch.n_seg > 0 ? ch.cost / ch.n_seg : 0.0;
    p->fft_d = (int32_t)odd_part(p->M);
    p->fft_n2 = p->M / 2 / p->fft_d;

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
        const double kexp = -M_PI * M_PI * p->B / M_LN2;
        const double dlt = sp[i] * (double)p->P / (double)p->M;
        s.dlt = (float)dlt;
        s.q2 = (float)exp2(2.0 * kexp * (double)s.dlt * (double)s.dlt);
        s.wsuf = (int32_t)std::min<int64_t>(p->P, hi - lo + 1);
    }
    for (size_t i = host.size(); i-- > 1;)
        host[i - 1].wsuf = std::max(host[i - 1].wsuf, host[i].wsuf);
    // Fold pairs: scales 2j and 2j + 1 of the table (whose bands nest when
    // their ratio is near 1) share a walk over the union of their bands when
    // both weights stay >= 1e-20 on it (the Gaussian's minimum over the
    // union is at one of its ends).
    for (size_t i = 0; i + 1 < host.size(); i += 2) {
        const int64_t lo = std::min(host[i].q_lo, host[i + 1].q_lo);
        const int64_t hi = std::max(host[i].q_hi, host[i + 1].q_hi);
        bool ok = true;
        for (size_t k = i; k <= i + 1; ++k)
            for (int64_t q : {lo, hi}) {
                const double u = (double)q * sp[k] / (double)p->M - p->C;
                if (-M_PI * M_PI * p->B * u * u < log(1e-20)) ok = false;
            }
        host[i].pair = ok ? 1 : 0;
    }
    cudaError_t e = cudaSuccess;
    if (p->n_fd > 0) {
        double rows = 0;
        p->fd_groups = fd_make_groups(fd_h, &p->fd_taps_n, &p->fd_hw, &rows);
        p->fd_fst = p->seg_frames | 1;
        // Columns of group g are fused scales fd_idx[row[j]]: the generator
        // reads their scale and support through gidx, the kernel writes
        // output row fd_idx[...].
        const int ng = (int)p->fd_groups.size();
        std::vector<int32_t> gidx((size_t)ng * cwth::kFdMaxG, 0);
        std::vector<double> fsc(fd_idx.size());
        for (size_t i = 0; i < fd_idx.size(); ++i) fsc[i] = p->scales[fd_idx[i]];
        for (int g = 0; g < ng; ++g)
            for (int j = 0; j < p->fd_groups[g].n; ++j) {
                const int i = p->fd_groups[g].row[j];
                gidx[(size_t)g * cwth::kFdMaxG + j] = i;
                p->fd_groups[g].row[j] = fd_idx[i];
            }
        double* d_sc = nullptr;
        int32_t *d_h = nullptr, *d_gi = nullptr;
        e = cudaMalloc(&p->d_fd_taps, sizeof(float2) * (size_t)p->fd_taps_n);
        if (e == cudaSuccess) e = cudaMalloc(&p->d_fd_grp, sizeof(cwth::FdGroup) * (size_t)ng);
        if (e == cudaSuccess) e = cudaMalloc(&d_sc, sizeof(double) * fsc.size());
        if (e == cudaSuccess) e = cudaMalloc(&d_h, sizeof(int32_t) * fd_h.size());
        if (e == cudaSuccess) e = cudaMalloc(&d_gi, sizeof(int32_t) * gidx.size());
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->d_fd_grp, p->fd_groups.data(), sizeof(cwth::FdGroup) * (size_t)ng,
                                cudaMemcpyHostToDevice, p->setup);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_sc, fsc.data(), sizeof(double) * fsc.size(),
                                cudaMemcpyHostToDevice, p->setup);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_h, fd_h.data(), sizeof(int32_t) * fd_h.size(),
                                cudaMemcpyHostToDevice, p->setup);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_gi, gidx.data(), sizeof(int32_t) * gidx.size(),
                                cudaMemcpyHostToDevice, p->setup);
        if (e == cudaSuccess)
            e = cwth::spectral_make_fd_taps(d_sc, d_h, d_gi, p->d_fd_grp, ng, p->fd_taps_n, p->B,
                                            p->C, p->d_fd_taps, p->setup);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->setup);
        cudaFree(d_sc);
        cudaFree(d_h);
        cudaFree(d_gi);
        if (e != cudaSuccess) return cuda_status(e);
        p->table_bytes += (int64_t)(sizeof(float2) * (size_t)p->fd_taps_n +
                                    sizeof(cwth::FdGroup) * (size_t)ng);
    }
    if (p->n_sp == 0) {
        e = cwth::spectral_prepare_device();
        if (e != cudaSuccess) return cuda_status(e);
        return cuda_status(cudaStreamSynchronize(p->setup));
    }
    const int threads = spectral_threads(p->M, p->P, fd_bytes(p));
    p->spec_prune = spectral_prune_pays(host, p->P, threads);
    // Decided once per plan, for its largest pass, so that every launch (any
    // scale grouping, any host chunk) runs the same inverse FFTs and gives
    // the same bytes.
    {
        const int nc = spectral_nconc(p->M, p->P, p->n_sp, threads, fd_bytes(p));
        p->inv_r8 = inverse_fft_radix8(p->P, nc, threads, p->spec_prune);
        p->inv_r8_model = p->inv_r8;
        p->inv_r8_ok = !p->spec_prune && threads == cwth::kSpecThreadsPair &&
                       (int64_t)nc * p->P <= 8 * (int64_t)threads;
    }
    const size_t ntw = (size_t)cwth::spectral_twiddle_entries(p->M);
    e = cudaMalloc(&p->d_tw, sizeof(float2) * ntw);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaMalloc(&p->d_sp, sizeof(SpecScale) * host.size());
    if (e != cudaSuccess) return cuda_status(e);
    p->table_bytes += (int64_t)(sizeof(float2) * ntw + sizeof(SpecScale) * host.size());
    e = cudaMemcpyAsync(p->d_sp, host.data(), sizeof(SpecScale) * host.size(), cudaMemcpyHostToDevice,
                        p->setup);
    if (e != cudaSuccess) return cuda_status(e);
    e = cwth::spectral_make_twiddles(p->d_tw, p->M, p->setup);
    if (e != cudaSuccess) return cuda_status(e);
    e = cwth::spectral_prepare_device();
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaStreamSynchronize(p->setup);
    return cuda_status(e);
}

// Several spectral parts when the cost model prefers them: the smallest
// spectral scales (shortest supports) in a child plan whose segments need
// only their own, short halo, so more of each segment's frames are valid;
// the rest (and the fused scales) stay in this plan.  Every split point of
// the ascending scale list is costed with each part's best segment length;
// a split is kept only if it saves at least a tenth of the cost before it
// (each part repeats the forward FFTs).  The remaining scales are then
// offered the same split again, up to kMaxSpectralParts parts (children
// chained in split order).  Not for forced segment lengths.
constexpr double kSplitGain = 0.9;
constexpr int kMaxSpectralParts = 4;

cwth_status split_spectral(cwth_plan_s* p) {
    if (p->no_split || p->seg_force > 0 || !spectral_hop_ok(p->hop)) return CWTH_OK;
    std::vector<int32_t> fd_idx;
    for (int s = 0; s < p->S; ++s)
        if (p->scale_path[s] == kPathFused) fd_idx.push_back(s);
    std::stable_sort(fd_idx.begin(), fd_idx.end(),
                     [&](int32_t i, int32_t j) { return p->scales[i] > p->scales[j]; });
    std::vector<int32_t> fd_h;
    for (int32_t s : fd_idx) fd_h.push_back(fd_half_support(p->scales[s], p->B));
    const std::vector<int32_t> none;
    cwth_plan_s** tail = &p->child;
    for (int part = 1; part < kMaxSpectralParts; ++part) {
        std::vector<int32_t> order;
        for (int s = 0; s < p->S; ++s)
            if (p->scale_path[s] == CWTH_PATH_SPECTRAL) order.push_back(s);
        if (order.size() < 2) break;
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t i, int32_t j) { return p->scales[i] < p->scales[j]; });
        std::vector<double> sp;
        for (int32_t s : order) sp.push_back(p->scales[s]);
        SegChoice one;
        if (!choose_segment(*p, sp, fd_h, &one)) break;
        double best = one.cost;
        size_t best_j = 0;
        // At most ~128 candidate split points (plan time grows with their
        // number times the scale count).
        const size_t step = std::max<size_t>(1, sp.size() / 128);
        for (size_t j = step; j < sp.size(); j += step) {
            const std::vector<double> a(sp.begin(), sp.begin() + j), b(sp.begin() + j, sp.end());
            SegChoice ca, cb;
            if (!choose_segment(*p, a, none, &ca) || !choose_segment(*p, b, fd_h, &cb)) continue;
            if (ca.cost + cb.cost < best) {
                best = ca.cost + cb.cost;
                best_j = j;
            }
        }
        if (best_j == 0 || best > kSplitGain * one.cost) break;
        cwth_plan_s* q = new (std::nothrow) cwth_plan_s();
        if (!q) return CWTH_ERR_OOM;
        q->device = p->device;
        q->B = p->B;
        q->C = p->C;
        q->fs = p->fs;
        q->S = p->S;
        q->hop = p->hop;
        q->precision = p->precision;
        q->path = p->path;
        q->max_len = p->max_len;
        q->frames_max = p->frames_max;
        q->scales = p->scales;
        q->scale_path.assign(p->S, CWTH_PATH_DIRECT);
        for (size_t j = 0; j < best_j; ++j) q->scale_path[order[j]] = CWTH_PATH_SPECTRAL;
        q->no_split = true;
        q->setup = p->setup;
        cwth_status st = build_spectral(q);
        q->setup = nullptr;
        if (st != CWTH_OK) {
            free_plan_memory(q);
            delete q;
            return st;
        }
        *tail = q;
        tail = &q->child;
        for (size_t j = 0; j < best_j; ++j) p->scale_path[order[j]] = kPathSpectralChild;
        p->table_bytes += q->table_bytes;
    }
    return CWTH_OK;
}

// The spectral kernel's launch record of a plan for one batch: scale
// groups (enough CTAs for two waves, each group at least 8 scales, since
// every group repeats its segment's forward FFT; one group when fill_gpu is
// false, i.e. when the launch shares the GPU with other work of the same
// batch), the fused tap groups dealt round-robin over them, the CTA shape
// and the dynamic shared memory.
void spectral_record(const cwth_plan_s* p, const float* d_x, int64_t ld_x, const int64_t* d_len,
                     int32_t batch, float* d_out, bool fill_gpu, SpecLaunch* out, int* threads_out,
                     int* n_groups_out, size_t* smem_out) {
    const int64_t base = std::max<int64_t>(1, (int64_t)p->n_seg * batch);
    const int64_t want = (2 * (int64_t)num_sms(p->device) + base - 1) / base;
    const int fdg = (int)p->fd_groups.size();
    int n_groups = 1, gs = 0;
    if (p->n_sp > 0) {
        n_groups = !fill_gpu ? 1 : (int)std::min<int64_t>(want, std::max(1, p->n_sp / 8));
        n_groups = std::max(1, n_groups);
        gs = (p->n_sp + n_groups - 1) / n_groups;
        // Groups and passes of an even number of scales: the fold walks
        // table pairs (2j, 2j + 1), so every launch shape pairs the same
        // scales and gives the same bytes.
        gs += gs & 1;
        n_groups = (p->n_sp + gs - 1) / gs;
    } else {
        n_groups = !fill_gpu ? 1 : (int)std::max<int64_t>(1, std::min<int64_t>(want, fdg));
    }
    const size_t fdb = fd_bytes(p);
    const int threads = spectral_threads(p->M, p->P, fdb);
    int nconc = spectral_nconc(p->M, p->P, std::max(1, gs), threads, fdb);
    if (nconc > 1) nconc &= ~1;

    SpecLaunch L;
    memset(&L, 0, sizeof(L));
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
    L.vec4 = (p->fft_d == 1 && ld_x % 4 == 0 && ((uintptr_t)d_x & 15) == 0 && p->halo % 4 == 0 &&
              ((int64_t)p->seg_frames * p->hop) % 4 == 0)
                 ? 1
                 : 0;
    L.fd_groups = fdg;
    L.fd_hw = p->fd_hw;
    L.fd_fst = p->fd_fst;
    L.fd_taps_n = p->fd_taps_n;
    L.fd_taps = p->d_fd_taps;
    L.fd_grp = p->d_fd_grp;
    L.inv_r8 = p->inv_r8 ? 1 : 0;
    L.fft_d = p->fft_d;
    L.fft_n2 = p->fft_n2;
    *out = L;
    *threads_out = threads;
    *n_groups_out = n_groups;
    *smem_out = cwth::spectral_smem_bytes(p->M, p->P, nconc, fdb);
}

cwth_status launch_spectral(cwth_plan_s* p, const float* d_x, int64_t ld_x,
                            const int64_t* d_len, int32_t batch, float* d_out, cudaStream_t st,
                            bool fill_gpu, bool dependent = false) {
    if ((p->n_sp == 0 && p->n_fd == 0) || batch == 0) return CWTH_OK;
    if (batch > 65535 || p->n_seg > 0x7fffffff) return CWTH_ERR_UNSUPPORTED;
    SpecLaunch L;
    int threads = 0, n_groups = 1;
    size_t smem = 0;
    spectral_record(p, d_x, ld_x, d_len, batch, d_out, fill_gpu, &L, &threads, &n_groups, &smem);
    return cuda_status(
        cwth::spectral_launch(L, threads, p->spec_prune, p->n_seg, batch, n_groups, smem, st,
                              dependent));
}

// Rows of one clip in the direct path's staged signal (the clip with its
// zero margins, in whole hops) and the staged elements of a batch.
struct DirStageShape {
    int64_t rows_per_clip, lpad, total_rows, total;
};

DirStageShape dir_stage_shape(const cwth_plan_s* p, int32_t batch) {
    DirStageShape d;
    const int64_t hop = p->hop;
    d.rows_per_clip = (2 * (int64_t)p->dir_front + p->frames_max * hop + p->dir_taps + hop - 1) / hop;
    d.lpad = d.rows_per_clip * hop;
    d.total_rows = (int64_t)batch * d.rows_per_clip;
    d.total = (int64_t)batch * d.lpad + p->dir_front + p->dir_taps + 64;
    return d;
}

// Grows the staged bf16 signal to `total` elements per part.  Growing frees
// the old buffers first (cudaFree waits for the device to finish the work
// that may still read them).
// Elements of one staged part in a caller-bound buffer: rounded up to 128
// (256 bytes), so each part starts aligned for the tensor maps.
int64_t dir_stage_part(int64_t total) { return (total + 127) / 128 * 128; }

// Bytes a caller-bound staging buffer needs for `batch` clips (0: the plan
// stages nothing).
size_t dir_stage_bytes(const cwth_plan_s* p, int32_t batch) {
    if (p->n_dir == 0 || p->precision == CWTH_PREC_FP32 || batch <= 0) return 0;
    const DirStageShape sh = dir_stage_shape(p, batch);
    return (size_t)direct_parts(p->precision) * (size_t)dir_stage_part(sh.total) *
           sizeof(__nv_bfloat16);
}

cwth_status dir_stage_grow(cwth_plan_s* p, int64_t total) {
    const int nparts = direct_parts(p->precision);
    if ((size_t)total > p->x_elems) {
        cudaFree(p->d_xhi);
        cudaFree(p->d_xlo);
        cudaFree(p->d_xlo2);
        p->d_xhi = nullptr;
        p->d_xlo = nullptr;
        p->d_xlo2 = nullptr;
        p->x_elems = 0;
        p->x_maps_ptr = nullptr;
        cudaError_t e = cudaMalloc(&p->d_xhi, sizeof(__nv_bfloat16) * (size_t)total);
        if (e == cudaSuccess) e = cudaMalloc(&p->d_xlo, sizeof(__nv_bfloat16) * (size_t)total);
        if (e == cudaSuccess && nparts > 2)
            e = cudaMalloc(&p->d_xlo2, sizeof(__nv_bfloat16) * (size_t)total);
        if (e != cudaSuccess) return cuda_status(e);
        p->x_elems = (size_t)total;
    }
    return CWTH_OK;
}

cwth_status launch_direct(cwth_plan_s* p, const float* d_x, int64_t ld_x, const int64_t* d_len,
                          int32_t batch, float* d_out, cudaStream_t st) {
    if (p->n_dir == 0 || batch == 0) return CWTH_OK;
    cwth::DirLaunch L;
    memset(&L, 0, sizeof(L));
    L.out = d_out;
    L.frames_max = p->frames_max;
    L.S_total = p->S;
    L.hop = p->hop;
    L.lengths = d_len;
    L.max_len = p->max_len;
    L.batch = batch;
    L.status = p->d_status;
    if (p->precision == CWTH_PREC_FP32) {
        for (auto& g : p->groups) {
            L.ncols = g.ncols;
            L.k_pad = g.k_pad;
            L.h_group = g.h;
            L.n_scales = g.n_scales;
            L.rows = g.d_rows;
            cudaError_t e = cwth::direct_launch_f32(d_x, ld_x, p->d_bank_f32 + g.f32_off, g.d_h, L, st);
            if (e != cudaSuccess) return cuda_status(e);
        }
        return CWTH_OK;
    }
    const int nparts = direct_parts(p->precision);
    const int64_t hop = p->hop;
    const DirStageShape sh = dir_stage_shape(p, batch);
    const int64_t rows_per_clip = sh.rows_per_clip;
    const int64_t lpad = sh.lpad;
    const int64_t total_rows = sh.total_rows;
    const int64_t total = sh.total;
    if (total_rows > (int64_t(1) << 31) - 256) return CWTH_ERR_UNSUPPORTED;
    {
        if (!p->ext_stage) {
            cwth_status gs = dir_stage_grow(p, total);
            if (gs != CWTH_OK) return gs;
        }
    }
    // The staged parts: the plan's own buffers, or consecutive parts of a
    // caller-bound buffer.
    __nv_bfloat16* xhi = p->d_xhi;
    __nv_bfloat16* xlo = p->d_xlo;
    __nv_bfloat16* xlo2 = p->d_xlo2;
    if (p->ext_stage) {
        if (p->ext_stage_bytes < dir_stage_bytes(p, batch)) {
            char msg[160];
            snprintf(msg, sizeof(msg), "the bound staging buffer holds %zu bytes; this batch needs %zu",
                     p->ext_stage_bytes, dir_stage_bytes(p, batch));
            note_error(msg);
            return CWTH_ERR_INVALID_ARG;
        }
        const int64_t part = dir_stage_part(total);
        xhi = static_cast<__nv_bfloat16*>(p->ext_stage);
        xlo = nparts > 1 ? xhi + part : xhi;
        xlo2 = nparts > 2 ? xhi + 2 * part : xlo;
    }
    if (p->x_maps_ptr != xhi || p->x_maps_rows != total_rows) {
        p->maps_a_hi.assign(p->groups.size(), CUtensorMap());
        p->maps_a_lo.assign(p->groups.size(), CUtensorMap());
        p->maps_a_lo2.assign(p->groups.size(), CUtensorMap());
        for (size_t gi = 0; gi < p->groups.size(); ++gi) {
            const cwth::DirGroup& g = p->groups[gi];
            const int64_t off = p->dir_front - g.h;
            if (!encode_bf16_2d(&p->maps_a_hi[gi], xhi + off, g.k_pad, total_rows, hop * 2, 32) ||
                !encode_bf16_2d(&p->maps_a_lo[gi], xlo + off, g.k_pad, total_rows, hop * 2, 32) ||
                (nparts > 2 && !encode_bf16_2d(&p->maps_a_lo2[gi], xlo2 + off, g.k_pad,
                                               total_rows, hop * 2, 32))) {
                note_error("cuTensorMapEncodeTiled rejected the frame-matrix tensor map");
                return CWTH_ERR_UNSUPPORTED;
            }
        }
        p->x_maps_ptr = xhi;
        p->x_maps_rows = total_rows;
    }
    cudaError_t e = cwth::direct_stage(d_x, ld_x, d_len, p->max_len, batch, xhi,
                                       nparts > 1 ? xlo : nullptr, nparts > 2 ? xlo2 : nullptr,
                                       lpad, p->dir_front, total, st);
    if (e != cudaSuccess) return cuda_status(e);
    L.rows_per_clip = rows_per_clip;
    L.total_rows = total_rows;
    for (size_t gi = 0; gi < p->groups.size(); ++gi) {
        const cwth::DirGroup& g = p->groups[gi];
        CUtensorMap maps[6] = {p->maps_a_hi[gi], p->maps_a_lo[gi], p->maps_a_lo2[gi],
                               g.map_b_hi,        g.map_b_lo,        g.map_b_lo2};
        L.ncols = g.ncols;
        L.k_pad = g.k_pad;
        L.h_group = g.h;
        L.n_scales = g.n_scales;
        L.rows = g.d_rows;
        L.stages = g.shape.stages;
        L.sched = g.d_sched;
        L.nsteps = g.nsteps;
        L.win_rows = g.shape.win_rows;
        L.a_shift = g.shape.win_rows ? cwth::direct_window_shift((int)hop) : 0;
        L.a_phases = g.shape.win_rows ? g.shape.phases : 1;
        L.unit = g.shape.unit;
        L.win_sets = g.shape.win_sets;
        L.acc_sets = g.shape.acc_sets;
        L.tmem_cols = g.shape.tmem_cols;
        e = cwth::direct_launch_mma(maps, L, nparts, st);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return CWTH_OK;
}

cwth_status launch_all(cwth_plan_s* p, const float* d_x, int64_t ld_x, const int64_t* d_len,
                       int32_t batch, float* d_out, cudaStream_t st, bool fill_gpu = true) {
    cwth_status s = launch_direct(p, d_x, ld_x, d_len, batch, d_out, st);
    // After the direct path's kernels (other rows, the same input), the
    // spectral part may start on the SMs they leave as they finish.
    if (s == CWTH_OK)
        s = launch_spectral(p, d_x, ld_x, d_len, batch, d_out, st, fill_gpu,
                            p->n_dir > 0 && batch > 0);
    // Later parts read the same input and write other rows: each may start
    // on the SMs the part before it leaves idle in its last wave.
    for (cwth_plan_s* q = p->child; q && s == CWTH_OK; q = q->child)
        s = launch_spectral(q, d_x, ld_x, d_len, batch, d_out, st, fill_gpu, true);
    return s;
}

// Samples each input row must hold: the longest clip, or for a
// resample-first plan the longest clip before re-sampling.
int64_t input_len(const cwth_plan_s* p) { return p->resample > 1 ? p->in_len : p->max_len; }

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

// The transform of rows [row0, row0 + batch) of a plan's workspace: a
// resample-first plan first re-samples the inputs into its own buffer (rows
// from row0 on, so concurrent chunks use disjoint rows).  `ws_rows` is the
// number of rows the workspace must hold.
cwth_status launch_transform(cwth_plan_s* p, const float* d_x, int64_t ld_x, const int64_t* d_len,
                             int32_t batch, float* d_out, cudaStream_t st, bool fill_gpu,
                             int64_t row0, int64_t ws_rows) {
    if (p->resample <= 1) return launch_all(p, d_x, ld_x, d_len, batch, d_out, st, fill_gpu);
    cwth_status s = grow(&p->d_res, &p->res_elems, (size_t)ws_rows * (size_t)p->max_len);
    if (s == CWTH_OK && d_len) s = grow(&p->d_res_len, &p->res_len_elems, (size_t)ws_rows);
    if (s != CWTH_OK) return s;
    float* y = p->d_res + (size_t)row0 * (size_t)p->max_len;
    int64_t* ly = d_len ? p->d_res_len + row0 : nullptr;
    cudaError_t e = cwth::resample_launch(d_x, ld_x, d_len, p->in_len, p->resample, y, p->max_len,
                                          ly, batch, st);
    if (e != cudaSuccess) return cuda_status(e);
    return launch_all(p, y, p->max_len, ly, batch, d_out, st, fill_gpu);
}

}  // namespace

namespace cwth {
void set_last_error(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }
}  // namespace cwth

extern "C" {

int64_t cwth_num_frames(int64_t n, int32_t hop) {
    if (n <= 0 || hop <= 0) return 0;
    return (n + hop - 1) / hop;
}

const char* cwth_last_error(void) { return g_last_error; }

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

namespace {
cwth_status plan_create(const cwth_morlet* w, const double* scales, int32_t S, int32_t hop,
                        double sample_rate, int64_t max_len, int32_t precision, int32_t path,
                        int32_t seg_len, cwth_plan_t* out);
}

cwth_status cwth_plan(const cwth_morlet* w, const double* scales, int32_t S, int32_t hop,
                      double sample_rate, int64_t max_len, int32_t precision, int32_t path,
                      cwth_plan_t* out) {
    return plan_create(w, scales, S, hop, sample_rate, max_len, precision, path, 0, out);
}

cwth_status cwth_plan_segment(const cwth_morlet* w, const double* scales, int32_t S,
                              int32_t hop, double sample_rate, int64_t max_len,
                              int32_t precision, int32_t path, int32_t seg_len,
                              cwth_plan_t* out) {
    if (out) *out = nullptr;
    if (seg_len < 0 || (seg_len > 0 && (seg_len < 512 || seg_len > 32768 ||
                                         !spectral_odd_ok(odd_part(seg_len)))))
        return CWTH_ERR_INVALID_ARG;
    return plan_create(w, scales, S, hop, sample_rate, max_len, precision, path, seg_len, out);
}

namespace {
cwth_status plan_create(const cwth_morlet* w, const double* scales, int32_t S, int32_t hop,
                        double sample_rate, int64_t max_len, int32_t precision, int32_t path,
                        int32_t seg_len, cwth_plan_t* out) {
    cwth::NvtxRange nvtx_range("cwth_plan");
    if (out) *out = nullptr;
    if (!w || !scales || !out) return CWTH_ERR_INVALID_ARG;
    if (S < 1 || hop < 1 || max_len < 1) return CWTH_ERR_INVALID_ARG;
    if (!(isfinite(w->bandwidth) && w->bandwidth > 0)) return CWTH_ERR_INVALID_ARG;
    if (!(isfinite(w->center_freq) && w->center_freq > 0)) return CWTH_ERR_INVALID_ARG;
    if (!(isfinite(sample_rate) && sample_rate > 0)) return CWTH_ERR_INVALID_ARG;
    if (precision < CWTH_PREC_FP32 || precision > CWTH_PREC_BF16X3) return CWTH_ERR_INVALID_ARG;
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
        p->seg_force = seg_len;
        p->frames_max = cwth_num_frames(max_len, hop);
        p->scales.assign(scales, scales + S);
        p->scale_path.assign(S, CWTH_PATH_SPECTRAL);
        const bool spectral_ok = spectral_hop_ok(hop);
        for (int32_t s = 0; s < S && st == CWTH_OK; ++s) {
            const bool direct_ok = direct_eligible(*p, scales[s]);
            int32_t choice;
            if (path == CWTH_PATH_SPECTRAL)
                choice = spectral_ok ? CWTH_PATH_SPECTRAL : -1;
            else if (path == CWTH_PATH_DIRECT)
                choice = direct_ok ? CWTH_PATH_DIRECT : -1;
            else if (precision == CWTH_PREC_FP32)
                choice = spectral_ok ? CWTH_PATH_SPECTRAL : (direct_ok ? CWTH_PATH_DIRECT : -1);
            else
                choice = direct_ok ? CWTH_PATH_DIRECT : (spectral_ok ? CWTH_PATH_SPECTRAL : -1);
            if (choice < 0)
                st = CWTH_ERR_UNSUPPORTED;
            else
                p->scale_path[s] = choice;
        }
        // Float32 automatic plans with a power-of-two hop: the cost model
        // moves the short-support scales, whose hop fold would cost more
        // than their direct sums, into the spectral kernel's time-domain
        // phase.
        if (st == CWTH_OK && path == CWTH_PATH_AUTO && precision == CWTH_PREC_FP32 && spectral_ok &&
            is_pow2(hop)) {
            std::vector<int32_t> asc(S);
            for (int32_t s = 0; s < S; ++s) asc[s] = s;
            std::stable_sort(asc.begin(), asc.end(),
                             [&](int32_t i, int32_t j) { return scales[i] < scales[j]; });
            const int nf = choose_fused_count(*p, asc);
            for (int i = 0; i < nf; ++i) p->scale_path[asc[i]] = kPathFused;
        }
        // Tables are made on a private non-blocking stream and only that
        // stream is waited for, so planning never stalls other work.
        if (st == CWTH_OK && cudaStreamCreateWithFlags(&p->setup, cudaStreamNonBlocking) != cudaSuccess)
            st = CWTH_ERR_CUDA;
        if (st == CWTH_OK) st = build_direct(p);
        if (st == CWTH_OK) st = split_spectral(p);
        if (st == CWTH_OK) st = build_spectral(p);
        if (p->setup) {
            cudaStreamSynchronize(p->setup);
            cudaStreamDestroy(p->setup);
            p->setup = nullptr;
        }
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

}  // namespace

cwth_status cwth_plan_resampled(const cwth_morlet* w, const double* scales, int32_t S, int32_t hop,
                                double sample_rate, int64_t max_len, int32_t precision,
                                int32_t path, cwth_plan_t* out) {
    if (out) *out = nullptr;
    if (!w || !scales || !out) return CWTH_ERR_INVALID_ARG;
    if (S < 1 || hop < 1 || max_len < 1) return CWTH_ERR_INVALID_ARG;
    if (!(isfinite(sample_rate) && sample_rate > 0)) return CWTH_ERR_INVALID_ARG;
    std::vector<double> sc(scales, scales + S);
    for (double& a : sc) {
        if (!(isfinite(a) && a > 0)) return CWTH_ERR_INVALID_ARG;
        a /= hop;
    }
    cwth_status st = cwth_plan(w, sc.data(), S, 1, sample_rate / hop, cwth_num_frames(max_len, hop),
                               precision, path, out);
    if (st != CWTH_OK) return st;
    (*out)->resample = hop;
    (*out)->in_len = max_len;
    return CWTH_OK;
}

cwth_status cwth_execute(cwth_plan_t p, const float* d_x, int64_t ld_x, const int64_t* d_lengths,
                         int32_t batch, float* d_out, void* stream) {
    cwth::NvtxRange nvtx_range("cwth_execute");
    if (!valid_plan(p)) return CWTH_ERR_BAD_PLAN;
    if (batch < 0) return CWTH_ERR_INVALID_ARG;
    if (batch == 0) return CWTH_OK;
    if (!d_x || !d_out || ld_x < input_len(p)) return CWTH_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    if (!g.ok) return CWTH_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    return launch_transform(p, d_x, ld_x, d_lengths, batch, d_out, st, true, 0, batch);
}

cwth_status cwth_execute_host(cwth_plan_t p, const float* h_x, int64_t ld_x,
                              const int64_t* h_lengths, int32_t batch, float* h_out,
                              void* stream) {
    cwth::NvtxRange nvtx_range("cwth_execute_host");
    if (!valid_plan(p)) return CWTH_ERR_BAD_PLAN;
    if (batch < 0) return CWTH_ERR_INVALID_ARG;
    if (batch == 0) return CWTH_OK;
    if (!h_x || !h_out || ld_x < input_len(p)) return CWTH_ERR_INVALID_ARG;
    DeviceGuard g(p->device);
    if (!g.ok) return CWTH_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nx = (size_t)batch * (size_t)ld_x;
    const size_t per_clip = (size_t)p->S * (size_t)p->frames_max;
    const size_t no = (size_t)batch * per_clip;
    cwth_status s = grow(&p->d_stage_x, &p->stage_x_elems, nx);
    if (s == CWTH_OK) s = grow(&p->d_stage_out, &p->stage_out_elems, no);
    if (s == CWTH_OK && h_lengths) s = grow(&p->d_stage_len, &p->stage_len_elems, (size_t)batch);
    if (s != CWTH_OK) return s;
    cudaError_t e = host_pipeline_init(p);
    if (e != cudaSuccess) return cuda_status(e);

    // Frames written per clip (only the written prefix of a short clip's
    // rows is copied back; the rest of h_out stays untouched).
    std::vector<int64_t> F;
    if (h_lengths) {
        F.resize(batch);
        for (int32_t i = 0; i < batch; ++i) {
            const int64_t len = std::min<int64_t>(std::max<int64_t>(h_lengths[i], 0), input_len(p));
            F[i] = cwth_num_frames(len, p->hop * p->resample);
        }
    }
    // Chunk c: upload on h2d, transform on `stream`, download on d2h.  Each
    // event is waited for right after it is recorded, so one event per edge
    // serves every chunk.  The plan's streams start after the work already
    // on `stream`, and `stream` ends with the last download.  A plan without
    // direct-path scales (whose launches share one staging workspace)
    // transforms odd chunks on a second stream, so that a chunk's last wave
    // of CTAs overlaps the next chunk's first.
    const int32_t nch = host_chunk_count(p, batch, ld_x);
    const bool two = nch > 1 && p->n_dir == 0;
    e = cudaEventRecord(p->ev_start, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->h2d, p->ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->d2h, p->ev_start, 0);
    if (e == cudaSuccess && two) e = cudaStreamWaitEvent(p->cs2, p->ev_start, 0);
    if (e == cudaSuccess && h_lengths)
        e = cudaMemcpyAsync(p->d_stage_len, h_lengths, (size_t)batch * sizeof(int64_t),
                            cudaMemcpyHostToDevice, p->h2d);
    for (int32_t c = 0; c < nch && e == cudaSuccess && s == CWTH_OK; ++c) {
        const int32_t b0 = (int32_t)((int64_t)batch * c / nch);
        const int32_t b1 = (int32_t)((int64_t)batch * (c + 1) / nch);
        const int32_t nb = b1 - b0;
        float* dx = p->d_stage_x + (size_t)b0 * ld_x;
        float* dout = p->d_stage_out + (size_t)b0 * per_clip;
        e = cudaMemcpyAsync(dx, h_x + (size_t)b0 * ld_x, (size_t)nb * ld_x * sizeof(float),
                            cudaMemcpyHostToDevice, p->h2d);
        cudaStream_t cs = (two && (c & 1)) ? p->cs2 : st;
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_in, p->h2d);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, p->ev_in, 0);
        if (e != cudaSuccess) break;
        s = launch_transform(p, dx, ld_x, h_lengths ? p->d_stage_len + b0 : nullptr, nb, dout, cs,
                             nch == 1, b0, batch);
        if (s != CWTH_OK) break;
        e = cudaEventRecord(p->ev_comp, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->d2h, p->ev_comp, 0);
        if (e != cudaSuccess) break;
        if (!h_lengths) {
            e = cudaMemcpyAsync(h_out + (size_t)b0 * per_clip, dout, (size_t)nb * per_clip * sizeof(float),
                                cudaMemcpyDeviceToHost, p->d2h);
        } else {
            for (int32_t i = b0; i < b1 && e == cudaSuccess; ++i) {
                if (F[i] == 0) continue;
                e = cudaMemcpy2DAsync(h_out + (size_t)i * per_clip, (size_t)p->frames_max * sizeof(float),
                                      p->d_stage_out + (size_t)i * per_clip,
                                      (size_t)p->frames_max * sizeof(float), (size_t)F[i] * sizeof(float),
                                      (size_t)p->S, cudaMemcpyDeviceToHost, p->d2h);
            }
        }
    }
    // Join whatever was enqueued, also after a failure part-way.
    cudaError_t ej = cudaEventRecord(p->ev_out, p->d2h);
    if (ej == cudaSuccess) ej = cudaStreamWaitEvent(st, p->ev_out, 0);
    if (ej != cudaSuccess) {
        cudaStreamSynchronize(p->h2d);
        cudaStreamSynchronize(p->cs2);
        cudaStreamSynchronize(p->d2h);
    }
    cudaError_t es = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    if (s != CWTH_OK) return s;
    if (ej != cudaSuccess) return cuda_status(ej);
    return cuda_status(es);
}

cwth_status cwth_plan_reserve(cwth_plan_t p, int32_t batch, int64_t ld_x, int32_t host) {
    if (!valid_plan(p)) return CWTH_ERR_BAD_PLAN;
    if (batch < 0 || (host && ld_x < input_len(p))) return CWTH_ERR_INVALID_ARG;
    if (batch == 0) return CWTH_OK;
    DeviceGuard g(p->device);
    if (!g.ok) return CWTH_ERR_CUDA;
    cwth_status s = CWTH_OK;
    if (p->n_dir > 0 && p->precision != CWTH_PREC_FP32) {
        const DirStageShape sh = dir_stage_shape(p, batch);
        if (sh.total_rows > (int64_t(1) << 31) - 256) return CWTH_ERR_UNSUPPORTED;
        s = dir_stage_grow(p, sh.total);
    }
    if (s == CWTH_OK && p->resample > 1) {
        s = grow(&p->d_res, &p->res_elems, (size_t)batch * (size_t)p->max_len);
        if (s == CWTH_OK) s = grow(&p->d_res_len, &p->res_len_elems, (size_t)batch);
    }
    if (s == CWTH_OK && host) {
        s = grow(&p->d_stage_x, &p->stage_x_elems, (size_t)batch * (size_t)ld_x);
        if (s == CWTH_OK)
            s = grow(&p->d_stage_out, &p->stage_out_elems,
                     (size_t)batch * (size_t)p->S * (size_t)p->frames_max);
        if (s == CWTH_OK) s = grow(&p->d_stage_len, &p->stage_len_elems, (size_t)batch);
        if (s == CWTH_OK) s = cuda_status(host_pipeline_init(p));
    }
    return s;
}

cwth_status cwth_plan_stage_bytes(cwth_plan_t p, int32_t batch, size_t* bytes) {
    if (!valid_plan(p)) return CWTH_ERR_BAD_PLAN;
    if (!bytes || batch < 0) return CWTH_ERR_INVALID_ARG;
    *bytes = dir_stage_bytes(p, batch);
    return CWTH_OK;
}

cwth_status cwth_plan_bind_stage(cwth_plan_t p, void* buf, size_t bytes) {
    if (!valid_plan(p)) return CWTH_ERR_BAD_PLAN;
    if (buf && (bytes == 0 || ((uintptr_t)buf & 15) != 0)) return CWTH_ERR_INVALID_ARG;
    p->ext_stage = buf;
    p->ext_stage_bytes = buf ? bytes : 0;
    return CWTH_OK;
}

cwth_status cwth_plan_set_host_chunks(cwth_plan_t p, int32_t chunks) {
    if (!valid_plan(p)) return CWTH_ERR_BAD_PLAN;
    if (chunks < 0) return CWTH_ERR_INVALID_ARG;
    p->host_chunks = chunks;
    return CWTH_OK;
}

cwth_status cwth_plan_set_inverse_radix(cwth_plan_t p, int32_t radix) {
    if (!valid_plan(p)) return CWTH_ERR_BAD_PLAN;
    if (radix != 0 && radix != 8 && radix != 16) return CWTH_ERR_INVALID_ARG;
    for (const cwth_plan_s* q = p; q; q = q->child)
        if (radix == 8 && q->n_sp > 0 && !q->inv_r8_ok) return CWTH_ERR_UNSUPPORTED;
    for (cwth_plan_s* q = p; q; q = q->child)
        q->inv_r8 = q->n_sp > 0 && (radix == 0 ? q->inv_r8_model : radix == 8);
    return CWTH_OK;
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
    info->spectral_parts = p->n_sp + p->n_fd > 0 ? 1 : 0;
    for (const cwth_plan_s* q = p->child; q; q = q->child) {
        info->num_spectral += q->n_sp;
        info->spectral_parts += 1;
    }
    info->num_direct = p->n_dir + p->n_fd;
    info->num_fused = p->n_fd;
    info->seg_len = p->M;
    info->seg_frames = p->seg_frames;
    info->seg_halo = p->halo;
    info->fold_len = p->P;
    info->num_segments = p->n_seg;
    info->direct_taps = p->dir_taps;
    info->table_bytes = p->table_bytes;
    info->sample_rate = p->fs;
    info->resample = p->resample;
    if (p->n_sp > 0 || p->n_fd > 0) {
        info->spectral_threads = spectral_threads(p->M, p->P, fd_bytes(p));
        int nc = p->n_sp > 0 ? spectral_nconc(p->M, p->P, p->n_sp, info->spectral_threads,
                                              fd_bytes(p))
                             : 0;
        if (nc > 1) nc &= ~1;  // passes hold whole fold pairs (see spectral_record)
        info->spectral_pass_scales = nc;
        info->spectral_pruned = p->spec_prune ? 1 : 0;
        info->inverse_radix = p->n_sp > 0 ? (p->inv_r8 ? 8 : 16) : 0;
    }
    const int64_t xparts = p->x_elems ? (p->d_xlo2 ? 3 : 2) : 0;
    info->workspace_bytes = (int64_t)(p->x_elems * xparts * sizeof(__nv_bfloat16) +
                                      p->res_elems * sizeof(float) +
                                      p->res_len_elems * sizeof(int64_t) +
                                      p->stage_x_elems * sizeof(float) +
                                      p->stage_out_elems * sizeof(float) +
                                      p->stage_len_elems * sizeof(int64_t));
    return CWTH_OK;
}

cwth_status cwth_sync(cwth_plan_t p, void* stream) {
    if (!valid_plan(p)) return CWTH_ERR_BAD_PLAN;
    DeviceGuard g(p->device);
    if (!g.ok) return CWTH_ERR_CUDA;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (p->d_status) {
        int flag = 0;
        e = cudaMemcpy(&flag, p->d_status, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_status(e);
        if (flag != 0) {
            cudaMemset(p->d_status, 0, sizeof(int));
            return (cwth_status)flag;
        }
    }
    return CWTH_OK;
}

cwth_status cwth_selftest_wait_timeout(cwth_plan_t p, int64_t budget_cycles, void* stream) {
    if (budget_cycles < 1 || budget_cycles > kMaxSelftestBudget) return CWTH_ERR_INVALID_ARG;
    if (!p) {
        // The allocation-free entry point's status word on the current device.
        int* word = nullptr;
        const cwth_status st = cwth::noalloc_status_word(&word);
        if (st != CWTH_OK) return st;
        return cuda_status(
            cwth::direct_wait_selftest(word, (long long)budget_cycles, (cudaStream_t)stream));
    }
    if (!valid_plan(p)) return CWTH_ERR_BAD_PLAN;
    DeviceGuard g(p->device);
    if (!g.ok) return CWTH_ERR_CUDA;
    if (!p->d_status) {
        cudaError_t e = cudaMalloc((void**)&p->d_status, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
        if (e != cudaSuccess) return cuda_status(e);
    }
    return cuda_status(
        cwth::direct_wait_selftest(p->d_status, (long long)budget_cycles, (cudaStream_t)stream));
}

cwth_status cwth_plan_scale_paths(cwth_plan_t p, int32_t* paths) {
    if (!valid_plan(p)) return CWTH_ERR_BAD_PLAN;
    if (!paths) return CWTH_ERR_INVALID_ARG;
    for (int s = 0; s < p->S; ++s)
        paths[s] = p->scale_path[s] == kPathFused
                       ? CWTH_PATH_DIRECT
                       : (p->scale_path[s] == kPathSpectralChild ? CWTH_PATH_SPECTRAL
                                                                 : p->scale_path[s]);
    return CWTH_OK;
}

cwth_status cwth_batch_create(int32_t n, const cwth_plan_t* plans, const float* const* d_x,
                              const int64_t* ld_x, const int64_t* const* d_lengths,
                              const int64_t* const* h_lengths, const int32_t* batch,
                              float* const* d_out, cwth_batch_t* out) {
    if (out) *out = nullptr;
    if (!out || !plans || !d_x || !ld_x || !batch || !d_out) return CWTH_ERR_INVALID_ARG;
    if (n < 1 || n > cwth::kMaxBatchGroups) return CWTH_ERR_INVALID_ARG;
    int dev = -1;
    for (int32_t i = 0; i < n; ++i) {
        const cwth_plan_s* p = plans[i];
        if (!valid_plan(p)) return CWTH_ERR_BAD_PLAN;
        if (batch[i] < 0 || batch[i] > 65535) return CWTH_ERR_INVALID_ARG;
        if (batch[i] > 0 && (!d_x[i] || !d_out[i] || ld_x[i] < input_len(p)))
            return CWTH_ERR_INVALID_ARG;
        if (dev >= 0 && p->device != dev) return CWTH_ERR_INVALID_ARG;
        dev = p->device;
        // One launch of the paired spectral kernel serves plans whose every
        // scale is spectral or fused, without pruned inverse FFTs or
        // re-sampling.
        if (p->n_dir > 0 || p->resample > 1 || p->spec_prune || p->child) {
            note_error("batched plans must be one-part float32 spectral/fused plans without "
                       "pruning or re-sampling");
            return CWTH_ERR_UNSUPPORTED;
        }
        if ((p->n_sp > 0 || p->n_fd > 0) &&
            spectral_threads(p->M, p->P, fd_bytes(p)) != cwth::kSpecThreadsPair) {
            note_error("a batched plan needs the two-CTAs-per-SM (512-thread) shape");
            return CWTH_ERR_UNSUPPORTED;
        }
    }
    cwth_batch_s* b = new (std::nothrow) cwth_batch_s();
    if (!b) return CWTH_ERR_OOM;
    b->wl = new (std::nothrow) cwth::SpecWorkList();
    if (!b->wl) {
        delete b;
        return CWTH_ERR_OOM;
    }
    b->device = dev;
    memset(b->wl, 0, sizeof(cwth::SpecWorkList));
    // Items of every group: each clip's segments up to its length, each
    // segment's scale groups.  Ordered by the cost model's work per segment,
    // largest first (stable within a group).
    std::vector<std::pair<double, int4>> items;
    try {
        for (int32_t i = 0; i < n; ++i) {
            cwth_plan_s* p = plans[i];
            if (batch[i] == 0 || (p->n_sp == 0 && p->n_fd == 0)) continue;
            SpecLaunch L;
            int threads = 0, ngrp = 1;
            size_t smem = 0;
            spectral_record(p, d_x[i], ld_x[i], d_lengths ? d_lengths[i] : nullptr, batch[i],
                            d_out[i], false, &L, &threads, &ngrp, &smem);
            b->wl->g[i] = L;
            b->smem = std::max(b->smem, smem);
            for (int32_t c = 0; c < batch[i]; ++c) {
                int64_t len = p->max_len;
                if (h_lengths && h_lengths[i])
                    len = std::min<int64_t>(std::max<int64_t>(h_lengths[i][c], 0), p->max_len);
                const int64_t F = cwth_num_frames(len, p->hop);
                const int64_t nseg = (F + p->seg_frames - 1) / p->seg_frames;
                for (int64_t sgm = 0; sgm < nseg; ++sgm)
                    for (int g = 0; g < ngrp; ++g)
                        items.push_back({p->seg_cost / ngrp,
                                         make_int4(i, (int)sgm, (int)c, g | (ngrp << 16))});
            }
        }
    } catch (...) {
        delete b->wl;
        delete b;
        return CWTH_ERR_OOM;
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<double, int4>& x, const std::pair<double, int4>& y) {
                         return x.first > y.first;
                     });
    if (items.size() > 0x7fffffff) {
        delete b->wl;
        delete b;
        return CWTH_ERR_UNSUPPORTED;
    }
    b->n_items = (int64_t)items.size();
    b->wl->n_items = (int32_t)items.size();
    b->wl->n_groups = n;
    DeviceGuard gd(dev);
    cudaError_t e = gd.ok ? cudaSuccess : cudaErrorInvalidDevice;
    if (e == cudaSuccess && !items.empty()) {
        std::vector<int4> h(items.size());
        for (size_t k = 0; k < items.size(); ++k) h[k] = items[k].second;
        e = cudaMalloc(&b->d_items, sizeof(int4) * h.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_items, h.data(), sizeof(int4) * h.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cwth::spectral_prepare_device();
    if (e != cudaSuccess) {
        cudaFree(b->d_items);
        delete b->wl;
        delete b;
        return cuda_status(e);
    }
    b->wl->items = b->d_items;
    b->magic = cwth::kPlanMagic ^ 0x5A5A5A5Au;
    *out = b;
    return CWTH_OK;
}

cwth_status cwth_batch_execute(cwth_batch_t b, void* stream) {
    cwth::NvtxRange nvtx_range("cwth_batch_execute");
    if (!b || b->magic != (cwth::kPlanMagic ^ 0x5A5A5A5Au)) return CWTH_ERR_BAD_PLAN;
    DeviceGuard g(b->device);
    if (!g.ok) return CWTH_ERR_CUDA;
    return cuda_status(cwth::spectral_worklist_launch(*b->wl, b->smem, (cudaStream_t)stream));
}

int64_t cwth_batch_items(cwth_batch_t b) {
    if (!b || b->magic != (cwth::kPlanMagic ^ 0x5A5A5A5Au)) return -1;
    return b->n_items;
}

cwth_status cwth_batch_destroy(cwth_batch_t b) {
    if (!b) return CWTH_OK;
    if (b->magic != (cwth::kPlanMagic ^ 0x5A5A5A5Au)) return CWTH_ERR_BAD_PLAN;
    DeviceGuard g(b->device);
    b->magic = 0;
    cudaFree(b->d_items);
    delete b->wl;
    delete b;
    return CWTH_OK;
}

}  // extern "C"
