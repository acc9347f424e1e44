// Internal declarations shared by the translation units of libcwth.so.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include <algorithm>

#include <nvtx3/nvToolsExt.h>

#include "cwth.h"

namespace cwth {

// A named NVTX range for the duration of a scope (plan, execute, batch,
// server launch), visible in timeline profilers; header-only NVTX v3, a
// no-op unless a tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr uint32_t kPlanMagic = 0xC0A7B17Eu;
// Spectral CTA shapes (64 registers per thread either way): two 512-thread
// CTAs per SM, so one CTA's phase barriers are covered by the other's work,
// or one 1024-thread CTA per SM, which has the whole SM's shared memory and
// so inverts more scales per pass when the inverse FFTs are long.  The pair
// holds 16 points per thread and so runs radix-16 FFT passes; measured on
// GB300 (64 x 10 s clips, 64 scales) it is 5-20 % faster wherever one scale
// per pass fits its shared memory, except at hop 32 (6 % slower); the
// single CTA runs only where the pair does not fit (hop 2 at M = 16384).
constexpr int kSpecThreadsPair = 512;
constexpr int kSpecThreadsSolo = 1024;
// Largest batched shared-memory FFT (complex points) one CTA performs: 16
// points per thread per pass for the 512-thread shape, 8 for 1024.
constexpr int kMaxFftPoints = 8192;

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
    float dlt;       // a P / M: argument step between the bins a residue visits
    float q2;        // 2^(2 kexp dlt^2): ratio of successive weight ratios
    // Upper bound on the folded band width, min(P, q_hi - q_lo + 1), of this
    // and every later scale in the table (a suffix maximum): the band of
    // any chunk of scales starting here fits in wsuf residues once shifted
    // to start at residue 0.
    int32_t wsuf;
    // 1: this scale and the next one of the table share one fold walk over
    // the union of their bands (both weights stay above 1e-20 there, so the
    // weight recurrence cannot lose either to underflow)
    int32_t pair;
};

// Short-support scales evaluated inside the spectral CTA as time-domain
// sums over the segment's staged samples (Eq. 1 at the hop positions, taps
// g[t] = a^{-1/2} conj(psi(t/a)) for |t| <= h): their Morlet bands are wide,
// so folding them by the hop costs about H/a spectrum bins per frame, while
// the direct sum costs 2h + 1 ~ 11 a taps per frame.  Scales are packed in
// groups of up to kFdMaxG with a common tap range; one warp item is one
// group over 32 consecutive frames of the segment.
constexpr int kFdMaxG = 2;
struct FdGroup {
    int32_t off;   // first complex tap of the group's table (an even index)
    int32_t hg;    // the group's half support: table rows tau = 0 .. 2 hg (t = tau - hg)
    int32_t n;     // scales in the group, 1 .. kFdMaxG
    int32_t gp;    // table row length: n rounded up to even (zero taps beyond n)
    int32_t row[kFdMaxG];  // output row of each scale
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
    const float2* tw;  // two-level table: exp(-2 pi i 128 i / M), i < M/128, then exp(-2 pi i j / M), j < 128
    const SpecScale* sc;
    int32_t vec4;      // 1: x rows and segment starts are 16-byte aligned (float4 staging)
    // fused time-domain scales (none when fd_groups == 0)
    int32_t fd_groups;   // tap groups; scale group z of the grid takes groups z, z + nz, ...
    int32_t fd_hw;       // half width of the frame windows: max hg over the groups
    int32_t fd_fst;      // row stride (floats) of the window buffer, odd, >= seg_frames
    int32_t fd_taps_n;   // complex taps of all group tables
    const float2* fd_taps;   // group tables, [2 hg + 1][gp] complex each
    const FdGroup* fd_grp;
    // 1: the inverse FFTs of the 512-thread shape use the radix-8 plan (one
    // radix-8 butterfly per thread: nc * P <= 4096), else radix 16
    int32_t inv_r8;
    // forward FFT of M/2 = fft_d * fft_n2 points: fft_d (the odd part of the
    // hop, 1 for power-of-two hops) column FFTs of fft_n2 = 2^k points, the
    // staged samples permuted into columns, then radix-3/5/7 passes
    int32_t fft_d;
    int32_t fft_n2;
};

// Plan records of a persistent batch launch, passed by value (the launch
// parameters hold up to 32 KB).
constexpr int kMaxBatchGroups = 96;
struct SpecWorkList {
    const int4* items;   // device, {group, segment, clip, scale group | groups << 16}
    int32_t n_items;
    int32_t n_groups;
    SpecLaunch g[kMaxBatchGroups];
};

// Direct (GEMM) path launch parameters; one launch per scale group.
constexpr int kMaxDirStages = 6;
// Schedule steps of one group: at most 4096 taps = 64 tap blocks, each
// visited once per bank part (up to three parts in the split variants).
constexpr int kMaxDirSteps = 192;
struct DirLaunch {
    float* out;
    int64_t frames_max;
    int32_t S_total;
    int32_t hop;
    const int64_t* lengths;
    int64_t max_len;
    int32_t batch;
    int64_t rows_per_clip;  // GEMM rows (frames) reserved per clip
    int64_t total_rows;     // batch * rows_per_clip
    int32_t ncols;          // N: 2 * scales, padded to a multiple of 16
    int32_t k_pad;          // K: padded taps, a multiple of 64
    int32_t h_group;        // half support of the group (taps -h_group .. h_group)
    int32_t n_scales;
    const int32_t* rows;    // output row of each scale of the group
    int32_t stages;
    uint32_t tmem_cols;
    int* status;            // device status word (CWTH_ERR_TIMEOUT on a bounded-wait expiry)
    const int2* sched;      // per K step: {tap blocks, columns used | bank part bits}
    int32_t nsteps;
    int32_t a_shift;        // frame-view rows per tap block (64 / hop; per a_phases blocks
                            // when a_phases > 1) when windows serve all blocks, else 0
    int32_t a_phases;       // frame windows per tile: hop / 64 for hops 128..256, else 1
    int32_t win_rows;       // rows of that window (a multiple of 32)
    int32_t unit;           // 128-frame tiles sharing each bank tile (1 or 2)
    int32_t win_sets;       // frame-window sets (2: the next unit's windows load early)
    int32_t acc_sets;       // tensor-memory accumulator sets (2: epilogue overlaps MMAs)
};

// Launch shape of one direct-path group.
struct DirShape {
    int32_t unit = 0, acc_sets = 0, win_sets = 0, win_rows = 0, stages = 0, phases = 1;
    uint32_t tmem_cols = 0;
};

// Records the detail string cwth_last_error() returns in the calling thread.
void set_last_error(const char* msg);
// Device address of the allocation-free entry point's status word on the
// current device (noalloc.cu).
cwth_status noalloc_status_word(int** word);

size_t spectral_smem_bytes(int M, int P, int nconc, size_t fd_bytes = 0);
// Shared-memory bytes of the fused time-domain scales, held in the fold's
// buffer before the fold: their tap tables (taps_n complex), the n_groups
// group records and the frame windows ((2 hw + 1) rows of fst floats, plus
// slack).
size_t spectral_fd_bytes(int taps_n, int hw, int fst, int n_groups);
cudaError_t spectral_make_fd_taps(const double* d_scales, const int32_t* d_h, const int32_t* d_gidx,
                                  const FdGroup* d_grp, int n_groups, int taps_n, double B,
                                  double C, float2* d_taps, cudaStream_t st);
int spectral_twiddle_entries(int M);
cudaError_t spectral_prepare_device();
cudaError_t spectral_make_twiddles(float2* d_tw, int M, cudaStream_t st);
// dependent: launch as a programmatic dependent of the kernel before it on
// st (a plan's second and later spectral parts; the kernel makes the
// grid complete after its predecessor).
cudaError_t spectral_launch(const SpecLaunch& L, int threads, bool prune, int n_seg, int batch,
                            int n_groups, size_t smem, cudaStream_t st, bool dependent);
// The 1024-thread instantiations (compiled in their own translation unit).
cudaError_t spectral_prepare_solo();
cudaError_t spectral_launch_solo(const SpecLaunch& L, bool prune, dim3 grid, size_t smem,
                                 cudaStream_t st, bool dependent);
// One launch of the paired shape over a work list: block i runs item i,
// {group, segment, clip, scale group | scale groups << 16}, of the plan
// records g[] (passed by value).
cudaError_t spectral_worklist_launch(const SpecWorkList& wl, size_t smem, cudaStream_t st);

// nparts: bf16 parts of each operand (1 = bf16, 2 = bf16x2, 3 = bf16x3).
size_t direct_smem_bytes(int ncols, int stages, int nparts, int win_rows, int unit,
                         int win_sets, int phases);
int direct_max_stages(int ncols, int nparts, int win_rows, int unit, int win_sets, int phases);
DirShape direct_shape(int ncols, int nparts, int hop, int k_pad);
// Rows of the frame window for hops dividing 64 (0: per-step frame tiles).
int direct_window_rows(int hop, int k_pad);
int direct_window_phases(int hop);
int direct_window_shift(int hop);
// The split variants' schedule: every step of `in` nparts times, bank part
// j = 0 .. nparts - 1 in bit 16 (j & 1) and bits 19-20 (j >> 1) of .y;
// returns nparts * n.
int direct_split_schedule(const int2* in, int n, int nparts, int2* out);
cudaError_t direct_prepare_device();
cudaError_t direct_wait_selftest(int* status, long long budget, cudaStream_t st);
cudaError_t resample_launch(const float* x, int64_t ld_x, const int64_t* lengths, int64_t in_len,
                            int32_t H, float* y, int64_t ld_y, int64_t* len_y, int batch,
                            cudaStream_t st);
cudaError_t direct_prepare_f32(size_t smem);
cudaError_t direct_make_bank(const double* d_scales, const int32_t* d_h, int n_scales, int ncols,
                             int k_pad, int h_group, double B, double C, __nv_bfloat16* hi,
                             __nv_bfloat16* lo, __nv_bfloat16* lo2, float2* f32bank,
                             cudaStream_t st);
cudaError_t direct_stage(const float* x, int64_t ld_x, const int64_t* lengths, int64_t max_len,
                         int batch, __nv_bfloat16* hi, __nv_bfloat16* lo, __nv_bfloat16* lo2,
                         int64_t lpad, int64_t h_front, int64_t total, cudaStream_t st);
// maps: {A part 0, 1, 2, bank part 0, 1, 2}; parts past nparts unused.
cudaError_t direct_launch_mma(const CUtensorMap* maps, const DirLaunch& L, int nparts,
                              cudaStream_t st);
// Centre-out K-block schedule of one group (supports in descending order):
// out[i] = {tap block, columns}; returns the number of steps (<= k_pad / 64).
int direct_schedule(const int32_t* h_desc, int n, int h_group, int k_pad, int stage_pieces,
                    int a_pieces, int2* out);
int direct_a_pieces(int nparts, int unit, bool windowed);
cudaError_t direct_launch_f32(const float* x, int64_t ld_x, const float2* bank, const int32_t* d_h,
                              const DirLaunch& L, cudaStream_t st);

// One group of direct-path scales (contiguous in support order).
struct DirGroup {
    int32_t n_scales = 0;
    int32_t ncols = 0;
    int32_t h = 0;       // group half support, a multiple of 8
    int32_t k_pad = 0;   // multiple of 64, >= 2h + 1
    DirShape shape;
    int64_t bank_off = 0;   // element offset into the bf16 banks ([ncols][k_pad])
    int64_t f32_off = 0;    // element offset into the float32 bank ([n_scales][k_pad])
    int32_t* d_rows = nullptr;
    int32_t* d_h = nullptr;
    double* d_scales = nullptr;
    int2* d_sched = nullptr;
    int32_t nsteps = 0;
    CUtensorMap map_b_hi, map_b_lo, map_b_lo2;
};

}  // namespace cwth

struct cwth_plan_s {
    uint32_t magic = 0;
    int device = 0;
    cudaStream_t setup = nullptr;   // private stream used while the plan is built
    double B = 0, C = 0, fs = 0;
    int32_t S = 0, hop = 0, precision = 0, path = 0;
    int64_t max_len = 0, frames_max = 0;
    std::vector<double> scales;
    std::vector<int32_t> scale_path;

    // spectral path
    int32_t n_sp = 0;
    int32_t M = 0, P = 0, halo = 0, kp0 = 0, seg_frames = 0, n_seg = 0;
    bool spec_prune = false;  // narrow bands let inverse FFTs skip passes
    bool inv_r8 = false;      // inverse FFTs on the radix-8 plan
    bool inv_r8_model = false;  // the cost model's choice (cwth_plan_set_inverse_radix 0)
    bool inv_r8_ok = false;     // the radix-8 plan can serve every pass of the plan
    int32_t fft_d = 1, fft_n2 = 0;  // forward FFT: fft_d column FFTs of fft_n2 points
    double seg_cost = 0;      // cost model's lane operations per segment
    int32_t seg_force = 0;    // segment length fixed by cwth_plan_segment (0: cost model)
    // The smallest spectral scales may run as further parts with their own
    // (shorter-halo) segmentations: child plans holding the same scale list
    // and output rows, chained through `child` and launched after this one
    // (null: one part).
    cwth_plan_s* child = nullptr;
    bool no_split = false;    // a child never splits again
    float2* d_tw = nullptr;
    cwth::SpecScale* d_sp = nullptr;
    // short-support scales summed in the time domain inside the spectral
    // kernel (chosen by the cost model of CWTH_PATH_AUTO at float32)
    int32_t n_fd = 0;
    int32_t fd_hw = 0, fd_fst = 0, fd_taps_n = 0;
    std::vector<cwth::FdGroup> fd_groups;
    float2* d_fd_taps = nullptr;
    cwth::FdGroup* d_fd_grp = nullptr;

    // direct path
    int32_t n_dir = 0;
    int32_t dir_taps = 0;      // largest padded tap count over the groups
    int32_t dir_front = 0;     // zero samples before each clip in the staged signal
    std::vector<cwth::DirGroup> groups;
    __nv_bfloat16* d_bank_hi = nullptr;
    __nv_bfloat16* d_bank_lo = nullptr;
    __nv_bfloat16* d_bank_lo2 = nullptr;
    float2* d_bank_f32 = nullptr;
    int* d_status = nullptr;
    // staged bf16 signal (workspace), grown on demand
    __nv_bfloat16* d_xhi = nullptr;
    __nv_bfloat16* d_xlo = nullptr;
    __nv_bfloat16* d_xlo2 = nullptr;
    size_t x_elems = 0;
    // caller-bound staging (cwth_plan_bind_stage): used instead of the
    // plan's own while set
    void* ext_stage = nullptr;
    size_t ext_stage_bytes = 0;
    // A-operand tensor maps per group, valid for (x_maps_ptr, x_maps_rows)
    std::vector<CUtensorMap> maps_a_hi, maps_a_lo, maps_a_lo2;
    const void* x_maps_ptr = nullptr;
    int64_t x_maps_rows = -1;

    int64_t table_bytes = 0;

    // host-API staging (grown on demand)
    float* d_stage_x = nullptr;
    size_t stage_x_elems = 0;
    float* d_stage_out = nullptr;
    size_t stage_out_elems = 0;
    int64_t* d_stage_len = nullptr;
    size_t stage_len_elems = 0;
    // host-API pipeline: clip chunks whose upload, transform and download
    // overlap (copy-in stream, caller's stream, copy-out stream)
    int32_t host_chunks = 0;        // 0 = chosen from the batch size
    // resample-first plans (cwth_plan_resampled): inputs of in_len samples are
    // re-sampled by `resample` into d_res before the hop-1 transform
    int32_t resample = 1;
    int64_t in_len = 0;
    float* d_res = nullptr;
    size_t res_elems = 0;
    int64_t* d_res_len = nullptr;
    size_t res_len_elems = 0;
    cudaStream_t h2d = nullptr, d2h = nullptr, cs2 = nullptr;
    cudaEvent_t ev_start = nullptr, ev_in = nullptr, ev_comp = nullptr, ev_out = nullptr;
};

// A bound uneven batch (cwth_batch_create): the plan records of its groups
// and a device work list, run as one launch of the spectral kernel.
struct cwth_batch_s {
    uint32_t magic = 0;
    int device = 0;
    int64_t n_items = 0;
    size_t smem = 0;
    int4* d_items = nullptr;
    cwth::SpecWorkList* wl = nullptr;  // host copy, passed by value at launch
};

