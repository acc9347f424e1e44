// cwth_execute_direct_noalloc: the tensor-core direct path with every piece of
// scratch memory (tap bank, per-scale tables, staged bf16 signal, status
// word) carved out of one fixed array compiled into the library, for callers
// that must not allocate device memory while they run (see include/cwth.h).
#include <limits.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "cwth_internal.h"

namespace {

// Scratch shared by every call on a device.  Each GPU that loads libcwth.so
// holds this much device memory until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)CWTH_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
constexpr int kMaxScales = 1024;
constexpr int kScalesPerGroup = 128;     // N = 256 columns per GEMM
constexpr double kEpsTaps = 1e-9;        // tap truncation, as the planned direct path
constexpr int kMaxTaps = 4096;

std::mutex g_mu;
void* g_scratch_dev[kMaxDevices];        // device address of the array, per device
bool g_ready[kMaxDevices];

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                             CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                             CUtensorMapFloatOOBfill);
EncodeFn g_encode = nullptr;

int64_t rup(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

int32_t half_support(double a, double B) {
    return (int32_t)rup((int64_t)ceil(a * sqrt(B * log(1.0 / kEpsTaps))), 8);
}

bool encode(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer, uint64_t stride,
            uint32_t box_outer) {
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {stride};
    const cuuint32_t box[2] = {64, box_outer};
    const cuuint32_t estr[2] = {1, 1};
    return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cwth_status fail(cwth_status s, const char* msg) {
    cwth::set_last_error(msg);
    return s;
}

cwth_status fail_cuda(cudaError_t e) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    cwth::set_last_error(buf);
    return e == cudaErrorMemoryAllocation ? CWTH_ERR_OOM : CWTH_ERR_CUDA;
}

// Once per device, with that device current: the array's device address
// (its name is only a host-side stand-in in host code), the kernels'
// shared-memory opt-in and the driver's tensor-map encoder.
cwth_status setup(int dev, void** scratch) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (dev < 0 || dev >= kMaxDevices) return fail(CWTH_ERR_UNSUPPORTED, "device index out of range");
    if (!g_ready[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return fail_cuda(e);
        e = cwth::direct_prepare_device();
        if (e != cudaSuccess) return fail_cuda(e);
        if (!g_encode) {
            void* fn = nullptr;
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                 cudaEnableDefault, &q) != cudaSuccess ||
                q != cudaDriverEntryPointSuccess)
                return fail(CWTH_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
            g_encode = (EncodeFn)fn;
        }
        g_scratch_dev[dev] = ptr;
        g_ready[dev] = true;
    }
    *scratch = g_scratch_dev[dev];
    return CWTH_OK;
}

}  // namespace

namespace cwth {
// Device address of the allocation-free entry point's status word on the
// current device (the first word of its scratch array), setting the device
// up on first use.
cwth_status noalloc_status_word(int** word) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e);
    void* base = nullptr;
    const cwth_status st = setup(dev, &base);
    if (st != CWTH_OK) return st;
    *word = (int*)base;
    return CWTH_OK;
}
}  // namespace cwth

extern "C" {

cwth_status cwth_noalloc_status(void* stream) {
    int* word = nullptr;
    cwth_status st = cwth::noalloc_status_word(&word);
    if (st != CWTH_OK) return st;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&flag, word, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && flag != 0) e = cudaMemset(word, 0, sizeof(int));
    if (e != cudaSuccess) return fail_cuda(e);
    return flag != 0 ? (cwth_status)flag : CWTH_OK;
}


cwth_status cwth_execute_direct_noalloc(const cwth_morlet* w, const double* scales, int32_t S,
                                        int32_t hop, int32_t precision, const float* d_x,
                                        int64_t ld_x, int64_t max_len, const int64_t* d_lengths,
                                        int32_t batch, float* d_out, void* stream) {
    cwth::NvtxRange nvtx_range("cwth_execute_direct_noalloc");
    if (!w || !scales) return fail(CWTH_ERR_INVALID_ARG, "NULL wavelet or scale list");
    if (S < 1 || S > kMaxScales) return fail(CWTH_ERR_INVALID_ARG, "S must be in [1, 1024]");
    if (hop < 8 || hop % 8 != 0) return fail(CWTH_ERR_INVALID_ARG, "hop must be a positive multiple of 8");
    if (precision != CWTH_PREC_BF16 && precision != CWTH_PREC_BF16X2 &&
        precision != CWTH_PREC_BF16X3)
        return fail(CWTH_ERR_INVALID_ARG,
                    "precision must be CWTH_PREC_BF16, CWTH_PREC_BF16X2 or CWTH_PREC_BF16X3");
    const int nparts = precision == CWTH_PREC_BF16X3 ? 3 : (precision == CWTH_PREC_BF16X2 ? 2 : 1);
    if (!(isfinite(w->bandwidth) && w->bandwidth > 0 && isfinite(w->center_freq) &&
          w->center_freq > 0))
        return fail(CWTH_ERR_INVALID_ARG, "bandwidth and centre frequency must be positive");
    if (max_len < 1 || batch < 0) return fail(CWTH_ERR_INVALID_ARG, "max_len < 1 or batch < 0");
    for (int32_t s = 0; s < S; ++s)
        if (!(isfinite(scales[s]) && scales[s] > 0))
            return fail(CWTH_ERR_INVALID_ARG, "scales must be finite and positive");
    if (batch == 0) return CWTH_OK;
    if (!d_x || !d_out || ld_x < max_len) return fail(CWTH_ERR_INVALID_ARG, "NULL buffer or ld_x < max_len");
    if ((int64_t)S * ((max_len + hop - 1) / hop) > INT32_MAX)
        return fail(CWTH_ERR_UNSUPPORTED, "one clip's output exceeds 2^31 elements");

    // Per-scale supports (stack arrays only).
    int32_t order[kMaxScales], hs[kMaxScales];
    double sc[kMaxScales];
    for (int32_t s = 0; s < S; ++s) {
        order[s] = s;
        hs[s] = half_support(scales[s], w->bandwidth);
        if (rup(2 * (int64_t)hs[s] + 1, 64) > kMaxTaps)
            return fail(CWTH_ERR_UNSUPPORTED, "a scale needs more than 4096 taps");
    }
    // Insertion sort (stable), descending scale - the planned direct path's
    // order, so that both put the same scales in each 128-scale group and
    // give the same bytes; supports then descend too.
    for (int32_t i = 1; i < S; ++i) {
        const int32_t v = order[i];
        int32_t j = i - 1;
        while (j >= 0 && scales[order[j]] < scales[v]) {
            order[j + 1] = order[j];
            --j;
        }
        order[j + 1] = v;
    }
    int32_t h_sorted[kMaxScales];
    for (int32_t i = 0; i < S; ++i) {
        h_sorted[i] = hs[order[i]];
        sc[i] = scales[order[i]];
    }

    const int n_groups = (S + kScalesPerGroup - 1) / kScalesPerGroup;
    int32_t front = 0, max_taps = 0;
    for (int g = 0; g < n_groups; ++g) {
        const int first = g * kScalesPerGroup;
        front = std::max(front, h_sorted[first]);
        max_taps = std::max<int32_t>(max_taps, (int32_t)rup(2 * (int64_t)h_sorted[first] + 1, 64));
    }
    const int64_t frames_max = (max_len + hop - 1) / hop;
    const int64_t rows_per_clip = (2 * (int64_t)front + frames_max * hop + max_taps + hop - 1) / hop;
    const int64_t lpad = rows_per_clip * hop;
    const int64_t total_rows = (int64_t)batch * rows_per_clip;
    const int64_t sig_elems = (int64_t)batch * lpad + front + max_taps + 64;

    // Scratch layout (256-byte aligned pieces).
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = (size_t)rup((int64_t)(off + bytes), 256);
        return o;
    };
    const size_t o_status = take(sizeof(int));  // 0: cwth_noalloc_status reads it there
    const size_t o_rows = take(sizeof(int32_t) * S);
    const size_t o_h = take(sizeof(int32_t) * S);
    const size_t o_sc = take(sizeof(double) * S);
    const size_t o_sched = take(sizeof(int2) * 3 * (kMaxTaps / 64) * ((kMaxScales + kScalesPerGroup - 1) / kScalesPerGroup));
    size_t o_bank[(kMaxScales + kScalesPerGroup - 1) / kScalesPerGroup];
    int32_t ncols[(kMaxScales + kScalesPerGroup - 1) / kScalesPerGroup];
    int32_t kpad[(kMaxScales + kScalesPerGroup - 1) / kScalesPerGroup];
    for (int g = 0; g < n_groups; ++g) {
        const int first = g * kScalesPerGroup;
        const int n = std::min(S, first + kScalesPerGroup) - first;
        ncols[g] = (int32_t)rup(2 * n, 16);
        kpad[g] = (int32_t)rup(2 * (int64_t)h_sorted[first] + 1, 64);
        o_bank[g] = take((size_t)ncols[g] * kpad[g] * (nparts > 2 ? 3 : 2) * sizeof(__nv_bfloat16));
    }
    if (total_rows > (int64_t(1) << 31) - 256)
        return fail(CWTH_ERR_INVALID_ARG, "batch too large for one launch");
    const size_t o_sig = take((size_t)sig_elems * (nparts > 2 ? 3 : 2) * sizeof(__nv_bfloat16));
    if (off > kNoAllocScratchBytes) {
        char buf[256];
        snprintf(buf, sizeof(buf),
                 "request needs %zu bytes of scratch; the allocation-free entry point holds "
                 "%zu bytes (reduce batch, max_len or scales)",
                 off, kNoAllocScratchBytes);
        cwth::set_last_error(buf);
        return CWTH_ERR_INVALID_ARG;
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e);
    void* base_v = nullptr;
    cwth_status st = setup(dev, &base_v);
    if (st != CWTH_OK) return st;
    unsigned char* base = (unsigned char*)base_v;
    cudaStream_t strm = (cudaStream_t)stream;

    int* d_status = (int*)(base + o_status);
    int32_t* d_rows = (int32_t*)(base + o_rows);
    int32_t* d_h = (int32_t*)(base + o_h);
    double* d_sc = (double*)(base + o_sc);
    __nv_bfloat16* d_xhi = (__nv_bfloat16*)(base + o_sig);
    __nv_bfloat16* d_xlo = d_xhi + sig_elems;
    __nv_bfloat16* d_xlo2 = d_xlo + sig_elems;

    // The small tables are rewritten on every call, the banks and the staged
    // signal in full by their kernels.  The status word is not: it keeps a
    // bounded-wait timeout until cwth_noalloc_status reads and clears it
    // (the array starts zeroed when the library loads).
    e = cudaMemcpyAsync(d_rows, order, sizeof(int32_t) * S, cudaMemcpyHostToDevice, strm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_h, h_sorted, sizeof(int32_t) * S, cudaMemcpyHostToDevice, strm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_sc, sc, sizeof(double) * S, cudaMemcpyHostToDevice, strm);
    if (e != cudaSuccess) return fail_cuda(e);

    // Centre-out K schedules of all groups, one slot of kMaxTaps/64 steps each.
    const bool split = nparts > 1;
    int2 sched[(kMaxScales + kScalesPerGroup - 1) / kScalesPerGroup][3 * (kMaxTaps / 64)];
    int32_t nsteps[(kMaxScales + kScalesPerGroup - 1) / kScalesPerGroup];
    int2* d_sched = (int2*)(base + o_sched);
    for (int g = 0; g < n_groups; ++g) {
        const int first = g * kScalesPerGroup;
        const int n = std::min(S, first + kScalesPerGroup) - first;
        int2 one[kMaxTaps / 64];
        const cwth::DirShape sh = cwth::direct_shape(ncols[g], nparts, hop, kpad[g]);
        nsteps[g] = cwth::direct_schedule(h_sorted + first, n, h_sorted[first], kpad[g],
                                          (ncols[g] + 63) / 64,
                                          cwth::direct_a_pieces(nparts, sh.unit, sh.win_rows > 0),
                                          one);
        if (split)
            nsteps[g] = cwth::direct_split_schedule(one, nsteps[g], nparts, sched[g]);
        else
            for (int i = 0; i < nsteps[g]; ++i) sched[g][i] = one[i];
    }
    e = cudaMemcpyAsync(d_sched, sched, sizeof(sched[0]) * n_groups, cudaMemcpyHostToDevice, strm);
    if (e != cudaSuccess) return fail_cuda(e);

    for (int g = 0; g < n_groups; ++g) {
        const int first = g * kScalesPerGroup;
        const int n = std::min(S, first + kScalesPerGroup) - first;
        __nv_bfloat16* bhi = (__nv_bfloat16*)(base + o_bank[g]);
        __nv_bfloat16* blo = bhi + (size_t)ncols[g] * kpad[g];
        e = cwth::direct_make_bank(d_sc + first, d_h + first, n, ncols[g], kpad[g],
                                   h_sorted[first], w->bandwidth, w->center_freq, bhi, blo,
                                   nparts > 2 ? blo + (size_t)ncols[g] * kpad[g] : nullptr,
                                   nullptr, strm);
        if (e != cudaSuccess) return fail_cuda(e);
    }
    e = cwth::direct_stage(d_x, ld_x, d_lengths, max_len, batch, d_xhi, split ? d_xlo : nullptr,
                           nparts > 2 ? d_xlo2 : nullptr,
                           lpad, front, sig_elems, strm);
    if (e != cudaSuccess) return fail_cuda(e);

    cwth::DirLaunch L;
    memset(&L, 0, sizeof(L));
    L.out = d_out;
    L.frames_max = frames_max;
    L.S_total = S;
    L.hop = hop;
    L.lengths = d_lengths;
    L.max_len = max_len;
    L.batch = batch;
    L.rows_per_clip = rows_per_clip;
    L.total_rows = total_rows;
    L.status = d_status;
    for (int g = 0; g < n_groups; ++g) {
        const int first = g * kScalesPerGroup;
        const int n = std::min(S, first + kScalesPerGroup) - first;
        const int32_t hg = h_sorted[first];
        __nv_bfloat16* bhi = (__nv_bfloat16*)(base + o_bank[g]);
        __nv_bfloat16* blo = bhi + (size_t)ncols[g] * kpad[g];
        CUtensorMap maps[6];
        __nv_bfloat16* blo2 = blo + (size_t)ncols[g] * kpad[g];
        const int64_t aoff = front - hg;
        if (!encode(&maps[0], d_xhi + aoff, kpad[g], total_rows, (uint64_t)hop * 2, 32) ||
            !encode(&maps[1], d_xlo + aoff, kpad[g], total_rows, (uint64_t)hop * 2, 32) ||
            (nparts > 2 &&
             !encode(&maps[2], d_xlo2 + aoff, kpad[g], total_rows, (uint64_t)hop * 2, 32)) ||
            !encode(&maps[3], bhi, kpad[g], ncols[g], (uint64_t)kpad[g] * 2, 64) ||
            !encode(&maps[4], blo, kpad[g], ncols[g], (uint64_t)kpad[g] * 2, 64) ||
            (nparts > 2 && !encode(&maps[5], blo2, kpad[g], ncols[g], (uint64_t)kpad[g] * 2, 64)))
            return fail(CWTH_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled rejected a tensor map");
        L.ncols = ncols[g];
        L.k_pad = kpad[g];
        L.h_group = hg;
        L.n_scales = n;
        L.rows = d_rows + first;
        const cwth::DirShape sh = cwth::direct_shape(ncols[g], nparts, hop, kpad[g]);
        L.stages = sh.stages;
        L.win_rows = sh.win_rows;
        L.a_shift = sh.win_rows ? cwth::direct_window_shift(hop) : 0;
        L.a_phases = sh.win_rows ? sh.phases : 1;
        L.unit = sh.unit;
        L.win_sets = sh.win_sets;
        L.acc_sets = sh.acc_sets;
        L.sched = d_sched + (size_t)g * 3 * (kMaxTaps / 64);
        L.nsteps = nsteps[g];
        L.tmem_cols = sh.tmem_cols;
        if (L.stages == 0) return fail(CWTH_ERR_UNSUPPORTED, "tile does not fit in shared memory");
        e = cwth::direct_launch_mma(maps, L, nparts, strm);
        if (e != cudaSuccess) return fail_cuda(e);
    }
    return CWTH_OK;
}

}  // extern "C"
