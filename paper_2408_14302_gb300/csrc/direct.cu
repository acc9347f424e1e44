// Direct path of the hop-size CWT (paper Sec. II.A Eq. 1 + Sec. II.B hop):
//
//     W_s[k] = sum_{t=-h}^{h} x[kH + t] * g_s[t],   g_s[t] = a_s^{-1/2} conj(psi(t/a_s)),
//
// evaluated as a GEMM C[frames x 2S] = A[frames x taps] * B[taps x 2S] with
// A[k, tau] = x[kH - h + tau] (the hop-strided frame matrix, never
// materialised: a TMA view of the padded signal whose row stride is H) and B
// the real/imaginary columns of the zero-padded tap bank.  Scales are
// grouped by support (at most 128 per group, columns in descending support);
// each group is one GEMM whose K loop starts at the centre tap block and
// then walks outwards, each block's MMA covering only the columns of the
// scales whose support reaches it (a pyramid of MMAs instead of a padded
// rectangle).
//
// tcgen05 kernel (bf16 operands, f32 accumulation in tensor memory): a
// persistent CTA per SM walks 128-frame tiles of one group with 10 warps:
//   warp 0      TMA producer (frame windows or A tiles, bank tiles, 128B swizzle)
//   warp 1      TMEM allocation + elected-lane MMA issue (M=128, N<=256, K=16)
//   warps 2..9  epilogue: tcgen05.ld, |re + i im|, coalesced stores along k
// The split variants represent x and g as sums of bf16 parts, x = x_0 + x_1
// (+ x_2), each part the bf16 rounding of what the earlier ones leave, and
// accumulate the part products into the same tensor-memory accumulator:
// "bf16x2" (two parts, within 2^-18 of each value) takes all four products,
// so every tap product is within about 2^-17 relative of x * g; "bf16x3"
// (three parts, within 2^-26) takes the six products x_i g_j with
// i + j <= 2, within about 2^-24 relative (the dropped ones are smaller
// still), which holds the sum to float32 accuracy even where the tap
// products cancel.  Every mbarrier wait is bounded; on a timeout the CTA
// records CWTH_ERR_TIMEOUT in a device status word, drains its own TMA
// copies (bounded), releases tensor memory and returns.
#include <cuda_bf16.h>

#include <stdlib.h>

#include <algorithm>

#include "cwth_internal.h"
#include "sm100.cuh"

namespace cwth {
namespace {

using namespace sm100;

constexpr int kBM = 128;             // frames per tile
constexpr int kBK = 64;              // taps per stage (128 bytes of bf16)
constexpr int kDirThreads = 320;
constexpr int kEpiWarps = 8;         // two per tensor-memory lane quarter
constexpr int kAPieceRows = 32;      // frame-map box height (rows per TMA copy)
constexpr int kMaxGroupScales = 128; // scales per GEMM group (256 columns)
constexpr int kMaxPhases = 4;        // frame windows per tile (hops up to 256)
constexpr long long kWaitBudget = 4000000000LL;  // ~2 s of SM clock

// Square root by the hardware approximation (relative error about 2^-22),
// well inside every accuracy class of the direct path.
__device__ __forceinline__ float sqrt_approx(float v) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// ------------------------------------------------------------ staging
// x_pad[b][j] = x[b][j - h_front] for j - h_front in [0, len_b), else 0;
// part 0 = bf16(x), part 1 = bf16(x - part 0), part 2 = bf16(x - part 0 -
// part 1) (the differences are exact in float32).  Row b = batch is the
// zero tail after the last clip.  Each thread writes 8 consecutive bf16
// (one 16-byte store per buffer); rows and the tail are multiples of 8
// elements long.  Null part buffers are not written.  vec: x, ld_x and
// h_front keep every 8-element source run of a row 16-byte aligned, so runs
// wholly inside the clip are read as two float4 loads.
__global__ void stage_bf16_kernel(const float* __restrict__ x, int64_t ld_x,
                                  const int64_t* __restrict__ lengths, int64_t max_len, int batch,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                  __nv_bfloat16* __restrict__ lo2, int64_t lpad, int64_t h_front,
                                  int64_t total, bool vec) {
    // The tensor-core kernel that follows may start its prologue now; it
    // waits for this grid's completion before reading the staged signal.
    asm volatile("griddepcontrol.launch_dependents;");
    const int b = blockIdx.y;
    const int64_t row_len = b < batch ? lpad : total - (int64_t)batch * lpad;
    int64_t len = 0;
    if (b < batch) {
        len = lengths ? lengths[b] : max_len;
        len = len < 0 ? 0 : (len > max_len ? max_len : len);
    }
    const float* xr = x + (int64_t)(b < batch ? b : 0) * ld_x;
    const int64_t base = (int64_t)b * lpad;
    for (int64_t j0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8; j0 < row_len;
         j0 += (int64_t)gridDim.x * blockDim.x * 8) {
        uint32_t wh[4], wl[4], w2[4];
        float xv[8];
        const int64_t n0 = j0 - h_front;
        if (vec && n0 >= 0 && n0 + 8 <= len) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(xr + n0));
            const float4 c = __ldg(reinterpret_cast<const float4*>(xr + n0 + 4));
            xv[0] = a.x, xv[1] = a.y, xv[2] = a.z, xv[3] = a.w;
            xv[4] = c.x, xv[5] = c.y, xv[6] = c.z, xv[7] = c.w;
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int64_t n = n0 + e;
                xv[e] = (n >= 0 && n < len) ? __ldg(xr + n) : 0.f;
            }
        }
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            const float v[2] = {xv[e], xv[e + 1]};
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[0], v[1]);
            const float2 hf = __bfloat1622float2(h2);
            const float r0 = v[0] - hf.x, r1 = v[1] - hf.y;
            const __nv_bfloat162 l2 = __floats2bfloat162_rn(r0, r1);
            const float2 lf = __bfloat1622float2(l2);
            const __nv_bfloat162 m2 = __floats2bfloat162_rn(r0 - lf.x, r1 - lf.y);
            wh[e >> 1] = *reinterpret_cast<const uint32_t*>(&h2);
            wl[e >> 1] = *reinterpret_cast<const uint32_t*>(&l2);
            w2[e >> 1] = *reinterpret_cast<const uint32_t*>(&m2);
        }
        *reinterpret_cast<uint4*>(hi + base + j0) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
        if (lo) *reinterpret_cast<uint4*>(lo + base + j0) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
        if (lo2) *reinterpret_cast<uint4*>(lo2 + base + j0) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
    }
}

// ------------------------------------------------------------ tap bank (float64)
// bank[n][tau] for column n of a group (parts as the staged signal's: hi,
// lo = bf16 of the remainder, lo2 = bf16 of what is left; lo2 may be
// null): scale j = n / 2 (real part for even n,
// imaginary for odd n), tap t = tau - h_group, value a^{-1/2} conj(psi(t/a))
// for |t| <= h_j, else 0.  Columns past 2 * n_scales are zero.
__global__ void bank_kernel(const double* __restrict__ scales, const int32_t* __restrict__ h_of,
                            int n_scales, int ncols, int k_pad, int h_group, double B, double C,
                            __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                            __nv_bfloat16* __restrict__ lo2, float2* __restrict__ f32bank) {
    const int64_t total = (int64_t)ncols * k_pad;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(i / k_pad);
        const int tau = (int)(i - (int64_t)n * k_pad);
        const int j = n >> 1;
        double v = 0.0;
        if (j < n_scales) {
            const int t = tau - h_group;
            if (t >= -h_of[j] && t <= h_of[j]) {
                const double a = scales[j];
                const double u = (double)t / a;
                const double env = exp(-(u * u) / B) / sqrt(a * M_PI * B);
                double s, c;
                sincospi(2.0 * C * u, &s, &c);
                v = (n & 1) ? -env * s : env * c;
            }
        }
        const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
        hi[i] = h;
        const double r = v - (double)__bfloat162float(h);
        const __nv_bfloat16 l = __float2bfloat16_rn((float)r);
        lo[i] = l;
        if (lo2) lo2[i] = __float2bfloat16_rn((float)(r - (double)__bfloat162float(l)));
        if (f32bank && j < n_scales) {
            // float32 copy for the SIMT kernel: [scale][tau] as (re, im)
            float* f = reinterpret_cast<float*>(f32bank + (int64_t)j * k_pad + tau);
            f[n & 1] = (float)v;
        }
    }
}

// ------------------------------------------------------------ tcgen05 GEMM
// Persistent kernel: one CTA per SM walks units of p.unit (1 or 2) 128-frame
// tiles, unit u covering tiles u * unit .. u * unit + unit - 1, units
// blockIdx.x, blockIdx.x + gridDim.x, ...  Every bank tile a stage brings in
// feeds the MMAs of all tiles of the unit, so the bank is read once per unit
// rather than once per tile.  TMA stages stream without a break between
// units; frame windows come in p.win_sets sets and tensor-memory
// accumulators in p.acc_sets sets (two sets: the next unit's loads / MMAs
// overlap this unit's MMAs / epilogue).
//
// Shared-memory layout (1024-byte aligned pieces):
//   windows: [set][tile][part][phase]   only when p.a_shift > 0 (see below)
//   stage s: [A tile 0 part 0][A tile 0 part 1]..[A tile 1 part 0].. [B]
//            (A parts only without a window; NP parts per tile)
// Schedule step j: up to four tap blocks, block b in bits 8b..8b+7 of
// sched[j].x; sched[j].y = columns used (low 16 bits, a multiple of 16) |
// bank part (bit 16: 0 = hi, 1 = lo; bits 19-20: part 2) | blocks - 1
// (bits 17-18).  A step of
// several blocks carries all their tiles in one stage, each block as [A
// tiles (without a window)][bank tile] at the same column count, so the
// narrow outer blocks of the pyramid share stage turns (4 MMAs per block).
// The split variants visit every step once per bank part (NP times); the
// plain variant uses the hi part only.  Bank part j meets the A parts
// 0 .. NP - 1 (two parts: all four products) or, with three parts, 0 ..
// 2 - j (the six products x_i g_j with i + j <= 2).
// When 64 is a multiple of the hop, the frame tile of tap block kb is the
// tile of block 0 moved down by kb * 64 / H rows of the frame view, so one
// window of 128 + (blocks - 1) * 64/H rows per tile, loaded once, serves
// every K step through descriptors that start kb * 64/H rows into it.  When
// the hop is r = H / 64 times 64 (r <= 4), block kb = r j + ph reads taps
// 64 ph .. 64 ph + 63 of frame rows moved down by j: r windows ("phases",
// loaded at tap offset 64 ph) of 128 + ceil(blocks / r) - 1 rows serve all
// blocks the same way.
template <int NP>
__global__ void __launch_bounds__(kDirThreads, 1)
    direct_mma_kernel(const __grid_constant__ CUtensorMap mA_hi,
                      const __grid_constant__ CUtensorMap mA_lo,
                      const __grid_constant__ CUtensorMap mA_lo2,
                      const __grid_constant__ CUtensorMap mB_hi,
                      const __grid_constant__ CUtensorMap mB_lo,
                      const __grid_constant__ CUtensorMap mB_lo2, const DirLaunch p) {
    extern __shared__ uint8_t dsmem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kMaxDirStages];
    __shared__ __align__(8) uint64_t empty_bar[kMaxDirStages];
    __shared__ __align__(8) uint64_t win_full[2], win_empty[2];
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    __shared__ int32_t rowoff_sh[kMaxGroupScales];
    __shared__ int2 sched_sh[kMaxDirSteps];

    uint8_t* smem = (uint8_t*)(((uintptr_t)dsmem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int kParts = NP;
    const int N = p.ncols;
    const int T = p.unit;
    const int stages = p.stages;
    const int shift = p.a_shift;       // window rows per block (per r blocks with phases)
    const int phases = p.a_phases, lgph = __ffs(phases) - 1;
    const int wsets = p.win_sets, asets = p.acc_sets;
    constexpr uint32_t kPiece = kAPieceRows * kBK * 2;  // one frame-map box
    const uint32_t win_bytes = (uint32_t)p.win_rows * kBK * 2;
    const uint32_t win_span = (win_bytes + 1023) & ~1023u;
    const uint32_t win_region = shift ? win_span * kParts * T * wsets * phases : 0u;
    const uint32_t a_tile = kBM * kBK * 2;
    const uint32_t a_step = shift ? 0u : a_tile * kParts * T;
    const uint32_t b_bytes = (uint32_t)((N + 63) / 64 * 64) * kBK * 2;
    const uint32_t stage_bytes = a_step + b_bytes;
    uint8_t* stage0 = smem + win_region;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nsteps = p.nsteps;
    const int ntiles = (int)((p.total_rows + kBM - 1) / kBM);
    // A spectral part of the same plan, launched next as a programmatic
    // dependent, takes each SM this persistent grid's CTAs leave.
    asm volatile("griddepcontrol.launch_dependents;");
    const int nunits = (ntiles + T - 1) / T;
    const uint32_t acc_cols = p.tmem_cols / (uint32_t)(asets * T);  // columns per tile accumulator

    // Per-scale output offsets (elements from the clip's first row) and the
    // schedule, both read at every step or store, live in shared memory.
    for (int i = threadIdx.x; i < p.n_scales; i += blockDim.x)
        rowoff_sh[i] = (int32_t)(__ldg(p.rows + i) * p.frames_max);
    for (int i = threadIdx.x; i < nsteps; i += blockDim.x) sched_sh[i] = __ldg(p.sched + i);
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&win_full[b], 1);
            mbar_init(&win_empty[b], 1);
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kEpiWarps);  // one arrival per epilogue warp
        }
        // A CTA of a launch that already timed out, or handed a schedule
        // longer than its table, does no work.
        abort_sh = (*(volatile int*)p.status != 0 || nsteps > kMaxDirSteps) ? 1 : 0;
        fence_mbar_init();
        prefetch_tensormap(&mA_hi);
        prefetch_tensormap(&mB_hi);
        if (NP > 1) {
            prefetch_tensormap(&mA_lo);
            prefetch_tensormap(&mB_lo);
        }
        if (NP > 2) {
            prefetch_tensormap(&mA_lo2);
            prefetch_tensormap(&mB_lo2);
        }
    }
    if (warp == 1) {
        tmem_alloc(&tmem_base_sh, p.tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    auto win_ptr = [&](int set, int tile, int part, int ph) {
        return smem + (((size_t)(set * T + tile) * kParts + part) * phases + ph) * win_span;
    };
    auto amap = [&](int part) { return part == 0 ? &mA_hi : (part == 1 ? &mA_lo : &mA_lo2); };
    auto aborted = [&]() { return *(volatile int*)&abort_sh != 0; };
    auto fail = [&]() { atomicExch(&abort_sh, 1); };

    // The producer and the MMA issuer run as whole warps (control flow stays
    // warp-uniform) and one elected lane issues the copies, MMAs and commits.
    // Ring positions advance by counters, never by division: MMA issue is
    // serial (each tcgen05.mma waits for the one before it to be accepted),
    // so any latency between two issues adds to the tensor-core time.
    if (warp == 0) {
        // Producer.  The kernel is launched as a programmatic dependent of
        // the staging kernel (its prologue above overlaps that kernel's
        // tail); the staged signal is read only after the preceding grid
        // has completed and its writes are visible.  Nothing else in the
        // kernel reads memory the preceding grid writes, and the epilogue's
        // stores follow the producer's copies.
        asm volatile("griddepcontrol.wait;" ::: "memory");
        uint32_t g = 0;            // steps issued over all units
        int s = 0;                 // stage of step g
        uint32_t sph = 0;          // parity of stage s's current fill
        int ws = 0, wins = 0;      // window set of the next unit, window sets issued
        uint32_t wph = 0;
        for (int u = blockIdx.x; u < nunits && !aborted(); u += gridDim.x) {
            if (shift) {
                if (wins >= wsets && !mbar_wait_warp(&win_empty[ws], wph ^ 1, kWaitBudget)) {
                    if (lane == 0) fail();
                    break;
                }
                if (elect_one()) {
                    mbar_arrive_expect_tx(&win_full[ws], win_bytes * kParts * T * phases);
                    for (int tt = 0; tt < T; ++tt) {
                        const int m0 = (u * T + tt) * kBM;
                        for (int ph = 0; ph < phases; ++ph)
                            for (int j = 0; j < p.win_rows / kAPieceRows; ++j)
                                for (int part = 0; part < kParts; ++part)
                                    tma_load_2d(win_ptr(ws, tt, part, ph) + j * kPiece, amap(part),
                                                &win_full[ws], ph * kBK, m0 + j * kAPieceRows);
                    }
                }
                __syncwarp();
                ++wins;
                if (++ws == wsets) {
                    ws = 0;
                    wph ^= 1;
                }
            }
            bool ok = true;
            for (int j = 0; j < nsteps; ++j) {
                if (aborted()) {
                    ok = false;
                    break;
                }
                if (g >= (uint32_t)stages && !mbar_wait_warp(&empty_bar[s], sph ^ 1, kWaitBudget)) {
                    if (lane == 0) fail();
                    ok = false;
                    break;
                }
                const int2 step = sched_sh[j];
                if (elect_one()) {
                    const int pieces = ((step.y & 0xFFFF) + 63) >> 6;
                    const int nblk = 1 + ((step.y >> 17) & 3);
                    const int bpart = ((step.y >> 16) & 1) | (((step.y >> 19) & 3) << 1);
                    const CUtensorMap* mb =
                        (NP > 1 && bpart == 1) ? &mB_lo : ((NP > 2 && bpart == 2) ? &mB_lo2 : &mB_hi);
                    uint8_t* st = stage0 + (size_t)s * stage_bytes;
                    mbar_arrive_expect_tx(&full_bar[s],
                                          (uint32_t)nblk * (a_step + (uint32_t)pieces * 64 * kBK * 2));
                    // block b of the stage: [A tiles (without a window)][bank tile]
                    const uint32_t blk = a_step + (uint32_t)pieces * 64 * kBK * 2;
                    for (int b = 0; b < nblk; ++b) {
                        const int kxb = ((step.x >> (8 * b)) & 0xFF) * kBK;
                        uint8_t* sb = st + b * blk;
                        if (!shift) {
                            for (int tt = 0; tt < T; ++tt) {
                                const int m0 = (u * T + tt) * kBM;
                                for (int q = 0; q < kBM / kAPieceRows; ++q)
                                    for (int part = 0; part < kParts; ++part)
                                        tma_load_2d(sb + (tt * kParts + part) * a_tile + q * kPiece,
                                                    amap(part), &full_bar[s], kxb,
                                                    m0 + q * kAPieceRows);
                            }
                        }
                        for (int q = 0; q < pieces; ++q)
                            tma_load_2d(sb + a_step + q * 64 * kBK * 2, mb, &full_bar[s], kxb,
                                        q * 64);
                    }
                }
                __syncwarp();
                ++g;
                if (++s == stages) {
                    s = 0;
                    sph ^= 1;
                }
            }
            if (!ok) break;
        }
        // Drain: every copy issued must have landed before the CTA exits.
        if (lane == 0) {
            for (uint32_t gg = g > (uint32_t)stages ? g - stages : 0; gg < g; ++gg)
                if (!mbar_wait(&full_bar[gg % stages], (gg / stages) & 1, kWaitBudget)) {
                    fail();
                    break;
                }
            for (int w = wins > wsets ? wins - wsets : 0; w < wins; ++w)
                if (!mbar_wait(&win_full[w % wsets], (w / wsets) & 1, kWaitBudget)) {
                    fail();
                    break;
                }
        }
    } else if (warp == 1) {
        // MMA issuer: one elected lane runs the loop.  Each unit's first step
        // is the centre tap block (hi part), which every scale reaches: its N
        // covers all columns and its first MMA per tile initialises that
        // tile's accumulator.  Descriptors are built from 32-bit low words
        // (start address >> 4) that advance by additions.
        if (elect_one()) {
            int s = 0;
            uint32_t sph = 0;
            int as = 0, ws = 0, i = 0;
            uint32_t aph = 0, wph = 0;
            const uint32_t stage_base = smem_u32(stage0);
            const uint32_t b_lo0 = desc_sw128_lo(stage_base + a_step);
            const uint32_t stage16 = stage_bytes >> 4;
            const uint32_t a_step16 = a_step >> 4;
            // distance between the A operands of consecutive (tile, part) pairs
            const uint32_t pitch16 = (shift ? win_span * phases : a_tile) >> 4;
            const uint32_t span16 = win_span >> 4;
            const uint32_t idesc0 = idesc_bf16_f32(kBM, 0);
            uint32_t b_lo = b_lo0;
            for (int u = blockIdx.x; u < nunits && !aborted(); u += gridDim.x, ++i) {
                if (i >= asets && !mbar_wait(&acc_empty[as], aph ^ 1, kWaitBudget)) {
                    fail();
                    break;
                }
                if (shift && !mbar_wait(&win_full[ws], wph, kWaitBudget)) {
                    fail();
                    break;
                }
                tc_fence_after();
                const uint32_t dacc0 = tmem + (uint32_t)(as * T) * acc_cols;
                const uint32_t win_lo = desc_sw128_lo(smem_u32(win_ptr(ws, 0, 0, 0)));
                bool ok = true;
                int2 step = sched_sh[0];
                for (int j = 0; j < nsteps; ++j) {
                    // Everything but the MMAs is computed before the wait.
                    const int2 next = sched_sh[j + 1 < nsteps ? j + 1 : j];
                    const uint32_t idesc = idesc0 | ((uint32_t)(step.y & 0xFFFF) >> 3 << 17);
                    const int nblk = 1 + ((step.y >> 17) & 3);
                    // block b's A tiles (without a window) and bank tile follow block
                    // b-1's, a_step + pieces x 8 KB further
                    const uint32_t b_next16 =
                        a_step16 + (uint32_t)(((step.y & 0xFFFF) + 63) >> 6) * 512u;
                    const uint32_t kb_all = (uint32_t)step.x;
                    const uint32_t acc0 = j > 0 ? 1u : 0u;
                    // A parts this bank part meets (see the kernel comment)
                    const int bpart = ((step.y >> 16) & 1) | (((step.y >> 19) & 3) << 1);
                    const int na = NP == 3 ? 3 - bpart : NP;
                    if (!mbar_wait(&full_bar[s], sph, kWaitBudget)) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // unrolled: constant shifts, no loop bookkeeping between MMAs
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        if (b >= nblk) break;
                        const uint32_t kb = (kb_all >> (8 * b)) & 0xFFu;
                        const uint32_t a_lo = shift ? win_lo + (kb & (uint32_t)(phases - 1)) * span16 +
                                                          (kb >> lgph) * (uint32_t)shift * 8u
                                                    : b_lo - a_step16 + (uint32_t)b * b_next16;
                        const uint32_t bb = b_lo + (uint32_t)b * b_next16;
                        for (int tt = 0; tt < T; ++tt) {
                            const uint32_t dacc = dacc0 + (uint32_t)tt * acc_cols;
                            const uint32_t ah = a_lo + (uint32_t)(tt * kParts) * pitch16;
#pragma unroll
                            for (int k = 0; k < kBK / 16; ++k) {
                                // 16 bf16 = 32 bytes along K -> +2 in the address field
                                const uint64_t bd = desc_words(bb + 2 * k, kDescSw128Hi);
                                mma_f16(dacc, desc_words(ah + 2 * k, kDescSw128Hi), bd, idesc,
                                        (acc0 | (uint32_t)b | (uint32_t)k) ? 1u : 0u);
#pragma unroll
                                for (int ap = 1; ap < NP; ++ap)
                                    if (ap < na)
                                        mma_f16(dacc,
                                                desc_words(ah + (uint32_t)ap * pitch16 + 2 * k,
                                                           kDescSw128Hi),
                                                bd, idesc, 1u);
                            }
                        }
                    }
                    mma_commit(&empty_bar[s]);
                    step = next;
                    if (++s == stages) {
                        s = 0;
                        sph ^= 1;
                        b_lo = b_lo0;
                    } else {
                        b_lo += stage16;
                    }
                }
                if (!ok) break;
                mma_commit(&acc_full[as]);
                if (shift) mma_commit(&win_empty[ws]);
                if (++as == asets) {
                    as = 0;
                    aph ^= 1;
                }
                if (++ws == wsets) {
                    ws = 0;
                    wph ^= 1;
                }
            }
        }
        __syncwarp();
    } else {
        // Epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (one frame each);
        // the two warps of a lane quarter take alternate 64-column chunks.
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        int as = 0;
        uint32_t aph = 0;
        for (int u = blockIdx.x; u < nunits && !aborted(); u += gridDim.x) {
            if (!mbar_wait(&acc_full[as], aph, kWaitBudget)) {
                fail();
                break;
            }
            tc_fence_after();
            for (int tt = 0; tt < T; ++tt) {
                const int64_t row = (int64_t)(u * T + tt) * kBM + quarter * 32 + lane;
                const int64_t b = row / p.rows_per_clip;
                const int64_t k = row - b * p.rows_per_clip;
                bool valid = b < p.batch;
                if (valid) {
                    int64_t len = p.lengths ? p.lengths[b] : p.max_len;
                    len = len < 0 ? 0 : (len > p.max_len ? p.max_len : len);
                    valid = k < (len + p.hop - 1) / p.hop;
                }
                const uint32_t tlane = tmem + (uint32_t)(as * T + tt) * acc_cols +
                                       ((uint32_t)(quarter * 32) << 16);
                float* obase = p.out + (valid ? (b * p.S_total) * p.frames_max + k : 0);
                // 64 columns (32 scales) per wait: four loads in flight at a time.
                for (int c0 = half * 64; c0 < N; c0 += 128) {
                    uint32_t r[64];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (c0 + 16 * q < N) tmem_ld16_nowait(tlane + (uint32_t)(c0 + 16 * q), r + 16 * q);
                    tmem_ld_wait();
                    if (valid) {
                        const int nsc = min(32, p.n_scales - (c0 >> 1));
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) {
                            if (jj < nsc) {
                                const float re = __uint_as_float(r[2 * jj]);
                                const float im = __uint_as_float(r[2 * jj + 1]);
                                __stcs(obase + rowoff_sh[(c0 >> 1) + jj],
                                       sqrt_approx(fmaf(re, re, im * im)));
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[as]);
            if (++as == asets) {
                as = 0;
                aph ^= 1;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, p.tmem_cols);
    }
    if (threadIdx.x == 0 && abort_sh) atomicExch(p.status, (int)CWTH_ERR_TIMEOUT);
    // Every CTA, also one that gave up before its producer waited, ends
    // after the grid it depends on, so work after this kernel on the
    // stream also follows that grid.
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ------------------------------------------------------------ float32 SIMT
// One CTA per (128-frame tile, clip, scale); taps of the scale staged in
// shared memory; each thread sums one frame in float32.
__global__ void __launch_bounds__(128) direct_f32_kernel(const float* __restrict__ x, int64_t ld_x,
                                                         const float2* __restrict__ bank,
                                                         const DirLaunch p,
                                                         const int32_t* __restrict__ h_of) {
    extern __shared__ float2 taps[];
    const int sl = blockIdx.z;
    const int64_t b = blockIdx.y;
    const int h = h_of[sl];
    const int hg = p.h_group;
    for (int t = threadIdx.x; t <= 2 * h; t += blockDim.x)
        taps[t] = bank[(int64_t)sl * p.k_pad + (hg - h) + t];
    __syncthreads();
    int64_t len = p.lengths ? p.lengths[b] : p.max_len;
    len = len < 0 ? 0 : (len > p.max_len ? p.max_len : len);
    const int64_t F = (len + p.hop - 1) / p.hop;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= F) return;
    const float* xr = x + b * ld_x;
    const int64_t c = k * p.hop;
    const int64_t t0 = c - h < 0 ? -c : -h;
    const int64_t t1 = c + h > len - 1 ? len - 1 - c : h;
    float re = 0.f, im = 0.f;
    for (int64_t t = t0; t <= t1; ++t) {
        const float xv = __ldg(xr + c + t);
        const float2 g = taps[t + h];
        re = fmaf(xv, g.x, re);
        im = fmaf(xv, g.y, im);
    }
    const int orow = p.rows[sl];
    p.out[(b * p.S_total + orow) * p.frames_max + k] = sqrtf(fmaf(re, re, im * im));
}

}  // namespace

// Dynamic shared memory of a launch: two frame windows, the stages, 1 KB of
// alignment slack, and at least kDirSmemMin so that one CTA holds an SM (the
// CTA allocates both tensor-memory accumulators).
constexpr size_t kDirSmemMin = 120 * 1024;

size_t direct_smem_bytes(int ncols, int stages, int nparts, int win_rows, int unit,
                         int win_sets, int phases) {
    const size_t parts = (size_t)nparts;
    const size_t brows = (size_t)(ncols + 63) / 64 * 64;
    const size_t a = win_rows > 0 ? 0 : (size_t)kBM * kBK * 2 * parts * unit;
    const size_t stage = a + brows * kBK * 2;
    const size_t win_span = ((size_t)win_rows * kBK * 2 + 1023) / 1024 * 1024;
    const size_t bytes = (win_rows > 0 ? win_span * parts * unit * win_sets * phases : 0) +
                         stage * stages + 1024;
    return bytes < kDirSmemMin ? kDirSmemMin : bytes;
}

// Frame windows (see direct_mma_kernel): hops dividing 64 use one window
// moved 64/H rows per tap block; hops of r * 64 (r <= kMaxPhases) use r
// phase windows moved one row per r blocks; other hops load A per stage.
int direct_window_phases(int hop) {
    return (hop > kBK && hop % kBK == 0 && hop / kBK <= kMaxPhases) ? hop / kBK : 1;
}

int direct_window_shift(int hop) { return hop > 0 && kBK % hop == 0 ? kBK / hop : 1; }

int direct_window_rows(int hop, int k_pad) {
    if (hop <= 0) return 0;
    const int nkb = k_pad / kBK;
    int rows;
    if (kBK % hop == 0) {
        rows = kBM + (nkb - 1) * (kBK / hop);
    } else if (direct_window_phases(hop) > 1) {
        const int r = direct_window_phases(hop);
        rows = kBM + (nkb + r - 1) / r - 1;
    } else {
        return 0;
    }
    return (rows + kAPieceRows - 1) / kAPieceRows * kAPieceRows;
}

int direct_split_schedule(const int2* in, int n, int nparts, int2* out) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < nparts; ++j)
            out[nparts * i + j] = make_int2(in[i].x, in[i].y | ((j & 1) << 16) | ((j >> 1) << 19));
    return nparts * n;
}

// Dynamic shared memory a direct CTA may request: the 227 KB opt-in limit
// less room for the kernel's static shared memory (barriers, the per-scale
// output offsets and the schedule: under 3 KB).
constexpr size_t kDirSmemLimit = 227 * 1024 - 3072;

// A stage's A tiles (frames; none with a frame window) in 8 KB pieces.
int direct_a_pieces(int nparts, int unit, bool windowed) {
    return windowed ? 0 : kBM * nparts * unit / 64;
}

int direct_max_stages(int ncols, int nparts, int win_rows, int unit, int win_sets, int phases) {
    int s = kMaxDirStages;
    while (s > 2 &&
           direct_smem_bytes(ncols, s, nparts, win_rows, unit, win_sets, phases) > kDirSmemLimit)
        --s;
    return direct_smem_bytes(ncols, s, nparts, win_rows, unit, win_sets, phases) <= kDirSmemLimit
               ? s
               : 0;
}

// Launch shape of a group: frame tiles per unit, window and accumulator
// sets, stages.  Two tiles share each bank tile only while two accumulator
// sets still fit in tensor memory (N <= 128): measured on GB300, exposing
// the epilogue (two 256-column tiles filling all 512 columns) costs more
// than the halved bank traffic saves.
DirShape direct_shape(int ncols, int nparts, int hop, int k_pad) {
    DirShape best{};
    int cpow = 32;
    while (cpow < ncols) cpow <<= 1;
    const int win = direct_window_rows(hop, k_pad);
    for (int unit = 2; unit >= 1; --unit) {
        const int asets = std::min(2, 512 / (unit * cpow));
        if (asets < 1 || (unit == 2 && asets < 2)) continue;
        for (int wrows : {win, 0}) {
            if (wrows == 0 && win > 0 && best.stages > 0) continue;
            const int ph = wrows ? direct_window_phases(hop) : 1;
            for (int wsets = (wrows ? 2 : 1); wsets >= 1; --wsets) {
                const int st = direct_max_stages(ncols, nparts, wrows, unit, wsets, ph);
                if (st >= (wsets == 2 ? 3 : 2)) {
                    best.unit = unit;
                    best.acc_sets = asets;
                    best.win_sets = wsets;
                    best.win_rows = wrows;
                    best.phases = ph;
                    best.stages = st;
                    best.tmem_cols = asets * unit * cpow;
                    return best;
                }
            }
        }
    }
    return best;
}

cudaError_t direct_prepare_device() {
    cudaError_t e = cudaSuccess;
    for (const void* f : {(const void*)direct_mma_kernel<1>, (const void*)direct_mma_kernel<2>,
                          (const void*)direct_mma_kernel<3>})
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kDirSmemLimit);
    return e;
}

cudaError_t direct_make_bank(const double* d_scales, const int32_t* d_h, int n_scales, int ncols,
                             int k_pad, int h_group, double B, double C, __nv_bfloat16* hi,
                             __nv_bfloat16* lo, __nv_bfloat16* lo2, float2* f32bank,
                             cudaStream_t st) {
    const int64_t total = (int64_t)ncols * k_pad;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
    bank_kernel<<<blocks, 256, 0, st>>>(d_scales, d_h, n_scales, ncols, k_pad, h_group, B, C, hi,
                                        lo, lo2, f32bank);
    return cudaGetLastError();
}

cudaError_t direct_stage(const float* x, int64_t ld_x, const int64_t* lengths, int64_t max_len,
                         int batch, __nv_bfloat16* hi, __nv_bfloat16* lo, __nv_bfloat16* lo2,
                         int64_t lpad, int64_t h_front, int64_t total, cudaStream_t st) {
    // lpad and the tail are multiples of 8 elements (hop % 8 == 0, supports
    // and tap counts multiples of 8), so every 16-byte store is aligned.
    const int64_t longest = std::max<int64_t>(lpad, total - (int64_t)batch * lpad);
    const unsigned bx = (unsigned)std::min<int64_t>((longest / 8 + 255) / 256, 1024);
    dim3 grid(bx > 0 ? bx : 1, (unsigned)batch + 1);
    const bool vec = ((uintptr_t)x & 15) == 0 && (ld_x & 3) == 0 && (h_front & 3) == 0;
    stage_bf16_kernel<<<grid, 256, 0, st>>>(x, ld_x, lengths, max_len, batch, hi, lo, lo2, lpad,
                                            h_front, total, vec);
    return cudaGetLastError();
}

// maps: {A part 0, 1, 2, bank part 0, 1, 2}; parts past nparts are unused.
cudaError_t direct_launch_mma(const CUtensorMap* maps, const DirLaunch& L, int nparts,
                              cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t units = ((L.total_rows + kBM - 1) / kBM + L.unit - 1) / L.unit;
    const int64_t tiles = std::min<int64_t>(units, sms);
    const size_t smem = direct_smem_bytes(L.ncols, L.stages, nparts, L.a_shift ? L.win_rows : 0,
                                          L.unit, L.win_sets, L.a_phases);
    // Programmatic stream serialisation: the kernel may begin while the
    // preceding kernel (the bf16 staging) finishes; its producer waits for
    // that grid (griddepcontrol.wait) before the first copy of the signal.
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)tiles);
    cfg.blockDim = dim3(kDirThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (nparts == 3)
        return cudaLaunchKernelEx(&cfg, direct_mma_kernel<3>, maps[0], maps[1], maps[2], maps[3],
                                  maps[4], maps[5], L);
    if (nparts == 2)
        return cudaLaunchKernelEx(&cfg, direct_mma_kernel<2>, maps[0], maps[1], maps[1], maps[3],
                                  maps[4], maps[4], L);
    return cudaLaunchKernelEx(&cfg, direct_mma_kernel<1>, maps[0], maps[0], maps[0], maps[3],
                              maps[3], maps[3], L);
}

cudaError_t direct_launch_f32(const float* x, int64_t ld_x, const float2* bank, const int32_t* d_h,
                              const DirLaunch& L, cudaStream_t st) {
    const int64_t ftiles = (L.frames_max + 127) / 128;
    dim3 grid((unsigned)ftiles, (unsigned)L.batch, (unsigned)L.n_scales);
    const size_t smem = (size_t)(2 * L.h_group + 1) * sizeof(float2);
    direct_f32_kernel<<<grid, 128, smem, st>>>(x, ld_x, bank, L, d_h);
    return cudaGetLastError();
}

int direct_schedule(const int32_t* h_desc, int n, int h_group, int k_pad, int stage_pieces,
                    int a_pieces, int2* out) {
    const int nkb = k_pad / kBK;
    const int center = h_group / kBK;
    int blocks = 0;
    int kbs[kMaxDirSteps], cols[kMaxDirSteps];
    for (int r = 0; r < 2 * nkb; ++r) {
        // centre, centre-1, centre+1, centre-2, centre+2, ...
        const int kb = center + ((r & 1) ? -((r + 1) >> 1) : (r >> 1));
        if (kb < 0 || kb >= nkb) continue;
        const int t0 = kb * kBK - h_group, t1 = t0 + kBK - 1;
        const int d = (t0 <= 0 && t1 >= 0) ? 0 : std::min(std::abs(t0), std::abs(t1));
        int cnt = 0;
        while (cnt < n && h_desc[cnt] >= d) ++cnt;  // supports are in descending order
        if (cnt == 0) continue;
        kbs[blocks] = kb;
        cols[blocks++] = (2 * cnt + 15) / 16 * 16;
    }
    // Consecutive blocks (after the centre block, which initialises the
    // accumulators alone) share a stage while their tiles fit: g blocks of
    // nc columns need g (a_pieces + ceil(nc / 64)) of the stage's
    // a_pieces + stage_pieces 8 KB pieces.
    int steps = 0;
    for (int i = 0; i < blocks;) {
        int g = 1, nc = cols[i];
        while (i > 0 && g < 4 && i + g < blocks) {
            const int nc2 = std::max(nc, cols[i + g]);
            if ((g + 1) * (a_pieces + (nc2 + 63) / 64) > a_pieces + stage_pieces) break;
            nc = nc2;
            ++g;
        }
        int x = 0;
        for (int b = 0; b < g; ++b) x |= kbs[i + b] << (8 * b);
        out[steps++] = make_int2(x, nc | ((g - 1) << 17));
        i += g;
    }
    return steps;
}

cudaError_t direct_prepare_f32(size_t smem) {
    return cudaFuncSetAttribute(direct_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)std::max<size_t>(smem, 48 * 1024));
}

}  // namespace cwth
