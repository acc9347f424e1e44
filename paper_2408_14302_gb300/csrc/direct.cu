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
// tcgen05 kernel (bf16 operands, f32 accumulation in tensor memory), one CTA
// per 128-frame tile of one group, 6 warps:
//   warp 0      TMA producer (A and B tiles, 64 taps per stage, 128B swizzle)
//   warp 1      TMEM allocation + single-thread MMA issue (M=128, N<=256, K=16)
//   warps 2..5  epilogue: tcgen05.ld, |re + i im|, coalesced stores along k
// The split variant ("bf16x2") represents x = x_hi + x_lo and g = g_hi + g_lo
// (each pair within 2^-18 of its value) and accumulates all four products
// into the same tensor-memory accumulator, so every tap product is within
// about 2^-17 relative of x * g even when a frame has a single tap.  Every mbarrier wait is bounded; on a timeout the CTA
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
constexpr int kDirThreads = 192;
constexpr int kAPieceRows = 32;      // frame-map box height (rows per TMA copy)
constexpr int kMaxGroupScales = 128; // scales per GEMM group (256 columns)
constexpr long long kWaitBudget = 4000000000LL;  // ~2 s of SM clock

// ------------------------------------------------------------ staging
// x_pad[b][j] = x[b][j - h_front] for j - h_front in [0, len_b), else 0;
// hi = bf16(x), lo = bf16(x - hi).  Row b = batch is the zero tail after the
// last clip.  Each thread writes 8 consecutive bf16 (one 16-byte store per
// buffer); rows and the tail are multiples of 8 elements long.
__global__ void stage_bf16_kernel(const float* __restrict__ x, int64_t ld_x,
                                  const int64_t* __restrict__ lengths, int64_t max_len, int batch,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                  int64_t lpad, int64_t h_front, int64_t total) {
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
        uint32_t wh[4], wl[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            float v[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int64_t n = j0 + e + q - h_front;
                v[q] = (n >= 0 && n < len) ? __ldg(xr + n) : 0.f;
            }
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[0], v[1]);
            const float2 hf = __bfloat1622float2(h2);
            const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[0] - hf.x, v[1] - hf.y);
            wh[e >> 1] = *reinterpret_cast<const uint32_t*>(&h2);
            wl[e >> 1] = *reinterpret_cast<const uint32_t*>(&l2);
        }
        *reinterpret_cast<uint4*>(hi + base + j0) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
        if (lo) *reinterpret_cast<uint4*>(lo + base + j0) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
    }
}

// ------------------------------------------------------------ tap bank (float64)
// bank[n][tau] for column n of a group: scale j = n / 2 (real part for even n,
// imaginary for odd n), tap t = tau - h_group, value a^{-1/2} conj(psi(t/a))
// for |t| <= h_j, else 0.  Columns past 2 * n_scales are zero.
__global__ void bank_kernel(const double* __restrict__ scales, const int32_t* __restrict__ h_of,
                            int n_scales, int ncols, int k_pad, int h_group, double B, double C,
                            __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                            float2* __restrict__ f32bank) {
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
        lo[i] = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
        if (f32bank && j < n_scales) {
            // float32 copy for the SIMT kernel: [scale][tau] as (re, im)
            float* f = reinterpret_cast<float*>(f32bank + (int64_t)j * k_pad + tau);
            f[n & 1] = (float)v;
        }
    }
}

// ------------------------------------------------------------ tcgen05 GEMM
// Shared-memory layout (1024-byte aligned pieces):
//   [window hi][window lo]          only when p.a_shift > 0 (see below)
//   stage s: [A hi][A lo][B]        A parts only without a window; A lo only
//                                   for the split variant
// Schedule step i: tap block sched[i].x; sched[i].y = columns used (low 16
// bits, a multiple of 16) | bank part (bit 16: 0 = hi, 1 = lo).  The split
// variant visits every block twice, once per bank part, so a stage holds one
// bank tile; the plain variant uses the hi part only.
// When 64 is a multiple of the hop, the frame tile of tap block kb is the
// tile of block 0 moved down by kb * 64 / H rows of the frame view, so one
// window of 128 + (blocks - 1) * 64/H rows, loaded once, serves every K step
// through descriptors that start kb * 64/H rows into it.
template <bool SPLIT>
__global__ void __launch_bounds__(kDirThreads, 1)
    direct_mma_kernel(const __grid_constant__ CUtensorMap mA_hi,
                      const __grid_constant__ CUtensorMap mA_lo,
                      const __grid_constant__ CUtensorMap mB_hi,
                      const __grid_constant__ CUtensorMap mB_lo, const DirLaunch p) {
    extern __shared__ uint8_t dsmem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kMaxDirStages];
    __shared__ __align__(8) uint64_t empty_bar[kMaxDirStages];
    __shared__ __align__(8) uint64_t accum_bar;
    __shared__ __align__(8) uint64_t win_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    __shared__ int rows_sh[kMaxGroupScales];

    uint8_t* smem = (uint8_t*)(((uintptr_t)dsmem_raw + 1023) & ~(uintptr_t)1023);
    const int N = p.ncols;
    for (int i = threadIdx.x; i < p.n_scales; i += blockDim.x) rows_sh[i] = __ldg(p.rows + i);
    const int stages = p.stages;
    const int shift = p.a_shift;
    constexpr uint32_t kPiece = kAPieceRows * kBK * 2;  // one frame-map box
    const uint32_t win_bytes = (uint32_t)p.win_rows * kBK * 2;
    const uint32_t win_span = (win_bytes + 1023) & ~1023u;
    const uint32_t a_tile = kBM * kBK * 2;
    const uint32_t a_step = shift ? 0u : a_tile * (SPLIT ? 2 : 1);
    const uint32_t b_bytes = (uint32_t)((N + 63) / 64 * 64) * kBK * 2;
    const uint32_t stage_bytes = a_step + b_bytes;
    uint8_t* win_hi = smem;
    uint8_t* win_lo = smem + win_span;
    uint8_t* stage0 = smem + (shift ? win_span * (SPLIT ? 2 : 1) : 0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM;
    const int nsteps = p.nsteps;
    const uint32_t tcols = p.tmem_cols;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&accum_bar, 1);
        mbar_init(&win_bar, 1);
        // A CTA of a launch that already timed out does no work.
        abort_sh = *(volatile int*)p.status != 0 ? 1 : 0;
        fence_mbar_init();
        prefetch_tensormap(&mA_hi);
        prefetch_tensormap(&mB_hi);
        if (SPLIT) {
            prefetch_tensormap(&mA_lo);
            prefetch_tensormap(&mB_lo);
        }
    }
    if (warp == 1) {
        tmem_alloc(&tmem_base_sh, tcols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    auto stage_ptr = [&](int s) { return stage0 + (size_t)s * stage_bytes; };

    if (warp == 0) {
        if (lane == 0) {
            // Producer.
            bool win_issued = false;
            if (shift && !*(volatile int*)&abort_sh) {
                mbar_arrive_expect_tx(&win_bar, win_bytes * (SPLIT ? 2 : 1));
                for (int j = 0; j < p.win_rows / kAPieceRows; ++j) {
                    tma_load_2d(win_hi + j * kPiece, &mA_hi, &win_bar, 0, m0 + j * kAPieceRows);
                    if (SPLIT)
                        tma_load_2d(win_lo + j * kPiece, &mA_lo, &win_bar, 0, m0 + j * kAPieceRows);
                }
                win_issued = true;
            }
            int issued = 0;
            for (int i = 0; i < nsteps; ++i) {
                const int s = i % stages;
                const uint32_t use = (uint32_t)(i / stages);
                if (*(volatile int*)&abort_sh) break;
                if (i >= stages && !mbar_wait(&empty_bar[s], (use & 1) ^ 1, kWaitBudget)) {
                    atomicExch(&abort_sh, 1);
                    break;
                }
                const int2 step = __ldg(p.sched + i);
                const int kx = step.x * kBK;
                const int pieces = ((step.y & 0xFFFF) + 63) >> 6;
                const CUtensorMap* mb = (SPLIT && (step.y >> 16)) ? &mB_lo : &mB_hi;
                uint8_t* st = stage_ptr(s);
                mbar_arrive_expect_tx(&full_bar[s], a_step + (uint32_t)pieces * 64 * kBK * 2);
                if (!shift) {
                    for (int j = 0; j < kBM / kAPieceRows; ++j) {
                        tma_load_2d(st + j * kPiece, &mA_hi, &full_bar[s], kx, m0 + j * kAPieceRows);
                        if (SPLIT)
                            tma_load_2d(st + a_tile + j * kPiece, &mA_lo, &full_bar[s], kx,
                                        m0 + j * kAPieceRows);
                    }
                }
                for (int j = 0; j < pieces; ++j)
                    tma_load_2d(st + a_step + j * 64 * kBK * 2, mb, &full_bar[s], kx, j * 64);
                ++issued;
            }
            // Drain: every copy issued must have landed before the CTA exits.
            for (int i = (issued > stages ? issued - stages : 0); i < issued; ++i) {
                const int s = i % stages;
                if (!mbar_wait(&full_bar[s], (uint32_t)(i / stages) & 1, kWaitBudget)) {
                    atomicExch(&abort_sh, 1);
                    break;
                }
            }
            if (win_issued && !mbar_wait(&win_bar, 0, kWaitBudget)) atomicExch(&abort_sh, 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer.  The first step is the centre tap block (hi part),
            // which every scale reaches: its N covers all columns and its first
            // MMA initialises them.
            bool ok = true;
            if (shift && !*(volatile int*)&abort_sh && !mbar_wait(&win_bar, 0, kWaitBudget)) {
                atomicExch(&abort_sh, 1);
                ok = false;
            }
            for (int i = 0; i < nsteps && ok; ++i) {
                const int s = i % stages;
                if (*(volatile int*)&abort_sh) break;
                if (!mbar_wait(&full_bar[s], (uint32_t)(i / stages) & 1, kWaitBudget)) {
                    atomicExch(&abort_sh, 1);
                    break;
                }
                tc_fence_after();
                const int2 step = __ldg(p.sched + i);
                const uint32_t idesc = idesc_bf16_f32(kBM, step.y & 0xFFFF);
                const uint32_t st = smem_u32(stage_ptr(s));
                const uint32_t rows = (uint32_t)(step.x * shift) * 128u;
                const uint64_t a_hi = desc_kmajor_sw128(shift ? smem_u32(win_hi) + rows : st);
                const uint64_t a_lo =
                    desc_kmajor_sw128(shift ? smem_u32(win_lo) + rows : st + a_tile);
                const uint64_t bd = desc_kmajor_sw128(st + a_step);
#pragma unroll
                for (int k = 0; k < kBK / 16; ++k) {
                    // 16 bf16 = 32 bytes along K -> +2 in the >>4 address field
                    const uint32_t acc = (i > 0 || k > 0) ? 1u : 0u;
                    mma_f16(tmem, a_hi + 2 * k, bd + 2 * k, idesc, acc);
                    if (SPLIT) mma_f16(tmem, a_lo + 2 * k, bd + 2 * k, idesc, 1u);
                }
                mma_commit(&empty_bar[s]);
            }
            mma_commit(&accum_bar);
        }
    } else {
        // Epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (one frame each).
        const int quarter = warp & 3;
        const bool ready = mbar_wait(&accum_bar, 0, kWaitBudget);
        if (!ready) atomicExch(&abort_sh, 1);
        tc_fence_after();
        const int64_t row = (int64_t)m0 + quarter * 32 + lane;
        const int64_t b = row / p.rows_per_clip;
        const int64_t k = row - b * p.rows_per_clip;
        bool valid = ready && b < p.batch;
        if (valid) {
            int64_t len = p.lengths ? p.lengths[b] : p.max_len;
            len = len < 0 ? 0 : (len > p.max_len ? p.max_len : len);
            valid = k < (len + p.hop - 1) / p.hop;
        }
        if (ready && !*(volatile int*)&abort_sh) {
            const uint32_t tlane = tmem + ((uint32_t)(quarter * 32) << 16);
            for (int c0 = 0; c0 < N; c0 += 16) {
                float v[16];
                tmem_ld16(tlane + (uint32_t)c0, v);
                if (valid) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int sl = (c0 >> 1) + j;
                        if (sl < p.n_scales) {
                            const float re = v[2 * j], im = v[2 * j + 1];
                            const int orow = rows_sh[sl];
                            p.out[(b * p.S_total + orow) * p.frames_max + k] =
                                sqrtf(fmaf(re, re, im * im));
                        }
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, tcols);
    }
    if (threadIdx.x == 0 && abort_sh) atomicExch(p.status, (int)CWTH_ERR_TIMEOUT);
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

size_t direct_smem_bytes(int ncols, int stages, bool split, int win_rows) {
    const size_t brows = (size_t)(ncols + 63) / 64 * 64;
    const size_t a = win_rows > 0 ? 0 : (size_t)kBM * kBK * 2 * (split ? 2 : 1);
    const size_t stage = a + brows * kBK * 2;
    const size_t win_span = ((size_t)win_rows * kBK * 2 + 1023) / 1024 * 1024;
    return win_span * (split ? 2 : 1) + stage * stages + 1024;  // + alignment slack
}

int direct_window_rows(int hop, int k_pad) {
    if (hop <= 0 || kBK % hop != 0) return 0;
    const int rows = kBM + (k_pad / kBK - 1) * (kBK / hop);
    return (rows + kAPieceRows - 1) / kAPieceRows * kAPieceRows;
}

int direct_split_schedule(const int2* in, int n, int2* out) {
    for (int i = 0; i < n; ++i) {
        out[2 * i] = in[i];
        out[2 * i + 1] = make_int2(in[i].x, in[i].y | (1 << 16));
    }
    return 2 * n;
}

// Dynamic shared memory a direct CTA may request: the 227 KB opt-in limit
// less room for the kernel's static barriers.
constexpr size_t kDirSmemLimit = 227 * 1024 - 1024;

// Stages: as many as fit while two CTAs still share an SM (one CTA's
// pipeline fill and epilogue then overlap the other's MMAs); if even two
// stages do not fit that way, as many as fit in one CTA's opt-in limit.
constexpr size_t kDirSmemTwoPerSm = 113 * 1024;

int direct_max_stages(int ncols, bool split, int win_rows) {
    int s = kMaxDirStages;
    while (s > 2 && direct_smem_bytes(ncols, s, split, win_rows) > kDirSmemTwoPerSm) --s;
    if (direct_smem_bytes(ncols, s, split, win_rows) <= kDirSmemTwoPerSm) return s;
    s = kMaxDirStages;
    while (s > 2 && direct_smem_bytes(ncols, s, split, win_rows) > kDirSmemLimit) --s;
    return direct_smem_bytes(ncols, s, split, win_rows) <= kDirSmemLimit ? s : 0;
}

cudaError_t direct_prepare_device() {
    cudaError_t e = cudaFuncSetAttribute(direct_mma_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kDirSmemLimit);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(direct_mma_kernel<true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDirSmemLimit);
}

cudaError_t direct_make_bank(const double* d_scales, const int32_t* d_h, int n_scales, int ncols,
                             int k_pad, int h_group, double B, double C, __nv_bfloat16* hi,
                             __nv_bfloat16* lo, float2* f32bank, cudaStream_t st) {
    const int64_t total = (int64_t)ncols * k_pad;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
    bank_kernel<<<blocks, 256, 0, st>>>(d_scales, d_h, n_scales, ncols, k_pad, h_group, B, C, hi,
                                        lo, f32bank);
    return cudaGetLastError();
}

cudaError_t direct_stage(const float* x, int64_t ld_x, const int64_t* lengths, int64_t max_len,
                         int batch, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t lpad,
                         int64_t h_front, int64_t total, cudaStream_t st) {
    // lpad and the tail are multiples of 8 elements (hop % 8 == 0, supports
    // and tap counts multiples of 8), so every 16-byte store is aligned.
    const int64_t longest = std::max<int64_t>(lpad, total - (int64_t)batch * lpad);
    const unsigned bx = (unsigned)std::min<int64_t>((longest / 8 + 255) / 256, 1024);
    dim3 grid(bx > 0 ? bx : 1, (unsigned)batch + 1);
    stage_bf16_kernel<<<grid, 256, 0, st>>>(x, ld_x, lengths, max_len, batch, hi, lo, lpad,
                                            h_front, total);
    return cudaGetLastError();
}

cudaError_t direct_launch_mma(const CUtensorMap* maps, const DirLaunch& L, bool split,
                              cudaStream_t st) {
    const int64_t tiles = (L.total_rows + kBM - 1) / kBM;
    const size_t smem = direct_smem_bytes(L.ncols, L.stages, split, L.a_shift ? L.win_rows : 0);
    if (split)
        direct_mma_kernel<true><<<(unsigned)tiles, kDirThreads, smem, st>>>(maps[0], maps[1],
                                                                           maps[2], maps[3], L);
    else
        direct_mma_kernel<false><<<(unsigned)tiles, kDirThreads, smem, st>>>(maps[0], maps[0],
                                                                            maps[2], maps[2], L);
    return cudaGetLastError();
}

cudaError_t direct_launch_f32(const float* x, int64_t ld_x, const float2* bank, const int32_t* d_h,
                              const DirLaunch& L, cudaStream_t st) {
    const int64_t ftiles = (L.frames_max + 127) / 128;
    dim3 grid((unsigned)ftiles, (unsigned)L.batch, (unsigned)L.n_scales);
    const size_t smem = (size_t)(2 * L.h_group + 1) * sizeof(float2);
    direct_f32_kernel<<<grid, 128, smem, st>>>(x, ld_x, bank, L, d_h);
    return cudaGetLastError();
}

int direct_schedule(const int32_t* h_desc, int n, int h_group, int k_pad, int2* out) {
    const int nkb = k_pad / kBK;
    const int center = h_group / kBK;
    int steps = 0;
    for (int r = 0; r < 2 * nkb; ++r) {
        // centre, centre-1, centre+1, centre-2, centre+2, ...
        const int kb = center + ((r & 1) ? -((r + 1) >> 1) : (r >> 1));
        if (kb < 0 || kb >= nkb) continue;
        const int t0 = kb * kBK - h_group, t1 = t0 + kBK - 1;
        const int d = (t0 <= 0 && t1 >= 0) ? 0 : std::min(std::abs(t0), std::abs(t1));
        int cnt = 0;
        while (cnt < n && h_desc[cnt] >= d) ++cnt;  // supports are in descending order
        if (cnt == 0) continue;
        out[steps++] = make_int2(kb, (2 * cnt + 15) / 16 * 16);
    }
    return steps;
}

cudaError_t direct_prepare_f32(size_t smem) {
    return cudaFuncSetAttribute(direct_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)std::max<size_t>(smem, 48 * 1024));
}

}  // namespace cwth
