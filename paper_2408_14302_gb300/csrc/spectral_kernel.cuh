// Spectral path of the hop-size CWT (paper Sec. II.A Eq. 1 + Sec. II.B hop):
// the device code, included by spectral.cu (512-thread CTAs, the batch
// work list, tables and launches) and spectral_solo.cu (1024-thread CTAs),
// which compile in parallel.
//
// One CTA owns one (clip, segment, scale group).  A segment is M consecutive
// samples whose left `halo` samples (a multiple of the hop) and right tail are
// context, so that the circular correlation over the segment equals the
// linear one of Eq. 1 at the segment's `seg_frames` valid frames
// (overlap-save).  Everything after the input load stays in shared memory:
//
//   a1  stage    z[n] = x[s0+2n] + i x[s0+2n+1], zero outside [0, len)
//   a2  FFT      Stockham FFT of the M/2 complex points (radix 16 with a
//                leading 8 / 4 in the 512-thread shape, radix 8 with a
//                leading 4 in the 1024-thread one), then the real-input
//                split to X[q], q = 0 .. M/2
//   a3  fold     Z_s[r] = sum_{q = r (mod P)} X[q] * sqrt(a)/M * Psi(a q/M)
//                over the unwrapped Morlet band of scale s (P = M/H); the
//                spectrum is summed over the H aliases of each bin, which is
//                decimation by the hop done in frequency
//   a4  IFFT     length-P inverse FFT of every Z_s, |.|, store the valid
//                frames of row s
//
// Short-support scales, whose bands span many hop aliases, skip a2-a4: the
// plan's cost model hands them to a time-domain phase in the same CTA that
// sums x[kH + t] g[t] over the staged samples (see fd_item below).
//
// The correlation taps g[t] = a^{-1/2} conj(psi(t/a)) have the real
// spectrum sqrt(a) sum_m Psi(a(nu - m)) (Poisson summation of the sampled
// Gaussian), so no complex multiplier is needed; bins q > M/2 come from
// conj(X[M - q]) because x is real.
//
// Shared-memory layouts: buffers are in natural order between phases.  The
// FFT passes in between write an XOR-swizzled order (element i lives at
// i ^ ((i >> 4) & 15)), which spreads every Stockham write stride over all
// banks; the last pass writes natural order again.
#pragma once
#include "cwth_internal.h"

namespace cwth {
namespace {

__device__ __forceinline__ int lay(int i, bool swz) { return swz ? (i ^ ((i >> 4) & 15)) : i; }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// times -i (forward transform) or +i (inverse transform)
template <bool INV>
__device__ __forceinline__ float2 rot90(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
    static __device__ __forceinline__ void run(float2* v) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <bool INV>
struct Dft<4, INV> {
    static __device__ __forceinline__ void run(float2* v) {
        const float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        const float2 t2 = cadd(v[1], v[3]), t3 = rot90<INV>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};

template <bool INV>
struct Dft<8, INV> {
    static __device__ __forceinline__ void run(float2* v) {
        float2 e[4] = {v[0], v[2], v[4], v[6]};
        float2 o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, INV>::run(e);
        Dft<4, INV>::run(o);
        const float h = 0.70710678118654752440f;
        // o[k] *= exp(-+ i pi k / 4)
        const float2 o1 = INV ? make_float2(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
                              : make_float2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
        const float2 o2 = rot90<INV>(o[2]);
        const float2 o3 = INV ? make_float2(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
                              : make_float2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
};

// 16 points: two 8-point DFTs of the even and odd samples joined by
// W16^k = exp(-+ 2 pi i k / 16).
template <bool INV>
struct Dft<16, INV> {
    static __device__ __forceinline__ void run(float2* v) {
        float2 e[8] = {v[0], v[2], v[4], v[6], v[8], v[10], v[12], v[14]};
        float2 o[8] = {v[1], v[3], v[5], v[7], v[9], v[11], v[13], v[15]};
        Dft<8, INV>::run(e);
        Dft<8, INV>::run(o);
        const float c1 = 0.92387953251128675613f;  // cos(pi / 8)
        const float s1 = 0.38268343236508977173f;  // sin(pi / 8)
        const float h = 0.70710678118654752440f;
        const float sg = INV ? 1.f : -1.f;        // sign of the imaginary parts
        const float2 w[8] = {make_float2(1.f, 0.f),    make_float2(c1, sg * s1),
                             make_float2(h, sg * h),   make_float2(s1, sg * c1),
                             make_float2(0.f, sg),     make_float2(-s1, sg * c1),
                             make_float2(-h, sg * h),  make_float2(-c1, sg * s1)};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float2 t = k == 0 ? o[0] : (k == 4 ? rot90<INV>(o[4]) : cmul(o[k], w[k]));
            v[k] = cadd(e[k], t);
            v[k + 8] = csub(e[k], t);
        }
    }
};

// Twiddle table in shared memory, two levels: exp(-2 pi i m / M) =
// t1[m >> 7] * t2[m & 127], t1[i] = exp(-2 pi i 128 i / M), t2[j] =
// exp(-2 pi i j / M), both generated in float64 (one extra rounding).
struct TwTab {
    const float2* t1;
    const float2* t2;
};

__device__ __forceinline__ float2 tw_at(const TwTab& t, int m) {
    return cmul(t.t1[m >> 7], t.t2[m & 127]);
}

// Multiplies v[r] by w^r, w = exp(-+ 2 pi i k / (Ns R)) = table[k * tstride]
// (conjugated for the inverse).  The powers come from a product tree of
// depth <= 4, a few roundings each (~3e-7 relative).
template <int R, bool INV>
__device__ __forceinline__ void twiddle(float2* v, const TwTab& tw, int idx) {
    float2 w1 = tw_at(tw, idx);
    if (INV) w1.y = -w1.y;
    v[1] = cmul(v[1], w1);
    if (R >= 4) {
        const float2 w2 = cmul(w1, w1);
        const float2 w3 = cmul(w2, w1);
        v[2] = cmul(v[2], w2);
        v[3] = cmul(v[3], w3);
        if (R >= 8) {
            const float2 w4 = cmul(w2, w2);
            v[4] = cmul(v[4], w4);
            v[5] = cmul(v[5], cmul(w4, w1));
            v[6] = cmul(v[6], cmul(w4, w2));
            v[7] = cmul(v[7], cmul(w4, w3));
            if (R >= 16) {
                const float2 w8 = cmul(w4, w4);
                v[8] = cmul(v[8], w8);
                v[9] = cmul(v[9], cmul(w8, w1));
                v[10] = cmul(v[10], cmul(w8, w2));
                v[11] = cmul(v[11], cmul(w8, w3));
                v[12] = cmul(v[12], cmul(w8, w4));
                v[13] = cmul(v[13], cmul(w8, cmul(w4, w1)));
                v[14] = cmul(v[14], cmul(w8, cmul(w4, w2)));
                v[15] = cmul(v[15], cmul(w8, cmul(w4, w3)));
            }
        }
    }
}

// One Stockham autosort pass over `nbatch` independent transforms of length
// L (a power of two) stored back to back in `buf`.  Ns is the length of the
// sub-transforms already done; each butterfly j reads R points spaced L/R
// apart, multiplies point r by w^{r*k} (k = j mod Ns, w = exp(-+2 pi i /
// (Ns R))), does a length-R DFT and writes the points spaced Ns apart at
// (j - k) R + k.  All reads finish before any write (barrier), so the pass
// runs in place; rs / ws select the layout read and written.  tstride is
// the twiddle-table step for one unit of r*k.
// BC: the passes before this one, of total size Ns, were skipped because
// every input is zero from index L / Ns on; their result is read in place:
// element i of transform b is x[b L + (i >> log2 Ns)] (x in natural order),
// since each skipped sub-transform saw a single nonzero sample.
template <int R, int MAXB, bool INV, bool BC = false>
__device__ __forceinline__ void fft_pass(float2* __restrict__ buf, int L, int nbatch, int Ns,
                                         const TwTab& tw, int tstride, bool rs, bool ws) {
    const int LR = L / R;
    const int lg_lr = __ffs(LR) - 1;
    const int nb = nbatch * LR;
    float2 v[MAXB][R];
#pragma unroll
    for (int u = 0; u < MAXB; ++u) {
        const int j = threadIdx.x + u * blockDim.x;
        if (j < nb) {
            const int b = j >> lg_lr;
            const int jj = j & (LR - 1);
            const int base = b * L + jj;
            // The swizzle only mixes bits 4..7 into bits 0..3, so a stride
            // that is a multiple of 256 moves a swizzled address linearly.
            if constexpr (BC) {
                const int lgN = __ffs(Ns) - 1;
#pragma unroll
                for (int r = 0; r < R; ++r) v[u][r] = buf[b * L + ((jj + r * LR) >> lgN)];
            } else if (!rs) {
#pragma unroll
                for (int r = 0; r < R; ++r) v[u][r] = buf[base + r * LR];
            } else if ((LR & 255) == 0) {
                const int a0 = lay(base, true);
#pragma unroll
                for (int r = 0; r < R; ++r) v[u][r] = buf[a0 + r * LR];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) v[u][r] = buf[lay(base + r * LR, true)];
            }
            const int k = jj & (Ns - 1);
            if (Ns > 1) twiddle<R, INV>(v[u], tw, k * tstride);
            Dft<R, INV>::run(v[u]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < MAXB; ++u) {
        const int j = threadIdx.x + u * blockDim.x;
        if (j < nb) {
            const int b = j >> lg_lr;
            const int jj = j & (LR - 1);
            const int k = jj & (Ns - 1);
            const int d = b * L + (jj - k) * R + k;
            if (!ws) {
#pragma unroll
                for (int r = 0; r < R; ++r) buf[d + r * Ns] = v[u][r];
            } else if ((Ns & 255) == 0) {
                const int a0 = lay(d, true);
#pragma unroll
                for (int r = 0; r < R; ++r) buf[a0 + r * Ns] = v[u][r];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) buf[lay(d + r * Ns, true)] = v[u][r];
            }
        }
    }
    __syncthreads();
}

// The forward FFT's pass sequence unrolled at compile time for each
// transform length: every pass's radix, stride, butterflies per thread and
// layouts are constants, and no run-time pass loop holds registers across
// passes (the run-time loop spills under the 64-register bound of the
// paired shape; each pass alone does not).  Plans: with 16 or more points
// per thread radix 16 where possible, the remainder of the exponent as a
// leading 8, 4 or 8,4 (8192 points: 8,4,16,16); with fewer, radix 8 and a
// leading 4 or 4,4.
__host__ __device__ constexpr int ct_npass(int ppt, int e) {
    return ppt >= 16 ? ((e & 3) == 3 || (e & 3) == 1 ? 1 : 0) + ((e & 3) == 2 || (e & 3) == 1 ? 1 : 0) +
                           (e - 3 * ((e & 3) == 3 || (e & 3) == 1 ? 1 : 0) -
                            2 * ((e & 3) == 2 || (e & 3) == 1 ? 1 : 0)) / 4
                     : (e % 3 == 1 ? 2 : e % 3 == 2 ? 1 : 0) +
                           (e - 2 * (e % 3 == 1 ? 2 : e % 3 == 2 ? 1 : 0)) / 3;
}
__host__ __device__ constexpr int ct_radix(int ppt, int e, int i) {
    return ppt >= 16 ? (i < ((e & 3) == 3 || (e & 3) == 1 ? 1 : 0)
                            ? 8
                            : (i < ((e & 3) == 3 || (e & 3) == 1 ? 1 : 0) +
                                       ((e & 3) == 2 || (e & 3) == 1 ? 1 : 0)
                                   ? 4
                                   : 16))
                     : (i < (e % 3 == 1 ? 2 : e % 3 == 2 ? 1 : 0) ? 4 : 8);
}

// PLAN: 16 (radix 16 with a leading 8, 4 or 8, 4) or 8 (radix 8 with a
// leading 4 or 4, 4); CAP: points a thread may hold (butterflies per thread
// of a pass <= CAP / R, the caller keeps nbatch * 2^LG <= CAP * THREADS).
// PRUNE: passes before i0 are skipped and pass i0 reads their result in
// place (see fft_pass's BC).
template <bool INV, int PLAN, int CAP, int LG, bool PRUNE, int I = 0, int NS = 1>
__device__ __forceinline__ void fft_ct(float2* buf, int nbatch, const TwTab& tw, int ts, int i0) {
    constexpr int NP = ct_npass(PLAN, LG);
    if constexpr (I < NP) {
        constexpr int R = ct_radix(PLAN, LG, I);
        constexpr int L = 1 << LG;
        constexpr int MAXB = CAP / R > 0 ? CAP / R : 1;
        constexpr int TS = L / (NS * R);
        if (!PRUNE || I >= i0) {
            if (PRUNE && I > 0 && I == i0)
                fft_pass<R, MAXB, INV, true>(buf, L, nbatch, NS, tw, ts * TS, false, I + 1 < NP);
            else
                fft_pass<R, MAXB, INV, false>(buf, L, nbatch, NS, tw, ts * TS, I > 0, I + 1 < NP);
        }
        fft_ct<INV, PLAN, CAP, LG, PRUNE, I + 1, NS * R>(buf, nbatch, tw, ts, i0);
    }
}

// Leading passes a pruned transform skips: those whose radices multiply to
// at most L / wmax, never the last (every input is zero from wmax on).
template <int PLAN>
__device__ __forceinline__ int fft_skip(int lg, int wmax) {
    const int np = ct_npass(PLAN, lg);
    int i = 0, ns = 1;
    while (i + 1 < np && (int64_t)wmax * ns * ct_radix(PLAN, lg, i) <= (1 << lg))
        ns *= ct_radix(PLAN, lg, i++);
    return i;
}

// log2 of the product of the radices fft_skip skips: the pruned transform
// reads only the first L >> fft_skip_lg entries of each input.
template <int PLAN>
__device__ __forceinline__ int fft_skip_lg(int lg, int wmax) {
    const int np = ct_npass(PLAN, lg);
    int i = 0, ns = 1, l = 0;
    while (i + 1 < np && (int64_t)wmax * ns * ct_radix(PLAN, lg, i) <= (1 << lg)) {
        const int r = ct_radix(PLAN, lg, i++);
        ns *= r;
        l += r == 16 ? 4 : (r == 8 ? 3 : (r == 4 ? 2 : 1));
    }
    return l;
}

// The forward FFT's power-of-two part: nbatch transforms of L = 2^8 ..
// 2^13 points back to back (nbatch * L <= kMaxFftPoints), the pass
// sequence unrolled at compile time for each length.
template <bool INV, int THREADS>
__device__ __forceinline__ void fft_one(float2* buf, int L, int nbatch, const TwTab& tw, int ts) {
    constexpr int PPT = kMaxFftPoints / THREADS;
    switch (__ffs(L) - 1) {
        case 8: fft_ct<INV, PPT, PPT, 8, false>(buf, nbatch, tw, ts, 0); break;
        case 9: fft_ct<INV, PPT, PPT, 9, false>(buf, nbatch, tw, ts, 0); break;
        case 10: fft_ct<INV, PPT, PPT, 10, false>(buf, nbatch, tw, ts, 0); break;
        case 11: fft_ct<INV, PPT, PPT, 11, false>(buf, nbatch, tw, ts, 0); break;
        case 12: fft_ct<INV, PPT, PPT, 12, false>(buf, nbatch, tw, ts, 0); break;
        default: fft_ct<INV, PPT, PPT, 13, false>(buf, nbatch, tw, ts, 0); break;
    }
}

// One Stockham pass of radix R (3, 5 or 7) over the block index of d blocks
// of N2 points: element n of column c sits at n N2 + c.  Butterfly (j, c),
// j < d / R, reads the R points n = j + r d / R of column c, multiplies
// point r by w_{Ns R}^{r k} (k = j mod Ns), does a length-R DFT and writes
// its outputs r to (j - k) R + k + r Ns: the mixed-radix form of fft_pass.
// FIRST (Ns = 1) also applies the decimation-in-time twiddle w_N^{n c}
// between the column FFTs and this dimension.  Twiddles come from the
// table of exp(-2 pi i m / M), M = 2N: w_N^m = tab[2m], and the DFT's own
// roots exp(-2 pi i m / R) = w_N^{m N / R}.  All reads of the pass finish
// before its writes (barrier), so it runs in place.
template <int R, int THREADS>
__device__ __forceinline__ void odd_pass(float2* X, int N2, int lgN2, int d, int Ns, bool first,
                                         const TwTab& tw) {
    constexpr int MAXB = (kMaxFftPoints / R + THREADS - 1) / THREADS;
    const int N = d * N2;
    const int dR = d / R;
    const int nb = dR * N2;
    float2 W[R];
#pragma unroll
    for (int m = 0; m < R; ++m) W[m] = tw_at(tw, 2 * m * (N / R));
    const int tstep = 2 * (N / (Ns * R));
    float2 y[MAXB][R];
#pragma unroll
    for (int u = 0; u < MAXB; ++u) {
        const int t = threadIdx.x + u * THREADS;
        if (t < nb) {
            const int c = t & (N2 - 1);
            const int j = t >> lgN2;
            const int k = j % Ns;
            float2 v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int n = j + r * dR;
                v[r] = X[n * N2 + c];
                if (first) {
                    if (n > 0) v[r] = cmul(v[r], tw_at(tw, 2 * n * c));
                } else if (r > 0) {
                    v[r] = cmul(v[r], tw_at(tw, r * k * tstep));
                }
            }
#pragma unroll
            for (int q = 0; q < R; ++q) {
                float2 a = v[0];
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const float2 w = W[(r * q) % R];
                    a.x = fmaf(v[r].x, w.x, fmaf(-v[r].y, w.y, a.x));
                    a.y = fmaf(v[r].x, w.y, fmaf(v[r].y, w.x, a.y));
                }
                y[u][q] = a;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < MAXB; ++u) {
        const int t = threadIdx.x + u * THREADS;
        if (t < nb) {
            const int c = t & (N2 - 1);
            const int j = t >> lgN2;
            const int k = j % Ns;
            const int o = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) X[(o + r * Ns) * N2 + c] = y[u][r];
        }
    }
    __syncthreads();
}

// The forward FFT of N = d N2 points, d odd (3^a 5^b 7^c <= 27), after the
// d column FFTs of N2 points: decimation in time by d,
//   X[k2 + N2 k1] = sum_{n1 < d} w_N^{n1 k2} F_{n1}[k2] w_d^{n1 k1},
// F_{n1} the N2-point DFT of x[d n2 + n1] (block n1 of the staged buffer),
// as Stockham passes of radix 7, 5, 3 over the block index; natural order
// out.  Out of line: its butterflies hold up to 18 complex values per
// thread, which must not raise the register pressure of the kernel around it.
template <int THREADS>
__device__ __noinline__ void odd_passes(float2* X, int N2, int d, const TwTab tw) {
    const int lgN2 = __ffs(N2) - 1;
    int rest = d, Ns = 1;
    while (rest > 1) {
        const bool first = Ns == 1;
        if (rest % 7 == 0) {
            odd_pass<7, THREADS>(X, N2, lgN2, d, Ns, first, tw);
            Ns *= 7;
            rest /= 7;
        } else if (rest % 5 == 0) {
            odd_pass<5, THREADS>(X, N2, lgN2, d, Ns, first, tw);
            Ns *= 5;
            rest /= 5;
        } else {
            odd_pass<3, THREADS>(X, N2, lgN2, d, Ns, first, tw);
            Ns *= 3;
            rest /= 3;
        }
    }
}

// One pass of fft_many: radix R at sub-transform length Ns, pass index i of
// np; with PRUNE the passes before i0 are skipped and pass i0 reads their
// result in place (fft_pass's BC).
template <int R, int CAP, bool INV, bool PRUNE>
__device__ __forceinline__ void fft_many_pass(float2* buf, int L, int nbatch, int Ns,
                                              const TwTab& tw, int ts, int i, int np, int i0) {
    if (PRUNE && i < i0) return;
    if (PRUNE && i > 0 && i == i0)
        fft_pass<R, CAP / R, INV, true>(buf, L, nbatch, Ns, tw, ts * (L / (Ns * R)), false,
                                        i + 1 < np);
    else
        fft_pass<R, CAP / R, INV, false>(buf, L, nbatch, Ns, tw, ts * (L / (Ns * R)), i > 0,
                                         i + 1 < np);
}

// nbatch transforms of L points (the plan's radices, as ct_radix): the
// leading radix-8 / radix-4 passes in line, then a loop whose body is the
// plan's main radix alone (a loop over every radix holds too many registers
// for the 64-register bound of the paired shape).
template <bool INV, int PLAN, int CAP, bool PRUNE = false>
__device__ __forceinline__ void fft_many(float2* buf, int L, int nbatch, const TwTab& tw, int ts,
                                         int wmax = 0) {
    const int e = __ffs(L) - 1;
    const int np = ct_npass(PLAN, e);
    const int i0 = PRUNE ? fft_skip<PLAN>(e, wmax) : 0;
    int i = 0, Ns = 1;
    if constexpr (PLAN >= 16) {
        const int m = e & 3;
        if (m == 3 || m == 1) {
            fft_many_pass<8, CAP, INV, PRUNE>(buf, L, nbatch, Ns, tw, ts, i, np, i0);
            Ns *= 8;
            ++i;
        }
        if (m == 2 || m == 1) {
            fft_many_pass<4, CAP, INV, PRUNE>(buf, L, nbatch, Ns, tw, ts, i, np, i0);
            Ns *= 4;
            ++i;
        }
        for (; i < np; ++i, Ns *= 16)
            fft_many_pass<16, CAP, INV, PRUNE>(buf, L, nbatch, Ns, tw, ts, i, np, i0);
    } else {
        const int n4 = (e % 3 == 1) ? 2 : (e % 3 == 2) ? 1 : 0;
        for (; i < n4; ++i, Ns *= 4)
            fft_many_pass<4, CAP, INV, PRUNE>(buf, L, nbatch, Ns, tw, ts, i, np, i0);
        for (; i < np; ++i, Ns *= 8)
            fft_many_pass<8, CAP, INV, PRUNE>(buf, L, nbatch, Ns, tw, ts, i, np, i0);
    }
}

__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Hardware square-root approximation (sqrt.approx), a few ulp, far below
// the path's 1e-5 tolerance; |z| of the inverse transforms.
__device__ __forceinline__ float fast_sqrt(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Sums of X[q] * exp2(kexp * (qf * a_over_m - C)^2) over n bins of one run,
// for NS = 1 or 2 scales at once (adjacent scales of the ascending list,
// whose Morlet bands nest, share one walk and one load of each bin):
// indices q0, q0 + dq, ... (dq = +-P) and unwrapped bin positions qf,
// qf + P, ... .  The weight is a sampled Gaussian: with u_j the argument at
// bin j and D = a P / M its step, g_{j+1} = g_j r_j, r_j = 2^{kexp (2 u_j D
// + D^2)} and r_{j+1} = r_j Q, Q = 2^{2 kexp D^2}.  The recurrence is
// anchored at the exact argument (ex2.approx, ~2^-22 relative) every 8
// bins, including a run's last, partial chunk (at most ~3.5e-6 relative
// drift at a chunk's end; D <= 0.35 where runs are long, so the ratios stay
// in range).  LGP > 0 fixes the stride at compile time (dq = SIGN * 2^LGP),
// so the loads of a chunk address X with immediate offsets; LGP = 0 takes
// dq as passed.
template <int LGP, int SIGN, int NS>
__device__ __forceinline__ void fold_run(const float2* __restrict__ X, int q0, int dq_rt, int n,
                                         float qf, float pf, const SpecScale* sc, float cneg,
                                         float kexp, float2* acc) {
    const int dq = LGP ? SIGN * (1 << LGP) : dq_rt;
    const float2* xp = X + q0;
    if (n <= 2) {
        // Runs of one or two bins (small hops): an exact weight per bin is
        // cheaper than anchoring the recurrence.
        for (int t = 0; t < n; ++t) {
            const float2 v = xp[t * dq];
#pragma unroll
            for (int k = 0; k < NS; ++k) {
                const float u = fmaf(qf + (float)t * pf, sc[k].a_over_m, cneg);
                const float g = fast_exp2(kexp * u * u);
                acc[k].x = fmaf(v.x, g, acc[k].x);
                acc[k].y = fmaf(v.y, g, acc[k].y);
            }
        }
        return;
    }
    for (int j = 0; j < n; j += 8) {
        float g[NS], r[NS];
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            const float u = fmaf(qf, sc[k].a_over_m, cneg);
            const float d = sc[k].dlt;
            g[k] = fast_exp2(kexp * u * u);
            r[k] = fast_exp2(kexp * fmaf(2.f * u, d, d * d));
        }
        if (j + 8 <= n) {
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const float2 v = xp[t * dq];
#pragma unroll
                for (int k = 0; k < NS; ++k) {
                    acc[k].x = fmaf(v.x, g[k], acc[k].x);
                    acc[k].y = fmaf(v.y, g[k], acc[k].y);
                    g[k] *= r[k];
                    r[k] *= sc[k].q2;
                }
            }
        } else {
            for (int t = 0; t < n - j; ++t) {
                const float2 v = xp[t * dq];
#pragma unroll
                for (int k = 0; k < NS; ++k) {
                    acc[k].x = fmaf(v.x, g[k], acc[k].x);
                    acc[k].y = fmaf(v.y, g[k], acc[k].y);
                    g[k] *= r[k];
                    r[k] *= sc[k].q2;
                }
            }
        }
        xp += 8 * dq;
        qf += 8.f * pf;
    }
}

// Z_k[r] = gscale_k * sum over the unwrapped band of the bins q_u = r
// (mod P) of X[q_u mod M] * Psi_k-weight, for the NS scales sc[0..NS-1]
// walked together over the union of their bands (outside its own band a
// scale's weights are below the band threshold and add next to nothing);
// bins above M/2 are read as conj(X[M - q]).  The walk is split into runs
// that stay on one side of M/2, so the inner loop is branch-free.
// LGP > 0: P = 2^LGP at compile time.
template <int LGP, int NS, bool MODM>
__device__ __forceinline__ void fold_residue(const float2* __restrict__ X, const SpecScale* sc,
                                             int r, int M, int Mh, int P_rt, int lgP_rt, float cneg,
                                             float kexp, float2* out) {
    const int P = LGP ? (1 << LGP) : P_rt;
    const int lgP = LGP ? LGP : lgP_rt;
    int q_lo = sc[0].q_lo, q_hi = sc[0].q_hi;
    if (NS > 1) {
        q_lo = min(q_lo, sc[NS - 1].q_lo);
        q_hi = max(q_hi, sc[NS - 1].q_hi);
    }
    int qu = q_lo + ((r - q_lo) & (P - 1));
    int left = qu <= q_hi ? ((q_hi - qu) >> lgP) + 1 : 0;
    const float pf = (float)P;
    float2 ad[NS], am[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) ad[k] = am[k] = make_float2(0.f, 0.f);
    while (left > 0) {
        int q;
        if (MODM) {
            q = qu % M;
            q += q < 0 ? M : 0;
        } else {
            q = qu & (M - 1);
        }
        int n;
        if (q <= Mh) {
            n = min(left, ((Mh - q) >> lgP) + 1);
            fold_run<LGP, 1, NS>(X, q, P, n, (float)qu, pf, sc, cneg, kexp, ad);
        } else {
            n = min(left, ((M - 1 - q) >> lgP) + 1);
            fold_run<LGP, -1, NS>(X, M - q, -P, n, (float)qu, pf, sc, cneg, kexp, am);
        }
        qu += n * P;
        left -= n;
    }
#pragma unroll
    for (int k = 0; k < NS; ++k)
        out[k] = make_float2(sc[k].gscale * (ad[k].x + am[k].x), sc[k].gscale * (ad[k].y - am[k].y));
}

// Fused time-domain scales.  The window buffer Xw[tau][f] =
// xs[halo + f H - hw + tau] (tau = 0 .. 2 hw, f < seg_frames, rows fst
// floats apart, fst odd) is copied from the staged samples before the
// forward FFT overwrites them: each warp reads consecutive samples and
// writes a column with an odd stride, both free of bank conflicts.  (The
// taps and group records were copied during staging.)
__device__ __forceinline__ void fd_copy_windows(const SpecLaunch& p, const float* __restrict__ xs,
                                                float* __restrict__ Xw, float2* __restrict__ T) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int wlen = 2 * p.fd_hw + 1, fst = p.fd_fst, H = p.hop;
    const float* src = xs + p.halo - p.fd_hw;
    // Four rows chunks of 32 per step: loads first, then stores.
    for (int f = warp; f < p.seg_frames; f += nwarps) {
        const float* sf = src + f * H;
        for (int t0 = lane; t0 < wlen; t0 += 128) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = t0 + 32 * u < wlen ? sf[t0 + 32 * u] : 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (t0 + 32 * u < wlen) Xw[(t0 + 32 * u) * fst + f] = v[u];
        }
    }
}

// One fused item: the n scales of tap group g over the 32 frames
// f = fb * 32 + lane of the segment, W[f] = sum_tau Xw[tau'][f] T[tau] with
// tau' = tau + hw - hg and T[tau] the group's taps at t = tau - hg (zero
// beyond each scale's own support).  Lanes read one window row per tap
// (consecutive frames: conflict-free); every lane reads the same taps
// (a broadcast through L1).  GP2 = gp / 2 float4 tap loads per row.
template <int GP2>
__device__ __forceinline__ void fd_sum(const float* __restrict__ xc, int fst,
                                       const float4* __restrict__ tp, int ntau, float2* acc) {
#pragma unroll
    for (int j = 0; j < 2 * GP2; ++j) acc[j] = make_float2(0.f, 0.f);
    int tau = 0;
    // Four rows per step, every load of the step issued before its FMAs.
    for (; tau + 4 <= ntau; tau += 4) {
        float x[4];
        float4 t[4][GP2];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            x[u] = xc[u * fst];
#pragma unroll
            for (int j = 0; j < GP2; ++j) t[u][j] = tp[u * GP2 + j];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < GP2; ++j) {
                acc[2 * j].x = fmaf(x[u], t[u][j].x, acc[2 * j].x);
                acc[2 * j].y = fmaf(x[u], t[u][j].y, acc[2 * j].y);
                acc[2 * j + 1].x = fmaf(x[u], t[u][j].z, acc[2 * j + 1].x);
                acc[2 * j + 1].y = fmaf(x[u], t[u][j].w, acc[2 * j + 1].y);
            }
        xc += 4 * fst;
        tp += 4 * GP2;
    }
    for (; tau < ntau; ++tau) {
        const float x0 = xc[0];
#pragma unroll
        for (int j = 0; j < GP2; ++j) {
            const float4 t0 = tp[j];
            acc[2 * j].x = fmaf(x0, t0.x, acc[2 * j].x);
            acc[2 * j].y = fmaf(x0, t0.y, acc[2 * j].y);
            acc[2 * j + 1].x = fmaf(x0, t0.z, acc[2 * j + 1].x);
            acc[2 * j + 1].y = fmaf(x0, t0.w, acc[2 * j + 1].y);
        }
        xc += fst;
        tp += GP2;
    }
}

__device__ __forceinline__ void fd_item(const SpecLaunch& p, const float* __restrict__ Xw,
                                        const float2* __restrict__ T, const FdGroup* G, int clip,
                                        int64_t k0, int64_t F, int g, int fb) {
    const int lane = threadIdx.x & 31;
    const FdGroup gr = G[g];
    const int Fs = p.seg_frames, fst = p.fd_fst;
    const int f = fb * 32 + lane;
    const int fc = f < Fs ? f : Fs - 1;  // idle lanes re-read a valid column
    const float* xc = Xw + (p.fd_hw - gr.hg) * fst + fc;
    const float4* tp = reinterpret_cast<const float4*>(T + gr.off);
    const int ntau = 2 * gr.hg + 1;
    float2 acc[kFdMaxG];
    if (gr.gp <= 2)
        fd_sum<1>(xc, fst, tp, ntau, acc);
    else
        fd_sum<2>(xc, fst, tp, ntau, acc);
    const int64_t k = k0 + f;
    if (f < Fs && k < F) {
        float* o = p.out + (int64_t)clip * p.S_total * p.frames_max + k;
#pragma unroll
        for (int j = 0; j < kFdMaxG; ++j)
            if (j < gr.n)
                o[(int64_t)gr.row[j] * p.frames_max] =
                    fast_sqrt(fmaf(acc[j].x, acc[j].x, acc[j].y * acc[j].y));
    }
}

// Fused items of the CTA of scale group grp (of ngrp): tap groups grp,
// grp + ngrp, ... times the frame blocks; item i is (group grp + (i / nfb)
// ngrp, frame block i % nfb).
struct FdWork {
    const float* Xw;
    const float2* T;
    const FdGroup* G;
    int clip, grp, ngrp, nfb, nitems;
    int64_t k0, F;
};

__device__ __forceinline__ FdWork fd_work(const SpecLaunch& p, const float* Xw, const float2* T,
                                          const FdGroup* G, int clip, int64_t k0, int64_t F,
                                          int grp, int ngrp) {
    FdWork w;
    w.Xw = Xw;
    w.T = T;
    w.G = G;
    w.clip = clip;
    w.grp = grp;
    w.ngrp = ngrp;
    w.nfb = (p.seg_frames + 31) >> 5;
    w.nitems = grp < p.fd_groups ? ((p.fd_groups - grp + ngrp - 1) / ngrp) * w.nfb : 0;
    w.k0 = k0;
    w.F = F;
    return w;
}

__device__ __forceinline__ void fd_run(const SpecLaunch& p, const FdWork& w, int i) {
    const int q = i / w.nfb;
    fd_item(p, w.Xw, w.T, w.G, w.clip, w.k0, w.F, w.grp + q * w.ngrp, i - q * w.nfb);
}

// a3 for one chunk of scales: band multiply + hop fold.  Scales are taken
// in adjacent pairs (c, c + 1), whose bands nest, and folded together; the
// chunk's (pair, residue) items are numbered g = c2 P + r; one item = 32
// consecutive g (32 residues of one pair, or 32 / P whole pairs when
// P < 32), one lane each; the loop walks the unwrapped band.  Items are
// ordered by decreasing band width (scales ascend); they are dealt to warps
// in a snake order to balance the work.
//
// SHIFT (the pruned kernel): each band is stored shifted to residue 0 and
// the inverse FFT reads only the first 2^lgneed residues of each scale
// (the rest of a skipped pass's input is zero), so only those are folded,
// one scale per lane: item g = c 2^lgneed + r' folds residue r' + q_lo.
template <int LGP, bool SHIFT, bool MODM = false>
__device__ __forceinline__ void fold_items(const SpecLaunch& p, const float2* __restrict__ X,
                                           float2* __restrict__ Z, int c0, int nc, int M, int P,
                                           int lgP, int lgneed = 0) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const float cneg = -p.center;
    if constexpr (SHIFT) {
        const int nitems = ((nc << lgneed) + 31) >> 5;
        for (int round = 0;; ++round) {
            const int it = round * nwarps + ((round & 1) ? nwarps - 1 - warp : warp);
            if (it >= nitems) break;
            const int g = (it << 5) + lane;
            const int c = g >> lgneed;
            if (c >= nc) continue;
            const int rs = g & ((1 << lgneed) - 1);
            const SpecScale sc = p.sc[c0 + c];
            if (sc.q_hi - sc.q_lo + 1 > 2 * P) {
                // Bands of several bins per residue: the recurrence walk.
                float2 z;
                fold_residue<LGP, 1, MODM>(X, &sc, (rs + sc.q_lo) & (P - 1), M, M >> 1, P, lgP,
                                           cneg, p.kexp, &z);
                Z[c * P + rs] = z;
                continue;
            }
            // One or two bins per residue: a plain walk with an exact weight
            // per bin.
            float2 acc = make_float2(0.f, 0.f);
            for (int qu = sc.q_lo + rs; qu <= sc.q_hi; qu += P) {
                int q;
                if (MODM) {
                    q = qu % M;
                    q += q < 0 ? M : 0;
                } else {
                    q = qu & (M - 1);
                }
                float2 v;
                if (q <= (M >> 1)) {
                    v = X[q];
                } else {
                    v = X[M - q];
                    v.y = -v.y;
                }
                const float u = fmaf((float)qu, sc.a_over_m, cneg);
                const float g = fast_exp2(p.kexp * u * u);
                acc.x = fmaf(v.x, g, acc.x);
                acc.y = fmaf(v.y, g, acc.y);
            }
            Z[c * P + rs] = make_float2(sc.gscale * acc.x, sc.gscale * acc.y);
        }
        return;
    }
    const int npairs = (nc + 1) >> 1;
    const int nitems = (npairs * P + 31) >> 5;
    for (int round = 0;; ++round) {
        const int it = round * nwarps + ((round & 1) ? nwarps - 1 - warp : warp);
        if (it >= nitems) break;
        const int g = (it << 5) + lane;
        const int c = (g >> lgP) * 2;
        const int r = g & (P - 1);
        if (c >= nc) continue;
        SpecScale sc[2];
        sc[0] = p.sc[c0 + c];
        float2 z[2];
        if (c + 1 < nc) {
            sc[1] = p.sc[c0 + c + 1];
            if (sc[0].pair) {
                fold_residue<LGP, 2, MODM>(X, sc, r, M, M >> 1, P, lgP, cneg, p.kexp, z);
            } else {
                fold_residue<LGP, 1, MODM>(X, sc, r, M, M >> 1, P, lgP, cneg, p.kexp, z);
                fold_residue<LGP, 1, MODM>(X, sc + 1, r, M, M >> 1, P, lgP, cneg, p.kexp, z + 1);
            }
            Z[(c + 1) * P + r] = z[1];
        } else {
            fold_residue<LGP, 1, MODM>(X, sc, r, M, M >> 1, P, lgP, cneg, p.kexp, z);
        }
        Z[c * P + r] = z[0];
    }
}

// Clip length (clamped to [0, max_len]), frame count and first frame of the
// CTA's segment.  reload: read the length again with a load the compiler
// may not merge with an earlier one.
__device__ __forceinline__ void cta_pos(const SpecLaunch& p, bool reload, int seg, int clip,
                                        int64_t* len, int64_t* F, int64_t* k0) {
    int64_t n = p.max_len;
    if (p.lengths) {
        const int64_t* a = p.lengths + clip;
        if (reload)
            asm volatile("ld.global.nc.s64 %0, [%1];" : "=l"(n) : "l"(a));
        else
            n = __ldg(a);
    }
    n = n < 0 ? 0 : (n > p.max_len ? p.max_len : n);
    *len = n;
    *F = (n + p.hop - 1) / p.hop;
    *k0 = (int64_t)seg * p.seg_frames;
}

template <int THREADS, bool PRUNE>
__device__ __forceinline__ void spectral_body(const SpecLaunch& p, int seg, int clip, int grp);

// One work item: segment `seg` of clip `clip`, scale group `grp` of `ngrp`
// (the spectral scales of the group and the fused tap groups grp, grp +
// ngrp, ...).  Every thread of the CTA calls it with the same arguments.
// PRUNE: inverse FFTs skip the passes that a chunk's narrow bands leave
// trivial (plans whose narrowest folded band fits a small fraction of P).
template <int THREADS, bool PRUNE>
__device__ __forceinline__ void spectral_item(const SpecLaunch& p, int seg, int clip, int grp,
                                              int ngrp) {
    extern __shared__ float2 smem[];
    const int M = p.M, Mh = M >> 1;
    const int ntw = (M >> 7) + 128;
    float2* T = smem;                 // two-level twiddle table, ntw entries
    float2* X = smem + ntw;           // Mh + 1 used
    float2* Z = smem + ntw + Mh + 2;  // nconc * P used
    const TwTab tab{T, T + (M >> 7)};

    int64_t len, F, k0;
    cta_pos(p, false, seg, clip, &len, &F, &k0);
    const bool has_sp = grp * p.group_size < p.n_sp;
    const bool has_fd = grp < p.fd_groups;
    if (k0 >= F || !(has_sp || has_fd)) return;

    if (has_sp)
        for (int i = threadIdx.x; i < ntw; i += blockDim.x) T[i] = __ldg(p.tw + i);

    // a1: stage the segment as M/2 complex points (x[s0 + i] is float i of X).
    const int64_t s0 = k0 * p.hop - p.halo;
    const float* xr = p.x + (int64_t)clip * p.ld_x;
    if (p.vec4 && s0 >= 0 && s0 + M <= len) {
        // Interior segment: plain float4 copies, loads issued together.
        float4* X4 = reinterpret_cast<float4*>(X);
        const float4* x4 = reinterpret_cast<const float4*>(xr + s0);
        const int n4 = M >> 2;
        for (int base = threadIdx.x; base < n4; base += 4 * blockDim.x) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int n = base + u * blockDim.x;
                if (n < n4) v[u] = __ldg(x4 + n);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int n = base + u * blockDim.x;
                if (n < n4) X4[n] = v[u];
            }
        }
    } else if (p.vec4) {
        // Four samples per load; the loads of a thread are issued together.
        float4* X4 = reinterpret_cast<float4*>(X);
        const int n4 = M >> 2;
        for (int base = threadIdx.x; base < n4; base += 4 * blockDim.x) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int n = base + u * blockDim.x;
                const int64_t i0 = s0 + 4 * (int64_t)n;
                if (n < n4 && i0 >= 0 && i0 + 3 < len) {
                    v[u] = __ldg(reinterpret_cast<const float4*>(xr + i0));
                } else {
                    float e[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        e[q] = (n < n4 && i0 + q >= 0 && i0 + q < len) ? __ldg(xr + i0 + q) : 0.f;
                    v[u] = make_float4(e[0], e[1], e[2], e[3]);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int n = base + u * blockDim.x;
                if (n < n4) X4[n] = v[u];
            }
        }
    } else {
        // Scalar pairs; with an odd factor d in M/2 = d N2, complex point n
        // goes to column n mod d, row n / d (the forward FFT's column layout).
        const int d = p.fft_d, n2 = p.fft_n2;
        for (int n = threadIdx.x; n < Mh; n += blockDim.x) {
            const int64_t i0 = s0 + 2 * (int64_t)n;
            const float a = (i0 >= 0 && i0 < len) ? __ldg(xr + i0) : 0.f;
            const float b = (i0 + 1 >= 0 && i0 + 1 < len) ? __ldg(xr + i0 + 1) : 0.f;
            int at = n;
            if (d > 1) {
                const int q = n / d;
                at = (n - q * d) * n2 + q;
            }
            X[at] = make_float2(a, b);
        }
    }
    if (has_fd) {
        // The fused scales' taps and group records, into the fold's buffer
        // (unused until the fold) while the sample loads are in flight.
        float2* Tfd = Z;
        for (int i = threadIdx.x; i < p.fd_taps_n; i += blockDim.x) Tfd[i] = __ldg(p.fd_taps + i);
        int* Gw = reinterpret_cast<int*>(Tfd + p.fd_taps_n);
        const int* Gr = reinterpret_cast<const int*>(p.fd_grp);
        const int nw = p.fd_groups * (int)(sizeof(FdGroup) / sizeof(int));
        for (int i = threadIdx.x; i < nw; i += blockDim.x) Gw[i] = __ldg(Gr + i);
    }
    __syncthreads();

    // Short-support scales: summed here, before the forward FFT overwrites
    // the staged samples.
    if (has_fd) {
        // Fused time-domain scales: taps and frame windows in the fold's
        // buffer (unused until the fold), items dealt to whichever warp is
        // free (a shared counter, largest groups first).
        float2* Tfd = Z;
        const FdGroup* Gfd = reinterpret_cast<const FdGroup*>(Tfd + p.fd_taps_n);
        float* Xw = reinterpret_cast<float*>(const_cast<FdGroup*>(Gfd) + p.fd_groups);
        __shared__ int s_ctr;
        if (threadIdx.x == 0) s_ctr = 0;
        fd_copy_windows(p, reinterpret_cast<const float*>(X), Xw, Tfd);
        __syncthreads();
        const FdWork fw = fd_work(p, Xw, Tfd, Gfd, clip, k0, F, grp, ngrp);
        const int lane = threadIdx.x & 31;
        for (;;) {
            int it = 0;
            if (lane == 0) it = atomicAdd(&s_ctr, 1);
            it = __shfl_sync(0xffffffffu, it, 0);
            if (it >= fw.nitems) break;
            fd_run(p, fw, it);
        }
        __syncthreads();
    }
    if (!has_sp) return;
    spectral_body<THREADS, PRUNE>(p, seg, clip, grp);
}

// One CTA per (segment, clip, scale group) of one plan.
template <int THREADS, bool PRUNE>
__global__ void __launch_bounds__(THREADS, THREADS >= 1024 ? 1 : 2)
    spectral_segment_kernel(const SpecLaunch p) {
    // The plan's next spectral part, launched as a programmatic dependent,
    // may start on the SMs this grid's last CTAs leave idle.
    asm volatile("griddepcontrol.launch_dependents;");
    spectral_item<THREADS, PRUNE>(p, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.z);
    // As such a dependent (the parts read the same input and write disjoint
    // rows, so nothing waits at the start), the grid completes only after
    // the part before it, and whatever follows on the stream still follows
    // every part; in any other launch this returns at once.
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Launches kern with programmatic stream serialisation: it may begin once
// every CTA of the kernel before it on st has started.
inline cudaError_t spectral_launch_dependent(void (*kern)(SpecLaunch), const SpecLaunch& L,
                                             dim3 grid, int threads, size_t smem,
                                             cudaStream_t st) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, L);
}

// One launch over a device work list spanning several plans (the groups
// of an uneven batch): block i runs item i, {group, segment, clip, scale
// group | scale groups << 16}, with its plan's record read from the launch
// parameters as in the one-plan kernel.  Items come longest first, so the
// hardware's block scheduler, which starts blocks in order as SMs free up,
// deals them longest-first to whichever SM is free.  (A loop over items
// inside one block keeps the item's state in registers across iterations
// and spills; one item per block does not.)
template <int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS >= 1024 ? 1 : 2)
    spectral_worklist_kernel(const __grid_constant__ SpecWorkList wl) {
    const int4 w = __ldg(wl.items + blockIdx.x);
    spectral_item<THREADS, false>(wl.g[w.x], w.y, w.z, w.w & 0xffff, w.w >> 16);
}

// Everything from the forward FFT on.  Its per-CTA values are derived again
// from the launch parameters (the clip length reloaded), so that none of
// them occupies a register through the FFT passes.
template <int THREADS, bool PRUNE>
__device__ __forceinline__ void spectral_body(const SpecLaunch& p, int seg, int clip, int grp) {
    constexpr int kPPT = kMaxFftPoints / THREADS;  // FFT points per thread
    extern __shared__ float2 smem[];
    const int M = p.M, Mh = M >> 1;
    const int ntw = (M >> 7) + 128;
    float2* T = smem;
    float2* X = smem + ntw;
    const TwTab tab{T, T + (M >> 7)};

    // a2: forward FFT of the M/2 points, twiddles exp(-2 pi i m/(M/2)) = tw[2m]:
    // fft_d column FFTs of fft_n2 points (one when M/2 is a power of two),
    // then the odd-radix passes across the columns.
    {
        const int d = p.fft_d;
        fft_one<false, THREADS>(X, p.fft_n2, d, tab, 2 * d);
        if (d > 1) odd_passes<THREADS>(X, p.fft_n2, d, tab);
    }

    // Real-input split: with Z = FFT(z), E = (Z[q] + conj Z[Mh-q])/2 and
    // O = (Z[q] - conj Z[Mh-q])/(2i) are the spectra of the even and odd
    // samples, X[q] = E + exp(-2 pi i q/M) O and X[Mh-q] = conj(E - exp(-2 pi i q/M) O).
    // Each pair (q, Mh-q) is read and written by one thread only.
    for (int q = threadIdx.x; q <= (Mh >> 1); q += blockDim.x) {
        const int qm = q == 0 ? 0 : Mh - q;
        const float2 zq = X[q];
        const float2 zm = X[qm];
        const float2 E = make_float2(0.5f * (zq.x + zm.x), 0.5f * (zq.y - zm.y));
        const float2 O = make_float2(0.5f * (zq.y + zm.y), 0.5f * (zm.x - zq.x));
        const float2 t = cmul(tw_at(tab, q), O);
        const float2 xq = cadd(E, t);
        const float2 xm = csub(E, t);
        X[q] = xq;
        X[Mh - q] = make_float2(xm.x, -xm.y);
    }
    __syncthreads();

    const int P = p.P;
    float2* Z = smem + ntw + Mh + 2;
    // The CTA's position lives in shared memory through the chunk loop and
    // is read back (volatile) where it is needed, so that nothing but the
    // chunk index holds a register through the inverse FFT's passes.
    __shared__ int s_pos[3];
    if (threadIdx.x == 0) {
        s_pos[0] = seg;
        s_pos[1] = clip;
        s_pos[2] = grp;
    }
    __syncthreads();
    const volatile int* vpos = s_pos;
    const int lgP = __ffs(P) - 1;
    for (int c0 = vpos[2] * p.group_size;; c0 += p.nconc) {
        const int sp_end = min(p.n_sp, vpos[2] * p.group_size + p.group_size);
        if (c0 >= sp_end) break;
        const int nc = min(p.nconc, sp_end - c0);

        // a3: the band walks of 8 or more bins per residue occur for P up to
        // M/16; those periods get a compile-time stride.  A segment length
        // with an odd factor takes the run-time stride and reduces bins
        // modulo M by division.
        const int lgneed = PRUNE ? lgP - fft_skip_lg<kPPT>(lgP, p.sc[c0].wsuf) : lgP;
        if (p.fft_d > 1) fold_items<0, PRUNE, true>(p, X, Z, c0, nc, M, P, lgP, lgneed);
        else switch (lgP) {
            case 4: fold_items<4, PRUNE>(p, X, Z, c0, nc, M, P, lgP, lgneed); break;
            case 5: fold_items<5, PRUNE>(p, X, Z, c0, nc, M, P, lgP, lgneed); break;
            case 6: fold_items<6, PRUNE>(p, X, Z, c0, nc, M, P, lgP, lgneed); break;
            case 7: fold_items<7, PRUNE>(p, X, Z, c0, nc, M, P, lgP, lgneed); break;
            case 8: fold_items<8, PRUNE>(p, X, Z, c0, nc, M, P, lgP, lgneed); break;
            case 9: fold_items<9, PRUNE>(p, X, Z, c0, nc, M, P, lgP, lgneed); break;
            case 10: fold_items<10, PRUNE>(p, X, Z, c0, nc, M, P, lgP, lgneed); break;
            default: fold_items<0, PRUNE>(p, X, Z, c0, nc, M, P, lgP, lgneed); break;
        }
        __syncthreads();

        // a4: inverse FFT of length P for every scale of the chunk; the 1/M
        // normalisation is already in gscale.  exp(+2 pi i m/P) = conj(tw[m H]).
        // With PRUNE every band of the chunk lies in its first sc[c0].wsuf
        // residues.
        // Few points per thread: the radix-8 plan (radix 8 with a leading 4
        // or 4, 4) keeps more warps busy than radix-16 butterflies would.
        if (!PRUNE && kPPT > 8 && p.inv_r8)
            fft_many<true, 8, 8>(Z, P, nc, tab, p.hop);
        else
            fft_many<true, kPPT, kPPT, PRUNE>(Z, P, nc, tab, p.hop, PRUNE ? p.sc[c0].wsuf : 0);

        // Stores: one warp per scale row, or (fewer rows than warps) warp
        // items of 32 consecutive frames of one row; the row is read once
        // per row or item, stores are coalesced and reads conflict-free.
        {
            const int clip = vpos[1];
            const int nc = min(p.nconc, min(p.n_sp, vpos[2] * p.group_size + p.group_size) - c0);
            int64_t len, F, k0;
            cta_pos(p, true, vpos[0], clip, &len, &F, &k0);
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            const int nwarps = blockDim.x >> 5;
            const int Fs = p.seg_frames;
            const int fend = (int)(F - k0 < (int64_t)Fs ? F - k0 : (int64_t)Fs);
            if (nc >= nwarps) {
                // One warp per row while there are rows for every warp.
                for (int c = warp; c < nc; c += nwarps) {
                    float* o = p.out +
                               ((int64_t)clip * p.S_total + p.sc[c0 + c].row) * p.frames_max + k0;
                    const float2* z = Z + c * P + p.kp0;
                    for (int f = lane; f < fend; f += 32) {
                        const float2 w = z[f];
                        o[f] = fast_sqrt(fmaf(w.x, w.x, w.y * w.y));
                    }
                }
            } else {
                // Fewer rows than warps (small hops, long rows): the whole
                // CTA strides over one row's frames at a time, independent
                // iterations, so loads and stores overlap.
                for (int c = 0; c < nc; ++c) {
                    float* o = p.out +
                               ((int64_t)clip * p.S_total + p.sc[c0 + c].row) * p.frames_max + k0;
                    const float2* z = Z + c * P + p.kp0;
#pragma unroll 4
                    for (int f = threadIdx.x; f < fend; f += blockDim.x) {
                        const float2 w = z[f];
                        o[f] = fast_sqrt(fmaf(w.x, w.x, w.y * w.y));
                    }
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace cwth
