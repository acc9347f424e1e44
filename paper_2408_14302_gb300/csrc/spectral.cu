// Spectral path of the hop-size CWT (paper Sec. II.A Eq. 1 + Sec. II.B hop).
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
// The correlation taps g[t] = a^{-1/2} conj(psi(t/a)) have the real
// spectrum sqrt(a) sum_m Psi(a(nu - m)) (Poisson summation of the sampled
// Gaussian), so no complex multiplier is needed; bins q > M/2 come from
// conj(X[M - q]) because x is real.
//
// Shared-memory layouts: buffers are in natural order between phases.  The
// FFT passes in between write an XOR-swizzled order (element i lives at
// i ^ ((i >> 4) & 15)), which spreads every Stockham write stride over all
// banks; the last pass writes natural order again.
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

template <int R, bool INV, int PPT, bool BC = false>
__device__ __forceinline__ void fft_pass_dispatch(float2* buf, int L, int nbatch, int Ns,
                                                  const TwTab& tw, int tstride, bool rs, bool ws) {
    const int nb = nbatch * (L / R);
    const int per = (nb + blockDim.x - 1) / blockDim.x;
    // Up to PPT complex values per thread: the caller keeps nbatch * L <=
    // kMaxFftPoints = PPT * blockDim.x.
    constexpr int kMaxB = PPT / R;
    if (per <= 1 || kMaxB <= 1)
        fft_pass<R, 1, INV, BC>(buf, L, nbatch, Ns, tw, tstride, rs, ws);
    else if (per <= 2 || kMaxB <= 2)
        fft_pass<R, 2, INV, BC>(buf, L, nbatch, Ns, tw, tstride, rs, ws);
    else if (per <= 4 || kMaxB <= 4)
        fft_pass<R, (kMaxB < 4 ? kMaxB : 4), INV, BC>(buf, L, nbatch, Ns, tw, tstride, rs, ws);
    else
        fft_pass<R, kMaxB, INV, BC>(buf, L, nbatch, Ns, tw, tstride, rs, ws);
}

// Radix of pass i of a transform of 2^e points.  With 16 or more points
// per thread: 16 where possible, the remainder of e as a leading 8, 4 or
// 8,4 (8192 points: 8,4,16,16); with fewer: 8 where possible, a leading 4
// (or 4,4).
template <int PPT>
__device__ __forceinline__ int fft_radix(int e, int i) {
    if constexpr (PPT >= 16) {
        const int m = e & 3;
        const int n8 = (m == 3 || m == 1) ? 1 : 0;
        const int n4 = (m == 2 || m == 1) ? 1 : 0;
        return i < n8 ? 8 : (i < n8 + n4 ? 4 : 16);
    } else {
        const int n4 = (e % 3 == 1) ? 2 : (e % 3 == 2) ? 1 : 0;
        return i < n4 ? 4 : 8;
    }
}

template <int PPT>
__device__ __forceinline__ int fft_npass(int e) {
    if constexpr (PPT >= 16) {
        const int m = e & 3;
        const int n8 = (m == 3 || m == 1) ? 1 : 0;
        const int n4 = (m == 2 || m == 1) ? 1 : 0;
        return n8 + n4 + (e - 3 * n8 - 2 * n4) / 4;
    } else {
        const int n4 = (e % 3 == 1) ? 2 : (e % 3 == 2) ? 1 : 0;
        return n4 + (e - 2 * n4) / 3;
    }
}

template <bool INV, int PPT, bool BC>
__device__ __forceinline__ void fft_pass_radix(int R, float2* buf, int L, int nbatch, int Ns,
                                               const TwTab& tw, int ts, bool rs, bool ws) {
    if (R == 4) {
        fft_pass_dispatch<4, INV, PPT, BC>(buf, L, nbatch, Ns, tw, ts * (L / (Ns * 4)), rs, ws);
    } else if (R == 8) {
        fft_pass_dispatch<8, INV, PPT, BC>(buf, L, nbatch, Ns, tw, ts * (L / (Ns * 8)), rs, ws);
    } else if constexpr (PPT >= 16) {
        fft_pass_dispatch<16, INV, PPT, BC>(buf, L, nbatch, Ns, tw, ts * (L / (Ns * 16)), rs, ws);
    }
}

// Batched power-of-two FFT in shared memory, natural order in and out.
// ts = M / L maps the transform's twiddles onto the table of exp(-2 pi i m/M).
// PRUNE: every input is zero from index wmax on, so the leading passes
// whose radices multiply to at most L / wmax (all but the last, at most)
// are skipped and the next pass reads their result directly (see BC).
template <bool INV, int PPT, bool PRUNE = false>
__device__ __forceinline__ void fft_block(float2* buf, int L, int nbatch, const TwTab& tw, int ts,
                                          int wmax = 0) {
    const int e = __ffs(L) - 1;  // L >= 8: the plan keeps P = M/H >= 8 and M/2 >= 256
    int Ns = 1;
    if constexpr (PRUNE) {
        const int npass = fft_npass<PPT>(e);
        int i = 0;
        while (i + 1 < npass && (int64_t)wmax * Ns * fft_radix<PPT>(e, i) <= L)
            Ns *= fft_radix<PPT>(e, i++);
        if (i > 0) {
            const int R = fft_radix<PPT>(e, i);
            fft_pass_radix<INV, PPT, true>(R, buf, L, nbatch, Ns, tw, ts, false, i + 1 < npass);
            Ns *= R;
            ++i;
        }
        for (; i < npass; ++i) {
            const int R = fft_radix<PPT>(e, i);
            fft_pass_radix<INV, PPT, false>(R, buf, L, nbatch, Ns, tw, ts, i > 0, i + 1 < npass);
            Ns *= R;
        }
    } else if constexpr (PPT >= 16) {
        // The same plan as fft_radix, with the passes unrolled by kind
        // (measured faster than dispatching on the radix at run time).
        const int m = e & 3;
        const int n8 = (m == 3 || m == 1) ? 1 : 0;
        const int n4 = (m == 2 || m == 1) ? 1 : 0;
        const int npass = n8 + n4 + (e - 3 * n8 - 2 * n4) / 4;
        for (int i = 0; i < npass; ++i) {
            const bool rs = i > 0, ws = i + 1 < npass;
            if (i < n8) {
                fft_pass_dispatch<8, INV, PPT>(buf, L, nbatch, Ns, tw, ts * (L / (Ns * 8)), rs, ws);
                Ns *= 8;
            } else if (i < n8 + n4) {
                fft_pass_dispatch<4, INV, PPT>(buf, L, nbatch, Ns, tw, ts * (L / (Ns * 4)), rs, ws);
                Ns *= 4;
            } else {
                fft_pass_dispatch<16, INV, PPT>(buf, L, nbatch, Ns, tw, ts * (L / (Ns * 16)), rs,
                                                ws);
                Ns *= 16;
            }
        }
    } else {
        const int n4 = (e % 3 == 1) ? 2 : (e % 3 == 2) ? 1 : 0;
        const int npass = n4 + (e - 2 * n4) / 3;
        for (int i = 0; i < npass; ++i) {
            const bool rs = i > 0, ws = i + 1 < npass;
            if (i < n4) {
                fft_pass_dispatch<4, INV, PPT>(buf, L, nbatch, Ns, tw, ts * (L / (Ns * 4)), rs, ws);
                Ns *= 4;
            } else {
                fft_pass_dispatch<8, INV, PPT>(buf, L, nbatch, Ns, tw, ts * (L / (Ns * 8)), rs, ws);
                Ns *= 8;
            }
        }
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

// Sum of X[q] * exp2(kexp * (qf * a_over_m - C)^2) over n bins of one run:
// indices q0, q0 + dq, ... (dq = +-P) and unwrapped bin positions qf,
// qf + P, ... .  The weight is a sampled Gaussian: with u_j the argument at
// bin j and D = a P / M its step, g_{j+1} = g_j r_j, r_j = 2^{kexp (2 u_j D
// + D^2)} and r_{j+1} = r_j Q, Q = 2^{2 kexp D^2}.  Runs of 8 or more bins
// take g_j this way, re-anchored from the exact argument every 8 bins (at
// most ~3.5e-6 relative drift at a chunk's end; D <= 0.35 there, so the
// ratios stay in range); shorter runs and the remainder use one
// ex2.approx (~2^-22 relative) per bin.  LGP > 0 fixes the stride at
// compile time (dq = SIGN * 2^LGP), so the eight loads of a chunk address X
// with immediate offsets; LGP = 0 takes dq as passed.
template <int LGP, int SIGN>
__device__ __forceinline__ float2 fold_run(const float2* __restrict__ X, int q0, int dq_rt, int n,
                                           float qf, float pf, const SpecScale& sc, float cneg,
                                           float kexp) {
    const int dq = LGP ? SIGN * (1 << LGP) : dq_rt;
    float2 acc = make_float2(0.f, 0.f);
    const float2* xp = X + q0;
    int j = 0;
    if (n >= 8) {
        const float dlt = sc.dlt, q2 = sc.q2;
        for (; j + 8 <= n; j += 8) {
            const float u = fmaf(qf, sc.a_over_m, cneg);
            float g = fast_exp2(kexp * u * u);
            float r = fast_exp2(kexp * fmaf(2.f * u, dlt, dlt * dlt));
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const float2 v = xp[t * dq];
                acc.x = fmaf(v.x, g, acc.x);
                acc.y = fmaf(v.y, g, acc.y);
                g *= r;
                r *= q2;
            }
            xp += 8 * dq;
            qf += 8.f * pf;
        }
    }
    for (; j < n; ++j) {
        const float2 v = *xp;
        xp += dq;
        const float u = fmaf(qf, sc.a_over_m, cneg);
        qf += pf;
        const float g = fast_exp2(kexp * u * u);
        acc.x = fmaf(v.x, g, acc.x);
        acc.y = fmaf(v.y, g, acc.y);
    }
    return acc;
}

// Z[r] = gscale * sum over the unwrapped band [q_lo, q_hi] of the bins
// q_u = r (mod P) of X[q_u mod M] * Psi-weight; bins above M/2 are read as
// conj(X[M - q]).  The walk is split into runs that stay on one side of M/2,
// so the inner loop is branch-free.  LGP > 0: P = 2^LGP at compile time.
template <int LGP>
__device__ __forceinline__ float2 fold_residue(const float2* __restrict__ X, const SpecScale& sc,
                                               int r, int M, int Mh, int P_rt, int lgP_rt,
                                               float cneg, float kexp) {
    const int P = LGP ? (1 << LGP) : P_rt;
    const int lgP = LGP ? LGP : lgP_rt;
    int qu = sc.q_lo + ((r - sc.q_lo) & (P - 1));
    int left = qu <= sc.q_hi ? ((sc.q_hi - qu) >> lgP) + 1 : 0;
    const float pf = (float)P;
    float2 ad = make_float2(0.f, 0.f), am = make_float2(0.f, 0.f);
    while (left > 0) {
        const int q = qu & (M - 1);
        int n;
        if (q <= Mh) {
            n = min(left, ((Mh - q) >> lgP) + 1);
            const float2 t = fold_run<LGP, 1>(X, q, P, n, (float)qu, pf, sc, cneg, kexp);
            ad.x += t.x;
            ad.y += t.y;
        } else {
            n = min(left, ((M - 1 - q) >> lgP) + 1);
            const float2 t = fold_run<LGP, -1>(X, M - q, -P, n, (float)qu, pf, sc, cneg, kexp);
            am.x += t.x;
            am.y += t.y;
        }
        qu += n * P;
        left -= n;
    }
    return make_float2(sc.gscale * (ad.x + am.x), sc.gscale * (ad.y - am.y));
}

// a3 for one chunk of scales: band multiply + hop fold.  The chunk's
// (scale, residue) pairs are numbered g = c P + r; one item = 32
// consecutive g (32 residues of one scale, or 32 / P whole scales when
// P < 32), one lane each; the loop walks the unwrapped band.  Items are
// ordered by decreasing band width (scales ascend); they are dealt to warps
// in a snake order to balance the work.
template <int LGP, bool SHIFT>
__device__ __forceinline__ void fold_items(const SpecLaunch& p, const float2* __restrict__ X,
                                           float2* __restrict__ Z, int c0, int nc, int M, int P,
                                           int lgP) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int nitems = (nc * P + 31) >> 5;
    const float cneg = -p.center;
    for (int round = 0;; ++round) {
        const int it = round * nwarps + ((round & 1) ? nwarps - 1 - warp : warp);
        if (it >= nitems) break;
        const int g = (it << 5) + lane;
        const int c = g >> lgP;
        const int r = g & (P - 1);
        if (c >= nc) continue;
        const SpecScale sc = p.sc[c0 + c];
        // SHIFT: stored shifted by the band's first residue (a unit-modulus
        // phase on the inverse transform, so |W| is unchanged); the band
        // then occupies residues [0, min(P, q_hi - q_lo + 1)).
        const int zr = SHIFT ? ((r - sc.q_lo) & (P - 1)) : r;
        Z[c * P + zr] = fold_residue<LGP>(X, sc, r, M, M >> 1, P, lgP, cneg, p.kexp);
    }
}

// PRUNE: inverse FFTs skip the passes that a chunk's narrow bands leave
// trivial (plans whose narrowest folded band fits a small fraction of P).
template <int THREADS, bool PRUNE>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) spectral_segment_kernel(const SpecLaunch p) {
    constexpr int kPPT = kMaxFftPoints / THREADS;  // FFT points per thread
    extern __shared__ float2 smem[];
    const int M = p.M, Mh = M >> 1, P = p.P;
    const int ntw = (M >> 7) + 128;
    float2* T = smem;                 // two-level twiddle table, ntw entries
    float2* X = smem + ntw;           // Mh + 1 used
    float2* Z = smem + ntw + Mh + 2;  // nconc * P used
    const TwTab tab{T, T + (M >> 7)};

    const int seg = blockIdx.x, clip = blockIdx.y, grp = blockIdx.z;
    int64_t len = p.lengths ? p.lengths[clip] : p.max_len;
    len = len < 0 ? 0 : (len > p.max_len ? p.max_len : len);
    const int64_t F = (len + p.hop - 1) / p.hop;
    const int64_t k0 = (int64_t)seg * p.seg_frames;
    const int sp_begin = grp * p.group_size;
    if (k0 >= F || sp_begin >= p.n_sp) return;
    const int sp_end = min(p.n_sp, sp_begin + p.group_size);

    for (int i = threadIdx.x; i < ntw; i += blockDim.x) T[i] = __ldg(p.tw + i);

    // a1: stage the segment as M/2 complex points.
    const int64_t s0 = k0 * p.hop - p.halo;
    const float* xr = p.x + (int64_t)clip * p.ld_x;
    for (int n = threadIdx.x; n < Mh; n += blockDim.x) {
        const int64_t i0 = s0 + 2 * (int64_t)n;
        const float a = (i0 >= 0 && i0 < len) ? __ldg(xr + i0) : 0.f;
        const float b = (i0 + 1 >= 0 && i0 + 1 < len) ? __ldg(xr + i0 + 1) : 0.f;
        X[n] = make_float2(a, b);
    }
    __syncthreads();

    // a2: forward FFT of the M/2 points, twiddles exp(-2 pi i m/(M/2)) = tw[2m].
    fft_block<false, kPPT>(X, Mh, 1, tab, 2);

    // Real-input split: with Z = FFT(z), E = (Z[q] + conj Z[Mh-q])/2 and
    // O = (Z[q] - conj Z[Mh-q])/(2i) are the spectra of the even and odd
    // samples, X[q] = E + exp(-2 pi i q/M) O and X[Mh-q] = conj(E - exp(-2 pi i q/M) O).
    // Each pair (q, Mh-q) is read and written by one thread only.
    for (int q = threadIdx.x; q <= (Mh >> 1); q += blockDim.x) {
        const int qm = (Mh - q) & (Mh - 1);
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

    const int lgP = __ffs(P) - 1;
    for (int c0 = sp_begin; c0 < sp_end; c0 += p.nconc) {
        const int nc = min(p.nconc, sp_end - c0);

        // a3: the band walks of 8 or more bins per residue occur for P up to
        // M/16; those periods get a compile-time stride.
        switch (lgP) {
            case 4: fold_items<4, PRUNE>(p, X, Z, c0, nc, M, P, lgP); break;
            case 5: fold_items<5, PRUNE>(p, X, Z, c0, nc, M, P, lgP); break;
            case 6: fold_items<6, PRUNE>(p, X, Z, c0, nc, M, P, lgP); break;
            case 7: fold_items<7, PRUNE>(p, X, Z, c0, nc, M, P, lgP); break;
            case 8: fold_items<8, PRUNE>(p, X, Z, c0, nc, M, P, lgP); break;
            case 9: fold_items<9, PRUNE>(p, X, Z, c0, nc, M, P, lgP); break;
            case 10: fold_items<10, PRUNE>(p, X, Z, c0, nc, M, P, lgP); break;
            default: fold_items<0, PRUNE>(p, X, Z, c0, nc, M, P, lgP); break;
        }
        __syncthreads();

        // a4: inverse FFT of length P for every scale of the chunk; the 1/M
        // normalisation is already in gscale.  exp(+2 pi i m/P) = conj(tw[m H]).
        // With PRUNE every band of the chunk lies in its first sc[c0].wsuf
        // residues.
        fft_block<true, kPPT, PRUNE>(Z, P, nc, tab, p.hop, PRUNE ? p.sc[c0].wsuf : 0);

        // Stores.  i < 2^24, so the float quotient is off by at most one
        // and one correction step gives c = i / Fs exactly.
        const int Fs = p.seg_frames;
        const float inv_fs = 1.0f / (float)Fs;
        for (int i = threadIdx.x; i < nc * Fs; i += blockDim.x) {
            int c = (int)((float)i * inv_fs);
            int f = i - c * Fs;
            if (f < 0) {
                --c;
                f += Fs;
            } else if (f >= Fs) {
                ++c;
                f -= Fs;
            }
            const int64_t k = k0 + f;
            if (k < F) {
                const float2 w = Z[c * P + p.kp0 + f];
                const int row = p.sc[c0 + c].row;
                p.out[((int64_t)clip * p.S_total + row) * p.frames_max + k] =
                    fast_sqrt(fmaf(w.x, w.x, w.y * w.y));
            }
        }
        __syncthreads();
    }
}

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

}  // namespace

size_t spectral_smem_bytes(int M, int P, int nconc) {
    return (size_t)(spectral_twiddle_entries(M) + M / 2 + 2 + (long)nconc * P) * sizeof(float2);
}

int spectral_twiddle_entries(int M) { return (M >> 7) + 128; }

cudaError_t spectral_prepare_device() {
    cudaError_t e = cudaSuccess;
    for (const void* f : {(const void*)spectral_segment_kernel<kSpecThreadsPair, false>,
                          (const void*)spectral_segment_kernel<kSpecThreadsPair, true>,
                          (const void*)spectral_segment_kernel<kSpecThreadsSolo, false>,
                          (const void*)spectral_segment_kernel<kSpecThreadsSolo, true>})
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     227 * 1024 - 1024);
    return e;
}

cudaError_t spectral_make_twiddles(float2* d_tw, int M, cudaStream_t st) {
    twiddle_kernel<<<(spectral_twiddle_entries(M) + 255) / 256, 256, 0, st>>>(d_tw, M);
    return cudaGetLastError();
}

cudaError_t spectral_launch(const SpecLaunch& L, int threads, bool prune, int n_seg, int batch,
                            int n_groups, size_t smem, cudaStream_t st) {
    dim3 grid(n_seg, batch, n_groups);
    if (threads == kSpecThreadsSolo) {
        if (prune)
            spectral_segment_kernel<kSpecThreadsSolo, true><<<grid, kSpecThreadsSolo, smem, st>>>(L);
        else
            spectral_segment_kernel<kSpecThreadsSolo, false><<<grid, kSpecThreadsSolo, smem, st>>>(L);
    } else {
        if (prune)
            spectral_segment_kernel<kSpecThreadsPair, true><<<grid, kSpecThreadsPair, smem, st>>>(L);
        else
            spectral_segment_kernel<kSpecThreadsPair, false><<<grid, kSpecThreadsPair, smem, st>>>(L);
    }
    return cudaGetLastError();
}

}  // namespace cwth
