// Fourier-form backprojection after the row pass (Eq. fftadj, Sec. 4-5).
//
//   colfft  : second pass of the 2D FFT of every projection (along detector
//             rows v), keeping the k_v >= 0 half of the spectrum and writing
//             it plane-major: G[l][k][m]. Real projections make the planes
//             -l the conjugates of planes l (the x3 pass uses 2 Re), and the
//             column -m the conjugate of the column m read backwards in k_v:
//             one transform of each column m >= 0 gives both. Also writes
//             per-chunk bounds of the values for the gridding.
//   grid    : per k_v plane l and band of T2 rows of the oversampled x2 grid,
//             Gaussian spreading of every point (k, m) at the frequency of
//             Eq. uneqspace onto a shared-memory band of the 2x oversampled
//             plane (the adjoint USFFT's "convolution" step), then the inverse
//             FFT along x1 of each band row, cropping to n0 and dividing by
//             M1 psi1(x1). Output V[l][x1][s2] (s2 fastest).
//   colifft : inverse FFT along x2 of each (l, x1) line, crop to n1, divide
//             by M2 psi2(x2): P[l][x2][x1]. This completes the 2D USFFT of
//             the split of Eq. fftfwdsplit.
//   zusfft  : per column (x1, x2), the 1D USFFT along x3 over the planes
//             (points xi3 = l cos(phi)/Hf, identical for every column):
//             gather onto the oversampled x3 grid through a fixed tap table,
//             inverse FFT, crop, divide by M3 psi3(x3), take the real part.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace lam {
namespace {

// Pitch (complex values) of the C sequences of length n of the x2 and x3
// passes: ld = 16/C (mod 16), so that when a half-warp reads element s (and
// s + 1, ...) of C consecutive sequences (lanes c = 0..C-1 over 16/C
// consecutive s), the 8-byte slots c ld + s fall on 16 different bank pairs.
__host__ __device__ constexpr int seq_pitch(int n, int C) {
    return n + ((((16 / C) - n) % 16 + 16) % 16 == 0 ? 16 : (((16 / C) - n) % 16 + 16) % 16);
}

// ---------------------------------------------------------------- colfft
template <int E>
__global__ void __launch_bounds__(512, 2) k_colfft(const float2* __restrict__ R, float2* __restrict__ G,
                                                 float2* __restrict__ st, int k0,
                                                 int nproj, int H, int Wf, int L, int offv, FftDesc fh,
                                                 const float2* __restrict__ phv, FastDiv fC) {
    extern __shared__ float2 sm[];
    const int C = fC.d;
    const int Hf = fh.n, ld = Hf + 1, half = Wf / 2;
    const int k = k0 + blockIdx.y, m0 = blockIdx.x * C;
    // load the C columns m0 .. m0 + C - 1 (R holds m in [0, Wf/2)) of
    // projection k, zero-padded rows, into sequences of length Hf (8
    // independent loads in flight per thread)
    constexpr int U = 8;
    const int total = C * Hf;
    for (int base = threadIdx.x; base < total; base += U * blockDim.x) {
        float2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * blockDim.x;
            const int q = fC.div(idx), c = idx - q * C, r = q - offv;
            v[u] = (idx < total && r >= 0 && r < H) ? R[((size_t)k * H + r) * half + m0 + c]
                                                    : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * blockDim.x;
            const int q = fC.div(idx);
            if (idx < total) sm[(idx - q * C) * ld + q] = v[u];
        }
    }
    __syncthreads();
    fft_many<E>(sm, ld, C, fh, -1.f);
    // With S the transform of column m (slot j = k_v mod Hf):
    //   G(m, l) = phv(l) S(l),  G(-m, l) = phv(l) conj S((Hf - l) mod Hf),
    // since R(v, -m) = conj R(v, m). Write both halves (column 0 once) and
    // keep them in shared memory for the statistics: G(m, l) in slot l,
    // G(-m, l) in slot Hf - l (slot Hf is the sequence's pad). A thread reads
    // and writes only its own two slots (L = Hf/2, so Hf - l > l).
    for (int idx = threadIdx.x; idx < C * L; idx += blockDim.x) {
        const int l = fC.div(idx), c = idx - l * C, m = m0 + c;
        const float2 ph = __ldg(phv + l);
        float2 sn = sm[c * ld + (l ? Hf - l : 0)];
        sn.y = -sn.y;
        const float2 gp = cmul(sm[c * ld + l], ph), gn = cmul(sn, ph);
        float2* Gl = G + ((size_t)l * nproj + k) * Wf + half;
        Gl[m] = gp;
        if (m > 0) Gl[-m] = gn;
        sm[c * ld + l] = gp;
        sm[c * ld + Hf - l] = gn;
    }
    __syncthreads();
    // per plane, the sum and the maximum of max(|Re|, |Im|) over the block's C
    // columns m and over their C mirror columns -m: the gridding kernel's
    // bound on its fixed-point range. Layout st[k][chunk][l], chunk m0 / C
    // for the columns m >= 0 and nch + m0 / C for -m (nch = Wf / 2C).
    const int nch = half / C;
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        float sp = 0.f, mp = 0.f, sn = 0.f, mn = 0.f;
        for (int c = 0; c < C; ++c) {
            const float2 g = sm[c * ld + l];
            const float av = fmaxf(fabsf(g.x), fabsf(g.y));
            sp += av;
            mp = fmaxf(mp, av);
            if (m0 + c == 0) continue;               // column 0 is not a mirror
            const float2 h = sm[c * ld + Hf - l];
            const float an = fmaxf(fabsf(h.x), fabsf(h.y));
            sn += an;
            mn = fmaxf(mn, an);
        }
        float2* sk = st + (size_t)k * 2 * nch * L;
        sk[(size_t)(m0 / C) * L + l] = make_float2(sp, mp);
        sk[(size_t)(nch + m0 / C) * L + l] = make_float2(sn, mn);
    }
}

// ---------------------------------------------------------------- grid
struct GridArgs {
    const float2* G;
    const float2* st;      // [nproj][Wf / ch][L] (sum, max) of max(|Re|, |Im|) per chunk of ch columns
    float2* V;
    const float2* trig;
    const float* dec1;
    int nproj, Wf, Hf, n0, M1, M2, T2, ld;   // ld: row pitch of the band accumulator
    FastDiv fT2, fNR;                        // division by T2 and by the transpose's rows T2 + 2W - 1
    int ch;                                  // column chunk of the statistics
    int L, l0;                               // planes of the half spectrum; first plane of
                                             // the launch (blockIdx.y = l - l0; V is [l - l0])
    int lchunk;                              // lines per band-list chunk (>= nproj: one chunk)
    int civ_cap;                             // entries of the group table (0: none)
    float sinphi, c1, c2;  // c = -1/(4t) per axis
    float q1, q2;          // exp(2 c) per axis (gauss_taps)
    FftDesc f1;
};

// Candidate points of one line for one band: the m in [mlo, mhi] with
// Y(m) = A m + B inside the periodic band [lo + p M2, hi + p M2) for some p,
// widened by one point on each side (the tap loop decides exactly which rows
// a point reaches). Returns up to 4 disjoint intervals [ms, me], ascending.
__device__ __forceinline__ int band_intervals(float A, float B, int mlo, int mhi, float lo, float hi,
                                              int M2, int* ms, int* me) {
    if (fabsf(A) * (float)(mhi - mlo + 1) < 0.5f) {
        // the line moves less than half a cell across the band: all or nothing,
        // tested one cell wider on each side (the tap loop decides exactly)
        float y = A * 0.5f * (float)(mlo + mhi) + B;
        y -= floorf(y / M2) * M2;  // in [0, M2]
        bool in = (hi - lo + 2.f >= (float)M2);
        for (int pp = -1; pp <= 1 && !in; ++pp) {
            float yy = y + (float)pp * M2;
            in = (yy >= lo - 1.f && yy < hi + 1.f);
        }
        if (!in) return 0;
        ms[0] = mlo;
        me[0] = mhi;
        return 1;
    }
    float y0 = A * mlo + B, y1 = A * mhi + B;
    float ymin = fminf(y0, y1), ymax = fmaxf(y0, y1);
    int p0 = (int)floorf((ymin - hi) / M2), p1 = (int)ceilf((ymax - lo) / M2);
    int rs[6], re[6], nr = 0;
    const float flo = (float)mlo - 2.f, fhi = (float)mhi + 2.f;
    for (int pp = p0; pp <= p1 && nr < 6; ++pp) {
        float a = lo + (float)pp * M2, b = hi + (float)pp * M2;   // Y in [a, b)
        float ma = (A > 0) ? (a - B) / A : (b - B) / A;
        float mb = (A > 0) ? (b - B) / A : (a - B) / A;
        ma = fminf(fmaxf(ma, flo), fhi);    // keep the int conversion in range
        mb = fminf(fmaxf(mb, flo), fhi);
        int s = max(mlo, (int)floorf(ma) - 1);
        int e = min(mhi, (int)ceilf(mb) + 1);
        if (s <= e) { rs[nr] = s; re[nr] = e; ++nr; }
    }
    // sort by start (A < 0 yields them in descending order) and merge overlaps
    for (int i = 1; i < nr; ++i)
        for (int j = i; j > 0 && rs[j] < rs[j - 1]; --j) {
            int t = rs[j]; rs[j] = rs[j - 1]; rs[j - 1] = t;
            t = re[j]; re[j] = re[j - 1]; re[j - 1] = t;
        }
    int n = 0;
    for (int i = 0; i < nr; ++i) {
        if (n > 0 && rs[i] <= me[n - 1] + 1) {
            me[n - 1] = max(me[n - 1], re[i]);
        } else if (n < 4) {
            ms[n] = rs[i];
            me[n] = re[i];
            ++n;
        }
    }
    return n;
}

// The 2W Gaussian weights exp(c (d0 + j)^2), j = 0 .. N-1, of one point along
// one axis (d0 = offset of its first cell), by the factorisation of fast
// Gaussian gridding (Greengard & Lee, SIAM Rev. 2004): the ratio of
// consecutive weights is exp(c (2 (d0 + j) + 1)) = r0 q^j with q = exp(2c),
// so two exponentials and two products per weight replace N exponentials.
// Every weight and ratio stays within exp(+-c (2N)^2), far inside float range.
template <int N>
__device__ __forceinline__ void gauss_taps(float (&g)[N], float c, float q, float d0) {
    float v = __expf(c * d0 * d0);
    float r = __expf(c * fmaf(2.f, d0, 1.f));
#pragma unroll
    for (int j = 0; j < N; ++j) {
        g[j] = v;
        v *= r;
        r *= q;
    }
}

// Exclusive prefix sum of n ints in shared memory (in place), whole block;
// returns the total. Uses `tmp` (>= 32 ints).
__device__ __forceinline__ int block_scan(int* v, int n, int* tmp) {
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per, e = min(n, b + per);
    int s = 0;
    for (int i = b; i < e; ++i) s += v[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = (lane < nw) ? tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) tmp[lane] = t;   // inclusive warp totals
    }
    __syncthreads();
    int run = x - s + (warp > 0 ? tmp[warp - 1] : 0);
    const int total = tmp[nw - 1];
    for (int i = b; i < e; ++i) {
        int c = v[i];
        v[i] = run;
        run += c;
    }
    __syncthreads();
    return total;
}

// Gridding of one band of T2 rows of plane l, accumulated in fixed point.
//
// Shared-memory float atomics are emulated (about 5x slower than the native
// int32 shared atomics), so the band accumulates integers. S1 >= the sum of
// max(|Re v|, |Im v|) over the band's points and Smax >= the largest such
// value come from the column FFT's chunk statistics (every chunk of C columns
// that holds a point of a line interval); every tap is scaled by
// q = min(2^30/S1, 2^21/Smax), so no single contribution reaches 2^22 (the
// range of the float-to-int rounding below) and no cell sum can reach 2^31 (a
// cell never holds more than all the band's points). The rounding error is at
// most 1/2 per tap. Taps are rounded to integers with one FMA against
// 1.5*2^23 (the integer then sits in the low mantissa bits) instead of a
// float-to-int conversion.
//
// The band's points (every line's m-intervals) are numbered through a block
// prefix sum; each warp takes 32 consecutive points, and each thread loops
// only over the rows of its point that fall inside the band.
constexpr float kRoundMagic = 12582912.0f;   // 1.5 * 2^23
constexpr int kRoundMagicBits = 0x4B400000;  // its bit pattern

// Upper bounds on the sum and the maximum of max(|Re|, |Im|) over the band's
// points, from the column FFT's chunk statistics of every chunk that holds a
// point of a line's intervals (lines k = threadIdx.x + j blockDim; per-thread
// partial results).
// Adds the chunk statistics (sum, max) of the m-interval [ms, me] of one line
// (sl: the line's st rows, chunks ch wide, stride sstride): chunks m / ch of
// its m >= 0 part and Wf / 2ch + (-m) / ch of its m < 0 part, as k_colfft
// writes them.
__device__ __forceinline__ void interval_stats(const float2* __restrict__ sl, int sstride, int Wf, int ch,
                                               int ms, int me, float& ssum, float& smax) {
    const int nch = Wf / (2 * ch);
    // chunks c0 .. c1 of the rows from off on: eight loads in flight at a time
    auto add = [&](int c0, int c1, int off) {
        for (int c = c0; c <= c1; c += 8) {
            float2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                v[u] = (c + u <= c1) ? __ldg(sl + (size_t)(off + c + u) * sstride) : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                ssum += v[u].x;
                smax = fmaxf(smax, v[u].y);
            }
        }
    };
    if (me >= 0) add(max(ms, 0) / ch, me / ch, 0);
    if (ms < 0) add(max(1, -me) / ch, -ms / ch, nch);
}

__device__ __forceinline__ void band_stats(const float2* __restrict__ trig, int nproj, int Wf, int M2,
                                           float rho, float lo, float hi, const float2* __restrict__ st,
                                           int ch, int sstride, float& ssum, float& smax) {
    const int half = Wf / 2;
    for (int k = threadIdx.x; k < nproj; k += blockDim.x) {
        int ms[4], me[4];
        const float2 cs = __ldg(trig + k);
        const float AY = (float)M2 * cs.y / (float)Wf, BY = -(float)M2 * rho * cs.x;
        const int n = band_intervals(AY, BY, -half + 1, half - 1, lo, hi, M2, ms, me);
        const float2* sl = st + (size_t)k * (Wf / ch) * sstride;
        for (int i = 0; i < n; ++i) interval_stats(sl, sstride, Wf, ch, ms[i], me[i], ssum, smax);
    }
}

// The band's points of the lines k0 .. k0 + nk - 1, as a compact list of
// non-empty m-intervals: every line k contributes the m in [-Wf/2 + 1,
// Wf/2 - 1] with Y(m) inside [lo, hi) (mod M2) (band_intervals). ioff[i] =
// first point number of interval i, ikm[i] = (k << 13) | (m start + 4096),
// ioff[nintv] = total. lcnt is [nk] scratch; nk <= 4 blockDim. With st, also
// the band_stats bounds of these lines. Whole block; returns the number of
// points.
__device__ __forceinline__ int band_list(const float2* __restrict__ trig, int k0, int nproj, int Wf, int M2,
                                         float rho, float lo, float hi, int* ioff, int* ikm,
                                         int* lcnt, int* scan_tmp, int& nintv_out,
                                         const float2* __restrict__ st = nullptr, int ch = 1,
                                         int sstride = 0, float* bsum = nullptr,
                                         float* bmax = nullptr, int* civ = nullptr,
                                         int civ_cap = 0) {
    const int half = Wf / 2;
    const int per = (nproj + blockDim.x - 1) / blockDim.x;   // lines per thread (<= 4)
    int ms[4][4], me[4][4], nint[4];
    float ssum = 0.f, smax = 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        nint[t] = 0;
        const int kl = threadIdx.x * per + t, k = k0 + kl;
        if (t < per && kl < nproj) {
            const float2 cs = __ldg(trig + k);
            const float AY = (float)M2 * cs.y / (float)Wf, BY = -(float)M2 * rho * cs.x;
            nint[t] = band_intervals(AY, BY, -half + 1, half - 1, lo, hi, M2, ms[t], me[t]);
            lcnt[kl] = nint[t];
            if (st) {
                // every chunk that holds a point of the line's intervals: an
                // upper bound on the band's sum and maximum
                const float2* sl = st + (size_t)k * (Wf / ch) * sstride;
                for (int i = 0; i < nint[t]; ++i)
                    interval_stats(sl, sstride, Wf, ch, ms[t][i], me[t][i], ssum, smax);
            }
        }
    }
    if (bsum) { *bsum = ssum; *bmax = smax; }
    __syncthreads();
    const int nintv = block_scan(lcnt, nproj, scan_tmp);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int kl = threadIdx.x * per + t, k = k0 + kl;
        if (t < per && kl < nproj) {
            const int o = lcnt[kl];
            for (int i = 0; i < nint[t]; ++i) {
                ioff[o + i] = me[t][i] - ms[t][i] + 1;
                ikm[o + i] = (k << 13) | (ms[t][i] + 4096);
            }
        }
    }
    __syncthreads();
    const int total = block_scan(ioff, nintv, scan_tmp);
    if (threadIdx.x == 0) ioff[nintv] = total;
    __syncthreads();
    if (civ && total <= 32 * civ_cap) {
        // group table: civ[g] = the interval that holds point 32 g
        for (int i = threadIdx.x; i < nintv; i += blockDim.x)
            for (int g = (ioff[i] + 31) >> 5; 32 * g < ioff[i + 1]; ++g) civ[g] = i;
        __syncthreads();
    }
    nintv_out = nintv;
    return total;
}

// Point number base + lane of a band list -> (line k, m); the interval of
// `base` (a multiple of 32) comes from the group table civ when there is one,
// else lane 0 finds it by bisection; every lane steps forward from it. Must be
// called by the whole warp; false for lanes past the end.
__device__ __forceinline__ bool band_locate(const int* ioff, const int* ikm, int nintv, int total,
                                            int base, int lane, int& k, int& m,
                                            const int* civ = nullptr) {
    int iv = 0;
    if (civ) {
        iv = civ[base >> 5];
    } else {
        if (lane == 0) {
            int a0 = 0, b0 = nintv;   // ioff[a0] <= base < ioff[b0]
            while (b0 - a0 > 1) {
                const int mid = (a0 + b0) >> 1;
                if (ioff[mid] <= base) a0 = mid; else b0 = mid;
            }
            iv = a0;
        }
        iv = __shfl_sync(0xffffffffu, iv, 0);
    }
    const int p = base + lane;
    if (p >= total) return false;
    while (ioff[iv + 1] <= p) ++iv;
    const int km = ikm[iv];
    k = km >> 13;
    m = (km & 8191) - 4096 + (p - ioff[iv]);
    return true;
}

// Shared-memory int32 reduction at a byte offset known at compile time.
template <int OFF>
__device__ __forceinline__ void red_s32(uint32_t addr, int v) {
    asm volatile("red.shared.add.s32 [%0+%2], %1;" ::"r"(addr), "r"(v), "n"(OFF) : "memory");
}
__device__ __forceinline__ int round_to_int(float a, float b) {
    return __float_as_int(fmaf(a, b, kRoundMagic)) - kRoundMagicBits;
}
// The 2W taps of one point row: consecutive cells starting at byte address bre
// (real plane) and bim (imaginary plane).
template <int C, int N>
struct TapRow {
    static __device__ __forceinline__ void run(uint32_t bre, uint32_t bim, float vr, float vi,
                                               const float (&gx)[N]) {
        red_s32<4 * C>(bre, round_to_int(vr, gx[C]));
        red_s32<4 * C>(bim, round_to_int(vi, gx[C]));
        TapRow<C + 1, N>::run(bre, bim, vr, vi, gx);
    }
};
template <int N>
struct TapRow<N, N> {
    static __device__ __forceinline__ void run(uint32_t, uint32_t, float, float, const float (&)[N]) {}
};

template <int E, int W>
__global__ void __launch_bounds__(1024, 1) k_grid(GridArgs a) {
    extern __shared__ float smf[];
    const int M1 = a.M1, M2 = a.M2, T2 = a.T2, ld = a.ld;
    const int nproj = a.nproj;
    float* Ure = smf;                       // [T2][ld] int32 during accumulation, then float
    float* Uim = smf + (size_t)T2 * ld;
    // compact list of the band's non-empty m-intervals: ioff[i] = first point
    // number, ikm[i] = (line << 13) | (m start + 4096); ioff[n] = total
    // (for one chunk of CH lines at a time when the lines do not fit at once)
    const int CH = min(a.lchunk, nproj);
    int* ioff = reinterpret_cast<int*>(Uim + (size_t)T2 * ld);
    int* ikm = ioff + 4 * CH + 1;
    int* lcnt = ikm + 4 * CH;               // [CH] per-line interval counts (scan)
    int* civ = lcnt + CH;                   // [civ_cap] group table of the band list
    __shared__ float red_s[32], red_m[32];
    __shared__ int scan_tmp[32];
    const int band = blockIdx.x, l = a.l0 + blockIdx.y;
    const int s20 = band * T2;
    int* Ui_re = reinterpret_cast<int*>(Ure);
    int* Ui_im = reinterpret_cast<int*>(Uim);
    for (int i = threadIdx.x; i < T2 * ld; i += blockDim.x) { Ui_re[i] = 0; Ui_im[i] = 0; }

    const float rho = (float)l * a.sinphi / (float)a.Hf;   // k_v sin(phi)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int half = a.Wf / 2;
    // points whose 2W rows reach the band: Y in [s20 - W, s20 + T2 + W - 1);
    // the chunk statistics of the column pass bound the band's values
    int nintv = 0, total = 0;
    float lsum = 0.f, lmax = 0.f;
    const float lo = (float)(s20 - W), hi = (float)(s20 + T2 + W - 1);
    if (CH >= nproj)
        total = band_list(a.trig, 0, nproj, a.Wf, M2, rho, lo, hi, ioff, ikm, lcnt, scan_tmp, nintv,
                          a.st + l, a.ch, a.L, &lsum, &lmax, civ, a.civ_cap);
    else   // the scale needs every line's bound before any chunk is spread
        band_stats(a.trig, nproj, a.Wf, M2, rho, lo, hi, a.st + l, a.ch, a.L, lsum, lmax);

    const float2* Gl = a.G + (size_t)l * nproj * a.Wf;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    }
    if (lane == 0) { red_s[warp] = lsum; red_m[warp] = lmax; }
    __syncthreads();
    float S1 = 0.f, Smax = 0.f;
    for (int i = 0; i < nwarps; ++i) { S1 += red_s[i]; Smax = fmaxf(Smax, red_m[i]); }
    // the sums run in float: 1 % headroom covers their rounding
    S1 *= 1.01f;
    const float q = (S1 > 0.f) ? fminf(1073741824.0f / S1, 2097152.0f / Smax) : 1.0f;

    // spread, chunk of lines by chunk of lines
    const uint32_t s_re = (uint32_t)__cvta_generic_to_shared(Ui_re);
    const uint32_t plane_bytes = 4u * (uint32_t)(T2 * ld);
    for (int k0 = 0; k0 < nproj; k0 += CH) {
    if (CH < nproj) {
        __syncthreads();   // every warp is done with the previous chunk's list
        total = band_list(a.trig, k0, min(CH, nproj - k0), a.Wf, M2, rho, lo, hi, ioff, ikm, lcnt,
                          scan_tmp, nintv, nullptr, 1, 0, nullptr, nullptr, civ, a.civ_cap);
    }
    const int* civ_t = (total <= 32 * a.civ_cap) ? civ : nullptr;
    for (int base = warp * 32; base < total; base += nwarps * 32) {
        int k, m;
        if (!band_locate(ioff, ikm, nintv, total, base, lane, k, m, civ_t)) continue;
        float2 g = Gl[(size_t)k * a.Wf + (m + half)];
        g.x *= q;
        g.y *= q;
        const float2 cs = __ldg(a.trig + k);
        // Eq. uneqspace in grid cells: X = M1 (m/Wf cos t + rho sin t),
        //                               Y = M2 (m/Wf sin t - rho cos t)
        const float AX = (float)M1 * cs.x / (float)a.Wf, BX = (float)M1 * rho * cs.y;
        const float AY = (float)M2 * cs.y / (float)a.Wf, BY = -(float)M2 * rho * cs.x;
        float X = fmaf(AX, (float)m, BX);
        const float Y = fmaf(AY, (float)m, BY);
        X -= floorf(X / M1) * M1;          // X in [0, M1]
        const float fx = floorf(X), fy = floorf(Y);
        float gx[2 * W];
        const int sx0 = (int)fx - W + 1;
        gauss_taps(gx, a.c1, a.q1, fx - W + 1 - X);
        const bool wraps = sx0 < 0 || sx0 + 2 * W > M1;   // rare: within W of the grid edge
        // rows of the point: s2 = fy - W + 1 + jy; band row rr = s2 - s20 (mod M2)
        int r0 = (int)fy - W + 1 - s20;                 // in (-2 M2 - W, M2)
        r0 += (r0 < 0) ? M2 : 0;
        r0 += (r0 < 0) ? M2 : 0;
        r0 -= (r0 >= M2) ? M2 : 0;                      // now in [0, M2); 2W <= M2
        float gyv[2 * W];
        gauss_taps(gyv, a.c2, a.q2, fy - W + 1 - Y);
#pragma unroll
        for (int jy = 0; jy < 2 * W; ++jy) {
            int rr = r0 + jy;
            rr -= (rr >= M2) ? M2 : 0;
            if ((unsigned)rr >= (unsigned)T2) continue;
            const float gy = gyv[jy];
            const float vr = g.x * gy, vi = g.y * gy;
            const uint32_t row = s_re + 4u * (uint32_t)(rr * ld);
            if (!wraps) {
                const uint32_t b = row + 4u * (uint32_t)sx0;
                TapRow<0, 2 * W>::run(b, b + plane_bytes, vr, vi, gx);
            } else {
#pragma unroll
                for (int c = 0; c < 2 * W; ++c) {
                    int s1 = sx0 + c;
                    s1 += (s1 < 0) ? M1 : 0;
                    s1 -= (s1 >= M1) ? M1 : 0;
                    red_s32<0>(row + 4u * (uint32_t)s1, round_to_int(vr, gx[c]));
                    red_s32<0>(row + plane_bytes + 4u * (uint32_t)s1, round_to_int(vi, gx[c]));
                }
            }
        }
    }
    }   // chunks of lines
    __syncthreads();
    // back to float
    const float inv_q = 1.0f / q;
    for (int i = threadIdx.x; i < T2 * ld; i += blockDim.x) {
        Ure[i] = (float)Ui_re[i] * inv_q;
        Uim[i] = (float)Ui_im[i] * inv_q;
    }
    __syncthreads();
    // inverse FFT of each band row along x1 (sum_s U(s) exp(+2 pi i x s/M1))
    fft_many_planar<E>(Ure, Uim, ld, T2, a.f1, +1.f, true);
    // crop x1 in [-n0/2, n0/2), deconvolve, write V[l][i0][s2] (s2 fastest)
    const int n0 = a.n0;
    for (int idx = threadIdx.x; idx < T2 * n0; idx += blockDim.x) {
        const int i0 = a.fT2.div(idx), rr = idx - i0 * T2;
        int s1 = i0 - n0 / 2;
        s1 += (s1 < 0) ? M1 : 0;
        s1 = fft_planar_pos<E>(a.f1, s1, true);
        const float dd = __ldg(a.dec1 + i0);
        a.V[((size_t)blockIdx.y * n0 + i0) * M2 + s20 + rr] = make_float2(Ure[rr * ld + s1] * dd, Uim[rr * ld + s1] * dd);
    }
}

// ---------------------------------------------------------------- colifft
template <int E, int MT>
__global__ void __launch_bounds__(MT, MT > 512 ? 1 : 2) k_colifft(const float2* __restrict__ V, float2* __restrict__ P,
                                                  int n0, int n1, FftDesc f2,
                                                  const float* __restrict__ dec2, FastDiv fC, FastDiv fM2,
                                                  int l0) {
    extern __shared__ float2 sm[];
    const int C = fC.d;
    const int M2 = f2.n, ld = seq_pitch(M2, C);
    const int lv = blockIdx.y, l = l0 + lv, i00 = blockIdx.x * C;   // V holds planes [l0, ...)
    constexpr int U = 8;
    const int total = C * M2;
    for (int base = threadIdx.x; base < total; base += U * blockDim.x) {
        float2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * blockDim.x;
            const int q = fM2.div(idx), i0 = i00 + q;
            v[u] = (idx < total && i0 < n0) ? V[((size_t)lv * n0 + i0) * M2 + (idx - q * M2)] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * blockDim.x;
            const int q = fM2.div(idx);
            if (idx < total) sm[q * ld + (idx - q * M2)] = v[u];
        }
    }
    __syncthreads();
    fft_many<E>(sm, ld, C, f2, +1.f);
    for (int idx = threadIdx.x; idx < C * n1; idx += blockDim.x) {
        const int i1 = fC.div(idx), c = idx - i1 * C, i0 = i00 + c;
        if (i0 >= n0) continue;
        int s2 = i1 - n1 / 2;
        s2 += (s2 < 0) ? M2 : 0;
        P[((size_t)l * n1 + i1) * n0 + i0] = cscale(sm[c * ld + s2], __ldg(dec2 + i1));
    }
}

// ---------------------------------------------------------------- zusfft
// Row pitch (complex values) of the block's plane values [L][C]: C + 2 keeps
// 16-byte rows and an odd number of 16-byte units per row, so the 16-byte
// loads of a warp's consecutive planes spread over all banks.
__host__ __device__ constexpr int zus_pitch(int C) { return C >= 2 ? C + 2 : 1; }

template <int E, int CB>
__global__ void __launch_bounds__(512, 2) k_zusfft(const float2* __restrict__ P, float* __restrict__ vol,
                                                 int L, int n0, int n1, int n2, FftDesc f3,
                                                 const int* __restrict__ zoff, const int* __restrict__ zl,
                                                 const float* __restrict__ zw,
                                                 const int2* __restrict__ zrange, const float* __restrict__ zwt,
                                                 const float* __restrict__ dec3, int i10) {
    extern __shared__ float2 sm[];
    constexpr int C = CB, PP = zus_pitch(CB);
    const int M3 = f3.n, ld = seq_pitch(M3, C);
    const int i1 = i10 + blockIdx.y, i00 = blockIdx.x * C;
    float2* Pl = sm;                    // [L][PP]
    float2* U = sm + (size_t)L * PP;    // [C][M3 + 1]
    constexpr int NB = 8;
    const int total = C * L;
    for (int base = threadIdx.x; base < total; base += NB * blockDim.x) {
        float2 v[NB];
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int idx = base + u * blockDim.x;
            const int i0 = i00 + idx % C;
            v[u] = (idx < total && i0 < n0) ? P[((size_t)(idx / C) * n1 + i1) * n0 + i0] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int idx = base + u * blockDim.x;
            if (idx < total) Pl[(idx / C) * PP + idx % C] = v[u];
        }
    }
    __syncthreads();
    // gather onto the oversampled x3 grid: a thread per cell for all C
    // columns, so every tap's (plane, weight) entry is read once per block
    for (int s3 = threadIdx.x; s3 < M3; s3 += blockDim.x) {
        float2 acc[C];
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] = make_float2(0.f, 0.f);
        // taps: planes l0 .. l0 + n - 1 with weights zwt[t][s3] (coalesced
        // across the warp's cells), else the CSR list of the cell
        int t0, n, l0 = 0;
        if (zrange) {
            const int2 r = __ldg(zrange + s3);
            t0 = 0;
            n = r.y;
            l0 = r.x;
        } else {
            t0 = __ldg(zoff + s3);
            n = __ldg(zoff + s3 + 1) - t0;
        }
        for (int t = 0; t < n; ++t) {
            const float wgt = zrange ? __ldg(zwt + (size_t)t * M3 + s3) : __ldg(zw + t0 + t);
            const float2* row = Pl + (zrange ? l0 + t : __ldg(zl + t0 + t)) * PP;
            if constexpr (C >= 2) {
#pragma unroll
                for (int j = 0; j < C / 2; ++j) {
                    const float4 v = reinterpret_cast<const float4*>(row)[j];
                    acc[2 * j].x = fmaf(wgt, v.x, acc[2 * j].x);
                    acc[2 * j].y = fmaf(wgt, v.y, acc[2 * j].y);
                    acc[2 * j + 1].x = fmaf(wgt, v.z, acc[2 * j + 1].x);
                    acc[2 * j + 1].y = fmaf(wgt, v.w, acc[2 * j + 1].y);
                }
            } else {
                const float2 v = row[0];
                acc[0].x = fmaf(wgt, v.x, acc[0].x);
                acc[0].y = fmaf(wgt, v.y, acc[0].y);
            }
        }
#pragma unroll
        for (int c = 0; c < C; ++c) U[c * ld + s3] = acc[c];
    }
    __syncthreads();
    fft_many<E>(U, ld, C, f3, +1.f);
    for (int idx = threadIdx.x; idx < C * n2; idx += blockDim.x) {
        int c = idx % C, i2 = idx / C, i0 = i00 + c;
        if (i0 >= n0) continue;
        int s3 = i2 - n2 / 2;
        s3 += (s3 < 0) ? M3 : 0;
        vol[((size_t)i2 * n1 + i1) * n0 + i0] = U[c * ld + s3].x * __ldg(dec3 + i2);
    }
}

template <typename K>
void set_smem(K kern, size_t smem) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Threads of a block that transforms C sequences with fft_many: a warp per
// 512-point sequence, a pair of warps per 1024-point one (the register-resident
// paths), else f.t per sequence; 128 to 512.
int fft_block_threads(const FftDesc& f, int C) {
    const int per = (f.e == 8 && f.n == 512) ? 32 : (f.e == 8 && f.n == 1024) ? 64 : f.t;
    return std::min(f.t > 512 ? 1024 : 512, std::max(128, C * per));
}

// Kernels whose blocks hold at most 512 threads refuse sequences that need more.
int refuse_long_fft(lamino_plan_t p, const FftDesc& f, const char* what) {
    return fail(p, LAMINO_EUNSUPPORTED, "%s supports FFT lengths up to 4096 (2^k) or 6144 (3*2^k), "
                "not %d", what, f.n);
}


// ============================================================================
// Transpose of the Fourier-form backprojection (the forward operator of
// Eq. fftfwd in this discretisation). Every stage is the conjugate transpose
// of its forward stage, in reverse order; the gridding becomes interpolation
// (a gather: no atomics), the inverse FFTs become forward FFTs and vice versa.
// ============================================================================

// x3: vol column -> x dec3, embed, forward FFT, gather each plane's 2wz taps.
template <int E>
__global__ void __launch_bounds__(512, 2) k_zusfft_t(const float* __restrict__ vol, float2* __restrict__ Pt,
                                                     int L, int n0, int n1, int n2, FftDesc f3,
                                                     const int2* __restrict__ ztap, int wz,
                                                     const float* __restrict__ dec3, FastDiv fC) {
    extern __shared__ float2 sm[];
    const int C = fC.d;
    const int M3 = f3.n, ld = M3 + 1;
    const int i1 = blockIdx.y, i00 = blockIdx.x * C;
    for (int i = threadIdx.x; i < C * ld; i += blockDim.x) sm[i] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int idx = threadIdx.x; idx < C * n2; idx += blockDim.x) {
        const int i2 = fC.div(idx), c = idx - i2 * C, i0 = i00 + c;
        int s3 = i2 - n2 / 2;
        s3 += (s3 < 0) ? M3 : 0;
        const float v = (i0 < n0) ? vol[((size_t)i2 * n1 + i1) * n0 + i0] * __ldg(dec3 + i2) : 0.f;
        sm[c * ld + s3] = make_float2(v, 0.f);
    }
    __syncthreads();
    fft_many<E>(sm, ld, C, f3, -1.f);
    for (int idx = threadIdx.x; idx < C * L; idx += blockDim.x) {
        const int l = fC.div(idx), c = idx - l * C, i0 = i00 + c;
        if (i0 >= n0) continue;
        float2 acc = make_float2(0.f, 0.f);
        for (int t = 0; t < 2 * wz; ++t) {
            const int2 tp = __ldg(ztap + (size_t)l * 2 * wz + t);
            const float w = __int_as_float(tp.y);
            const float2 u = sm[c * ld + tp.x];
            acc.x = fmaf(w, u.x, acc.x);
            acc.y = fmaf(w, u.y, acc.y);
        }
        Pt[((size_t)l * n1 + i1) * n0 + i0] = acc;
    }
}

// x2: column of plane l at x1 -> x dec2, embed, forward FFT -> Vt[l][x1][s2].
template <int E>
__global__ void __launch_bounds__(512, 2) k_colifft_t(const float2* __restrict__ Pt, float2* __restrict__ Vt,
                                                      int n0, int n1, FftDesc f2,
                                                      const float* __restrict__ dec2, FastDiv fC, FastDiv fM2,
                                                      int l0) {
    extern __shared__ float2 sm[];
    const int C = fC.d;
    const int M2 = f2.n, ld = M2 + 1;
    const int lv = blockIdx.y, l = l0 + lv, i00 = blockIdx.x * C;   // Vt holds planes [l0, ...)
    for (int i = threadIdx.x; i < C * ld; i += blockDim.x) sm[i] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int idx = threadIdx.x; idx < C * n1; idx += blockDim.x) {
        const int i1 = fC.div(idx), c = idx - i1 * C, i0 = i00 + c;
        int s2 = i1 - n1 / 2;
        s2 += (s2 < 0) ? M2 : 0;
        sm[c * ld + s2] = (i0 < n0) ? cscale(Pt[((size_t)l * n1 + i1) * n0 + i0], __ldg(dec2 + i1))
                                    : make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft_many<E>(sm, ld, C, f2, -1.f);
    for (int idx = threadIdx.x; idx < C * M2; idx += blockDim.x) {
        const int c = fM2.div(idx), s = idx - c * M2, i0 = i00 + c;
        if (i0 < n0) Vt[((size_t)lv * n0 + i0) * M2 + s] = sm[c * ld + s];
    }
}

// Gridding transpose: CTA = (plane l, band of T2 rows) + a halo of 2W - 1 rows
// below it. Each row s2: x dec1, embed along s1, forward FFT; then every point
// whose first tap row lies in the band (each point has exactly one such band)
// gathers its (2W)^2 taps.
template <int E, int W>
__global__ void __launch_bounds__(512, 1) k_grid_t(GridArgs a, const float2* __restrict__ Vt,
                                                   float2* __restrict__ Gt) {
    extern __shared__ float2 smx[];
    const int M1 = a.M1, M2 = a.M2, T2 = a.T2, ld = a.ld, NR = T2 + 2 * W - 1;
    const int nproj = a.nproj, n0 = a.n0;
    float2* X = smx;                                           // [NR][ld]
    const int CH = min(a.lchunk, nproj);                       // lines per band-list chunk
    int* ioff = reinterpret_cast<int*>(X + (size_t)NR * ld);
    int* ikm = ioff + 4 * CH + 1;
    int* lcnt = ikm + 4 * CH;
    __shared__ int scan_tmp[32];
    const int band = blockIdx.x, l = a.l0 + blockIdx.y, s20 = band * T2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int half = a.Wf / 2;
    for (int i = threadIdx.x; i < NR * ld; i += blockDim.x) X[i] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int idx = threadIdx.x; idx < NR * n0; idx += blockDim.x) {
        const int i0 = a.fNR.div(idx), rr = idx - i0 * NR;
        int s2 = s20 + rr;
        s2 -= (s2 >= M2) ? M2 : 0;
        int s1 = i0 - n0 / 2;
        s1 += (s1 < 0) ? M1 : 0;
        X[rr * ld + s1] = cscale(Vt[((size_t)blockIdx.y * n0 + i0) * M2 + s2], __ldg(a.dec1 + i0));
    }
    __syncthreads();
    fft_many<E>(X, ld, NR, a.f1, -1.f);

    const float rho = (float)l * a.sinphi / (float)a.Hf;
    // owners: first tap row fy - W + 1 in [s20, s20 + T2), i.e. Y in [s20 + W - 1, s20 + T2 + W - 1)
    float2* Gl = Gt + (size_t)l * nproj * a.Wf;
    if (band == 0)   // the dropped Nyquist column m = -Wf/2
        for (int k = threadIdx.x; k < nproj; k += blockDim.x) Gl[(size_t)k * a.Wf] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < nproj; k0 += CH) {
    if (k0 > 0) __syncthreads();   // every warp is done with the previous chunk's list
    int nintv = 0;
    const int total = band_list(a.trig, k0, min(CH, nproj - k0), a.Wf, M2, rho, (float)(s20 + W - 1),
                                (float)(s20 + T2 + W - 1), ioff, ikm, lcnt, scan_tmp, nintv);
    for (int base = warp * 32; base < total; base += nwarps * 32) {
        int k, m;
        if (!band_locate(ioff, ikm, nintv, total, base, lane, k, m)) continue;
        const float2 cs = __ldg(a.trig + k);
        const float AX = (float)M1 * cs.x / (float)a.Wf, BX = (float)M1 * rho * cs.y;
        const float AY = (float)M2 * cs.y / (float)a.Wf, BY = -(float)M2 * rho * cs.x;
        float X0 = fmaf(AX, (float)m, BX);
        const float Y = fmaf(AY, (float)m, BY);
        X0 -= floorf(X0 / M1) * M1;
        const float fx = floorf(X0), fy = floorf(Y);
        int r0 = (int)fy - W + 1 - s20;
        r0 += (r0 < 0) ? M2 : 0;
        r0 += (r0 < 0) ? M2 : 0;
        r0 -= (r0 >= M2) ? M2 : 0;
        if (r0 >= T2) continue;                 // owned by another band
        float gx[2 * W], gyv[2 * W];
        int col[2 * W];
        const int sx0 = (int)fx - W + 1;
        gauss_taps(gx, a.c1, a.q1, fx - W + 1 - X0);
        gauss_taps(gyv, a.c2, a.q2, fy - W + 1 - Y);
#pragma unroll
        for (int c = 0; c < 2 * W; ++c) {
            int s1 = sx0 + c;
            s1 += (s1 < 0) ? M1 : 0;
            s1 -= (s1 >= M1) ? M1 : 0;
            col[c] = s1;
        }
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int jy = 0; jy < 2 * W; ++jy) {
            const float gy = gyv[jy];
            const float2* row = X + (size_t)(r0 + jy) * ld;
            float2 racc = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < 2 * W; ++c) {
                const float2 u = row[col[c]];
                racc.x = fmaf(gx[c], u.x, racc.x);
                racc.y = fmaf(gx[c], u.y, racc.y);
            }
            acc.x = fmaf(gy, racc.x, acc.x);
            acc.y = fmaf(gy, racc.y, acc.y);
        }
        Gl[(size_t)k * a.Wf + (m + half)] = acc;
    }
    }   // chunks of lines
}

// Column pass transpose: plane values of one (projection, column) x conj(phase)
// -> inverse FFT over l (only l < Hf/2 non-zero) -> detector rows.
template <int E>
__global__ void __launch_bounds__(512, 2) k_colfft_t(const float2* __restrict__ Gt, float2* __restrict__ Rt,
                                                     int nproj, int H, int Wf, int L, int offv, FftDesc fh,
                                                     const float2* __restrict__ phv, FastDiv fC) {
    extern __shared__ float2 sm[];
    const int C = fC.d;
    const int Hf = fh.n, ld = Hf + 1;
    const int k = blockIdx.y, m0 = blockIdx.x * C;
    for (int idx = threadIdx.x; idx < C * Hf; idx += blockDim.x) {
        const int l = fC.div(idx), c = idx - l * C;
        float2 v = make_float2(0.f, 0.f);
        if (l < L) {
            float2 ph = __ldg(phv + l);
            ph.y = -ph.y;
            v = cmul(Gt[((size_t)l * nproj + k) * Wf + m0 + c], ph);
        }
        sm[c * ld + l] = v;
    }
    __syncthreads();
    fft_many<E>(sm, ld, C, fh, +1.f);
    for (int idx = threadIdx.x; idx < C * H; idx += blockDim.x) {
        const int r = fC.div(idx), c = idx - r * C;
        Rt[((size_t)k * H + r) * Wf + m0 + c] = sm[c * ld + r + offv];
    }
}

// Row pass transpose: x conj(phase), inverse FFT over m, real part at the
// detector columns, times nproj/pi (lamino_project omits the pi/nproj weight).
template <int E>
__global__ void __launch_bounds__(512, 2) k_rowfft_t(const float2* __restrict__ Rt, float* __restrict__ d,
                                                     long nrows, int W, int offu, FftDesc ff,
                                                     const float2* __restrict__ phu, float unscale,
                                                     int rows_per_block) {
    extern __shared__ float2 sm[];
    const int Nf = ff.n, T = ff.t;
    const int seq = threadIdx.x / T, tid = threadIdx.x % T;
    const long row = (long)blockIdx.x * rows_per_block + seq;
    const bool active = seq < rows_per_block && row < nrows;
    float2* x = sm + (size_t)min(seq, rows_per_block - 1) * Nf;
    if (active)
        for (int mi = tid; mi < Nf; mi += T) {
            float2 ph = __ldg(phu + mi);
            ph.y = -ph.y;
            int m = mi - Nf / 2;
            m += (m < 0) ? Nf : 0;
            x[m] = cmul(Rt[(size_t)row * Nf + mi], ph);
        }
    __syncthreads();
    fft_run<E>(x, ff, tid, active, +1.f);
    if (active)
        for (int j = tid; j < W; j += T) d[(size_t)row * W + j] = x[j + offu].x * unscale;
}

int largest_pow2_divisor_upto(int n, int cap) {
    int c = 1;
    while (c * 2 <= cap && n % (c * 2) == 0) c *= 2;
    return c;
}

template <int E, int W>
void launch_grid_kernel(const GridArgs& a, dim3 grid, int threads, size_t smem, cudaStream_t s) {
    set_smem(k_grid<E, W>, smem);
    k_grid<E, W><<<grid, threads, smem, s>>>(a);
}

template <int E>
int dispatch_grid_w(int w, const GridArgs& a, dim3 grid, int threads, size_t smem, cudaStream_t s) {
    switch (w) {
        case 2: launch_grid_kernel<E, 2>(a, grid, threads, smem, s); break;
        case 3: launch_grid_kernel<E, 3>(a, grid, threads, smem, s); break;
        case 4: launch_grid_kernel<E, 4>(a, grid, threads, smem, s); break;
        case 5: launch_grid_kernel<E, 5>(a, grid, threads, smem, s); break;
        case 6: launch_grid_kernel<E, 6>(a, grid, threads, smem, s); break;
        case 7: launch_grid_kernel<E, 7>(a, grid, threads, smem, s); break;
        default: launch_grid_kernel<E, 8>(a, grid, threads, smem, s); break;
    }
    return 0;
}

}  // namespace

// Columns per block of the column FFT (a power of two dividing Wf/2, at most
// 16, with the block's sequences within 100 KB of shared memory); also the
// chunk of the statistics it writes for the gridding kernel.
int colfft_chunk(lamino_plan_t p) {
    int C = largest_pow2_divisor_upto(p->Wf / 2, 16);
    while (C > 1 && (size_t)C * (p->Hf + 1) * sizeof(float2) > 100 * 1024) C /= 2;
    return C;
}

// Planes per F3-F5 chunk: the plan's z_chunk, or every plane (no chunking).
int plane_chunk(lamino_plan_t p) {
    return (p->z_chunk > 0 && p->z_chunk < p->L) ? p->z_chunk : p->L;
}

// Workspace sizes (bytes) of A and B for the layouts described at FourierBufs.
int fourier_workspace(lamino_plan_t p, size_t* a_bytes, size_t* b_bytes) {
    const int zc = plane_chunk(p);
    size_t R = (size_t)p->nproj * p->H * p->Wf;    // row spectra
    size_t G = (size_t)p->L * p->nproj * p->Wf;    // half spectra, plane-major
    G += G / colfft_chunk(p);                      // + chunk statistics (sum, max)
    size_t P = (size_t)p->L * p->n1 * p->n0;       // deconvolved planes
    size_t V = (size_t)zc * p->n0 * p->M2;         // x1-pass planes of one chunk
    if (zc >= p->L) {
        *a_bytes = sizeof(float2) * std::max(R, V);
        *b_bytes = sizeof(float2) * std::max(G, P);
    } else {
        *a_bytes = sizeof(float2) * std::max(R, P + V);
        *b_bytes = sizeof(float2) * G;
    }
    return LAMINO_OK;
}

FourierBufs fourier_bufs(lamino_plan_t p, void* a, void* b) {
    FourierBufs f;
    f.CH = colfft_chunk(p);
    f.zc = plane_chunk(p);
    f.R = (float2*)a;                                        // [nproj][H][Wf/2] (Rt: [nproj][H][Wf])
    f.G = (float2*)b;                                        // [L][nproj][Wf]
    f.st = f.G + (size_t)p->L * p->nproj * p->Wf;           // [nproj][Wf/CH][L]
    if (f.zc >= p->L) {
        f.V = (float2*)a;                                    // [L][n0][M2]  (R is dead by then)
        f.P = (float2*)b;                                    // [L][n1][n0]  (G is dead by then)
    } else {
        f.P = (float2*)a;                                    // [L][n1][n0]  (R is dead by then)
        f.V = f.P + (size_t)p->L * p->n1 * p->n0;            // [zc][n0][M2]
    }
    return f;
}

int launch_colfft(lamino_plan_t p, const FourierBufs& fb, int k0, int k1, cudaStream_t s) {
    if (k1 <= k0) return LAMINO_OK;
    // column FFT (+ chunk statistics for the gridding bound, after G in B)
    const FftDesc& f = p->fHf;
    if (f.t > 512) return refuse_long_fft(p, f, "the column FFT (padded detector height)");
    const int C = fb.CH;
    size_t smem = (size_t)C * (f.n + 1) * sizeof(float2);
    dim3 grid(p->Wf / 2 / C, k1 - k0);         // the columns m >= 0 (R holds those)
    int threads = fft_block_threads(f, C);
    ProfScope prof(p, "colfft", s);
    if (f.e == 8) {
        set_smem(k_colfft<8>, smem);
        k_colfft<8><<<grid, threads, smem, s>>>(fb.R, fb.G, fb.st, k0, p->nproj, p->H, p->Wf, p->L, p->offv, f,
                                                 p->d_phv, FastDiv(C));
    } else {
        set_smem(k_colfft<12>, smem);
        k_colfft<12><<<grid, threads, smem, s>>>(fb.R, fb.G, fb.st, k0, p->nproj, p->H, p->Wf, p->L, p->offv, f,
                                                  p->d_phv, FastDiv(C));
    }
    LAM_LAUNCH_CHECK(p, "column FFT kernel");
    return LAMINO_OK;
}

// Lines per band-list chunk of the gridding kernels: all nproj lines if their
// lists (9 ints per line) fit in shared memory beside a band of band_bytes,
// else the most that do (at least 512 and at most 4 per thread, maxlines), with
// 4 KB kept for the group table; 0 if not even 512 fit.
static int line_chunk(int nproj, size_t band_bytes, int maxlines) {
    const size_t avail = 220 * 1024 - 4096;
    if (band_bytes + sizeof(int) * 10 >= avail) return 0;
    const long fit = (long)((avail - band_bytes - sizeof(int)) / (9 * sizeof(int)));
    const long ch = std::min<long>(std::min<long>(fit, maxlines), nproj);
    return ch >= std::min(nproj, 512) ? (int)ch : 0;
}

// Arguments of the gridding kernel and of its transpose shared by both.
static GridArgs grid_args(lamino_plan_t p) {
    GridArgs a;
    a.G = nullptr; a.V = nullptr; a.st = nullptr;
    a.trig = p->d_trig; a.dec1 = p->d_dec1;
    a.ch = 1; a.civ_cap = 0;
    a.nproj = p->nproj; a.Wf = p->Wf; a.Hf = p->Hf; a.n0 = p->n0; a.M1 = p->M1; a.M2 = p->M2;
    a.L = p->L; a.l0 = 0; a.lchunk = p->nproj;
    a.sinphi = (float)sin(p->tilt);
    a.c1 = (float)(-1.0 / (4.0 * p->t1));
    a.c2 = (float)(-1.0 / (4.0 * p->t2));
    a.q1 = (float)exp(-2.0 / (4.0 * p->t1));
    a.q2 = (float)exp(-2.0 / (4.0 * p->t2));
    a.f1 = p->fM1;
    return a;
}

int launch_grid(lamino_plan_t p, const FourierBufs& fb, int l0, int l1, cudaStream_t s) {
    if (l1 <= l0) return LAMINO_OK;
    // gridding + x1 inverse FFT of planes [l0, l1) into V
    GridArgs a = grid_args(p);
    a.G = fb.G; a.V = fb.V; a.st = fb.st; a.ch = fb.CH;
    a.l0 = l0;
    // Row pitch = 13 (mod 32) words. Lanes hold consecutive points of one
    // line (steps of ~1.33 cells), so a warp's reductions span ~42 cells along
    // the line and some banks take two lanes whatever the pitch; simulating the
    // reductions of the 512x512x256 workload's bands over all residues gives
    // 2.11 wavefronts per reduction at 13 (and 19), 2.25 at 5, 2.66 at 1 (which
    // stacks near-anti-diagonal lines into one bank), 3.35 at 0.
    a.ld = p->M1 + ((13 - p->M1) % 32 + 32) % 32;
    int T2 = p->grid_rows > 0 ? p->grid_rows : 16;
    while (T2 > 1 && (size_t)T2 * a.ld * sizeof(float2) > 132 * 1024) T2 /= 2;
    while (p->M2 % T2) T2 /= 2;
    a.T2 = T2;
    a.fT2 = FastDiv(T2);
    // band accumulator (planar) + compact interval list + per-line counts, for
    // chunks of lines when every line's list does not fit beside the band
    if (p->Wf > 8192) return fail(p, LAMINO_EUNSUPPORTED, "gridding supports Wf <= 8192");
    const size_t band_bytes = (size_t)T2 * a.ld * sizeof(float2);
    a.lchunk = line_chunk(p->nproj, band_bytes, 4 * 1024);
    if (a.lchunk <= 0)
        return fail(p, LAMINO_EUNSUPPORTED, "gridding tile of %zu bytes exceeds shared memory", band_bytes);
    size_t smem = band_bytes + sizeof(int) * (9 * (size_t)std::min(a.lchunk, p->nproj) + 1);
    // group table in what is left (bands with more points bisect instead)
    a.civ_cap = (int)std::min<size_t>(16384, (224 * 1024 - smem) / sizeof(int));
    smem += sizeof(int) * (size_t)a.civ_cap;
    int threads = 1024;
    dim3 grid(p->M2 / T2, l1 - l0);
    ProfScope prof(p, "grid", s);
    if (p->fM1.e == 8) dispatch_grid_w<8>(p->w, a, grid, threads, smem, s);
    else dispatch_grid_w<12>(p->w, a, grid, threads, smem, s);
    LAM_LAUNCH_CHECK(p, "gridding kernel");
    return LAMINO_OK;
}

// Columns per block of the x2 pass: <= ~72 KB per block so that several
// blocks share an SM and one block's loads overlap another's FFT.
static int x2_chunk(const FftDesc& f) {
    int C = 16;
    while (C > 1 && (size_t)C * seq_pitch(f.n, C) * sizeof(float2) > 72 * 1024) C /= 2;
    return C;
}

int launch_colifft(lamino_plan_t p, const FourierBufs& fb, int l0, int l1, cudaStream_t s) {
    if (l1 <= l0) return LAMINO_OK;
    // x2 inverse FFT of planes [l0, l1): V (chunk-relative) -> P (absolute)
    const FftDesc& f = p->fM2;
    const int C = x2_chunk(f);
    size_t smem = (size_t)C * seq_pitch(f.n, C) * sizeof(float2);
    dim3 grid((p->n0 + C - 1) / C, l1 - l0);
    int threads = fft_block_threads(f, C);
    ProfScope prof(p, "colifft", s);
    auto go = [&](auto kern) {
        set_smem(kern, smem);
        kern<<<grid, threads, smem, s>>>(fb.V, fb.P, p->n0, p->n1, f, p->d_dec2, FastDiv(C), FastDiv(f.n), l0);
    };
    if (threads > 512) go(k_colifft<8, 1024>);          // 8192-point x2 grids
    else if (f.e == 8) go(k_colifft<8, 512>);
    else go(k_colifft<12, 512>);
    LAM_LAUNCH_CHECK(p, "x2 inverse FFT kernel");
    return LAMINO_OK;
}

template <int E, int CB>
static void launch_zusfft_cb(lamino_plan_t p, const FourierBufs& fb, float* vol, int i10, dim3 grid,
                             int threads, size_t smem, cudaStream_t s) {
    set_smem(k_zusfft<E, CB>, smem);
    k_zusfft<E, CB><<<grid, threads, smem, s>>>(fb.P, vol, p->L, p->n0, p->n1, p->n2, p->fM3, p->d_zoff,
                                                 p->d_zl, p->d_zw, p->d_zrange, p->d_zwt, p->d_dec3, i10);
}

template <int E>
static void dispatch_zusfft(int C, lamino_plan_t p, const FourierBufs& fb, float* vol, int i10, dim3 grid,
                            int threads, size_t smem, cudaStream_t s) {
    switch (C) {
        case 16: launch_zusfft_cb<E, 16>(p, fb, vol, i10, grid, threads, smem, s); break;
        case 8: launch_zusfft_cb<E, 8>(p, fb, vol, i10, grid, threads, smem, s); break;
        case 4: launch_zusfft_cb<E, 4>(p, fb, vol, i10, grid, threads, smem, s); break;
        case 2: launch_zusfft_cb<E, 2>(p, fb, vol, i10, grid, threads, smem, s); break;
        default: launch_zusfft_cb<E, 1>(p, fb, vol, i10, grid, threads, smem, s); break;
    }
}

int launch_zusfft(lamino_plan_t p, const FourierBufs& fb, float* vol, int i10, int i11, cudaStream_t s) {
    if (i11 <= i10) return LAMINO_OK;
    // x3 USFFT of the columns of x2 rows [i10, i11)
    const FftDesc& f = p->fM3;
    if (f.t > 512) return refuse_long_fft(p, f, "the x3 USFFT");
    int C = 16;
    auto bytes = [&](int c) { return ((size_t)zus_pitch(c) * p->L + (size_t)c * seq_pitch(f.n, c)) * sizeof(float2); };
    while (C > 1 && bytes(C) > 72 * 1024) C /= 2;
    size_t smem = bytes(C);
    dim3 grid((p->n0 + C - 1) / C, i11 - i10);
    int threads = fft_block_threads(f, C);
    ProfScope prof(p, "zusfft", s);
    if (f.e == 8) dispatch_zusfft<8>(C, p, fb, vol, i10, grid, threads, smem, s);
    else dispatch_zusfft<12>(C, p, fb, vol, i10, grid, threads, smem, s);
    LAM_LAUNCH_CHECK(p, "x3 USFFT kernel");
    return LAMINO_OK;
}

// F3-F5 over chunks of zc k_v planes (the 2D USFFT of the split of
// Eq. fftfwdsplit, chunked by slices as in Sec. 5).
int run_planes(lamino_plan_t p, const FourierBufs& fb, cudaStream_t s) {
    int rc;
    for (int l0 = 0; l0 < p->L; l0 += fb.zc) {
        const int l1 = std::min(p->L, l0 + fb.zc);
        if ((rc = launch_grid(p, fb, l0, l1, s))) return rc;
        if ((rc = launch_colifft(p, fb, l0, l1, s))) return rc;
    }
    return LAMINO_OK;
}

int run_fourier_after_rows(lamino_plan_t p, const FourierBufs& fb, float* vol, cudaStream_t s) {
    int rc;
    if ((rc = launch_colfft(p, fb, 0, p->nproj, s))) return rc;
    if ((rc = run_planes(p, fb, s))) return rc;
    // F6 by column chunks (x2 rows), as many chunks as plane chunks
    const int nch = (p->L + fb.zc - 1) / fb.zc;
    for (int c = 0; c < nch; ++c) {
        const int i10 = (int)((long)p->n1 * c / nch), i11 = (int)((long)p->n1 * (c + 1) / nch);
        if ((rc = launch_zusfft(p, fb, vol, i10, i11, s))) return rc;
    }
    return LAMINO_OK;
}


int launch_project_fourier(lamino_plan_t p, const FourierBufs& fb, const float* vol, float* d,
                           cudaStream_t s) {
    // the backprojection's views in reverse order: Pt = P, Vt = V (one plane
    // chunk at a time), Gt = G, Rt = R (P and V are dead by then)
    float2* Pt = fb.P;   // [L][n1][n0]
    float2* Vt = fb.V;   // [zc][n0][M2]
    float2* Gt = fb.G;   // [L][nproj][Wf]
    float2* Rt = fb.R;   // [nproj][H][Wf]
    for (const FftDesc* f : {&p->fM3, &p->fM2, &p->fM1, &p->fHf, &p->fWf})
        if (f->t > 512) return refuse_long_fft(p, *f, "the Fourier projector");
    {   // x3
        const FftDesc& f = p->fM3;
        int C = 16;
        while (C > 1 && (size_t)C * (f.n + 1) * sizeof(float2) > 72 * 1024) C /= 2;
        size_t smem = (size_t)C * (f.n + 1) * sizeof(float2);
        dim3 grid((p->n0 + C - 1) / C, p->n1);
        int threads = fft_block_threads(f, C);
        ProfScope prof(p, "zusfft_t", s);
        if (f.e == 8) {
            set_smem(k_zusfft_t<8>, smem);
            k_zusfft_t<8><<<grid, threads, smem, s>>>(vol, Pt, p->L, p->n0, p->n1, p->n2, f, p->d_ztap, p->wz, p->d_dec3, FastDiv(C));
        } else {
            set_smem(k_zusfft_t<12>, smem);
            k_zusfft_t<12><<<grid, threads, smem, s>>>(vol, Pt, p->L, p->n0, p->n1, p->n2, f, p->d_ztap, p->wz, p->d_dec3,
                                                        FastDiv(C));
        }
        LAM_LAUNCH_CHECK(p, "x3 USFFT transpose kernel");
    }
    GridArgs a = grid_args(p);
    a.ld = p->M1 + 1;
    int T2 = 8;
    while (T2 > 1 && (size_t)(T2 + 2 * p->w - 1) * a.ld * sizeof(float2) > 150 * 1024) T2 /= 2;
    while (p->M2 % T2) T2 /= 2;
    a.T2 = T2;
    a.fNR = FastDiv(T2 + 2 * p->w - 1);
    const size_t tile = (size_t)(T2 + 2 * p->w - 1) * a.ld * sizeof(float2);
    a.lchunk = line_chunk(p->nproj, tile, 4 * 512);
    if (a.lchunk <= 0)
        return fail(p, LAMINO_EUNSUPPORTED, "gridding transpose tile of %zu bytes exceeds shared memory", tile);
    const size_t gsmem = tile + sizeof(int) * (9 * (size_t)std::min(a.lchunk, p->nproj) + 1);
    for (int l0 = 0; l0 < p->L; l0 += fb.zc) {
        const int l1 = std::min(p->L, l0 + fb.zc);
        {   // x2 of planes [l0, l1): Pt -> Vt (chunk-relative)
            const FftDesc& f = p->fM2;
            const int C = x2_chunk(f);
            size_t smem = (size_t)C * (f.n + 1) * sizeof(float2);
            dim3 grid((p->n0 + C - 1) / C, l1 - l0);
            int threads = fft_block_threads(f, C);
            ProfScope prof(p, "colifft_t", s);
            if (f.e == 8) {
                set_smem(k_colifft_t<8>, smem);
                k_colifft_t<8><<<grid, threads, smem, s>>>(Pt, Vt, p->n0, p->n1, f, p->d_dec2, FastDiv(C),
                                                           FastDiv(f.n), l0);
            } else {
                set_smem(k_colifft_t<12>, smem);
                k_colifft_t<12><<<grid, threads, smem, s>>>(Pt, Vt, p->n0, p->n1, f, p->d_dec2, FastDiv(C),
                                                            FastDiv(f.n), l0);
            }
            LAM_LAUNCH_CHECK(p, "x2 FFT transpose kernel");
        }
        {   // gridding transpose of planes [l0, l1): Vt -> Gt (absolute planes)
            a.l0 = l0;
            dim3 grid(p->M2 / T2, l1 - l0);
            ProfScope prof(p, "grid_t", s);
            auto go = [&](auto kern) {
                set_smem(kern, gsmem);
                kern<<<grid, 512, gsmem, s>>>(a, Vt, Gt);
            };
            const bool e8 = p->fM1.e == 8;
            switch (p->w) {
                case 2: e8 ? go(k_grid_t<8, 2>) : go(k_grid_t<12, 2>); break;
                case 3: e8 ? go(k_grid_t<8, 3>) : go(k_grid_t<12, 3>); break;
                case 4: e8 ? go(k_grid_t<8, 4>) : go(k_grid_t<12, 4>); break;
                case 5: e8 ? go(k_grid_t<8, 5>) : go(k_grid_t<12, 5>); break;
                case 6: e8 ? go(k_grid_t<8, 6>) : go(k_grid_t<12, 6>); break;
                case 7: e8 ? go(k_grid_t<8, 7>) : go(k_grid_t<12, 7>); break;
                default: e8 ? go(k_grid_t<8, 8>) : go(k_grid_t<12, 8>); break;
            }
            LAM_LAUNCH_CHECK(p, "gridding transpose kernel");
        }
    }
    {   // column pass transpose
        const FftDesc& f = p->fHf;
        int C = largest_pow2_divisor_upto(p->Wf, 16);
        while (C > 1 && (size_t)C * (f.n + 1) * sizeof(float2) > 100 * 1024) C /= 2;
        size_t smem = (size_t)C * (f.n + 1) * sizeof(float2);
        dim3 grid(p->Wf / C, p->nproj);
        int threads = fft_block_threads(f, C);
        ProfScope prof(p, "colfft_t", s);
        if (f.e == 8) {
            set_smem(k_colfft_t<8>, smem);
            k_colfft_t<8><<<grid, threads, smem, s>>>(Gt, Rt, p->nproj, p->H, p->Wf, p->L, p->offv, f, p->d_phv,
                                                      FastDiv(C));
        } else {
            set_smem(k_colfft_t<12>, smem);
            k_colfft_t<12><<<grid, threads, smem, s>>>(Gt, Rt, p->nproj, p->H, p->Wf, p->L, p->offv, f, p->d_phv,
                                                       FastDiv(C));
        }
        LAM_LAUNCH_CHECK(p, "column FFT transpose kernel");
    }
    {   // row pass transpose
        const FftDesc& f = p->fWf;
        int rows = 1;
        while (rows * 2 * f.t <= 512 && (size_t)rows * 2 * f.n * sizeof(float2) <= 64 * 1024) rows *= 2;
        long nrows = (long)p->nproj * p->H;
        size_t smem = (size_t)rows * f.n * sizeof(float2);
        dim3 grid((unsigned)((nrows + rows - 1) / rows));
        const float unscale = (float)(p->nproj / 3.14159265358979323846);
        ProfScope prof(p, "rowfft_t", s);
        if (f.e == 8) {
            set_smem(k_rowfft_t<8>, smem);
            k_rowfft_t<8><<<grid, rows * f.t, smem, s>>>(Rt, d, nrows, p->W, p->offu, f, p->d_phu, unscale, rows);
        } else {
            set_smem(k_rowfft_t<12>, smem);
            k_rowfft_t<12><<<grid, rows * f.t, smem, s>>>(Rt, d, nrows, p->W, p->offu, f, p->d_phu, unscale, rows);
        }
        LAM_LAUNCH_CHECK(p, "row FFT transpose kernel");
    }
    return LAMINO_OK;
}

}  // namespace lam
