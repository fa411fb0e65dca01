// Row kernels: the filter W of Eq. recon and the detector-row pass of the 2D
// FFT of the Fourier form (F_2D of Eq. fftadj).
//
// Both work on pairs of detector rows packed into one complex sequence
// z = a + i b. The filter transfer function H(f) is real and even, so
// IFFT(H . FFT(a + i b)) = (H*a) + i (H*b) with both parts real: one complex
// FFT pair filters two rows. For the Fourier row pass the two real spectra
// are separated afterwards with A(m) = (Z(m) + conj Z(-m))/2 and
// B(m) = (Z(m) - conj Z(-m))/(2i).
#include <algorithm>

#include "common.cuh"

namespace lam {
namespace {

// Rows rA and rA + 1 (if hasB) into x[j] = (a[j - off], b[j - off]) for j in
// [0, N), zero outside [off, off + W), x a padded sequence (SeqCP layout);
// 8 independent loads in flight per thread.
template <typename Tin>
__device__ __forceinline__ void load_pair_rows(const Tin* __restrict__ d, float2* x, long rA, bool hasB,
                                               int W, int N, int off, int tid, int T) {
    constexpr int U = 8;
    const size_t ra = (size_t)rA * W, rb = ra + W;
    for (int base = tid; base < N; base += U * T) {
        float a[U], b[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int src = base + u * T - off;
            const bool in = base + u * T < N && src >= 0 && src < W;
            a[u] = in ? load_f(d, ra + src) : 0.f;
            b[u] = (in && hasB) ? load_f(d, rb + src) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (base + u * T < N) x[fpad(base + u * T)] = make_float2(a[u], b[u]);
    }
}

// Filter: rows of length W zero-padded to Wp, FFT, x H(f)/Wp, IFFT, crop.
// One CTA handles `pairs` row pairs; each pair uses t = Wp/E threads.
template <int E, typename Tin, int MT>
__global__ void __launch_bounds__(MT, 1) k_filter(const Tin* __restrict__ d, float* __restrict__ q,
                                                long row0, long row1, int W, FftDesc fp,
                                                const float* __restrict__ filt, int pairs) {
    extern __shared__ float2 sm[];
    const int T = fp.t, N = fp.n;
    const int seq = threadIdx.x / T, tid = threadIdx.x % T;
    const long pair = (long)blockIdx.x * pairs + seq;
    const long rA = row0 + 2 * pair, rB = rA + 1;
    const bool active = seq < pairs && rA < row1;
    const bool hasB = rB < row1;
    float2* x = sm + (size_t)seq * fpad_len(N);
    if (active) load_pair_rows(d, x, rA, hasB, W, N, 0, tid, T);
    __syncthreads();
    fft_run<E>(SeqCP{x}, fp, tid, active, -1.f);
    if (active)
        for (int j = tid; j < N; j += T) {
            float h = __ldg(filt + j);
            const float2 v = x[fpad(j)];
            x[fpad(j)] = make_float2(v.x * h, v.y * h);
        }
    __syncthreads();
    fft_run<E>(SeqCP{x}, fp, tid, active, +1.f);
    if (active)
        for (int j = tid; j < W; j += T) {
            float2 v = x[fpad(j)];
            q[(size_t)rA * W + j] = v.x;
            if (hasB) q[(size_t)rB * W + j] = v.y;
        }
}

// Fourier row pass. Optionally filters first (EP > 0: FFT of length Wp), then
// places the W samples at offset offu of a length-Wf row, FFTs it, splits the
// two real spectra and writes, multiplied by the centring phase
// exp(2 pi i m cu/Wf), the frequencies m in [0, Wf/2) only: a real row's
// spectrum at -m is the conjugate of that at m (and so is the phase), which
// the column pass uses. Output R[row][m], row = k*H + r, pitch Wf/2.
template <int EP, int EF, typename Tin, int MT>
__global__ void __launch_bounds__(MT, 1) k_rowfft(const Tin* __restrict__ d, float2* __restrict__ R,
                                                long row0, long row1, int W, int offu, FftDesc fp,
                                                FftDesc ff, const float* __restrict__ filt,
                                                const float2* __restrict__ phu, int pairs, int T) {
    extern __shared__ float2 sm[];
    const int Np = (EP > 0) ? fp.n : 0, Nf = ff.n;
    const int seq = threadIdx.x / T, tid = threadIdx.x % T;
    const long pair = (long)blockIdx.x * pairs + seq;
    const long rA = row0 + 2 * pair, rB = rA + 1;
    const bool active = seq < pairs && rA < row1;
    const bool hasB = rB < row1;
    const int Lp = (EP > 0) ? fpad_len(Np) : 0;
    float2* xp = sm + (size_t)seq * (Lp + fpad_len(Nf));
    float2* xf = xp + Lp;
    if constexpr (EP > 0) {
        if (active) load_pair_rows(d, xp, rA, hasB, W, Np, 0, tid, T);
        __syncthreads();
        fft_run<EP>(SeqCP{xp}, fp, tid, active, -1.f);
        if (active)
            for (int j = tid; j < Np; j += T) {
                float h = __ldg(filt + j);
                const float2 v = xp[fpad(j)];
                xp[fpad(j)] = make_float2(v.x * h, v.y * h);
            }
        __syncthreads();
        fft_run<EP>(SeqCP{xp}, fp, tid, active, +1.f);
        if (active)
            for (int j = tid; j < Nf; j += T) {
                int src = j - offu;
                xf[fpad(j)] = (src >= 0 && src < W) ? xp[fpad(src)] : make_float2(0.f, 0.f);
            }
    } else {
        if (active) load_pair_rows(d, xf, rA, hasB, W, Nf, offu, tid, T);
    }
    __syncthreads();
    fft_run<EF>(SeqCP{xf}, ff, tid, active, -1.f);
    if (active) {
        const int half = Nf / 2;
        for (int m = tid; m < half; m += T) {
            const int i2 = m > 0 ? Nf - m : 0;    // index of -m
            float2 Z = xf[fpad(m)], Zc = xf[fpad(i2)];
            Zc.y = -Zc.y;
            float2 A = make_float2(0.5f * (Z.x + Zc.x), 0.5f * (Z.y + Zc.y));
            float2 Dm = csub(Z, Zc);
            float2 B = make_float2(0.5f * Dm.y, -0.5f * Dm.x);   // (Z - conj Z(-m)) / (2i)
            float2 ph = __ldg(phu + half + m);
            R[(size_t)rA * half + m] = cmul(A, ph);
            if (hasB) R[(size_t)rB * half + m] = cmul(B, ph);
        }
    }
}

// ---------------------------------------------------------------------------
// Rows of length 3N (N = 256 or 512, one warp per N-point transform). A row
// pair z = a + i b is kept 3-way decimated in shared memory, buffer b holding
// z[3i + b] (b = 0, 1, 2; buffers LB slots apart). A length-3N DFT is then
// three N-point DFTs of the buffers (one warp each, register-resident:
// fft256_warp / fft512_warp) and a radix-3 step per frequency k < N:
//   X[k + N j] = sum_b exp(-2 pi i b k / 3N) Y_b[k] exp(-2 pi i b j / 3)
// (decimation in time), which reads and writes the three buffers at index k
// only. The filter multiplies X by H and inverts the radix-3 step in the same
// pass, so forward transform, multiplication and inverse transform meet in
// registers; the 3N-point Stockham stages (six shared-memory round trips each
// way) become two warp transposes each way.
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void fft_warp(float2* x, const float2* __restrict__ tw, float s, int lane) {
    static_assert(N == 256 || N == 512, "warp FFT length");
    if constexpr (N == 256) fft256_warp(x, tw, s, lane);
    else fft512_warp(x, tw, s, lane);
}

// Pitch of the three decimated buffers of a row pair: 11 (mod 16) slots, so
// that a half-warp's accesses to z[j] .. z[j + 15] (slots (j % 3) LB + j / 3)
// fall on 16 different bank pairs (with LB = 0 (mod 16), three consecutive j
// shared one).
__host__ __device__ constexpr int pitch3(int n) { return n + ((11 - n) % 16 + 16) % 16; }

// barrier of the 96 threads (three warps) of sequence `seq` of a block
__device__ __forceinline__ void seq_sync(int seq) {
    asm volatile("bar.sync %0, 96;" ::"r"(seq + 1) : "memory");
}

// Rows rA and rA + 1 (if hasB) placed at offset `off` of a length-3NB row,
// 3-way decimated into buf (buffers LB apart), zero elsewhere. Sixteen loads
// of a thread are in flight at a time.
template <typename Tin>
__device__ __forceinline__ void load_rows3(const Tin* __restrict__ d, float2* buf, int LB, int NB,
                                           long rA, bool hasB, int W, int off, int t96) {
    constexpr int U = 8;
    const size_t ra = (size_t)rA * W, rb = ra + W;
    for (int j0 = t96; j0 < 3 * NB; j0 += U * 96) {
        float a[U], b[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = j0 + u * 96, src = j - off;
            const bool in = j < 3 * NB && src >= 0 && src < W;
            a[u] = in ? load_f(d, ra + src) : 0.f;
            b[u] = (in && hasB) ? load_f(d, rb + src) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = j0 + u * 96;
            if (j < 3 * NB) buf[(j % 3) * LB + j / 3] = make_float2(a[u], b[u]);
        }
    }
}

// The filter of a decimated row pair of length 3N in place: forward DFT,
// x H(f)/3N (the filter table), inverse DFT (unnormalised, the 1/3N is in
// the table). Ends with the sequence's barrier.
template <int N>
__device__ __forceinline__ void filter_rows3(float2* buf, int LB, const float2* __restrict__ twN,
                                             const float2* __restrict__ tw3N, const float* __restrict__ filt,
                                             int t96, int lane, int seq) {
    const int w3 = t96 >> 5;
    fft_warp<N>(buf + w3 * LB, twN, -1.f, lane);
    seq_sync(seq);
    for (int k = t96; k < N; k += 96) {
        float2 y[3] = {buf[k], buf[LB + k], buf[2 * LB + k]};
        const float2 w1 = __ldg(tw3N + k), w2 = __ldg(tw3N + 2 * k);
        y[1] = cmul(y[1], w1);
        y[2] = cmul(y[2], w2);
        bfly<3>(y, -1.f);                         // X[k + N j], j = 0, 1, 2
#pragma unroll
        for (int j = 0; j < 3; ++j) y[j] = cscale(y[j], __ldg(filt + k + N * j));
        bfly<3>(y, +1.f);                         // inverse radix-3 step
        y[1] = cmul(y[1], make_float2(w1.x, -w1.y));
        y[2] = cmul(y[2], make_float2(w2.x, -w2.y));
        buf[k] = y[0];
        buf[LB + k] = y[1];
        buf[2 * LB + k] = y[2];
    }
    seq_sync(seq);
    fft_warp<N>(buf + w3 * LB, twN, +1.f, lane);
    seq_sync(seq);
}

// Filter (direct form) for Wp = 3N: a block holds blockDim/96 row pairs.
template <int N, typename Tin>
__global__ void __launch_bounds__(384) k_filter3(const Tin* __restrict__ d, float* __restrict__ q, long row0,
                                                 long row1, int W, const float2* __restrict__ twN,
                                                 const float2* __restrict__ tw3N, const float* __restrict__ filt) {
    extern __shared__ float2 sm[];
    const int seq = threadIdx.x / 96, t96 = threadIdx.x % 96, lane = threadIdx.x & 31;
    const long rA = row0 + 2 * ((long)blockIdx.x * (blockDim.x / 96) + seq);
    if (rA >= row1) return;                       // the whole sequence leaves: no barrier waits on it
    const bool hasB = rA + 1 < row1;
    constexpr int LB = pitch3(N);
    float2* buf = sm + (size_t)seq * 3 * LB;
    load_rows3(d, buf, LB, N, rA, hasB, W, 0, t96);
    seq_sync(seq);
    filter_rows3<N>(buf, LB, twN, tw3N, filt, t96, lane, seq);
    for (int j = t96; j < W; j += 96) {
        const float2 v = buf[(j % 3) * LB + j / 3];
        q[(size_t)rA * W + j] = v.x;
        if (hasB) q[(size_t)(rA + 1) * W + j] = v.y;
    }
}

// Fourier row pass for Wf = 3 NF (NF = 256 or 512), optionally after the
// filter (N > 0: Wp = 3N, NF <= N, offu a multiple of 3): the filtered row
// stays decimated, and since offu = 3 o, the decimated subsequences of the
// padded row are the filter's buffers shifted by o slots (zero past W). Then
// the NF-point warp FFTs, the radix-3 step written back in natural order
// (X[k + NF j] in buffer j, slot k), and the same epilogue as k_rowfft: the
// two real spectra, the centring phase, R[row][m] for m in [0, Wf/2).
template <int N, int NF, typename Tin>
__global__ void __launch_bounds__(384, 2) k_rowfft3(const Tin* __restrict__ d, float2* __restrict__ R,
                                                 long row0, long row1, int W, int offu,
                                                 const float2* __restrict__ twN, const float2* __restrict__ tw3N,
                                                 const float* __restrict__ filt,
                                                 const float2* __restrict__ twNF, const float2* __restrict__ tw3NF,
                                                 const float2* __restrict__ phu) {
    extern __shared__ float2 sm[];
    constexpr int LB = pitch3((N > NF) ? N : NF);
    const int seq = threadIdx.x / 96, t96 = threadIdx.x % 96, lane = threadIdx.x & 31, w3 = t96 >> 5;
    const long rA = row0 + 2 * ((long)blockIdx.x * (blockDim.x / 96) + seq);
    if (rA >= row1) return;
    const bool hasB = rA + 1 < row1;
    float2* buf = sm + (size_t)seq * 3 * LB;
    if constexpr (N > 0) {
        load_rows3(d, buf, LB, N, rA, hasB, W, 0, t96);
        seq_sync(seq);
        filter_rows3<N>(buf, LB, twN, tw3N, filt, t96, lane, seq);
        // shift buffer w3 by o = offu/3 slots, zero past the row (each warp its own buffer)
        const int o = offu / 3;
        float2 v[NF / 32];
        float2* bw = buf + w3 * LB;
#pragma unroll
        for (int i = 0; i < NF / 32; ++i) {
            const int a = lane + 32 * i, src = a - o, j = 3 * src + w3;
            v[i] = (src >= 0 && j < W) ? bw[src] : make_float2(0.f, 0.f);
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < NF / 32; ++i) bw[lane + 32 * i] = v[i];
        __syncwarp();
    } else {
        load_rows3(d, buf, LB, NF, rA, hasB, W, offu, t96);
        seq_sync(seq);
    }
    fft_warp<NF>(buf + w3 * LB, twNF, -1.f, lane);
    seq_sync(seq);
    for (int k = t96; k < NF; k += 96) {
        float2 y[3] = {buf[k], buf[LB + k], buf[2 * LB + k]};
        y[1] = cmul(y[1], __ldg(tw3NF + k));
        y[2] = cmul(y[2], __ldg(tw3NF + 2 * k));
        bfly<3>(y, -1.f);
        buf[k] = y[0];
        buf[LB + k] = y[1];
        buf[2 * LB + k] = y[2];
    }
    seq_sync(seq);
    constexpr int Nf = 3 * NF, half = Nf / 2;
    auto X = [&](int i) { return buf[(i / NF) * LB + i % NF]; };
    for (int m = t96; m < half; m += 96) {
        const int i2 = m > 0 ? Nf - m : 0;          // index of -m
        float2 Z = X(m), Zc = X(i2);
        Zc.y = -Zc.y;
        const float2 A = make_float2(0.5f * (Z.x + Zc.x), 0.5f * (Z.y + Zc.y));
        const float2 Dm = csub(Z, Zc);
        const float2 B = make_float2(0.5f * Dm.y, -0.5f * Dm.x);   // (Z - conj Z(-m)) / (2i)
        const float2 ph = __ldg(phu + half + m);
        R[(size_t)rA * half + m] = cmul(A, ph);
        if (hasB) R[(size_t)(rA + 1) * half + m] = cmul(B, ph);
    }
}

// Row pairs per block: blocks of about 128 threads (one pair for rows of
// 1024 or more): small blocks wait on fewer warps at each FFT barrier and
// more of them share an SM.
int pairs_for(int T, size_t bytes_per_pair) {
    int pairs = 1;
    while (pairs * 2 * T <= 128 && (pairs * 2) * bytes_per_pair <= 64 * 1024) pairs *= 2;
    return pairs;
}

template <typename Tin>
int filter_typed(lamino_plan_t p, const Tin* d, float* q, int kind, cudaStream_t s, long row0,
                 long row1) {
    const FftDesc& f = p->fWp;
    long npairs = (row1 - row0 + 1) / 2;
    if (npairs <= 0) return LAMINO_OK;
    const float* filt3 = p->d_filt + (size_t)kind * p->Wp;
    if (p->fWp3.n == 512 || p->fWp3.n == 256) {
        // three one-warp transforms per row pair, four row pairs per block
        const int N = p->fWp3.n;
        const size_t smem = sizeof(float2) * 3 * pitch3(N) * 4;
        dim3 grid((unsigned)((npairs + 3) / 4));
        ProfScope prof(p, "filter", s);
        if (N == 512) {
            cudaFuncSetAttribute(k_filter3<512, Tin>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_filter3<512, Tin><<<grid, 384, smem, s>>>(d, q, row0, row1, p->W, p->fWp3.tw, f.tw, filt3);
        } else {
            cudaFuncSetAttribute(k_filter3<256, Tin>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_filter3<256, Tin><<<grid, 384, smem, s>>>(d, q, row0, row1, p->W, p->fWp3.tw, f.tw, filt3);
        }
        LAM_LAUNCH_CHECK(p, "filter kernel");
        return LAMINO_OK;
    }
    int pairs = pairs_for(f.t, sizeof(float2) * fpad_len(f.n));
    size_t smem = sizeof(float2) * fpad_len(f.n) * pairs;
    dim3 grid((unsigned)((npairs + pairs - 1) / pairs));
    const float* filt = p->d_filt + (size_t)kind * p->Wp;
    ProfScope prof(p, "filter", s);
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<grid, pairs * f.t, smem, s>>>(d, q, row0, row1, p->W, f, filt, pairs);
    };
    if (pairs * f.t > 512) go(k_filter<8, Tin, 1024>);      // 8192-point rows
    else if (f.e == 8) go(k_filter<8, Tin, 512>);
    else go(k_filter<12, Tin, 512>);
    LAM_LAUNCH_CHECK(p, "filter kernel");
    return LAMINO_OK;
}

template <int EP, int EF, typename Tin>
int rowfft_launch(lamino_plan_t p, const Tin* d, float2* R, const float* filt, cudaStream_t s,
                  long row0, long row1) {
    const int Tp = (EP > 0) ? p->fWp.t : 0;
    const int T = std::max(Tp, p->fWf.t);
    const size_t per_pair = sizeof(float2) * ((EP > 0 ? fpad_len(p->Wp) : 0) + fpad_len(p->Wf));
    int pairs = pairs_for(T, per_pair);
    long npairs = (row1 - row0 + 1) / 2;
    if (npairs <= 0) return LAMINO_OK;
    size_t smem = per_pair * pairs;
    dim3 grid((unsigned)((npairs + pairs - 1) / pairs));
    // 1024 threads per row pair only for 8192-point rows (filter length 2^13:
    // EP = 8, or an unfiltered 2^13 Fourier row: EP = 0, EF = 8)
    auto kern = k_rowfft<EP, EF, Tin, 512>;
    if constexpr (EP == 8 || (EP == 0 && EF == 8)) {
        if (pairs * T > 512) kern = k_rowfft<EP, EF, Tin, 1024>;
    } else {
        if (pairs * T > 512) return fail(p, LAMINO_EUNSUPPORTED, "row FFT block of %d threads", pairs * T);
    }
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    ProfScope prof(p, EP > 0 ? "filter_rowfft" : "rowfft", s);
    kern<<<grid, pairs * T, smem, s>>>(d, R, row0, row1, p->W, p->offu, p->fWp, p->fWf, filt,
                                       p->d_phu, pairs, T);
    LAM_LAUNCH_CHECK(p, "row FFT kernel");
    return LAMINO_OK;
}

template <int N, int NF, typename Tin>
int rowfft3_launch(lamino_plan_t p, const Tin* d, float2* R, const float* filt, cudaStream_t s,
                   long row0, long row1) {
    long npairs = (row1 - row0 + 1) / 2;
    if (npairs <= 0) return LAMINO_OK;
    constexpr int LB = pitch3((N > NF) ? N : NF);
    const size_t smem = sizeof(float2) * 3 * LB * 4;
    dim3 grid((unsigned)((npairs + 3) / 4));
    auto kern = k_rowfft3<N, NF, Tin>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    ProfScope prof(p, N > 0 ? "filter_rowfft" : "rowfft", s);
    kern<<<grid, 384, smem, s>>>(d, R, row0, row1, p->W, p->offu, N > 0 ? p->fWp3.tw : nullptr,
                                 N > 0 ? p->fWp.tw : nullptr, filt, p->fWf3.tw, p->fWf.tw, p->d_phu);
    LAM_LAUNCH_CHECK(p, "row FFT kernel");
    return LAMINO_OK;
}

// The decimated-by-3 row kernels apply when the lengths are 3 x (256 or 512)
// and, after the filter, the row offset in the padded Fourier row is a
// multiple of 3 with the Fourier length not above the filter's.
template <typename Tin>
int rowfft3_typed(lamino_plan_t p, const Tin* d, float2* R, const float* filt, cudaStream_t s, long r0,
                  long r1, bool* done) {
    *done = false;
    const int nf = p->fWf3.n, np = filt ? p->fWp3.n : 0;
    const bool nf_ok = nf == 256 || nf == 512;
    if (!nf_ok) return LAMINO_OK;
    if (filt && !((np == 256 || np == 512) && nf <= np && p->offu % 3 == 0)) return LAMINO_OK;
    *done = true;
    if (!filt) return nf == 256 ? rowfft3_launch<0, 256, Tin>(p, d, R, filt, s, r0, r1)
                                : rowfft3_launch<0, 512, Tin>(p, d, R, filt, s, r0, r1);
    if (np == 512) return nf == 256 ? rowfft3_launch<512, 256, Tin>(p, d, R, filt, s, r0, r1)
                                    : rowfft3_launch<512, 512, Tin>(p, d, R, filt, s, r0, r1);
    return rowfft3_launch<256, 256, Tin>(p, d, R, filt, s, r0, r1);
}

template <typename Tin>
int rowfft_typed(lamino_plan_t p, const Tin* d, float2* R, int kind, cudaStream_t s, long r0,
                 long r1) {
    const float* filt = kind >= 0 ? p->d_filt + (size_t)kind * p->Wp : nullptr;
    bool done = false;
    int rc3 = rowfft3_typed(p, d, R, filt, s, r0, r1, &done);
    if (done) return rc3;
    const int ef = p->fWf.e;
    if (kind < 0) {
        return ef == 8 ? rowfft_launch<0, 8, Tin>(p, d, R, filt, s, r0, r1)
                        : rowfft_launch<0, 12, Tin>(p, d, R, filt, s, r0, r1);
    }
    const int ep = p->fWp.e;
    if (ep == 8 && ef == 8) return rowfft_launch<8, 8, Tin>(p, d, R, filt, s, r0, r1);
    if (ep == 8 && ef == 12) return rowfft_launch<8, 12, Tin>(p, d, R, filt, s, r0, r1);
    if (ep == 12 && ef == 8) return rowfft_launch<12, 8, Tin>(p, d, R, filt, s, r0, r1);
    return rowfft_launch<12, 12, Tin>(p, d, R, filt, s, r0, r1);
}

}  // namespace

int launch_filter(lamino_plan_t p, const void* d, int dtype, float* q, int kind, cudaStream_t s,
                  long row0, long row1) {
    if (row1 < 0) row1 = (long)p->nproj * p->H;
    switch (dtype) {
        case LAMINO_F32: return filter_typed(p, (const float*)d, q, kind, s, row0, row1);
        case LAMINO_F16: return filter_typed(p, (const __half*)d, q, kind, s, row0, row1);
        default: return filter_typed(p, (const __nv_bfloat16*)d, q, kind, s, row0, row1);
    }
}

int launch_rowfft(lamino_plan_t p, const void* d, int dtype, float2* R, int kind, cudaStream_t s,
                  long row0, long row1) {
    if (row1 < 0) row1 = (long)p->nproj * p->H;
    switch (dtype) {
        case LAMINO_F32: return rowfft_typed(p, (const float*)d, R, kind, s, row0, row1);
        case LAMINO_F16: return rowfft_typed(p, (const __half*)d, R, kind, s, row0, row1);
        default: return rowfft_typed(p, (const __nv_bfloat16*)d, R, kind, s, row0, row1);
    }
}

}  // namespace lam
