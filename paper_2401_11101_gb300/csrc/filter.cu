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
template <int E, typename Tin>
__global__ void __launch_bounds__(512, 1) k_filter(const Tin* __restrict__ d, float* __restrict__ q,
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
// two real spectra and writes them in signed frequency order mi = m + Wf/2,
// multiplied by the centring phase exp(2 pi i m cu/Wf) (zero at m = -Wf/2).
// Output R[row][mi], row = k*H + r.
template <int EP, int EF, typename Tin>
__global__ void __launch_bounds__(512, 1) k_rowfft(const Tin* __restrict__ d, float2* __restrict__ R,
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
        for (int mi = tid; mi < Nf; mi += T) {
            int m = mi - half;
            int i1 = m < 0 ? m + Nf : m;          // index of +m
            int i2 = m > 0 ? Nf - m : -m;         // index of -m
            float2 Z = xf[fpad(i1)], Zc = xf[fpad(i2)];
            Zc.y = -Zc.y;
            float2 A = make_float2(0.5f * (Z.x + Zc.x), 0.5f * (Z.y + Zc.y));
            float2 Dm = csub(Z, Zc);
            float2 B = make_float2(0.5f * Dm.y, -0.5f * Dm.x);   // (Z - conj Z(-m)) / (2i)
            float2 ph = __ldg(phu + mi);
            R[(size_t)rA * Nf + mi] = cmul(A, ph);
            if (hasB) R[(size_t)rB * Nf + mi] = cmul(B, ph);
        }
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
    int pairs = pairs_for(f.t, sizeof(float2) * fpad_len(f.n));
    size_t smem = sizeof(float2) * fpad_len(f.n) * pairs;
    dim3 grid((unsigned)((npairs + pairs - 1) / pairs));
    const float* filt = p->d_filt + (size_t)kind * p->Wp;
    ProfScope prof(p, "filter", s);
    if (f.e == 8) {
        cudaFuncSetAttribute(k_filter<8, Tin>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_filter<8, Tin><<<grid, pairs * f.t, smem, s>>>(d, q, row0, row1, p->W, f, filt, pairs);
    } else {
        cudaFuncSetAttribute(k_filter<12, Tin>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_filter<12, Tin><<<grid, pairs * f.t, smem, s>>>(d, q, row0, row1, p->W, f, filt, pairs);
    }
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
    auto kern = k_rowfft<EP, EF, Tin>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    ProfScope prof(p, EP > 0 ? "filter_rowfft" : "rowfft", s);
    kern<<<grid, pairs * T, smem, s>>>(d, R, row0, row1, p->W, p->offu, p->fWp, p->fWf, filt,
                                       p->d_phu, pairs, T);
    LAM_LAUNCH_CHECK(p, "row FFT kernel");
    return LAMINO_OK;
}

template <typename Tin>
int rowfft_typed(lamino_plan_t p, const Tin* d, float2* R, int kind, cudaStream_t s, long r0,
                 long r1) {
    const float* filt = kind >= 0 ? p->d_filt + (size_t)kind * p->Wp : nullptr;
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
