// Internal declarations of the laminographic FBP library: plan object, error
// handling and the shared-memory FFT used by every Fourier-side kernel.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lamino.h"

namespace lam {

// Largest FFT length any kernel handles (one sequence fits in shared memory),
// and the most threads one sequence may take (n / elements per thread): a
// block must hold at least one whole sequence. So 2^k lengths go up to 8192,
// 3*2^k up to 6144. Most FFT kernels run blocks of at most 512 threads
// (lengths up to 4096); the filter, the row pass, the gridding and the x2 pass
// also have 1024-thread instantiations for 8192-point sequences, and the
// others refuse such lengths (EUNSUPPORTED).
constexpr int kMaxFft = 8192;
constexpr int kMaxFftThreads = 1024;

// Radix schedule of one FFT length: n = product of the stage radices, stage
// st having radix (rads >> 4 st) & 15; power-of-two radices come first and a
// radix-3 stage last, so every partial length ns is a power of two. Each stage
// is done by t = n/e threads holding e complex values in registers.
struct FftDesc {
    int n = 0, e = 0, t = 0, nst = 0;
    unsigned rads = 0;
    const float2* tw = nullptr;  // device table exp(-2 pi i s/n), s in [0, n)
};

// Quotient and remainder by a divisor d >= 1 fixed at launch, for dividends
// 0 <= n with n d < 2^32, by one high multiply with M = ceil(2^32 / d):
// n M / 2^32 = n/d + n e / (d 2^32) with e = M d - 2^32 in [0, d), and the
// second term is below n / 2^32 < 1/d, so the floor stays floor(n/d). The
// kernels' index loops divide by launch-time sizes (columns per block, grid
// lengths), where a division by a runtime value costs ~20 instructions.
struct FastDiv {
    unsigned M = 0;
    int d = 1;
    FastDiv() = default;
    explicit FastDiv(int dd) : M(dd > 1 ? (unsigned)((0x100000000ull + (unsigned)dd - 1) / (unsigned)dd) : 0u), d(dd) {}
    __device__ __forceinline__ int div(int n) const { return d == 1 ? n : (int)__umulhi((unsigned)n, M); }
    __device__ __forceinline__ int mod(int n) const { return n - div(n) * d; }
};

// Elements per thread: 8 for 2^k lengths (radix-8 stages, one radix-4/2), 12
// for 3*2^k lengths (radix-4/2 stages and one radix-3 stage).
int fft_elems(int n);
bool fft_len_ok(int n);
int fft_size_at_least(double n);   // smallest 2^k or 3*2^k >= n

struct DirectCfg {
    int tx = 32, ty = 16, tz = 16;   // voxel tile of one CTA (x1, x2, x3)
    int bw = 0, bh = 0;              // detector footprint box (columns, rows)
    int stages = 6;                  // TMA pipeline depth
};

}  // namespace lam

struct lamino_plan_s {
    int device = 0;
    int n0 = 0, n1 = 0, n2 = 0, nproj = 0, W = 0, H = 0;
    double tilt = 0.0;
    std::vector<double> theta;

    // derived sizes
    int Wp = 0, Wf = 0, Hf = 0, L = 0, M1 = 0, M2 = 0, M3 = 0;
    int w = 4, wz = 6, offu = 0, offv = 0;
    double err_est = 0.0;                // predicted USFFT relL2 error (usfft_err_est)
    int grid_rows = 0;                   // band height of the gridding kernel (0: default)
    int z_chunk = 0;                     // k_v planes per F3-F5 chunk and output slices per
                                         // direct launch (0: no chunking)
    double t1 = 0, t2 = 0, t3 = 0;       // Gaussian widths (grid cells^2) per axis
    lam::FftDesc fWp, fWf, fHf, fM1, fM2, fM3;
    lam::FftDesc fWp3, fWf3;             // Wp/3 and Wf/3 (decimated-by-3 row kernels; n = 0 if unused)
    int zmax = 0;                        // taps per cell of the x3 gridding table

    // device tables (owned)
    float2* d_trig = nullptr;      // [nproj] (cos t, sin t) float
    double* d_trig64 = nullptr;    // [nproj][2] (cos t, sin t) double
    float* d_filt = nullptr;       // [3][Wp] H(f)/Wp per filter kind, FFT order
    float2* d_phu = nullptr;       // [Wf] centring phase of column frequency m (signed order)
    float2* d_phv = nullptr;       // [L]  centring phase of row frequency l
    float* d_dec1 = nullptr;       // [n0] 1/(M1 psi1(x1))
    float* d_dec2 = nullptr;       // [n1] 1/(M2 psi2(x2))
    float* d_dec3 = nullptr;       // [n2] scale/(M3 psi3(x3))
    int* d_zoff = nullptr;         // [M3+1] CSR offsets of the x3 gridding table
    int* d_zl = nullptr;           // taps: plane index
    float* d_zw = nullptr;         // taps: weight (Gaussian x Hermitian factor)
    int2* d_zrange = nullptr;      // [M3] (first plane, taps) of each cell when its planes are consecutive
    float* d_zwt = nullptr;        // [zmax][M3] the same weights tap-major (d_zrange set only then)
    int2* d_ztap = nullptr;        // [L][2 wz] (cell, weight bits) per plane: the same taps by plane
    float2* d_tw = nullptr;        // all FFT twiddle tables
    int* d_err = nullptr;          // device error word (bounded waits)
    size_t table_bytes = 0;        // device bytes of the tables above

    // workspaces (owned, allocated on first use)
    void* ws_a = nullptr; size_t ws_a_bytes = 0;   // row spectra R / gridded planes V
    void* ws_b = nullptr; size_t ws_b_bytes = 0;   // half spectra G / planes P
    float* q_buf = nullptr; size_t q_buf_bytes = 0; // filtered rows (direct FBP)
    float* q_pad = nullptr; size_t q_pad_bytes = 0; // rows padded to a 16-byte pitch (TMA)
    void* h_in = nullptr; size_t h_in_bytes = 0;   // device copy of host input
    float* h_vol = nullptr; size_t h_vol_bytes = 0;
    void* lent = nullptr; size_t lent_bytes = 0;   // caller-owned workspace (lamino_set_workspace)
    cudaStream_t copy_stream = nullptr;            // host pipeline: copies overlap kernels
    std::vector<cudaEvent_t> pipe_ev;              // host pipeline: chunk events

    lam::DirectCfg dcfg;           // backprojector (k_direct): 32 x 16 x 16 tile, TMA box
    lam::DirectCfg pcfg;           // direct projector (k_project): 32 x 8 x 32 tile
    bool filter_ok = false;        // Wp is a supported FFT length
    bool fourier_ok = false;       // Wf, Hf, M1..M3 supported and n even
    std::string fourier_why;

    // tracing
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Rec { std::string name; int a, b; };
    std::vector<Rec> recs;
    int ev_used = 0;

    std::string err;
};

namespace lam {

// error helpers -------------------------------------------------------------
int fail(lamino_plan_t p, int code, const char* fmt, ...);
int cuda_fail(lamino_plan_t p, cudaError_t e, const char* what);
void set_global_error(const char* msg);

#define LAM_CUDA(p, call)                                         \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return lam::cuda_fail((p), e_, #call); \
    } while (0)

#define LAM_LAUNCH_CHECK(p, what)                                 \
    do {                                                          \
        cudaError_t e_ = cudaGetLastError();                      \
        if (e_ != cudaSuccess) return lam::cuda_fail((p), e_, what); \
    } while (0)

int ensure_buffer(lamino_plan_t p, void** buf, size_t* have, size_t need, const char* what);
// Workspaces of the direct form: the filtered rows (lamino_fbp) and the copy of
// the projections at a 16-byte row pitch (TMA), from the caller's lent buffer
// (rows at 0, padded copy at lent_pad_offset) or plan-owned allocations.
int rows_buffer(lamino_plan_t p, float** q);
int pad_buffer(lamino_plan_t p, size_t need, float** q);
inline size_t lent_align(size_t b) { return (b + 255) / 256 * 256; }
int set_device(lamino_plan_t p);

// tracing: bracket a launch with events when profiling is on
void prof_begin(lamino_plan_t p, const char* name, cudaStream_t s);
void prof_end(lamino_plan_t p, cudaStream_t s);
struct ProfScope {
    lamino_plan_t p;
    cudaStream_t s;
    ProfScope(lamino_plan_t p_, const char* name, cudaStream_t s_) : p(p_), s(s_) { prof_begin(p, name, s); }
    ~ProfScope() { prof_end(p, s); }
};

// kernels' host launchers (defined in the .cu files) ---------------------------
// Row kernels take the detector rows [row0, row1) (row = k H + r; row1 < 0:
// all rows), so that a host pipeline can start on the projections already copied.
int launch_filter(lamino_plan_t p, const void* d, int dtype, float* q, int kind,
                  cudaStream_t s, long row0 = 0, long row1 = -1);
int validate_dtype_kind(lamino_plan_t p, int dtype, int kind);
int launch_rowfft(lamino_plan_t p, const void* d, int dtype, float2* R, int kind /* -1: no filter */,
                  cudaStream_t s, long row0 = 0, long row1 = -1);
// Views of the Fourier form's two workspaces A and B (fourier_bufs). R, the
// row spectra (frequencies m >= 0 only, [nproj][H][Wf/2]), and G, the
// plane-major half spectra (followed by the column FFT's chunk statistics
// st), are whole; V holds the x1-pass planes of one chunk of zc planes and P
// the deconvolved planes of all L planes.
//   zc == L (no z chunking): A = R, then V [L][n0][M2]; B = G + st, then P.
//   zc <  L: A = R, then P [L][n1][n0] followed by V [zc][n0][M2]; B = G + st
//            (G must outlive every plane chunk).
// The transpose (lamino_project) uses the same views in reverse order, with
// full row spectra in R ([nproj][H][Wf], the workspace is sized for them).
struct FourierBufs {
    float2 *R, *G, *st, *V, *P;
    int CH;    // columns per column-FFT block = statistics chunk
    int zc;    // planes per chunk (F3-F5)
};
int fourier_workspace(lamino_plan_t p, size_t* a_bytes, size_t* b_bytes);
FourierBufs fourier_bufs(lamino_plan_t p, void* a, void* b);
int colfft_chunk(lamino_plan_t p);
int plane_chunk(lamino_plan_t p);    // zc: planes per F3-F5 chunk (L when not chunked)

// The Fourier form after the row pass, stage by stage: column FFT of the
// projections [k0, k1), gridding + x1 inverse FFT of the planes [l0, l1) into
// V, x2 inverse FFT of those planes from V into P, and the x3 USFFT of the x2
// rows [i10, i11) of the volume. run_fourier_after_rows runs them all, plane
// chunk by plane chunk (F3-F5) and column chunk by column chunk (F6).
int launch_colfft(lamino_plan_t p, const FourierBufs& fb, int k0, int k1, cudaStream_t s);
int launch_grid(lamino_plan_t p, const FourierBufs& fb, int l0, int l1, cudaStream_t s);
int launch_colifft(lamino_plan_t p, const FourierBufs& fb, int l0, int l1, cudaStream_t s);
int launch_zusfft(lamino_plan_t p, const FourierBufs& fb, float* vol, int i10, int i11, cudaStream_t s);
int run_planes(lamino_plan_t p, const FourierBufs& fb, cudaStream_t s);   // F3-F5, all chunks
int run_fourier_after_rows(lamino_plan_t p, const FourierBufs& fb, float* vol, cudaStream_t s);
int launch_direct(lamino_plan_t p, const float* q, float* vol, cudaStream_t s);
int launch_project_direct(lamino_plan_t p, const float* vol, float* d, cudaStream_t s);
int launch_project_fourier(lamino_plan_t p, const FourierBufs& fb, const float* vol, float* d,
                           cudaStream_t s);

// device helpers --------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by s*i (s = +-1)
__device__ __forceinline__ float2 cmul_si(float2 a, float s) { return make_float2(-s * a.y, s * a.x); }

template <typename T> __device__ __forceinline__ float load_f(const T* p, size_t i);
template <> __device__ __forceinline__ float load_f<float>(const float* p, size_t i) { return __ldg(p + i); }
template <> __device__ __forceinline__ float load_f<__half>(const __half* p, size_t i) { return __half2float(p[i]); }
template <> __device__ __forceinline__ float load_f<__nv_bfloat16>(const __nv_bfloat16* p, size_t i) {
    return __bfloat162float(p[i]);
}

// DFT of length R in registers, exponent sign s (-1 forward, +1 inverse):
// X_k = sum_r v_r exp(s 2 pi i r k / R).
template <int R> __device__ __forceinline__ void bfly(float2* v, float s);

template <> __device__ __forceinline__ void bfly<2>(float2* v, float) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}
template <> __device__ __forceinline__ void bfly<3>(float2* v, float s) {
    const float h = 0.86602540378443864676f;  // sqrt(3)/2
    float2 t = cadd(v[1], v[2]);
    float2 u = cmul_si(csub(v[1], v[2]), s * h);
    float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, u);
    v[2] = csub(m, u);
}
template <> __device__ __forceinline__ void bfly<4>(float2* v, float s) {
    float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    float2 t2 = cadd(v[1], v[3]), t3 = cmul_si(csub(v[1], v[3]), s);
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
}
template <> __device__ __forceinline__ void bfly<8>(float2* v, float s) {
    // split into even / odd halves, two DFT4s, then combine with w8^k
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    bfly<4>(e, s);
    bfly<4>(o, s);
    const float r = 0.70710678118654752440f;
    // w8^1 = r (1 + s i), w8^2 = s i, w8^3 = r (-1 + s i)
    float2 o1 = make_float2(r * (o[1].x - s * o[1].y), r * (o[1].y + s * o[1].x));
    float2 o2 = cmul_si(o[2], s);
    float2 o3 = make_float2(r * (-o[3].x - s * o[3].y), r * (-o[3].y + s * o[3].x));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
}

// Storage views of one FFT sequence in shared memory: interleaved complex
// (float2) or planar (separate real and imaginary arrays).
struct SeqC {
    float2* p;
    __device__ __forceinline__ float2 ld(int i) const { return p[i]; }
    __device__ __forceinline__ void st(int i, float2 v) const { p[i] = v; }
};
// Interleaved complex with one empty slot after every 16 elements: the
// strided accesses of the first radix-8 / radix-4 Stockham stages then spread
// over all banks instead of 2-4 of them.
__device__ __forceinline__ int fpad(int i) { return i + (i >> 4); }
// slots a padded sequence of n elements occupies
__host__ __device__ constexpr int fpad_len(int n) { return n + ((n - 1) >> 4); }
struct SeqCP {
    float2* p;
    __device__ __forceinline__ float2 ld(int i) const { return p[fpad(i)]; }
    __device__ __forceinline__ void st(int i, float2 v) const { p[fpad(i)] = v; }
};
struct SeqP {
    float* re;
    float* im;
    __device__ __forceinline__ float2 ld(int i) const { return make_float2(re[i], im[i]); }
    __device__ __forceinline__ void st(int i, float2 v) const { re[i] = v.x; im[i] = v.y; }
};

// Barrier of the threads that share one FFT sequence: the whole block
// (mode 0), the warp (mode 1: groups of at most 32 threads) or named barrier
// 1 + gid over the group's T threads (mode 2). Every thread of the group
// reaches every call, active or not.
__device__ __forceinline__ void fft_sync(int mode, int gid, int T) {
    if (mode == 0) {
        __syncthreads();
    } else if (mode == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(T) : "memory");
    }
}

// One Stockham autosort stage of radix R on a sequence of length n held in
// shared memory (the decimation-in-time autosort formulation, see e.g.
// Govindaraju et al., SC 2008). Each of the t threads of the sequence stages
// its E/R butterflies' inputs in registers, the threads of the sequence
// synchronise (fft_sync), and the outputs are written back in place (the
// barrier separates all reads from all writes). Butterfly j reads
// x[j + r n/R]; with k = j mod ns it twiddles by exp(-+2 pi i k r/(ns R)),
// transforms and writes x[(j - k) R + k + r ns].
template <int E, int R, typename S>
__device__ __forceinline__ void fft_stage(S x, const FftDesc& f, int tid, bool active, int ns,
                                          float s, int smode = 0, int gid = 0, int gT = 0) {
    static_assert(E % R == 0, "radix must divide the elements per thread");
    float2 v[E];
    const int n = f.n, t = f.t, nr = n / R;
    if (active) {
#pragma unroll
        for (int i = 0; i < E / R; ++i) {
            int j = tid + i * t;
#pragma unroll
            for (int r = 0; r < R; ++r) v[i * R + r] = x.ld(j + r * nr);
        }
    }
    fft_sync(smode, gid, gT);
    if (active) {
        const int stride = n / (ns * R);
#pragma unroll
        for (int i = 0; i < E / R; ++i) {
            int j = tid + i * t;
            int k = j & (ns - 1);  // ns is a power of two
            if (ns > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    // table holds exp(-2 pi i u/n); the inverse uses its conjugate
                    float2 w = __ldg(f.tw + k * r * stride);
                    if (s > 0.f) w.y = -w.y;
                    v[i * R + r] = cmul(v[i * R + r], w);
                }
            }
            bfly<R>(&v[i * R], s);
            int d = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) x.st(d + r * ns, v[i * R + r]);
        }
    }
    fft_sync(smode, gid, gT);
}

// Complex FFT of the length-f.n sequence x (shared memory), exponent sign s.
// Must be called by every thread of the block (it synchronises); threads with
// active == false only take part in the barriers. Output is in natural order,
// unnormalised.
template <int E, typename S>
__device__ __forceinline__ void fft_run(S x, const FftDesc& f, int tid, bool active, float s,
                                        int smode = 0, int gid = 0, int gT = 0) {
    active = active && tid < f.t;
    int ns = 1;
    for (int st = 0; st < f.nst; ++st) {
        const int R = (f.rads >> (4 * st)) & 15u;
        if constexpr (E % 8 == 0) {
            if (R == 8) fft_stage<E, 8>(x, f, tid, active, ns, s, smode, gid, gT);
            else if (R == 4) fft_stage<E, 4>(x, f, tid, active, ns, s, smode, gid, gT);
            else fft_stage<E, 2>(x, f, tid, active, ns, s, smode, gid, gT);
        } else {
            if (R == 4) fft_stage<E, 4>(x, f, tid, active, ns, s, smode, gid, gT);
            else if (R == 2) fft_stage<E, 2>(x, f, tid, active, ns, s, smode, gid, gT);
            else fft_stage<E, 3>(x, f, tid, active, ns, s, smode, gid, gT);
        }
        ns *= R;
    }
}

// Barrier mode of fft_many: per-group barriers when the block splits into
// whole groups of T threads (at most 15 named barriers), else the block.
__device__ __forceinline__ int fft_group_mode(int T) {
    const int nb = blockDim.x;
    if (nb % T != 0 || nb % 32 != 0) return 0;
    if (T <= 32) return 1;
    return (nb / T <= 15) ? 2 : 0;
}

template <int E>
__device__ __forceinline__ void fft_run(float2* x, const FftDesc& f, int tid, bool active, float s) {
    fft_run<E>(SeqC{x}, f, tid, active, s);
}

// v * exp(s i a) for the angle a with cosine c and sine sn.
__device__ __forceinline__ float2 ctw(float2 v, float c, float sn, float s) {
    const float y = s * sn;
    return make_float2(v.x * c - v.y * y, v.x * y + v.y * c);
}

// DFT of length 16 in registers, exponent sign s, as 4 x 4: with n = 4a + b
// and k = c + 4d, X[c + 4d] = sum_b w4^(bd) w16^(bc) sum_a v[4a + b] w4^(ac),
// w_m = exp(s 2 pi i / m).
__device__ __forceinline__ void dft16(float2* v, float s) {
    const float c1 = 0.92387953251128675613f;   // cos(pi/8)
    const float c3 = 0.38268343236508977173f;   // cos(3pi/8)
    const float r = 0.70710678118654752440f;    // cos(pi/4)
    float2 A[4][4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        float2 u[4] = {v[b], v[4 + b], v[8 + b], v[12 + b]};
        bfly<4>(u, s);
#pragma unroll
        for (int c = 0; c < 4; ++c) A[b][c] = u[c];
    }
    // w16^(bc): angles pi bc / 8 for bc = 1, 2, 3, 4, 6, 9
    A[1][1] = ctw(A[1][1], c1, c3, s);
    A[1][2] = ctw(A[1][2], r, r, s);
    A[1][3] = ctw(A[1][3], c3, c1, s);
    A[2][1] = ctw(A[2][1], r, r, s);
    A[2][2] = cmul_si(A[2][2], s);
    A[2][3] = ctw(A[2][3], -r, r, s);
    A[3][1] = ctw(A[3][1], c3, c1, s);
    A[3][2] = ctw(A[3][2], -r, r, s);
    A[3][3] = ctw(A[3][3], -c1, -c3, s);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float2 u[4] = {A[0][c], A[1][c], A[2][c], A[3][c]};
        bfly<4>(u, s);
#pragma unroll
        for (int d = 0; d < 4; ++d) v[c + 4 * d] = u[d];
    }
}

// v[c] *= w^(u c) for c = 1..15, w = exp(s 2 pi i / n), from the table
// tw[j] = exp(-2 pi i j / n) (12 u < n): w^(u c) = tw[4 q u] tw[u]^r for
// c = 4q + r, four table loads and at most two products per twiddle (fewer
// live registers than fifteen loads).
__device__ __forceinline__ void twiddle16(float2* v, const float2* __restrict__ tw, int u, float s) {
    const float sg = (s > 0.f) ? -1.f : 1.f;
    float2 w1 = __ldg(tw + u);
    w1.y *= sg;
    const float2 w2 = cmul(w1, w1), w3 = cmul(w2, w1);
    v[1] = cmul(v[1], w1);
    v[2] = cmul(v[2], w2);
    v[3] = cmul(v[3], w3);
#pragma unroll
    for (int q = 1; q < 4; ++q) {
        float2 wq = __ldg(tw + 4 * q * u);
        wq.y *= sg;
        v[4 * q] = cmul(v[4 * q], wq);
        v[4 * q + 1] = cmul(v[4 * q + 1], cmul(wq, w1));
        v[4 * q + 2] = cmul(v[4 * q + 2], cmul(wq, w2));
        v[4 * q + 3] = cmul(v[4 * q + 3], cmul(wq, w3));
    }
}

// v[c] *= w^(u c) for c = 1..7, w = exp(s 2 pi i / n), from the table
// tw[j] = exp(-2 pi i j / n) (4 u < n): three table loads and four products.
__device__ __forceinline__ void twiddle8(float2* v, const float2* __restrict__ tw, int u, float s) {
    const float sg = (s > 0.f) ? -1.f : 1.f;
    float2 w1 = __ldg(tw + u), w2 = __ldg(tw + 2 * u), w4 = __ldg(tw + 4 * u);
    w1.y *= sg;
    w2.y *= sg;
    w4.y *= sg;
    const float2 w3 = cmul(w2, w1);
    v[1] = cmul(v[1], w1);
    v[2] = cmul(v[2], w2);
    v[3] = cmul(v[3], w3);
    v[4] = cmul(v[4], w4);
    v[5] = cmul(v[5], cmul(w4, w1));
    v[6] = cmul(v[6], cmul(w4, w2));
    v[7] = cmul(v[7], cmul(w4, w3));
}

// 256-point FFT of the sequence x (shared memory, natural order in and out,
// unnormalised, exponent sign s) by the 32 lanes of one warp: 256 = 8 x 32.
// With n = 32a + t and k = c + 8e,
//   X[c + 8e] = sum_t w32^(te) [w256^(tc) sum_a x[32a + t] w8^(ac)].
// Lane t takes the 8-point DFT over a and its twiddles; after a transpose
// through x (row c rotated by 4c slots, so that the column reads below hit
// 16 distinct 8-byte slots per half-warp), lane (c, r) = (lane / 4, lane % 4)
// takes the 8-point DFT D_r over the samples t = 4m + r of row c and the
// twiddles w32^(re); a radix-4 DFT over r between the lanes of a quad (two
// shuffle butterflies, as in fft1024_pair) gives X[c + 8e + 64q], lane r
// producing q = 2 (r % 2) + r / 2. tw: exp(-2 pi i u / 256), u in [0, 256).
template <typename S>
__device__ __forceinline__ void fft256_warp_s(S x, const float2* __restrict__ tw, float s, int lane) {
    float2 v[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) v[a] = x.ld(32 * a + lane);
    bfly<8>(v, s);
    twiddle8(v, tw, lane, s);
    __syncwarp();
#pragma unroll
    for (int c = 0; c < 8; ++c) x.st(32 * c + ((lane + 4 * c) & 31), v[c]);
    __syncwarp();
    const int c = lane >> 2, r = lane & 3;
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = x.ld(32 * c + ((4 * m + r + 4 * c) & 31));
    bfly<8>(v, s);
    twiddle8(v, tw, 8 * r, s);
    const int b1 = r >> 1, b0 = r & 1;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        float2 o;
        o.x = __shfl_xor_sync(0xffffffffu, v[e].x, 2);
        o.y = __shfl_xor_sync(0xffffffffu, v[e].y, 2);
        float2 t = b1 ? csub(o, v[e]) : cadd(v[e], o);
        if (b1 & b0) t = cmul_si(t, s);
        v[e] = t;
    }
    __syncwarp();   // every read of x precedes the writes below
    const int q = 2 * b0 + b1;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        float2 o;
        o.x = __shfl_xor_sync(0xffffffffu, v[e].x, 1);
        o.y = __shfl_xor_sync(0xffffffffu, v[e].y, 1);
        x.st(c + 8 * e + 64 * q, b0 ? csub(o, v[e]) : cadd(v[e], o));
    }
}

__device__ __forceinline__ void fft256_warp(float2* x, const float2* __restrict__ tw, float s, int lane) {
    fft256_warp_s(SeqC{x}, tw, s, lane);
}

// 512-point FFT of the sequence x (shared memory, natural order in and out,
// unnormalised, exponent sign s) by the 32 lanes of one warp: the four-step
// split 512 = 16 x 32. With n = 32a + t and k = c + 16e,
//   X[c + 16e] = sum_t w32^(te) [w512^(tc) sum_a x[32a + t] w16^(ac)].
// Lane t takes the inner 16-point DFT of column t and its twiddles; after one
// transpose through x itself, lane (c, p) = (lane / 2, lane % 2) takes the
// 16-point DFT over the samples t = 2m + p of row c, and a radix-2 exchange
// between the two lanes of a pair (shuffles) completes the 32-point DFT over t:
// X[c + 16e + 256p] = E[e] + (-1)^p w32^e O[e]. Two shared-memory round trips
// instead of one per radix-8 stage, and only warp barriers. The transpose
// rotates row c by 2c slots so that its row writes and its column reads both
// take the minimum two wavefronts. tw: exp(-2 pi i u / 512), u in [0, 512).
template <typename S>
__device__ __forceinline__ void fft512_warp_s(S x, const float2* __restrict__ tw, float s, int lane) {
    float2 v[16];
#pragma unroll
    for (int a = 0; a < 16; ++a) v[a] = x.ld(32 * a + lane);
    dft16(v, s);
    twiddle16(v, tw, lane, s);
    __syncwarp();
#pragma unroll
    for (int c = 0; c < 16; ++c) x.st(32 * c + ((lane + 2 * c) & 31), v[c]);
    __syncwarp();
    const int c = lane >> 1, p = lane & 1;
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = x.ld(32 * c + ((2 * m + p + 2 * c) & 31));
    dft16(v, s);
    // odd lanes: w32^e, cos and sin of pi e / 16
    const float a1 = 0.98078528040323044913f, a3 = 0.83146961230254523708f;
    const float a5 = 0.55557023301960222474f, a7 = 0.19509032201612826785f;
    const float c1 = 0.92387953251128675613f, c3 = 0.38268343236508977173f;
    const float r = 0.70710678118654752440f;
    if (p) {
        v[1] = ctw(v[1], a1, a7, s);
        v[2] = ctw(v[2], c1, c3, s);
        v[3] = ctw(v[3], a3, a5, s);
        v[4] = ctw(v[4], r, r, s);
        v[5] = ctw(v[5], a5, a3, s);
        v[6] = ctw(v[6], c3, c1, s);
        v[7] = ctw(v[7], a7, a1, s);
        v[8] = cmul_si(v[8], s);
        v[9] = ctw(v[9], -a7, a1, s);
        v[10] = ctw(v[10], -c3, c1, s);
        v[11] = ctw(v[11], -a5, a3, s);
        v[12] = ctw(v[12], -r, r, s);
        v[13] = ctw(v[13], -a3, a5, s);
        v[14] = ctw(v[14], -c1, c3, s);
        v[15] = ctw(v[15], -a1, a7, s);
    }
    __syncwarp();
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        float2 o;
        o.x = __shfl_xor_sync(0xffffffffu, v[e].x, 1);
        o.y = __shfl_xor_sync(0xffffffffu, v[e].y, 1);
        x.st(c + 16 * e + 256 * p, p ? csub(o, v[e]) : cadd(v[e], o));
    }
}

__device__ __forceinline__ void fft512_warp(float2* x, const float2* __restrict__ tw, float s, int lane) {
    fft512_warp_s(SeqC{x}, tw, s, lane);
}

// 1024-point FFT of the sequence x (as fft512_warp) by the 64 threads of one
// pair of warps, tid in [0, 64), synchronised on named barrier bar (64
// threads): 1024 = 16 x 64. With n = 64a + t and k = c + 16e,
//   X[c + 16e] = sum_t w64^(te) [w1024^(tc) sum_a x[64a + t] w16^(ac)].
// Thread t takes the inner 16-point DFT of column t and its twiddles; after a
// transpose through x (row c rotated by 4c slots), thread (c, r) = (tid / 4,
// tid % 4) takes the 16-point DFT D_r over the samples t = 4m + r of row c and
// its twiddles w64^(re); the radix-4 DFT over r between the four lanes of a
// quad (two shuffle butterflies) gives X[c + 16e + 256q] = sum_r w4^(rq)
// w64^(re) D_r[e], lane r producing q = 2 (r % 2) + r / 2.
// The sequence is any storage view (SeqC, SeqP); the pair synchronises with
// fft_sync(smode, gid, 64), i.e. named barrier 1 + gid, or the whole block
// (smode 0) when every pair of the block runs one sequence in step. A pair
// with active == false touches no memory and only takes part in the barriers.
// With swz, output k is stored at k ^ (((k >> 8) & 3) << 3) (fft1024_pos):
// the last stores of a warp then fill all 32 banks of 4-byte words instead of
// 8 (four quads' q outputs share their low five bits), which pays for planar
// sequences.
template <typename S>
__device__ __forceinline__ void fft1024_pair_s(S x, const float2* __restrict__ tw, float s, int tid,
                                               int smode, int gid, bool active = true, bool swz = false) {
    float2 v[16];
#pragma unroll
    for (int a = 0; a < 16; ++a) v[a] = active ? x.ld(64 * a + tid) : make_float2(0.f, 0.f);
    dft16(v, s);
    twiddle16(v, tw, tid, s);
    fft_sync(smode, gid, 64);
#pragma unroll
    for (int c = 0; c < 16; ++c)
        if (active) x.st(64 * c + ((tid + 4 * c) & 63), v[c]);
    fft_sync(smode, gid, 64);
    const int c = tid >> 2, r = tid & 3;
#pragma unroll
    for (int m = 0; m < 16; ++m)
        v[m] = active ? x.ld(64 * c + ((4 * m + r + 4 * c) & 63)) : make_float2(0.f, 0.f);
    dft16(v, s);
    twiddle16(v, tw, 16 * r, s);
    const int b1 = r >> 1, b0 = r & 1;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        // butterfly over r and r ^ 2; lane 3 then takes the w4 factor
        float2 o;
        o.x = __shfl_xor_sync(0xffffffffu, v[e].x, 2);
        o.y = __shfl_xor_sync(0xffffffffu, v[e].y, 2);
        float2 a = b1 ? csub(o, v[e]) : cadd(v[e], o);
        if (b1 & b0) a = cmul_si(a, s);
        v[e] = a;
    }
    fft_sync(smode, gid, 64);   // every read of x precedes the writes below
    const int q = 2 * b0 + b1;
    const int xo = swz ? (q << 3) : 0;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        float2 o;
        o.x = __shfl_xor_sync(0xffffffffu, v[e].x, 1);
        o.y = __shfl_xor_sync(0xffffffffu, v[e].y, 1);
        if (active) x.st((c + 16 * e + 256 * q) ^ xo, b0 ? csub(o, v[e]) : cadd(v[e], o));
    }
}

__device__ __forceinline__ void fft1024_pair(float2* x, const float2* __restrict__ tw, float s, int tid,
                                             int bar) {
    fft1024_pair_s(SeqC{x}, tw, s, tid, 2, bar - 1);
}

// FFTs of nseq sequences at base + i*ld with every thread of the block: groups
// of blockDim/f.t sequences run side by side (blockDim must be >= f.t). Length
// 512 goes one sequence per warp (fft512_warp) when blockDim is whole warps,
// length 1024 one per pair of warps (fft1024_pair) when blockDim is whole
// pairs and at most 15 of them (named barriers 1..15). Ends with a block-wide
// barrier.
template <int E>
__device__ __forceinline__ void fft_many(float2* base, int ld, int nseq, const FftDesc& f, float s) {
    if constexpr (E == 8) {
        if (f.n == 512 && (blockDim.x & 31) == 0) {
            const int lane = threadIdx.x & 31;
            for (int seq = threadIdx.x >> 5; seq < nseq; seq += blockDim.x >> 5)
                fft512_warp(base + (size_t)seq * ld, f.tw, s, lane);
            __syncthreads();
            return;
        }
        if (f.n == 1024 && (blockDim.x & 63) == 0 && blockDim.x <= 15 * 64) {
            const int g = threadIdx.x >> 6, tid = threadIdx.x & 63;
            for (int seq = g; seq < nseq; seq += blockDim.x >> 6)
                fft1024_pair(base + (size_t)seq * ld, f.tw, s, tid, g + 1);
            __syncthreads();
            return;
        }
    }
    const int T = f.t;
    const int par = blockDim.x / T;
    if (par == 0) return;   // a sequence needs more threads than the block has (the plan refuses this)
    const int g = threadIdx.x / T;
    const int mode = fft_group_mode(T);
    for (int s0 = 0; s0 < nseq; s0 += par) {
        const int seq = s0 + g;
        fft_run<E>(SeqC{base + (size_t)min(seq, nseq - 1) * ld}, f, threadIdx.x % T,
                   g < par && seq < nseq, s, mode, g, T);
    }
    if (mode != 0) __syncthreads();
}

// Whether fft_many_planar<E> takes the pair path for f (see below).
template <int E>
__device__ __forceinline__ bool fft_planar_pair(const FftDesc& f) {
    return E == 8 && f.n == 1024 && (blockDim.x & 63) == 0;
}
// Where output i of fft_many_planar<E>(..., swz) sits in its sequence.
template <int E>
__device__ __forceinline__ int fft_planar_pos(const FftDesc& f, int i, bool swz) {
    return (swz && fft_planar_pair<E>(f)) ? i ^ (((i >> 8) & 3) << 3) : i;
}

// The same for planar sequences re + i*ld, im + i*ld: lengths 256 and 512
// one sequence per warp, 1024 one per pair of warps (named barriers for at
// most 15 pairs, else block barriers with every pair in step, idle pairs
// taking part in the barriers only; outputs permuted as fft_planar_pos says
// when swz). Ends with a block-wide barrier.
template <int E>
__device__ __forceinline__ void fft_many_planar(float* re, float* im, int ld, int nseq,
                                                const FftDesc& f, float s, bool swz = false) {
    if constexpr (E == 8) {
        if ((f.n == 256 || f.n == 512) && (blockDim.x & 31) == 0) {
            const int lane = threadIdx.x & 31;
            for (int seq = threadIdx.x >> 5; seq < nseq; seq += blockDim.x >> 5) {
                const size_t o = (size_t)seq * ld;
                if (f.n == 256) fft256_warp_s(SeqP{re + o, im + o}, f.tw, s, lane);
                else fft512_warp_s(SeqP{re + o, im + o}, f.tw, s, lane);
            }
            __syncthreads();
            return;
        }
        if (fft_planar_pair<E>(f)) {
            const int np = blockDim.x >> 6, g = threadIdx.x >> 6, tid = threadIdx.x & 63;
            const int mode = (np <= 15) ? 2 : 0;
            for (int s0 = 0; s0 < nseq; s0 += np) {
                const size_t o = (size_t)min(s0 + g, nseq - 1) * ld;
                fft1024_pair_s(SeqP{re + o, im + o}, f.tw, s, tid, mode, g, s0 + g < nseq, swz);
            }
            __syncthreads();
            return;
        }
    }
    const int T = f.t;
    const int par = blockDim.x / T;
    if (par == 0) return;   // a sequence needs more threads than the block has (the plan refuses this)
    const int g = threadIdx.x / T;
    const int mode = fft_group_mode(T);
    for (int s0 = 0; s0 < nseq; s0 += par) {
        const size_t o = (size_t)min(s0 + g, nseq - 1) * ld;
        fft_run<E>(SeqP{re + o, im + o}, f, threadIdx.x % T, g < par && s0 + g < nseq, s, mode, g, T);
    }
    if (mode != 0) __syncthreads();
}

}  // namespace lam
