// Plan object and C ABI entry points of the laminographic FBP library.
//
// lamino_plan computes, on the host in double precision, everything that
// depends only on the geometry (Nikitin et al., Sec. 4): trigonometric node
// tables of the rotation angles, the filter transfer function |f| cos(phi) w(f),
// the detector-centring phases of the Fourier form, the Gaussian-kernel
// deconvolution factors of the USFFT (one per axis) and the fixed x3 gridding
// table, and uploads them once as float32. Kernels only read these tables.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"

namespace {

std::string g_last_error;  // failures of lamino_plan (no plan to hold them)
const double kPi = 3.14159265358979323846;

bool is_pow2(long n) { return n > 0 && (n & (n - 1)) == 0; }

}  // namespace

namespace lam {

void set_global_error(const char* msg) { g_last_error = msg; }

int fail(lamino_plan_t p, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (p) p->err = buf; else g_last_error = buf;
    return code;
}

int cuda_fail(lamino_plan_t p, cudaError_t e, const char* what) {
    int code = (e == cudaErrorMemoryAllocation) ? LAMINO_ENOMEM : LAMINO_ECUDA;
    return fail(p, code, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

int set_device(lamino_plan_t p) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != p->device) {
        LAM_CUDA(p, cudaSetDevice(p->device));
    }
    return LAMINO_OK;
}

int ensure_buffer(lamino_plan_t p, void** buf, size_t* have, size_t need, const char* what) {
    if (*buf && *have >= need) return LAMINO_OK;
    if (*buf) {
        cudaFree(*buf);
        *buf = nullptr;
        *have = 0;
    }
    if (need == 0) return LAMINO_OK;
    cudaError_t e = cudaMalloc(buf, need);
    if (e != cudaSuccess) {
        *buf = nullptr;
        cudaGetLastError();
        return fail(p, LAMINO_ENOMEM, "cudaMalloc of %zu bytes for %s failed: %s", need, what,
                    cudaGetErrorString(e));
    }
    *have = need;
    return LAMINO_OK;
}

static cudaEvent_t prof_event(lamino_plan_t p) {
    if (p->ev_used >= (int)p->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        p->ev_pool.push_back(e);
    }
    return p->ev_pool[p->ev_used++];
}

void prof_begin(lamino_plan_t p, const char* name, cudaStream_t s) {
    if (!p->profiling) return;
    cudaEvent_t e = prof_event(p);
    if (!e) return;
    cudaEventRecord(e, s);
    p->recs.push_back({name, p->ev_used - 1, -1});
}

void prof_end(lamino_plan_t p, cudaStream_t s) {
    if (!p->profiling || p->recs.empty() || p->recs.back().b >= 0) return;
    cudaEvent_t e = prof_event(p);
    if (!e) return;
    cudaEventRecord(e, s);
    p->recs.back().b = p->ev_used - 1;
}

int fft_elems(int n) { return (n % 3 == 0) ? 12 : 8; }

bool fft_len_ok(int n) {
    if (n <= 0 || n > kMaxFft) return false;
    if (is_pow2(n)) return n >= 8 && n / 8 <= kMaxFftThreads;
    return n % 3 == 0 && is_pow2(n / 3) && n >= 12 && n / 12 <= kMaxFftThreads;
}

int fft_size_at_least(double n) {
    long best = -1;
    for (long p = 1; p <= (1L << 40); p <<= 1) {
        if (p >= n && (best < 0 || p < best)) best = p;
        if (3 * p >= n && (best < 0 || 3 * p < best)) best = 3 * p;
        if (p >= n) break;
    }
    return (int)std::min<long>(best, 1L << 30);
}

}  // namespace lam

using namespace lam;

namespace {

// Radix schedule. 2^k (k >= 3, 8 elements per thread): radix-8 stages and one
// radix-4 or radix-2 stage for k mod 3 = 2 or 1. 3*2^k (k >= 2, 12 per
// thread): radix-4 stages, a radix-2 stage if k is odd, then one radix-3 stage.
FftDesc make_desc(int n) {
    FftDesc f;
    f.n = n;
    f.e = fft_elems(n);
    f.t = n / f.e;
    int k = 0;
    for (int m = (n % 3 == 0) ? n / 3 : n; m > 1; m >>= 1) ++k;
    auto push = [&](unsigned r) { f.rads |= r << (4 * f.nst++); };
    if (n % 3 == 0) {
        for (; k >= 2; k -= 2) push(4);
        if (k == 1) push(2);
        push(3);
    } else {
        for (int i = 0; i < k / 3; ++i) push(8);
        if (k % 3 == 2) push(4);
        if (k % 3 == 1) push(2);
    }
    return f;
}

// Gaussian spreading width (grid cells^2) of the USFFT for half-width w and
// oversampling R = M/n: the choice that balances the truncation of the
// kernel at w cells against the aliasing of the grid (fast Gaussian gridding,
// Greengard & Lee, SIAM Rev. 46 (2004)), written in cells: t = w R /(4 pi (R - 1/2)).
double gauss_t(int w, double R) { return w * R / (4.0 * kPi * (R - 0.5)); }

// Error model of the Gaussian USFFT along one axis of n voxels on an M-cell
// grid with half-width w, as a mean square over the voxels. After the
// deconvolution by psi(x), voxel x carries two relative errors: the kernel's
// truncation at w cells, exp(-w^2/(4t)) amplified by 1/psi(x) ~ exp(4 pi^2 t
// (x/M)^2), and the aliasing of the first image of the grid, psi(M - |x|) /
// psi(x) = exp(-4 pi^2 t (1 - 2|x|/M)). With t from gauss_t both equal
// exp(-pi w (R - 1)/(R - 1/2)) at the edge |x| = n/2 (2.3e-4 for w = 4, R = 2)
// and fall off inside, so small axes (a larger share of voxels near the
// edge) and R = 2 exactly (no spare oversampling) fare worst.
double usfft_axis_err2(int n, int M, int w) {
    const double t = gauss_t(w, (double)M / n), c = 4.0 * kPi * kPi * t;
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
        const double u = fabs((double)(i - n / 2)) / M;
        const double e = exp(-w * (double)w / (4.0 * t) + c * u * u) + exp(-c * (1.0 - 2.0 * u));
        s += e * e;
    }
    return s / n;
}

// Predicted relative L2 error of the Fourier form against the exact type-1
// sum for a volume whose energy is spread evenly over the voxels (random
// projections: the worst of the parity workloads). The root of the summed
// axis models overestimates the measured FP32 error; measured / model was
// 0.35-0.36 on random projections (8x8x8: 7.3e-5, 8x8x256: 1.02e-4,
// 16x16x256: 8.8e-5 at w = 4), and that calibration is folded in here.
constexpr double kErrCalib = 0.36;
double usfft_err_est(int n0, int n1, int n2, int M1, int M2, int M3, int w, int wz) {
    return kErrCalib * sqrt(usfft_axis_err2(n0, M1, w) + usfft_axis_err2(n1, M2, w) +
                            usfft_axis_err2(n2, M3, wz));
}

// Half-widths the plan uses unless the caller sets them: the smallest
// w in [4, 8] whose predicted error stays below kErrTarget (w = 4 for axes of
// 24 voxels or more at R = 2, w = 5 for the smallest grids), and along x3 the
// smallest wz whose axis term alone stays below 5 % of that (wz = 6; the x3
// pass is cheap: 2 wz taps per plane and cell).
constexpr double kErrTarget = 0.9e-4;
void choose_widths(lamino_plan_t p, bool fix_w, bool fix_wz) {
    if (!fix_wz) {
        p->wz = 4;
        while (p->wz < 8 && kErrCalib * sqrt(usfft_axis_err2(p->n2, p->M3, p->wz)) > 0.05 * kErrTarget) ++p->wz;
    }
    if (!fix_w) {
        p->w = 4;
        while (p->w < 8 && usfft_err_est(p->n0, p->n1, p->n2, p->M1, p->M2, p->M3, p->w, p->wz) > kErrTarget)
            ++p->w;
    }
}

// Deconvolution factor of one axis: the spread kernel exp(-d^2/(4t)) (d in
// cells) has the continuous Fourier transform psi(x) = sqrt(4 pi t)/M *
// exp(-4 pi^2 t (x/M)^2) at integer x; dividing the inverse DFT of the grid by
// M psi(x) recovers the type-1 sum (Sec. 4, USFFT step "division by psi").
std::vector<float> deconv(int n, int M, double t, double scale) {
    std::vector<float> d(n);
    for (int i = 0; i < n; ++i) {
        double x = i - n / 2;
        d[i] = (float)(scale * exp(4.0 * kPi * kPi * t * (x / M) * (x / M)) / sqrt(4.0 * kPi * t));
    }
    return d;
}

double window(double f, int kind) {
    double af = fabs(f);
    if (kind == LAMINO_SHEPP) return af == 0.0 ? 1.0 : sin(kPi * f) / (kPi * f);
    if (kind == LAMINO_PARZEN) {
        double z = af / 0.5;
        if (z <= 0.5) return 1 - 6 * z * z + 6 * z * z * z;
        if (z <= 1.0) return 2 * (1 - z) * (1 - z) * (1 - z);
        return 0.0;
    }
    return 1.0;
}

template <typename T>
int upload(lamino_plan_t p, T** dst, const std::vector<T>& v, const char* what) {
    size_t bytes = sizeof(T) * std::max<size_t>(v.size(), 1);
    cudaError_t e = cudaMalloc((void**)dst, bytes);
    if (e != cudaSuccess) return cuda_fail(p, e, what);
    p->table_bytes += bytes;
    if (!v.empty()) {
        e = cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(p, e, what);
    }
    return LAMINO_OK;
}

void free_plan(lamino_plan_t p) {
    void* bufs[] = {p->d_trig, p->d_trig64, p->d_filt, p->d_phu, p->d_phv, p->d_dec1,
                    p->d_dec2, p->d_dec3, p->d_zoff, p->d_zl, p->d_zw, p->d_zrange, p->d_zwt,
                    p->d_ztap, p->d_tw, p->d_err,
                    p->ws_a, p->ws_b, p->q_buf, p->q_pad, p->h_in, p->h_vol};
    for (void* b : bufs)
        if (b) cudaFree(b);
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : p->pipe_ev) cudaEventDestroy(e);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    delete p;
}

int build_tables(lamino_plan_t p) {
    const int nproj = p->nproj;
    // angle tables
    std::vector<float2> trig(nproj);
    std::vector<double> trig64(2 * nproj);
    for (int k = 0; k < nproj; ++k) {
        double c = cos(p->theta[k]), s = sin(p->theta[k]);
        trig[k] = make_float2((float)c, (float)s);
        trig64[2 * k] = c;
        trig64[2 * k + 1] = s;
    }
    int rc;
    if ((rc = upload(p, &p->d_trig, trig, "trig table"))) return rc;
    if ((rc = upload(p, &p->d_trig64, trig64, "trig64 table"))) return rc;

    // filter H(f)/Wp per kind, FFT order (the 1/Wp of the inverse DFT folded in)
    std::vector<float> filt(3 * (size_t)p->Wp);
    for (int kind = 0; kind < 3; ++kind)
        for (int j = 0; j < p->Wp; ++j) {
            double f = (double)(j < p->Wp / 2 ? j : j - p->Wp) / p->Wp;
            filt[(size_t)kind * p->Wp + j] =
                (float)(fabs(f) * cos(p->tilt) * window(f, kind) / p->Wp);
        }
    if ((rc = upload(p, &p->d_filt, filt, "filter table"))) return rc;

    // error word
    {
        cudaError_t e = cudaMalloc((void**)&p->d_err, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(p, e, "error word");
        e = cudaMemset(p->d_err, 0, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(p, e, "error word");
    }

    // FFT twiddles exp(-2 pi i s/n) of every length in use, computed in double
    std::vector<int> lens = {p->Wp, p->Wf, p->Hf, p->M1, p->M2, p->M3};
    // the decimated-by-3 row kernels use 256- and 512-point tables for Wp, Wf = 3 x 256 or 3 x 512
    for (int n : {p->Wp, p->Wf})
        if (n % 3 == 0 && (n / 3 == 256 || n / 3 == 512)) lens.push_back(n / 3);
    std::vector<int> uniq;
    for (int n : lens)
        if (fft_len_ok(n) && std::find(uniq.begin(), uniq.end(), n) == uniq.end()) uniq.push_back(n);
    std::vector<float2> tw;
    std::vector<size_t> off;
    for (int n : uniq) {
        off.push_back(tw.size());
        for (int s = 0; s < n; ++s) {
            double a = -2.0 * kPi * s / n;
            tw.push_back(make_float2((float)cos(a), (float)sin(a)));
        }
    }
    if ((rc = upload(p, &p->d_tw, tw, "twiddle tables"))) return rc;
    auto desc_for = [&](int n) {
        if (!fft_len_ok(n)) return FftDesc();
        FftDesc f = make_desc(n);
        size_t i = std::find(uniq.begin(), uniq.end(), n) - uniq.begin();
        f.tw = p->d_tw + off[i];
        return f;
    };
    p->fWp = desc_for(p->Wp);
    p->fWf = desc_for(p->Wf);
    p->fHf = desc_for(p->Hf);
    p->fM1 = desc_for(p->M1);
    p->fM2 = desc_for(p->M2);
    p->fM3 = desc_for(p->M3);
    p->fWp3 = (p->Wp % 3 == 0 && (p->Wp / 3 == 256 || p->Wp / 3 == 512)) ? desc_for(p->Wp / 3) : FftDesc();
    p->fWf3 = (p->Wf % 3 == 0 && (p->Wf / 3 == 256 || p->Wf / 3 == 512)) ? desc_for(p->Wf / 3) : FftDesc();

    // centring phases: data sit at padded column j' = j + offu, so the type-1 sum
    // carries exp(2 pi i m cu / Wf), cu = W/2 + offu (and likewise for rows);
    // the Nyquist column m = -Wf/2 is dropped (weight 0).
    const double cu = p->W / 2.0 + p->offu, cv = p->H / 2.0 + p->offv;
    std::vector<float2> phu(p->Wf), phv(p->L);
    for (int mi = 0; mi < p->Wf; ++mi) {
        int m = mi - p->Wf / 2;
        double a = 2.0 * kPi * m * cu / p->Wf;
        phu[mi] = (mi == 0) ? make_float2(0.f, 0.f) : make_float2((float)cos(a), (float)sin(a));
    }
    for (int l = 0; l < p->L; ++l) {
        double a = 2.0 * kPi * l * cv / p->Hf;
        phv[l] = make_float2((float)cos(a), (float)sin(a));
    }
    if ((rc = upload(p, &p->d_phu, phu, "phase table u"))) return rc;
    if ((rc = upload(p, &p->d_phv, phv, "phase table v"))) return rc;

    // deconvolution factors; the global scale (pi/Ntheta)/(Wf Hf) rides on x3
    const double scale = (kPi / nproj) / ((double)p->Wf * p->Hf);
    if ((rc = upload(p, &p->d_dec1, deconv(p->n0, p->M1, p->t1, 1.0), "deconv x1"))) return rc;
    if ((rc = upload(p, &p->d_dec2, deconv(p->n1, p->M2, p->t2, 1.0), "deconv x2"))) return rc;
    if ((rc = upload(p, &p->d_dec3, deconv(p->n2, p->M3, p->t3, scale), "deconv x3"))) return rc;

    // x3 gridding table: plane l sits at Z_l = M3 l cos(phi)/Hf cells and carries
    // the Hermitian factor c_l (1 for l = 0, 2 otherwise: planes -l are the
    // conjugates of planes l). Every cell lists its (l, weight) taps.
    std::vector<std::vector<std::pair<int, float>>> cells(p->M3);
    std::vector<int2> ztap((size_t)p->L * 2 * p->wz);
    for (int l = 0; l < p->L; ++l) {
        double Z = (double)p->M3 * l * cos(p->tilt) / p->Hf;
        long fz = (long)floor(Z);
        double cl = (l == 0) ? 1.0 : 2.0;
        for (long s = fz - p->wz + 1; s <= fz + p->wz; ++s) {
            double dd = s - Z;
            double wgt = cl * exp(-dd * dd / (4.0 * p->t3));
            long cell = ((s % p->M3) + p->M3) % p->M3;
            cells[cell].push_back({l, (float)wgt});
            float fw = (float)wgt;
            int bits;
            memcpy(&bits, &fw, sizeof bits);
            ztap[(size_t)l * 2 * p->wz + (s - (fz - p->wz + 1))] = make_int2((int)cell, bits);
        }
    }
    std::vector<int> zoff(p->M3 + 1, 0), zl;
    std::vector<float> zw;
    int zmax = 0;
    for (int c = 0; c < p->M3; ++c) {
        zoff[c] = (int)zl.size();
        zmax = std::max(zmax, (int)cells[c].size());
        for (auto& t : cells[c]) {
            zl.push_back(t.first);
            zw.push_back(t.second);
        }
    }
    zoff[p->M3] = (int)zl.size();
    p->zmax = zmax;
    // When every cell's planes are consecutive (always but for x3 grids of a
    // few cells, where a cell can see both images of the periodic grid), the
    // x3 pass reads (first plane, count) per cell and the weights tap-major,
    // so that the lanes of a warp (consecutive cells) read consecutive words.
    bool consecutive = true;
    for (int c = 0; c < p->M3 && consecutive; ++c)
        for (size_t t = 1; t < cells[c].size(); ++t)
            if (cells[c][t].first != cells[c][0].first + (int)t) consecutive = false;
    if (consecutive) {
        std::vector<int2> zrange(p->M3);
        std::vector<float> zwt((size_t)std::max(zmax, 1) * p->M3, 0.f);
        for (int c = 0; c < p->M3; ++c) {
            zrange[c] = make_int2(cells[c].empty() ? 0 : cells[c][0].first, (int)cells[c].size());
            for (size_t t = 0; t < cells[c].size(); ++t) zwt[t * p->M3 + c] = cells[c][t].second;
        }
        if ((rc = upload(p, &p->d_zrange, zrange, "x3 table ranges"))) return rc;
        if ((rc = upload(p, &p->d_zwt, zwt, "x3 table weights by tap"))) return rc;
    }
    if ((rc = upload(p, &p->d_zoff, zoff, "x3 table offsets"))) return rc;
    if ((rc = upload(p, &p->d_zl, zl, "x3 table planes"))) return rc;
    if ((rc = upload(p, &p->d_zw, zw, "x3 table weights"))) return rc;
    if ((rc = upload(p, &p->d_ztap, ztap, "x3 table by plane"))) return rc;
    return LAMINO_OK;
}

// TMA box of the direct backprojector: the detector footprint of one voxel
// tile (tx x ty columns, tz slices) at any angle, plus the bilinear
// neighbour, one guard column/row before the footprint, and alignment slack
// of the box start (x rounded down to a multiple of 4).
void box_for(DirectCfg& c, double tilt) {
    double diag = sqrt((double)(c.tx - 1) * (c.tx - 1) + (double)(c.ty - 1) * (c.ty - 1));
    int need_w = (int)floor(diag) + 1 /*guard*/ + 2 /*floor+neighbour*/ + 3 /*align*/ + 1;
    c.bw = (need_w + 3) / 4 * 4;
    // row pitch = 12 or 20 mod 32 words: rows 1..7 apart fall in different banks
    while (c.bw % 32 != 12 && c.bw % 32 != 20) c.bw += 4;
    double span_r = fabs(sin(tilt)) * diag + cos(tilt) * (c.tz - 1);
    c.bh = (int)floor(span_r) + 1 /*guard*/ + 2 /*floor+neighbour*/ + 2;
}

void direct_config(lamino_plan_t p) {
    p->dcfg = DirectCfg();                      // 32 x 16 x 32
    p->dcfg.tz = 32;
    box_for(p->dcfg, p->tilt);
    p->pcfg = DirectCfg();
    p->pcfg.ty = 8;
    p->pcfg.tz = 32;
    box_for(p->pcfg, p->tilt);
}

}  // namespace

namespace lam {

int validate_dtype_kind(lamino_plan_t p, int dtype, int kind) {
    if (dtype != LAMINO_F32 && dtype != LAMINO_F16 && dtype != LAMINO_BF16)
        return fail(p, LAMINO_EINVAL, "unknown dtype %d", dtype);
    if (kind != LAMINO_RAMP && kind != LAMINO_SHEPP && kind != LAMINO_PARZEN)
        return fail(p, LAMINO_EINVAL, "unknown filter kind %d", kind);
    return LAMINO_OK;
}

// The plan's two Fourier workspaces for its current z chunking: views of the
// caller's lent buffer (A at 0, B 256-byte aligned after it), or plan-owned
// buffers allocated (or kept) here.
int fourier_buffers(lamino_plan_t p, FourierBufs* fb) {
    size_t a, b;
    fourier_workspace(p, &a, &b);
    if (p->lent) {
        const size_t need = lent_align(a) + b;
        if (need > p->lent_bytes)
            return fail(p, LAMINO_ENOMEM, "the lent workspace holds %zu bytes; the Fourier form needs %zu",
                        p->lent_bytes, need);
        *fb = fourier_bufs(p, p->lent, static_cast<char*>(p->lent) + lent_align(a));
        return LAMINO_OK;
    }
    int rc = ensure_buffer(p, &p->ws_a, &p->ws_a_bytes, a, "Fourier workspace A");
    if (rc) return rc;
    if ((rc = ensure_buffer(p, &p->ws_b, &p->ws_b_bytes, b, "Fourier workspace B"))) return rc;
    *fb = fourier_bufs(p, p->ws_a, p->ws_b);
    return LAMINO_OK;
}

int rows_buffer(lamino_plan_t p, float** q) {
    const size_t need = sizeof(float) * (size_t)p->nproj * p->H * p->W;
    if (p->lent) {
        if (need > p->lent_bytes)
            return fail(p, LAMINO_ENOMEM, "the lent workspace holds %zu bytes; the filtered rows need %zu",
                        p->lent_bytes, need);
        *q = static_cast<float*>(p->lent);
        return LAMINO_OK;
    }
    int rc = ensure_buffer(p, (void**)&p->q_buf, &p->q_buf_bytes, need, "filtered rows");
    *q = p->q_buf;
    return rc;
}

int pad_buffer(lamino_plan_t p, size_t need, float** q) {
    if (p->lent) {
        const size_t off = lent_align(sizeof(float) * (size_t)p->nproj * p->H * p->W);
        if (off + need > p->lent_bytes)
            return fail(p, LAMINO_ENOMEM, "the lent workspace holds %zu bytes; the padded projections "
                        "need %zu", p->lent_bytes, off + need);
        *q = reinterpret_cast<float*>(static_cast<char*>(p->lent) + off);
        return LAMINO_OK;
    }
    int rc = ensure_buffer(p, (void**)&p->q_pad, &p->q_pad_bytes, need, "padded projections");
    *q = p->q_pad;
    return rc;
}

}  // namespace lam

extern "C" {

int lamino_plan(lamino_plan_t* out, int n0, int n1, int n2, int nproj, int det_w, int det_h,
                double tilt, const double* angles, const lamino_opts* opts) {
    if (!out) return fail(nullptr, LAMINO_EINVAL, "lamino_plan: out is NULL");
    *out = nullptr;
    if (n0 < 1 || n1 < 1 || n2 < 1 || n0 > 8192 || n1 > 8192 || n2 > 8192)
        return fail(nullptr, LAMINO_EINVAL, "volume size %dx%dx%d out of range [1, 8192]", n0, n1, n2);
    if (nproj < 1 || nproj > (1 << 20))
        return fail(nullptr, LAMINO_EINVAL, "nproj %d out of range", nproj);
    if (det_w < 1 || det_h < 1 || det_w > 16384 || det_h > 8192)
        return fail(nullptr, LAMINO_EINVAL, "detector %dx%d out of range [1, 16384]x[1, 8192]", det_w, det_h);
    if (!isfinite(tilt) || fabs(tilt) >= kPi / 2)
        return fail(nullptr, LAMINO_EINVAL, "tilt %g rad must be finite with |tilt| < pi/2", tilt);
    if (angles)
        for (int k = 0; k < nproj; ++k)
            if (!isfinite(angles[k])) return fail(nullptr, LAMINO_EINVAL, "angle %d is not finite", k);

    lamino_plan_t p = nullptr;
    try {
        p = new lamino_plan_s();
    } catch (const std::bad_alloc&) {
        return fail(nullptr, LAMINO_ENOMEM, "host allocation of the plan failed");
    }
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return fail(nullptr, LAMINO_ECUDA, "no CUDA device");
    }
    p->n0 = n0; p->n1 = n1; p->n2 = n2; p->nproj = nproj; p->W = det_w; p->H = det_h;
    p->tilt = tilt;
    p->theta.resize(nproj);
    for (int k = 0; k < nproj; ++k) p->theta[k] = angles ? angles[k] : 2.0 * kPi * k / nproj;

    // sizes (Sec. 4 filter padding; the Fourier grid must hold the projected
    // footprint u_max, v_max so that trigonometric interpolation never wraps)
    double umax = 0.5 * hypot((double)n0, (double)n1);
    double vmax = umax * fabs(sin(tilt)) + 0.5 * n2 * cos(tilt);
    p->Wp = fft_size_at_least(2.0 * det_w);
    p->Wf = fft_size_at_least(std::max((double)det_w, 2.0 * umax + 2.0));
    p->Hf = fft_size_at_least(std::max((double)det_h, 2.0 * vmax + 2.0));
    if (opts && opts->wf) p->Wf = opts->wf;
    if (opts && opts->hf) p->Hf = opts->hf;
    p->w = (opts && opts->usfft_w) ? opts->usfft_w : 4;
    p->wz = (opts && opts->usfft_wz) ? opts->usfft_wz : 6;
    p->grid_rows = (opts && opts->grid_rows > 0) ? opts->grid_rows : 0;
    p->z_chunk = (opts && opts->z_chunk > 0) ? opts->z_chunk : 0;
    if (opts && opts->z_chunk < 0) {
        free_plan(p);
        return fail(nullptr, LAMINO_EINVAL, "z_chunk must be >= 0");
    }
    if (p->grid_rows & (p->grid_rows - 1)) {
        free_plan(p);
        return fail(nullptr, LAMINO_EINVAL, "grid_rows must be a power of two");
    }
    if (p->w < 2 || p->w > 8 || p->wz < 2 || p->wz > 8) {
        free_plan(p);
        return fail(nullptr, LAMINO_EINVAL, "usfft half-widths must be in [2, 8]");
    }
    if (p->Wf < det_w || p->Hf < det_h) {
        free_plan(p);
        return fail(nullptr, LAMINO_EINVAL, "Fourier grid %dx%d must cover the %dx%d detector",
                    p->Wf, p->Hf, det_w, det_h);
    }
    p->L = p->Hf / 2;
    p->offu = (p->Wf - det_w) / 2;
    p->offv = (p->Hf - det_h) / 2;
    p->M1 = std::max(16, fft_size_at_least(2.0 * n0));
    p->M2 = std::max(16, fft_size_at_least(2.0 * n1));
    p->M3 = std::max(16, fft_size_at_least(2.0 * n2));
    choose_widths(p, opts && opts->usfft_w, opts && opts->usfft_wz);
    p->err_est = usfft_err_est(n0, n1, n2, p->M1, p->M2, p->M3, p->w, p->wz);
    p->t1 = gauss_t(p->w, (double)p->M1 / n0);
    p->t2 = gauss_t(p->w, (double)p->M2 / n1);
    p->t3 = gauss_t(p->wz, (double)p->M3 / n2);
    // forms whose FFT lengths this build cannot handle are refused at call time
    p->filter_ok = fft_len_ok(p->Wp);
    p->fourier_ok = true;
    {
        const int lens[] = {p->Wf, p->Hf, p->M1, p->M2, p->M3};
        char buf[256];
        for (int n : lens)
            if (!fft_len_ok(n) && p->fourier_ok) {
                snprintf(buf, sizeof buf, "FFT length %d of the Fourier form is not 2^k (8 .. 8192) "
                         "or 3*2^k (12 .. 6144)", n);
                p->fourier_why = buf;
                p->fourier_ok = false;
            }
        if (p->fourier_ok && ((n0 & 1) || (n1 & 1) || (n2 & 1))) {
            p->fourier_why = "the Fourier form needs even volume sizes (x = i - n/2 integer)";
            p->fourier_ok = false;
        }
    }
    direct_config(p);
    if (p->dcfg.bh > 256 || p->dcfg.bw > 256 || p->pcfg.bh > 256 || p->pcfg.bw > 256) {
        free_plan(p);
        return fail(nullptr, LAMINO_EUNSUPPORTED, "detector footprint tile too large");
    }
    int rc = build_tables(p);
    if (rc) {
        g_last_error = p->err;
        free_plan(p);
        return rc;
    }
    *out = p;
    return LAMINO_OK;
}

int lamino_get_info(lamino_plan_t p, lamino_plan_info* info) {
    if (!p || !info) return fail(p, LAMINO_EINVAL, "lamino_get_info: NULL argument");
    info->n0 = p->n0; info->n1 = p->n1; info->n2 = p->n2; info->nproj = p->nproj;
    info->det_w = p->W; info->det_h = p->H;
    info->wp = p->Wp; info->wf = p->Wf; info->hf = p->Hf;
    info->m1 = p->M1; info->m2 = p->M2; info->m3 = p->M3;
    info->usfft_w = p->w; info->usfft_wz = p->wz; info->planes = p->L;
    info->usfft_err_est = (float)p->err_est;
    info->z_chunk = p->z_chunk;
    info->plane_chunk = plane_chunk(p);
    return LAMINO_OK;
}

int lamino_filter(lamino_plan_t p, const void* d, int dtype, float* q, int kind,
                  cudaStream_t stream) {
    if (!p) return fail(nullptr, LAMINO_EINVAL, "NULL plan");
    if (!d || !q) return fail(p, LAMINO_EINVAL, "lamino_filter: NULL data pointer");
    int rc = validate_dtype_kind(p, dtype, kind);
    if (rc) return rc;
    if (!p->filter_ok) return fail(p, LAMINO_EUNSUPPORTED, "filter length %d is not a supported FFT length", p->Wp);
    if ((rc = set_device(p))) return rc;
    return launch_filter(p, d, dtype, q, kind, stream);
}

int lamino_backproject_direct(lamino_plan_t p, const float* q, float* vol, cudaStream_t stream) {
    if (!p) return fail(nullptr, LAMINO_EINVAL, "NULL plan");
    if (!q || !vol) return fail(p, LAMINO_EINVAL, "lamino_backproject_direct: NULL data pointer");
    int rc = set_device(p);
    if (rc) return rc;
    return launch_direct(p, q, vol, stream);
}

static int fourier_common(lamino_plan_t p, const void* d, int dtype, float* vol, int kind,
                          cudaStream_t stream) {
    if (!p->fourier_ok) return fail(p, LAMINO_EUNSUPPORTED, "%s", p->fourier_why.c_str());
    if (kind >= 0 && !p->filter_ok)
        return fail(p, LAMINO_EUNSUPPORTED, "filter length %d is not a supported FFT length", p->Wp);
    FourierBufs fb;
    int rc = fourier_buffers(p, &fb);
    if (rc) return rc;
    if ((rc = launch_rowfft(p, d, dtype, fb.R, kind, stream))) return rc;
    return run_fourier_after_rows(p, fb, vol, stream);
}

int lamino_backproject_fourier(lamino_plan_t p, const void* q, int dtype, float* vol,
                               cudaStream_t stream) {
    if (!p) return fail(nullptr, LAMINO_EINVAL, "NULL plan");
    if (!q || !vol) return fail(p, LAMINO_EINVAL, "lamino_backproject_fourier: NULL data pointer");
    int rc = validate_dtype_kind(p, dtype, LAMINO_RAMP);
    if (rc) return rc;
    if ((rc = set_device(p))) return rc;
    return fourier_common(p, q, dtype, vol, -1, stream);
}

int lamino_fbp(lamino_plan_t p, int form, const void* d, int dtype, float* vol, int kind,
               cudaStream_t stream) {
    if (!p) return fail(nullptr, LAMINO_EINVAL, "NULL plan");
    if (!d || !vol) return fail(p, LAMINO_EINVAL, "lamino_fbp: NULL data pointer");
    int rc = validate_dtype_kind(p, dtype, kind);
    if (rc) return rc;
    if ((rc = set_device(p))) return rc;
    if (form == LAMINO_FOURIER) return fourier_common(p, d, dtype, vol, kind, stream);
    if (form != LAMINO_DIRECT) return fail(p, LAMINO_EINVAL, "unknown form %d", form);
    if (!p->filter_ok) return fail(p, LAMINO_EUNSUPPORTED, "filter length %d is not a supported FFT length", p->Wp);
    float* qb = nullptr;
    if ((rc = rows_buffer(p, &qb))) return rc;
    if ((rc = launch_filter(p, d, dtype, qb, kind, stream))) return rc;
    return launch_direct(p, qb, vol, stream);
}

// Host pipeline of lamino_fbp_host: the projections go up in chunks of whole
// projections on a copy stream while the row (and, for the Fourier form,
// column) passes of the chunks already copied run on the caller's stream; the
// Fourier volume comes back in slabs of x2 rows while the x3 pass computes the
// next slab. Every dependency is an event; the call returns after both
// streams have drained.
static int ensure_pipeline(lamino_plan_t p, size_t nev) {
    if (!p->copy_stream)
        LAM_CUDA(p, cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
    while (p->pipe_ev.size() < nev) {
        cudaEvent_t e;
        LAM_CUDA(p, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        p->pipe_ev.push_back(e);
    }
    return LAMINO_OK;
}

int lamino_fbp_host(lamino_plan_t p, int form, const void* d_host, int dtype, float* vol_host,
                    int kind, cudaStream_t stream) {
    if (!p) return fail(nullptr, LAMINO_EINVAL, "NULL plan");
    if (!d_host || !vol_host) return fail(p, LAMINO_EINVAL, "lamino_fbp_host: NULL host pointer");
    int rc = validate_dtype_kind(p, dtype, kind);
    if (rc) return rc;
    if ((rc = set_device(p))) return rc;
    if (form != LAMINO_FOURIER && form != LAMINO_DIRECT) return fail(p, LAMINO_EINVAL, "unknown form %d", form);
    if (form == LAMINO_FOURIER) {
        if (!p->fourier_ok) return fail(p, LAMINO_EUNSUPPORTED, "%s", p->fourier_why.c_str());
    }
    if (!p->filter_ok) return fail(p, LAMINO_EUNSUPPORTED, "filter length %d is not a supported FFT length", p->Wp);
    const size_t esz = dtype == LAMINO_F32 ? 4 : 2;
    const size_t proj_bytes = esz * (size_t)p->H * p->W;
    const size_t din = proj_bytes * p->nproj;
    const size_t dvol = sizeof(float) * (size_t)p->n0 * p->n1 * p->n2;
    if ((rc = ensure_buffer(p, &p->h_in, &p->h_in_bytes, din, "device copy of projections"))) return rc;
    if ((rc = ensure_buffer(p, (void**)&p->h_vol, &p->h_vol_bytes, dvol, "device volume"))) return rc;
    FourierBufs fb;
    if (form == LAMINO_FOURIER) {
        if ((rc = fourier_buffers(p, &fb))) return rc;
    }
    float* qb = nullptr;
    if (form != LAMINO_FOURIER && (rc = rows_buffer(p, &qb))) return rc;
    const int nin = std::min(8, p->nproj);                          // projection chunks
    const int nout = form == LAMINO_FOURIER ? std::min(8, p->n1) : 1;   // volume slabs
    if ((rc = ensure_pipeline(p, (size_t)nin + nout + 2))) return rc;
    cudaEvent_t* ev = p->pipe_ev.data();
    cudaStream_t cs = p->copy_stream;
    // the copies start after whatever the caller queued before (which may
    // still read the plan's buffers)
    LAM_CUDA(p, cudaEventRecord(ev[0], stream));
    LAM_CUDA(p, cudaStreamWaitEvent(cs, ev[0], 0));
    for (int c = 0; c < nin; ++c) {
        const long k0 = (long)p->nproj * c / nin, k1 = (long)p->nproj * (c + 1) / nin;
        LAM_CUDA(p, cudaMemcpyAsync((char*)p->h_in + k0 * proj_bytes, (const char*)d_host + k0 * proj_bytes,
                                    (k1 - k0) * proj_bytes, cudaMemcpyHostToDevice, cs));
        LAM_CUDA(p, cudaEventRecord(ev[1 + c], cs));
    }
    for (int c = 0; c < nin; ++c) {
        const long k0 = (long)p->nproj * c / nin, k1 = (long)p->nproj * (c + 1) / nin;
        LAM_CUDA(p, cudaStreamWaitEvent(stream, ev[1 + c], 0));
        if (form == LAMINO_FOURIER) {
            if ((rc = launch_rowfft(p, p->h_in, dtype, fb.R, kind, stream, k0 * p->H, k1 * p->H)))
                return rc;
            if ((rc = launch_colfft(p, fb, (int)k0, (int)k1, stream))) return rc;
        } else {
            if ((rc = launch_filter(p, p->h_in, dtype, qb, kind, stream, k0 * p->H, k1 * p->H)))
                return rc;
        }
    }
    cudaEvent_t* evo = ev + 1 + nin;
    if (form == LAMINO_FOURIER) {
        if ((rc = run_planes(p, fb, stream))) return rc;
        const size_t row = sizeof(float) * (size_t)p->n0, slice = row * p->n1;
        for (int v = 0; v < nout; ++v) {
            const int i10 = (int)((long)p->n1 * v / nout), i11 = (int)((long)p->n1 * (v + 1) / nout);
            if ((rc = launch_zusfft(p, fb, p->h_vol, i10, i11, stream))) return rc;
            LAM_CUDA(p, cudaEventRecord(evo[v], stream));
            LAM_CUDA(p, cudaStreamWaitEvent(cs, evo[v], 0));
            // slab [x3][x2 in i10..i11)[x1]: n2 pieces of (i11 - i10) rows
            LAM_CUDA(p, cudaMemcpy2DAsync((char*)vol_host + i10 * row, slice, (const char*)p->h_vol + i10 * row,
                                          slice, (i11 - i10) * row, p->n2, cudaMemcpyDeviceToHost, cs));
        }
    } else {
        if ((rc = launch_direct(p, qb, p->h_vol, stream))) return rc;
        LAM_CUDA(p, cudaEventRecord(evo[0], stream));
        LAM_CUDA(p, cudaStreamWaitEvent(cs, evo[0], 0));
        LAM_CUDA(p, cudaMemcpyAsync(vol_host, p->h_vol, dvol, cudaMemcpyDeviceToHost, cs));
    }
    LAM_CUDA(p, cudaEventRecord(evo[nout], cs));
    LAM_CUDA(p, cudaStreamWaitEvent(stream, evo[nout], 0));
    LAM_CUDA(p, cudaStreamSynchronize(stream));
    return LAMINO_OK;
}

int lamino_project(lamino_plan_t p, int form, const float* vol, float* d, cudaStream_t stream) {
    if (!p) return fail(nullptr, LAMINO_EINVAL, "NULL plan");
    if (!vol || !d) return fail(p, LAMINO_EINVAL, "lamino_project: NULL data pointer");
    int rc = set_device(p);
    if (rc) return rc;
    if (form == LAMINO_DIRECT) return launch_project_direct(p, vol, d, stream);
    if (form == LAMINO_FOURIER) {
        if (!p->fourier_ok) return fail(p, LAMINO_EUNSUPPORTED, "%s", p->fourier_why.c_str());
        FourierBufs fb;
        if ((rc = fourier_buffers(p, &fb))) return rc;
        return launch_project_fourier(p, fb, vol, d, stream);
    }
    return fail(p, LAMINO_EINVAL, "unknown form %d", form);
}

int lamino_device_bytes(lamino_plan_t p, size_t* bytes) {
    if (!p || !bytes) return fail(p, LAMINO_EINVAL, "lamino_device_bytes: NULL argument");
    *bytes = p->table_bytes + sizeof(int) + p->ws_a_bytes + p->ws_b_bytes + p->q_buf_bytes +
             p->q_pad_bytes + p->h_in_bytes + p->h_vol_bytes;
    return LAMINO_OK;
}

int lamino_set_workspace(lamino_plan_t p, void* ws, size_t bytes) {
    if (!p) return fail(nullptr, LAMINO_EINVAL, "NULL plan");
    if ((ws == nullptr) != (bytes == 0))
        return fail(p, LAMINO_EINVAL, "lamino_set_workspace: pointer and size must both be set or both be 0");
    if ((uintptr_t)ws % 256)
        return fail(p, LAMINO_EINVAL, "lamino_set_workspace: the buffer must be 256-byte aligned");
    int rc = set_device(p);
    if (rc) return rc;
    if (ws && (p->ws_a || p->ws_b || p->q_buf || p->q_pad)) {
        // the plan's own workspaces are no longer used; cudaFree waits for the device
        void* own[] = {p->ws_a, p->ws_b, p->q_buf, p->q_pad};
        for (void* b : own)
            if (b) LAM_CUDA(p, cudaFree(b));
        p->ws_a = p->ws_b = nullptr;
        p->q_buf = p->q_pad = nullptr;
        p->ws_a_bytes = p->ws_b_bytes = p->q_buf_bytes = p->q_pad_bytes = 0;
    }
    p->lent = ws;
    p->lent_bytes = bytes;
    return LAMINO_OK;
}

int lamino_set_z_chunk(lamino_plan_t p, int z_chunk) {
    if (!p) return fail(nullptr, LAMINO_EINVAL, "NULL plan");
    if (z_chunk < 0) return fail(p, LAMINO_EINVAL, "z_chunk must be >= 0, not %d", z_chunk);
    int rc = set_device(p);
    if (rc) return rc;
    if (z_chunk == p->z_chunk) return LAMINO_OK;
    // the workspaces follow the new layout at the next call; cudaFree waits
    // for the device, so nothing in flight still uses them
    if (p->ws_a) LAM_CUDA(p, cudaFree(p->ws_a));
    if (p->ws_b) LAM_CUDA(p, cudaFree(p->ws_b));
    p->ws_a = p->ws_b = nullptr;
    p->ws_a_bytes = p->ws_b_bytes = 0;
    p->z_chunk = z_chunk;
    return LAMINO_OK;
}

int lamino_workspace_bytes(lamino_plan_t p, int form, size_t* bytes) {
    if (!p || !bytes) return fail(p, LAMINO_EINVAL, "lamino_workspace_bytes: NULL argument");
    if (form == LAMINO_FOURIER) {
        size_t a, b;
        fourier_workspace(p, &a, &b);
        *bytes = a + b;
    } else if (form == LAMINO_DIRECT) {
        *bytes = sizeof(float) * (size_t)p->nproj * p->H * p->W;
        // rows whose width is not a multiple of 4 floats are staged at a
        // 16-byte pitch for the TMA loads (after the filtered rows, aligned)
        if (p->W % 4) *bytes = lent_align(*bytes) + sizeof(float) * (size_t)p->nproj * p->H * ((p->W + 3) / 4 * 4);
    } else {
        return fail(p, LAMINO_EINVAL, "unknown form %d", form);
    }
    return LAMINO_OK;
}

int lamino_status(lamino_plan_t p, cudaStream_t stream) {
    if (!p) return fail(nullptr, LAMINO_EINVAL, "NULL plan");
    int rc = set_device(p);
    if (rc) return rc;
    LAM_CUDA(p, cudaStreamSynchronize(stream));
    int h = 0;
    LAM_CUDA(p, cudaMemcpy(&h, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        LAM_CUDA(p, cudaMemset(p->d_err, 0, sizeof(int)));
        return fail(p, LAMINO_ETIMEOUT, "a bounded device wait gave up (code %d); results of the "
                    "calls since the last status check are invalid", h);
    }
    return LAMINO_OK;
}

int lamino_profile(lamino_plan_t p, int enable) {
    if (!p) return fail(nullptr, LAMINO_EINVAL, "NULL plan");
    p->profiling = enable != 0;
    p->recs.clear();
    p->ev_used = 0;
    return LAMINO_OK;
}

int lamino_profile_read(lamino_plan_t p, lamino_kernel_time* out, int max, int* n) {
    if (!p || !n || (max > 0 && !out)) return fail(p, LAMINO_EINVAL, "lamino_profile_read: bad argument");
    int rc = set_device(p);
    if (rc) return rc;
    int k = 0;
    for (auto& r : p->recs) {
        if (r.b < 0) continue;
        LAM_CUDA(p, cudaEventSynchronize(p->ev_pool[r.b]));
        if (k < max) {
            float ms = 0.f;
            LAM_CUDA(p, cudaEventElapsedTime(&ms, p->ev_pool[r.a], p->ev_pool[r.b]));
            snprintf(out[k].name, sizeof out[k].name, "%s", r.name.c_str());
            out[k].ms = ms;
        }
        ++k;
    }
    *n = std::min(k, max);
    p->recs.clear();
    p->ev_used = 0;
    return LAMINO_OK;
}

const char* lamino_last_error(lamino_plan_t p) { return p ? p->err.c_str() : g_last_error.c_str(); }

int lamino_destroy(lamino_plan_t p) {
    if (!p) return LAMINO_OK;
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    free_plan(p);
    return LAMINO_OK;
}

}  // extern "C"
