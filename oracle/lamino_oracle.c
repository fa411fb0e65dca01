/*
 * FP64 CPU oracle for laminographic backprojection -- TEST INFRASTRUCTURE.
 *
 * Plain, slow, obviously correct loops; nothing here is tuned. Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load this
 * library. It shares no code with the CUDA path.
 *
 * Geometry (Nikitin et al., Sec. 4, the two delta functions after Eq. fwd):
 *   u = a.x = x1 cos t + x2 sin t
 *   v = b.x = x1 sin t sin phi - x2 cos t sin phi + x3 cos phi
 * Voxel index i on an axis of size n sits at x = i - n/2; detector column j at
 * u = j - W/2, row r at v = r - H/2. Volumes are [n2][n1][n0], projections
 * [nproj][H][W], both C order.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the OpenMP loops from now on (timing of the CPU baseline). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Detector value with zero outside [0,W) x [0,H). */
static double tap(const double* q, int H, int W, long r, long j) {
    if (r < 0 || r >= H || j < 0 || j >= W) return 0.0;
    return q[(size_t)r * W + j];
}

/* Bilinear interpolation on the integer pixel lattice (linear interpolation of
 * the line-integral discretisation, Sec. 4 after Eq. adj). */
static double bilinear(const double* q, int H, int W, double j, double r) {
    double jf = floor(j), rf = floor(r);
    double fj = j - jf, fr = r - rf;
    long j0 = (long)jf, r0 = (long)rf;
    return (1.0 - fj) * (1.0 - fr) * tap(q, H, W, r0, j0)
         + fj * (1.0 - fr) * tap(q, H, W, r0, j0 + 1)
         + (1.0 - fj) * fr * tap(q, H, W, r0 + 1, j0)
         + fj * fr * tap(q, H, W, r0 + 1, j0 + 1);
}

/* One voxel of the direct backprojection, Eq. adj discretised with the
 * rectangle rule over theta:  (pi/Ntheta) * sum_k q_k(a_k.x + W/2, b_k.x + H/2).
 * The factor pi/Ntheta is half of 2*pi/Ntheta: the full-circle FBP carries a
 * 1/2 because every Fourier point is reached twice over [0, 2 pi). */
static double bp_direct_voxel(const double* q, int nproj, int H, int W,
                              const double* theta, double phi,
                              double x1, double x2, double x3) {
    double sp = sin(phi), cp = cos(phi), acc = 0.0;
    for (int k = 0; k < nproj; ++k) {
        double ct = cos(theta[k]), st = sin(theta[k]);
        double u = x1 * ct + x2 * st;
        double v = x1 * st * sp - x2 * ct * sp + x3 * cp;
        acc += bilinear(q + (size_t)k * H * W, H, W, u + 0.5 * W, v + 0.5 * H);
    }
    return acc * ORC_PI / nproj;
}

/* Direct backprojection of slices z in [z0, z1): out[(z-z0)][n1][n0]. */
void orc_bp_direct(const double* q, int nproj, int H, int W, const double* theta,
                   double phi, int n0, int n1, int n2, int z0, int z1, double* out) {
    (void)n2;
    long nz = z1 - z0;
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (long z = 0; z < nz; ++z)
        for (long i1 = 0; i1 < n1; ++i1)
            for (long i0 = 0; i0 < n0; ++i0)
                out[(z * n1 + i1) * n0 + i0] = bp_direct_voxel(
                    q, nproj, H, W, theta, phi, i0 - 0.5 * n0, i1 - 0.5 * n1,
                    (z + z0) - 0.5 * n2);
}

/* Direct backprojection on whole columns: cols[c] = (i0, i1); out[c][n2]. */
void orc_bp_direct_columns(const double* q, int nproj, int H, int W, const double* theta,
                           double phi, int n0, int n1, int n2, const int* cols, int ncol,
                           double* out) {
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (long c = 0; c < ncol; ++c)
        for (long i2 = 0; i2 < n2; ++i2)
            out[c * n2 + i2] = bp_direct_voxel(q, nproj, H, W, theta, phi,
                                               cols[2 * c] - 0.5 * n0,
                                               cols[2 * c + 1] - 0.5 * n1, i2 - 0.5 * n2);
}

/* Exact transpose of the bilinear backprojection sum (without the pi/Ntheta
 * factor): every voxel scatters its bilinear weights onto each projection. */
void orc_splat(const double* vol, int n0, int n1, int n2, int nproj, int H, int W,
               const double* theta, double phi, double* d) {
    double sp = sin(phi), cp = cos(phi);
    memset(d, 0, sizeof(double) * (size_t)nproj * H * W);
#pragma omp parallel for schedule(dynamic)
    for (long k = 0; k < nproj; ++k) {
        double ct = cos(theta[k]), st = sin(theta[k]);
        double* dk = d + (size_t)k * H * W;
        for (long i2 = 0; i2 < n2; ++i2)
            for (long i1 = 0; i1 < n1; ++i1)
                for (long i0 = 0; i0 < n0; ++i0) {
                    double x1 = i0 - 0.5 * n0, x2 = i1 - 0.5 * n1, x3 = i2 - 0.5 * n2;
                    double j = x1 * ct + x2 * st + 0.5 * W;
                    double r = x1 * st * sp - x2 * ct * sp + x3 * cp + 0.5 * H;
                    double jf = floor(j), rf = floor(r), fj = j - jf, fr = r - rf;
                    long j0 = (long)jf, r0 = (long)rf;
                    double m = vol[(i2 * n1 + i1) * n0 + i0];
                    double wt[4] = {(1 - fj) * (1 - fr), fj * (1 - fr), (1 - fj) * fr, fj * fr};
                    long jj[4] = {j0, j0 + 1, j0, j0 + 1}, rr[4] = {r0, r0, r0 + 1, r0 + 1};
                    for (int t = 0; t < 4; ++t)
                        if (rr[t] >= 0 && rr[t] < H && jj[t] >= 0 && jj[t] < W)
                            dk[rr[t] * W + jj[t]] += wt[t] * m;
                }
    }
}

/* Signed frequency of FFT index i for length N (N even): i or i - N. */
static int sfreq(int i, int N) { return i < N / 2 ? i : i - N; }

/*
 * Fourier-form backprojection, Eq. fftadj, evaluated as its exact definition:
 * the type-1 sum over the unequally spaced frequencies of Eq. uneqspace,
 *   vol(x) = scale * Re sum_k sum_{m,l} D_k(m,l) exp(2 pi i (m j'/Wf + l r'/Hf)),
 * j' = a_k.x + joff, r' = b_k.x + roff (padded detector indices), D_k the 2D DFT
 * of the zero-padded projection (Nyquist row/column already zeroed by the
 * caller). With k_u = m/Wf, k_v = l/Hf the exponent equals 2 pi i x.xi of
 * Eq. uneqspace plus the constant detector-centre phase.
 *
 * Evaluated separably (exact algebra, no approximation): per (k, column) the
 * inner sum over m is formed once, then the sum over l for every x3.
 * D is [nproj][Hf][Wf] complex as separate re/im arrays in FFT index order.
 */
void orc_bp_fourier_columns(const double* Dre, const double* Dim, int nproj, int Hf, int Wf,
                            double joff, double roff, const double* theta, double phi,
                            int n0, int n1, int n2, const int* cols, int ncol, double scale,
                            double* out) {
    double sp = sin(phi), cp = cos(phi);
#pragma omp parallel
    {
        double* gre = (double*)malloc(sizeof(double) * Hf);
        double* gim = (double*)malloc(sizeof(double) * Hf);
        double* ere = (double*)malloc(sizeof(double) * Wf);
        double* eim = (double*)malloc(sizeof(double) * Wf);
#pragma omp for schedule(dynamic)
        for (long c = 0; c < ncol; ++c) {
            double x1 = cols[2 * c] - 0.5 * n0, x2 = cols[2 * c + 1] - 0.5 * n1;
            for (long i2 = 0; i2 < n2; ++i2) out[c * n2 + i2] = 0.0;
            for (int k = 0; k < nproj; ++k) {
                double ct = cos(theta[k]), st = sin(theta[k]);
                double jp = x1 * ct + x2 * st + joff;
                for (int m = 0; m < Wf; ++m) {
                    double ang = 2.0 * ORC_PI * sfreq(m, Wf) * jp / Wf;
                    ere[m] = cos(ang);
                    eim[m] = sin(ang);
                }
                const double* dr = Dre + (size_t)k * Hf * Wf;
                const double* di = Dim + (size_t)k * Hf * Wf;
                for (int l = 0; l < Hf; ++l) {
                    double sr = 0.0, si = 0.0;
                    for (int m = 0; m < Wf; ++m) {
                        double ar = dr[(size_t)l * Wf + m], ai = di[(size_t)l * Wf + m];
                        sr += ar * ere[m] - ai * eim[m];
                        si += ar * eim[m] + ai * ere[m];
                    }
                    gre[l] = sr;
                    gim[l] = si;
                }
                double rbase = x1 * st * sp - x2 * ct * sp + roff;
                for (long i2 = 0; i2 < n2; ++i2) {
                    double rp = rbase + (i2 - 0.5 * n2) * cp;
                    double acc = 0.0;
                    for (int l = 0; l < Hf; ++l) {
                        double ang = 2.0 * ORC_PI * sfreq(l, Hf) * rp / Hf;
                        acc += gre[l] * cos(ang) - gim[l] * sin(ang);
                    }
                    out[c * n2 + i2] += acc;
                }
            }
            for (long i2 = 0; i2 < n2; ++i2) out[c * n2 + i2] *= scale;
        }
        free(gre); free(gim); free(ere); free(eim);
    }
}

/* The same sum with all four loops written out for every voxel (no
 * separation), for tiny volumes only. out is [n2][n1][n0]. */
void orc_bp_fourier_full4(const double* Dre, const double* Dim, int nproj, int Hf, int Wf,
                          double joff, double roff, const double* theta, double phi,
                          int n0, int n1, int n2, double scale, double* out) {
    double sp = sin(phi), cp = cos(phi);
    long nvox = (long)n0 * n1 * n2;
#pragma omp parallel for schedule(dynamic)
    for (long idx = 0; idx < nvox; ++idx) {
        long i0 = idx % n0, i1 = (idx / n0) % n1, i2 = idx / ((long)n0 * n1);
        double x1 = i0 - 0.5 * n0, x2 = i1 - 0.5 * n1, x3 = i2 - 0.5 * n2;
        double acc = 0.0;
        for (int k = 0; k < nproj; ++k) {
            double ct = cos(theta[k]), st = sin(theta[k]);
            double jp = x1 * ct + x2 * st + joff;
            double rp = x1 * st * sp - x2 * ct * sp + x3 * cp + roff;
            for (int l = 0; l < Hf; ++l)
                for (int m = 0; m < Wf; ++m) {
                    double ang = 2.0 * ORC_PI * (sfreq(m, Wf) * jp / Wf + sfreq(l, Hf) * rp / Hf);
                    size_t o = ((size_t)k * Hf + l) * Wf + m;
                    acc += Dre[o] * cos(ang) - Dim[o] * sin(ang);
                }
        }
        out[idx] = acc * scale;
    }
}

/* Coefficients of the transpose of the Fourier form:
 *   A_k(m,l) = sum_x vol(x) exp(2 pi i (m j'_k(x)/Wf + l r'_k(x)/Hf)),
 * brute force over every voxel; A is [nproj][Hf][Wf] in FFT index order. */
void orc_fourier_adjoint_coeffs(const double* vol, int n0, int n1, int n2, int nproj, int Hf,
                                int Wf, double joff, double roff, const double* theta,
                                double phi, double* Are, double* Aim) {
    double sp = sin(phi), cp = cos(phi);
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (long k = 0; k < nproj; ++k)
        for (long l = 0; l < Hf; ++l) {
            double ct = cos(theta[k]), st = sin(theta[k]);
            for (int m = 0; m < Wf; ++m) {
                double sr = 0.0, si = 0.0;
                for (long i2 = 0; i2 < n2; ++i2)
                    for (long i1 = 0; i1 < n1; ++i1)
                        for (long i0 = 0; i0 < n0; ++i0) {
                            double x1 = i0 - 0.5 * n0, x2 = i1 - 0.5 * n1, x3 = i2 - 0.5 * n2;
                            double jp = x1 * ct + x2 * st + joff;
                            double rp = x1 * st * sp - x2 * ct * sp + x3 * cp + roff;
                            double ang = 2.0 * ORC_PI * (sfreq(m, Wf) * jp / Wf +
                                                         sfreq((int)l, Hf) * rp / Hf);
                            double mu = vol[(i2 * n1 + i1) * n0 + i0];
                            sr += mu * cos(ang);
                            si += mu * sin(ang);
                        }
                size_t o = ((size_t)k * Hf + l) * Wf + m;
                Are[o] = sr;
                Aim[o] = si;
            }
        }
}

/* Periodic interpolation kernel of period N with the Nyquist term dropped:
 *   K_N(t) = (1/N) sum_{m=-N/2+1}^{N/2-1} exp(2 pi i m t / N)
 *          = sin(pi (N-1) t / N) / (N sin(pi t / N)),
 * a real, even, N-periodic function equal to (N-1)/N at multiples of N. */
static double periodic_kernel(double t, int N) {
    double tr = t - N * floor(t / N + 0.5);   /* reduce to [-N/2, N/2) */
    double s = sin(ORC_PI * tr / N);
    if (fabs(tr) < 1e-9) return (double)(N - 1) / N;
    return sin(ORC_PI * (N - 1) * tr / N) / (N * s);
}

/*
 * The Fourier form by its spatial reading. Substituting the 2D DFT of the
 * zero-padded projection into the type-1 sum of Eq. fftadj (Eq. uneqspace grid)
 * and summing the geometric series over m and l gives
 *   vol(x) = (pi/Ntheta) sum_k sum_{r,j} q_k(r, j) K_Wf(a_k.x + W/2 - j) K_Hf(b_k.x + H/2 - r):
 * direct backprojection with the periodic (trigonometric) interpolation
 * kernel of the padded detector in place of the bilinear one. The padding
 * offsets cancel; Wf and Hf enter only as the kernel periods. This route needs
 * no spectra, so it scales to paper-size projections; it and
 * orc_bp_fourier_columns are two independent evaluations of one sum.
 *
 * q holds nq projections at angles theta[0..nq); `weight` is the quadrature
 * weight per angle (pi/Ntheta of the full angle set). Columns cols[c] =
 * (i0, i1); out[c][n2] is overwritten.
 */
void orc_bp_trig_columns(const double* q, int nq, int H, int W, const double* theta, double phi,
                         int Wf, int Hf, int n0, int n1, int n2, const int* cols, int ncol,
                         double weight, double* out) {
    double sp = sin(phi), cp = cos(phi);
    double* rows = (double*)malloc(sizeof(double) * (size_t)nq * H);   /* per angle: rows at u */
    for (long c = 0; c < ncol; ++c) {
        double x1 = cols[2 * c] - 0.5 * n0, x2 = cols[2 * c + 1] - 0.5 * n1;
        /* interpolate every detector row of every projection at u = a_k.x */
#pragma omp parallel for schedule(dynamic)
        for (long k = 0; k < nq; ++k) {
            double ct = cos(theta[k]), st = sin(theta[k]);
            double u = x1 * ct + x2 * st + 0.5 * W;
            double* kr = (double*)malloc(sizeof(double) * W);
            for (int j = 0; j < W; ++j) kr[j] = periodic_kernel(u - j, Wf);
            const double* qk = q + (size_t)k * H * W;
            for (int r = 0; r < H; ++r) {
                double acc = 0.0;
                for (int j = 0; j < W; ++j) acc += qk[(size_t)r * W + j] * kr[j];
                rows[(size_t)k * H + r] = acc;
            }
            free(kr);
        }
        /* then along the detector column at v = b_k.x for every slice */
#pragma omp parallel for schedule(dynamic)
        for (long i2 = 0; i2 < n2; ++i2) {
            double x3 = i2 - 0.5 * n2, acc = 0.0;
            for (long k = 0; k < nq; ++k) {
                double ct = cos(theta[k]), st = sin(theta[k]);
                double v = x1 * st * sp - x2 * ct * sp + x3 * cp + 0.5 * H;
                for (int r = 0; r < H; ++r) acc += rows[(size_t)k * H + r] * periodic_kernel(v - r, Hf);
            }
            out[c * n2 + i2] = acc * weight;
        }
    }
    free(rows);
}
