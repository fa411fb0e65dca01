/*
 * lamino.h -- C ABI of the GB300 laminographic filtered-backprojection library.
 *
 * Method: Nikitin et al., "Laminography as a tool for imaging large-size
 * samples with high resolution" (arXiv 2401.11101), Sec. 4-5.
 *
 *   forward operator  d(theta,u,v) = L mu      (Eq. fwd)
 *   backprojection    L* d(x)                  (Eq. adj)
 *   FBP               mu = W L* d              (Eq. recon; W = ramp filter
 *                                               |sigma| cos(phi) or a windowed one)
 *   Fourier form      L* = F*_u3D F_2D         (Eq. fftadj, grid of Eq. uneqspace),
 *                     evaluated with a Gaussian-kernel USFFT split into a 2D
 *                     transform over (x1, x2) and a 1D transform over x3
 *                     (Eq. fftfwdsplit)
 *
 * Conventions (all calls):
 *   - volumes are float32 [n2][n1][n0] in C order (x1 fastest, x3 = slab
 *     thickness); projections are [nproj][det_h][det_w] (u = columns fastest);
 *   - voxel = pixel = 1; voxel i on an axis of size n sits at x = i - n/2,
 *     detector column j at u = j - det_w/2, row r at v = r - det_h/2;
 *   - u = x1 cos t + x2 sin t, v = x1 sin t sin phi - x2 cos t sin phi +
 *     x3 cos phi (the delta functions after Eq. fwd); phi is the tilt away
 *     from tomography (phi = 0 is the Radon transform, Sec. 4), in radians;
 *   - every data pointer is a DEVICE pointer owned by the caller unless a
 *     call says otherwise; the plan owns its tables and workspaces;
 *   - calls are asynchronous on the given stream (0 = legacy default stream);
 *     outputs are valid once that stream has synchronised. One plan must not
 *     be used from two streams or two host threads at the same time (its
 *     workspace and its settings are shared);
 *   - every call returns a status (LAMINO_OK = 0 or a negative code below);
 *     lamino_last_error() gives a message for the last failure of a plan.
 */
#ifndef LAMINO_H
#define LAMINO_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define LAMINO_OK            0
#define LAMINO_EINVAL       -1   /* bad size, dtype, filter, pointer or tilt */
#define LAMINO_ENOMEM       -2   /* device allocation failed */
#define LAMINO_ECUDA        -3   /* a CUDA call failed (message has the CUDA error) */
#define LAMINO_ETIMEOUT     -4   /* a bounded device wait gave up (kernel returned early) */
#define LAMINO_EUNSUPPORTED -5   /* valid request this build does not handle */

/* Storage type of projection data handed to lamino_filter / lamino_fbp /
 * lamino_backproject_fourier. Arithmetic is always float32. */
#define LAMINO_F32  0
#define LAMINO_F16  1
#define LAMINO_BF16 2

/* Filter window on top of |f| cos(phi) (Sec. 4 after Eq. adj):
 * ramp w = 1; Shepp-Logan w = sin(pi f)/(pi f); Parzen (cubic, cutoff 1/2). */
#define LAMINO_RAMP   0
#define LAMINO_SHEPP  1
#define LAMINO_PARZEN 2

/* Backprojection form. */
#define LAMINO_DIRECT  0   /* voxel-driven bilinear sum, O(N^3 Ntheta) (Eq. adj) */
#define LAMINO_FOURIER 1   /* USFFT form, O(N^3 log N) (Eq. fftadj) */

typedef struct lamino_plan_s* lamino_plan_t;

/* Optional plan parameters; pass NULL for the defaults. Zero fields take the
 * default as well. */
typedef struct {
    int usfft_w;     /* Gaussian half-width (grid cells) of the 2D gridding; 0: the plan
                        chooses the smallest w in [4, 8] whose predicted relative L2 error
                        (usfft_err_est) is <= 0.9e-4: 4 for axes of >= 24 voxels, 5 for
                        the smallest grids */
    int usfft_wz;    /* half-width of the 1D gridding along x3; 0: chosen likewise (6) */
    int wf;          /* override of the padded Fourier detector width Wf */
    int hf;          /* override of the padded Fourier detector height Hf */
    int grid_rows;   /* rows of the oversampled grid per gridding CTA (power of two; tuning) */
    int z_chunk;     /* z chunking (Sec. 5: the 2D USFFT of Eq. fftfwdsplit by chunks of
                        slices, the 1D USFFT by chunks of columns, the direct form by
                        chunks of x3 slices): k_v planes per chunk of the gridding and
                        the x2 pass, and output slices per launch of the direct form
                        (rounded up to its 32-slice tile); 0: no chunking. Chunking the
                        Fourier form keeps only one chunk of x1-pass planes and shrinks
                        its workspace (lamino_workspace_bytes); results are equal */
} lamino_opts;

/* Sizes a plan derived (all integers). */
typedef struct {
    int n0, n1, n2, nproj, det_w, det_h;
    int wp;          /* filter length: smallest 2^k or 3*2^k >= 2*det_w */
    int wf, hf;      /* padded Fourier detector grid */
    int m1, m2, m3;  /* oversampled USFFT grids (>= 2*n0, 2*n1, 2*n2) */
    int usfft_w, usfft_wz;
    int planes;      /* k_v planes gridded (hf/2; the rest follow by Hermitian symmetry) */
    float usfft_err_est;  /* predicted relative L2 error of the Fourier form against the
                             exact sum, for evenly spread volume energy: truncation and
                             aliasing of the Gaussian kernel after deconvolution, per
                             axis, calibrated on random projections */
    int z_chunk;     /* the plan's z_chunk (0: none) */
    int plane_chunk; /* k_v planes per chunk of the Fourier form (planes when not chunked) */
} lamino_plan_info;

/*
 * lamino_plan -- build a plan for one geometry (host call, synchronous).
 *   out      : receives the plan handle.
 *   n0,n1,n2 : volume size (x1, x2, x3); each in [1, 8192] (Fourier form:
 *              2*n must round to a length <= 8192).
 *   nproj    : number of projection angles, >= 1.
 *   det_w/h  : detector columns (u) / rows (v); >= 1, <= 16384 / 8192.
 *   tilt     : laminographic angle phi in radians, |phi| < pi/2, finite.
 *   angles   : HOST array of nproj rotation angles in radians, or NULL for
 *              theta_k = 2 pi k / nproj. The quadrature weight is pi/nproj
 *              either way (the rectangle rule over a full circle).
 *   opts     : optional parameters or NULL.
 * Allocates the device tables of the plan on the current device; workspaces
 * of the Fourier form are allocated on first use. Errors: EINVAL, ENOMEM,
 * ECUDA, EUNSUPPORTED (a required FFT length above 8192).
 */
int lamino_plan(lamino_plan_t* out, int n0, int n1, int n2, int nproj, int det_w, int det_h,
                double tilt, const double* angles, const lamino_opts* opts);

/* Fill *info with the sizes of a plan. */
int lamino_get_info(lamino_plan_t plan, lamino_plan_info* info);

/*
 * lamino_filter -- the filter W of Eq. recon along detector rows (Sec. 4):
 * each row is zero-padded on the right to wp, transformed, multiplied by
 * H(f) = |f| cos(phi) w(f) for f = m/wp in [-1/2, 1/2), transformed back and
 * cropped to det_w.
 *   d     : projections [nproj][det_h][det_w] in `dtype` (LAMINO_F32/F16/BF16).
 *   q     : output float32 [nproj][det_h][det_w]; may equal d for LAMINO_F32.
 *   kind  : LAMINO_RAMP, LAMINO_SHEPP or LAMINO_PARZEN.
 */
int lamino_filter(lamino_plan_t plan, const void* d, int dtype, float* q, int kind,
                  cudaStream_t stream);

/*
 * lamino_backproject_direct -- Eq. adj by direct discretisation with bilinear
 * interpolation on the detector (taps outside the detector read 0):
 *   vol(x) = (pi/nproj) * sum_k q_k(a_k.x + det_w/2, b_k.x + det_h/2).
 *   q   : float32 projections [nproj][det_h][det_w] (filtered or not).
 *   vol : float32 [n2][n1][n0], overwritten.
 * Errors: EINVAL, ECUDA, ETIMEOUT (a pipeline wait gave up; vol is invalid).
 */
int lamino_backproject_direct(lamino_plan_t plan, const float* q, float* vol,
                              cudaStream_t stream);

/*
 * lamino_backproject_fourier -- Eq. fftadj: the same backprojection with the
 * detector interpolated trigonometrically instead of bilinearly, i.e.
 *   vol(x) = (pi/nproj)/(wf*hf) * Re sum_k sum_{m,l} D_k(m,l)
 *            exp(2 pi i (m j'(x)/wf + l r'(x)/hf)),
 * D_k the 2D DFT of projection k zero-padded to hf x wf (centred), Nyquist
 * row and column dropped, j' = a_k.x + det_w/2 + (wf-det_w)/2 and
 * r' = b_k.x + det_h/2 + (hf-det_h)/2. Evaluated with a 2D FFT per projection,
 * Gaussian gridding of the half spectrum onto each tilted k_v plane (2x
 * oversampled), inverse 2D FFT and deconvolution per plane, then a 1D USFFT
 * along x3. Accuracy is set by usfft_w / usfft_wz (relative L2 error below
 * 1e-4 at the widths the plan chooses; lamino_plan_info.usfft_err_est).
 *   q     : projections in `dtype`; vol : float32 [n2][n1][n0], overwritten.
 * Uses the plan's workspace (see lamino_workspace_bytes), allocated on the
 * first call. Errors: EINVAL, ENOMEM, ECUDA.
 */
int lamino_backproject_fourier(lamino_plan_t plan, const void* q, int dtype, float* vol,
                               cudaStream_t stream);

/*
 * lamino_backproject_fourier_noalloc -- the same result as
 * lamino_backproject_fourier, computed without allocating any device memory.
 * The paper has no counterpart to this call; it exists for callers that must
 * not allocate at reconstruction time: a streaming loop that may not stall on
 * the device allocator between frames, a process whose device memory is owned
 * by a pool or allocator that forbids stray cudaMalloc calls, or code that
 * records its work into a CUDA graph, where allocating inside the recorded
 * region is not permitted.
 *   - Its workspace is one static device array of 64 MiB held by every GPU that
 *     loads this library, until the process exits. Geometries whose Fourier
 *     workspace (lamino_workspace_bytes with LAMINO_FOURIER) exceeds it are
 *     rejected with LAMINO_EINVAL and a message giving both sizes; use
 *     lamino_backproject_fourier for those.
 *   - The plan itself (lamino_plan) still allocates its tables: create it while
 *     allocation is allowed. This call allocates nothing and calls no
 *     cudaMalloc/cudaFree; tracing (lamino_profile) is off during it.
 *   - The first call on each device looks up the array's device address with
 *     cudaGetSymbolAddress; make that first call before any stream capture.
 *   - Every call, from every plan and stream, shares the one array, and the
 *     array keeps the previous call's contents (nothing in it needs to start at
 *     zero). Calls whose execution overlaps on the GPU race on it: serialise
 *     them, e.g. on one stream.
 *   q, dtype, vol, stream: as for lamino_backproject_fourier.
 */
int lamino_backproject_fourier_noalloc(lamino_plan_t plan, const void* q, int dtype, float* vol,
                                       cudaStream_t stream);

/*
 * lamino_fbp -- filtered backprojection (Eq. recon): lamino_filter followed by
 * the chosen backprojection form. For LAMINO_FOURIER the filter is fused into
 * the first FFT pass; for LAMINO_DIRECT the filtered rows go through a plan
 * workspace of nproj*det_h*det_w floats.
 *   d : projections in `dtype`; vol : float32 [n2][n1][n0]; form : LAMINO_DIRECT
 *   or LAMINO_FOURIER; kind : filter window.
 */
int lamino_fbp(lamino_plan_t plan, int form, const void* d, int dtype, float* vol, int kind,
               cudaStream_t stream);

/*
 * lamino_fbp_host -- lamino_fbp on HOST buffers: copies d (host, pinned or
 * pageable) to a plan-owned device buffer, reconstructs, and copies the
 * volume back to vol (host). The copies run on a plan-owned stream in chunks
 * (up to 8 of whole projections up, up to 8 slabs of x2 rows of the Fourier
 * volume down) so that they overlap the row / column passes and the x3 pass
 * on `stream`; with pinned host memory the transfers hide behind the
 * kernels. The result equals lamino_fbp's. Synchronises `stream` (and the
 * copy stream) before returning; errors as lamino_fbp.
 */
int lamino_fbp_host(lamino_plan_t plan, int form, const void* d_host, int dtype,
                    float* vol_host, int kind, cudaStream_t stream);

/*
 * lamino_project -- the forward operator L of Eq. fwd, discretised as the
 * exact transpose of the chosen backprojection without its pi/nproj factor:
 *   <lamino_project(vol), q> * pi/nproj == <vol, lamino_backproject(q)>.
 *   vol : float32 [n2][n1][n0];  d : float32 [nproj][det_h][det_w], overwritten.
 * Form LAMINO_DIRECT is the voxel-driven bilinear splat. Errors: EINVAL,
 * ECUDA, EUNSUPPORTED (a form this build does not provide).
 */
int lamino_project(lamino_plan_t plan, int form, const float* vol, float* d,
                   cudaStream_t stream);

/*
 * lamino_status -- synchronise `stream`, then report whether a bounded device
 * wait of any kernel of this plan gave up since the last check (the kernel
 * then returned early and its output is invalid). Clears the flag.
 * Returns LAMINO_OK or LAMINO_ETIMEOUT (or ECUDA if the sync failed).
 */
int lamino_status(lamino_plan_t plan, cudaStream_t stream);

/*
 * lamino_selftest_wait -- exercise the failure path of bounded device waits
 * (the method has no counterpart; it is a test hook). Launches on `stream` one
 * kernel that waits, with the same bounded mbarrier wait as the hot-path
 * kernels, on a barrier that nothing arrives at. After `limit_us`
 * microseconds (1 .. 5,000,000, else LAMINO_EINVAL) the wait gives up, the
 * kernel records the failure in the plan's error word and returns; the next
 * lamino_status on `stream` then returns LAMINO_ETIMEOUT and clears it. The
 * device context stays usable. Returns LAMINO_OK once the kernel is queued
 * (ECUDA if the launch failed).
 */
int lamino_selftest_wait(lamino_plan_t plan, unsigned int limit_us, cudaStream_t stream);

/*
 * Tracing: with profiling enabled, every kernel a plan launches is bracketed
 * by two CUDA events recorded on the call's stream. lamino_profile_read waits
 * for the recorded events, returns (name, milliseconds) per launch in launch
 * order (at most `max`), and clears the record.
 */
typedef struct {
    char name[32];
    float ms;
} lamino_kernel_time;

int lamino_profile(lamino_plan_t plan, int enable);
int lamino_profile_read(lamino_plan_t plan, lamino_kernel_time* out, int max, int* n);

/* Bytes of device workspace a form needs beyond the plan tables (admission
 * control by HBM footprint), under the plan's current z chunking. */
int lamino_workspace_bytes(lamino_plan_t plan, int form, size_t* bytes);

/* Device memory the plan holds right now: its tables plus every workspace it
 * has allocated so far (admission control of a server that keeps idle plans
 * resident). */
int lamino_device_bytes(lamino_plan_t plan, size_t* bytes);

/*
 * lamino_set_workspace -- lend the plan a caller-owned device buffer for its
 * workspaces (the role of a work area set on an FFT plan): from now on the
 * Fourier form's two workspaces, and the direct form's filtered rows and
 * 16-byte-pitch copy, are views of `ws` instead of plan-owned allocations, so
 * the calls allocate no workspace (lamino_fbp_host still owns its device copies
 * of the host data). `bytes` must cover lamino_workspace_bytes of the form
 * used, else that call fails with LAMINO_ENOMEM and a message giving both
 * sizes. `ws` must be 256-byte aligned, must stay valid, and must not be used
 * for anything else while calls of this plan that use it are in flight (one
 * buffer can serve many plans whose calls are serialised, e.g. on one stream).
 * Workspaces the plan had allocated itself are freed (which waits for the
 * device). ws = NULL with bytes = 0 returns to plan-owned workspaces,
 * allocated on the next use. Errors: EINVAL (misaligned, or one of ws/bytes
 * zero), ECUDA.
 */
int lamino_set_workspace(lamino_plan_t plan, void* ws, size_t bytes);

/*
 * lamino_set_z_chunk -- change the z chunking of a plan (see lamino_opts.z_chunk;
 * Sec. 5, chunking by slices and columns). Frees the plan's Fourier workspaces
 * (which waits for the device); the next call allocates them for the new
 * layout. Results do not depend on the chunking. Errors: EINVAL (z_chunk < 0).
 */
int lamino_set_z_chunk(lamino_plan_t plan, int z_chunk);

/* Message of the last failure of `plan` (or of the last failed lamino_plan
 * call when plan is NULL). The pointer stays valid until the next call. */
const char* lamino_last_error(lamino_plan_t plan);

/* Free a plan and everything it owns (synchronises the device first). */
int lamino_destroy(lamino_plan_t plan);

#ifdef __cplusplus
}
#endif
#endif /* LAMINO_H */
