// Fourier-form backprojection that allocates no device memory.
//
// lamino_backproject_fourier allocates its two workspaces (row spectra /
// gridded planes, and half spectra / deconvolved planes) with cudaMalloc the
// first time a plan uses the Fourier form. Some callers cannot allow that at
// reconstruction time: a streaming acquisition loop that must not stall on the
// device allocator between frames, a process that runs under an allocator or
// memory pool that owns all device memory (so a stray cudaMalloc would fail or
// fragment the pool), or code that records its work into a CUDA graph, where an
// allocation inside the recorded region is not permitted. For them,
// lamino_backproject_fourier_noalloc runs the same kernels with the workspaces
// placed in one fixed-size array in the library's device globals.
//
// The array is a file-scope __device__ variable: every GPU on which the library
// is loaded holds it until the process exits. Host code must not use its name
// as an address (on the host it is only a stand-in for the device symbol); the
// device address is obtained once per device with cudaGetSymbolAddress, with
// that device current, the first time the entry point runs there.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kScratchBytes = 64ull << 20;   // 64 MiB per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the plan's device (which is current).
int scratch_address(lamino_plan_t p, void** out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (p->device < 0 || p->device >= kMaxDevices)
        return lam::fail(p, LAMINO_EUNSUPPORTED, "device ordinal %d out of range", p->device);
    if (!g_scratch_addr[p->device]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess) return lam::cuda_fail(p, e, "cudaGetSymbolAddress(static scratch)");
        g_scratch_addr[p->device] = ptr;
    }
    *out = g_scratch_addr[p->device];
    return LAMINO_OK;
}

}  // namespace

extern "C" int lamino_backproject_fourier_noalloc(lamino_plan_t p, const void* q, int dtype, float* vol,
                                                  cudaStream_t stream) {
    if (!p) return lam::fail(nullptr, LAMINO_EINVAL, "NULL plan");
    if (!q || !vol) return lam::fail(p, LAMINO_EINVAL, "lamino_backproject_fourier_noalloc: NULL data pointer");
    int rc = lam::validate_dtype_kind(p, dtype, LAMINO_RAMP);
    if (rc) return rc;
    if (!p->fourier_ok) return lam::fail(p, LAMINO_EUNSUPPORTED, "%s", p->fourier_why.c_str());
    size_t a = 0, b = 0;
    lam::fourier_workspace(p, &a, &b);
    const size_t a_al = (a + 255) / 256 * 256;
    if (a_al + b > kScratchBytes)
        return lam::fail(p, LAMINO_EINVAL,
                         "this geometry needs %zu bytes of workspace; the static scratch array of "
                         "lamino_backproject_fourier_noalloc holds %zu bytes (use "
                         "lamino_backproject_fourier)", a_al + b, kScratchBytes);
    if ((rc = lam::set_device(p))) return rc;
    void* base = nullptr;
    if ((rc = scratch_address(p, &base))) return rc;

    // Run the Fourier kernels on views of the static array (no buffer of the
    // plan is touched or allocated), without the tracing events (creating
    // them would allocate).
    const lam::FourierBufs fb = lam::fourier_bufs(p, base, static_cast<unsigned char*>(base) + a_al);
    const bool keep_prof = p->profiling;
    p->profiling = false;
    rc = lam::launch_rowfft(p, q, dtype, fb.R, -1, stream);
    if (!rc) rc = lam::run_fourier_after_rows(p, fb, vol, stream);
    p->profiling = keep_prof;
    return rc;
}
