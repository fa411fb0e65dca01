// Direct form of the laminographic backprojection (Eq. adj, linear
// interpolation on the detector) and its exact transpose (the forward
// operator of Eq. fwd in the same discretisation).
//
// Backprojector: one CTA owns a tile of TX x TY columns (x1, x2) and TZ
// slices; each consumer thread keeps its column's TZ voxels in registers. For
// every angle a producer warp stages the detector footprint of the tile
// (rows/columns the tile projects onto, zero outside the detector) into
// shared memory with a TMA tiled copy; consumers wait on the stage's
// mbarrier, sample bilinearly, and release the stage. Along x3 the detector
// column j = a.x + W/2 is constant (a has no x3 part, Sec. 4), so the
// horizontal weight is computed once per angle and only the row advances.
//
// Every mbarrier wait is bounded (about 2 s of GPU time); on expiry the
// kernel writes an error word, drains its own copies in flight and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "sync.cuh"

namespace lam {
namespace {

constexpr int TX = 32, TY = 8, TZ = 32;
constexpr int kConsumers = TX * TY;              // 256 threads, 8 warps
constexpr int kThreads = kConsumers + 32;        // + 1 producer warp

struct StageMeta {
    float jb, rb;       // tile origin (x1 = X0, x2 = Y0, x3 = Z0) in box coordinates
    float ct, st;       // cos t, sin t
    float stsp, ctsp;   // sin t sin phi, cos t sin phi
    float pad0, pad1;
};

struct DirectArgs {
    const double* trig64;  // [nproj][2]
    float* vol;
    int* err;
    int nproj, n0, n1, n2, W, H;
    int bw, bh, stages, stage_floats;
    double sp, cp;
    float cpf, scale;
};

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

__global__ void __launch_bounds__(kThreads) k_direct(const __grid_constant__ CUtensorMap tmap,
                                                     DirectArgs a) {
    extern __shared__ __align__(128) unsigned char dsm[];
    float* tiles = reinterpret_cast<float*>(dsm);
    StageMeta* meta = reinterpret_cast<StageMeta*>(
        dsm + sizeof(float) * ((size_t)a.stages * a.stage_floats + (size_t)(TZ + 2) * a.bw));
    uint64_t* full = reinterpret_cast<uint64_t*>(meta + a.stages);
    uint64_t* empty = full + a.stages;
    const int S = a.stages;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_addr(full + s), 1);
            mbar_init(smem_addr(empty + s), kConsumers / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int X0i = blockIdx.x * TX, Y0i = blockIdx.y * TY, Z0i = blockIdx.z * TZ;
    if (threadIdx.x >= kConsumers) {
        // ---------------- producer warp (lane 0 issues) ----------------
        if (threadIdx.x != kConsumers) return;
        const double X0 = X0i - 0.5 * a.n0, Y0 = Y0i - 0.5 * a.n1, Z0 = Z0i - 0.5 * a.n2;
        const uint32_t bytes = (uint32_t)(sizeof(float) * a.bw * a.bh);
        int issued = 0;
        bool ok = true;
        for (int k = 0; k < a.nproj; ++k) {
            const int s = k % S;
            if (k >= S && !mbar_wait(smem_addr(empty + s), ((k / S) & 1) ^ 1)) {
                atomicExch(a.err, 1);
                ok = false;
                break;
            }
            const double ct = a.trig64[2 * k], st = a.trig64[2 * k + 1];
            const double cj1 = ct, cj2 = st;                          // j = cj1 x1 + cj2 x2 + W/2
            const double cr1 = st * a.sp, cr2 = -ct * a.sp, cr3 = a.cp; // r = cr.x + H/2
            double jmin = 0.5 * a.W + cj1 * (cj1 >= 0 ? X0 : X0 + TX - 1) + cj2 * (cj2 >= 0 ? Y0 : Y0 + TY - 1);
            double rmin = 0.5 * a.H + cr1 * (cr1 >= 0 ? X0 : X0 + TX - 1) +
                          cr2 * (cr2 >= 0 ? Y0 : Y0 + TY - 1) + cr3 * (cr3 >= 0 ? Z0 : Z0 + TZ - 1);
            // one guard column/row before the footprint keeps every rounded
            // coordinate >= 1 inside the box
            int js = (int)floor(jmin) - 1;
            js -= ((js % 4) + 4) % 4;                 // TMA: x offset a multiple of 16 bytes
            int rs = (int)floor(rmin) - 1;
            StageMeta m;
            m.jb = (float)(0.5 * a.W + cj1 * X0 + cj2 * Y0 - js);
            m.rb = (float)(0.5 * a.H + cr1 * X0 + cr2 * Y0 + cr3 * Z0 - rs);
            m.ct = (float)ct;
            m.st = (float)st;
            m.stsp = (float)cr1;
            m.ctsp = (float)(ct * a.sp);
            m.pad0 = m.pad1 = 0.f;
            meta[s] = m;
            mbar_expect_tx(smem_addr(full + s), bytes);
            tma_load_3d(smem_addr(tiles + (size_t)s * a.stage_floats), &tmap, js, rs, k, smem_addr(full + s));
            ++issued;
        }
        // drain: wait for the copies this thread issued last (bounded)
        for (int k = std::max(0, issued - S); k < issued; ++k)
            if (!mbar_wait(smem_addr(full + (k % S)), (k / S) & 1)) atomicExch(a.err, 2);
        (void)ok;
        return;
    }

    // ---------------- consumers ----------------
    // a warp covers an 8 x 4 patch of columns: its lanes then sample at most
    // ~5 detector rows instead of up to 11
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int tx = (lane & 7) + 8 * (wq & 3), ty = (lane >> 3) + 4 * (wq >> 2);
    float acc[TZ];
#pragma unroll
    for (int z = 0; z < TZ; ++z) acc[z] = 0.f;
    const float cpf = a.cpf;
    const int bw = a.bw, bh = a.bh;
    for (int k = 0; k < a.nproj; ++k) {
        const int s = k % S;
        if (!mbar_wait(smem_addr(full + s), (k / S) & 1)) {
            atomicExch(a.err, 3);
            return;
        }
        const StageMeta m = meta[s];
        const float* tile = tiles + (size_t)s * a.stage_floats;
        const float jl = m.jb + m.ct * (float)tx + m.st * (float)ty;
        const float jf = floorf(jl);
        const float fj = jl - jf;
        const int j0 = min(max((int)jf, 0), bw - 2);
        // row walk: r(z) = rl + cos(phi) z advances by at most one row per slice
        const float rl = m.rb + m.stsp * (float)tx - m.ctsp * (float)ty;
        const float rf = floorf(rl);
        float fr = rl - rf;
        int r0 = (int)rf;
        // the walk adds at most TZ rows; the stage buffers carry TZ + 2 rows of
        // slack after the last stage, so every read stays inside shared memory
        r0 = min(max(r0, 0), bh - 2);
        const float* p = tile + j0 + r0 * bw;
        float h_lo = fmaf(fj, p[1] - p[0], p[0]);              // row r0, lerped in u
        p += bw;                                               // row r0 + 1
        float h_hi = fmaf(fj, p[1] - p[0], p[0]);
#pragma unroll
        for (int z = 0; z < TZ; ++z) {
            acc[z] += fmaf(fr, h_hi - h_lo, h_lo);
            fr += cpf;
            const bool adv = fr >= 1.f;
            fr = adv ? fr - 1.f : fr;
            p += adv ? bw : 0;
            h_lo = adv ? h_hi : h_lo;
            h_hi = fmaf(fj, p[1] - p[0], p[0]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(empty + s));
    }
    const int i0 = X0i + tx, i1 = Y0i + ty;
    if (i0 < a.n0 && i1 < a.n1) {
#pragma unroll
        for (int z = 0; z < TZ; ++z) {
            const int i2 = Z0i + z;
            if (i2 < a.n2) a.vol[((size_t)i2 * a.n1 + i1) * a.n0 + i0] = acc[z] * a.scale;
        }
    }
}

// Transpose of the bilinear sum without the pi/nproj factor: every voxel adds
// its value times the four bilinear weights to the detector. A CTA owns a
// voxel tile; per angle it accumulates into a shared-memory footprint tile
// (shared atomics) and then adds the footprint to the projection (global
// atomics). d must be zeroed first.
__global__ void __launch_bounds__(kConsumers) k_project(const float* __restrict__ vol, float* d,
                                                        DirectArgs a) {
    extern __shared__ float foot[];
    const int bw = a.bw, bh = a.bh;
    const int X0i = blockIdx.x * TX, Y0i = blockIdx.y * TY, Z0i = blockIdx.z * TZ;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int i0 = X0i + tx, i1 = Y0i + ty;
    float val[TZ];
#pragma unroll
    for (int z = 0; z < TZ; ++z) {
        const int i2 = Z0i + z;
        val[z] = (i0 < a.n0 && i1 < a.n1 && i2 < a.n2) ? vol[((size_t)i2 * a.n1 + i1) * a.n0 + i0] : 0.f;
    }
    const double X0 = X0i - 0.5 * a.n0, Y0 = Y0i - 0.5 * a.n1, Z0 = Z0i - 0.5 * a.n2;
    for (int k = 0; k < a.nproj; ++k) {
        for (int i = threadIdx.x; i < bw * bh; i += blockDim.x) foot[i] = 0.f;
        const double ct = a.trig64[2 * k], st = a.trig64[2 * k + 1];
        const double cr1 = st * a.sp, cr2 = -ct * a.sp, cr3 = a.cp;
        double jmin = 0.5 * a.W + ct * (ct >= 0 ? X0 : X0 + TX - 1) + st * (st >= 0 ? Y0 : Y0 + TY - 1);
        double rmin = 0.5 * a.H + cr1 * (cr1 >= 0 ? X0 : X0 + TX - 1) + cr2 * (cr2 >= 0 ? Y0 : Y0 + TY - 1) +
                      cr3 * (cr3 >= 0 ? Z0 : Z0 + TZ - 1);
        const int js = (int)floor(jmin) - 1, rs = (int)floor(rmin) - 1;
        const float jb = (float)(0.5 * a.W + ct * X0 + st * Y0 - js);
        const float rb = (float)(0.5 * a.H + cr1 * X0 + cr2 * Y0 + cr3 * Z0 - rs);
        __syncthreads();
        const float jl = jb + (float)ct * tx + (float)st * ty;
        const float jf = floorf(jl), fj = jl - jf;
        const int j0 = min(max((int)jf, 0), bw - 2);
        const float rl = rb + (float)cr1 * tx + (float)cr2 * ty;
#pragma unroll
        for (int z = 0; z < TZ; ++z) {
            if (val[z] == 0.f) continue;
            const float r = fmaf(a.cpf, (float)z, rl);
            const float rf = floorf(r), fr = r - rf;
            const int r0 = min(max((int)rf, 0), bh - 2);
            float* p = foot + r0 * bw + j0;
            const float v = val[z];
            atomicAdd(p, (1.f - fj) * (1.f - fr) * v);
            atomicAdd(p + 1, fj * (1.f - fr) * v);
            atomicAdd(p + bw, (1.f - fj) * fr * v);
            atomicAdd(p + bw + 1, fj * fr * v);
        }
        __syncthreads();
        float* dk = d + (size_t)k * a.H * a.W;
        for (int i = threadIdx.x; i < bw * bh; i += blockDim.x) {
            const float v = foot[i];
            if (v == 0.f) continue;
            const int rr = rs + i / bw, jj = js + i % bw;
            if (rr >= 0 && rr < a.H && jj >= 0 && jj < a.W) atomicAdd(dk + (size_t)rr * a.W + jj, v);
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
    }
    return fn;
}

DirectArgs make_args(lamino_plan_t p) {
    DirectArgs a;
    a.trig64 = p->d_trig64;
    a.vol = nullptr;
    a.err = p->d_err;
    a.nproj = p->nproj; a.n0 = p->n0; a.n1 = p->n1; a.n2 = p->n2; a.W = p->W; a.H = p->H;
    a.bw = p->dcfg.bw; a.bh = p->dcfg.bh; a.stages = p->dcfg.stages;
    a.stage_floats = (a.bw * a.bh + 31) / 32 * 32;   // 128-byte aligned stages
    a.sp = sin(p->tilt);
    a.cp = cos(p->tilt);
    a.cpf = (float)a.cp;
    a.scale = (float)(3.14159265358979323846 / p->nproj);
    return a;
}

}  // namespace

int launch_direct(lamino_plan_t p, const float* q, float* vol, cudaStream_t s) {
    // TMA needs a 16-byte aligned base and row pitch; otherwise stage a padded copy
    const float* src = q;
    int pitch = p->W;
    if ((p->W % 4) || ((uintptr_t)q % 16)) {
        pitch = (p->W + 3) / 4 * 4;
        size_t need = sizeof(float) * (size_t)p->nproj * p->H * pitch;
        int rc = ensure_buffer(p, (void**)&p->q_buf, &p->q_buf_bytes, need, "padded projections");
        if (rc) return rc;
        if (p->q_buf == q) return fail(p, LAMINO_EUNSUPPORTED, "unaligned input aliases the plan buffer");
        LAM_CUDA(p, cudaMemsetAsync(p->q_buf, 0, need, s));
        LAM_CUDA(p, cudaMemcpy2DAsync(p->q_buf, sizeof(float) * pitch, q, sizeof(float) * p->W,
                                      sizeof(float) * p->W, (size_t)p->nproj * p->H, cudaMemcpyDeviceToDevice, s));
        src = p->q_buf;
    }
    PFN_cuTensorMapEncodeTiled_v12000 encode = get_encode();
    if (!encode) return fail(p, LAMINO_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    CUtensorMap map;
    cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)p->H, (cuuint64_t)p->nproj};
    cuuint64_t strides[2] = {sizeof(float) * (cuuint64_t)pitch, sizeof(float) * (cuuint64_t)pitch * p->H};
    cuuint32_t box[3] = {(cuuint32_t)p->dcfg.bw, (cuuint32_t)p->dcfg.bh, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult cr = encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)src, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return fail(p, LAMINO_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
    DirectArgs a = make_args(p);
    a.vol = vol;
    size_t smem = sizeof(float) * ((size_t)a.stages * a.stage_floats + (size_t)(TZ + 2) * a.bw) +
                  sizeof(StageMeta) * a.stages + 2 * sizeof(uint64_t) * a.stages;
    dim3 grid((p->n0 + TX - 1) / TX, (p->n1 + TY - 1) / TY, (p->n2 + TZ - 1) / TZ);
    cudaFuncSetAttribute(k_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    ProfScope prof(p, "direct", s);
    k_direct<<<grid, kThreads, smem, s>>>(map, a);
    LAM_LAUNCH_CHECK(p, "direct backprojection kernel");
    return LAMINO_OK;
}

int launch_project_direct(lamino_plan_t p, const float* vol, float* d, cudaStream_t s) {
    LAM_CUDA(p, cudaMemsetAsync(d, 0, sizeof(float) * (size_t)p->nproj * p->H * p->W, s));
    DirectArgs a = make_args(p);
    // the footprint box here needs no alignment slack but keep the same size
    size_t smem = sizeof(float) * (size_t)a.bw * a.bh;
    dim3 grid((p->n0 + TX - 1) / TX, (p->n1 + TY - 1) / TY, (p->n2 + TZ - 1) / TZ);
    cudaFuncSetAttribute(k_project, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    ProfScope prof(p, "project", s);
    k_project<<<grid, kConsumers, smem, s>>>(vol, d, a);
    LAM_LAUNCH_CHECK(p, "direct projector kernel");
    return LAMINO_OK;
}

}  // namespace lam
