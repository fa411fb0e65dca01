// Direct form of the laminographic backprojection (Eq. adj, linear
// interpolation on the detector) and its exact transpose (the forward
// operator of Eq. fwd in the same discretisation).
//
// Backprojector: one CTA owns a tile of BX x BY columns (x1, x2) and BZ
// slices; each consumer thread keeps the BZ voxels of its two columns in
// registers as packed pairs. For every angle a producer warp stages the
// detector footprint of the tile
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

// Backprojector tile: BX x BY columns x BZ slices; each of the 256 consumer
// threads owns two columns (x2 = y and y + BY/2) whose updates run as packed
// f32x2 arithmetic. Projector tile (k_project): TX x TY columns x TZ slices.
constexpr int BX = 32, BY = 16, BZ = 32;
constexpr int TX = 32, TY = 8, TZ = 32;
constexpr int kConsumers = 256;                  // 8 warps
constexpr int kThreads = kConsumers + 32;        // + 1 producer warp
static_assert(BX * BY == 2 * kConsumers && TX * TY == kConsumers, "thread layout");

// packed pairs of floats (one 64-bit register pair) and f32x2 arithmetic
__device__ __forceinline__ unsigned long long pk(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(unsigned long long r, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

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
    int z0;                // first slice of the launch (z chunking); blockIdx.z counts tiles from it
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
        dsm + sizeof(float) * ((size_t)a.stages * a.stage_floats + (size_t)(BZ + 2) * a.bw));
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

    const int X0i = blockIdx.x * BX, Y0i = blockIdx.y * BY, Z0i = a.z0 + blockIdx.z * BZ;
    if (threadIdx.x >= kConsumers) {
        // ---------------- producer warp (lane 0 issues) ----------------
        if (threadIdx.x != kConsumers) return;
        const double X0 = X0i - 0.5 * a.n0, Y0 = Y0i - 0.5 * a.n1, Z0 = Z0i - 0.5 * a.n2;
        const uint32_t bytes = (uint32_t)(sizeof(float) * a.bw * a.bh);
        int issued = 0;
        for (int k = 0; k < a.nproj; ++k) {
            const int s = k % S;
            if (k >= S && !mbar_wait(smem_addr(empty + s), ((k / S) & 1) ^ 1)) {
                atomicExch(a.err, 1);
                break;
            }
            const double ct = a.trig64[2 * k], st = a.trig64[2 * k + 1];
            const double cj1 = ct, cj2 = st;                          // j = cj1 x1 + cj2 x2 + W/2
            const double cr1 = st * a.sp, cr2 = -ct * a.sp, cr3 = a.cp; // r = cr.x + H/2
            double jmin = 0.5 * a.W + cj1 * (cj1 >= 0 ? X0 : X0 + BX - 1) + cj2 * (cj2 >= 0 ? Y0 : Y0 + BY - 1);
            double rmin = 0.5 * a.H + cr1 * (cr1 >= 0 ? X0 : X0 + BX - 1) +
                          cr2 * (cr2 >= 0 ? Y0 : Y0 + BY - 1) + cr3 * (cr3 >= 0 ? Z0 : Z0 + BZ - 1);
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
        return;
    }

    // ---------------- consumers ----------------
    // a warp covers an 8 x 4 patch of columns (and the patch 8 rows of x2
    // further): its lanes then sample at most ~5 detector rows per load
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int tx = (lane & 7) + 8 * (wq & 3), ty = (lane >> 3) + 4 * (wq >> 2);
    constexpr int DY = BY / 2;                  // second column: x2 = ty + DY
    unsigned long long acc[BZ];                 // (column ty, column ty + DY) per slice
#pragma unroll
    for (int z = 0; z < BZ; ++z) acc[z] = 0ull;   // +0.0f in both halves
    const float cpf = a.cpf;
    const unsigned long long cpf2 = pk(cpf, cpf);
    const int bw = a.bw, bh = a.bh;
    for (int k = 0; k < a.nproj; ++k) {
        const int s = k % S;
        if (!mbar_wait(smem_addr(full + s), (k / S) & 1)) {
            atomicExch(a.err, 3);
            return;
        }
        const StageMeta m = meta[s];
        const float* tile = tiles + (size_t)s * a.stage_floats;
        // per column: detector column j (constant along x3) and the row walk
        // r(z) = rl + cos(phi) z, which advances by at most one row per slice
        float fj[2], fr[2];
        const float* p[2];
        float lo[2], hi[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float y = (float)(ty + c * DY);
            const float jl = m.jb + m.ct * (float)tx + m.st * y;
            const float jf = floorf(jl);
            fj[c] = jl - jf;
            const int j0 = min(max((int)jf, 0), bw - 2);
            const float rl = m.rb + m.stsp * (float)tx - m.ctsp * y;
            const float rf = floorf(rl);
            fr[c] = rl - rf;
            // the walk adds at most BZ rows; the stage buffers carry BZ + 2
            // rows of slack after the last stage, so every read stays inside
            // shared memory
            const int r0 = min(max((int)rf, 0), bh - 2);
            const float* q = tile + j0 + r0 * bw;
            lo[c] = fmaf(fj[c], q[1] - q[0], q[0]);             // row r0, lerped in u
            q += bw;                                              // row r0 + 1
            hi[c] = fmaf(fj[c], q[1] - q[0], q[0]);
            p[c] = q;
        }
        const unsigned long long fj2 = pk(fj[0], fj[1]);
        unsigned long long fr2 = pk(fr[0], fr[1]);
        unsigned long long hlo = pk(lo[0], lo[1]), hhi = pk(hi[0], hi[1]);
#pragma unroll
        for (int z = 0; z < BZ; ++z) {
            acc[z] = add2(acc[z], fma2(fr2, sub2(hhi, hlo), hlo));
            fr2 = add2(fr2, cpf2);
            float f0, f1, h0, h1, l0, l1;
            upk(fr2, f0, f1);
            upk(hhi, h0, h1);
            upk(hlo, l0, l1);
            const bool a0 = f0 >= 1.f, a1 = f1 >= 1.f;
            f0 = a0 ? f0 - 1.f : f0;
            f1 = a1 ? f1 - 1.f : f1;
            p[0] += a0 ? bw : 0;
            p[1] += a1 ? bw : 0;
            l0 = a0 ? h0 : l0;
            l1 = a1 ? h1 : l1;
            fr2 = pk(f0, f1);
            hlo = pk(l0, l1);
            const unsigned long long s0 = pk(p[0][0], p[1][0]), s1 = pk(p[0][1], p[1][1]);
            hhi = fma2(fj2, sub2(s1, s0), s0);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(empty + s));
    }
    const int i0 = X0i + tx;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int i1 = Y0i + ty + c * DY;
        if (i0 >= a.n0 || i1 >= a.n1) continue;
#pragma unroll
        for (int z = 0; z < BZ; ++z) {
            float v0, v1;
            upk(acc[z], v0, v1);
            const int i2 = Z0i + z;
            if (i2 < a.n2) a.vol[((size_t)i2 * a.n1 + i1) * a.n0 + i0] = (c == 0 ? v0 : v1) * a.scale;
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

DirectArgs make_args(lamino_plan_t p, const DirectCfg& cfg) {
    DirectArgs a;
    a.trig64 = p->d_trig64;
    a.vol = nullptr;
    a.err = p->d_err;
    a.nproj = p->nproj; a.n0 = p->n0; a.n1 = p->n1; a.n2 = p->n2; a.W = p->W; a.H = p->H;
    a.z0 = 0;
    a.bw = cfg.bw; a.bh = cfg.bh; a.stages = cfg.stages;
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
        float* qp = nullptr;
        int rc = pad_buffer(p, need, &qp);
        if (rc) return rc;
        LAM_CUDA(p, cudaMemsetAsync(qp, 0, need, s));
        LAM_CUDA(p, cudaMemcpy2DAsync(qp, sizeof(float) * pitch, q, sizeof(float) * p->W,
                                      sizeof(float) * p->W, (size_t)p->nproj * p->H, cudaMemcpyDeviceToDevice, s));
        src = qp;
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
    DirectArgs a = make_args(p, p->dcfg);
    a.vol = vol;
    size_t smem = sizeof(float) * ((size_t)a.stages * a.stage_floats + (size_t)(BZ + 2) * a.bw) +
                  sizeof(StageMeta) * a.stages + 2 * sizeof(uint64_t) * a.stages;
    cudaFuncSetAttribute(k_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // z chunking: one launch per slab of zs output slices (a multiple of the
    // tile depth, so that the slabs' tiles never overlap); the last slab's
    // tiles stop at n2 inside the kernel
    const int zs = p->z_chunk > 0 ? (p->z_chunk + BZ - 1) / BZ * BZ : (p->n2 + BZ - 1) / BZ * BZ;
    for (int z0 = 0; z0 < p->n2; z0 += zs) {
        a.z0 = z0;
        const int nz = std::min(zs, p->n2 - z0);
        dim3 grid((p->n0 + BX - 1) / BX, (p->n1 + BY - 1) / BY, (nz + BZ - 1) / BZ);
        ProfScope prof(p, "direct", s);
        k_direct<<<grid, kThreads, smem, s>>>(map, a);
        LAM_LAUNCH_CHECK(p, "direct backprojection kernel");
    }
    return LAMINO_OK;
}

int launch_project_direct(lamino_plan_t p, const float* vol, float* d, cudaStream_t s) {
    LAM_CUDA(p, cudaMemsetAsync(d, 0, sizeof(float) * (size_t)p->nproj * p->H * p->W, s));
    DirectArgs a = make_args(p, p->pcfg);
    size_t smem = sizeof(float) * (size_t)a.bw * a.bh;
    dim3 grid((p->n0 + TX - 1) / TX, (p->n1 + TY - 1) / TY, (p->n2 + TZ - 1) / TZ);
    cudaFuncSetAttribute(k_project, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    ProfScope prof(p, "project", s);
    k_project<<<grid, kConsumers, smem, s>>>(vol, d, a);
    LAM_LAUNCH_CHECK(p, "direct projector kernel");
    return LAMINO_OK;
}

}  // namespace lam
