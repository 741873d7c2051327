// 3D convolution (3x3x3 taps, zero padding, stride 1) as an implicit GEMM on
// the fifth-generation tensor cores (tcgen05), for the small volume CNN of
// the learned initial proposal.
//
// GEMM view: D[m][n] = sum_k A[m][k] B[n][k], m = voxel (x fastest),
// n = output channel, k = tap * Cin + c with tap = (dz+1)*9 + (dy+1)*3 +
// (dx+1). A is the im2col of the channels-last bf16 input gathered on the
// fly; B is the bf16 weight matrix [Cout][Kp] (K padded with zeros to a
// multiple of 64). D accumulates in FP32 in tensor memory.
//
// One CTA = 128 voxels x Cout (Cout in {16, 32, 64}); 4 warps, one thread
// per voxel row.
//   * K is walked in steps of 64 (one 128-byte row chunk per voxel) through
//     two shared-memory stages in the canonical K-major, non-swizzled layout:
//     8 x 16-byte core matrices, 128 bytes each, adjacent along K (leading
//     byte offset 128) and 8-row groups 1024 bytes apart (stride byte
//     offset).
//   * Every thread gathers its voxel's 64 im2col values of the step (16-byte
//     loads when Cin is a multiple of 8), the CTA loads the step's weights,
//     and after a proxy fence and a barrier one thread issues four
//     tcgen05.mma (M = 128, N = Cout, K = 16 each) and commits them to the
//     stage's mbarrier, which the stage's next overwrite waits on.
//   * Epilogue: each warp reads its 32 accumulator lanes with tcgen05.ld,
//     adds the bias, applies ReLU if asked and stores the voxel's channels
//     (bf16 or fp32, channels-last).
// Every mbarrier wait is bounded; a wait that gives up sets a status word
// (sbp_cnn_status) and the CTA skips to its clean-up.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <cuda_pipeline.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "sbp_internal.cuh"

namespace {

constexpr int kTcRows = 128;     // voxels per CTA (the MMA's M)
constexpr int kTcBK = 64;        // K per stage
constexpr int kTcThreads = 128;
constexpr int kTcCols = 64;      // TMEM columns allocated (>= Cout, power of two >= 32)
constexpr long long kWaitLimit = 1LL << 24;

__device__ int g_cnn_status;  // 0, or 1 when a bounded wait gave up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// UMMA shared-memory descriptor: start >> 4 in bits 0-13, leading byte
// offset >> 4 in 16-29, stride byte offset >> 4 in 32-45, version 1 in
// 46-47, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 and 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in
// bits 24-28.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Waits for the phase with the given parity to complete; false after the
// iteration limit.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// 16 consecutive fp32 columns of this thread's lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Activation layouts: channels-last [V][C], or planar [C / 8][V][8] (planes
// of 8 channels, 16 bytes per voxel), which gives a tile's halo box rows of
// ten voxels (160 bytes) instead of one (16 bytes).
struct ConvArgs {
    const __nv_bfloat16* in;  // [V][Cin], or planar (in_planar)
    const __nv_bfloat16* w;   // [Cout][Kp]
    const float* bias;        // [Cout] or null
    void* out;                // [V][Cout], bf16 or fp32; or planar bf16 (out_planar)
    int nx, ny, nz;
    int Kp;
    int in_planar, out_planar;
    long long V;
};

// Stores channels c0 .. c0 + 15 (c0 a multiple of 16) of voxel q as bf16:
// one 32-byte run channels-last, or 16 bytes in each of two planes.
template <int C>
__device__ __forceinline__ void store16_bf16(const ConvArgs& a, long long q, int c0,
                                             const float* v) {
    __nv_bfloat162 h[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    __nv_bfloat16* const out = static_cast<__nv_bfloat16*>(a.out);
    uint4* o0;
    uint4* o1;
    if (a.out_planar) {
        o0 = reinterpret_cast<uint4*>(out + ((long long)(c0 >> 3) * a.V + q) * 8);
        o1 = reinterpret_cast<uint4*>(out + ((long long)((c0 >> 3) + 1) * a.V + q) * 8);
    } else {
        o0 = reinterpret_cast<uint4*>(out + q * C + c0);
        o1 = o0 + 1;
    }
    *o0 = *reinterpret_cast<uint4*>(&h[0]);
    *o1 = *reinterpret_cast<uint4*>(&h[4]);
}

template <int CIN, int COUT, bool RELU, bool OUT_F32>
__global__ void __launch_bounds__(kTcThreads) conv3d_tc_kernel(ConvArgs a) {
    static_assert(COUT % 16 == 0 && COUT >= 16 && COUT <= kTcCols, "Cout must be 16, 32 or 64");
    // two stages of A (128 rows x 64) then two of B (COUT rows x 64), bf16
    extern __shared__ __align__(1024) uint8_t s_dyn[];
    constexpr int kABytes = kTcRows * kTcBK * 2, kBBytes = COUT * kTcBK * 2;
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t s_tmem;

    const int tid = threadIdx.x, warp = tid >> 5;
    const long long V = (long long)a.nx * a.ny * a.nz;
    const long long m = (long long)blockIdx.x * kTcRows + tid;  // this thread's voxel
    const bool mv = m < V;
    int x = 0, y = 0, z = 0;
    if (mv) {
        x = (int)(m % a.nx);
        y = (int)((m / a.nx) % a.ny);
        z = (int)(m / ((long long)a.nx * a.ny));
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    constexpr uint32_t idesc = umma_idesc_bf16(kTcRows, COUT);
    const int nk = a.Kp / kTcBK;
    constexpr int K = 27 * CIN;
    uint32_t phase[2] = {0u, 0u};
    bool ok = true;

    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt & 1;
        if (kt >= 2) {  // the MMAs that read this stage two steps ago must be done
            if (!mbar_wait(&bar[st], phase[st])) ok = false;
            phase[st] ^= 1u;
        }
        if (!__syncthreads_and(ok)) break;
        // this thread's row: 8 chunks of 8 K-values (16 bytes each)
        uint8_t* rowA = s_dyn + st * kABytes + ((tid >> 3) * 8) * 128 + (tid & 7) * 16;
#pragma unroll
        for (int kc = 0; kc < 8; ++kc) {
            const int k0 = kt * kTcBK + kc * 8;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (mv && k0 < K) {
                if constexpr (CIN % 8 == 0) {
                    const int tap = k0 / CIN, c0 = k0 % CIN;
                    const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
                    const int xx = x + dx, yy = y + dy, zz = z + dz;
                    if (xx >= 0 && xx < a.nx && yy >= 0 && yy < a.ny && zz >= 0 && zz < a.nz) {
                        const long long q = ((long long)zz * a.ny + yy) * a.nx + xx;
                        v = *reinterpret_cast<const uint4*>(a.in + q * CIN + c0);
                    }
                } else {
                    union {
                        uint4 u;
                        __nv_bfloat16 h[8];
                    } e;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int k = k0 + j;
                        e.h[j] = __float2bfloat16(0.0f);
                        if (k < K) {
                            const int tap = k / CIN, c = k % CIN;
                            const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
                            const int xx = x + dx, yy = y + dy, zz = z + dz;
                            if (xx >= 0 && xx < a.nx && yy >= 0 && yy < a.ny && zz >= 0 &&
                                zz < a.nz)
                                e.h[j] = a.in[(((long long)zz * a.ny + yy) * a.nx + xx) * CIN + c];
                        }
                    }
                    v = e.u;
                }
            }
            *reinterpret_cast<uint4*>(rowA + kc * 128) = v;
        }
        // weights of the step: COUT rows x 8 chunks
        for (int t = tid; t < COUT * 8; t += kTcThreads) {
            const int n = t >> 3, kc = t & 7;
            const uint4 v =
                *reinterpret_cast<const uint4*>(a.w + (size_t)n * a.Kp + kt * kTcBK + kc * 8);
            *reinterpret_cast<uint4*>(s_dyn + 2 * kABytes + st * kBBytes + ((n >> 3) * 8 + kc) * 128 +
                                      (n & 7) * 16) = v;
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(s_dyn + st * kABytes);
            const uint32_t b0 = smem_u32(s_dyn + 2 * kABytes + st * kBBytes);
#pragma unroll
            for (int ks = 0; ks < kTcBK / 16; ++ks)  // K = 16 per MMA: two core matrices
                tc_mma(tmem, umma_desc(a0 + ks * 256, 128, 1024), umma_desc(b0 + ks * 256, 128, 1024),
                       idesc, (kt > 0 || ks > 0) ? 1u : 0u);
            tc_commit(&bar[st]);
        }
    }
    // wait for the last commit of each stage still outstanding
    if (ok) {
        for (int s = 0; s < 2; ++s) {
            const int uses = nk > s ? (nk - 1 - s) / 2 + 1 : 0;  // commits made on stage s
            const int waited = uses > 0 ? uses - 1 : 0;          // of them already waited on
            if (uses > waited && !mbar_wait(&bar[s], phase[s])) ok = false;
        }
    }
    tc_fence_after();
    if (!__syncthreads_and(ok)) {
        if (tid == 0) atomicExch(&g_cnn_status, 1);
    } else {
        // epilogue: lane = voxel row, columns = output channels (every lane
        // takes part in the warp-wide tcgen05.ld)
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int c0 = 0; c0 < COUT; c0 += 16) {
            float v[16];
            tc_ld16(taddr + c0, v);
            if (mv) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float r = v[j] + (a.bias ? a.bias[c0 + j] : 0.0f);
                    if (RELU) r = fmaxf(r, 0.0f);
                    v[j] = r;
                }
                if constexpr (OUT_F32) {
                    float4* o = reinterpret_cast<float4*>(static_cast<float*>(a.out) + m * COUT + c0);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                } else {
                    store16_bf16<COUT>(a, m, c0, v);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTcCols)
                     : "memory");
}

// Halo variant (Cin a multiple of 16). A CTA computes a tile of 8 x 16 x 1
// voxels (m = ty * 8 + tx, so the 16 groups of 8 MMA rows are the tile's 16
// rows along y). The tile's input halo (10 x 18 x 3 voxels, zeros outside the
// volume) is copied once into shared memory, chunk-major: [cc][hz][hy][hx]
// with 16 bytes (8 channels) per voxel. For tap (dx, dy, dz) the im2col rows
// of the 8 voxels of a tile row are then 8 consecutive 16-byte entries of
// one halo row, which is a canonical K-major core matrix: the A operand of
// the tap is a descriptor pointing into the halo (leading byte offset = one
// chunk plane, stride byte offset = one halo row), and no im2col copy is
// made. The weights of all 27 taps are staged once ([tap][cc][n] x 16
// bytes). One thread then issues the 27 * Cin / 16 MMAs (M = 128, N = Cout,
// K = 16) back to back and commits them to one mbarrier.
constexpr int kHTX = 8, kHTY = 16;                 // tile
constexpr int kHX = kHTX + 2, kHY = kHTY + 2, kHZ = 3;  // halo
constexpr int kHV = kHX * kHY * kHZ;

template <int CIN, int COUT>
constexpr int halo_smem_bytes() {
    return CIN / 8 * kHV * 16 + 27 * (CIN / 8) * COUT * 16;
}

// One input channel (the network's first layer). A CTA takes an 8 x 16 x 4
// block of voxels, four MMA tiles of 128 stacked along z, and stages the
// block's 10 x 18 x 6 input halo in shared memory (zero outside the volume).
// Each thread then writes its voxel row of every tile's im2col operand from
// the halo: the 27 taps padded with zeros to K = 32, in the canonical K-major
// layout (core matrices 128 bytes apart along K, 8-row groups 512 bytes
// apart). One thread issues two K = 16 MMAs per tile, each tile into its own
// COUT columns of TMEM, and one commit; the epilogue then reads all four.
// (The gather kernel read its 27 values per voxel from global memory and
// built one tile per CTA.)
constexpr int kC1Tiles = 4;                 // z-slices per CTA
constexpr int kC1HZ = kC1Tiles + 2;         // halo depth
constexpr int kC1K = 32;                    // 27 taps padded
constexpr int kC1TileBytes = kTcRows * kC1K * 2;

template <int COUT, bool RELU, bool OUT_F32>
__global__ void __launch_bounds__(kTcThreads) conv3d_c1_kernel(ConvArgs a) {
    static_assert(COUT % 16 == 0 && COUT * kC1Tiles <= kTcCols, "every tile needs its columns");
    __shared__ __align__(1024) uint8_t s_a[kC1Tiles * kC1TileBytes];
    __shared__ __align__(128) uint8_t s_b[COUT * kC1K * 2];
    __shared__ __nv_bfloat16 s_h[kC1HZ * kHY * kHX];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_tmem;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int x0 = blockIdx.x * kHTX, y0 = blockIdx.y * kHTY, z0 = blockIdx.z * kC1Tiles;
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the halo, x fastest
    for (int i = tid; i < kC1HZ * kHY * kHX; i += kTcThreads) {
        const int hx = i % kHX, hy = (i / kHX) % kHY, hz = i / (kHX * kHY);
        const int x = x0 - 1 + hx, y = y0 - 1 + hy, z = z0 - 1 + hz;
        __nv_bfloat16 v = __float2bfloat16(0.0f);
        if (x >= 0 && x < a.nx && y >= 0 && y < a.ny && z >= 0 && z < a.nz)
            v = a.in[((long long)z * a.ny + y) * a.nx + x];
        s_h[i] = v;
    }
    // the weights' first 32 K values: row n, chunk kc at (n / 8) 512 + kc 128 + (n % 8) 16
    for (int t = tid; t < COUT * (kC1K / 8); t += kTcThreads) {
        const int n = t / (kC1K / 8), kc = t % (kC1K / 8);
        *reinterpret_cast<uint4*>(s_b + (n >> 3) * 512 + kc * 128 + (n & 7) * 16) =
            *reinterpret_cast<const uint4*>(a.w + (size_t)n * a.Kp + kc * 8);
    }
    __syncthreads();
    // this thread's row m of each tile: voxel (x0 + m % 8, y0 + m / 8, z0 + t)
    const int m = tid, mx = m & 7, my = m >> 3;
#pragma unroll
    for (int t = 0; t < kC1Tiles; ++t) {
        union {
            uint4 u[4];
            __nv_bfloat16 h[32];
        } row;
#pragma unroll
        for (int k = 0; k < kC1K; ++k) {
            if (k < 27) {
                const int dx = k % 3, dy = (k / 3) % 3, dz = k / 9;
                row.h[k] = s_h[((t + dz) * kHY + my + dy) * kHX + mx + dx];
            } else {
                row.h[k] = __float2bfloat16(0.0f);
            }
        }
        uint8_t* dst = s_a + t * kC1TileBytes + (m >> 3) * 512 + (m & 7) * 16;
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) *reinterpret_cast<uint4*>(dst + kc * 128) = row.u[kc];
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (tid == 0) {
        constexpr uint32_t idesc = umma_idesc_bf16(kTcRows, COUT);
        const uint32_t a0 = smem_u32(s_a), b0 = smem_u32(s_b);
#pragma unroll
        for (int t = 0; t < kC1Tiles; ++t)
#pragma unroll
            for (int ks = 0; ks < kC1K / 16; ++ks)
                tc_mma(tmem + (uint32_t)(t * COUT),
                       umma_desc(a0 + t * kC1TileBytes + ks * 256, 128, 512),
                       umma_desc(b0 + ks * 256, 128, 512), idesc, ks > 0 ? 1u : 0u);
        tc_commit(&bar);
    }
    const bool ok = mbar_wait(&bar, 0u);
    tc_fence_after();
    if (!__syncthreads_and(ok)) {
        if (tid == 0) atomicExch(&g_cnn_status, 1);
    } else {
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        const int x = x0 + mx, y = y0 + my;
#pragma unroll
        for (int t = 0; t < kC1Tiles; ++t) {
            const int z = z0 + t;
            const bool mv = x < a.nx && y < a.ny && z < a.nz;
            const long long q = ((long long)z * a.ny + y) * a.nx + x;
#pragma unroll
            for (int c0 = 0; c0 < COUT; c0 += 16) {
                float v[16];
                tc_ld16(taddr + (uint32_t)(t * COUT + c0), v);
                if (mv) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        float r = v[j] + (a.bias ? a.bias[c0 + j] : 0.0f);
                        if (RELU) r = fmaxf(r, 0.0f);
                        v[j] = r;
                    }
                    if constexpr (OUT_F32) {
                        float4* o =
                            reinterpret_cast<float4*>(static_cast<float*>(a.out) + q * COUT + c0);
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                    } else {
                        store16_bf16<COUT>(a, q, c0, v);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTcCols)
                     : "memory");
}

template <int COUT, bool RELU, bool OUT_F32>
int launch_c1_t(const ConvArgs& a, cudaStream_t st) {
    const dim3 grid((a.nx + kHTX - 1) / kHTX, (a.ny + kHTY - 1) / kHTY,
                    (a.nz + kC1Tiles - 1) / kC1Tiles);
    conv3d_c1_kernel<COUT, RELU, OUT_F32><<<grid, kTcThreads, 0, st>>>(a);
    return SBP_OK;
}

template <int CIN, int COUT, bool RELU, bool OUT_F32>
__global__ void __launch_bounds__(kTcThreads) conv3d_halo_kernel(ConvArgs a) {
    static_assert(CIN % 16 == 0, "one MMA (K = 16) takes two channel chunks of one tap");
    static_assert(COUT % 16 == 0 && COUT >= 16 && COUT <= kTcCols, "Cout must be 16, 32 or 64");
    static_assert(kHTX * kHTY == kTcRows, "a tile is one MMA's M");
    extern __shared__ __align__(1024) uint8_t s_dyn[];
    constexpr int kChunks = CIN / 8;
    constexpr int kPlane = kHV * 16;    // bytes of one 8-channel chunk of the halo
    constexpr int kWBlock = COUT * 16;  // bytes of the weights of one (tap, chunk)
    uint8_t* const s_halo = s_dyn;
    uint8_t* const s_w = s_dyn + kChunks * kPlane;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_tmem;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int x0 = blockIdx.x * kHTX, y0 = blockIdx.y * kHTY, z0 = blockIdx.z;
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the halo: a voxel's chunks are adjacent in global memory (coalesced)
    for (int t = tid; t < kHV * kChunks; t += kTcThreads) {
        const int v = t / kChunks, cc = t - v * kChunks;
        const int hx = v % kHX, hy = (v / kHX) % kHY, hz = v / (kHX * kHY);
        const int xx = x0 + hx - 1, yy = y0 + hy - 1, zz = z0 + hz - 1;
        uint8_t* dst = s_halo + cc * kPlane + v * 16;
        if (xx >= 0 && xx < a.nx && yy >= 0 && yy < a.ny && zz >= 0 && zz < a.nz)
            __pipeline_memcpy_async(
                dst, a.in + (((long long)zz * a.ny + yy) * a.nx + xx) * CIN + cc * 8, 16);
        else
            *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
    // the weights: w[n][tap * CIN + cc * 8 ...] -> [tap][cc][n] (a row's chunks coalesced)
    for (int t = tid; t < COUT * 27 * kChunks; t += kTcThreads) {
        const int n = t / (27 * kChunks), r = t - n * (27 * kChunks);  // r = tap * kChunks + cc
        __pipeline_memcpy_async(s_w + r * kWBlock + n * 16, a.w + (size_t)n * a.Kp + r * 8, 16);
    }
    __pipeline_commit();
    __pipeline_wait_prior(0);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (tid == 0) {
        constexpr uint32_t idesc = umma_idesc_bf16(kTcRows, COUT);
        const uint32_t hb = smem_u32(s_halo), wb = smem_u32(s_w);
        // base descriptors plus compile-time offsets (>> 4) in the start-address
        // field, which cannot carry out of its 14 bits (shared addresses < 256 KB)
        const uint64_t da = umma_desc(hb, kPlane, kHX * 16);
        const uint64_t db = umma_desc(wb, kWBlock, 128);
#pragma unroll
        for (int tap = 0; tap < 27; ++tap) {
            // (dx, dy, dz) + 1 = (tap % 3, tap / 3 % 3, tap / 9): the tile's voxel (0, 0)
            // reads halo voxel (dx + 1, dy + 1, dz + 1)
            const uint32_t aoff = (uint32_t)(((tap / 9) * kHY + (tap / 3) % 3) * kHX + tap % 3) * 16;
#pragma unroll
            for (int kp = 0; kp < kChunks / 2; ++kp)
                tc_mma(tmem, da + ((aoff + 2 * kp * kPlane) >> 4),
                       db + (((tap * kChunks + 2 * kp) * kWBlock) >> 4), idesc,
                       (tap > 0 || kp > 0) ? 1u : 0u);
        }
        tc_commit(&bar);
    }
    const bool ok = mbar_wait(&bar, 0u);
    tc_fence_after();
    if (!__syncthreads_and(ok)) {
        if (tid == 0) atomicExch(&g_cnn_status, 1);
    } else {
        // epilogue: lane = tile row m = ty * 8 + tx, columns = output channels
        const int m = warp * 32 + (tid & 31);
        const int x = x0 + (m & 7), y = y0 + (m >> 3);
        const bool mv = x < a.nx && y < a.ny;
        const long long q = ((long long)z0 * a.ny + y) * a.nx + x;
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int c0 = 0; c0 < COUT; c0 += 16) {
            float v[16];
            tc_ld16(taddr + c0, v);
            if (mv) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float r = v[j] + (a.bias ? a.bias[c0 + j] : 0.0f);
                    if (RELU) r = fmaxf(r, 0.0f);
                    v[j] = r;
                }
                if constexpr (OUT_F32) {
                    float4* o = reinterpret_cast<float4*>(static_cast<float*>(a.out) + q * COUT + c0);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                } else {
                    store16_bf16<COUT>(a, q, c0, v);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTcCols)
                     : "memory");
}

template <int CIN, int COUT, bool RELU, bool OUT_F32>
int launch_halo_t(const ConvArgs& a, cudaStream_t st) {
    constexpr int smem = halo_smem_bytes<CIN, COUT>();
    auto k = conv3d_halo_kernel<CIN, COUT, RELU, OUT_F32>;
    if (sbp_cuda_check(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                       "conv3d_bf16: smem attribute"))
        return SBP_ERR_CUDA;
    const dim3 grid((a.nx + kHTX - 1) / kHTX, (a.ny + kHTY - 1) / kHTY, a.nz);
    k<<<grid, kTcThreads, smem, st>>>(a);
    return SBP_OK;
}

// Persistent TMA variant (Cin 16 or 32), warp-specialised. Each CTA stages
// the weights once and walks its tiles (tile i of the CTA is global tile
// blockIdx.x + i gridDim.x); one or two CTAs per SM, as shared memory allows.
// Each tile's halo comes in by TMA: a 4-D tensor map over the channels-last
// input (channel, x, y, z) and one box of 8 channels x 10 x 18 x 3 per
// 8-channel chunk, which lands as exactly the chunk plane the MMA
// descriptors read (rows of 16 bytes along x); outside the volume TMA fills
// zeros. Roles, linked only by mbarriers (no CTA-wide barrier per tile):
//   warp 0, one lane   producer: the halo of tile i into slot i % kSlots,
//                      once the MMAs of tile i - kSlots have released it
//   warp 1, one lane   MMA issuer: the 27 Cin / 16 MMAs of tile i into TMEM
//                      buffer i & 1, once its halo has landed and the
//                      epilogue of tile i - 2 has read that buffer; two
//                      commits then release the slot and publish the buffer
//   warps 2 - 5        epilogue: tcgen05.ld of the warp's quarter of the
//                      128 TMEM lanes, bias, ReLU, store; one arrive per warp
//                      frees the buffer
// So the producer runs up to kSlots tiles ahead and the MMAs of tile i + 1
// overlap the epilogue of tile i. Every wait is bounded; a role that gives up
// sets the status word and stops, and the others' waits then run out too.
constexpr int kWsThreads = 192;
constexpr int kPlanePad = (kHV * 16 + 127) / 128 * 128;  // a TMA destination is 128-byte aligned

template <int CIN, int COUT>
__host__ __device__ constexpr int tma_slots() { return CIN == 16 ? 4 : 3; }

template <int CIN, int COUT>
constexpr int tma_smem_bytes() {  // + 128: the base is rounded up to 128 bytes in the kernel
    return 27 * (CIN / 8) * COUT * 16 + tma_slots<CIN, COUT>() * (CIN / 8) * kPlanePad + 128;
}

// CTAs per SM: two where both fit the SM's 228 KB of shared memory (with the
// 1 KB each CTA reserves and the static part), else one
template <int CIN, int COUT>
constexpr int tma_ctas_per_sm() { return 2 * (tma_smem_bytes<CIN, COUT>() + 2048) <= 228 * 1024 ? 2 : 1; }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(smem_u32(bar))
        : "memory");
}

template <int CIN, int COUT, bool RELU, bool OUT_F32>
__global__ void __launch_bounds__(kWsThreads, 1)
conv3d_tma_kernel(const __grid_constant__ CUtensorMap tmap, ConvArgs a, int ntx, int nty,
                  int ntiles) {
    static_assert(CIN % 16 == 0 && CIN <= 32, "two or four channel chunks");
    static_assert(COUT % 16 == 0 && COUT >= 16 && COUT <= kTcCols, "Cout must be 16, 32 or 64");
    extern __shared__ __align__(1024) uint8_t s_dyn[];
    constexpr int kSlots = tma_slots<CIN, COUT>();
    constexpr int kChunks = CIN / 8;
    constexpr int kWBlock = COUT * 16;
    constexpr int kWBytes = 27 * kChunks * kWBlock;
    constexpr int kSlotBytes = kChunks * kPlanePad;
    constexpr uint32_t kTxBytes = kChunks * kHV * 16;  // one tile's halo
    static_assert(kWBytes % 128 == 0, "halo slots must stay 128-byte aligned");
    uint8_t* const s_w = s_dyn + ((128u - (smem_u32(s_dyn) & 127u)) & 127u);
    uint8_t* const s_halo = s_w + kWBytes;
    __shared__ __align__(8) uint64_t full[kSlots];   // halo of the slot landed
    __shared__ __align__(8) uint64_t empty[kSlots];  // the slot's MMAs are done
    __shared__ __align__(8) uint64_t tfull[2];       // accumulator buffer ready
    __shared__ __align__(8) uint64_t tempty[2];      // accumulator buffer read
    __shared__ uint32_t s_tmem;
    __shared__ float s_bias[COUT];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);  // one arrive per epilogue warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(2 * kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the weights, once: w[n][tap * CIN + cc * 8 ...] -> [tap][cc][n] x 16 bytes
    for (int t = tid; t < COUT * 27 * kChunks; t += kWsThreads) {
        const int n = t / (27 * kChunks), r = t - n * (27 * kChunks);
        __pipeline_memcpy_async(s_w + r * kWBlock + n * 16, a.w + (size_t)n * a.Kp + r * 8, 16);
    }
    for (int n = tid; n < COUT; n += kWsThreads) s_bias[n] = a.bias ? a.bias[n] : 0.0f;
    __pipeline_commit();
    __pipeline_wait_prior(0);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const int nmine = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    auto origin = [&](int i, int& x0, int& y0, int& z0) {
        const int t = (int)blockIdx.x + i * (int)gridDim.x;
        x0 = (t % ntx) * kHTX;
        y0 = ((t / ntx) % nty) * kHTY;
        z0 = t / (ntx * nty);
    };
    bool ok = true;
    if (warp == 0) {
        if (lane == 0) {
            for (int i = 0; i < nmine; ++i) {
                const int s = i % kSlots;
                if (i >= kSlots && !mbar_wait(&empty[s], (uint32_t)((i / kSlots - 1) & 1))) {
                    ok = false;
                    break;
                }
                int x0, y0, z0;
                origin(i, x0, y0, z0);
                mbar_expect_tx(&full[s], kTxBytes);
#pragma unroll
                for (int cc = 0; cc < kChunks; ++cc) {
                    const uint32_t dst = smem_u32(s_halo + s * kSlotBytes + cc * kPlanePad);
                    if (a.in_planar)  // (x * 8 + channel, y, z, plane)
                        tma_load_4d(dst, &tmap, (x0 - 1) * 8, y0 - 1, z0 - 1, cc, &full[s]);
                    else  // (channel, x, y, z)
                        tma_load_4d(dst, &tmap, cc * 8, x0 - 1, y0 - 1, z0 - 1, &full[s]);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = umma_idesc_bf16(kTcRows, COUT);
            const uint32_t wb = smem_u32(s_w);
            const uint64_t db = umma_desc(wb, kWBlock, 128);
            for (int i = 0; i < nmine; ++i) {
                const int s = i % kSlots, b = i & 1;
                if (!mbar_wait(&full[s], (uint32_t)((i / kSlots) & 1)) ||
                    (i >= 2 && !mbar_wait(&tempty[b], (uint32_t)(((i >> 1) - 1) & 1)))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t hb = smem_u32(s_halo + s * kSlotBytes);
                const uint32_t d = tmem + (uint32_t)(b * kTcCols);
                // the halo base descriptor; each MMA adds its compile-time
                // offset (>> 4) to the start-address field, which cannot
                // carry out of its 14 bits (shared addresses < 256 KB)
                const uint64_t da = umma_desc(hb, kPlanePad, kHX * 16);
#pragma unroll
                for (int tap = 0; tap < 27; ++tap) {
                    const uint32_t aoff =
                        (uint32_t)(((tap / 9) * kHY + (tap / 3) % 3) * kHX + tap % 3) * 16;
#pragma unroll
                    for (int kp = 0; kp < kChunks / 2; ++kp)
                        tc_mma(d, da + ((aoff + 2 * kp * kPlanePad) >> 4),
                               db + (((tap * kChunks + 2 * kp) * kWBlock) >> 4), idesc,
                               (tap > 0 || kp > 0) ? 1u : 0u);
                }
                tc_commit(&empty[s]);
                tc_commit(&tfull[b]);
            }
        }
    } else {
        // epilogue: warp w may read TMEM lanes 32 (w % 4) .. + 31
        const int qtr = warp & 3;
        const int m = qtr * 32 + lane;
        for (int i = 0; i < nmine; ++i) {
            const int b = i & 1;
            if (!mbar_wait(&tfull[b], (uint32_t)((i >> 1) & 1))) {
                ok = false;
                break;
            }
            tc_fence_after();
            int x0, y0, z0;
            origin(i, x0, y0, z0);
            const int x = x0 + (m & 7), y = y0 + (m >> 3);
            const bool mv = x < a.nx && y < a.ny;
            const long long q = ((long long)z0 * a.ny + y) * a.nx + x;
            const uint32_t taddr = tmem + (uint32_t)(b * kTcCols) + ((uint32_t)(qtr * 32) << 16);
#pragma unroll
            for (int c0 = 0; c0 < COUT; c0 += 16) {
                float v[16];
                tc_ld16(taddr + c0, v);
                if (mv) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        float r = v[k] + s_bias[c0 + k];
                        if (RELU) r = fmaxf(r, 0.0f);
                        v[k] = r;
                    }
                    if constexpr (OUT_F32) {
                        float4* o =
                            reinterpret_cast<float4*>(static_cast<float*>(a.out) + q * COUT + c0);
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            o[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
                    } else {
                        store16_bf16<COUT>(a, q, c0, v);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
    }
    if (!ok) atomicExch(&g_cnn_status, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(2 * kTcCols)
                     : "memory");
}

// cuTensorMapEncodeTiled from the driver (looked up once)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 1 when launched, 0 when the tensor map could not be made (the caller then
// uses the halo kernel), an sbp_status otherwise
template <int CIN, int COUT, bool RELU, bool OUT_F32>
int launch_tma_t(const ConvArgs& a, cudaStream_t st) {
    const auto encode = tensor_map_encoder();
    if (!encode) return 0;
    CUtensorMap map;
    // channels-last: (channel, x, y, z), a box of 8 channels x 10 x 18 x 3;
    // planar: (x * 8 + channel, y, z, plane), a box of 80 x 18 x 3 x 1, whose
    // rows are ten voxels of one plane (the same bytes in shared memory)
    const cuuint64_t V = (cuuint64_t)a.nx * a.ny * a.nz;
    const cuuint64_t dims_cl[4] = {(cuuint64_t)CIN, (cuuint64_t)a.nx, (cuuint64_t)a.ny,
                                   (cuuint64_t)a.nz};
    const cuuint64_t strides_cl[3] = {(cuuint64_t)CIN * 2, (cuuint64_t)a.nx * CIN * 2,
                                      (cuuint64_t)a.nx * a.ny * CIN * 2};
    const cuuint32_t box_cl[4] = {8, (cuuint32_t)kHX, (cuuint32_t)kHY, (cuuint32_t)kHZ};
    const cuuint64_t dims_pl[4] = {(cuuint64_t)a.nx * 8, (cuuint64_t)a.ny, (cuuint64_t)a.nz,
                                   (cuuint64_t)(CIN / 8)};
    const cuuint64_t strides_pl[3] = {(cuuint64_t)a.nx * 16, (cuuint64_t)a.nx * a.ny * 16, V * 16};
    const cuuint32_t box_pl[4] = {(cuuint32_t)kHX * 8, (cuuint32_t)kHY, (cuuint32_t)kHZ, 1};
    const cuuint64_t* dims = a.in_planar ? dims_pl : dims_cl;
    const cuuint64_t* strides = a.in_planar ? strides_pl : strides_cl;
    const cuuint32_t* box = a.in_planar ? box_pl : box_cl;
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(a.in), dims,
               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return 0;
    constexpr int smem = tma_smem_bytes<CIN, COUT>();
    auto k = conv3d_tma_kernel<CIN, COUT, RELU, OUT_F32>;
    if (sbp_cuda_check(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                       "conv3d_bf16: smem attribute"))
        return SBP_ERR_CUDA;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ntx = (a.nx + kHTX - 1) / kHTX, nty = (a.ny + kHTY - 1) / kHTY;
    const long long ntiles = (long long)ntx * nty * a.nz;
    const int grid = (int)std::min<long long>(
        (long long)std::max(1, sms) * tma_ctas_per_sm<CIN, COUT>(), ntiles);
    k<<<grid, kWsThreads, smem, st>>>(map, a, ntx, nty, (int)ntiles);
    return 1;
}

template <int CIN, int COUT, bool RELU, bool OUT_F32>
int launch_conv_t(const ConvArgs& a, unsigned blocks, cudaStream_t st) {
    constexpr int smem = 2 * (kTcRows + COUT) * kTcBK * 2;
    auto k = conv3d_tc_kernel<CIN, COUT, RELU, OUT_F32>;
    if (sbp_cuda_check(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                       "conv3d_bf16: smem attribute"))
        return SBP_ERR_CUDA;
    k<<<blocks, kTcThreads, smem, st>>>(a);
    return SBP_OK;
}

template <int CIN, int COUT>
int launch_conv(const ConvArgs& a, bool relu, bool out_f32, long long V, cudaStream_t st) {
    // one input channel: the staged-halo kernel, four tiles per CTA
    if constexpr (CIN == 1 && COUT * kC1Tiles <= kTcCols) {
        if ((a.ny + kHTY - 1) / kHTY <= 65535 && (a.nz + kC1Tiles - 1) / kC1Tiles <= 65535) {
            if (relu && out_f32) return launch_c1_t<COUT, true, true>(a, st);
            if (relu) return launch_c1_t<COUT, true, false>(a, st);
            if (out_f32) return launch_c1_t<COUT, false, true>(a, st);
            return launch_c1_t<COUT, false, false>(a, st);
        }
    }
    // the persistent TMA kernel for 16 or 32 input channels, where its three
    // halo slots and the weights fit one CTA's shared memory
    if constexpr (CIN % 16 == 0 && CIN <= 32 && tma_smem_bytes<CIN, COUT>() <= 220 * 1024) {
        if ((long long)((a.nx + kHTX - 1) / kHTX) * ((a.ny + kHTY - 1) / kHTY) * a.nz < (1LL << 31)) {
            int r = 0;
            if (relu && out_f32) r = launch_tma_t<CIN, COUT, true, true>(a, st);
            else if (relu) r = launch_tma_t<CIN, COUT, true, false>(a, st);
            else if (out_f32) r = launch_tma_t<CIN, COUT, false, true>(a, st);
            else r = launch_tma_t<CIN, COUT, false, false>(a, st);
            if (r != 0) return r == 1 ? SBP_OK : r;
        }
    }
    // planar input is read by the TMA kernel only
    if (a.in_planar) {
        sbp_set_error("conv3d: planar input needs the TMA kernel (Cin 16 or 32, a tensor map)");
        return SBP_ERR_ARG;
    }
    // the halo kernel where its staged halo and weights fit one CTA's shared
    // memory and the grid's y and z extents allow it
    if constexpr (CIN % 16 == 0 && halo_smem_bytes<CIN, COUT>() <= 200 * 1024) {
        if ((a.ny + kHTY - 1) / kHTY <= 65535 && a.nz <= 65535) {
            if (relu && out_f32) return launch_halo_t<CIN, COUT, true, true>(a, st);
            if (relu) return launch_halo_t<CIN, COUT, true, false>(a, st);
            if (out_f32) return launch_halo_t<CIN, COUT, false, true>(a, st);
            return launch_halo_t<CIN, COUT, false, false>(a, st);
        }
    }
    const unsigned blocks = (unsigned)((V + kTcRows - 1) / kTcRows);
    if (relu && out_f32) return launch_conv_t<CIN, COUT, true, true>(a, blocks, st);
    if (relu) return launch_conv_t<CIN, COUT, true, false>(a, blocks, st);
    if (out_f32) return launch_conv_t<CIN, COUT, false, true>(a, blocks, st);
    return launch_conv_t<CIN, COUT, false, false>(a, blocks, st);
}

// ---------------------------------------------------------------------------
// Weight gradient of a 3x3x3 convolution on the tensor cores.
//
// GEMM view: D[m][n] = sum_k A[m][k] B[n][k] with m = tap * Cin + c (the
// weight's input side), n = output channel, k = voxel:
//   A[m][v] = x[v + off(tap)][c] (the layer's input, shifted by the tap,
//   zero outside the volume), B[n][v] = g[v][n] (the loss gradient with
//   respect to the layer's output before its ReLU). Row m = 27 Cin
//   of A is all ones over the volume, so D's row 27 Cin is the bias gradient
//   sum_v g[v][n]. The reduction runs over voxels, but both tensors are
//   stored channels-last, so every staged 8 x 8 block (8 voxels x 8
//   channels, one 16-byte load per voxel) is transposed in registers into 8
//   rows of 8 voxels (one byte permute per output word) and stored in the
//   canonical K-major, non-swizzled layout of conv3d_tc_kernel.
// One CTA = one 128-row tile of m x one run of K-steps; a K-step is 64
// voxels of one x-row (x0 .. x0 + 63 at fixed y, z; columns past nx are
// zero). Every CTA writes its FP32 tile to partial[chunk][m][n]; a second
// kernel adds the chunks in chunk order (no atomics: the weight gradient is
// the same bit for bit on every run).
// ---------------------------------------------------------------------------

constexpr int kWgRows = 128;   // rows of m per CTA (the MMA's M)
constexpr int kWgBK = 64;      // voxels per K-step

// out[c] = the 8 channel-c values of the 8 voxels in[0..7] (8 bf16 each)
__device__ __forceinline__ void wg_transpose8(const uint4 (&in)[8], uint4 (&out)[8]) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(in);  // w[4 j + c / 2]
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint32_t sel = (c & 1) ? 0x7632u : 0x5410u;
        uint32_t o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            o[q] = __byte_perm(w[4 * (2 * q) + (c >> 1)], w[4 * (2 * q + 1) + (c >> 1)], sel);
        out[c] = make_uint4(o[0], o[1], o[2], o[3]);
    }
}

// Stores the 8 rows r0 .. r0 + 7 (r0 a multiple of 8) of voxel chunk k8 of
// a K-major tile.
__device__ __forceinline__ void wg_store8(uint8_t* tile, int r0, int k8, const uint4 (&rows)[8]) {
    uint8_t* p = tile + ((r0 >> 3) * 8 + k8) * 128;
#pragma unroll
    for (int c = 0; c < 8; ++c) *reinterpret_cast<uint4*>(p + c * 16) = rows[c];
}

struct WgradArgs {
    const __nv_bfloat16* g;  // [V][Cout], or planar (g_planar)
    const __nv_bfloat16* x;  // [V][Cin], or planar (x_planar)
    int x_planar, g_planar;
    long long V;
    float* partial;          // [chunks][m_pad][Cout]
    int nx, ny, nz;
    int xblocks;             // ceil(nx / 64)
    int steps;               // nz * ny * xblocks
    int steps_per_chunk;
    int m_pad;               // row tiles * 128
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(kTcThreads) wgrad_tc_kernel(WgradArgs a) {
    static_assert(COUT % 16 == 0 && COUT >= 16 && COUT <= kTcCols, "Cout must be 16, 32 or 64");
    static_assert(CIN == 1 || CIN % 8 == 0, "Cin must be 1 or a multiple of 8");
    extern __shared__ __align__(1024) uint8_t s_dyn[];
    constexpr int kABytes = kWgRows * kWgBK * 2, kBBytes = COUT * kWgBK * 2;
    constexpr int kRowsUsed = 27 * CIN + 1;  // weight rows and the bias row
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int mt = blockIdx.x;
    const int s0 = blockIdx.y * a.steps_per_chunk;
    const int s1 = min(a.steps, s0 + a.steps_per_chunk);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    constexpr uint32_t idesc = umma_idesc_bf16(kWgRows, COUT);
    uint32_t phase[2] = {0u, 0u};
    bool ok = true;
    // this thread's 8 x 8 block of each stage: rows r8 * 8 .. + 7, voxels k8 * 8 .. + 7
    const int r8 = tid >> 3, k8 = tid & 7;
    const int nsteps = s1 - s0;

    for (int it = 0; it < nsteps; ++it) {
        const int st = it & 1;
        if (it >= 2) {  // the MMAs that read this stage two steps ago must be done
            if (!mbar_wait(&bar[st], phase[st])) ok = false;
            phase[st] ^= 1u;
        }
        if (!__syncthreads_and(ok)) break;
        const int s = s0 + it;
        const int xb = s % a.xblocks;
        const int y = (s / a.xblocks) % a.ny;
        const int z = s / (a.xblocks * a.ny);
        const int xv = xb * kWgBK + k8 * 8;  // first voxel of this thread's 8
        uint8_t* tileA = s_dyn + st * kABytes;
        uint8_t* tileB = s_dyn + 2 * kABytes + st * kBBytes;
        // A: rows m0 .. m0 + 7 of the layer input shifted by the row's tap
        const int m0 = mt * kWgRows + r8 * 8;
        uint4 blk[8], rows[8];
        if constexpr (CIN % 8 == 0) {
            const int tap = m0 / CIN, c0 = m0 - tap * CIN;
            const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
            const int yy = y + dy, zz = z + dz;
            const bool row_in = m0 < 27 * CIN && yy >= 0 && yy < a.ny && zz >= 0 && zz < a.nz;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int xx = xv + j + dx;
                blk[j] = make_uint4(0u, 0u, 0u, 0u);
                if (row_in && xv + j < a.nx && xx >= 0 && xx < a.nx) {
                    const long long v = ((long long)zz * a.ny + yy) * a.nx + xx;
                    blk[j] = *reinterpret_cast<const uint4*>(
                        a.x + (a.x_planar ? ((long long)(c0 >> 3) * a.V + v) * 8 : v * CIN + c0));
                }
            }
            wg_transpose8(blk, rows);
            if (m0 == 27 * CIN) {  // the bias row: ones over the volume, then zero rows
                uint32_t o[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    o[q] = (xv + 2 * q < a.nx ? 0x3F80u : 0u) |
                           (xv + 2 * q + 1 < a.nx ? 0x3F800000u : 0u);
                rows[0] = make_uint4(o[0], o[1], o[2], o[3]);
            }
        } else {  // one input channel: row m is tap m, read voxel by voxel
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int m = m0 + i;
                uint32_t o[4] = {0u, 0u, 0u, 0u};
                if (m < 27) {
                    const int dx = m % 3 - 1, dy = (m / 3) % 3 - 1, dz = m / 9 - 1;
                    const int yy = y + dy, zz = z + dz;
                    if (yy >= 0 && yy < a.ny && zz >= 0 && zz < a.nz) {
                        const unsigned short* rowp = reinterpret_cast<const unsigned short*>(a.x) +
                                                     ((long long)zz * a.ny + yy) * a.nx;
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int xx = xv + j + dx;
                            const uint32_t h = (xv + j < a.nx && xx >= 0 && xx < a.nx) ? rowp[xx] : 0u;
                            o[j >> 1] |= h << (16 * (j & 1));
                        }
                    }
                } else if (m == 27) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        o[q] = (xv + 2 * q < a.nx ? 0x3F80u : 0u) |
                               (xv + 2 * q + 1 < a.nx ? 0x3F800000u : 0u);
                }
                rows[i] = make_uint4(o[0], o[1], o[2], o[3]);
            }
        }
        wg_store8(tileA, r8 * 8, k8, rows);
        // B: the output gradient, rows = output channels
        if (r8 < COUT / 8) {
            const long long vrow = ((long long)z * a.ny + y) * a.nx;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                blk[j] = make_uint4(0u, 0u, 0u, 0u);
                if (xv + j < a.nx) {
                    const long long v = vrow + xv + j;
                    blk[j] = *reinterpret_cast<const uint4*>(
                        a.g + (a.g_planar ? ((long long)r8 * a.V + v) * 8 : v * COUT + r8 * 8));
                }
            }
            wg_transpose8(blk, rows);
            wg_store8(tileB, r8 * 8, k8, rows);
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(tileA), b0 = smem_u32(tileB);
#pragma unroll
            for (int ks = 0; ks < kWgBK / 16; ++ks)  // K = 16 per MMA: two core matrices
                tc_mma(tmem, umma_desc(a0 + ks * 256, 128, 1024), umma_desc(b0 + ks * 256, 128, 1024),
                       idesc, (it > 0 || ks > 0) ? 1u : 0u);
            tc_commit(&bar[st]);
        }
    }

    // wait for the last commit of each stage still outstanding
    if (ok) {
        for (int s = 0; s < 2; ++s) {
            const int uses = nsteps > s ? (nsteps - 1 - s) / 2 + 1 : 0;  // commits made on stage s
            const int waited = uses > 0 ? uses - 1 : 0;                 // of them already waited on
            if (uses > waited && !mbar_wait(&bar[s], phase[s])) ok = false;
        }
    }
    tc_fence_after();
    const int row = mt * kWgRows + warp * 32 + (tid & 31);
    float* out = a.partial + ((size_t)blockIdx.y * a.m_pad + row) * COUT;
    if (!__syncthreads_and(ok)) {
        if (tid == 0) atomicExch(&g_cnn_status, 1);
    } else if (nsteps > 0) {
        // lane = row m, columns = output channels (every lane takes part in
        // the warp-wide tcgen05.ld)
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int c0 = 0; c0 < COUT; c0 += 16) {
            float v[16];
            tc_ld16(taddr + c0, v);
            if (row < kRowsUsed) {
                float4* o = reinterpret_cast<float4*>(out + c0);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            }
        }
    } else if (row < kRowsUsed) {
        for (int c = 0; c < COUT; ++c) out[c] = 0.0f;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTcCols)
                     : "memory");
}

// dW[n][tap][c] = sum over chunks (in chunk order) of row tap * Cin + c,
// db[n] = the same for the bias row 27 Cin.
template <int CIN, int COUT>
__global__ void wgrad_reduce_kernel(const float* __restrict__ partial, int chunks, int m_pad,
                                    float* __restrict__ dW, float* __restrict__ db) {
    constexpr int kOut = (27 * CIN + 1) * COUT;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < kOut; t += gridDim.x * blockDim.x) {
        const int m = t / COUT, n = t - m * COUT;
        float s = 0.0f;
        for (int k = 0; k < chunks; ++k) s += partial[((size_t)k * m_pad + m) * COUT + n];
        if (m < 27 * CIN) {
            const int tap = m / CIN, c = m - tap * CIN;
            dW[((size_t)n * 27 + tap) * CIN + c] = s;
        } else {
            db[n] = s;
        }
    }
}

// Chunks of K-steps for a layer: enough CTAs to fill the GPU about four
// times over, every chunk non-empty.
void wgrad_plan(int nx, int ny, int nz, int cin, int sms, int& xblocks, int& steps,
                int& steps_per, int& chunks, int& m_pad) {
    xblocks = (nx + kWgBK - 1) / kWgBK;
    steps = nz * ny * xblocks;
    const int tiles = (27 * cin + 1 + kWgRows - 1) / kWgRows;
    m_pad = tiles * kWgRows;
    const int want = std::max(1, (4 * sms + tiles - 1) / tiles);
    steps_per = std::max(1, (steps + want - 1) / want);
    chunks = (steps + steps_per - 1) / steps_per;
}

template <int CIN, int COUT>
int launch_wgrad_t(const WgradArgs& a, int chunks, float* dW, float* db, cudaStream_t st) {
    constexpr int smem = 2 * (kWgRows + COUT) * kWgBK * 2;
    auto k = wgrad_tc_kernel<CIN, COUT>;
    if (sbp_cuda_check(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                       "cnn wgrad: smem attribute"))
        return SBP_ERR_CUDA;
    const dim3 grid((unsigned)(a.m_pad / kWgRows), (unsigned)chunks);
    k<<<grid, kTcThreads, smem, st>>>(a);
    constexpr int kOut = (27 * CIN + 1) * COUT;
    wgrad_reduce_kernel<CIN, COUT><<<(kOut + 255) / 256, 256, 0, st>>>(a.partial, chunks, a.m_pad,
                                                                       dW, db);
    sbp_count_launches(2);
    return sbp_cuda_check(cudaGetLastError(), "cnn wgrad launch") ? SBP_ERR_CUDA : SBP_OK;
}

}  // namespace

// Weight and bias gradients of a 3x3x3 convolution (Cin, Cout) in (1, 16),
// (16, 32), (32, 64): see wgrad_tc_kernel. `partial` holds
// sbp_wgrad_scratch_floats(...) floats.
long long sbp_wgrad_scratch_floats(int nx, int ny, int nz, int cin, int cout, int sms) {
    int xb, steps, per, chunks, m_pad;
    wgrad_plan(nx, ny, nz, cin, sms, xb, steps, per, chunks, m_pad);
    return (long long)chunks * m_pad * cout;
}

int sbp_wgrad_bf16(const void* g_dev, const void* x_dev, int nx, int ny, int nz, int cin,
                   int cout, int sms, float* partial, float* dW, float* db, bool x_planar,
                   bool g_planar, cudaStream_t st) {
    WgradArgs a;
    int chunks;
    wgrad_plan(nx, ny, nz, cin, sms, a.xblocks, a.steps, a.steps_per_chunk, chunks, a.m_pad);
    a.g = static_cast<const __nv_bfloat16*>(g_dev);
    a.x = static_cast<const __nv_bfloat16*>(x_dev);
    a.x_planar = (x_planar && cin % 8 == 0) ? 1 : 0;
    a.g_planar = g_planar ? 1 : 0;
    a.V = (long long)nx * ny * nz;
    a.partial = partial;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    if (cin == 1 && cout == 16) return launch_wgrad_t<1, 16>(a, chunks, dW, db, st);
    if (cin == 16 && cout == 32) return launch_wgrad_t<16, 32>(a, chunks, dW, db, st);
    if (cin == 32 && cout == 64) return launch_wgrad_t<32, 64>(a, chunks, dW, db, st);
    sbp_set_error("cnn wgrad: unsupported (cin, cout)");
    return SBP_ERR_ARG;
}

namespace {

}  // namespace

int sbp_conv3d_layout(const void* in_dev, int nx, int ny, int nz, int cin, const void* w_dev,
                      int kp, const float* bias_dev, int cout, int relu, void* out_dev,
                      int out_f32, bool in_planar, bool out_planar, cudaStream_t st) {
    const long long V = (long long)nx * ny * nz;
    if (!in_dev || !w_dev || !out_dev || nx < 1 || ny < 1 || nz < 1 || kp < 27 * cin ||
        kp % kTcBK != 0 || V > (1LL << 31) * kTcRows) {
        sbp_set_error("conv3d_bf16: invalid argument");
        return SBP_ERR_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(in_dev) | reinterpret_cast<uintptr_t>(w_dev) |
         reinterpret_cast<uintptr_t>(out_dev)) & 15u) {
        sbp_set_error("conv3d_bf16: arrays must be 16-byte aligned");
        return SBP_ERR_ARG;
    }
    if ((in_planar && cin % 8 != 0) || (out_planar && (out_f32 || cout % 16 != 0))) {
        sbp_set_error("conv3d: planar layouts need Cin a multiple of 8, Cout of 16, bf16 output");
        return SBP_ERR_ARG;
    }
    ConvArgs a{static_cast<const __nv_bfloat16*>(in_dev),
               static_cast<const __nv_bfloat16*>(w_dev),
               bias_dev,
               out_dev,
               nx,
               ny,
               nz,
               kp,
               in_planar ? 1 : 0,
               out_planar ? 1 : 0,
               V};
    int rc = SBP_ERR_ARG + 100;  // "no case matched" until a case launches
#define SBP_CONV_CASE(CI, CO) \
    if (cin == CI && cout == CO) rc = launch_conv<CI, CO>(a, relu != 0, out_f32 != 0, V, st);
    SBP_CONV_CASE(1, 16)
    SBP_CONV_CASE(16, 16)
    SBP_CONV_CASE(16, 32)
    SBP_CONV_CASE(32, 32)
    SBP_CONV_CASE(32, 64)
    SBP_CONV_CASE(64, 64)
    SBP_CONV_CASE(64, 32)
    SBP_CONV_CASE(32, 16)
#undef SBP_CONV_CASE
    if (rc == SBP_ERR_ARG + 100) {
        sbp_set_error("conv3d_bf16: unsupported (cin, cout); supported: (1,16) (16,16) (16,32) "
                      "(32,32) (32,64) (64,64) (64,32) (32,16)");
        return SBP_ERR_ARG;
    }
    if (rc != SBP_OK) return rc;
    sbp_count_launches(1);
    return sbp_cuda_check(cudaGetLastError(), "conv3d_bf16 launch") ? SBP_ERR_CUDA : SBP_OK;
}

extern "C" {

int sbp_conv3d_bf16(const void* in_dev, int nx, int ny, int nz, int cin, const void* w_dev,
                    int kp, const float* bias_dev, int cout, int relu, void* out_dev, int out_f32,
                    sbp_stream stream) {
    return sbp_conv3d_layout(in_dev, nx, ny, nz, cin, w_dev, kp, bias_dev, cout, relu, out_dev,
                             out_f32, false, false, reinterpret_cast<cudaStream_t>(stream));
}

int sbp_cnn_status(sbp_stream stream, int* status) {
    if (!status) {
        sbp_set_error("cnn_status: null pointer");
        return SBP_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (sbp_cuda_check(cudaStreamSynchronize(st), "cnn_status: synchronise")) return SBP_ERR_CUDA;
    int v = 0, zero = 0;
    if (sbp_cuda_check(cudaMemcpyFromSymbol(&v, g_cnn_status, sizeof(int)), "cnn_status: read") ||
        sbp_cuda_check(cudaMemcpyToSymbol(g_cnn_status, &zero, sizeof(int)), "cnn_status: clear"))
        return SBP_ERR_CUDA;
    *status = v ? SBP_ERR_TIMEOUT : 0;
    return SBP_OK;
}

}  // extern "C"
