// Gaussian-profile radiator (the variant of Section 4.1 in which a ball is a
// Gaussian spherical source of peak p0 and standard deviation a, stored in
// the R row of the cloud).
//
// The outgoing spherical wave of the initial pressure p0 exp(-r^2 / 2a^2),
// seen at distance d (far field, d > 6a; nearer pairs are skipped and
// counted), is p(t) = p0 w (d - ct) exp(-(d - ct)^2 / 2a^2) / (2d), and its
// average over cell j of level k is
//     S_j = D_{j+1} - D_j,   D_j = p0 K g(b_j),   K = w a^2 / (2 d h),
// with boundary offsets b_j = d - j h (h = c dt_k) and g(b) = exp(-b^2 / 2a^2).
// A pair therefore contributes one value per cell boundary; boundaries with
// |b| >= 6a are left out (their values are below 1.5e-8 of the peak).
//
// Kernels:
//   gfwd_group     CTA = (32 sensors) x (chunk of 512 balls), warp = ball,
//                  lane = sensor, as the uniform-sphere forward: the
//                  boundary values are rounded to fixed point (2^-F, F from
//                  max |p0|) and added to the lane's window in shared memory
//                  as two 32-bit words, then flushed to int64 accumulators
//                  [M][T_k + 1] with global atomics; the traces are
//                  bitwise independent of accumulation order.
//   gfwd_finalize  S_j = (D_{j+1} - D_j) 2^-F, exact integer difference; clears D.
//   gadj           one thread per ball over all sensors: by summation by
//                  parts sum_j G_j S_j = p0 K sum_j c_j g(b_j) with
//                  c_j = G_{j-1} - G_j (G = 0 outside the record), and
//                      A0 = sum c_j g,  A1 = sum c_j g b,  A2 = sum c_j g b^2,
//                      dL/dp0 = K A0,
//                      dL/dd  = p0 K (-A0 / d - A1 / a^2),
//                      dL/da  = p0 K (2 A0 / a + A2 / a^3),
//                      dL/dw  = p0 a^2 A0 / (2 d h).
#include <algorithm>

#include "sbp_internal.cuh"

namespace {

constexpr float kSupport = 6.0f;  // |b| < 6a
constexpr int kGWarps = 16;
constexpr int kGWindow = 384;     // boundaries per lane held in shared memory
constexpr int kGChunk = 512;
constexpr int kGLoBits = 20;
static_assert(kGChunk * (1LL << kGLoBits) < (1LL << 32), "low word could overflow");

__device__ __forceinline__ long long g_f2ll(float x) {
    const float ax = fabsf(x);
    if (ax < 2147483520.0f) return (long long)__float2int_rn(x);
    const float hi = floorf(ax * 2.3283064365386963e-10f);
    const float rem = fmaf(-hi, 4294967296.0f, ax);
    const long long v = ((long long)__float2uint_rz(hi) << 32) + (long long)__float2uint_rn(rem);
    return x < 0.0f ? -v : v;
}

__device__ __forceinline__ int g_frac_bits(unsigned int bits) {
    const float pm = __uint_as_float(bits);
    int e = 0;
    if (pm > 0.0f) frexpf(pm, &e);
    const int F = 34 - e;
    return F < 0 ? 0 : (F > 60 ? 60 : F);
}

// Calls f(k, g(b_k), b_k) for k = klo .. khi, b_k = e - k h, g(b) = 2^(b^2 nc),
// by the ratio recurrence g_{k+1} = g_k r_k, r_{k+1} = r_k q with
// r_k = 2^((h^2 - 2 b_k h) nc) and q = 2^(2 h^2 nc), restarted from exp2f
// every 8 boundaries: two exp2f per 8 values instead of eight. Against the
// exact Gaussian, in float32 over a in [0.05, 0.4] mm and h from 0.019 to
// 0.15 mm, values above 1e-4 of the peak are off by 5e-7 rms and 9e-6 at
// worst (exp2f of the rounded argument alone: 2.5e-6 at worst).
template <typename F>
__device__ __forceinline__ void g_gauss_run(int klo, int khi, float e, float h, float nc, F&& f) {
    const float h2 = h * h;
    const float q = exp2f(2.0f * h2 * nc);
    for (int k0 = klo; k0 <= khi; k0 += 8) {
        const float b0 = fmaf(-(float)k0, h, e);
        float gk = exp2f(b0 * b0 * nc);
        float rk = exp2f(fmaf(-2.0f * h, b0, h2) * nc);
        const int kend = min(k0 + 7, khi);
        for (int k = k0; k <= kend; ++k) {
            f(k, gk, fmaf(-(float)k, h, e));
            gk *= rk;
            rk *= q;
        }
    }
}

__global__ void gpmax_kernel(const float* __restrict__ p0, const int* n_dev, int n_cap,
                             unsigned int* bits) {
    const int n = sbp_read_n(n_dev, n_cap);
    float m = 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(p0[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(bits, __float_as_uint(m));
}

// Boundary window [jlo, jhi] (clipped to 0 .. Tk) that any ball of the box
// can reach at this sensor, with a support radius of 6 x the box's largest a.
__device__ __forceinline__ void g_box_bounds(float sx, float sy, float sz, const float* box,
                                             float inv_h, int Tk, int& jlo, int& jhi) {
    const float ex = fmaxf(fmaxf(box[0] - sx, sx - box[3]), 0.0f);
    const float ey = fmaxf(fmaxf(box[1] - sy, sy - box[4]), 0.0f);
    const float ez = fmaxf(fmaxf(box[2] - sz, sz - box[5]), 0.0f);
    const float fx = fmaxf(fabsf(sx - box[0]), fabsf(sx - box[3]));
    const float fy = fmaxf(fabsf(sy - box[1]), fabsf(sy - box[4]));
    const float fz = fmaxf(fabsf(sz - box[2]), fabsf(sz - box[5]));
    const float dmin = sqrtf(ex * ex + ey * ey + ez * ez);
    const float dmax = sqrtf(fx * fx + fy * fy + fz * fz);
    const float Rs = kSupport * fmaxf(box[6], 0.0f);
    float lo = floorf((dmin - Rs) * inv_h) - 2.0f;
    float hi = ceilf((dmax + Rs) * inv_h) + 2.0f;
    lo = fminf(fmaxf(lo, 0.0f), (float)Tk + 1.0f);
    hi = fminf(fmaxf(hi, -1.0f), (float)Tk);
    jlo = (int)lo;
    jhi = (int)hi;
}

__global__ void __launch_bounds__(kGWarps * 32, 2)
gfwd_group_kernel(BallsDev b, const int* n_dev, int n_cap, const float* __restrict__ sens,
                  LevelGeo g, const unsigned int* __restrict__ pmax, SbpDevState* st,
                  unsigned long long* __restrict__ acc) {
    extern __shared__ unsigned int gacc[];  // [2][kGWindow][32]
    __shared__ float s_red[kGWarps * 7];
    __shared__ float s_box[7];
    __shared__ int s_jlo[32];
    const int n = sbp_read_n(n_dev, n_cap);
    const int c0 = blockIdx.x * kGChunk;
    if (c0 >= n) return;
    const int c1 = min(n, c0 + kGChunk);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Tk = g.Tk, M = g.M, W = Tk + 1;  // boundaries 0 .. Tk
    const int m = blockIdx.y * 32 + lane;
    const bool sv = m < M;
    sbp_chunk_box(b, c0, c1, s_red, s_box);
    float sx = 0.f, sy = 0.f, sz = 0.f, nx = 0.f, ny = 0.f, nz = 0.f;
    int jlo = 0, jhi = -1;
    if (sv) {
        sx = sens[m];
        sy = sens[M + m];
        sz = sens[2 * M + m];
        nx = sens[3 * M + m];
        ny = sens[4 * M + m];
        nz = sens[5 * M + m];
        g_box_bounds(sx, sy, sz, s_box, g.inv_h, Tk, jlo, jhi);
    }
    int wmax = max(0, jhi - jlo + 1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    const int passes = (wmax + kGWindow - 1) / kGWindow;
    if (warp == 0) s_jlo[lane] = jlo;
    const int used0 = min(wmax, kGWindow) * 32;
    for (int t = threadIdx.x; t < used0; t += blockDim.x) {
        gacc[t] = 0u;
        gacc[kGWindow * 32 + t] = 0u;
    }
    __syncthreads();
    const float scale = __int_as_float((127 + g_frac_bits(*pmax)) << 23);
    const float h = g.h_hi;
    unsigned int inside = 0;
    for (int p = 0; p < passes; ++p) {
        const int base = jlo + p * kGWindow;
        const int lim = min(jhi - base, kGWindow - 1);
        unsigned int* col = gacc + lane;
        for (int i = c0 + warp; i < c1; i += kGWarps) {
            const float a = b.R[i], p0 = b.p0[i];
            if (p0 == 0.0f || !(a > 0.0f) || !sv) continue;
            const PairDist pd = sbp_pair_distance(b.x[i], b.y[i], b.z[i], sx, sy, sz);
            if (!(pd.dh + pd.dl > kSupport * a)) {
                if (p == 0) ++inside;
                continue;
            }
            const float cosv = (nx * pd.dx + ny * pd.dy + nz * pd.dz) * pd.rd;
            float act;
            const float w = sbp_weight(g.wmode, cosv, act);
            if (w == 0.0f) continue;
            // reference boundary jr = floor(d / h), its offset e = b_jr exactly
            const float xr = pd.dh * g.inv_h;
            if (!(xr < (float)Tk + 4096.0f)) continue;
            const int jr = (int)floorf(xr);
            const float e = sbp_boundary(pd.dh, pd.dl, jr, g.h_hi, g.h_lo);
            const float span = kSupport * a;
            const int k0 = (int)ceilf((e - span) * g.inv_h);  // b_j = e - (j - jr) h < 6a
            const int k1 = (int)floorf((e + span) * g.inv_h);
            const float Ks = p0 * w * (a * a) * 0.5f * pd.rd * g.inv_h * scale;  // K p0 2^F
            const float nc = -0.72134752044448170f / (a * a);  // g(b) = 2^(b^2 nc)
            // boundaries j = jr + k inside this pass's cells [base, base + lim]
            // (which lie inside the record 0 .. Tk)
            const int klo = max(k0, base - jr), khi = min(k1, base + lim - jr);
            unsigned int* cb = col + (jr - base) * 32;
            // g at consecutive boundaries by the ratio recurrence (g_gauss_run);
            // every value is at most Ks, so below 2^30 a 32-bit conversion and
            // 32-bit words do (their arithmetic shift gives the 64-bit one's
            // high word)
            const bool small = fabsf(Ks) < 1073741824.0f;
            g_gauss_run(klo, khi, e, h, nc, [&](int k, float gk, float) {
                if (small) {
                    const int v = __float2int_rn(Ks * gk);
                    atomicAdd(cb + k * 32, (unsigned int)v);
                    atomicAdd(cb + k * 32 + kGWindow * 32, (unsigned int)(v >> kGLoBits));
                } else {
                    const long long v = g_f2ll(Ks * gk);
                    atomicAdd(cb + k * 32, (unsigned int)v);
                    atomicAdd(cb + k * 32 + kGWindow * 32, (unsigned int)(int)(v >> kGLoBits));
                }
            });
        }
        __syncthreads();
        const int used = min(wmax - p * kGWindow, kGWindow) * 32;
        for (int t = threadIdx.x; t < used; t += blockDim.x) {
            const unsigned int wa = gacc[t];
            const int hi = (int)gacc[kGWindow * 32 + t];
            if (wa | (unsigned)hi) {
                const unsigned int lo = wa - ((unsigned int)hi << kGLoBits);
                const long long v = (long long)hi * (1LL << kGLoBits) + (long long)lo;
                const int ln = t & 31, rel = t >> 5;
                const int j = s_jlo[ln] + p * kGWindow + rel;
                atomicAdd(acc + (size_t)(blockIdx.y * 32 + ln) * W + j, (unsigned long long)v);
                gacc[t] = 0u;
                gacc[kGWindow * 32 + t] = 0u;
            }
        }
        __syncthreads();
    }
    if (inside) atomicAdd(&st->inside_pairs, (unsigned long long)inside);
}

// one CTA per sensor row: S_j = (D_{j+1} - D_j) 2^-F; clears D
__global__ void gfwd_finalize_kernel(unsigned long long* __restrict__ acc, int Tk,
                                     const unsigned int* __restrict__ pmax, float* __restrict__ S) {
    const int m = blockIdx.x;
    unsigned long long* row = acc + (size_t)m * (Tk + 1);
    const float inv = __int_as_float((127 - g_frac_bits(*pmax)) << 23);
    for (int j = threadIdx.x; j < Tk; j += blockDim.x) {
        const long long x = (long long)row[j + 1] - (long long)row[j];
        S[(size_t)m * Tk + j] = fmaf((float)(int)(x >> 32), 4294967296.0f, (float)(unsigned)x) * inv;
    }
    __syncthreads();
    for (int j = threadIdx.x; j <= Tk; j += blockDim.x) row[j] = 0ull;
}

constexpr int kGAdjThreads = 128;
constexpr int kGSensTile = 128;

// grid.y CTAs share a chunk of kGAdjThreads balls, each taking 1/grid.y of
// the sensors; their partial sums go to scratch [chunk][part][5][ball] and
// the last of them to arrive (a ticket per chunk) adds the parts in rank
// order and writes the gradients, so the result does not depend on timing.
__global__ void __launch_bounds__(kGAdjThreads)
gadj_kernel(BallsDev b, const int* n_dev, int n_cap, const float* __restrict__ sens, LevelGeo g,
            const float* __restrict__ G, unsigned mask, float* gx_, float* gy_, float* gz_,
            float* ga_, float* gp_, float* __restrict__ part_all,
            unsigned int* __restrict__ tickets) {
    static_assert(kGAdjThreads == SBP_ADJ_CHUNK, "the partial-sum scratch holds 128-ball chunks");
    __shared__ float s[kGSensTile * 6];
    __shared__ bool s_last;
    const int n = sbp_read_n(n_dev, n_cap);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x * blockDim.x >= n) return;  // uniform over the chunk's CTAs
    const bool live = i < n;
    const float cx = live ? b.x[i] : 0.f, cy = live ? b.y[i] : 0.f, cz = live ? b.z[i] : 0.f;
    const float a0 = live ? b.R[i] : 1.f, p0 = live ? b.p0[i] : 0.f;
    const bool valid = live && a0 > 0.0f;  // a ball without width radiates nothing
    const float a = valid ? a0 : 1.f;
    const int Tk = g.Tk, M = g.M;
    const float h = g.h_hi, ia2 = 1.0f / (a * a);
    const float nc = -0.72134752044448170f * ia2;  // g(b) = exp(-b^2 / 2a^2) = 2^(b^2 nc)
    float ax = 0.f, ay = 0.f, az = 0.f, aa = 0.f, ap = 0.f;
    const int split = (int)gridDim.y, part = (int)blockIdx.y;
    const int per = (M + split - 1) / split;
    const int m_begin = min(M, part * per), m_end = min(M, m_begin + per);
    for (int m0 = m_begin; m0 < m_end; m0 += kGSensTile) {
        const int cnt = min(kGSensTile, m_end - m0);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt * 6; t += blockDim.x) {
            const int k = t / cnt, j = t % cnt;
            s[j * 6 + k] = sens[(size_t)k * M + m0 + j];
        }
        __syncthreads();
        if (!valid) continue;
        for (int q = 0; q < cnt; ++q) {
            const float* S6 = s + q * 6;
            const PairDist pd = sbp_pair_distance(cx, cy, cz, S6[0], S6[1], S6[2]);
            if (!(pd.dh + pd.dl > kSupport * a)) continue;
            const float ux = pd.dx * pd.rd, uy = pd.dy * pd.rd, uz = pd.dz * pd.rd;
            const float cosv = S6[3] * ux + S6[4] * uy + S6[5] * uz;
            float act;
            const float w = sbp_weight(g.wmode, cosv, act);
            if (w == 0.0f && act == 0.0f) continue;
            const float xr = pd.dh * g.inv_h;
            if (!(xr < (float)Tk + 4096.0f)) continue;
            const int jr = (int)floorf(xr);
            const float e = sbp_boundary(pd.dh, pd.dl, jr, g.h_hi, g.h_lo);
            const float span = kSupport * a;
            const int k0 = (int)ceilf((e - span) * g.inv_h);
            const int k1 = (int)floorf((e + span) * g.inv_h);
            const float* Gm = G + (size_t)(m0 + q) * Tk;
            float A0 = 0.f, A1 = 0.f, A2 = 0.f;
            // boundaries j = jr + k in 0 .. Tk; c_j = G[j-1] - G[j] with G = 0
            // outside the record, G[j-1] carried from the step before
            const int klo = max(k0, -jr), khi = min(k1, Tk - jr);
            int j = jr + klo;
            float gprev = j >= 1 ? Gm[j - 1] : 0.0f;
            // (one exp2f per boundary here: the ratio recurrence of the
            // forward made this loop, which waits on its loads of G, slower)
            for (int k = klo; k <= khi; ++k, ++j) {
                const float gcur = j < Tk ? Gm[j] : 0.0f;
                const float cj = gprev - gcur;
                gprev = gcur;
                const float bj = fmaf(-(float)k, h, e);
                const float gv = exp2f(bj * bj * nc) * cj;
                A0 += gv;
                A1 = fmaf(gv, bj, A1);
                A2 = fmaf(gv * bj, bj, A2);
            }
            const float K = w * a * a * 0.5f * pd.rd * g.inv_h;
            ap = fmaf(K, A0, ap);
            aa += p0 * K * (2.0f * A0 / a + A2 * ia2 / a);
            const float gd = p0 * K * (-A0 * pd.rd - A1 * ia2);
            const float gw = p0 * a * a * A0 * 0.5f * pd.rd * g.inv_h * act;
            ax += gd * ux + gw * (S6[3] - cosv * ux) * pd.rd;
            ay += gd * uy + gw * (S6[4] - cosv * uy) * pd.rd;
            az += gd * uz + gw * (S6[5] - cosv * uz) * pd.rd;
        }
    }
    const size_t chunk = blockIdx.x;
    const int t = threadIdx.x;
    float* __restrict__ mine = part_all + (chunk * split + part) * 5 * kGAdjThreads;
    mine[0 * kGAdjThreads + t] = ax;
    mine[1 * kGAdjThreads + t] = ay;
    mine[2 * kGAdjThreads + t] = az;
    mine[3 * kGAdjThreads + t] = aa;
    mine[4 * kGAdjThreads + t] = ap;
    __threadfence();
    __syncthreads();
    if (t == 0) s_last = atomicAdd(&tickets[chunk], 1u) == (unsigned int)(split - 1);
    __syncthreads();
    if (!s_last) return;  // uniform over the block
    __threadfence();
    if (live) {
        const float* __restrict__ all = part_all + chunk * split * 5 * kGAdjThreads + t;
        float a[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        for (int r = 0; r < split; ++r)
#pragma unroll
            for (int c = 0; c < 5; ++c) a[c] += __ldcg(all + ((size_t)r * 5 + c) * kGAdjThreads);
        const bool xyz = mask & SBP_MASK_XYZ;
        gx_[i] = xyz ? a[0] : 0.0f;
        gy_[i] = xyz ? a[1] : 0.0f;
        gz_[i] = xyz ? a[2] : 0.0f;
        ga_[i] = (mask & SBP_MASK_R) ? a[3] : 0.0f;
        gp_[i] = (mask & SBP_MASK_P0) ? a[4] : 0.0f;
    }
    if (t == 0) tickets[chunk] = 0u;  // ready for the next launch
}

}  // namespace

extern "C" {

int sbp_forward_gauss(sbp_array arr, sbp_balls balls, const int* n_dev, int n_cap, float* S_dev,
                      sbp_stream stream) {
    if (!arr || !balls.x || !balls.y || !balls.z || !balls.R || !balls.p0 || !S_dev || n_cap < 0 ||
        n_cap > arr->n_cap) {
        sbp_set_error("forward_gauss: invalid argument");
        return SBP_ERR_ARG;
    }
    const LevelGeo g = sbp_level_geo(arr, arr->level);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t cells = (size_t)g.M * (g.Tk + 1);
    if (arr->gauss_cells < cells) {
        if (sbp_cuda_check(cudaStreamSynchronize(st), "forward_gauss: synchronise")) return SBP_ERR_CUDA;
        cudaFree(arr->d_gacc);
        arr->d_gacc = nullptr;
        arr->gauss_cells = 0;
        if (sbp_cuda_check(cudaMalloc(&arr->d_gacc, sizeof(unsigned long long) * cells),
                           "forward_gauss: alloc") ||
            sbp_cuda_check(cudaMemset(arr->d_gacc, 0, sizeof(unsigned long long) * cells),
                           "forward_gauss: clear"))
            return SBP_ERR_CUDA;
        arr->gauss_cells = cells;
    }
    if (n_cap == 0) {
        return sbp_cuda_check(cudaMemsetAsync(S_dev, 0, sizeof(float) * (size_t)g.M * g.Tk, st),
                              "forward_gauss: clear S")
                   ? SBP_ERR_CUDA
                   : SBP_OK;
    }
    const size_t smem = (size_t)2 * kGWindow * 32 * sizeof(unsigned int);
    if (sbp_cuda_check(cudaFuncSetAttribute(gfwd_group_kernel,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                       "forward_gauss: smem attribute") ||
        sbp_cuda_check(cudaMemsetAsync(&arr->d_state->pmax_bits, 0, sizeof(unsigned int), st),
                       "forward_gauss: reset"))
        return SBP_ERR_CUDA;
    const BallsDev bd{balls.x, balls.y, balls.z, balls.R, balls.p0};
    gpmax_kernel<<<std::max(1, std::min(4 * arr->sm_count, (n_cap + 255) / 256)), 256, 0, st>>>(
        balls.p0, n_dev, n_cap, &arr->d_state->pmax_bits);
    dim3 grid((n_cap + kGChunk - 1) / kGChunk, (g.M + 31) / 32);
    gfwd_group_kernel<<<grid, kGWarps * 32, smem, st>>>(bd, n_dev, n_cap, arr->d_sens, g,
                                                       &arr->d_state->pmax_bits, arr->d_state,
                                                       arr->d_gacc);
    gfwd_finalize_kernel<<<g.M, 512, 0, st>>>(arr->d_gacc, g.Tk, &arr->d_state->pmax_bits, S_dev);
    sbp_count_launches(3);
    return sbp_cuda_check(cudaGetLastError(), "forward_gauss launch") ? SBP_ERR_CUDA : SBP_OK;
}

int sbp_adjoint_gauss(sbp_array arr, sbp_balls balls, const int* n_dev, int n_cap,
                      const float* G_dev, sbp_grads out, unsigned grad_mask, sbp_stream stream) {
    if (!arr || !balls.x || !balls.y || !balls.z || !balls.R || !balls.p0 || !G_dev || !out.gx ||
        !out.gy || !out.gz || !out.gR || !out.gp0 || n_cap < 0 || n_cap > arr->n_cap ||
        (grad_mask & ~SBP_MASK_ALL)) {
        sbp_set_error("adjoint_gauss: invalid argument");
        return SBP_ERR_ARG;
    }
    if (n_cap == 0) return SBP_OK;
    const LevelGeo g = sbp_level_geo(arr, arr->level);
    const BallsDev bd{balls.x, balls.y, balls.z, balls.R, balls.p0};
    // enough CTAs per chunk (each over a share of at least kGSensTile
    // sensors) for about four waves of resident CTAs (~8 per SM): one CTA
    // per chunk left the last wave mostly empty
    const int chunks = (n_cap + kGAdjThreads - 1) / kGAdjThreads;
    int split = 1;
    while (split < SBP_ADJ_MAX_SPLIT && (long long)chunks * split < 32LL * arr->sm_count &&
           2 * split * kGSensTile <= g.M)
        split *= 2;
    gadj_kernel<<<dim3(chunks, split), kGAdjThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        bd, n_dev, n_cap, arr->d_sens, g, G_dev, grad_mask, out.gx, out.gy, out.gz, out.gR,
        out.gp0, arr->d_adj_part, arr->d_adj_ticket);
    sbp_count_launches(1);
    return sbp_cuda_check(cudaGetLastError(), "adjoint_gauss launch") ? SBP_ERR_CUDA : SBP_OK;
}

}  // extern "C"
