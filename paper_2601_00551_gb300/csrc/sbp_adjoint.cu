// Level downsampling, residual of the per-level loss, and the adjoint of the
// forward radiator (the backpropagation step of Algorithm 1).
//
// Adjoint. With the per-pair cell values of the forward (first cell a, ramp
// D1 + n D2 on cells jL..jH-1, last cell e; see sbp_forward.cu), the pair's
// contribution to dL/dtheta for a trace gradient G is
//     g_f da + S0 dD1 + S1 dD2 + g_l de,
// g_f = G[jL-1], g_l = G[jH], S0 = sum_{j=jL}^{jH-1} G_j, S1 = sum (j-jL) G_j.
// The cell weights Q_j of a pair sum to zero (the N-wave has zero mean), so
// the pair's sum_j G_j Q_j equals sum_j (G_j - g_l) Q_j; written that way the
// sums only see differences of G and do not cancel when G varies slowly over
// the window. With Df = g_f - g_l, E0 = sum_n (G_{jL+n} - g_l),
// E1 = sum_n n (G_{jL+n} - g_l) (n = 0..L-1, L = jH - jL), Qf = R^2 - b0^2
// and K0 = w / (4 d h):
//     A'     = Df Qf + E0 h (2 b0 - h) - 2 h^2 E1        (= sum_j G_j Q_j)
//     B/2    = h E0 - b0 Df                             (= sum_j G_j dQ_j/dd / 2)
//     dL/dp0 = K0 A'
//     dL/dR  = 2 p0 K0 R Df
//     dL/dd  = p0 K0 (B - A'/d)
//     dL/dw  = p0 A' / (4 d h)
//     dL/dc  = dL/dd u + dL/dw (n - (n.u) u) / d       ([n.u > 0] when clamped)
//
// Kernels:
//   downsample   y_k = block mean over f_k samples (zero padded)
//   residual     G = 2 (S - y), L = sum (S - y)^2 (fixed-order last-block reduction)
//   adj_group    kAdjSplit consecutive CTAs share one chunk of consecutive
//                balls (one thread per ball) and split the sensors between
//                them. Each CTA walks its sensors in groups. For each group
//                it stages, per sensor, the window of G that the chunk's
//                bounding box can reach (past the record's end as zeros),
//                packed one after another into one
//                of two shared buffers with asynchronous copies, the next
//                group's copies in flight while the current group is
//                evaluated; a group takes as many sensor pairs as fill the
//                buffer. Every thread takes the group's sensors two at a
//                time, evaluating both pairs side by side in packed float2
//                arithmetic. A ball's five gradient components stay in its
//                thread's registers across the CTA's sensors. Each CTA then
//                writes its partial sums to global scratch; the last of the
//                chunk's CTAs to finish adds them in rank order and writes
//                every ball's gradients exactly once (no atomics on the
//                gradients, so the result is reproducible). A window longer
//                than half a buffer (e.g. an unsorted cloud) is not staged:
//                its pairs read the global row instead.

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include <cuda_pipeline.h>

#include "sbp_internal.cuh"

namespace {

constexpr int kAdjThreads = SBP_ADJ_CHUNK_MAX;  // balls (threads) per adjoint CTA
constexpr int kAdjSplit = 8;      // default CTAs per chunk, each taking 1/split of the sensors
constexpr int kAdjCap = 4096;     // cells per staging buffer (two buffers per CTA)
constexpr int kAdjCapP0 = 4096;   // the same for the p0-only adjoint
static_assert(SBP_FRAME_ALIGN % kAdjThreads == 0, "a chunk must not straddle two frames");
static_assert(kAdjThreads % SBP_ADJ_CHUNK == 0, "the scratch is sized in whole chunks");
constexpr int kAdjShare = 16;     // a CTA's share of the sensors is a multiple of this
constexpr int kAdjMeta = 128;     // sensors whose set-up is held in shared memory at once

__device__ __forceinline__ void downsample_one(const float* __restrict__ y, int T, int f,
                                               float* __restrict__ yk, long long t, int m, int j) {
    const float* row = y + (size_t)m * T;
    float s = 0.0f;
    for (int q = 0; q < f; ++q) {
        const int i = j * f + q;
        if (i < T) s += row[i];
    }
    yk[t] = s / (float)f;
}

__global__ void downsample_kernel(const float* __restrict__ y, int M, int T, int f, int Tk,
                                  float* __restrict__ yk) {
    const long long total = (long long)M * Tk;
    if (total < (1LL << 30)) {  // 32-bit index arithmetic (a 64-bit division is slow)
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < (int)total;
             t += gridDim.x * blockDim.x)
            downsample_one(y, T, f, yk, t, t / Tk, t % Tk);
        return;
    }
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x)
        downsample_one(y, T, f, yk, t, (int)(t / Tk), (int)(t % Tk));
}

// Sum of squares in float-float: hi + lo carries sum r^2 with the rounding
// error of every product and addition (relative error ~n 2^-48), so the
// per-thread sums need no double-precision arithmetic per element.
__device__ __forceinline__ void sq_acc(float r, float& hi, float& lo) {
    const float p = r * r;
    const float pe = fmaf(r, r, -p);
    float s, e;
    ff_two_sum(hi, p, s, e);
    hi = s;
    lo += e + pe;
}

// G = 2 (S - y) (S may be null: S = 0) and this thread's share of
// sum (S - y)^2 over [0, n), four elements per load when vec is set (then
// n is a multiple of 4 and the three arrays 16-byte aligned).
__device__ __forceinline__ void residual_span(const float* __restrict__ S,
                                              const float* __restrict__ y, float* __restrict__ G,
                                              long long n, bool vec, long long t0,
                                              long long stride, float& hi, float& lo) {
    if (vec) {
        const float4* y4 = reinterpret_cast<const float4*>(y);
        const float4* S4 = reinterpret_cast<const float4*>(S);
        float4* G4 = reinterpret_cast<float4*>(G);
        for (long long t = t0; t < n / 4; t += stride) {
            const float4 yv = y4[t];
            const float4 sv = S ? S4[t] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 r = make_float4(sv.x - yv.x, sv.y - yv.y, sv.z - yv.z, sv.w - yv.w);
            if (G) G4[t] = make_float4(2.0f * r.x, 2.0f * r.y, 2.0f * r.z, 2.0f * r.w);
            sq_acc(r.x, hi, lo);
            sq_acc(r.y, hi, lo);
            sq_acc(r.z, hi, lo);
            sq_acc(r.w, hi, lo);
        }
        return;
    }
    for (long long t = t0; t < n; t += stride) {
        const float r = (S ? S[t] : 0.0f) - y[t];
        if (G) G[t] = 2.0f * r;
        sq_acc(r, hi, lo);
    }
}

__device__ __forceinline__ double block_sum(double v, double* warp_sum) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = v;
    __syncthreads();
    double b = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (blockDim.x + 31) / 32; ++w) b += warp_sum[w];
    return b;  // valid in thread 0
}

// G = 2 (S - y); per-block sums of (S - y)^2 in double; the last block to
// finish adds the block sums in a fixed order (thread t takes blocks t,
// t + blockDim.x, ... in turn, then the fixed tree of block_sum).
__global__ void residual_kernel(const float* __restrict__ S, const float* __restrict__ y,
                                float* __restrict__ G, long long total, bool vec,
                                double* __restrict__ partials, SbpDevState* st,
                                double* loss) {
    __shared__ double warp_sum[32];
    __shared__ bool is_last;
    float hi = 0.f, lo = 0.f;
    residual_span(S, y, G, total, vec, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                  (long long)gridDim.x * blockDim.x, hi, lo);
    if (!loss) return;
    const double b = block_sum((double)hi + (double)lo, warp_sum);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = b;
        __threadfence();
        const unsigned int tk = atomicAdd(&st->loss_ticket, 1u);
        is_last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) {  // uniform over the block
        __threadfence();
        double v = 0.0;
        for (int bk = threadIdx.x; bk < (int)gridDim.x; bk += blockDim.x)
            v += __ldcg(partials + bk);
        const double L = block_sum(v, warp_sum);
        if (threadIdx.x == 0) {
            *loss = L;
            st->loss_ticket = 0;
        }
    }
}

struct GradOut {
    float* o[5];  // x, y, z, R, p0
};

// Window sums of one pair against the residual row of its sensor: the first
// cell gf = G[jL-1], the last cell gl = G[jH] (0 past the record) and, with
// d_q = G[jL+q] - gl over the L = min(jH, Tk) - jL ramp cells,
// Last cell any pair of the box can touch at this sensor, like sbp_box_cells
// but not clamped to the record: the staged window runs on past the record's
// end as zeros (G = 0 there), so the paired window sums need no clamps.
__device__ __forceinline__ int adj_box_hi(float sx, float sy, float sz, const float* box,
                                          const LevelGeo& g) {
    const float fx = fmaxf(fabsf(sx - box[0]), fabsf(sx - box[3]));
    const float fy = fmaxf(fabsf(sy - box[1]), fabsf(sy - box[4]));
    const float fz = fmaxf(fabsf(sz - box[2]), fabsf(sz - box[5]));
    const float dmax = sqrtf(fx * fx + fy * fy + fz * fz);
    const float hi = ceilf((dmax + fmaxf(box[6], 0.0f)) * g.inv_h) + 3.0f;
    return (int)fminf(fmaxf(hi, -1.0f), 2.0e9f);
}

// E0 = sum_q d_q and E1 = sum_q q d_q. Reads the staged window when it holds
// every needed cell, else the global row.
__device__ __forceinline__ void adj_window_sums(const float* __restrict__ sGrow, int jlo, int len,
                                                const float* __restrict__ Gm,
                                                int jL, int jH, int Tk, float& gf, float& gl,
                                                float& E0, float& E1) {
    const int L = min(jH, Tk) - jL;
    E0 = 0.f;
    E1 = 0.f;
    // the box bound puts cells jL-1 .. min(jH, Tk-1) inside the staged
    // window; checked anyway so that no read can leave it
    if (jL - 1 >= jlo && min(jH, Tk - 1) - jlo < len) {
        const float* Gw = sGrow - jlo + jL;
        gf = Gw[-1];
        gl = jH < Tk ? Gw[jH - jL] : 0.0f;
        // E1 = sum_q q d_q accumulated as the running sums of the tail
        float run = 0.0f;
        int q = L - 1;
        for (; q >= 2; q -= 2) {
            const float d1 = Gw[q] - gl, d0 = Gw[q - 1] - gl;
            run += d1;
            E1 += run;
            run += d0;
            E1 += run;
        }
        if (q == 1) {
            run += Gw[1] - gl;
            E1 += run;
        }
        E0 = L > 0 ? run + (Gw[0] - gl) : 0.0f;
    } else {
        gf = Gm[jL - 1];
        gl = jH < Tk ? Gm[jH] : 0.0f;
        for (int q = 0; q < L; ++q) {
            const float d = Gm[jL + q] - gl;
            E0 += d;
            E1 = fmaf((float)q, d, E1);
        }
    }
}

// P0_ONLY: only dL/dp0 is wanted (the zero-gradient pass), so the chain rule
// for R and the centre is skipped. WMODE: the orientation weight (SBP_W_*),
// fixed at compile time so that no pair branches on it.
// `split` CTAs share a chunk, each taking 1/split of the sensors.
template <bool P0_ONLY, int WMODE>
__global__ void __launch_bounds__(kAdjThreads, P0_ONLY ? 5 : 4)
adj_group_kernel(BallsDev b, FrameTable ft, const float* __restrict__ sens, LevelGeo g,
                 const float* __restrict__ G_all, unsigned mask, GradOut out,
                 float* __restrict__ part_all, unsigned int* __restrict__ tickets, int split,
                 bool vec) {
    // two staging buffers of kCap cells, each holding the windows of one
    // group of sensors packed one after another
    constexpr int kCap = P0_ONLY ? kAdjCapP0 : kAdjCap;
    constexpr int kWin = kCap / 2;  // longest window staged: a pair of them fills a buffer
    __shared__ __align__(16) float sG[2][kCap];
    // set-up of sensor pairs (2p, 2p + 1), each quantity of both sensors side
    // by side so that a pair's float2 operands load as one register pair
    __shared__ float4 s_q0[kAdjMeta / 2 + 1];  // sx, sy
    __shared__ float4 s_q1[kAdjMeta / 2 + 1];  // sz, nx
    __shared__ float4 s_q2[kAdjMeta / 2 + 1];  // ny, nz
    __shared__ int4 s_q3[kAdjMeta / 2 + 1];    // jlo, staged length (0: not staged)
    __shared__ int2 s_qo[kAdjMeta / 2 + 1];    // offset of the staged window in its group's buffer
    float* const q0f = reinterpret_cast<float*>(s_q0);
    float* const q1f = reinterpret_cast<float*>(s_q1);
    float* const q2f = reinterpret_cast<float*>(s_q2);
    int* const q3i = reinterpret_cast<int*>(s_q3);
    int* const qoi = reinterpret_cast<int*>(s_qo);
    // element of quantity c (0 or 1) of sensor t within its pair's record
    auto at = [](int t, int c) { return 4 * (t >> 1) + 2 * c + (t & 1); };
    __shared__ int s_gfirst[kAdjMeta / 2 + 2];  // first sensor of each group, then the count
    __shared__ int s_ng;
    __shared__ float s_red[(kAdjThreads / 32) * 7];
    __shared__ float s_box[7];
    static_assert(2 * kWin <= kCap, "a pair of staged windows must fit one buffer");
    // one-dimensional grid, chunk-major: the `split` CTAs of a chunk are
    // consecutive, so they run at about the same time and the partial sums
    // they leave for the chunk's last CTA are still in L2 when it reads them
    const int chunk_id = (int)(blockIdx.x / (unsigned)split);
    const int part = (int)blockIdx.x - chunk_id * split;
    const int c0 = chunk_id * kAdjThreads;
    const FrameSlot fs = sbp_frame_of(ft, c0);
    if (c0 >= fs.end) return;  // uniform over the chunk's CTAs
    const int c1 = min(fs.end, c0 + kAdjThreads);
    const int nb = c1 - c0;
    const int Tk = g.Tk, M = g.M;
    const float* __restrict__ G = G_all + (size_t)fs.f * M * Tk;
    // Threads take the chunk's balls in order of their window length class
    // floor(2R/h), so the lanes of a warp run window loops of nearly equal
    // length. (The order within a class is arbitrary; every ball's result is
    // computed by one thread and stored under the ball's own index.)
    __shared__ int s_cls[32], s_perm[kAdjThreads];
    if (threadIdx.x < 32) s_cls[threadIdx.x] = 0;
    sbp_chunk_box(b, c0, c1, s_red, s_box);  // also orders the clearing above
    int cls = 0;
    if ((int)threadIdx.x < nb) {
        const float Rk = b.R[c0 + threadIdx.x] * 2.0f * g.inv_h;
        cls = (int)fminf(fmaxf(Rk, 0.0f), 31.0f);  // NaN -> 0
        atomicAdd(&s_cls[cls], 1);
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan of the 32 class counts
        const int v = s_cls[threadIdx.x];
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, x, o);
            if ((int)threadIdx.x >= o) x += t;
        }
        s_cls[threadIdx.x] = x - v;
    }
    __syncthreads();
    if ((int)threadIdx.x < nb) s_perm[atomicAdd(&s_cls[cls], 1)] = threadIdx.x;
    __syncthreads();
    const bool valid = (int)threadIdx.x < nb;
    const int li = valid ? s_perm[threadIdx.x] : 0;  // this thread's ball, chunk-local
    const int i = c0 + li;
    float cx = 0.f, cy = 0.f, cz = 0.f, R = 0.f, p0 = 0.f;
    if (valid) {
        cx = b.x[i];
        cy = b.y[i];
        cz = b.z[i];
        R = b.R[i];
        p0 = b.p0[i];
    }
    const float h = g.h_hi;
    const float hh2 = 2.0f * h * h;
    float2 gx2 = f2(0.f), gy2 = f2(0.f), gz2 = f2(0.f), gR2 = f2(0.f), gp2 = f2(0.f);
    // this CTA's share of the sensors, whole groups
    const int per = ((M + split - 1) / split + kAdjShare - 1) / kAdjShare * kAdjShare;
    const int m_begin = min(M, part * per), m_end = min(M, m_begin + per);
    // The share is walked in blocks of up to kAdjMeta sensors whose positions,
    // normals and cell ranges are set up once, and within a block in groups of
    // consecutive sensor pairs whose residual windows, packed one after
    // another, fill one staging buffer (a window longer than kWin is not
    // staged: its pairs read the global row). Short windows (coarse levels,
    // compact chunks) so make long groups and few barriers. The windows of
    // group q + 1 are copied into the other buffer asynchronously while group
    // q is evaluated, so one barrier per group both publishes a group and
    // frees the buffer of the group before.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int mb = m_begin; mb < m_end; mb += kAdjMeta) {
        const int nsens = min(kAdjMeta, m_end - mb);
        __syncthreads();  // the previous block is done with every shared buffer
        for (int t = threadIdx.x; t < nsens; t += blockDim.x) {
            const int m = mb + t;
            const float sx = sens[m], sy = sens[M + m], sz = sens[2 * M + m];
            int jlo, jhi;
            sbp_box_cells(sx, sy, sz, s_box, g, jlo, jhi);
            // staged through the box's last cell even past the record (zeros there)
            jhi = max(jhi, adj_box_hi(sx, sy, sz, s_box, g));
            // with 16-byte copies a window starts on a 4-cell boundary and
            // holds a multiple of 4 cells
            if (vec) jlo &= ~3;
            int len = max(0, jhi - jlo + 1);
            if (vec) len = (len + 3) & ~3;
            if (len > kWin) len = 0;
            q0f[at(t, 0)] = sx;
            q0f[at(t, 1)] = sy;
            q1f[at(t, 0)] = sz;
            q1f[at(t, 1)] = sens[3 * M + m];
            q2f[at(t, 0)] = sens[4 * M + m];
            q2f[at(t, 1)] = sens[5 * M + m];
            q3i[at(t, 0)] = jlo;
            q3i[at(t, 1)] = len;
        }
        if ((nsens & 1) && threadIdx.x == 0) {  // odd count: a partner that no ball reaches
            const int t = nsens;
            q0f[at(t, 0)] = 1e6f;
            q0f[at(t, 1)] = 1e6f;
            q1f[at(t, 0)] = 1e6f;
            q1f[at(t, 1)] = 0.0f;
            q2f[at(t, 0)] = 0.0f;
            q2f[at(t, 1)] = 1.0f;
            q3i[at(t, 0)] = 0;
            q3i[at(t, 1)] = 0;
            qoi[t] = 0;
        }
        __syncthreads();
        if (warp == 0) {
            // Greedy packing of sensor pairs into groups: a group takes pairs
            // in order while their windows fit one buffer. With P the
            // inclusive prefix sums of the pairs' lengths, the group that
            // starts at pair g (exclusive prefix E_g) ends before the first
            // pair p with P_p - E_g > kCap; the window of pair p starts
            // E_p - E_g cells into its group's buffer. Lane l holds pairs l
            // and l + 32 (at most kAdjMeta / 2 = 64 pairs).
            static_assert(kAdjMeta <= 128, "two pairs per lane");
            const int npairs = (nsens + 1) >> 1;
            int la[2], w[2], P[2], E[2], gb[2] = {0, 0};
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int p = lane + 32 * hh;
                la[hh] = p < npairs ? q3i[at(2 * p, 1)] : 0;
                const int lb = 2 * p + 1 < nsens ? q3i[at(2 * p + 1, 1)] : 0;
                w[hh] = p < npairs ? la[hh] + lb : 0;
                int x = w[hh];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += t;
                }
                P[hh] = x;
            }
            P[1] += __shfl_sync(0xffffffffu, P[0], 31);
            E[0] = P[0] - w[0];
            E[1] = P[1] - w[1];
            int ng = 0, base = 0;  // ng: groups started so far, kept by lane 0 (which writes them)
            for (;;) {  // each pass starts a group at a later pair: at most npairs passes
                const unsigned m0 = __ballot_sync(0xffffffffu, lane < npairs && P[0] - base > kCap);
                const unsigned m1 =
                    __ballot_sync(0xffffffffu, lane + 32 < npairs && P[1] - base > kCap);
                if (!(m0 | m1)) break;
                const int first = m0 ? __ffs(m0) - 1 : 32 + __ffs(m1) - 1;
                base = __shfl_sync(0xffffffffu, first < 32 ? E[0] : E[1], first & 31);
                if (lane == 0) s_gfirst[++ng] = 2 * first;
                if (lane >= first) gb[0] = base;
                if (lane + 32 >= first) gb[1] = base;
            }
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int p = lane + 32 * hh;
                if (p < npairs) {
                    qoi[2 * p] = E[hh] - gb[hh];
                    if (2 * p + 1 < nsens) qoi[2 * p + 1] = E[hh] - gb[hh] + la[hh];
                }
            }
            if (lane == 0) {
                s_gfirst[0] = 0;
                s_gfirst[ng + 1] = nsens;
                s_ng = ng + 1;
            }
        }
        __syncthreads();
        const int ng = s_ng;
        // asynchronous copy of group q's windows into buffer q & 1, a warp per
        // sensor
        auto stage = [&](int q) {
            float* dst = sG[q & 1];
            for (int s = s_gfirst[q] + warp; s < s_gfirst[q + 1]; s += kAdjThreads / 32) {
                const int jlo = q3i[at(s, 0)], len = q3i[at(s, 1)];
                const float* row = G + (size_t)(mb + s) * Tk + jlo;
                float* d = dst + qoi[s];
                const int inrec = min(len, Tk - jlo);  // cells before the record's end
                if (vec) {
                    for (int r = 4 * lane; r < len; r += 128) {
                        if (r + 4 <= inrec) {
                            __pipeline_memcpy_async(d + r, row + r, 16);
                        } else {
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                if (r + c < inrec)
                                    __pipeline_memcpy_async(d + r + c, row + r + c, sizeof(float));
                                else
                                    d[r + c] = 0.0f;
                            }
                        }
                    }
                } else {
                    for (int r = lane; r < len; r += 32) {
                        if (r < inrec)
                            __pipeline_memcpy_async(d + r, row + r, sizeof(float));
                        else
                            d[r] = 0.0f;
                    }
                }
            }
        };
        stage(0);
        __pipeline_commit();
        for (int q = 0; q < ng; ++q) {
            __pipeline_wait_prior(0);  // this thread's copies of group q have landed
            __syncthreads();  // ... everyone's; and group q - 1 is no longer read
            if (q + 1 < ng) {
                stage(q + 1);
                __pipeline_commit();
            }
            const int gbase = s_gfirst[q];
            const int cnt = s_gfirst[q + 1] - gbase;
            const int m0 = mb + gbase;
            const int pbase = gbase >> 1;  // groups start at even sensors
            const float* __restrict__ sGb = sG[q & 1];
            if (!valid) continue;
            // two sensors at a time, evaluated side by side in the halves of float2
#pragma unroll 1
            for (int s = 0; s < cnt; s += 2) {
                const int pi = pbase + (s >> 1);
                const float4 Q0 = s_q0[pi], Q1 = s_q1[pi], Q2 = s_q2[pi];
                const int4 Q3 = s_q3[pi];
                const int2 QO = s_qo[pi];
                const float* __restrict__ sGA = sGb + QO.x;
                const float* __restrict__ sGB = sGb + QO.y;
                // dL/dp0 is continuous in the distance (the cell values are), so the
                // p0-only pass takes it in plain float; the full gradient, whose
                // centre and radius terms jump at the window's ends, needs the
                // exact one
                const PairDist2 pd =
                    P0_ONLY ? sbp_pair_distance2_f32(f2(cx), f2(cy), f2(cz),
                                                     make_float2(Q0.x, Q0.y),
                                                     make_float2(Q0.z, Q0.w),
                                                     make_float2(Q1.x, Q1.y))
                            : sbp_pair_distance2(f2(cx), f2(cy), f2(cz), make_float2(Q0.x, Q0.y),
                                                 make_float2(Q0.z, Q0.w),
                                                 make_float2(Q1.x, Q1.y));
                PairWindow wa, wb;
                bool okA, okB;
                sbp_window2(pd.dh, pd.dl, f2(R), g, wa, wb, okA, okB);
                if (!(okA || okB)) continue;
                const float2 ux = f2mul(pd.dx, pd.rd), uy = f2mul(pd.dy, pd.rd),
                             uz = f2mul(pd.dz, pd.rd);
                const float2 nx = make_float2(Q1.z, Q1.w), ny = make_float2(Q2.x, Q2.y),
                             nz = make_float2(Q2.z, Q2.w);
                const float2 cosv = f2fma(nx, ux, f2fma(ny, uy, f2mul(nz, uz)));
                float actA, actB;
                float wA = sbp_weight(WMODE, cosv.x, actA), wB = sbp_weight(WMODE, cosv.y, actB);
                okA = okA && !(wA == 0.0f && actA == 0.0f);
                okB = okB && !(wB == 0.0f && actB == 0.0f);
                if (!(okA || okB)) continue;
                // window sums; a pair that does not count gets zeros, so that its
                // half contributes exactly nothing below
                const int jloA = Q3.x, lenA = Q3.z;
                const int jloB = Q3.y, lenB = Q3.w;
                float2 gf = f2(0.f), gl = f2(0.f), E0 = f2(0.f), E1 = f2(0.f);
                // side by side when both windows are staged (cells past the
                // record staged as zeros, so no clamps) and differ by at most one
                // ramp cell: the shorter one then reads one cell further, its own
                // last cell G[jH], which adds d = 0
                const int LA = wa.jH - wa.jL, LB = wb.jH - wb.jL;
                const bool inA = okA && wa.jL - 1 >= jloA && wa.jH - jloA < lenA;
                const bool inB = okB && wb.jL - 1 >= jloB && wb.jH - jloB < lenB;
                if (inA && inB && abs(LA - LB) <= 1) {
                    const float* GwA = sGA - jloA + wa.jL;
                    const float* GwB = sGB - jloB + wb.jL;
                    gf = make_float2(GwA[-1], GwB[-1]);
                    gl = make_float2(GwA[LA], GwB[LB]);
                    const float2 ngl = f2neg(gl);
                    const int Lm = max(LA, LB);
                    float2 run = f2(0.f);
                    int q = Lm - 1;
                    if (q >= 2) {
                        // cells q and q - 1 loaded one step ahead (q - 3 >= -1
                        // stays inside the staged window)
                        float2 c1 = make_float2(GwA[q], GwB[q]);
                        float2 c0 = make_float2(GwA[q - 1], GwB[q - 1]);
                        for (; q >= 2; q -= 2) {
                            const float2 n1 = make_float2(GwA[q - 2], GwB[q - 2]);
                            const float2 n0 = make_float2(GwA[q - 3], GwB[q - 3]);
                            const float2 d1 = f2add(c1, ngl);
                            const float2 d0 = f2add(c0, ngl);
                            run = f2add(run, d1);
                            E1 = f2add(E1, run);
                            run = f2add(run, d0);
                            E1 = f2add(E1, run);
                            c1 = n1;
                            c0 = n0;
                        }
                    }
                    if (q == 1) {
                        run = f2add(run, f2add(make_float2(GwA[1], GwB[1]), ngl));
                        E1 = f2add(E1, run);
                    }
                    if (Lm > 0) E0 = f2add(run, f2add(make_float2(GwA[0], GwB[0]), ngl));
                } else {
                    if (okA)
                        adj_window_sums(sGA, jloA, lenA,
                                        G + (size_t)(m0 + s) * Tk, wa.jL, wa.jH, Tk, gf.x, gl.x, E0.x,
                                        E1.x);
                    if (okB)
                        adj_window_sums(sGB, jloB, lenB,
                                        G + (size_t)(m0 + s + 1) * Tk, wb.jL, wb.jH, Tk, gf.y, gl.y,
                                        E0.y, E1.y);
                }
                if (!okA) {
                    wA = 0.0f;
                    actA = 0.0f;
                }
                if (!okB) {
                    wB = 0.0f;
                    actB = 0.0f;
                }
                const float2 b0 = make_float2(okA ? wa.b0 : 0.0f, okB ? wb.b0 : 0.0f);
                const float2 Df = f2sub(gf, gl);
                const float2 ra = make_float2(fmaxf(R - b0.x, 0.0f), fmaxf(R - b0.y, 0.0f));
                const float2 A = f2fma(f2mul(Df, ra), f2add(f2(R), b0),
                                       f2fma(f2mul(E0, f2(h)), f2fma(f2(2.0f), b0, f2(-h)),
                                             f2mul(f2(-hh2), E1)));
                const float2 qd = f2mul(f2(g.inv_4h), pd.rd);  // 1 / (4 d h)
                const float2 K0 = f2mul(make_float2(wA, wB), qd);
                gp2 = f2fma(K0, A, gp2);
                if (P0_ONLY) continue;
                const float2 Bh = f2fma(f2(h), E0, f2neg(f2mul(b0, Df)));
                const float2 pK = f2mul(f2(p0), K0);
                gR2 = f2fma(f2mul(pK, f2(2.0f * R)), Df, gR2);
                const float2 gd = f2mul(pK, f2fma(f2(2.0f), Bh, f2neg(f2mul(A, pd.rd))));
                const float2 gw = f2mul(f2mul(f2mul(f2(p0), A), qd), make_float2(actA, actB));
                const float2 gwr = f2mul(gw, pd.rd);
                gx2 = f2fma(gd, ux, f2fma(gwr, f2fma(f2neg(cosv), ux, nx), gx2));
                gy2 = f2fma(gd, uy, f2fma(gwr, f2fma(f2neg(cosv), uy, ny), gy2));
                gz2 = f2fma(gd, uz, f2fma(gwr, f2fma(f2neg(cosv), uz, nz), gz2));
            }
        }
    }
    const float gx = gx2.x + gx2.y, gy = gy2.x + gy2.y, gz = gz2.x + gz2.y;
    const float gR = gR2.x + gR2.y, gp = gp2.x + gp2.y;
    // This CTA's partial sums go to global scratch [chunk][part][5][ball]. The
    // last of the chunk's CTAs to arrive (a ticket per chunk) adds the parts
    // in rank order and writes every ball's gradients exactly once, so the
    // result does not depend on which CTA finishes last, and no CTA waits
    // for another.
    const size_t chunk = chunk_id;
    float* __restrict__ mine = part_all + (chunk * split + part) * 5 * kAdjThreads;
    if (valid) {  // stored under the ball's chunk-local index
        if (!P0_ONLY) {
            mine[0 * kAdjThreads + li] = gx;
            mine[1 * kAdjThreads + li] = gy;
            mine[2 * kAdjThreads + li] = gz;
            mine[3 * kAdjThreads + li] = gR;
        }
        mine[4 * kAdjThreads + li] = gp;
    }
    __threadfence();
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&tickets[chunk], 1u) == (unsigned int)(split - 1);
    __syncthreads();
    if (!s_last) return;  // uniform over the block
    __threadfence();
    if (valid) {
        const float* __restrict__ all = part_all + chunk * split * 5 * kAdjThreads + li;
        float a[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        for (int r = 0; r < split; ++r) {
            const float* pr = all + (size_t)r * 5 * kAdjThreads;
#pragma unroll
            for (int c = P0_ONLY ? 4 : 0; c < 5; ++c) a[c] += __ldcg(pr + c * kAdjThreads);
        }
        const bool xyz = mask & SBP_MASK_XYZ;
        out.o[0][i] = xyz ? a[0] : 0.0f;
        out.o[1][i] = xyz ? a[1] : 0.0f;
        out.o[2][i] = xyz ? a[2] : 0.0f;
        out.o[3][i] = (mask & SBP_MASK_R) ? a[3] : 0.0f;
        out.o[4][i] = (mask & SBP_MASK_P0) ? a[4] : 0.0f;
    }
    if (threadIdx.x == 0) tickets[chunk] = 0u;  // ready for the next launch
}

}  // namespace

int sbp_launch_downsample(sbp_array_s* a, int k, const float* y_full, float* y_k,
                          cudaStream_t st) {
    const int Tk = sbp_level_T(a, k);
    const long long total = (long long)a->M * Tk;
    // about one output per thread, so that many loads are in flight
    const int blocks = (int)std::max<long long>(1, std::min<long long>(32768, (total + 255) / 256));
    downsample_kernel<<<blocks, 256, 0, st>>>(y_full, a->M, a->T, a->factors[k], Tk, y_k);
    sbp_count_launches(1);
    return sbp_cuda_check(cudaGetLastError(), "downsample launch") ? SBP_ERR_CUDA : SBP_OK;
}

// Downsample `rows` consecutive records of T samples (frames x sensors).
int sbp_launch_downsample_rows(sbp_array_s* a, int k, int rows, const float* y_full,
                               float* y_k, cudaStream_t st) {
    const int Tk = sbp_level_T(a, k);
    const long long total = (long long)rows * Tk;
    const int blocks = (int)std::max<long long>(1, std::min<long long>(32768, (total + 255) / 256));
    downsample_kernel<<<blocks, 256, 0, st>>>(y_full, rows, a->T, a->factors[k], Tk, y_k);
    sbp_count_launches(1);
    return sbp_cuda_check(cudaGetLastError(), "downsample launch") ? SBP_ERR_CUDA : SBP_OK;
}

namespace {

// The four-wide path needs n % 4 == 0 and 16-byte aligned arrays.
bool residual_vec(const float* S, const float* y, const float* G, long long n) {
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    return n % 4 == 0 && al(y) && (!S || al(S)) && (!G || al(G));
}

}  // namespace

int sbp_launch_residual(sbp_array_s* a, const float* S, const float* y, float* G,
                        double* loss, cudaStream_t st) {
    const int Tk = sbp_level_T(a, a->level);
    const long long total = (long long)a->M * Tk;
    const bool vec = residual_vec(S, y, G, total);
    const int blocks = (int)std::max<long long>(
        1, std::min<long long>(a->loss_blocks, (total / (vec ? 4 : 1) + 255) / 256));
    residual_kernel<<<blocks, 256, 0, st>>>(S, y, G, total, vec, a->d_lossp, a->d_state, loss);
    sbp_count_launches(1);
    return sbp_cuda_check(cudaGetLastError(), "residual launch") ? SBP_ERR_CUDA : SBP_OK;
}

namespace {

int launch_adj(sbp_array_s* a, const FrameTable& ft, int total, int split, const BallsDev& b,
               const LevelGeo& g, const float* G, unsigned mask, const GradOut& o,
               cudaStream_t st) {
    if (split != 1 && split != 2 && split != 4 && split != 8) split = kAdjSplit;
    static_assert(kAdjSplit <= SBP_ADJ_MAX_SPLIT, "the scratch holds at most 8 parts");
    const int chunks = (total + kAdjThreads - 1) / kAdjThreads;
    if ((long long)chunks * kAdjThreads > (long long)a->adj_chunks * SBP_ADJ_CHUNK) {
        sbp_set_error("adjoint: more balls than the array's capacity");
        return SBP_ERR_ARG;
    }
    const unsigned grid = (unsigned)chunks * (unsigned)split;
    // 16-byte staging copies need every residual row 16-byte aligned
    const bool vec = (g.Tk % 4 == 0) && ((reinterpret_cast<uintptr_t>(G) & 15u) == 0);
    auto go = [&](auto p0_only, auto wmode) {
        adj_group_kernel<decltype(p0_only)::value, decltype(wmode)::value>
            <<<grid, kAdjThreads, 0, st>>>(b, ft, a->d_sens, g, G, mask, o, a->d_adj_part,
                                           a->d_adj_ticket, split, vec);
    };
    auto by_mode = [&](auto p0_only) {
        if (g.wmode == SBP_W_NONE)
            go(p0_only, std::integral_constant<int, SBP_W_NONE>{});
        else if (g.wmode == SBP_W_COS)
            go(p0_only, std::integral_constant<int, SBP_W_COS>{});
        else
            go(p0_only, std::integral_constant<int, SBP_W_CLAMP>{});
    };
    if (mask == SBP_MASK_P0)
        by_mode(std::true_type{});
    else
        by_mode(std::false_type{});
    if (sbp_cuda_check(cudaGetLastError(), "adjoint: launch")) return SBP_ERR_CUDA;
    sbp_count_launches(1);
    return SBP_OK;
}

}  // namespace

int sbp_launch_adjoint(sbp_array_s* a, const BallsDev& b, const int* n_dev, int n_cap,
                       const float* G, sbp_grads out, unsigned mask, cudaStream_t st) {
    const LevelGeo g = sbp_level_geo(a, a->level);
    GradOut o;
    o.o[0] = out.gx;
    o.o[1] = out.gy;
    o.o[2] = out.gz;
    o.o[3] = out.gR;
    o.o[4] = out.gp0;
    const FrameTable ft{1, nullptr, n_dev, n_cap};
    const int split = a->adj_split_lvl[a->level] ? a->adj_split_lvl[a->level] : kAdjSplit;
    return launch_adj(a, ft, n_cap, split, b, g, G, mask, o, st);
}

// All frames of the packed layout in one launch (sbp_adjoint_frames).
int sbp_launch_adjoint_frames(sbp_array_s* a, const BallsDev& b, const int* n_dev,
                              const float* G, sbp_grads out, unsigned mask, cudaStream_t st) {
    const LevelGeo g = sbp_level_geo(a, a->level);
    GradOut o;
    o.o[0] = out.gx;
    o.o[1] = out.gy;
    o.o[2] = out.gz;
    o.o[3] = out.gR;
    o.o[4] = out.gp0;
    const int total = a->h_frame_off[a->frames];
    const FrameTable ft{a->frames, a->d_frame_off, n_dev, total};
    return launch_adj(a, ft, total, a->adj_split_frames ? a->adj_split_frames : kAdjSplit, b, g,
                      G, mask, o, st);
}

namespace {

// Per-frame sums of (S - y)^2: block partials, then one thread per frame adds
// them in block order (reproducible).
// Frame f = blockIdx.y: G = 2 (S - y) over the frame and, when partials is
// set, this block's sum of (S - y)^2 into partials[f][blockIdx.x].
__global__ void frame_loss_partial_kernel(const float* __restrict__ S, const float* __restrict__ y,
                                          float* __restrict__ G, long long per_frame, bool vec,
                                          double* __restrict__ partials) {
    __shared__ double warp_sum[32];
    const int f = blockIdx.y;
    const size_t o = (size_t)f * per_frame;
    float hi = 0.f, lo = 0.f;
    residual_span(S ? S + o : nullptr, y + o, G ? G + o : nullptr, per_frame, vec,
                  blockIdx.x * (long long)blockDim.x + threadIdx.x,
                  (long long)gridDim.x * blockDim.x, hi, lo);
    if (!partials) return;
    const double b = block_sum((double)hi + (double)lo, warp_sum);
    if (threadIdx.x == 0) partials[(size_t)f * gridDim.x + blockIdx.x] = b;
}

__global__ void frame_loss_final_kernel(const double* __restrict__ partials, int blocks, int F,
                                        double* __restrict__ loss) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    double L = 0.0;
    for (int k = 0; k < blocks; ++k) L += partials[(size_t)f * blocks + k];
    loss[f] = L;
}

}  // namespace

// G = 2 (S - y) over all frames and one loss per frame (sbp_residual_frames).
int sbp_launch_residual_frames(sbp_array_s* a, const float* S, const float* y, float* G,
                               double* loss, cudaStream_t st) {
    const int Tk = sbp_level_T(a, a->level);
    const long long per = (long long)a->M * Tk;
    const bool vec = residual_vec(S, y, G, per);  // per % 4 == 0 keeps every frame aligned
    // blocks per frame: enough to fill the GPU, at most the 16 partials a frame has room for
    const int fb = (int)std::max<long long>(
        1, std::min<long long>(
               {16LL, (4LL * a->sm_count + a->frames - 1) / a->frames,
                (per / (vec ? 4 : 1) + 255) / 256}));
    frame_loss_partial_kernel<<<dim3(fb, a->frames), 256, 0, st>>>(
        S, y, G, per, vec, loss ? a->d_frame_lossp : nullptr);
    int launched = 1;
    if (loss) {
        frame_loss_final_kernel<<<(a->frames + 127) / 128, 128, 0, st>>>(a->d_frame_lossp, fb,
                                                                          a->frames, loss);
        launched += 1;
    }
    sbp_count_launches(launched);
    return sbp_cuda_check(cudaGetLastError(), "residual_frames launch") ? SBP_ERR_CUDA : SBP_OK;
}
