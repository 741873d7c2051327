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
// the window. With Df = g_f - g_l, E0 = S0 - L g_l, E1 = S1 - L(L-1)/2 g_l
// (L = jH - jL), Qf = R^2 - b0^2 and K0 = w / (4 d h):
//     A'     = Df Qf + E0 h (2 b0 - h) - 2 h^2 E1        (= sum_j G_j Q_j)
//     B/2    = h E0 - b0 Df                             (= sum_j G_j dQ_j/dd / 2)
//     dL/dp0 = K0 A'
//     dL/dR  = 2 p0 K0 R Df
//     dL/dd  = p0 K0 (B - A'/d)
//     dL/dw  = p0 A' / (4 d h)
//     dL/dc  = dL/dd u + dL/dw (n - (n.u) u) / d       ([n.u > 0] when clamped)
// G is rounded per sensor to 31-bit fixed point; S0, S1 come from exclusive
// prefix sums of G and j G and every difference above is exact int64 before
// it is converted to float, so every pair costs O(1) work regardless of how
// many cells its window spans.
//
// Kernels:
//   downsample   y_k = block mean over f_k samples (zero padded)
//   residual     G = 2 (S - y), L = sum (S - y)^2 (fixed-order last-block reduction)
//   adj_prep     CTA = one sensor: quantise G, prefix sums -> records
//   adj_pair     thread = one ball, CTA column = one sensor group; gradients of
//                each ball accumulated in registers and written once
//   adj_reduce   fixed-order sum of per-group partials (only when sensors are split)
#include <algorithm>

#include "sbp_internal.cuh"
#include "sbp_scan.cuh"

namespace {

constexpr int kPrepThreads = 1024;
constexpr int kPairThreads = 128;
constexpr int kSensTile = 256;  // sensors staged in shared memory at a time

__global__ void downsample_kernel(const float* __restrict__ y, int M, int T, int f, int Tk,
                                  float* __restrict__ yk) {
    const long long total = (long long)M * Tk;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(t / Tk), j = (int)(t % Tk);
        const float* row = y + (size_t)m * T;
        float s = 0.0f;
        for (int q = 0; q < f; ++q) {
            const int i = j * f + q;
            if (i < T) s += row[i];
        }
        yk[t] = s / (float)f;
    }
}

// G = 2 (S - y); per-block sums of (S - y)^2 in double; the last block to
// finish adds the block sums in index order.
__global__ void residual_kernel(const float* __restrict__ S, const float* __restrict__ y,
                                float* __restrict__ G, long long total,
                                double* __restrict__ partials, SbpDevState* st,
                                double* loss) {
    __shared__ double warp_sum[32];
    __shared__ bool is_last;
    double acc = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const float r = (S ? S[t] : 0.0f) - y[t];
        G[t] = 2.0f * r;
        acc += (double)r * (double)r;
    }
    if (!loss) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (blockDim.x + 31) / 32; ++w) b += warp_sum[w];
        partials[blockIdx.x] = b;
        __threadfence();
        const unsigned int tk = atomicAdd(&st->loss_ticket, 1u);
        is_last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last && threadIdx.x == 0) {
        __threadfence();
        double L = 0.0;
        for (int bk = 0; bk < (int)gridDim.x; ++bk) L += ((volatile double*)partials)[bk];
        *loss = L;
        st->loss_ticket = 0;
    }
}

// One CTA per sensor. Records rec[m][j] = (sum_{j'<j} Gq, sum_{j'<j} j' Gq),
// j = 0..Tk, and gq[m][j] = Gq_j, with Gq = round(G * 2^s), |Gq| < 2^30;
// ginv[m] = 2^-s.
__global__ void __launch_bounds__(kPrepThreads)
adj_prep_kernel(const float* __restrict__ G, int Tk, longlong2* __restrict__ rec,
                int* __restrict__ gq, float* __restrict__ ginv) {
    __shared__ long long warp_tot[32];
    __shared__ float warp_max[32];
    const int m = blockIdx.x;
    const float* row = G + (size_t)m * Tk;
    longlong2* out = rec + (size_t)m * (Tk + 1);
    int* qout = gq + (size_t)m * Tk;
    float mx = 0.0f;
    for (int j = threadIdx.x; j < Tk; j += blockDim.x) mx = fmaxf(mx, fabsf(row[j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x + 31) / 32 ? warp_max[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) warp_max[0] = v;
    }
    __syncthreads();
    const float gmax = warp_max[0];
    int e = 0;
    if (gmax > 0.0f) frexpf(gmax, &e);  // gmax < 2^e
    int s = 30 - e;
    s = s < -100 ? -100 : (s > 100 ? 100 : s);
    if (threadIdx.x == 0) ginv[m] = ldexpf(1.0f, -s);

    long long c0 = 0, c1 = 0;
    constexpr int IPT = 4;
    const int tile = blockDim.x * IPT;
    for (int base = 0; base < Tk + 1; base += tile) {
        long long q[IPT], qj[IPT];
        const int i0 = base + threadIdx.x * IPT;
        long long r0 = 0, r1 = 0;
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const int i = i0 + k;
            q[k] = i < Tk ? (long long)llrintf(ldexpf(row[i], s)) : 0;
            qj[k] = q[k] * (long long)i;
            r0 += q[k];
            r1 += qj[k];
        }
        long long t0, t1;
        const long long x0 = sbp_block_incl_scan(r0, warp_tot, t0) - r0 + c0;
        const long long x1 = sbp_block_incl_scan(r1, warp_tot, t1) - r1 + c1;
        long long e0 = x0, e1 = x1;  // exclusive prefix at i0
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const int i = i0 + k;
            if (i <= Tk) out[i] = make_longlong2(e0, e1);
            if (i < Tk) qout[i] = (int)q[k];
            e0 += q[k];
            e1 += qj[k];
        }
        c0 += t0;
        c1 += t1;
    }
}

struct GradOut {
    float* o[5];  // x, y, z, R, p0
};

__global__ void __launch_bounds__(kPairThreads)
adj_pair_kernel(BallsDev b, const int* n_dev, int n_cap, const float* __restrict__ sens,
                LevelGeo g, const int* __restrict__ gq, const longlong2* __restrict__ rec,
                const float* __restrict__ ginv, int sens_per_group, unsigned mask, GradOut out,
                size_t group_stride) {
    __shared__ float s_sens[kSensTile][8];
    const int n = sbp_read_n(n_dev, n_cap);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    const int M = g.M, Tk = g.Tk;
    const int m_begin = blockIdx.y * sens_per_group;
    const int m_end = min(M, m_begin + sens_per_group);
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
    float gx = 0.f, gy = 0.f, gz = 0.f, gR = 0.f, gp = 0.f;
    for (int t0 = m_begin; t0 < m_end; t0 += kSensTile) {
        const int cnt = min(kSensTile, m_end - t0);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt * 7; t += blockDim.x) {
            const int s = t / 7, k = t % 7;
            s_sens[s][k] = k < 6 ? sens[k * M + t0 + s] : ginv[t0 + s];
        }
        __syncthreads();
        if (!valid) continue;
#pragma unroll 1
        for (int s = 0; s < cnt; ++s) {
            const int m = t0 + s;
            const PairDist pd =
                sbp_pair_distance(cx, cy, cz, s_sens[s][0], s_sens[s][1], s_sens[s][2]);
            if (!(pd.dh + pd.dl > R)) continue;
            PairWindow win;
            if (!sbp_window(pd, R, g, false, win)) continue;
            const int jL = win.jL, jH = win.jH;
            const float ux = pd.dx * pd.rd, uy = pd.dy * pd.rd, uz = pd.dz * pd.rd;
            const float nx = s_sens[s][3], ny = s_sens[s][4], nz = s_sens[s][5];
            const float cosv = nx * ux + ny * uy + nz * uz;
            float act;
            const float w = sbp_weight(g.wmode, cosv, act);
            if (w == 0.0f && act == 0.0f) continue;
            const float b0 = win.b0;
            const int* Gm = gq + (size_t)m * Tk;
            const long long qf = Gm[jL - 1];
            const long long ql = jH < Tk ? Gm[jH] : 0;
            const longlong2* rm = rec + (size_t)m * (Tk + 1);
            const int lo = min(jL, Tk), hi = min(jH, Tk);
            const longlong2 rl = rm[lo], rh = rm[hi];
            const long long S0 = rh.x - rl.x;
            const long long S1 = (rh.y - rl.y) - (long long)jL * S0;
            const long long L = jH - jL;
            const float sc = s_sens[s][6];
            const float Df = __ll2float_rn(qf - ql) * sc;
            const float E0 = __ll2float_rn(S0 - L * ql) * sc;
            const float E1 = __ll2float_rn(S1 - ((L * (L - 1)) >> 1) * ql) * sc;
            const float A = Df * fmaxf(R - b0, 0.0f) * (R + b0) + E0 * h * (2.0f * b0 - h) -
                            hh2 * E1;
            const float Bh = h * E0 - b0 * Df;
            const float q = g.inv_4h * pd.rd;  // 1 / (4 d h)
            const float K0 = w * q;
            gp += K0 * A;
            gR += 2.0f * p0 * K0 * R * Df;
            const float gd = p0 * K0 * (2.0f * Bh - A * pd.rd);
            const float gw = p0 * A * q * act;
            gx += gd * ux + gw * (nx - cosv * ux) * pd.rd;
            gy += gd * uy + gw * (ny - cosv * uy) * pd.rd;
            gz += gd * uz + gw * (nz - cosv * uz) * pd.rd;
        }
    }
    if (!valid) return;
    const size_t base = (size_t)blockIdx.y * group_stride;
    const bool xyz = mask & SBP_MASK_XYZ;
    out.o[0][base + i] = xyz ? gx : 0.0f;
    out.o[1][base + i] = xyz ? gy : 0.0f;
    out.o[2][base + i] = xyz ? gz : 0.0f;
    out.o[3][base + i] = (mask & SBP_MASK_R) ? gR : 0.0f;
    out.o[4][base + i] = (mask & SBP_MASK_P0) ? gp : 0.0f;
}

// grads[k][i] = sum over groups, in group order, of part[g][k][i].
__global__ void adj_reduce_kernel(const float* __restrict__ part, int groups, int n_cap,
                                  const int* n_dev, GradOut out) {
    const int n = sbp_read_n(n_dev, n_cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            float s = 0.0f;
            for (int gi = 0; gi < groups; ++gi) s += part[((size_t)gi * 5 + k) * n_cap + i];
            out.o[k][i] = s;
        }
    }
}

}  // namespace

int sbp_launch_downsample(sbp_array_s* a, int k, const float* y_full, float* y_k,
                          cudaStream_t st) {
    const int Tk = sbp_level_T(a, k);
    const long long total = (long long)a->M * Tk;
    const int blocks = (int)std::max<long long>(
        1, std::min<long long>(8LL * a->sm_count, (total + 255) / 256));
    downsample_kernel<<<blocks, 256, 0, st>>>(y_full, a->M, a->T, a->factors[k], Tk, y_k);
    return sbp_cuda_check(cudaGetLastError(), "downsample launch") ? SBP_ERR_CUDA : SBP_OK;
}

int sbp_launch_residual(sbp_array_s* a, const float* S, const float* y, float* G,
                        double* loss, cudaStream_t st) {
    const int Tk = sbp_level_T(a, a->level);
    const long long total = (long long)a->M * Tk;
    const int blocks = (int)std::max<long long>(
        1, std::min<long long>(a->loss_blocks, (total + 255) / 256));
    residual_kernel<<<blocks, 256, 0, st>>>(S, y, G, total, a->d_lossp, a->d_state, loss);
    return sbp_cuda_check(cudaGetLastError(), "residual launch") ? SBP_ERR_CUDA : SBP_OK;
}

int sbp_launch_adjoint(sbp_array_s* a, const BallsDev& b, const int* n_dev, int n_cap,
                       const float* G, sbp_grads out, unsigned mask, cudaStream_t st) {
    const LevelGeo g = sbp_level_geo(a, a->level);
    float* ginv = a->d_ginv;
    adj_prep_kernel<<<g.M, kPrepThreads, 0, st>>>(G, g.Tk, a->d_rec, a->d_gq, ginv);
    if (sbp_cuda_check(cudaGetLastError(), "adjoint: prep launch")) return SBP_ERR_CUDA;
    const int ball_blocks = (n_cap + kPairThreads - 1) / kPairThreads;
    // split sensors across CTAs when there are too few balls to fill the GPU
    int groups = std::max(1, (4 * a->sm_count + ball_blocks - 1) / ball_blocks);
    groups = std::min(groups, std::min(g.M, a->part_groups));
    const int per = (g.M + groups - 1) / groups;
    groups = (g.M + per - 1) / per;
    GradOut o;
    if (groups == 1) {
        o.o[0] = out.gx;
        o.o[1] = out.gy;
        o.o[2] = out.gz;
        o.o[3] = out.gR;
        o.o[4] = out.gp0;
    } else {
        for (int k = 0; k < 5; ++k) o.o[k] = a->d_part + (size_t)k * n_cap;
    }
    dim3 grid(ball_blocks, groups);
    adj_pair_kernel<<<grid, kPairThreads, 0, st>>>(b, n_dev, n_cap, a->d_sens, g, a->d_gq, a->d_rec,
                                                   ginv, per, mask, o, (size_t)5 * n_cap);
    if (sbp_cuda_check(cudaGetLastError(), "adjoint: pair launch")) return SBP_ERR_CUDA;
    if (groups > 1) {
        GradOut d;
        d.o[0] = out.gx;
        d.o[1] = out.gy;
        d.o[2] = out.gz;
        d.o[3] = out.gR;
        d.o[4] = out.gp0;
        const int blocks = std::max(1, std::min(4 * a->sm_count, (n_cap + 255) / 256));
        adj_reduce_kernel<<<blocks, 256, 0, st>>>(a->d_part, groups, n_cap, n_dev, d);
        if (sbp_cuda_check(cudaGetLastError(), "adjoint: reduce launch")) return SBP_ERR_CUDA;
    }
    return SBP_OK;
}
