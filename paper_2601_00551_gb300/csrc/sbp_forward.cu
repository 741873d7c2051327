// Forward radiator (the "Simulate" step of Sections 4.2-4.3): renders every
// (sensor, ball) pair's cell-averaged N-wave into the sensor traces.
//
// Per pair the trace is, cell by cell (b_j = d - j h, h = c dt_k, K = p0 w / (4 d h)):
//   first touched cell  jL-1 :  a  = K (R^2 - b_jL^2)
//   interior cells jL+n       :  D1 + n D2,   D1 = K h (2 b_jL - h),  D2 = -2 K h^2
//   last cell           jH   :  e  = -K (R^2 - b_jH^2)
// where jL..jH are the cell boundaries strictly inside the support |b| < R.
// This is the closed form E(e_a)^2 - E(e_b)^2 of the cell average with the
// clamp resolved: every interior cell has both boundaries inside the support,
// so its value is linear in j. A linear run has a second difference that is
// zero except at its ends, so each pair is written as at most six integer
// impulses of the second difference (positions jL-1, jL, jL+1, jH, jH+1,
// jH+2) and the trace is recovered by two inclusive prefix sums. The four
// coefficients are rounded to fixed point (2^-F units) and every later
// operation is exact integer arithmetic, so the traces do not depend on the
// order in which pairs are accumulated: the forward is bitwise deterministic.
//
// Kernels:
//   fwd_pmax      max |p0| over the cloud (chooses F so sums cannot overflow)
//   fwd_accum     CTA = (tile of ST sensors) x (chunk of balls); impulses go to
//                 per-sensor shared-memory accumulators with shared atomics,
//                 flushed once per CTA to global memory with global atomics
//   fwd_finalize  CTA = one sensor; two block scans turn impulses into the
//                 float32 trace and clear the accumulator row
#include <algorithm>

#include "sbp_internal.cuh"
#include "sbp_scan.cuh"

namespace {

constexpr int kAccumThreads = 256;
constexpr int kFinalizeThreads = 1024;
constexpr int kFracHeadroomBits = 38;  // F = 38 - ceil(log2 max|p0|)

__global__ void fwd_pmax_kernel(const float* __restrict__ p0, const int* n_dev, int n_cap,
                                SbpDevState* st) {
    const int n = sbp_read_n(n_dev, n_cap);
    float m = 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(p0[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(&st->pmax_bits, __float_as_uint(m));
}

// Fixed-point exponent F: values are stored as round(v * 2^F).
__device__ __forceinline__ int fwd_frac_bits(const SbpDevState* st) {
    const float pm = __uint_as_float(st->pmax_bits);
    int e = 0;
    if (pm > 0.0f) frexpf(pm, &e);  // pm < 2^e
    int F = kFracHeadroomBits - e;
    return F < 0 ? 0 : (F > 60 ? 60 : F);
}

__global__ void __launch_bounds__(kAccumThreads)
fwd_accum_kernel(BallsDev b, const int* n_dev, int n_cap, const float* __restrict__ sens,
                 LevelGeo g, int ST, int n_chunks, SbpDevState* st,
                 unsigned long long* __restrict__ acc) {
    extern __shared__ unsigned long long sacc[];  // [ST][Tk]
    __shared__ float s_sens[8][6];
    const int Tk = g.Tk, M = g.M;
    const int m0 = blockIdx.x * ST;
    const int ns = min(ST, M - m0);
    for (int t = threadIdx.x; t < ST * Tk; t += blockDim.x) sacc[t] = 0ull;
    if (threadIdx.x < ns * 6) {
        const int s = threadIdx.x / 6, k = threadIdx.x % 6;
        s_sens[s][k] = sens[k * M + m0 + s];
    }
    __syncthreads();

    const int n = sbp_read_n(n_dev, n_cap);
    const int chunk = (n + n_chunks - 1) / n_chunks;
    const int c0 = blockIdx.y * chunk;
    const int len = max(0, min(n, c0 + chunk) - c0);
    const float scale = __int_as_float((127 + fwd_frac_bits(st)) << 23);  // 2^F
    const float h = g.h_hi;
    const float d2c = -2.0f * h * h;
    // Lanes of a warp take balls len/32 apart so that a spatially sorted
    // cloud does not send a whole warp's impulses to the same few cells.
    const int cols = (len + 31) >> 5;
    const int slots = cols << 5;
    unsigned int inside = 0;
    for (int slot = threadIdx.x; slot < slots; slot += blockDim.x) {
        const int r = slot & 31, col = slot >> 5;
        const int off = r * cols + col;
        if (off >= len) continue;
        const int i = c0 + off;
        const float cx = __ldg(b.x + i), cy = __ldg(b.y + i), cz = __ldg(b.z + i);
        const float R = __ldg(b.R + i), p0 = __ldg(b.p0 + i);
        if (p0 == 0.0f) continue;
#pragma unroll 1
        for (int s = 0; s < ns; ++s) {
            const PairDist pd =
                sbp_pair_distance(cx, cy, cz, s_sens[s][0], s_sens[s][1], s_sens[s][2]);
            if (!(pd.dh + pd.dl > R)) {
                ++inside;
                continue;
            }
            PairWindow win;
            if (!sbp_window(pd, R, g, true, win)) continue;
            const int jL = win.jL, jH = win.jH;
            const float cosv =
                (s_sens[s][3] * pd.dx + s_sens[s][4] * pd.dy + s_sens[s][5] * pd.dz) * pd.rd;
            float act;
            const float w = sbp_weight(g.wmode, cosv, act);
            if (w == 0.0f) continue;
            const float b0 = win.b0, bL = win.bL;
            const float K = p0 * w * g.inv_4h * pd.rd;
            const float Ks = K * scale;
            const long long qa = __float2ll_rn(Ks * fmaxf(R - b0, 0.0f) * (R + b0));
            const long long qe = -__float2ll_rn(Ks * fmaxf(R + bL, 0.0f) * (R - bL));
            const long long q1 = __float2ll_rn(Ks * h * (2.0f * b0 - h));
            const long long q2 = __float2ll_rn(Ks * d2c);
            const long long L = jH - jL;
            unsigned long long* row = sacc + s * Tk;
            // second difference of the pair's cell values (valid for every L >= 0;
            // for L < 2 some positions coincide and the impulses add up)
            const long long imp[6] = {qa, q1 - 2 * qa, qa - q1 + q2,
                                      qe - q1 - L * q2, q1 + (L - 1) * q2 - 2 * qe, qe};
            const int pos[6] = {jL - 1, jL, jL + 1, jH, jH + 1, jH + 2};
#pragma unroll
            for (int q = 0; q < 6; ++q)
                if (pos[q] < Tk && imp[q] != 0)
                    atomicAdd(row + pos[q], (unsigned long long)imp[q]);
        }
    }
    if (inside) atomicAdd(&st->inside_pairs, (unsigned long long)inside);
    __syncthreads();
    for (int t = threadIdx.x; t < ns * Tk; t += blockDim.x) {
        const unsigned long long v = sacc[t];
        if (v) atomicAdd(acc + (size_t)(m0 + t / Tk) * Tk + (t % Tk), v);
    }
}

// One CTA per sensor: S = 2^-F * P(P(D)), then clear the accumulator row.
__global__ void __launch_bounds__(kFinalizeThreads)
fwd_finalize_kernel(unsigned long long* __restrict__ acc, int Tk, const SbpDevState* st,
                    float* __restrict__ S) {
    __shared__ long long warp_tot[32];
    const int m = blockIdx.x;
    unsigned long long* row = acc + (size_t)m * Tk;
    float* out = S + (size_t)m * Tk;
    const float inv = __int_as_float((127 - fwd_frac_bits(st)) << 23);  // 2^-F
    long long carry1 = 0, carry2 = 0;
    constexpr int IPT = 4;
    const int tile = blockDim.x * IPT;
    for (int base = 0; base < Tk; base += tile) {
        long long v[IPT];
        const int i0 = base + threadIdx.x * IPT;
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            const int i = i0 + q;
            v[q] = i < Tk ? (long long)row[i] : 0;
        }
        // first prefix sum
        long long run = 0;
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            run += v[q];
            v[q] = run;
        }
        long long tot;
        long long incl = sbp_block_incl_scan(run, warp_tot, tot);
        long long off = incl - run + carry1;
#pragma unroll
        for (int q = 0; q < IPT; ++q) v[q] += off;
        carry1 += tot;
        // second prefix sum
        run = 0;
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            run += v[q];
            v[q] = run;
        }
        incl = sbp_block_incl_scan(run, warp_tot, tot);
        off = incl - run + carry2;
        carry2 += tot;
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            const int i = i0 + q;
            if (i < Tk) {
                out[i] = __ll2float_rn(v[q] + off) * inv;
                row[i] = 0ull;
            }
        }
    }
}

}  // namespace

int sbp_launch_forward(sbp_array_s* a, const BallsDev& b, const int* n_dev, int n_cap,
                       float* S, cudaStream_t st) {
    const LevelGeo g = sbp_level_geo(a, a->level);
    const int Tk = g.Tk;
    // sensors per CTA: as many traces as fit in ~96 KB of shared memory, at most 8
    const size_t row_bytes = (size_t)Tk * sizeof(unsigned long long);
    int ST = (int)std::max<size_t>(1, std::min<size_t>(8, (96u * 1024u) / row_bytes));
    if ((size_t)ST * row_bytes > 200u * 1024u) {
        sbp_set_error("forward: a trace of T_k samples does not fit in shared memory");
        return SBP_ERR_ARG;
    }
    const int tiles = (g.M + ST - 1) / ST;
    // enough CTAs for ~4 waves at 2 CTAs per SM, chunks of at least 512 balls
    const int want = 8 * a->sm_count;
    int chunks = std::max(1, (want + tiles - 1) / tiles);
    chunks = std::min(chunks, std::max(1, (n_cap + 511) / 512));
    const size_t smem = (size_t)ST * row_bytes;
    if (sbp_cuda_check(cudaFuncSetAttribute(fwd_accum_kernel,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem),
                       "forward: smem attribute"))
        return SBP_ERR_CUDA;
    if (sbp_cuda_check(cudaMemsetAsync(&a->d_state->pmax_bits, 0, sizeof(unsigned int), st),
                       "forward: reset pmax"))
        return SBP_ERR_CUDA;
    fwd_pmax_kernel<<<std::max(1, std::min(4 * a->sm_count, (n_cap + 255) / 256)), 256, 0,
                      st>>>(b.p0, n_dev, n_cap, a->d_state);
    if (sbp_cuda_check(cudaGetLastError(), "forward: pmax launch")) return SBP_ERR_CUDA;
    dim3 grid(tiles, chunks);
    fwd_accum_kernel<<<grid, kAccumThreads, smem, st>>>(b, n_dev, n_cap, a->d_sens, g, ST,
                                                        chunks, a->d_state, a->d_acc);
    if (sbp_cuda_check(cudaGetLastError(), "forward: accumulate launch")) return SBP_ERR_CUDA;
    fwd_finalize_kernel<<<g.M, kFinalizeThreads, 0, st>>>(a->d_acc, Tk, a->d_state, S);
    if (sbp_cuda_check(cudaGetLastError(), "forward: finalize launch")) return SBP_ERR_CUDA;
    return SBP_OK;
}
