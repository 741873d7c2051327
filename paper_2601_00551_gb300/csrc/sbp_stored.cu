// Stored-window adjoint: the alternative to recomputing each pair's geometry
// in the backward pass (the backpropagation step of Algorithm 1). The
// forward pass then also writes, for every (sensor, ball) pair, the window
// and the factors the adjoint needs; the adjoint reads them back instead of
// evaluating the distance, the window and the orientation weight again.
// It exists to measure that trade: memory of 20 bytes per pair (about 2 GB
// for 200k balls x 512 sensors) against the recomputing adjoint, which
// keeps nothing but the cloud.
//
// Record of pair (m, i), five planes of [M][n_cap] (structure of arrays, so
// that consecutive balls of one sensor are consecutive words):
//   b0   float  offset of the first boundary inside the support, b_jL
//   w    float  orientation weight (0 when the pair does not count)
//   rd   float  ~1 / d
//   jL   int    first boundary inside the support; -1: the pair adds nothing
//   jHa  int    last boundary jH, with bit 31 set when dw/dc is non-zero
// The window comes from the same float-float distance and window helpers as
// the forward and the recomputing adjoint, so the three agree pair by pair.
//
// Kernels:
//   store_windows   one thread per (sensor, two consecutive balls)
//   adjoint_stored  one thread per ball, over every sensor: the window sums
//                   of G read from global memory (one pair at a time), then
//                   the same chain rule as the recomputing adjoint; each
//                   gradient written once.
#include <algorithm>

#include "sbp_internal.cuh"

namespace {

constexpr int kStoreThreads = 256;
constexpr int kAdjStoredThreads = 128;

struct StoredGradOut {
    float* o[5];  // x, y, z, R, p0
};

struct WindowRec {
    float* b0;
    float* w;
    float* rd;
    int* jL;
    int* jHa;
};

template <int WMODE>
__global__ void __launch_bounds__(kStoreThreads)
store_windows_kernel(BallsDev b, const int* n_dev, int n_cap, const float* __restrict__ sens,
                     LevelGeo g, WindowRec rec) {
    const int n = sbp_read_n(n_dev, n_cap);
    const int m = blockIdx.y;
    const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= n_cap) return;
    const int M = g.M;
    const float sx = sens[m], sy = sens[M + m], sz = sens[2 * M + m];
    const float nx = sens[3 * M + m], ny = sens[4 * M + m], nz = sens[5 * M + m];
    const bool hasA = i < n, hasB = i + 1 < n && i + 1 < n_cap;
    const float2 cx = make_float2(hasA ? b.x[i] : 0.f, hasB ? b.x[i + 1] : 0.f);
    const float2 cy = make_float2(hasA ? b.y[i] : 0.f, hasB ? b.y[i + 1] : 0.f);
    const float2 cz = make_float2(hasA ? b.z[i] : 0.f, hasB ? b.z[i + 1] : 0.f);
    const float2 R2 = make_float2(hasA ? b.R[i] : 0.f, hasB ? b.R[i + 1] : 0.f);
    const PairDist2 pd = sbp_pair_distance2(cx, cy, cz, f2(sx), f2(sy), f2(sz));
    PairWindow wa, wb;
    bool okA, okB;
    sbp_window2(pd.dh, pd.dl, R2, g, wa, wb, okA, okB);
    const float2 cosv = f2mul(
        f2fma(f2(nx), pd.dx, f2fma(f2(ny), pd.dy, f2mul(f2(nz), pd.dz))), pd.rd);
    float actA, actB;
    const float wA = sbp_weight(WMODE, cosv.x, actA), wB = sbp_weight(WMODE, cosv.y, actB);
    // the recomputing adjoint's test: a pair counts unless its weight and the
    // weight's derivative both vanish (p0 plays no part in the window)
    okA = hasA && okA && !(wA == 0.0f && actA == 0.0f);
    okB = hasB && okB && !(wB == 0.0f && actB == 0.0f);
    const size_t p = (size_t)m * n_cap + i;
    rec.b0[p] = okA ? wa.b0 : 0.0f;
    rec.w[p] = okA ? wA : 0.0f;
    rec.rd[p] = pd.rd.x;
    rec.jL[p] = okA ? wa.jL : -1;
    rec.jHa[p] = okA ? (wa.jH | (actA != 0.0f ? (int)0x80000000u : 0)) : 0;
    if (i + 1 < n_cap) {
        rec.b0[p + 1] = okB ? wb.b0 : 0.0f;
        rec.w[p + 1] = okB ? wB : 0.0f;
        rec.rd[p + 1] = pd.rd.y;
        rec.jL[p + 1] = okB ? wb.jL : -1;
        rec.jHa[p + 1] = okB ? (wb.jH | (actB != 0.0f ? (int)0x80000000u : 0)) : 0;
    }
}

template <bool P0_ONLY>
__global__ void __launch_bounds__(kAdjStoredThreads)
adjoint_stored_kernel(BallsDev b, const int* n_dev, int n_cap, const float* __restrict__ sens,
                      LevelGeo g, const float* __restrict__ G, WindowRec rec, unsigned mask,
                      StoredGradOut out) {
    const int n = sbp_read_n(n_dev, n_cap);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gx = 0.f, gy = 0.f, gz = 0.f, gR = 0.f, gp = 0.f;
    {
        const float cx = b.x[i], cy = b.y[i], cz = b.z[i], R = b.R[i], p0 = b.p0[i];
        const float h = g.h_hi, hh2 = 2.0f * h * h;
        const int M = g.M, Tk = g.Tk;
        for (int m = 0; m < M; ++m) {
            const size_t p = (size_t)m * n_cap + i;
            const int jL = rec.jL[p];
            if (jL < 0) continue;
            const int jHa = rec.jHa[p];
            const int jH = jHa & 0x7fffffff;
            const float act = jHa < 0 ? 1.0f : 0.0f;
            const float b0 = rec.b0[p], w = rec.w[p], rd = rec.rd[p];
            // window sums against the last cell's value (the recomputing
            // adjoint's form, which sees only differences of G)
            const float* __restrict__ Gm = G + (size_t)m * Tk;
            const int L = min(jH, Tk) - jL;
            const float gf = Gm[jL - 1];
            const float gl = jH < Tk ? Gm[jH] : 0.0f;
            float E0 = 0.f, E1 = 0.f;
            for (int q = 0; q < L; ++q) {
                const float d = Gm[jL + q] - gl;
                E0 += d;
                E1 = fmaf((float)q, d, E1);
            }
            const float Df = gf - gl;
            const float ra = fmaxf(R - b0, 0.0f);
            const float A = fmaf(Df * ra, R + b0, fmaf(E0 * h, fmaf(2.0f, b0, -h), -hh2 * E1));
            const float qd = g.inv_4h * rd;  // 1 / (4 d h)
            const float K0 = w * qd;
            gp = fmaf(K0, A, gp);
            if (P0_ONLY) continue;
            const float Bh = fmaf(h, E0, -(b0 * Df));
            const float pK = p0 * K0;
            gR = fmaf(pK * (2.0f * R), Df, gR);
            const float gd = pK * fmaf(2.0f, Bh, -(A * rd));
            const float gwr = p0 * A * qd * act * rd;
            // the unit vector from the sensor to the centre and n . u
            const float sx = sens[m], sy = sens[M + m], sz = sens[2 * M + m];
            const float nx = sens[3 * M + m], ny = sens[4 * M + m], nz = sens[5 * M + m];
            const float ux = (cx - sx) * rd, uy = (cy - sy) * rd, uz = (cz - sz) * rd;
            const float cosv = fmaf(nx, ux, fmaf(ny, uy, nz * uz));
            gx = fmaf(gd, ux, fmaf(gwr, fmaf(-cosv, ux, nx), gx));
            gy = fmaf(gd, uy, fmaf(gwr, fmaf(-cosv, uy, ny), gy));
            gz = fmaf(gd, uz, fmaf(gwr, fmaf(-cosv, uz, nz), gz));
        }
    }
    // every live ball's components written once; those outside the mask as zero
    out.o[0][i] = (mask & SBP_MASK_XYZ) ? gx : 0.0f;
    out.o[1][i] = (mask & SBP_MASK_XYZ) ? gy : 0.0f;
    out.o[2][i] = (mask & SBP_MASK_XYZ) ? gz : 0.0f;
    out.o[3][i] = (mask & SBP_MASK_R) ? gR : 0.0f;
    out.o[4][i] = (mask & SBP_MASK_P0) ? gp : 0.0f;
}

WindowRec rec_planes(void* rec_dev, int M, int n_cap) {
    const size_t plane = (size_t)M * n_cap;
    float* f = static_cast<float*>(rec_dev);
    int* k = static_cast<int*>(rec_dev);
    return WindowRec{f, f + plane, f + 2 * plane, k + 3 * plane, k + 4 * plane};
}

}  // namespace

int sbp_launch_store_windows(sbp_array_s* a, const BallsDev& b, const int* n_dev, int n_cap,
                             void* rec_dev, cudaStream_t st) {
    const LevelGeo g = sbp_level_geo(a, a->level);
    const WindowRec rec = rec_planes(rec_dev, g.M, n_cap);
    const dim3 grid((unsigned)((n_cap + 2 * kStoreThreads - 1) / (2 * kStoreThreads)),
                    (unsigned)g.M);
    if (g.wmode == SBP_W_NONE)
        store_windows_kernel<SBP_W_NONE><<<grid, kStoreThreads, 0, st>>>(b, n_dev, n_cap, a->d_sens,
                                                                        g, rec);
    else if (g.wmode == SBP_W_COS)
        store_windows_kernel<SBP_W_COS><<<grid, kStoreThreads, 0, st>>>(b, n_dev, n_cap, a->d_sens,
                                                                       g, rec);
    else
        store_windows_kernel<SBP_W_CLAMP><<<grid, kStoreThreads, 0, st>>>(b, n_dev, n_cap,
                                                                         a->d_sens, g, rec);
    sbp_count_launches(1);
    return sbp_cuda_check(cudaGetLastError(), "store_windows launch") ? SBP_ERR_CUDA : SBP_OK;
}

int sbp_launch_adjoint_stored(sbp_array_s* a, const BallsDev& b, const int* n_dev, int n_cap,
                              const void* rec_dev, const float* G, sbp_grads out, unsigned mask,
                              cudaStream_t st) {
    const LevelGeo g = sbp_level_geo(a, a->level);
    const WindowRec rec = rec_planes(const_cast<void*>(rec_dev), g.M, n_cap);
    StoredGradOut o;
    o.o[0] = out.gx;
    o.o[1] = out.gy;
    o.o[2] = out.gz;
    o.o[3] = out.gR;
    o.o[4] = out.gp0;
    const unsigned grid = (unsigned)((n_cap + kAdjStoredThreads - 1) / kAdjStoredThreads);
    if (mask == SBP_MASK_P0)
        adjoint_stored_kernel<true><<<grid, kAdjStoredThreads, 0, st>>>(b, n_dev, n_cap, a->d_sens,
                                                                       g, G, rec, mask, o);
    else
        adjoint_stored_kernel<false><<<grid, kAdjStoredThreads, 0, st>>>(
            b, n_dev, n_cap, a->d_sens, g, G, rec, mask, o);
    sbp_count_launches(1);
    return sbp_cuda_check(cudaGetLastError(), "adjoint_stored launch") ? SBP_ERR_CUDA : SBP_OK;
}
