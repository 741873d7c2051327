// Zero-gradient filtering (Section 4.2, Algorithm 1), adaptive growth
// (destroy / split / duplicate; Section 4.1, Algorithm 1) and the Adam step.
//
// Filtering and growth are one stable expansion: every input ball maps to 0,
// 1 or 2 output balls; a block-local scan of those counts (warp shuffles)
// plus a scan of the block totals gives each ball its output offset, the
// balls, gradients and carried arrays are scattered into library scratch and
// copied back in place, and the new count is written to n_dev on the device.
//   fg_count    per-block totals of the output counts
//   fg_scan     exclusive scan of the block totals, capacity check
//   fg_scatter  writes the outputs at their offsets
//   fg_copy     copies the outputs back and publishes the new count
#include <algorithm>
#include <cmath>
#include <cstring>

#include "sbp_internal.cuh"

namespace {

constexpr int kFgThreads = 256;
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

struct FgArrays {
    float* a[SBP_FG_ARRAYS];  // x, y, z, R, p0, gx, gy, gz, gR, gp0, extra...
    int count;                // 10 + n_extra
};

struct FgRule {
    int mode;
    sbp_grow_params gp;
};

__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Unit direction of ball i: SplitMix64 outputs 3i, 3i+1, 3i+2 of the stream
// seeded with `seed`, top 24 bits each, mapped to odd lattice points of
// (-1, 1) and normalised.
__device__ __forceinline__ float3 split_dir(uint64_t seed, int i) {
    float g[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const uint64_t u = sm64_mix(seed + (uint64_t)(3 * (long long)i + r + 1) * kGolden) >> 40;
        const int k = 2 * (int)u + 1 - 16777216;
        g[r] = (float)k * (1.0f / 16777216.0f);
    }
    const float inv = 1.0f / sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    return make_float3(g[0] * inv, g[1] * inv, g[2] * inv);
}

// 0 = drop, 1 = keep, 2 = split into two, 3 = keep and duplicate. `local`
// is the ball's index within its frame (the rules do not depend on it).
__device__ __forceinline__ int fg_action(const FgArrays& A, const FgRule& r, int i, int local) {
    (void)local;
    if (r.mode != SBP_GROW) {
        const float g = A.a[9][i];
        if (r.mode == SBP_KEEP_NEG) return g < 0.0f ? 1 : 0;
        if (r.mode == SBP_KEEP_NONPOS) return g <= 0.0f ? 1 : 0;
        return g != 0.0f ? 1 : 0;  // SBP_DROP_ZERO
    }
    const sbp_grow_params& gp = r.gp;
    if (gp.prune_zero) {
        bool any = false, all_zero = true;
        if (gp.grad_mask & SBP_MASK_XYZ) {
            any = true;
            all_zero = all_zero && A.a[5][i] == 0.0f && A.a[6][i] == 0.0f && A.a[7][i] == 0.0f;
        }
        if (gp.grad_mask & SBP_MASK_R) {
            any = true;
            all_zero = all_zero && A.a[8][i] == 0.0f;
        }
        if (gp.grad_mask & SBP_MASK_P0) {
            any = true;
            all_zero = all_zero && A.a[9][i] == 0.0f;
        }
        if (any && all_zero) return 0;
    }
    const float R = A.a[3][i], p0 = A.a[4][i];
    if (gp.destroy && (p0 < gp.p_min || R < gp.R_min)) return 0;
    if (gp.split && R > gp.R_max) return 2;
    if (gp.duplicate) {
        const double gx = A.a[5][i], gy = A.a[6][i], gz = A.a[7][i];
        const double t = (double)gp.g_dup;
        if (gx * gx + gy * gy + gz * gz > t * t) return 3;
    }
    return 1;
}

__device__ __forceinline__ int fg_out_count(int act) { return act == 0 ? 0 : (act == 1 ? 1 : 2); }

// exclusive block scan of small non-negative ints; returns the exclusive
// prefix and the block total
__device__ __forceinline__ int fg_block_excl_scan(int v, int* warp_tot, int& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    total = warp_tot[nw - 1];
    const int off = wid > 0 ? warp_tot[wid - 1] : 0;
    __syncthreads();
    return x - v + off;
}

// Every block of kFgThreads balls lies inside one frame (frame capacities are
// multiples of SBP_FRAME_ALIGN). Counts and offsets are per frame; n_new[f]
// receives frame f's new count, or -1 when it would exceed its capacity.
__global__ void __launch_bounds__(kFgThreads)
fg_count_kernel(FgArrays A, FgRule r, FrameTable ft, int* block_tot) {
    __shared__ int warp_tot[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const FrameSlot fs = sbp_frame_of(ft, blockIdx.x * blockDim.x);
    const int c = i < fs.end ? fg_out_count(fg_action(A, r, i, i - fs.off)) : 0;
    int tot;
    fg_block_excl_scan(c, warp_tot, tot);
    if (threadIdx.x == 0) block_tot[blockIdx.x] = tot;
}

// One CTA per frame: exclusive scan of the frame's block totals.
__global__ void fg_scan_kernel(int* block_tot, FrameTable ft, int* n_new, SbpDevState* st) {
    __shared__ int warp_tot[32];
    const int f = blockIdx.x;
    const int off = ft.ball_off ? ft.ball_off[f] : 0;
    const int cap = ft.ball_off ? ft.ball_off[f + 1] - off : ft.n_cap;
    const int b0 = off / kFgThreads, nblocks = (cap + kFgThreads - 1) / kFgThreads;
    int carry = 0;
    for (int base = 0; base < nblocks; base += blockDim.x) {
        const int b = base + threadIdx.x;
        const int v = b < nblocks ? block_tot[b0 + b] : 0;
        int tot;
        const int ex = fg_block_excl_scan(v, warp_tot, tot);
        if (b < nblocks) block_tot[b0 + b] = ex + carry;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        if (carry > cap) {
            n_new[f] = -1;
            sbp_latch(st, SBP_ERR_CAPACITY);
        } else {
            n_new[f] = carry;
        }
    }
}

__global__ void __launch_bounds__(kFgThreads)
fg_scatter_kernel(FgArrays A, FgRule r, FrameTable ft, const int* block_off, const int* n_new,
                  int total_cap, float* __restrict__ buf) {
    __shared__ int warp_tot[32];
    const FrameSlot fs = sbp_frame_of(ft, blockIdx.x * blockDim.x);
    if (n_new[fs.f] < 0) return;  // uniform: capacity exceeded, leave the frame as is
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int act = i < fs.end ? fg_action(A, r, i, i - fs.off) : 0;
    int tot;
    const int pos =
        fs.off + block_off[blockIdx.x] + fg_block_excl_scan(fg_out_count(act), warp_tot, tot);
    if (act == 0) return;
    const size_t cap = (size_t)total_cap;
    if (act == 1 || act == 3) {
        for (int k = 0; k < A.count; ++k) buf[k * cap + pos] = A.a[k][i];
    }
    if (act == 2 || act == 3) {
        const float x = A.a[0][i], y = A.a[1][i], z = A.a[2][i], R = A.a[3][i], p0 = A.a[4][i];
        const float3 v = split_dir(r.gp.seed, i - fs.off);  // index within the frame
        const float hr = 0.5f * R;
        if (act == 2) {
            const float Rc = R * 0.793700525984099737f;  // 2^(-1/3)
            buf[0 * cap + pos] = x + hr * v.x;
            buf[1 * cap + pos] = y + hr * v.y;
            buf[2 * cap + pos] = z + hr * v.z;
            buf[3 * cap + pos] = Rc;
            buf[4 * cap + pos] = p0;
            buf[0 * cap + pos + 1] = x - hr * v.x;
            buf[1 * cap + pos + 1] = y - hr * v.y;
            buf[2 * cap + pos + 1] = z - hr * v.z;
            buf[3 * cap + pos + 1] = Rc;
            buf[4 * cap + pos + 1] = p0;
            for (int k = 5; k < A.count; ++k) {
                buf[k * cap + pos] = 0.0f;
                buf[k * cap + pos + 1] = 0.0f;
            }
        } else {
            buf[0 * cap + pos + 1] = x + hr * v.x;
            buf[1 * cap + pos + 1] = y + hr * v.y;
            buf[2 * cap + pos + 1] = z + hr * v.z;
            buf[3 * cap + pos + 1] = R;
            buf[4 * cap + pos + 1] = p0;
            for (int k = 5; k < A.count; ++k) buf[k * cap + pos + 1] = 0.0f;
        }
    }
}

// grid.y = frame: copies the frame's outputs back and publishes its count.
__global__ void fg_copy_kernel(FgArrays A, FrameTable ft, int total_cap,
                               const float* __restrict__ buf, const int* n_new, int* n_dev) {
    const int f = blockIdx.y;
    const int nn = n_new[f];
    if (nn < 0) return;
    const int off = ft.ball_off ? ft.ball_off[f] : 0;
    const size_t cap = (size_t)total_cap;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x)
        for (int k = 0; k < A.count; ++k) A.a[k][off + i] = buf[k * cap + off + i];
    if (blockIdx.x == 0 && threadIdx.x == 0) n_dev[f] = nn;
}

struct AdamArgs {
    float* p[5];
    const float* g[5];
    float* m[5];
    float* v[5];
    float lr[5];
    float b1, b2, eps, c1, c2;
    unsigned mask;
};

// grid.y = frame
__global__ void adam_kernel(AdamArgs a, FrameTable ft) {
    const FrameSlot fs = sbp_frame_of(ft, ft.ball_off ? ft.ball_off[blockIdx.y] : 0);
    for (int i = fs.off + blockIdx.x * blockDim.x + threadIdx.x; i < fs.end;
         i += gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const unsigned bit = k < 3 ? SBP_MASK_XYZ : (k == 3 ? SBP_MASK_R : SBP_MASK_P0);
            if (!(a.mask & bit)) continue;
            float g = a.g[k][i];
            const bool sp = k == 3 && (a.mask & SBP_SOFTPLUS_R);
            float p = a.p[k][i];
            float u = p;
            if (sp) {
                // a = softplus^-1(R) = R + log(1 - exp(-R)); sigma(a) = 1 - exp(-R)
                p = fmaxf(p, 1e-30f);
                const float em = expf(-p);
                g *= 1.0f - em;
                u = p + log1pf(-em);
            }
            const float m = a.b1 * a.m[k][i] + (1.0f - a.b1) * g;
            const float v = a.b2 * a.v[k][i] + (1.0f - a.b2) * g * g;
            a.m[k][i] = m;
            a.v[k][i] = v;
            u -= a.lr[k] * (m / a.c1) / (sqrtf(v / a.c2) + a.eps);
            if (sp) u = fmaxf(u, 0.0f) + log1pf(expf(-fabsf(u)));  // softplus
            a.p[k][i] = u;
        }
    }
}

}  // namespace

namespace {

int launch_filter_grow(sbp_array_s* a, sbp_balls balls, sbp_grads grads, float* const* extra,
                       int n_extra, const FrameTable& ft, int total_cap, int* n_dev, int* n_new,
                       const sbp_grow_params* gp, int mode, cudaStream_t st) {
    FgArrays A;
    A.a[0] = balls.x;
    A.a[1] = balls.y;
    A.a[2] = balls.z;
    A.a[3] = balls.R;
    A.a[4] = balls.p0;
    A.a[5] = grads.gx;
    A.a[6] = grads.gy;
    A.a[7] = grads.gz;
    A.a[8] = grads.gR;
    A.a[9] = grads.gp0;
    for (int e = 0; e < n_extra; ++e) A.a[10 + e] = extra[e];
    A.count = 10 + n_extra;
    FgRule r;
    r.mode = mode;
    if (gp) r.gp = *gp;
    else memset(&r.gp, 0, sizeof(r.gp));
    const int blocks = (total_cap + kFgThreads - 1) / kFgThreads;
    if (blocks > a->fg_blocks) {
        sbp_set_error("filter_grow: capacity exceeds the array's capacity");
        return SBP_ERR_ARG;
    }
    fg_count_kernel<<<blocks, kFgThreads, 0, st>>>(A, r, ft, a->d_fg_counts);
    fg_scan_kernel<<<ft.F, 1024, 0, st>>>(a->d_fg_counts, ft, n_new, a->d_state);
    fg_scatter_kernel<<<blocks, kFgThreads, 0, st>>>(A, r, ft, a->d_fg_counts, n_new, total_cap,
                                                     a->d_fg_buf);
    const int per_frame = std::max(1, total_cap / ft.F);
    const int cblocks =
        std::max(1, std::min(std::max(1, 4 * a->sm_count / ft.F), (per_frame + 255) / 256));
    fg_copy_kernel<<<dim3(cblocks, ft.F), 256, 0, st>>>(A, ft, total_cap, a->d_fg_buf, n_new,
                                                        n_dev);
    sbp_count_launches(4);
    return sbp_cuda_check(cudaGetLastError(), "filter_grow launch") ? SBP_ERR_CUDA : SBP_OK;
}

int launch_adam(sbp_array_s* a, sbp_balls balls, sbp_grads grads, sbp_balls m, sbp_balls v,
                const FrameTable& ft, int per_frame_cap, int t, const sbp_adam_params* ap,
                unsigned mask, cudaStream_t st) {
    AdamArgs x;
    float* P[5] = {balls.x, balls.y, balls.z, balls.R, balls.p0};
    const float* Gr[5] = {grads.gx, grads.gy, grads.gz, grads.gR, grads.gp0};
    float* Mm[5] = {m.x, m.y, m.z, m.R, m.p0};
    float* Vv[5] = {v.x, v.y, v.z, v.R, v.p0};
    for (int k = 0; k < 5; ++k) {
        x.p[k] = P[k];
        x.g[k] = Gr[k];
        x.m[k] = Mm[k];
        x.v[k] = Vv[k];
        x.lr[k] = ap->lr[k];
    }
    x.b1 = ap->beta1;
    x.b2 = ap->beta2;
    x.eps = ap->eps;
    x.c1 = (float)(1.0 - pow((double)ap->beta1, (double)t));
    x.c2 = (float)(1.0 - pow((double)ap->beta2, (double)t));
    x.mask = mask;
    const int blocks =
        std::max(1, std::min(std::max(1, 4 * a->sm_count / ft.F), (per_frame_cap + 255) / 256));
    adam_kernel<<<dim3(blocks, ft.F), 256, 0, st>>>(x, ft);
    sbp_count_launches(1);
    return sbp_cuda_check(cudaGetLastError(), "adam launch") ? SBP_ERR_CUDA : SBP_OK;
}

}  // namespace

int sbp_launch_filter_grow(sbp_array_s* a, sbp_balls balls, sbp_grads grads,
                           float* const* extra, int n_extra, int* n_dev, int n_cap,
                           const sbp_grow_params* gp, int mode, cudaStream_t st) {
    const FrameTable ft{1, nullptr, n_dev, n_cap};
    return launch_filter_grow(a, balls, grads, extra, n_extra, ft, n_cap, n_dev,
                              &a->d_state->n_new, gp, mode, st);
}

int sbp_launch_filter_grow_frames(sbp_array_s* a, sbp_balls balls, sbp_grads grads,
                                  float* const* extra, int n_extra, int* n_dev,
                                  const sbp_grow_params* gp, int mode, cudaStream_t st) {
    const int total = a->h_frame_off[a->frames];
    const FrameTable ft{a->frames, a->d_frame_off, n_dev, total};
    return launch_filter_grow(a, balls, grads, extra, n_extra, ft, total, n_dev,
                              a->d_frame_n_new, gp, mode, st);
}

int sbp_launch_adam(sbp_array_s* a, sbp_balls balls, sbp_grads grads, sbp_balls m,
                    sbp_balls v, const int* n_dev, int n_cap, int t,
                    const sbp_adam_params* ap, unsigned mask, cudaStream_t st) {
    const FrameTable ft{1, nullptr, n_dev, n_cap};
    return launch_adam(a, balls, grads, m, v, ft, n_cap, t, ap, mask, st);
}

int sbp_launch_adam_frames(sbp_array_s* a, sbp_balls balls, sbp_grads grads, sbp_balls m,
                           sbp_balls v, const int* n_dev, int t, const sbp_adam_params* ap,
                           unsigned mask, cudaStream_t st) {
    const int total = a->h_frame_off[a->frames];
    const FrameTable ft{a->frames, a->d_frame_off, n_dev, total};
    return launch_adam(a, balls, grads, m, v, ft, total / a->frames, t, ap, mask, st);
}
