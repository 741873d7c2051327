// The reconstruction loop of Algorithm 1 on the device (host orchestration
// only: every step is one of the library's kernels, enqueued on one stream
// with no synchronisation, the ball count staying in device memory).
#include <algorithm>
#include <cstring>

#include "sbp_internal.cuh"

namespace {

int ensure_recon_scratch(sbp_array_s* a) {
    if (a->d_rc_state) return SBP_OK;
    const size_t MT = (size_t)a->M * a->T;
    bool ok = true;
    ok = ok && !sbp_cuda_check(cudaMalloc(&a->d_rc_yk, sizeof(float) * MT), "recon: alloc y_k");
    ok = ok && !sbp_cuda_check(cudaMalloc(&a->d_rc_S, sizeof(float) * MT), "recon: alloc S");
    ok = ok && !sbp_cuda_check(cudaMalloc(&a->d_rc_G, sizeof(float) * MT), "recon: alloc G");
    ok = ok && !sbp_cuda_check(cudaMalloc(&a->d_rc_state, sizeof(float) * 15 * (size_t)a->n_cap),
                               "recon: alloc state");
    return ok ? SBP_OK : SBP_ERR_CUDA;
}

}  // namespace

extern "C" int sbp_reconstruct(sbp_array arr, const float* y_full_dev, sbp_balls balls,
                               int* n_dev, int n_cap, const sbp_recon_params* rp,
                               sbp_stream stream) {
    if (!arr || !rp || !y_full_dev || !n_dev || !balls.x || !balls.y || !balls.z || !balls.R ||
        !balls.p0 || n_cap < 1 || n_cap > arr->n_cap || rp->n_stages < 0 ||
        rp->n_stages > SBP_MAX_STAGES || rp->zero_grad_mode < -1 ||
        rp->zero_grad_mode > SBP_DROP_ZERO) {
        sbp_set_error("reconstruct: invalid argument");
        return SBP_ERR_ARG;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != arr->device) {
        sbp_set_error("reconstruct: the array belongs to another device");
        return SBP_ERR_ARG;
    }
    if (rp->zero_grad_mode >= 0 &&
        (rp->zero_grad_level < 0 || rp->zero_grad_level >= arr->n_levels)) {
        sbp_set_error("reconstruct: zero_grad_level out of range");
        return SBP_ERR_LEVEL;
    }
    for (int s = 0; s < rp->n_stages; ++s) {
        const sbp_stage& st = rp->stages[s];
        if (st.level < 0 || st.level >= arr->n_levels || st.iterations < 0 ||
            (st.grad_mask & ~(SBP_MASK_ALL | SBP_SOFTPLUS_R))) {
            sbp_set_error("reconstruct: invalid stage");
            return SBP_ERR_ARG;
        }
    }
    if (int e = ensure_recon_scratch(arr)) return e;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const size_t cap = (size_t)n_cap;
    float* st = arr->d_rc_state;
    sbp_grads grads{st, st + cap, st + 2 * cap, st + 3 * cap, st + 4 * cap};
    sbp_balls m{st + 5 * cap, st + 6 * cap, st + 7 * cap, st + 8 * cap, st + 9 * cap};
    sbp_balls v{st + 10 * cap, st + 11 * cap, st + 12 * cap, st + 13 * cap, st + 14 * cap};
    float* extra[10] = {m.x, m.y, m.z, m.R, m.p0, v.x, v.y, v.z, v.R, v.p0};
    const BallsDev bd{balls.x, balls.y, balls.z, balls.R, balls.p0};
    if (sbp_cuda_check(cudaMemsetAsync(st, 0, sizeof(float) * 15 * cap, cs),
                       "reconstruct: clear state"))
        return SBP_ERR_CUDA;

    int level = -1;
    auto use_level = [&](int k) -> int {
        if (k == level) return SBP_OK;
        arr->level = k;
        level = k;
        return sbp_launch_downsample(arr, k, y_full_dev, arr->d_rc_yk, cs);
    };

    // spatial ordering of the initial cloud (its moments are still zero)
    if (rp->spatial_sort) {
        float* rows[5] = {balls.x, balls.y, balls.z, balls.R, balls.p0};
        if (int e = sbp_launch_sort(arr, rows, 5, n_dev, n_cap, cs)) return e;
    }
    // zero-gradient filtering (Section 4.2): all p0 = 0, so S = 0 and G = -2 y_k
    if (rp->zero_grad_mode >= 0) {
        if (int e = use_level(rp->zero_grad_level)) return e;
        if (int e = sbp_launch_residual(arr, nullptr, arr->d_rc_yk, arr->d_rc_G, nullptr, cs))
            return e;
        if (int e = sbp_launch_adjoint(arr, bd, n_dev, n_cap, arr->d_rc_G, grads, SBP_MASK_P0,
                                       cs))
            return e;
        if (int e = sbp_launch_filter_grow(arr, balls, grads, extra, 10, n_dev, n_cap, nullptr,
                                           rp->zero_grad_mode, cs))
            return e;
    }

    int t = 0;
    for (int s = 0; s < rp->n_stages; ++s) {
        const sbp_stage& stg = rp->stages[s];
        const unsigned gmask = stg.grad_mask & SBP_MASK_ALL;
        const bool softplus_starts = (stg.grad_mask & SBP_SOFTPLUS_R) &&
                                     !(s > 0 && (rp->stages[s - 1].grad_mask & SBP_SOFTPLUS_R));
        if (softplus_starts) {  // the free variable of the refinement starts with fresh moments
            if (sbp_cuda_check(cudaMemsetAsync(m.R, 0, sizeof(float) * cap, cs),
                               "reconstruct: reset m") ||
                sbp_cuda_check(cudaMemsetAsync(v.R, 0, sizeof(float) * cap, cs),
                               "reconstruct: reset v"))
                return SBP_ERR_CUDA;
        }
        for (int it = 0; it < stg.iterations; ++it) {
            if (int e = use_level(stg.level)) return e;
            if (rp->n_log_dev && t < rp->log_capacity &&
                sbp_cuda_check(cudaMemcpyAsync(rp->n_log_dev + t, n_dev, sizeof(int),
                                               cudaMemcpyDeviceToDevice, cs),
                               "reconstruct: log count"))
                return SBP_ERR_CUDA;
            if (int e = sbp_launch_forward(arr, bd, n_dev, n_cap, arr->d_rc_S, cs)) return e;
            double* loss = (rp->loss_log_dev && t < rp->log_capacity) ? rp->loss_log_dev + t
                                                                       : nullptr;
            if (int e = sbp_launch_residual(arr, arr->d_rc_S, arr->d_rc_yk, arr->d_rc_G, loss,
                                            cs))
                return e;
            if (int e = sbp_launch_adjoint(arr, bd, n_dev, n_cap, arr->d_rc_G, grads, gmask, cs))
                return e;
            ++t;
            if (int e = sbp_launch_adam(arr, balls, grads, m, v, n_dev, n_cap, t, &rp->adam,
                                        stg.grad_mask, cs))
                return e;
            if (stg.grow) {
                sbp_grow_params gp = rp->grow;
                gp.seed = rp->grow.seed + (uint64_t)t;
                gp.grad_mask = (int)gmask;
                gp.duplicate = stg.duplicate;
                if (int e = sbp_launch_filter_grow(arr, balls, grads, extra, 10, n_dev, n_cap, &gp,
                                                   SBP_GROW, cs))
                    return e;
            }
        }
    }
    return SBP_OK;
}
