// Batched reconstruction of many acquisitions (frames) against one sensor
// array: every step of the hot path runs once for all frames, each frame's
// balls in its own slice of one packed cloud and its traces in its own
// [M][T_k] block, so a whole iteration of all frames is a fixed sequence of
// kernel launches with no host round trip (capturable in a CUDA graph).
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "sbp_internal.cuh"

namespace {

bool balls_ok(const sbp_balls& b) { return b.x && b.y && b.z && b.R && b.p0; }
bool grads_ok(const sbp_grads& g) { return g.gx && g.gy && g.gz && g.gR && g.gp0; }

int check_frames(sbp_array a, const char* fn) {
    if (!a) {
        sbp_set_error(std::string(fn) + ": null array");
        return SBP_ERR_ARG;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != a->device) {
        sbp_set_error(std::string(fn) + ": the array belongs to another device");
        return SBP_ERR_ARG;
    }
    if (a->frames < 1 || !a->d_frame_off) {
        sbp_set_error(std::string(fn) + ": no frame layout (call sbp_set_frames first)");
        return SBP_ERR_ARG;
    }
    return SBP_OK;
}

int grow_buffer(float** p, size_t* cells, size_t need, const char* what) {
    if (*p && *cells >= need) return SBP_OK;
    cudaFree(*p);
    *p = nullptr;
    if (sbp_cuda_check(cudaMalloc(p, sizeof(float) * need), what)) return SBP_ERR_CUDA;
    *cells = need;
    return SBP_OK;
}

}  // namespace

extern "C" {

int sbp_set_frames(sbp_array arr, const int* frame_cap_host, int n_frames, int* frame_off_out) {
    if (!arr || !frame_cap_host || n_frames < 1 || n_frames > SBP_MAX_FRAMES) {
        sbp_set_error("set_frames: invalid argument");
        return SBP_ERR_ARG;
    }
    std::vector<int> off(n_frames + 1, 0);
    long long total = 0;
    for (int f = 0; f < n_frames; ++f) {
        if (frame_cap_host[f] < 1) {
            sbp_set_error("set_frames: every frame needs a capacity >= 1");
            return SBP_ERR_ARG;
        }
        total += (frame_cap_host[f] + SBP_FRAME_ALIGN - 1) / SBP_FRAME_ALIGN * SBP_FRAME_ALIGN;
        off[f + 1] = (int)std::min<long long>(total, 0x7fffffff);
    }
    if (total > arr->n_cap) {
        sbp_set_error("set_frames: the padded frame capacities exceed the array's n_cap");
        return SBP_ERR_CAPACITY;
    }
    if (sbp_cuda_check(cudaDeviceSynchronize(), "set_frames: synchronise")) return SBP_ERR_CUDA;
    cudaFree(arr->d_frame_off);
    cudaFree(arr->d_frame_n_new);
    cudaFree(arr->d_frame_lossp);
    cudaFree(arr->d_frame_pmax);
    arr->d_frame_off = nullptr;
    arr->d_frame_n_new = nullptr;
    arr->d_frame_lossp = nullptr;
    arr->d_frame_pmax = nullptr;
    delete[] arr->h_frame_off;
    arr->h_frame_off = new int[n_frames + 1];
    std::copy(off.begin(), off.end(), arr->h_frame_off);
    arr->frames = 0;
    bool ok = true;
    ok = ok && !sbp_cuda_check(cudaMalloc(&arr->d_frame_off, sizeof(int) * (n_frames + 1)),
                               "set_frames: alloc offsets");
    ok = ok && !sbp_cuda_check(cudaMalloc(&arr->d_frame_n_new, sizeof(int) * n_frames),
                               "set_frames: alloc counts");
    ok = ok && !sbp_cuda_check(cudaMalloc(&arr->d_frame_lossp, sizeof(double) * 16 * n_frames),
                               "set_frames: alloc loss partials");
    ok = ok && !sbp_cuda_check(cudaMalloc(&arr->d_frame_pmax, sizeof(unsigned int) * n_frames),
                               "set_frames: alloc scales");
    ok = ok && !sbp_cuda_check(cudaMemcpy(arr->d_frame_off, off.data(),
                                          sizeof(int) * (n_frames + 1), cudaMemcpyHostToDevice),
                               "set_frames: copy offsets");
    const size_t cells = (size_t)n_frames * arr->M * arr->T;
    if (ok && arr->acc_cells < cells) {
        cudaFree(arr->d_acc);
        arr->d_acc = nullptr;
        ok = !sbp_cuda_check(cudaMalloc(&arr->d_acc, sizeof(unsigned long long) * cells),
                             "set_frames: alloc accumulators") &&
             !sbp_cuda_check(cudaMemset(arr->d_acc, 0, sizeof(unsigned long long) * cells),
                             "set_frames: clear accumulators");
        arr->acc_cells = ok ? cells : 0;
    }
    if (!ok) return SBP_ERR_CUDA;
    arr->frames = n_frames;
    if (frame_off_out) std::copy(off.begin(), off.end(), frame_off_out);
    return SBP_OK;
}

int sbp_set_sampling_level_frames(sbp_array arr, int k, const float* y_full_dev, float* y_k_dev,
                                  sbp_stream stream) {
    if (int e = check_frames(arr, "set_sampling_level_frames")) return e;
    if (k < 0 || k >= arr->n_levels) {
        sbp_set_error("set_sampling_level_frames: level out of range");
        return SBP_ERR_LEVEL;
    }
    if (y_full_dev && !y_k_dev) {
        sbp_set_error("set_sampling_level_frames: y_k_dev is null");
        return SBP_ERR_ARG;
    }
    arr->level = k;
    if (!y_full_dev) return SBP_OK;
    return sbp_launch_downsample_rows(arr, k, arr->frames * arr->M, y_full_dev, y_k_dev,
                                      reinterpret_cast<cudaStream_t>(stream));
}

int sbp_forward_frames(sbp_array arr, sbp_balls balls, const int* n_dev, float* S_dev,
                       sbp_stream stream) {
    if (int e = check_frames(arr, "forward_frames")) return e;
    if (!balls_ok(balls) || !n_dev || !S_dev) {
        sbp_set_error("forward_frames: null pointer");
        return SBP_ERR_ARG;
    }
    const BallsDev b{balls.x, balls.y, balls.z, balls.R, balls.p0};
    return sbp_launch_forward_frames(arr, b, n_dev, S_dev, arr->fwd_chunk_frames,
                                     reinterpret_cast<cudaStream_t>(stream));
}

int sbp_residual_frames(sbp_array arr, const float* S_dev, const float* y_k_dev, float* G_dev,
                        double* loss_dev, sbp_stream stream) {
    if (int e = check_frames(arr, "residual_frames")) return e;
    if (!y_k_dev || !G_dev) {
        sbp_set_error("residual_frames: null pointer");
        return SBP_ERR_ARG;
    }
    return sbp_launch_residual_frames(arr, S_dev, y_k_dev, G_dev, loss_dev,
                                      reinterpret_cast<cudaStream_t>(stream));
}

int sbp_adjoint_frames(sbp_array arr, sbp_balls balls, const int* n_dev, const float* G_dev,
                       sbp_grads out, unsigned grad_mask, sbp_stream stream) {
    if (int e = check_frames(arr, "adjoint_frames")) return e;
    if (!balls_ok(balls) || !grads_ok(out) || !n_dev || !G_dev || (grad_mask & ~SBP_MASK_ALL)) {
        sbp_set_error("adjoint_frames: null pointer or unknown mask bit");
        return SBP_ERR_ARG;
    }
    const BallsDev b{balls.x, balls.y, balls.z, balls.R, balls.p0};
    return sbp_launch_adjoint_frames(arr, b, n_dev, G_dev, out, grad_mask,
                                     reinterpret_cast<cudaStream_t>(stream));
}

int sbp_filter_grow_frames(sbp_array arr, sbp_balls balls, sbp_grads grads, float* const* extra,
                           int n_extra, int* n_dev, const sbp_grow_params* gp, int mode,
                           sbp_stream stream) {
    if (int e = check_frames(arr, "filter_grow_frames")) return e;
    if (!balls_ok(balls) || !grads_ok(grads) || !n_dev || n_extra < 0 ||
        n_extra > SBP_MAX_EXTRA || (n_extra > 0 && !extra) || mode < SBP_KEEP_NEG ||
        mode > SBP_GROW || (mode == SBP_GROW && !gp)) {
        sbp_set_error("filter_grow_frames: invalid argument");
        return SBP_ERR_ARG;
    }
    for (int e = 0; e < n_extra; ++e)
        if (!extra[e]) {
            sbp_set_error("filter_grow_frames: null extra array");
            return SBP_ERR_ARG;
        }
    return sbp_launch_filter_grow_frames(arr, balls, grads, extra, n_extra, n_dev, gp, mode,
                                         reinterpret_cast<cudaStream_t>(stream));
}

int sbp_adam_step_frames(sbp_array arr, sbp_balls balls, sbp_grads grads, sbp_balls m,
                         sbp_balls v, const int* n_dev, int t, const sbp_adam_params* ap,
                         unsigned mask, sbp_stream stream) {
    if (int e = check_frames(arr, "adam_step_frames")) return e;
    if (!balls_ok(balls) || !grads_ok(grads) || !balls_ok(m) || !balls_ok(v) || !n_dev || !ap ||
        t < 1 || (mask & ~(SBP_MASK_ALL | SBP_SOFTPLUS_R))) {
        sbp_set_error("adam_step_frames: invalid argument");
        return SBP_ERR_ARG;
    }
    return sbp_launch_adam_frames(arr, balls, grads, m, v, n_dev, t, ap, mask,
                                  reinterpret_cast<cudaStream_t>(stream));
}

int sbp_reconstruct_frames(sbp_array arr, const float* y_full_dev, sbp_balls balls, int* n_dev,
                           const sbp_recon_params* rp, sbp_stream stream) {
    if (int e = check_frames(arr, "reconstruct_frames")) return e;
    if (!rp || !y_full_dev || !n_dev || !balls_ok(balls) || rp->n_stages < 0 ||
        rp->n_stages > SBP_MAX_STAGES || rp->zero_grad_mode < -1 ||
        rp->zero_grad_mode > SBP_DROP_ZERO || rp->spatial_sort != 0) {
        sbp_set_error("reconstruct_frames: invalid argument (spatial_sort is single-cloud only)");
        return SBP_ERR_ARG;
    }
    if (rp->zero_grad_mode >= 0 &&
        (rp->zero_grad_level < 0 || rp->zero_grad_level >= arr->n_levels)) {
        sbp_set_error("reconstruct_frames: zero_grad_level out of range");
        return SBP_ERR_LEVEL;
    }
    for (int s = 0; s < rp->n_stages; ++s) {
        const sbp_stage& st = rp->stages[s];
        if (st.level < 0 || st.level >= arr->n_levels || st.iterations < 0 ||
            (st.grad_mask & ~(SBP_MASK_ALL | SBP_SOFTPLUS_R))) {
            sbp_set_error("reconstruct_frames: invalid stage");
            return SBP_ERR_ARG;
        }
    }
    const int F = arr->frames;
    const size_t cells = (size_t)F * arr->M * arr->T;
    size_t c1 = arr->fr_cells, c2 = arr->fr_cells, c3 = arr->fr_cells;
    if (int e = grow_buffer(&arr->d_fr_yk, &c1, cells, "reconstruct_frames: alloc y_k")) return e;
    if (int e = grow_buffer(&arr->d_fr_S, &c2, cells, "reconstruct_frames: alloc S")) return e;
    if (int e = grow_buffer(&arr->d_fr_G, &c3, cells, "reconstruct_frames: alloc G")) return e;
    arr->fr_cells = std::min(c1, std::min(c2, c3));
    if (!arr->d_rc_state &&
        sbp_cuda_check(cudaMalloc(&arr->d_rc_state, sizeof(float) * 15 * (size_t)arr->n_cap),
                       "reconstruct_frames: alloc state"))
        return SBP_ERR_CUDA;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const size_t cap = (size_t)arr->n_cap;
    float* st = arr->d_rc_state;
    sbp_grads grads{st, st + cap, st + 2 * cap, st + 3 * cap, st + 4 * cap};
    sbp_balls m{st + 5 * cap, st + 6 * cap, st + 7 * cap, st + 8 * cap, st + 9 * cap};
    sbp_balls v{st + 10 * cap, st + 11 * cap, st + 12 * cap, st + 13 * cap, st + 14 * cap};
    float* extra[10] = {m.x, m.y, m.z, m.R, m.p0, v.x, v.y, v.z, v.R, v.p0};
    const BallsDev bd{balls.x, balls.y, balls.z, balls.R, balls.p0};
    if (sbp_cuda_check(cudaMemsetAsync(st, 0, sizeof(float) * 15 * cap, cs),
                       "reconstruct_frames: clear state"))
        return SBP_ERR_CUDA;
    int level = -1;
    auto use_level = [&](int k) -> int {
        if (k == level) return SBP_OK;
        arr->level = k;
        level = k;
        return sbp_launch_downsample_rows(arr, k, F * arr->M, y_full_dev, arr->d_fr_yk, cs);
    };
    if (rp->zero_grad_mode >= 0) {
        if (int e = use_level(rp->zero_grad_level)) return e;
        if (int e = sbp_launch_residual_frames(arr, nullptr, arr->d_fr_yk, arr->d_fr_G, nullptr,
                                               cs))
            return e;
        if (int e = sbp_launch_adjoint_frames(arr, bd, n_dev, arr->d_fr_G, grads, SBP_MASK_P0, cs))
            return e;
        if (int e = sbp_launch_filter_grow_frames(arr, balls, grads, extra, 10, n_dev, nullptr,
                                                  rp->zero_grad_mode, cs))
            return e;
    }
    int t = 0;
    for (int s = 0; s < rp->n_stages; ++s) {
        const sbp_stage& stg = rp->stages[s];
        const unsigned gmask = stg.grad_mask & SBP_MASK_ALL;
        const bool softplus_starts = (stg.grad_mask & SBP_SOFTPLUS_R) &&
                                     !(s > 0 && (rp->stages[s - 1].grad_mask & SBP_SOFTPLUS_R));
        if (softplus_starts) {
            if (sbp_cuda_check(cudaMemsetAsync(m.R, 0, sizeof(float) * cap, cs),
                               "reconstruct_frames: reset m") ||
                sbp_cuda_check(cudaMemsetAsync(v.R, 0, sizeof(float) * cap, cs),
                               "reconstruct_frames: reset v"))
                return SBP_ERR_CUDA;
        }
        for (int it = 0; it < stg.iterations; ++it) {
            if (int e = use_level(stg.level)) return e;
            if (rp->n_log_dev && t < rp->log_capacity &&
                sbp_cuda_check(cudaMemcpyAsync(rp->n_log_dev + (size_t)t * F, n_dev,
                                               sizeof(int) * F, cudaMemcpyDeviceToDevice, cs),
                               "reconstruct_frames: log counts"))
                return SBP_ERR_CUDA;
            if (int e = sbp_launch_forward_frames(arr, bd, n_dev, arr->d_fr_S,
                                                  arr->fwd_chunk_frames, cs))
                return e;
            double* loss = (rp->loss_log_dev && t < rp->log_capacity)
                               ? rp->loss_log_dev + (size_t)t * F
                               : nullptr;
            if (int e = sbp_launch_residual_frames(arr, arr->d_fr_S, arr->d_fr_yk, arr->d_fr_G,
                                                   loss, cs))
                return e;
            if (int e = sbp_launch_adjoint_frames(arr, bd, n_dev, arr->d_fr_G, grads, gmask, cs))
                return e;
            ++t;
            if (int e = sbp_launch_adam_frames(arr, balls, grads, m, v, n_dev, t, &rp->adam,
                                               stg.grad_mask, cs))
                return e;
            if (stg.grow) {
                sbp_grow_params gp = rp->grow;
                gp.seed = rp->grow.seed + (uint64_t)t;
                gp.grad_mask = (int)gmask;
                gp.duplicate = stg.duplicate;
                if (int e = sbp_launch_filter_grow_frames(arr, balls, grads, extra, 10, n_dev,
                                                          &gp, SBP_GROW, cs))
                    return e;
            }
        }
    }
    return SBP_OK;
}

int sbp_set_frame_tiles(sbp_array arr, int fwd_chunk, int adj_split) {
    if (int e = check_frames(arr, "set_frame_tiles")) return e;
    // a chunk must not straddle two frames: at most one alignment unit
    const bool chunk_ok = fwd_chunk == 0 || (sbp_fwd_tile_valid(fwd_chunk) &&
                                             (fwd_chunk & ~SBP_TILE_WIDE) <= SBP_FRAME_ALIGN);
    const bool split_ok = adj_split == 0 || adj_split == 1 || adj_split == 2 || adj_split == 4 ||
                          adj_split == 8;
    if (!chunk_ok || !split_ok) {
        sbp_set_error("set_frame_tiles: chunk must be 0 or a power of two in [32, 1024] "
                      "(optionally with SBP_TILE_WIDE), split 0, 1, 2, 4 or 8");
        return SBP_ERR_ARG;
    }
    arr->fwd_chunk_frames = fwd_chunk;
    arr->adj_split_frames = adj_split;
    return SBP_OK;
}

int sbp_get_frame_tiles(sbp_array arr, int* fwd_chunk, int* adj_split) {
    if (int e = check_frames(arr, "get_frame_tiles")) return e;
    if (fwd_chunk) *fwd_chunk = arr->fwd_chunk_frames;
    if (adj_split) *adj_split = arr->adj_split_frames;
    return SBP_OK;
}

int sbp_autotune_frames(sbp_array arr, sbp_balls balls, const int* n_dev, float* S_dev,
                        float* G_dev, int* fwd_chunk_out, int* adj_split_out) {
    if (int e = check_frames(arr, "autotune_frames")) return e;
    if (!balls_ok(balls) || !n_dev || !S_dev || !G_dev) {
        sbp_set_error("autotune_frames: null pointer");
        return SBP_ERR_ARG;
    }
    cudaStream_t s;
    if (sbp_cuda_check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking),
                       "autotune_frames: stream"))
        return SBP_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const BallsDev bd{balls.x, balls.y, balls.z, balls.R, balls.p0};
    float* g = nullptr;
    const size_t cap = (size_t)arr->n_cap;
    int rc = SBP_OK;
    if (sbp_cuda_check(cudaMalloc(&g, sizeof(float) * 5 * cap), "autotune_frames: alloc"))
        rc = SBP_ERR_CUDA;
    auto time_it = [&](auto&& fn) -> float {
        fn();  // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r) fn();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    int best_chunk = 512, best_split = 4;
    if (rc == SBP_OK) {
        float best = 1e30f;
        for (int chunk : {256, 512, 1024, 1024 | SBP_TILE_WIDE}) {
            const float ms = time_it([&] {
                sbp_launch_forward_frames(arr, bd, n_dev, S_dev, chunk, s);
            });
            if (ms < best) {
                best = ms;
                best_chunk = chunk;
            }
        }
        sbp_grads gr{g, g + cap, g + 2 * cap, g + 3 * cap, g + 4 * cap};
        best = 1e30f;
        for (int split : {1, 2, 4, 8}) {
            arr->adj_split_frames = split;
            const float ms = time_it([&] {
                sbp_launch_adjoint_frames(arr, bd, n_dev, G_dev, gr, SBP_MASK_ALL, s);
            });
            if (ms < best) {
                best = ms;
                best_split = split;
            }
        }
        if (sbp_cuda_check(cudaStreamSynchronize(s), "autotune_frames: run")) rc = SBP_ERR_CUDA;
    }
    arr->fwd_chunk_frames = best_chunk;
    arr->adj_split_frames = best_split;
    if (fwd_chunk_out) *fwd_chunk_out = best_chunk;
    if (adj_split_out) *adj_split_out = best_split;
    cudaFree(g);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    return rc;
}

}  // extern "C"
