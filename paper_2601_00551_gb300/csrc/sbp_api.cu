// C ABI of libslingbag: argument checking, the array object and its
// scratch, and dispatch to the kernel launchers.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <string>
#include <vector>

#include "sbp_internal.cuh"

namespace {

thread_local std::string g_last_error = "no error";
std::atomic<long long> g_launches{0};

cudaStream_t as_stream(sbp_stream s) { return reinterpret_cast<cudaStream_t>(s); }

bool balls_ok(const sbp_balls& b) { return b.x && b.y && b.z && b.R && b.p0; }
bool grads_ok(const sbp_grads& g) { return g.gx && g.gy && g.gz && g.gR && g.gp0; }

BallsDev to_dev(const sbp_balls& b) { return BallsDev{b.x, b.y, b.z, b.R, b.p0}; }

int check_array(sbp_array a, const char* fn) {
    if (!a) {
        sbp_set_error(std::string(fn) + ": null array");
        return SBP_ERR_ARG;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != a->device) {
        sbp_set_error(std::string(fn) + ": the array belongs to another device");
        return SBP_ERR_ARG;
    }
    return SBP_OK;
}

int check_cap(sbp_array a, int n_cap, const char* fn) {
    if (n_cap < 1 || n_cap > a->n_cap) {
        sbp_set_error(std::string(fn) + ": n_cap must be in [1, capacity of the array]");
        return SBP_ERR_ARG;
    }
    return SBP_OK;
}

void free_array(sbp_array_s* a) {
    if (!a) return;
    cudaFree(a->d_sens);
    cudaFree(a->d_acc);
    cudaFree(a->d_lossp);
    cudaFree(a->d_fg_counts);
    cudaFree(a->d_fg_buf);
    cudaFree(a->d_state);
    cudaFree(a->d_adj_part);
    cudaFree(a->d_adj_ticket);
    cudaFree(a->d_rc_yk);
    cudaFree(a->d_rc_S);
    cudaFree(a->d_rc_G);
    cudaFree(a->d_rc_state);
    cudaFree(a->d_frame_off);
    cudaFree(a->d_frame_n_new);
    cudaFree(a->d_frame_lossp);
    cudaFree(a->d_frame_pmax);
    cudaFree(a->d_gacc);
    cudaFree(a->d_fr_yk);
    cudaFree(a->d_fr_S);
    cudaFree(a->d_fr_G);
    cudaFree(a->d_sort_keys);
    cudaFree(a->d_sort_tmp);
    delete[] a->h_frame_off;
    delete a;
}

}  // namespace

void sbp_set_error(const std::string& msg) { g_last_error = msg; }

void sbp_count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int sbp_cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return 0;
    sbp_set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return 1;
}

int sbp_level_T(const sbp_array_s* a, int k) {
    const int f = a->factors[k];
    return (a->T + f - 1) / f;
}

LevelGeo sbp_level_geo(const sbp_array_s* a, int k) {
    LevelGeo g;
    const double h = a->c * (double)a->factors[k] / a->fs;  // mm per sample
    g.M = a->M;
    g.Tk = sbp_level_T(a, k);
    g.h_hi = (float)h;
    g.h_lo = (float)(h - (double)g.h_hi);
    g.inv_h = (float)(1.0 / h);
    g.inv_4h = (float)(0.25 / h);
    g.wmode = a->wmode;
    g.pad = 0;
    return g;
}

extern "C" {

const char* sbp_last_error(void) { return g_last_error.c_str(); }

const char* sbp_version(void) { return "slingbag-gb300 0.1 (sm_103a)"; }

long long sbp_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int sbp_create_array(const float* pos_host, const float* normal_host, int M, double c_mm_per_us,
                     double fs_mhz, int T, const int* factors_host, int n_levels, int n_cap,
                     const sbp_params* params, sbp_array* out) {
    if (!out) {
        sbp_set_error("create_array: out is null");
        return SBP_ERR_ARG;
    }
    *out = nullptr;
    if (!pos_host || !normal_host || !factors_host || M < 1 || T < 1 || n_levels < 1 ||
        n_levels > SBP_MAX_LEVELS || n_cap < 1 || !(c_mm_per_us > 0) || !(fs_mhz > 0) ||
        !std::isfinite(c_mm_per_us) || !std::isfinite(fs_mhz)) {
        sbp_set_error("create_array: invalid argument");
        return SBP_ERR_ARG;
    }
    for (int k = 0; k < n_levels; ++k)
        if (factors_host[k] < 1 || factors_host[k] > T) {
            sbp_set_error("create_array: level factors must be in [1, T]");
            return SBP_ERR_ARG;
        }
    if ((long long)T * 8 > 200LL * 1024) {
        sbp_set_error("create_array: T larger than 25600 samples is not supported");
        return SBP_ERR_ARG;
    }
    if (params && (params->weight_mode < SBP_W_CLAMP || params->weight_mode > SBP_W_COS)) {
        sbp_set_error("create_array: unknown weight mode");
        return SBP_ERR_ARG;
    }
    // host copy of the sensors as [6][M], normals normalised
    std::vector<float> sens((size_t)6 * M);
    for (int m = 0; m < M; ++m) {
        const double nx = normal_host[3 * m], ny = normal_host[3 * m + 1],
                     nz = normal_host[3 * m + 2];
        const double nn = std::sqrt(nx * nx + ny * ny + nz * nz);
        for (int k = 0; k < 3; ++k) {
            if (!std::isfinite(pos_host[3 * m + k])) {
                sbp_set_error("create_array: non-finite sensor position");
                return SBP_ERR_NUMERIC;
            }
            sens[(size_t)k * M + m] = pos_host[3 * m + k];
        }
        if (!(nn > 0) || !std::isfinite(nn)) {
            sbp_set_error("create_array: zero or non-finite sensor normal");
            return SBP_ERR_NUMERIC;
        }
        sens[(size_t)3 * M + m] = (float)(nx / nn);
        sens[(size_t)4 * M + m] = (float)(ny / nn);
        sens[(size_t)5 * M + m] = (float)(nz / nn);
    }
    sbp_array_s* a = new sbp_array_s();
    memset(a, 0, sizeof(*a));
    if (sbp_cuda_check(cudaGetDevice(&a->device), "create_array: device")) {
        delete a;
        return SBP_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&a->sm_count, cudaDevAttrMultiProcessorCount, a->device);
    if (a->sm_count < 1) a->sm_count = 1;
    a->M = M;
    a->T = T;
    a->n_levels = n_levels;
    a->n_cap = n_cap;
    a->level = 0;
    for (int k = 0; k < n_levels; ++k) a->factors[k] = factors_host[k];
    a->c = c_mm_per_us;
    a->fs = fs_mhz;
    a->wmode = params ? params->weight_mode : SBP_W_CLAMP;
    a->loss_blocks = 4 * a->sm_count;
    a->fg_blocks = (n_cap + 255) / 256;
    bool ok = true;
    ok = ok && !sbp_cuda_check(cudaMalloc(&a->d_sens, sizeof(float) * 6 * M), "alloc sensors");
    ok = ok && !sbp_cuda_check(cudaMalloc(&a->d_acc, sizeof(unsigned long long) * (size_t)M * T),
                               "alloc trace accumulators");
    a->acc_cells = (size_t)M * T;
    ok = ok && !sbp_cuda_check(cudaMalloc(&a->d_lossp, sizeof(double) * a->loss_blocks),
                               "alloc loss partials");
    ok = ok && !sbp_cuda_check(cudaMalloc(&a->d_fg_counts, sizeof(int) * (a->fg_blocks + 1)),
                               "alloc filter counts");
    ok = ok && !sbp_cuda_check(cudaMalloc(&a->d_fg_buf, sizeof(float) * (size_t)SBP_FG_ARRAYS *
                                                            (size_t)n_cap),
                               "alloc filter buffer");
    ok = ok && !sbp_cuda_check(cudaMalloc(&a->d_state, sizeof(SbpDevState)), "alloc state");
    // in scratch units of SBP_ADJ_CHUNK balls, for n_cap rounded up to whole
    // chunks of the largest size (both adjoints' partial sums and tickets fit)
    a->adj_chunks = (n_cap + SBP_ADJ_CHUNK_MAX - 1) / SBP_ADJ_CHUNK_MAX *
                    (SBP_ADJ_CHUNK_MAX / SBP_ADJ_CHUNK);
    ok = ok && !sbp_cuda_check(cudaMalloc(&a->d_adj_part, sizeof(float) * (size_t)a->adj_chunks *
                                                              SBP_ADJ_MAX_SPLIT * 5 * SBP_ADJ_CHUNK),
                               "alloc adjoint partials");
    ok = ok && !sbp_cuda_check(cudaMalloc(&a->d_adj_ticket, sizeof(unsigned int) * a->adj_chunks),
                               "alloc adjoint tickets");
    ok = ok && !sbp_cuda_check(cudaMemset(a->d_adj_ticket, 0, sizeof(unsigned int) * a->adj_chunks),
                               "clear adjoint tickets");
    ok = ok && !sbp_cuda_check(cudaMemcpy(a->d_sens, sens.data(), sizeof(float) * 6 * M,
                                          cudaMemcpyHostToDevice),
                               "copy sensors");
    ok = ok && !sbp_cuda_check(
                   cudaMemset(a->d_acc, 0, sizeof(unsigned long long) * (size_t)M * T),
                   "clear accumulators");
    ok = ok && !sbp_cuda_check(cudaMemset(a->d_state, 0, sizeof(SbpDevState)), "clear state");
    ok = ok && !sbp_cuda_check(cudaDeviceSynchronize(), "create_array: synchronise");
    if (!ok) {
        free_array(a);
        return SBP_ERR_CUDA;
    }
    *out = a;
    return SBP_OK;
}

int sbp_destroy_array(sbp_array arr) {
    if (!arr) return SBP_OK;
    cudaDeviceSynchronize();
    free_array(arr);
    return SBP_OK;
}

int sbp_level_info(sbp_array arr, int k, int* T_k, double* dt_k) {
    if (!arr) {
        sbp_set_error("level_info: null array");
        return SBP_ERR_ARG;
    }
    if (k < 0 || k >= arr->n_levels) {
        sbp_set_error("level_info: level out of range");
        return SBP_ERR_LEVEL;
    }
    if (T_k) *T_k = sbp_level_T(arr, k);
    if (dt_k) *dt_k = (double)arr->factors[k] / arr->fs;
    return SBP_OK;
}

int sbp_set_sampling_level(sbp_array arr, int k, const float* y_full_dev, float* y_k_dev,
                           sbp_stream stream) {
    if (int e = check_array(arr, "set_sampling_level")) return e;
    if (k < 0 || k >= arr->n_levels) {
        sbp_set_error("set_sampling_level: level out of range");
        return SBP_ERR_LEVEL;
    }
    if (y_full_dev && !y_k_dev) {
        sbp_set_error("set_sampling_level: y_k_dev is null");
        return SBP_ERR_ARG;
    }
    arr->level = k;
    if (y_full_dev) return sbp_launch_downsample(arr, k, y_full_dev, y_k_dev, as_stream(stream));
    return SBP_OK;
}

int sbp_forward(sbp_array arr, sbp_balls balls, const int* n_dev, int n_cap, float* S_dev,
                unsigned flags, sbp_stream stream) {
    if (int e = check_array(arr, "forward")) return e;
    if (int e = check_cap(arr, n_cap, "forward")) return e;
    if (!balls_ok(balls) || !S_dev || (flags & ~SBP_DETERMINISTIC)) {
        sbp_set_error("forward: null pointer or unknown flag");
        return SBP_ERR_ARG;
    }
    return sbp_launch_forward(arr, to_dev(balls), n_dev, n_cap, S_dev, as_stream(stream));
}

int sbp_residual(sbp_array arr, const float* S_dev, const float* y_k_dev, float* G_dev,
                 double* loss_dev, sbp_stream stream) {
    if (int e = check_array(arr, "residual")) return e;
    if (!y_k_dev || !G_dev) {
        sbp_set_error("residual: null pointer");
        return SBP_ERR_ARG;
    }
    return sbp_launch_residual(arr, S_dev, y_k_dev, G_dev, loss_dev, as_stream(stream));
}

int sbp_adjoint(sbp_array arr, sbp_balls balls, const int* n_dev, int n_cap, const float* G_dev,
                sbp_grads out, unsigned grad_mask, sbp_stream stream) {
    if (int e = check_array(arr, "adjoint")) return e;
    if (int e = check_cap(arr, n_cap, "adjoint")) return e;
    if (!balls_ok(balls) || !grads_ok(out) || !G_dev || (grad_mask & ~SBP_MASK_ALL)) {
        sbp_set_error("adjoint: null pointer or unknown mask bit");
        return SBP_ERR_ARG;
    }
    return sbp_launch_adjoint(arr, to_dev(balls), n_dev, n_cap, G_dev, out, grad_mask,
                              as_stream(stream));
}

int sbp_store_windows(sbp_array arr, sbp_balls balls, const int* n_dev, int n_cap,
                      void* rec_dev, sbp_stream stream) {
    if (int e = check_array(arr, "store_windows")) return e;
    if (int e = check_cap(arr, n_cap, "store_windows")) return e;
    if (!balls_ok(balls) || !rec_dev || (reinterpret_cast<uintptr_t>(rec_dev) & 3u)) {
        sbp_set_error("store_windows: null or misaligned pointer");
        return SBP_ERR_ARG;
    }
    if (n_cap == 0) return SBP_OK;
    return sbp_launch_store_windows(arr, to_dev(balls), n_dev, n_cap, rec_dev, as_stream(stream));
}

int sbp_adjoint_stored(sbp_array arr, sbp_balls balls, const int* n_dev, int n_cap,
                       const void* rec_dev, const float* G_dev, sbp_grads out,
                       unsigned grad_mask, sbp_stream stream) {
    if (int e = check_array(arr, "adjoint_stored")) return e;
    if (int e = check_cap(arr, n_cap, "adjoint_stored")) return e;
    if (!balls_ok(balls) || !grads_ok(out) || !rec_dev || !G_dev ||
        (reinterpret_cast<uintptr_t>(rec_dev) & 3u) || (grad_mask & ~SBP_MASK_ALL)) {
        sbp_set_error("adjoint_stored: null or misaligned pointer, or unknown mask bit");
        return SBP_ERR_ARG;
    }
    if (n_cap == 0) return SBP_OK;
    return sbp_launch_adjoint_stored(arr, to_dev(balls), n_dev, n_cap, rec_dev, G_dev, out,
                                     grad_mask, as_stream(stream));
}

namespace {

bool fwd_chunk_ok(int c) { return c == 0 || sbp_fwd_tile_valid(c); }
bool adj_split_ok(int s) { return s == 0 || s == 1 || s == 2 || s == 4 || s == 8; }

}  // namespace

int sbp_set_tiles(sbp_array arr, int k, int fwd_chunk, int adj_split) {
    if (int e = check_array(arr, "set_tiles")) return e;
    if (k < 0 || k >= arr->n_levels) {
        sbp_set_error("set_tiles: level out of range");
        return SBP_ERR_LEVEL;
    }
    if (!fwd_chunk_ok(fwd_chunk) || !adj_split_ok(adj_split)) {
        sbp_set_error("set_tiles: chunk must be 0 or a power of two in [32, 2048] (optionally "
                      "with SBP_TILE_WIDE), split 0, 1, 2, 4 or 8");
        return SBP_ERR_ARG;
    }
    arr->fwd_chunk_lvl[k] = fwd_chunk;
    arr->adj_split_lvl[k] = adj_split;
    return SBP_OK;
}

int sbp_get_tiles(sbp_array arr, int k, int* fwd_chunk, int* adj_split) {
    if (int e = check_array(arr, "get_tiles")) return e;
    if (k < 0 || k >= arr->n_levels) {
        sbp_set_error("get_tiles: level out of range");
        return SBP_ERR_LEVEL;
    }
    if (fwd_chunk) *fwd_chunk = arr->fwd_chunk_lvl[k];
    if (adj_split) *adj_split = arr->adj_split_lvl[k];
    return SBP_OK;
}

int sbp_autotune(sbp_array arr, sbp_balls balls, const int* n_dev, int n_cap, float* S_dev,
                 const float* G_dev, int* fwd_chunk_out, int* adj_split_out) {
    if (int e = check_array(arr, "autotune")) return e;
    if (int e = check_cap(arr, n_cap, "autotune")) return e;
    if (!balls_ok(balls) || !S_dev || !G_dev) {
        sbp_set_error("autotune: null pointer");
        return SBP_ERR_ARG;
    }
    cudaStream_t s;
    if (sbp_cuda_check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "autotune: stream"))
        return SBP_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const BallsDev bd = to_dev(balls);
    const size_t cap = (size_t)n_cap;
    float* g = nullptr;
    int rc = SBP_OK;
    if (sbp_cuda_check(cudaMalloc(&g, sizeof(float) * 5 * std::max<size_t>(cap, 1)),
                       "autotune: alloc"))
        rc = SBP_ERR_CUDA;
    // a failed launch latches rc and ends the search with the defaults
    auto time_it = [&](auto&& fn) -> float {
        if (rc != SBP_OK) return 1e30f;
        rc = fn();  // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < 5 && rc == SBP_OK; ++r) rc = fn();
        cudaEventRecord(e1, s);
        if (sbp_cuda_check(cudaEventSynchronize(e1), "autotune: run")) rc = SBP_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return rc == SBP_OK ? ms : 1e30f;
    };
    // the default tile (0) is timed first; another choice replaces it only
    // when it is faster by more than kMargin, so timing noise and a cloud
    // that differs from the one tuned on do not move the choice for little
    constexpr float kMargin = 0.97f;
    const int k = arr->level;
    auto pick = [&](std::initializer_list<int> cands, int* field, auto&& launch) {
        *field = 0;
        const float base = time_it(launch);
        float best = base * kMargin;
        int choice = 0;
        for (int c : cands) {
            *field = c;
            const float ms = time_it(launch);
            if (ms < best) {
                best = ms;
                choice = c;
            }
        }
        *field = choice;
        return choice;
    };
    const sbp_grads gr{g, g + cap, g + 2 * cap, g + 3 * cap, g + 4 * cap};
    int best_chunk = pick({128, 256, 512, 1024, 2048, 1024 | SBP_TILE_WIDE, 2048 | SBP_TILE_WIDE},
                          &arr->fwd_chunk_lvl[k], [&] {
        return sbp_launch_forward(arr, bd, n_dev, n_cap, S_dev, s);
    });
    int best_split = pick({1, 2, 4, 8}, &arr->adj_split_lvl[k], [&] {
        return sbp_launch_adjoint(arr, bd, n_dev, n_cap, G_dev, gr, SBP_MASK_ALL, s);
    });
    if (rc != SBP_OK) best_chunk = best_split = 0;
    arr->fwd_chunk_lvl[k] = best_chunk;
    arr->adj_split_lvl[k] = best_split;
    if (fwd_chunk_out) *fwd_chunk_out = best_chunk;
    if (adj_split_out) *adj_split_out = best_split;
    cudaFree(g);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    return rc;
}

int sbp_filter_grow(sbp_array arr, sbp_balls balls, sbp_grads grads, float* const* extra,
                    int n_extra, int* n_dev, int n_cap, const sbp_grow_params* gp, int mode,
                    sbp_stream stream) {
    if (int e = check_array(arr, "filter_grow")) return e;
    if (int e = check_cap(arr, n_cap, "filter_grow")) return e;
    if (!balls_ok(balls) || !grads_ok(grads) || !n_dev || n_extra < 0 ||
        n_extra > SBP_MAX_EXTRA || (n_extra > 0 && !extra) || mode < SBP_KEEP_NEG ||
        mode > SBP_GROW || (mode == SBP_GROW && !gp)) {
        sbp_set_error("filter_grow: invalid argument");
        return SBP_ERR_ARG;
    }
    for (int e = 0; e < n_extra; ++e)
        if (!extra[e]) {
            sbp_set_error("filter_grow: null extra array");
            return SBP_ERR_ARG;
        }
    if (gp && (gp->grad_mask & ~SBP_MASK_ALL)) {
        sbp_set_error("filter_grow: unknown grad_mask bit");
        return SBP_ERR_ARG;
    }
    return sbp_launch_filter_grow(arr, balls, grads, extra, n_extra, n_dev, n_cap, gp, mode,
                                  as_stream(stream));
}

int sbp_adam_step(sbp_array arr, sbp_balls balls, sbp_grads grads, sbp_balls m, sbp_balls v,
                  const int* n_dev, int n_cap, int t, const sbp_adam_params* ap,
                  unsigned mask, sbp_stream stream) {
    if (int e = check_array(arr, "adam_step")) return e;
    if (int e = check_cap(arr, n_cap, "adam_step")) return e;
    if (!balls_ok(balls) || !grads_ok(grads) || !balls_ok(m) || !balls_ok(v) || !ap || t < 1 ||
        (mask & ~(SBP_MASK_ALL | SBP_SOFTPLUS_R))) {
        sbp_set_error("adam_step: invalid argument");
        return SBP_ERR_ARG;
    }
    return sbp_launch_adam(arr, balls, grads, m, v, n_dev, n_cap, t, ap, mask,
                           as_stream(stream));
}

int sbp_sync_status(sbp_array arr, sbp_stream stream) {
    if (int e = check_array(arr, "sync_status")) return e;
    if (sbp_cuda_check(cudaStreamSynchronize(as_stream(stream)), "sync_status"))
        return SBP_ERR_CUDA;
    int err = 0;
    if (sbp_cuda_check(cudaMemcpy(&err, &arr->d_state->err, sizeof(int), cudaMemcpyDeviceToHost),
                       "sync_status: read"))
        return SBP_ERR_CUDA;
    if (err) {
        int zero = 0;
        cudaMemcpy(&arr->d_state->err, &zero, sizeof(int), cudaMemcpyHostToDevice);
        sbp_set_error(err == SBP_ERR_CAPACITY ? "device: growth exceeded n_cap"
                                              : "device: latched error");
    }
    return err;
}

int sbp_get_inside_pairs(sbp_array arr, sbp_stream stream, long long* count) {
    if (int e = check_array(arr, "get_inside_pairs")) return e;
    if (!count) {
        sbp_set_error("get_inside_pairs: null pointer");
        return SBP_ERR_ARG;
    }
    if (sbp_cuda_check(cudaStreamSynchronize(as_stream(stream)), "get_inside_pairs"))
        return SBP_ERR_CUDA;
    unsigned long long c = 0;
    if (sbp_cuda_check(cudaMemcpy(&c, &arr->d_state->inside_pairs, sizeof(c),
                                  cudaMemcpyDeviceToHost),
                       "get_inside_pairs: read"))
        return SBP_ERR_CUDA;
    *count = (long long)c;
    return SBP_OK;
}

}  // extern "C"
