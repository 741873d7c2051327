// Spatial ordering of a point cloud: the live balls are put in Morton
// (Z-curve) order of their centres, so that consecutive balls are spatial
// neighbours. The forward and adjoint take balls in chunks of consecutive
// indices and bound each chunk's cells by its bounding box: on a cloud in
// random order (the random initialisation of Algorithm 1, Section 4.1)
// every chunk spans the whole region and its windows cover most of the
// record. Growth keeps the order (children take their parent's place), so
// one sort before the iterations keeps chunks compact.
//
// Key of a ball (30 bits): with lo / hi the componentwise min / max of the
// live centres, span = the largest of hi - lo over the three axes and
// inv = 1024 / span (float32, correctly rounded), each axis is quantised to
// q = min(1023, floor((c - lo) * inv)), every operation rounded once in
// float32 (no fused multiply-add), and the key interleaves the bits of
// (q_x, q_y, q_z) with x in the lowest position. span = 0 gives key 0.
// The order is the stable ascending order of the keys: equal keys keep
// their index order. Balls past the live count keep key 2^32 - 1 and stay
// behind the live ones.
#include <cub/device/device_radix_sort.cuh>

#include <algorithm>

#include "sbp_internal.cuh"

namespace {

// float <-> unsigned int order-preserving maps (for atomicMin / atomicMax)
__device__ __forceinline__ unsigned int ord_of(float f) {
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float float_of(unsigned int o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// box[0..2] = ord(min), box[3..5] = ord(max) over the live balls (box
// preset to UINT_MAX / 0)
__global__ void sort_box_kernel(BallsDev b, const int* n_dev, int n_cap, unsigned int* box) {
    const int n = sbp_read_n(n_dev, n_cap);
    unsigned int lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned int o[3] = {ord_of(b.x[i]), ord_of(b.y[i]), ord_of(b.z[i])};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = min(lo[k], o[k]);
            hi[k] = max(hi[k], o[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], s));
            hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], s));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            atomicMin(&box[k], lo[k]);
            atomicMax(&box[3 + k], hi[k]);
        }
    }
}

__device__ __forceinline__ unsigned int spread10(unsigned int v) {  // bit i -> bit 3i
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ unsigned int quant(float c, float lo, float inv) {
    const float t = __fmul_rn(__fsub_rn(c, lo), inv);
    const float f = floorf(t);
    return f >= 1023.0f ? 1023u : (f > 0.0f ? (unsigned int)f : 0u);
}

__global__ void sort_key_kernel(BallsDev b, const int* n_dev, int n_cap,
                                const unsigned int* box, unsigned int* keys,
                                int* idx) {
    const int n = sbp_read_n(n_dev, n_cap);
    const float lx = float_of(box[0]), ly = float_of(box[1]), lz = float_of(box[2]);
    const float span = fmaxf(fmaxf(__fsub_rn(float_of(box[3]), lx), __fsub_rn(float_of(box[4]), ly)),
                             __fsub_rn(float_of(box[5]), lz));
    const float inv = span > 0.0f ? __fdiv_rn(1024.0f, span) : 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_cap; i += gridDim.x * blockDim.x) {
        unsigned int key = 0xffffffffu;
        if (i < n) {
            key = spread10(quant(b.x[i], lx, inv)) | (spread10(quant(b.y[i], ly, inv)) << 1) |
                  (spread10(quant(b.z[i], lz, inv)) << 2);
        }
        keys[i] = key;
        idx[i] = i;
    }
}

// dst[r][j] = src[r][perm[j]] for the live balls into the scratch, then back
struct SortRows {
    float* r[SBP_FG_ARRAYS];
};

__global__ void sort_gather_rows_kernel(SortRows rows, int nrows, const int* __restrict__ perm,
                                        const int* n_dev, int n_cap, float* __restrict__ tmp) {
    const int n = sbp_read_n(n_dev, n_cap);
    const long long total = (long long)nrows * n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(t / n), j = (int)(t - (long long)r * n);
        tmp[(size_t)r * n_cap + j] = rows.r[r][perm[j]];
    }
}

__global__ void sort_copy_rows_kernel(SortRows rows, int nrows, const int* n_dev, int n_cap,
                                      const float* __restrict__ tmp) {
    const int n = sbp_read_n(n_dev, n_cap);
    const long long total = (long long)nrows * n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(t / n), j = (int)(t - (long long)r * n);
        rows.r[r][j] = tmp[(size_t)r * n_cap + j];
    }
}

}  // namespace

int sbp_launch_sort(sbp_array_s* a, float* const* rows, int nrows, const int* n_dev, int n_cap,
                    cudaStream_t st) {
    if (nrows < 5 || nrows > SBP_FG_ARRAYS || n_cap < 1 || n_cap > a->n_cap || !a->d_fg_buf) {
        sbp_set_error("sort: invalid argument");
        return SBP_ERR_ARG;
    }
    const size_t cap = (size_t)a->n_cap;
    if (!a->d_sort_keys) {  // first use: keys, indices and the radix sort's storage
        size_t bytes = 0;
        if (sbp_cuda_check(cub::DeviceRadixSort::SortPairs(nullptr, bytes, (unsigned int*)nullptr,
                                                           (unsigned int*)nullptr, (int*)nullptr,
                                                           (int*)nullptr, a->n_cap, 0, 32, st),
                           "sort: storage query") ||
            sbp_cuda_check(cudaMalloc(&a->d_sort_keys, sizeof(unsigned int) * (4 * cap + 8)),
                           "sort: alloc keys") ||
            sbp_cuda_check(cudaMalloc(&a->d_sort_tmp, std::max<size_t>(bytes, 16)),
                           "sort: alloc storage")) {
            cudaFree(a->d_sort_keys);
            a->d_sort_keys = nullptr;
            return SBP_ERR_CUDA;
        }
        a->sort_tmp_bytes = std::max<size_t>(bytes, 16);
    }
    unsigned int* k_in = a->d_sort_keys;
    unsigned int* k_out = k_in + cap;
    int* i_in = reinterpret_cast<int*>(k_out + cap);
    int* i_out = i_in + cap;
    unsigned int* box = reinterpret_cast<unsigned int*>(i_out + cap);
    const BallsDev b{rows[0], rows[1], rows[2], rows[3], rows[4]};
    if (sbp_cuda_check(cudaMemsetAsync(box, 0xff, 3 * sizeof(unsigned int), st), "sort: box") ||
        sbp_cuda_check(cudaMemsetAsync(box + 3, 0, 3 * sizeof(unsigned int), st), "sort: box"))
        return SBP_ERR_CUDA;
    const int blocks = std::max(1, std::min(4 * a->sm_count, (n_cap + 255) / 256));
    sort_box_kernel<<<blocks, 256, 0, st>>>(b, n_dev, n_cap, box);
    sort_key_kernel<<<blocks, 256, 0, st>>>(b, n_dev, n_cap, box, k_in, i_in);
    if (sbp_cuda_check(cudaGetLastError(), "sort: key launches")) return SBP_ERR_CUDA;
    // keys past the live count are 2^32 - 1: sorting all 32 bits keeps them last
    size_t bytes = a->sort_tmp_bytes;
    if (sbp_cuda_check(cub::DeviceRadixSort::SortPairs(a->d_sort_tmp, bytes, k_in, k_out, i_in,
                                                       i_out, n_cap, 0, 32, st),
                       "sort: radix sort"))
        return SBP_ERR_CUDA;
    SortRows sr{};
    for (int r = 0; r < nrows; ++r) sr.r[r] = rows[r];
    const int gblocks = std::max(1, std::min(8 * a->sm_count,
                                             (int)(((long long)nrows * n_cap + 255) / 256)));
    sort_gather_rows_kernel<<<gblocks, 256, 0, st>>>(sr, nrows, i_out, n_dev, n_cap, a->d_fg_buf);
    sort_copy_rows_kernel<<<gblocks, 256, 0, st>>>(sr, nrows, n_dev, n_cap, a->d_fg_buf);
    sbp_count_launches(4);
    return sbp_cuda_check(cudaGetLastError(), "sort: launches") ? SBP_ERR_CUDA : SBP_OK;
}

extern "C" int sbp_sort_cloud(sbp_array arr, sbp_balls balls, const int* n_dev, int n_cap,
                              float* const* extra, int n_extra, sbp_stream stream) {
    if (!arr || !balls.x || !balls.y || !balls.z || !balls.R || !balls.p0 || n_cap < 1 ||
        n_cap > arr->n_cap || n_extra < 0 || n_extra > SBP_FG_ARRAYS - 5 ||
        (n_extra > 0 && !extra)) {
        sbp_set_error("sort_cloud: invalid argument");
        return SBP_ERR_ARG;
    }
    float* rows[SBP_FG_ARRAYS] = {balls.x, balls.y, balls.z, balls.R, balls.p0};
    for (int e = 0; e < n_extra; ++e) {
        if (!extra[e]) {
            sbp_set_error("sort_cloud: null extra row");
            return SBP_ERR_ARG;
        }
        rows[5 + e] = extra[e];
    }
    return sbp_launch_sort(arr, rows, 5 + n_extra, n_dev, n_cap,
                           reinterpret_cast<cudaStream_t>(stream));
}
