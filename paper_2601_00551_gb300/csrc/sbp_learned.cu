// Learned initial proposal (an extension of the initialisation step of
// Algorithm 1; the paper itself initialises at random and filters by zero
// gradients, Section 4.2):
//   * delay-and-sum volume of the measured traces on a voxel grid;
//   * a small 3D CNN on that volume, 1 -> 16 -> 32 -> 64 channels of 3x3x3
//     convolutions with ReLU (tcgen05 implicit GEMMs, sbp_cnn.cu) and a
//     1x1x1 head with two outputs per voxel: the logit of "a source lies
//     here" and its pressure;
//   * its training step: binary cross-entropy on the occupancy logit (with a
//     positive-class weight), squared error on the pressure of occupied
//     voxels, backpropagation (the data gradient of a convolution is the
//     convolution of the output gradient with the flipped, transposed
//     weights, on the tensor cores again; the weight gradients are GEMMs
//     over voxels on the tensor cores too, sbp_wgrad_bf16, reduced in a
//     fixed order so that a training step is reproducible bit for bit) and
//     Adam on FP32 master weights;
//   * the proposal: a given number of balls in every voxel whose occupancy
//     probability exceeds a threshold, each at a seeded random point of the
//     voxel, in voxel order.
// The hidden activations h1, h2 and their gradients g1, g2 are kept planar
// ([C / 8][V][8]), so that the TMA-fed convolutions that read them copy halo
// rows of ten voxels instead of one; h3 and g3 are channels-last.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "sbp_internal.cuh"
#include "sbp_scan.cuh"

namespace {

constexpr int kC1 = 16, kC2 = 32, kC3 = 64, kHead = 2;
// parameter blocks (FP32 masters), weights as [cout][27][cin]
constexpr int kW1 = kC1 * 27 * 1, kB1 = kC1;
constexpr int kW2 = kC2 * 27 * kC1, kB2 = kC2;
constexpr int kW3 = kC3 * 27 * kC2, kB3 = kC3;
constexpr int kWh = kHead * kC3, kBh = kHead;
constexpr int kOW1 = 0, kOB1 = kOW1 + kW1, kOW2 = kOB1 + kB1, kOB2 = kOW2 + kW2;
constexpr int kOW3 = kOB2 + kB2, kOB3 = kOW3 + kW3, kOWh = kOB3 + kB3, kOBh = kOWh + kWh;
constexpr int kParams = kOBh + kBh;

int padded_k(int cin) { return (27 * cin + 63) / 64 * 64; }

}  // namespace

struct sbp_cnn_s {
    int device = -1;
    int nx = 0, ny = 0, nz = 0;
    long long V = 0;
    int step = 0;
    float* p = nullptr;  // [kParams] masters, then m, v, grads: 4 blocks
    __nv_bfloat16* w1 = nullptr;   // [16][64]
    __nv_bfloat16* w2 = nullptr;   // [32][padded_k(16)]
    __nv_bfloat16* w3 = nullptr;   // [64][padded_k(32)]
    __nv_bfloat16* w2t = nullptr;  // dgrad of conv2: [16][padded_k(32)]
    __nv_bfloat16* w3t = nullptr;  // dgrad of conv3: [32][padded_k(64)]
    __nv_bfloat16* x0 = nullptr;   // [V] scaled input
    __nv_bfloat16* h1 = nullptr;   // [2][V][8] (planar)
    __nv_bfloat16* h2 = nullptr;   // [4][V][8] (planar)
    __nv_bfloat16* h3 = nullptr;   // [V][64]
    __nv_bfloat16* g3 = nullptr;   // [V][64] gradient before conv3's ReLU
    __nv_bfloat16* g2 = nullptr;   // [4][V][8] (planar)
    __nv_bfloat16* g1 = nullptr;   // [2][V][8] (planar)
    float* out = nullptr;          // [V][2]
    float* dout = nullptr;         // [V][2]
    unsigned int* vmax = nullptr;  // bits of max |volume|
    double* loss = nullptr;        // [2]: data term sums
    int* cnt = nullptr;            // proposal scratch: per-block counts ([blocks + 1])
    long long cnt_cap = 0;
    int sms = 1;                   // SMs of the device (sizes the weight-gradient grids)
    float* wg_part = nullptr;      // weight-gradient partial tiles (largest layer)
    float* hd_part = nullptr;      // head parameter-gradient partials [blocks][kWh + kBh]
};

namespace {

// ---------------------------------------------------------------------------
// delay-and-sum
// ---------------------------------------------------------------------------

constexpr int kDasThreads = 256;
constexpr int kDasTile = 256;

struct VoxGeo {
    float o[3];
    float h;
    int n[3];
};

__global__ void __launch_bounds__(kDasThreads)
das_kernel(const float* __restrict__ y, int M, int T, const float* __restrict__ sens, float inv_cdt,
           int wmode, VoxGeo g, float* __restrict__ vol) {
    __shared__ float s[kDasTile * 6];
    const long long V = (long long)g.n[0] * g.n[1] * g.n[2];
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = v < V;
    float px = 0.f, py = 0.f, pz = 0.f;
    if (act) {
        const int ix = (int)(v % g.n[0]), iy = (int)((v / g.n[0]) % g.n[1]);
        const int iz = (int)(v / ((long long)g.n[0] * g.n[1]));
        px = g.o[0] + ((float)ix + 0.5f) * g.h;
        py = g.o[1] + ((float)iy + 0.5f) * g.h;
        pz = g.o[2] + ((float)iz + 0.5f) * g.h;
    }
    float acc = 0.f;
    for (int m0 = 0; m0 < M; m0 += kDasTile) {
        const int cnt = min(kDasTile, M - m0);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt * 6; t += blockDim.x) {
            const int k = t / cnt, j = t % cnt;
            s[j * 6 + k] = sens[(size_t)k * M + m0 + j];
        }
        __syncthreads();
        if (!act) continue;
        for (int j = 0; j < cnt; ++j) {
            const float* S = s + j * 6;
            const float dx = px - S[0], dy = py - S[1], dz = pz - S[2];
            const float d = sqrtf(dx * dx + dy * dy + dz * dz);
            float w = 1.0f;
            if (wmode != SBP_W_NONE) {
                const float cs = (S[3] * dx + S[4] * dy + S[5] * dz) / d;
                w = wmode == SBP_W_COS ? cs : fmaxf(cs, 0.0f);
            }
            if (w == 0.0f) continue;
            const float q = d * inv_cdt - 0.5f;
            const float fl = floorf(q);
            if (!(fl >= -1.0f && fl < (float)T)) continue;
            const int i0 = (int)fl;
            const float f = q - fl;
            const float* row = y + (size_t)(m0 + j) * T;
            const float y0 = i0 >= 0 ? row[i0] : 0.0f;
            const float y1 = i0 + 1 < T ? row[i0 + 1] : 0.0f;
            acc += w * fmaf(f, y1 - y0, y0);
        }
    }
    if (act) vol[v] = acc;
}

// ---------------------------------------------------------------------------
// CNN pieces on the CUDA cores
// ---------------------------------------------------------------------------

__global__ void absmax_kernel(const float* __restrict__ x, long long n, unsigned int* bits) {
    float m = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(bits, __float_as_uint(m));
}

// x0 = vol / max|vol| in bf16
__global__ void scale_input_kernel(const float* __restrict__ vol, long long n,
                                   const unsigned int* bits, __nv_bfloat16* __restrict__ x0) {
    const float mx = __uint_as_float(*bits);
    const float inv = mx > 0.f ? 1.0f / mx : 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        x0[i] = __float2bfloat16(vol[i] * inv);
}

// out[v][j] = bh[j] + sum_c h3[v][c] Wh[j][c]
__global__ void head_fwd_kernel(const __nv_bfloat16* __restrict__ h3, long long V,
                                const float* __restrict__ P, float* __restrict__ out) {
    __shared__ float w[kWh + kBh];
    for (int t = threadIdx.x; t < kWh + kBh; t += blockDim.x) w[t] = P[kOWh + t];
    __syncthreads();
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x) {
        float a0 = w[kWh], a1 = w[kWh + 1];
        const __nv_bfloat16* r = h3 + v * kC3;
#pragma unroll
        for (int c = 0; c < kC3; ++c) {
            const float hv = __bfloat162float(r[c]);
            a0 = fmaf(hv, w[c], a0);
            a1 = fmaf(hv, w[kC3 + c], a1);
        }
        out[2 * v] = a0;
        out[2 * v + 1] = a1;
    }
}

// Loss per voxel and its gradient:
//   logit z: pos_weight * t * softplus(-z) + (1 - t) * softplus(z),
//   pressure q (occupied voxels only): (q - p)^2,
// both divided by V. dout = d loss / d (z, q); loss sums in double.
__global__ void loss_kernel(const float* __restrict__ out, const float* __restrict__ occ,
                            const float* __restrict__ p0, long long V, float pos_weight,
                            float* __restrict__ dout, double* __restrict__ loss) {
    __shared__ double red[2][32];
    double l0 = 0.0, l1 = 0.0;
    const float invV = 1.0f / (float)V;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x) {
        const float z = out[2 * v], q = out[2 * v + 1];
        const float t = occ[v];
        const float sp_pos = fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));  // softplus(z)
        const float sp_neg = sp_pos - z;                                // softplus(-z)
        const float sg = 1.0f / (1.0f + expf(-z));
        l0 += (double)(pos_weight * t * sp_neg + (1.0f - t) * sp_pos);
        dout[2 * v] = (pos_weight * t * (sg - 1.0f) + (1.0f - t) * sg) * invV;
        const float e = t > 0.f ? q - p0[v] : 0.0f;
        l1 += (double)(e * e);
        dout[2 * v + 1] = 2.0f * e * invV;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l0 += __shfl_xor_sync(0xffffffffu, l0, o);
        l1 += __shfl_xor_sync(0xffffffffu, l1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = l0;
        red[1][threadIdx.x >> 5] = l1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        atomicAdd(&loss[0], a / (double)V);
        atomicAdd(&loss[1], b / (double)V);
    }
}

// head backward, data part: g3[v][c] = (sum_j dout[v][j] Wh[j][c]) [h3 > 0]
__global__ void head_bwd_data_kernel(const __nv_bfloat16* __restrict__ h3,
                                     const float* __restrict__ dout, long long V,
                                     const float* __restrict__ P, __nv_bfloat16* __restrict__ g3) {
    __shared__ float w[kWh];
    for (int t = threadIdx.x; t < kWh; t += blockDim.x) w[t] = P[kOWh + t];
    __syncthreads();
    const long long n = V * kC3;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long v = i / kC3;
        const int c = (int)(i - v * kC3);
        const float hv = __bfloat162float(h3[i]);
        g3[i] = __float2bfloat16(hv > 0.f ? fmaf(dout[2 * v], w[c], dout[2 * v + 1] * w[kC3 + c])
                                          : 0.0f);
    }
}

// head backward, parameter part: dWh[j][c] = sum_v dout[v][j] h3[v][c] and
// dbh[j] = sum_v dout[v][j]. A block takes `chunk` voxels; thread j kC3 + c
// sums its weight over them (reading a voxel's channels coalesced), threads
// 2 kC3 and 2 kC3 + 1 the biases, into the block's row of partials; the
// rows are then added in block order (head_param_reduce_kernel).
__global__ void head_bwd_param_kernel(const __nv_bfloat16* __restrict__ h3,
                                      const float* __restrict__ dout, long long V, int chunk,
                                      float* __restrict__ part) {
    const int t = threadIdx.x;
    if (t >= kWh + kBh) return;
    const long long v0 = (long long)blockIdx.x * chunk, v1 = min(V, v0 + chunk);
    const int j = t < kWh ? t / kC3 : t - kWh, c = t < kWh ? t % kC3 : 0;
    float acc = 0.f;
    for (long long v = v0; v < v1; ++v) {
        const float d = dout[2 * v + j];
        acc = t < kWh ? fmaf(d, __bfloat162float(h3[v * kC3 + c]), acc) : acc + d;
    }
    part[(size_t)blockIdx.x * (kWh + kBh) + t] = acc;
}

__global__ void head_param_reduce_kernel(const float* __restrict__ part, int blocks,
                                         float* __restrict__ G) {
    const int t = threadIdx.x;
    if (t >= kWh + kBh) return;
    float s = 0.0f;
    for (int b = 0; b < blocks; ++b) s += part[(size_t)b * (kWh + kBh) + t];
    G[kOWh + t] = s;
}

// g[v][c] *= [h[v][c] > 0] (the ReLU of the layer that produced h)
__global__ void relu_mask_kernel(__nv_bfloat16* __restrict__ g, const __nv_bfloat16* __restrict__ h,
                                 long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        if (!(__bfloat162float(h[i]) > 0.f)) g[i] = __float2bfloat16(0.0f);
}

// forward weights [cout][27][cin] -> bf16 [cout][kp]; dgrad weights
// W'[c][tap][n] = W[n][26 - tap][c] -> bf16 [cin][kp'] (kp' for cin' = cout)
__global__ void pack_kernel(const float* __restrict__ W, int cout, int cin, int kp,
                            __nv_bfloat16* __restrict__ fwd, int kpt, __nv_bfloat16* __restrict__ bwd) {
    const int total = cout * kp;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int n = t / kp, k = t % kp;
        fwd[t] = __float2bfloat16(k < 27 * cin ? W[(size_t)n * 27 * cin + k] : 0.0f);
    }
    if (!bwd) return;
    const int total2 = cin * kpt;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total2; t += gridDim.x * blockDim.x) {
        const int c = t / kpt, k = t % kpt;
        float v = 0.0f;
        if (k < 27 * cout) {
            const int tap = k / cout, n = k % cout;
            v = W[((size_t)n * 27 + (26 - tap)) * cin + c];
        }
        bwd[t] = __float2bfloat16(v);
    }
}

__global__ void adam_flat_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                                 float* __restrict__ g, int n, float lr, float b1, float b2,
                                 float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        g[i] = 0.0f;
    }
}

// ---------------------------------------------------------------------------
// proposal
// ---------------------------------------------------------------------------

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float unit24(uint64_t seed, long long k) {
    return (float)(mix64(seed + (uint64_t)(k + 1) * kGamma) >> 40) * (1.0f / 16777216.0f);
}

__global__ void propose_count_kernel(const float* __restrict__ out, long long V, float zthr,
                                     int* __restrict__ cnt) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool on = v < V && out[2 * v] > zthr;
    const int c = __syncthreads_count(on);
    if (threadIdx.x == 0) cnt[blockIdx.x] = c;
}

__global__ void propose_scan_kernel(int* __restrict__ cnt, int nb) {
    __shared__ long long warp_tot[32];
    long long carry = 0;
    for (int b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int b = b0 + threadIdx.x;
        const long long v = b < nb ? cnt[b] : 0;
        long long tot;
        const long long incl = sbp_block_incl_scan(v, warp_tot, tot);
        if (b < nb) cnt[b] = (int)(carry + incl - v);
        carry += tot;
    }
    if (threadIdx.x == 0) cnt[nb] = (int)carry;
}

// Occupied voxel number q (in voxel order) gets balls q k .. q k + k - 1, ball
// j at the seeded uniform point of counter outputs 3 (v k + j) .. + 2.
__global__ void propose_write_kernel(const float* __restrict__ out, long long V, float zthr,
                                     const int* __restrict__ off, VoxGeo g, uint64_t seed, float R,
                                     float p_min, float p_max, int k, sbp_balls balls, int n_cap,
                                     int* __restrict__ n_dev) {
    __shared__ long long warp_tot[32];
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int on = (v < V && out[2 * v] > zthr) ? 1 : 0;
    long long tot;
    const long long incl = sbp_block_incl_scan(on, warp_tot, tot);
    const long long q = off[blockIdx.x] + incl - on;
    if (on) {
        const int ix = (int)(v % g.n[0]), iy = (int)((v / g.n[0]) % g.n[1]);
        const int iz = (int)(v / ((long long)g.n[0] * g.n[1]));
        const float p = fminf(fmaxf(out[2 * v + 1], p_min), p_max);
        for (int j = 0; j < k; ++j) {
            const long long pos = q * k + j, c = 3 * (v * k + j);
            if (pos >= n_cap) break;
            balls.x[pos] = g.o[0] + ((float)ix + unit24(seed, c)) * g.h;
            balls.y[pos] = g.o[1] + ((float)iy + unit24(seed, c + 1)) * g.h;
            balls.z[pos] = g.o[2] + ((float)iz + unit24(seed, c + 2)) * g.h;
            balls.R[pos] = R;
            balls.p0[pos] = p;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        *n_dev = (int)min((long long)off[gridDim.x] * k, (long long)n_cap);
}

int blocks_for(long long n, int threads = 256, int cap = 4096) {
    return (int)std::max<long long>(1, std::min<long long>(cap, (n + threads - 1) / threads));
}

int check(sbp_cnn c, const char* what) {
    int dev = -1;
    if (!c) {
        sbp_set_error(std::string(what) + ": null cnn");
        return SBP_ERR_ARG;
    }
    if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device) {
        sbp_set_error(std::string(what) + ": the cnn belongs to another device");
        return SBP_ERR_ARG;
    }
    return SBP_OK;
}

int pack_all(sbp_cnn c, cudaStream_t st) {
    const float* P = c->p;
    pack_kernel<<<64, 256, 0, st>>>(P + kOW1, kC1, 1, padded_k(1), c->w1, 0, nullptr);
    pack_kernel<<<64, 256, 0, st>>>(P + kOW2, kC2, kC1, padded_k(kC1), c->w2, padded_k(kC2),
                                    c->w2t);
    pack_kernel<<<64, 256, 0, st>>>(P + kOW3, kC3, kC2, padded_k(kC2), c->w3, padded_k(kC3),
                                    c->w3t);
    sbp_count_launches(3);
    return sbp_cuda_check(cudaGetLastError(), "cnn: pack") ? SBP_ERR_CUDA : SBP_OK;
}

// input scaling and the three convolutions and the head
int forward(sbp_cnn c, const float* vol, cudaStream_t st) {
    const long long V = c->V;
    if (sbp_cuda_check(cudaMemsetAsync(c->vmax, 0, sizeof(unsigned int), st), "cnn: reset"))
        return SBP_ERR_CUDA;
    absmax_kernel<<<blocks_for(V), 256, 0, st>>>(vol, V, c->vmax);
    scale_input_kernel<<<blocks_for(V), 256, 0, st>>>(vol, V, c->vmax, c->x0);
    sbp_count_launches(2);
    // h1 and h2 are planar ([C / 8][V][8]): the next layer's TMA halo boxes
    // then have rows of ten voxels; h3 is channels-last for the head
    if (int e = sbp_conv3d_layout(c->x0, c->nx, c->ny, c->nz, 1, c->w1, padded_k(1), c->p + kOB1,
                                  kC1, 1, c->h1, 0, false, true, st))
        return e;
    if (int e = sbp_conv3d_layout(c->h1, c->nx, c->ny, c->nz, kC1, c->w2, padded_k(kC1),
                                  c->p + kOB2, kC2, 1, c->h2, 0, true, true, st))
        return e;
    if (int e = sbp_conv3d_layout(c->h2, c->nx, c->ny, c->nz, kC2, c->w3, padded_k(kC2),
                                  c->p + kOB3, kC3, 1, c->h3, 0, true, false, st))
        return e;
    head_fwd_kernel<<<blocks_for(V), 256, 0, st>>>(c->h3, V, c->p, c->out);
    sbp_count_launches(1);
    return sbp_cuda_check(cudaGetLastError(), "cnn: forward") ? SBP_ERR_CUDA : SBP_OK;
}

}  // namespace

extern "C" {

int sbp_das_volume(sbp_array arr, const float* y_full_dev, const double* origin3, double spacing,
                   int nx, int ny, int nz, float* vol_dev, sbp_stream stream) {
    if (!arr || !y_full_dev || !origin3 || !vol_dev || !(spacing > 0.0) || nx < 1 || ny < 1 ||
        nz < 1) {
        sbp_set_error("das_volume: invalid argument");
        return SBP_ERR_ARG;
    }
    VoxGeo g;
    for (int k = 0; k < 3; ++k) g.o[k] = (float)origin3[k];
    g.h = (float)spacing;
    g.n[0] = nx;
    g.n[1] = ny;
    g.n[2] = nz;
    const long long V = (long long)nx * ny * nz;
    const double cdt = arr->c / arr->fs;  // mm per sample at the full rate
    das_kernel<<<(unsigned)((V + kDasThreads - 1) / kDasThreads), kDasThreads, 0,
                 reinterpret_cast<cudaStream_t>(stream)>>>(y_full_dev, arr->M, arr->T, arr->d_sens,
                                                           (float)(1.0 / cdt), arr->wmode, g,
                                                           vol_dev);
    sbp_count_launches(1);
    return sbp_cuda_check(cudaGetLastError(), "das_volume launch") ? SBP_ERR_CUDA : SBP_OK;
}

int sbp_cnn_create(int nx, int ny, int nz, uint64_t seed, sbp_cnn* out) {
    if (!out || nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz > (1LL << 28)) {
        sbp_set_error("cnn_create: invalid argument");
        return SBP_ERR_ARG;
    }
    *out = nullptr;
    sbp_cnn c = new sbp_cnn_s();
    cudaGetDevice(&c->device);
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->V = (long long)nx * ny * nz;
    const size_t V = (size_t)c->V;
    bool ok = true;
    auto alloc = [&](void** p, size_t bytes) {
        ok = ok && !sbp_cuda_check(cudaMalloc(p, bytes), "cnn_create: alloc");
    };
    alloc((void**)&c->p, sizeof(float) * 4 * kParams);
    alloc((void**)&c->w1, 2 * (size_t)kC1 * padded_k(1));
    alloc((void**)&c->w2, 2 * (size_t)kC2 * padded_k(kC1));
    alloc((void**)&c->w3, 2 * (size_t)kC3 * padded_k(kC2));
    alloc((void**)&c->w2t, 2 * (size_t)kC1 * padded_k(kC2));
    alloc((void**)&c->w3t, 2 * (size_t)kC2 * padded_k(kC3));
    alloc((void**)&c->x0, 2 * V);
    alloc((void**)&c->h1, 2 * V * kC1);
    alloc((void**)&c->h2, 2 * V * kC2);
    alloc((void**)&c->h3, 2 * V * kC3);
    alloc((void**)&c->g3, 2 * V * kC3);
    alloc((void**)&c->g2, 2 * V * kC2);
    alloc((void**)&c->g1, 2 * V * kC1);
    alloc((void**)&c->out, sizeof(float) * 2 * V);
    alloc((void**)&c->dout, sizeof(float) * 2 * V);
    alloc((void**)&c->vmax, sizeof(unsigned int));
    alloc((void**)&c->loss, sizeof(double) * 2);
    {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        c->sms = sms > 0 ? sms : 1;
        const long long wg = std::max({sbp_wgrad_scratch_floats(nx, ny, nz, 1, kC1, c->sms),
                                       sbp_wgrad_scratch_floats(nx, ny, nz, kC1, kC2, c->sms),
                                       sbp_wgrad_scratch_floats(nx, ny, nz, kC2, kC3, c->sms)});
        alloc((void**)&c->wg_part, sizeof(float) * (size_t)wg);
        alloc((void**)&c->hd_part, sizeof(float) * (size_t)((V + 511) / 512) * (kWh + kBh));
    }
    if (!ok) {
        sbp_cnn_destroy(c);
        return SBP_ERR_CUDA;
    }
    // He-normal weights from SplitMix64 + Box-Muller, zero biases; zero Adam state
    std::vector<float> h(4 * (size_t)kParams, 0.0f);
    uint64_t k = 0;
    auto normal = [&]() {
        auto u01 = [&]() {
            uint64_t z = seed + (++k) * 0x9E3779B97F4A7C15ull;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        };
        const double a = u01(), b = u01();
        return std::sqrt(-2.0 * std::log(a)) * std::cos(6.283185307179586 * b);
    };
    auto fill = [&](int off, int n, double std_) {
        for (int i = 0; i < n; ++i) h[off + i] = (float)(normal() * std_);
    };
    fill(kOW1, kW1, std::sqrt(2.0 / 27.0));
    fill(kOW2, kW2, std::sqrt(2.0 / (27.0 * kC1)));
    fill(kOW3, kW3, std::sqrt(2.0 / (27.0 * kC2)));
    fill(kOWh, kWh, std::sqrt(1.0 / kC3));
    h[kOBh] = -2.0f;  // start from "mostly empty"
    if (sbp_cuda_check(cudaMemcpy(c->p, h.data(), sizeof(float) * h.size(),
                                  cudaMemcpyHostToDevice),
                       "cnn_create: copy") ||
        pack_all(c, 0) || sbp_cuda_check(cudaDeviceSynchronize(), "cnn_create: pack")) {
        sbp_cnn_destroy(c);
        return SBP_ERR_CUDA;
    }
    *out = c;
    return SBP_OK;
}

int sbp_cnn_destroy(sbp_cnn c) {
    if (!c) return SBP_OK;
    cudaDeviceSynchronize();
    void* ptrs[] = {c->p,  c->w1, c->w2, c->w3,  c->w2t, c->w3t, c->x0,   c->h1,   c->h2, c->h3,
                    c->g3, c->g2, c->g1, c->out, c->dout, c->vmax, c->loss, c->cnt,
                    c->wg_part, c->hd_part};
    for (void* q : ptrs) cudaFree(q);
    delete c;
    return SBP_OK;
}

int sbp_cnn_num_params(void) { return kParams; }

int sbp_cnn_params(sbp_cnn c, float* host, int set) {
    if (int e = check(c, "cnn_params")) return e;
    if (!host) {
        sbp_set_error("cnn_params: null pointer");
        return SBP_ERR_ARG;
    }
    if (sbp_cuda_check(cudaDeviceSynchronize(), "cnn_params: synchronise")) return SBP_ERR_CUDA;
    if (set) {
        if (sbp_cuda_check(cudaMemcpy(c->p, host, sizeof(float) * kParams, cudaMemcpyHostToDevice),
                           "cnn_params: copy") ||
            pack_all(c, 0) || sbp_cuda_check(cudaDeviceSynchronize(), "cnn_params: pack"))
            return SBP_ERR_CUDA;
        return SBP_OK;
    }
    return sbp_cuda_check(cudaMemcpy(host, c->p, sizeof(float) * kParams, cudaMemcpyDeviceToHost),
                          "cnn_params: copy")
               ? SBP_ERR_CUDA
               : SBP_OK;
}

int sbp_cnn_forward(sbp_cnn c, const float* vol_dev, float* out_dev, sbp_stream stream) {
    if (int e = check(c, "cnn_forward")) return e;
    if (!vol_dev) {
        sbp_set_error("cnn_forward: null volume");
        return SBP_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (int e = forward(c, vol_dev, st)) return e;
    if (out_dev &&
        sbp_cuda_check(cudaMemcpyAsync(out_dev, c->out, sizeof(float) * 2 * c->V,
                                       cudaMemcpyDeviceToDevice, st),
                       "cnn_forward: copy"))
        return SBP_ERR_CUDA;
    return SBP_OK;
}

namespace {

// Forward, loss and backward of one volume: every parameter's gradient is
// written (not accumulated) into the gradient block G = p + 3 kParams, in a
// fixed order of additions, and the two loss terms into c->loss.
int backward(sbp_cnn c, const float* vol_dev, const float* occ_dev, const float* p0_dev,
             float pos_weight, cudaStream_t st) {
    const long long V = c->V;
    const int nx = c->nx, ny = c->ny, nz = c->nz;
    if (int e = forward(c, vol_dev, st)) return e;
    if (sbp_cuda_check(cudaMemsetAsync(c->loss, 0, sizeof(double) * 2, st), "cnn: loss reset"))
        return SBP_ERR_CUDA;
    float* G = c->p + 3 * kParams;
    loss_kernel<<<blocks_for(V), 256, 0, st>>>(c->out, occ_dev, p0_dev, V, pos_weight, c->dout,
                                               c->loss);
    head_bwd_data_kernel<<<blocks_for(V * kC3), 256, 0, st>>>(c->h3, c->dout, V, c->p, c->g3);
    static_assert(kWh + kBh <= 256, "one thread per head parameter");
    const unsigned hb = (unsigned)((V + 511) / 512);
    head_bwd_param_kernel<<<hb, 256, 0, st>>>(c->h3, c->dout, V, 512, c->hd_part);
    head_param_reduce_kernel<<<1, 256, 0, st>>>(c->hd_part, (int)hb, G);
    sbp_count_launches(4);
    // conv3: weights (tensor cores), then the data gradient into g2 (masked by conv2's ReLU)
    // g3 is channels-last like h3; g2 and g1 are planar like h2 and h1
    if (int e = sbp_wgrad_bf16(c->g3, c->h2, nx, ny, nz, kC2, kC3, c->sms, c->wg_part, G + kOW3,
                               G + kOB3, true, false, st))
        return e;
    if (int e = sbp_conv3d_layout(c->g3, nx, ny, nz, kC3, c->w3t, padded_k(kC3), nullptr, kC2, 0,
                                  c->g2, 0, false, true, st))
        return e;
    relu_mask_kernel<<<blocks_for(V * kC2), 256, 0, st>>>(c->g2, c->h2, V * kC2);
    sbp_count_launches(1);
    if (int e = sbp_wgrad_bf16(c->g2, c->h1, nx, ny, nz, kC1, kC2, c->sms, c->wg_part, G + kOW2,
                               G + kOB2, true, true, st))
        return e;
    if (int e = sbp_conv3d_layout(c->g2, nx, ny, nz, kC2, c->w2t, padded_k(kC2), nullptr, kC1, 0,
                                  c->g1, 0, true, true, st))
        return e;
    relu_mask_kernel<<<blocks_for(V * kC1), 256, 0, st>>>(c->g1, c->h1, V * kC1);
    sbp_count_launches(1);
    if (int e = sbp_wgrad_bf16(c->g1, c->x0, nx, ny, nz, 1, kC1, c->sms, c->wg_part, G + kOW1,
                               G + kOB1, false, true, st))
        return e;
    return sbp_cuda_check(cudaGetLastError(), "cnn backward") ? SBP_ERR_CUDA : SBP_OK;
}

}  // namespace

int sbp_cnn_train_step(sbp_cnn c, const float* vol_dev, const float* occ_dev, const float* p0_dev,
                       float pos_weight, float lr, double* loss_dev, sbp_stream stream) {
    if (int e = check(c, "cnn_train_step")) return e;
    if (!vol_dev || !occ_dev || !p0_dev || !(lr > 0.f) || !(pos_weight > 0.f)) {
        sbp_set_error("cnn_train_step: invalid argument");
        return SBP_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (int e = backward(c, vol_dev, occ_dev, p0_dev, pos_weight, st)) return e;
    float* G = c->p + 3 * kParams;
    ++c->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)c->step), c2 = 1.0f - std::pow(b2, (float)c->step);
    adam_flat_kernel<<<64, 256, 0, st>>>(c->p, c->p + kParams, c->p + 2 * kParams, G, kParams, lr,
                                         b1, b2, 1e-8f, c1, c2);
    sbp_count_launches(1);
    if (int e = pack_all(c, st)) return e;
    if (loss_dev && sbp_cuda_check(cudaMemcpyAsync(loss_dev, c->loss, sizeof(double) * 2,
                                                   cudaMemcpyDeviceToDevice, st),
                                   "cnn: loss copy"))
        return SBP_ERR_CUDA;
    return sbp_cuda_check(cudaGetLastError(), "cnn_train_step") ? SBP_ERR_CUDA : SBP_OK;
}

int sbp_cnn_grad(sbp_cnn c, const float* vol_dev, const float* occ_dev, const float* p0_dev,
                 float pos_weight, double* loss_dev, float* grad_dev, sbp_stream stream) {
    if (int e = check(c, "cnn_grad")) return e;
    if (!vol_dev || !occ_dev || !p0_dev || !grad_dev || !(pos_weight > 0.f)) {
        sbp_set_error("cnn_grad: invalid argument");
        return SBP_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (int e = backward(c, vol_dev, occ_dev, p0_dev, pos_weight, st)) return e;
    if (sbp_cuda_check(cudaMemcpyAsync(grad_dev, c->p + 3 * kParams, sizeof(float) * kParams,
                                       cudaMemcpyDeviceToDevice, st),
                       "cnn_grad: copy"))
        return SBP_ERR_CUDA;
    if (loss_dev && sbp_cuda_check(cudaMemcpyAsync(loss_dev, c->loss, sizeof(double) * 2,
                                                   cudaMemcpyDeviceToDevice, st),
                                   "cnn_grad: loss copy"))
        return SBP_ERR_CUDA;
    return SBP_OK;
}

int sbp_cnn_propose(sbp_cnn c, const float* vol_dev, float prob_threshold, uint64_t seed,
                    const double* origin3, double spacing, float R, float p_min, float p_max,
                    int per_voxel, sbp_balls out, int n_cap, int* n_dev, sbp_stream stream) {
    if (int e = check(c, "cnn_propose")) return e;
    if (!vol_dev || !origin3 || !(spacing > 0.0) || !n_dev || n_cap < 0 || !out.x || !out.y ||
        !out.z || !out.R || !out.p0 || !(prob_threshold > 0.f && prob_threshold < 1.f) ||
        !(R > 0.f) || !(p_max >= p_min) || per_voxel < 1 || per_voxel > 4096) {
        sbp_set_error("cnn_propose: invalid argument");
        return SBP_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const long long V = c->V;
    const int nb = (int)((V + 255) / 256);
    if (c->cnt_cap < nb + 1) {
        if (sbp_cuda_check(cudaStreamSynchronize(st), "cnn_propose: synchronise")) return SBP_ERR_CUDA;
        cudaFree(c->cnt);
        c->cnt = nullptr;
        c->cnt_cap = 0;
        if (sbp_cuda_check(cudaMalloc(&c->cnt, sizeof(int) * (size_t)(nb + 1)), "cnn_propose: alloc"))
            return SBP_ERR_CUDA;
        c->cnt_cap = nb + 1;
    }
    if (int e = forward(c, vol_dev, st)) return e;
    const float zthr = std::log(prob_threshold / (1.0f - prob_threshold));
    VoxGeo g;
    for (int k = 0; k < 3; ++k) g.o[k] = (float)origin3[k];
    g.h = (float)spacing;
    g.n[0] = c->nx;
    g.n[1] = c->ny;
    g.n[2] = c->nz;
    propose_count_kernel<<<nb, 256, 0, st>>>(c->out, V, zthr, c->cnt);
    propose_scan_kernel<<<1, 1024, 0, st>>>(c->cnt, nb);
    propose_write_kernel<<<nb, 256, 0, st>>>(c->out, V, zthr, c->cnt, g, seed, R, p_min, p_max,
                                             per_voxel, out, n_cap, n_dev);
    sbp_count_launches(3);
    return sbp_cuda_check(cudaGetLastError(), "cnn_propose") ? SBP_ERR_CUDA : SBP_OK;
}

}  // extern "C"
