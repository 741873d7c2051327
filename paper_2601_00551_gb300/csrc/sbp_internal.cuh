// Internal declarations shared by the CUDA translation units of libslingbag.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "slingbag.h"

#define SBP_MAX_LEVELS 16
#define SBP_ADJ_CHUNK 128      // balls per Gaussian-adjoint CTA: the adjoint scratch's unit
#define SBP_ADJ_CHUNK_MAX 256  // balls per sphere-adjoint CTA, the largest chunk
#define SBP_ADJ_MAX_SPLIT 8  // most CTAs sharing one adjoint chunk
#define SBP_MAX_EXTRA 16
#define SBP_FG_ARRAYS (10 + SBP_MAX_EXTRA)

// Device-resident state of an array object: latched status and counters.
struct SbpDevState {
    int err;                          // first latched sbp_status (0 = none)
    unsigned int pmax_bits;           // bits of max |p0| seen by the forward pre-pass
    unsigned long long inside_pairs;  // pairs with d <= R skipped
    unsigned int loss_ticket;         // last-block ticket of the loss reduction
    int n_new;                        // result count of the last filter/grow
    int pad[2];
};

// Geometry of the current sampling level, passed by value to kernels.
struct LevelGeo {
    int M;         // sensors
    int Tk;        // samples at this level
    float h_hi;    // c * dt_k (mm per sample), float-float high part
    float h_lo;    //   ... low part
    float inv_h;   // 1 / h
    float inv_4h;  // 1 / (4 h)
    int wmode;     // SBP_W_*
    int pad;
};

struct BallsDev {
    const float* __restrict__ x;
    const float* __restrict__ y;
    const float* __restrict__ z;
    const float* __restrict__ R;
    const float* __restrict__ p0;
};

// Multi-frame layout. Frame f owns balls [ball_off[f], ball_off[f+1]) of the
// packed arrays (every frame's capacity is a multiple of kFrameAlign, so a
// chunk of up to kFrameAlign balls never straddles two frames) and traces
// [f*M*T_k, (f+1)*M*T_k); its live count is n_dev[f]. A single cloud is
// F = 1 with ball_off = null, capacity n_cap and count n_dev (may be null).
#define SBP_FRAME_ALIGN 1024
#define SBP_MAX_FRAMES 1024

struct FrameTable {
    int F;
    const int* __restrict__ ball_off;  // device, F + 1 entries, or null when F == 1
    const int* n_dev;                  // device, F entries (null: n = capacity)
    int n_cap;                         // capacity of the single cloud when ball_off is null
};

struct FrameSlot {
    int f;    // frame
    int off;  // first ball of the frame in the packed arrays
    int end;  // one past the frame's last live ball
};

// Frame of packed ball index `ball` (binary search over the frame offsets).
__device__ __forceinline__ FrameSlot sbp_frame_of(const FrameTable& ft, int ball) {
    FrameSlot s;
    if (ft.ball_off == nullptr) {
        s.f = 0;
        s.off = 0;
        int n = ft.n_dev ? *ft.n_dev : ft.n_cap;
        s.end = n < 0 ? 0 : (n > ft.n_cap ? ft.n_cap : n);
        return s;
    }
    int lo = 0, hi = ft.F;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (ft.ball_off[mid] <= ball) lo = mid;
        else hi = mid;
    }
    s.f = lo;
    s.off = ft.ball_off[lo];
    const int cap = ft.ball_off[lo + 1] - s.off;
    int n = ft.n_dev ? ft.n_dev[lo] : cap;
    n = n < 0 ? 0 : (n > cap ? cap : n);
    s.end = s.off + n;
    return s;
}

struct sbp_array_s {
    int device;
    int sm_count;
    int M, T, n_levels, n_cap, level;
    int factors[SBP_MAX_LEVELS];
    double c, fs;
    int wmode;
    // sensors on the device, structure of arrays [6][M]: sx, sy, sz, nx, ny, nz
    float* d_sens;
    // forward: fixed-point second-difference accumulators [frames][M][T_k] (int64)
    unsigned long long* d_acc;
    size_t acc_cells;
    // multi-frame layout (sbp_set_frames)
    int frames;
    int* d_frame_off;      // [frames + 1]
    int* h_frame_off;      // host copy
    int* d_frame_n_new;    // [frames] result counts of a frame-wise filter/grow
    unsigned int* d_frame_pmax;  // [frames] bits of max |p0| per frame (forward scale)
    double* d_frame_lossp; // [frames][loss blocks]
    // residual loss partials
    double* d_lossp;
    int loss_blocks;
    // filter/grow scratch
    int* d_fg_counts;  // block totals / offsets
    int fg_blocks;
    float* d_fg_buf;   // [SBP_FG_ARRAYS][n_cap]
    SbpDevState* d_state;
    // reconstruction scratch (allocated by the first sbp_reconstruct)
    float* d_rc_yk;     // [M][T]
    float* d_rc_S;      // [M][T]
    float* d_rc_G;      // [M][T]
    float* d_rc_state;  // [15][n_cap]: grads (5), Adam m (5), Adam v (5)
    // multi-frame reconstruction scratch ([frames][M][T] each)
    float* d_fr_yk;
    float* d_fr_S;
    float* d_fr_G;
    size_t fr_cells;
    // Gaussian-profile forward: boundary accumulators [M][T_k + 1] (int64)
    unsigned long long* d_gacc;
    size_t gauss_cells;
    int fwd_chunk_frames;  // forward balls per CTA chosen by sbp_autotune_frames (0: default)
    int adj_split_frames;  // adjoint CTAs per ball chunk chosen by sbp_autotune_frames (0: default)
    // single-cloud tiles per level chosen by sbp_autotune (0: default)
    int fwd_chunk_lvl[SBP_MAX_LEVELS];
    int adj_split_lvl[SBP_MAX_LEVELS];
    // adjoint: partial sums of the CTAs that split a chunk's sensors
    // [chunk][part][5][128] and one arrival ticket per chunk (left zero)
    float* d_adj_part;
    unsigned int* d_adj_ticket;
    int adj_chunks;  // chunks the two hold
    // spatial sort (allocated by its first use): keys and indices in and out
    // (4 n_cap words) and the box (8 words); the radix sort's temporary storage
    unsigned int* d_sort_keys;
    void* d_sort_tmp;
    size_t sort_tmp_bytes;
};

// ----------------------------------------------------------------------------
// host helpers (sbp_api.cu)
// ----------------------------------------------------------------------------
void sbp_set_error(const std::string& msg);
void sbp_count_launches(int k);  // adds k to the process-wide kernel launch count
int sbp_cuda_check(cudaError_t e, const char* what);
LevelGeo sbp_level_geo(const sbp_array_s* a, int k);
int sbp_level_T(const sbp_array_s* a, int k);

// ----------------------------------------------------------------------------
// launchers (one per translation unit family); each returns an sbp_status
// ----------------------------------------------------------------------------
// A forward tile value: a power of two in [32, SBP_FRAME_ALIGN] balls per
// CTA, optionally or'ed with SBP_TILE_WIDE.
bool sbp_fwd_tile_valid(int tile);
int sbp_launch_forward(sbp_array_s* a, const BallsDev& b, const int* n_dev, int n_cap,
                       float* S, cudaStream_t st);
int sbp_launch_residual(sbp_array_s* a, const float* S, const float* y, float* G,
                        double* loss, cudaStream_t st);
int sbp_launch_downsample(sbp_array_s* a, int k, const float* y_full, float* y_k,
                          cudaStream_t st);
int sbp_launch_adjoint(sbp_array_s* a, const BallsDev& b, const int* n_dev, int n_cap,
                       const float* G, sbp_grads out, unsigned mask, cudaStream_t st);
int sbp_launch_filter_grow(sbp_array_s* a, sbp_balls balls, sbp_grads grads,
                           float* const* extra, int n_extra, int* n_dev, int n_cap,
                           const sbp_grow_params* gp, int mode, cudaStream_t st);
int sbp_launch_adam(sbp_array_s* a, sbp_balls balls, sbp_grads grads, sbp_balls m,
                    sbp_balls v, const int* n_dev, int n_cap, int t,
                    const sbp_adam_params* ap, unsigned mask, cudaStream_t st);
// the same over every frame of the packed layout of sbp_set_frames
int sbp_launch_forward_frames(sbp_array_s* a, const BallsDev& b, const int* n_dev, float* S,
                              int chunk, cudaStream_t st);
int sbp_launch_residual_frames(sbp_array_s* a, const float* S, const float* y, float* G,
                               double* loss, cudaStream_t st);
int sbp_launch_adjoint_frames(sbp_array_s* a, const BallsDev& b, const int* n_dev,
                              const float* G, sbp_grads out, unsigned mask, cudaStream_t st);
int sbp_launch_filter_grow_frames(sbp_array_s* a, sbp_balls balls, sbp_grads grads,
                                  float* const* extra, int n_extra, int* n_dev,
                                  const sbp_grow_params* gp, int mode, cudaStream_t st);
int sbp_launch_adam_frames(sbp_array_s* a, sbp_balls balls, sbp_grads grads, sbp_balls m,
                           sbp_balls v, const int* n_dev, int t, const sbp_adam_params* ap,
                           unsigned mask, cudaStream_t st);
int sbp_launch_downsample_rows(sbp_array_s* a, int k, int rows, const float* y_full,
                               float* y_k, cudaStream_t st);

// Morton order of the live balls of a single cloud, carrying `nrows` float
// rows (the five ball rows first, then any state) through the permutation
// (sbp_sort.cu); nrows <= SBP_FG_ARRAYS.
int sbp_launch_sort(sbp_array_s* a, float* const* rows, int nrows, const int* n_dev, int n_cap,
                    cudaStream_t st);

// Stored-window forward records and the adjoint that reads them (sbp_stored.cu):
// rec_dev holds five [M][n_cap] planes of 4-byte words.
int sbp_launch_store_windows(sbp_array_s* a, const BallsDev& b, const int* n_dev, int n_cap,
                             void* rec_dev, cudaStream_t st);
int sbp_launch_adjoint_stored(sbp_array_s* a, const BallsDev& b, const int* n_dev, int n_cap,
                              const void* rec_dev, const float* G, sbp_grads out, unsigned mask,
                              cudaStream_t st);

// weight gradient of the proposal CNN's convolutions on the tensor cores (sbp_cnn.cu)
long long sbp_wgrad_scratch_floats(int nx, int ny, int nz, int cin, int cout, int sms);
// The 3x3x3 convolution of sbp_conv3d_bf16 with a choice of activation
// layouts: channels-last [V][C] or planar [C / 8][V][8] for the input (Cin a
// multiple of 8, read by the TMA kernel only) and the bf16 output (Cout a
// multiple of 16).
int sbp_conv3d_layout(const void* in_dev, int nx, int ny, int nz, int cin, const void* w_dev,
                      int kp, const float* bias_dev, int cout, int relu, void* out_dev,
                      int out_f32, bool in_planar, bool out_planar, cudaStream_t st);
// x and g are channels-last or planar (x_planar, g_planar; Cin = 1 is [V]).
int sbp_wgrad_bf16(const void* g_dev, const void* x_dev, int nx, int ny, int nz, int cin,
                   int cout, int sms, float* partial, float* dW, float* db, bool x_planar,
                   bool g_planar, cudaStream_t st);

// ----------------------------------------------------------------------------
// device helpers
// ----------------------------------------------------------------------------

__device__ __forceinline__ int sbp_read_n(const int* n_dev, int n_cap) {
    if (!n_dev) return n_cap;
    int n = *n_dev;
    return n < 0 ? 0 : (n > n_cap ? n_cap : n);
}

// Error-free transforms (Knuth's TwoSum, Dekker's FastTwoSum and the FMA
// product error): a + b = s + e and a * b = p + e exactly.
__device__ __forceinline__ void ff_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void ff_fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// Distance from sensor to ball centre as an unevaluated sum dh + dl that is
// accurate to ~1e-13 relative, plus the rounded difference vector and 1/dh.
// The difference of the float32 coordinates is taken exactly (TwoSum), the
// squared norm in float-float, and the square root is corrected once.
struct PairDist {
    float dh, dl;      // d = dh + dl
    float dx, dy, dz;  // c - s rounded to float
    float rd;          // ~1/dh (relative error ~1e-7)
};

__device__ __forceinline__ PairDist sbp_pair_distance(float cx, float cy, float cz, float sx,
                                                      float sy, float sz) {
    PairDist p;
    float ex, ey, ez;
    ff_two_sum(cx, -sx, p.dx, ex);
    ff_two_sum(cy, -sy, p.dy, ey);
    ff_two_sum(cz, -sz, p.dz, ez);
    const float qx = __fmul_rn(p.dx, p.dx), rx = fmaf(p.dx, p.dx, -qx);
    const float qy = __fmul_rn(p.dy, p.dy), ry = fmaf(p.dy, p.dy, -qy);
    const float qz = __fmul_rn(p.dz, p.dz), rz = fmaf(p.dz, p.dz, -qz);
    float s1, e1, s2, e2;
    ff_two_sum(qx, qy, s1, e1);
    ff_two_sum(s1, qz, s2, e2);
    // cross terms 2 * dx * ex (the ex^2 terms are below 1e-20 relative)
    float lo = (rx + ry) + (rz + (e1 + e2));
    lo = fmaf(2.0f * p.dx, ex, lo);
    lo = fmaf(2.0f * p.dy, ey, lo);
    lo = fmaf(2.0f * p.dz, ez, lo);
    float Sh, Sl;
    ff_fast_two_sum(s2, lo, Sh, Sl);
    const float rs = rsqrtf(Sh);
    p.dh = __fmul_rn(Sh, rs);
    const float res = fmaf(-p.dh, p.dh, Sh) + Sl;  // Sh + Sl - dh^2
    p.rd = rs;
    p.dl = res * 0.5f * rs;
    return p;
}

// ----------------------------------------------------------------------------
// Two pairs at once. Blackwell issues the FP32 add, multiply and fused
// multiply-add of both halves of a float2 as one instruction, so a thread
// that evaluates two pairs side by side spends half the issue slots on their
// floating-point arithmetic. Every operation below rounds each half exactly
// as its scalar counterpart does, so a pair's result does not depend on
// which half it was evaluated in.
// ----------------------------------------------------------------------------

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b: b * (-1) + a rounds once, to the same value as the subtraction
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) {
    return __ffma2_rn(a, b, c);
}
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ void ff2_two_sum(float2 a, float2 b, float2& s, float2& e) {
    s = f2add(a, b);
    const float2 bb = f2sub(s, a);
    e = f2add(f2sub(a, f2sub(s, bb)), f2sub(b, bb));
}

struct PairDist2 {
    float2 dh, dl;      // d = dh + dl, per half
    float2 dx, dy, dz;  // c - s rounded to float
    float2 rd;          // ~1/dh
};

// sbp_pair_distance for two (ball, sensor) pairs; every half equals the
// scalar result bit for bit.
__device__ __forceinline__ PairDist2 sbp_pair_distance2(float2 cx, float2 cy, float2 cz,
                                                        float2 sx, float2 sy, float2 sz) {
    PairDist2 p;
    float2 ex, ey, ez;
    ff2_two_sum(cx, f2neg(sx), p.dx, ex);
    ff2_two_sum(cy, f2neg(sy), p.dy, ey);
    ff2_two_sum(cz, f2neg(sz), p.dz, ez);
    const float2 qx = f2mul(p.dx, p.dx), rx = f2fma(p.dx, p.dx, f2neg(qx));
    const float2 qy = f2mul(p.dy, p.dy), ry = f2fma(p.dy, p.dy, f2neg(qy));
    const float2 qz = f2mul(p.dz, p.dz), rz = f2fma(p.dz, p.dz, f2neg(qz));
    float2 s1, e1, s2, e2;
    ff2_two_sum(qx, qy, s1, e1);
    ff2_two_sum(s1, qz, s2, e2);
    float2 lo = f2add(f2add(rx, ry), f2add(rz, f2add(e1, e2)));
    lo = f2fma(f2add(p.dx, p.dx), ex, lo);
    lo = f2fma(f2add(p.dy, p.dy), ey, lo);
    lo = f2fma(f2add(p.dz, p.dz), ez, lo);
    const float2 Sh = f2add(s2, lo);
    const float2 Sl = f2sub(lo, f2sub(Sh, s2));
    const float2 rs = make_float2(rsqrtf(Sh.x), rsqrtf(Sh.y));
    p.dh = f2mul(Sh, rs);
    const float2 res = f2add(f2fma(f2neg(p.dh), p.dh, Sh), Sl);
    p.rd = rs;
    p.dl = f2mul(f2mul(res, f2(0.5f)), rs);
    return p;
}

// The same in plain float (relative error ~1e-7 of d; dl = 0), for results
// that are continuous in the distance.
__device__ __forceinline__ PairDist2 sbp_pair_distance2_f32(float2 cx, float2 cy, float2 cz,
                                                            float2 sx, float2 sy, float2 sz) {
    PairDist2 p;
    p.dx = f2sub(cx, sx);
    p.dy = f2sub(cy, sy);
    p.dz = f2sub(cz, sz);
    const float2 q = f2fma(p.dx, p.dx, f2fma(p.dy, p.dy, f2mul(p.dz, p.dz)));
    p.rd = make_float2(rsqrtf(q.x), rsqrtf(q.y));
    p.dh = f2mul(q, p.rd);
    p.dl = f2(0.0f);
    return p;
}

// Offset of cell boundary j from the wave front: b_j = d - j h, evaluated as
// (dh - j h_hi) + (dl - err(j h_hi) - j h_lo); the first difference is exact
// when j h_hi lies within a factor of two of dh.
__device__ __forceinline__ float sbp_boundary(float dh, float dl, int j, float h_hi,
                                              float h_lo) {
    const float jf = (float)j;
    const float p = __fmul_rn(jf, h_hi);
    const float pe = fmaf(jf, h_hi, -p);
    const float t = __fsub_rn(dh, p);
    return t + ((dl - pe) - jf * h_lo);
}

// Cell boundaries of a pair inside the support: jL = min{j : b_j < R} and
// jH = max{j : b_j > -R}, b_j = d - j h. The offset e = d - jr h of one
// reference boundary jr = floor(d / h) is taken in float-float; every other
// boundary is b_j = e - (j - jr) h with a small integer j - jr, so the window
// and its end offsets b0 = b_jL, bL = b_jH follow from small-magnitude float
// arithmetic (abs. error ~1e-8 mm) and are then checked against R directly.
// Returns false when no boundary lies inside the support (every cell
// integral is zero), when the sensor is inside the ball (d <= R), or when the
// first touched cell jL - 1 is past the record.
struct PairWindow {
    int jL, jH;
    float b0, bL;
};

// The window of two pairs at once. For each: jr = floor(d / h), the offset
// e = b_jr taken in float-float (sbp_boundary), then jL and jH from small
// integer steps kL and kH carried as exact floats (below 2^24), and the end
// offsets b0 = e - kL h and bL = e - kH h, each rounded once (one FMA).
// kL is the first step with b0 < R, kH the last with bL > -R, both decided
// on those float offsets. The estimates kL = floor((e - R) / h - kBias) + 1
// and kH = ceil((e + R) / h + kBias) - 1 are biased so that each is the
// answer or one step short of it on one known side (kL below, kH above):
// the bias of 2^-10 cells exceeds the rounding error of (e -+ R) / h, about
// 3 |e -+ R| / h 2^-24 cells, for windows shorter than 2^11 cells. One
// comparison per end then settles it. Where the float offset lands exactly
// on +-R the cell it drops or keeps contributes zero, so either choice gives
// the same cell values. Valid when d > R, the far end lies inside the record
// and jH >= jL >= 1; pairs whose window is not valid (ok = false) may carry
// any values.
__device__ __forceinline__ void sbp_window2(float2 dh, float2 dl, float2 R, const LevelGeo& g,
                                            PairWindow& wa, PairWindow& wb, bool& okA,
                                            bool& okB) {
    constexpr float kBias = 0.0009765625f;  // 2^-10 cells
    const float h = g.h_hi;
    const float2 xr = f2mul(dh, f2(g.inv_h));
    const float2 dd = f2add(dh, dl);
    const float lim = (float)g.Tk + 4096.0f;
    okA = xr.x < lim && dd.x > R.x;  // also false for NaN
    okB = xr.y < lim && dd.y > R.y;
    const float2 jr = make_float2(floorf(xr.x), floorf(xr.y));
    // b_jr = (dh - jr h_hi) + (dl - err(jr h_hi) - jr h_lo)
    const float2 p = f2mul(jr, f2(g.h_hi));
    const float2 pe = f2fma(jr, f2(g.h_hi), f2neg(p));
    const float2 e = f2add(f2sub(dh, p), f2sub(f2sub(dl, pe), f2mul(jr, f2(g.h_lo))));
    const float2 tL = f2fma(f2sub(e, R), f2(g.inv_h), f2(-kBias));
    const float2 tH = f2fma(f2add(e, R), f2(g.inv_h), f2(kBias));
    float2 kL = f2add(make_float2(floorf(tL.x), floorf(tL.y)), f2(1.0f));
    float2 kH = f2add(make_float2(ceilf(tH.x), ceilf(tH.y)), f2(-1.0f));
    const float2 b0t = f2fma(kL, f2(-h), e);
    const float2 bLt = f2fma(kH, f2(-h), e);
    kL = f2add(kL, make_float2(b0t.x >= R.x ? 1.0f : 0.0f, b0t.y >= R.y ? 1.0f : 0.0f));
    kH = f2add(kH, make_float2(bLt.x <= -R.x ? -1.0f : 0.0f, bLt.y <= -R.y ? -1.0f : 0.0f));
    const float2 b0 = f2fma(kL, f2(-h), e);
    const float2 bL = f2fma(kH, f2(-h), e);
    const float2 jL = f2add(jr, kL), jH = f2add(jr, kH);
    okA = okA && jH.x >= jL.x && jL.x >= 1.0f && jL.x <= (float)g.Tk;
    okB = okB && jH.y >= jL.y && jL.y >= 1.0f && jL.y <= (float)g.Tk;
    wa.jL = __float2int_rz(jL.x);
    wa.jH = __float2int_rz(jH.x);
    wb.jL = __float2int_rz(jL.y);
    wb.jH = __float2int_rz(jH.y);
    wa.b0 = b0.x;
    wa.bL = bL.x;
    wb.b0 = b0.y;
    wb.bL = bL.y;
}

// Orientation weight and its switch (1 where d w / d c is non-zero).
__device__ __forceinline__ float sbp_weight(int wmode, float cosv, float& active) {
    if (wmode == SBP_W_NONE) {
        active = 0.0f;
        return 1.0f;
    }
    if (wmode == SBP_W_COS) {
        active = 1.0f;
        return cosv;
    }
    active = cosv > 0.0f ? 1.0f : 0.0f;
    return fmaxf(cosv, 0.0f);
}

// Bounding box of the centres of balls [c0, c1) and their largest radius,
// reduced over the block: box[0..2] = min, box[3..5] = max, box[6] = max R.
// `red` needs 7 floats per warp of shared memory. Contains __syncthreads()
// and must be reached by every thread of the block.
__device__ __forceinline__ void sbp_chunk_box(const BallsDev& b, int c0, int c1, float* red,
                                              float* box) {
    const float inf = __int_as_float(0x7f800000);
    float v[7] = {inf, inf, inf, -inf, -inf, -inf, -inf};
    for (int i = c0 + (int)threadIdx.x; i < c1; i += blockDim.x) {
        const float x = b.x[i], y = b.y[i], z = b.z[i], R = b.R[i];
        v[0] = fminf(v[0], x);
        v[1] = fminf(v[1], y);
        v[2] = fminf(v[2], z);
        v[3] = fmaxf(v[3], x);
        v[4] = fmaxf(v[4], y);
        v[5] = fmaxf(v[5], z);
        v[6] = fmaxf(v[6], R);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] = fminf(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
#pragma unroll
        for (int k = 3; k < 7; ++k) v[k] = fmaxf(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 7; ++k) red[wid * 7 + k] = v[k];
    __syncthreads();
    if (threadIdx.x < 7) {
        const int k = threadIdx.x, nw = (blockDim.x + 31) >> 5;
        float r = red[k];
        for (int w = 1; w < nw; ++w) r = k < 3 ? fminf(r, red[w * 7 + k]) : fmaxf(r, red[w * 7 + k]);
        box[k] = r;
    }
    __syncthreads();
}

// Cells [jlo, jhi] (clipped to the record) that any pair of the sensor at
// (sx, sy, sz) and a ball of the box can touch: the first touched cell jL-1
// and the last impulse jH+2 of every such pair lie inside. Empty when
// jhi < jlo. The bound uses the nearest and farthest points of the box and
// the largest radius, with two cells of slack for float rounding.
__device__ __forceinline__ void sbp_box_cells(float sx, float sy, float sz, const float* box,
                                              const LevelGeo& g, int& jlo, int& jhi) {
    const float ex = fmaxf(fmaxf(box[0] - sx, sx - box[3]), 0.0f);
    const float ey = fmaxf(fmaxf(box[1] - sy, sy - box[4]), 0.0f);
    const float ez = fmaxf(fmaxf(box[2] - sz, sz - box[5]), 0.0f);
    const float fx = fmaxf(fabsf(sx - box[0]), fabsf(sx - box[3]));
    const float fy = fmaxf(fabsf(sy - box[1]), fabsf(sy - box[4]));
    const float fz = fmaxf(fabsf(sz - box[2]), fabsf(sz - box[5]));
    const float dmin = sqrtf(ex * ex + ey * ey + ez * ez);
    const float dmax = sqrtf(fx * fx + fy * fy + fz * fz);
    const float Rm = fmaxf(box[6], 0.0f);
    float lo = floorf((dmin - Rm) * g.inv_h) - 2.0f;
    float hi = ceilf((dmax + Rm) * g.inv_h) + 3.0f;
    lo = fminf(fmaxf(lo, 0.0f), (float)g.Tk);
    hi = fminf(fmaxf(hi, -1.0f), (float)g.Tk - 1.0f);
    jlo = (int)lo;
    jhi = (int)hi;
}

__device__ __forceinline__ void sbp_latch(SbpDevState* st, int code) {
    atomicCAS(&st->err, 0, code);
}
