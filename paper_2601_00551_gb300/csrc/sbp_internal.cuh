// Internal declarations shared by the CUDA translation units of libslingbag.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "slingbag.h"

#define SBP_MAX_LEVELS 16
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

struct sbp_array_s {
    int device;
    int sm_count;
    int M, T, n_levels, n_cap, level;
    int factors[SBP_MAX_LEVELS];
    double c, fs;
    int wmode;
    // sensors on the device, structure of arrays [6][M]: sx, sy, sz, nx, ny, nz
    float* d_sens;
    // forward: fixed-point second-difference accumulators [M][T_k] (int64)
    unsigned long long* d_acc;
    // adjoint: per-sensor prefix records [M][T_k + 1] of (sum G, sum j G), int64
    longlong2* d_rec;
    int* d_gq;      // [M][T_k] G rounded to fixed point (int32)
    float* d_ginv;  // [M] 2^-s, the inverse quantisation scale of G per sensor
    // adjoint partial gradients when sensors are split across CTAs: [groups][5][n_cap]
    float* d_part;
    int part_groups;
    // residual loss partials
    double* d_lossp;
    int loss_blocks;
    // filter/grow scratch
    int* d_fg_counts;  // block totals / offsets
    int fg_blocks;
    float* d_fg_buf;   // [SBP_FG_ARRAYS][n_cap]
    SbpDevState* d_state;
};

// ----------------------------------------------------------------------------
// host helpers (sbp_api.cu)
// ----------------------------------------------------------------------------
void sbp_set_error(const std::string& msg);
int sbp_cuda_check(cudaError_t e, const char* what);
LevelGeo sbp_level_geo(const sbp_array_s* a, int k);
int sbp_level_T(const sbp_array_s* a, int k);

// ----------------------------------------------------------------------------
// launchers (one per translation unit family); each returns an sbp_status
// ----------------------------------------------------------------------------
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
// jH = max{j : b_j > -R}, b_j = d - j h. A float32 estimate of (d -+ R)/h is
// good to ~1e-3 cells; when it falls within 2e-3 of an integer the decision is
// taken on the float-float offsets b_j instead, so the window agrees with an
// exact evaluation except within ~1e-9 mm of a kink (where the loss is not
// differentiable anyway). Returns false when no boundary lies inside the
// support (every cell integral is then zero) or the window starts beyond
// the record. jH is capped near Tk + 3: boundaries past the record are never
// stored or read. b0 = b_jL; bL = b_jH only when want_bL.
struct PairWindow {
    int jL, jH;
    float b0, bL;
};

__device__ __forceinline__ bool sbp_window(const PairDist& pd, float R, const LevelGeo& g,
                                           bool want_bL, PairWindow& w) {
    const int Tk = g.Tk;
    const float dli = pd.dl * g.inv_h;
    const float xlo = fmaf(pd.dh - R, g.inv_h, dli);
    if (!(xlo < (float)Tk + 1.0f)) return false;  // also rejects NaN
    const float flo = floorf(xlo);
    int jL = max(1, (int)flo + 1);
    float b0 = sbp_boundary(pd.dh, pd.dl, jL, g.h_hi, g.h_lo);
    const float rlo = xlo - flo;
    if (rlo < 2e-3f || rlo > 1.0f - 2e-3f) {
        if (b0 >= R) {
            ++jL;
            b0 = sbp_boundary(pd.dh, pd.dl, jL, g.h_hi, g.h_lo);
        } else if (jL > 1) {
            const float bp = sbp_boundary(pd.dh, pd.dl, jL - 1, g.h_hi, g.h_lo);
            if (bp < R) {
                --jL;
                b0 = bp;
            }
        }
    }
    if (jL - 1 >= Tk) return false;
    // clamped to [-1, Tk + 4] so that jH + 2 stays far from int overflow
    const float xhi = fmaxf(fminf(fmaf(pd.dh + R, g.inv_h, dli), (float)Tk + 4.0f), -1.0f);
    const float chi = ceilf(xhi);
    int jH = (int)chi - 1;
    float bL = 0.0f;
    const float rhi = chi - xhi;
    const bool near = (rhi < 2e-3f || rhi > 1.0f - 2e-3f) && jH < Tk + 2;
    if (near || want_bL) bL = sbp_boundary(pd.dh, pd.dl, jH, g.h_hi, g.h_lo);
    if (near) {
        if (bL <= -R) {
            --jH;
            bL = sbp_boundary(pd.dh, pd.dl, jH, g.h_hi, g.h_lo);
        } else {
            const float bn = sbp_boundary(pd.dh, pd.dl, jH + 1, g.h_hi, g.h_lo);
            if (bn > -R) {
                ++jH;
                bL = bn;
            }
        }
    }
    if (jH < jL) return false;
    w.jL = jL;
    w.jH = jH;
    w.b0 = b0;
    w.bL = bL;
    return true;
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

__device__ __forceinline__ void sbp_latch(SbpDevState* st, int code) {
    atomicCAS(&st->err, 0, code);
}
