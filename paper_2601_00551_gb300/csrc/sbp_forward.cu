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
//   fwd_group     CTA = (group of 32 sensors) x (chunk of consecutive balls).
//                 A warp takes one ball at a time and its 32 lanes take the 32
//                 sensors, so ball data is warp-uniform and every lane keeps
//                 its sensor in registers. The cells a chunk can touch at a
//                 sensor are bounded from the chunk's bounding box; each
//                 lane's window is privatised in shared memory laid out
//                 [cell][lane], so the shared atomics of a warp never
//                 conflict on a bank, and flushed once per CTA to the global
//                 int64 accumulators with global atomics. Where a window is
//                 longer than the shared buffer, the impulses past its end
//                 go straight to the global accumulators.
//                 Two shapes: narrow (416 cells per sensor, 16 warps, two
//                 CTAs per SM) and wide (832 cells, 32 warps, one CTA per
//                 SM). The flush costs about one global atomic per window
//                 cell, i.e. (window cells) / (balls per chunk) per pair, and
//                 the window grows with the chunk's extent in cells; at the
//                 finest sampling rates the wide shape lets a chunk of 2048
//                 balls keep its window on chip where the narrow one spills.
//                 A 64-bit shared atomic add costs several times a 32-bit one
//                 on this GPU, so each int64 impulse v is added as two 32-bit
//                 words: v mod 2^32 and v >> kLoBits (signed). The sum of the
//                 low kLoBits-bit parts (at most 2 impulses per ball and
//                 cell, at most kMaxChunk balls) stays below 2^32, so the
//                 flush recovers it from the first word and the high word
//                 and recombines the sum exactly. The high word is a signed
//                 32-bit sum of v >> kLoBits: with K h R 2^F < 2^32 R / d
//                 (F below) every impulse is below K h (10 R + 3 h) 2^F in
//                 magnitude, so 2 kMaxChunk of them overflow it only for a
//                 ball within (10 R + 3 h) / 64 of a sensor.
//   fwd_finalize  CTA = one sensor; two block scans turn impulses into the
//                 float32 trace and clear the accumulator row
#include <algorithm>
#include <cuda.h>
#include <mutex>

#include "sbp_internal.cuh"
#include "sbp_scan.cuh"

namespace {

constexpr int kWarpsNarrow = 16;    // warps per forward CTA, narrow shape
constexpr int kWindowNarrow = 416;  // cells per sensor held in shared memory, narrow shape
constexpr int kWarpsWide = 32;      // the same for the wide shape
constexpr int kWindowWide = 832;
constexpr int kChunk = 512;         // default number of balls per CTA
constexpr int kMaxChunk = 2 * SBP_FRAME_ALIGN;  // largest (single cloud; frames: SBP_FRAME_ALIGN)
constexpr int kLoBits = 19;         // 2 * kMaxChunk * 2^kLoBits <= 2^32
static_assert(2LL * kMaxChunk * ((1LL << kLoBits) - 1) < (1LL << 32), "low word could overflow");
constexpr int kFinalizeThreads = 1024;
constexpr int kFracHeadroomBits = 34;  // F = 34 - ceil(log2 max|p0|)

// pmax[f] = max |p0| over frame f (grid.y = frame). A live ball with a
// non-finite coordinate, radius or pressure latches SBP_ERR_NUMERIC (its
// pairs would otherwise be dropped silently: fmaxf ignores a NaN p0).
__global__ void fwd_pmax_kernel(BallsDev b, FrameTable ft, unsigned int* __restrict__ pmax,
                                SbpDevState* st) {
    const int f = blockIdx.y;
    const FrameSlot fs = sbp_frame_of(ft, ft.ball_off ? ft.ball_off[f] : 0);
    float m = 0.0f;
    bool bad = false;
    for (int i = fs.off + blockIdx.x * blockDim.x + threadIdx.x; i < fs.end;
         i += gridDim.x * blockDim.x) {
        const float p = b.p0[i];
        // x * 0 is 0 for every finite x and NaN for an infinity or a NaN
        const float z = (b.x[i] + b.y[i] + b.z[i] + b.R[i] + p) * 0.0f;
        bad |= z != 0.0f;
        m = fmaxf(m, fabsf(p));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(&pmax[f], __float_as_uint(m));
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) sbp_latch(st, SBP_ERR_NUMERIC);
}

// Round a float to the nearest int64. Values below 2^31 in magnitude (nearly
// all of them) take one 32-bit conversion; larger ones are split exactly
// into two 32-bit halves. (A direct float -> int64 conversion would run on
// the double-precision pipe, which is narrow on this GPU.)
__device__ __forceinline__ long long fwd_f2ll(float x) {
    const float ax = fabsf(x);
    if (ax < 2147483520.0f) return (long long)__float2int_rn(x);  // largest float < 2^31
    const float hi = floorf(ax * 2.3283064365386963e-10f);          // |x| / 2^32
    const float rem = fmaf(-hi, 4294967296.0f, ax);                 // exact, in [0, 2^32)
    const long long v = ((long long)__float2uint_rz(hi) << 32) + (long long)__float2uint_rn(rem);
    return x < 0.0f ? -v : v;
}

// Adds the int64 impulse v to the split accumulator word pair at `lo` (the
// high word sits WIN * 32 words further on).
template <int WIN>
__device__ __forceinline__ void fwd_add(unsigned int* lo, long long v) {
    atomicAdd(lo, (unsigned int)v);
    atomicAdd(lo + WIN * 32, (unsigned int)(int)(v >> kLoBits));
}

// The same for an impulse that fits in 32 bits (its arithmetic shift gives
// the same high word as the 64-bit one).
template <int WIN>
__device__ __forceinline__ void fwd_add32(unsigned int* lo, int v) {
    atomicAdd(lo, (unsigned int)v);
    atomicAdd(lo + WIN * 32, (unsigned int)(v >> kLoBits));
}

// Adds one pair's six second-difference impulses to the lane's column of the
// split accumulator: three at cells ra .. ra+2 (relative to the lane's first
// window cell) from the first-cell, ramp and slope coefficients fa, f1, f2,
// three at rb .. rb+2 from the last-cell coefficient fe, with L = jH - jL
// ramp cells. Cells in [0, lim] are held in shared memory; other cells
// inside the record (relative cells -base .. glim) are added straight to the
// lane's global accumulator row grow (indexed relative to the window start);
// cells past the record are dropped (they cannot reach a stored sample).
template <int WIN>
__device__ __forceinline__ void fwd_emit(unsigned int* col, unsigned long long* grow, int ra,
                                         int rb, int L, int lim, int base, int glim, float fa,
                                         float fe, float f1, float f2) {
    const bool fast_a = ra >= 0 && ra + 2 <= lim, fast_b = rb >= 0 && rb + 2 <= lim;
    // impulses are sums of at most four coefficient terms; below 2^28 each
    // they fit in 32 bits (the usual case)
    const float big = fmaxf(fmaxf(fabsf(fa), fabsf(fe)), fmaxf(fabsf(f1), fabsf(f2) * (float)(L + 2)));
    if (big < 268435456.0f && fast_a && fast_b) {
        const int qa = __float2int_rn(fa), qe = __float2int_rn(fe);
        const int q1 = __float2int_rn(f1), q2 = __float2int_rn(f2);
        const int Lq2 = L * q2;
        unsigned int* a = col + ra * 32;
        fwd_add32<WIN>(a, qa);
        fwd_add32<WIN>(a + 32, q1 - 2 * qa);
        fwd_add32<WIN>(a + 64, qa - q1 + q2);
        unsigned int* c = col + rb * 32;
        fwd_add32<WIN>(c, qe - q1 - Lq2);
        fwd_add32<WIN>(c + 32, q1 + Lq2 - q2 - 2 * qe);
        fwd_add32<WIN>(c + 64, qe);
        return;
    }
    const long long qa = fwd_f2ll(fa), qe = fwd_f2ll(fe);
    const long long q1 = fwd_f2ll(f1), q2 = fwd_f2ll(f2);
    const long long Lq2 = (long long)L * q2;
    // second difference of the pair's cell values: three impulses at
    // jL-1 .. jL+1 and three at jH .. jH+2 (valid for every jH >= jL; when
    // the two triples overlap the impulses add up)
    const long long ia0 = qa, ia1 = q1 - 2 * qa, ia2 = qa - q1 + q2;
    const long long ib0 = qe - q1 - Lq2, ib1 = q1 + Lq2 - q2 - 2 * qe, ib2 = qe;
    auto put = [&](int r, long long v) {
        if (r >= 0 && r <= lim)
            fwd_add<WIN>(col + r * 32, v);
        else if (r >= -base && r <= glim)
            atomicAdd(grow + r, (unsigned long long)v);
    };
    if (fast_a) {
        unsigned int* a = col + ra * 32;
        fwd_add<WIN>(a, ia0);
        fwd_add<WIN>(a + 32, ia1);
        fwd_add<WIN>(a + 64, ia2);
    } else {
        put(ra, ia0);
        put(ra + 1, ia1);
        put(ra + 2, ia2);
    }
    if (fast_b) {
        unsigned int* c = col + rb * 32;
        fwd_add<WIN>(c, ib0);
        fwd_add<WIN>(c + 32, ib1);
        fwd_add<WIN>(c + 64, ib2);
    } else {
        put(rb, ib0);
        put(rb + 1, ib1);
        put(rb + 2, ib2);
    }
}

// Fixed-point exponent F: values are stored as round(v * 2^F).
__device__ __forceinline__ int fwd_frac_bits(unsigned int pmax_bits) {
    const float pm = __uint_as_float(pmax_bits);
    int e = 0;
    if (pm > 0.0f) frexpf(pm, &e);  // pm < 2^e
    int F = kFracHeadroomBits - e;
    return F < 0 ? 0 : (F > 60 ? 60 : F);
}

// WMODE: the orientation weight (SBP_W_*), fixed at compile time so that no
// pair branches on it; WIDE: the wide shape. FwdTile picks the instance.
template <int WMODE, bool WIDE>
__global__ void __launch_bounds__((WIDE ? kWarpsWide : kWarpsNarrow) * 32, WIDE ? 1 : 2)
fwd_group_kernel(BallsDev b, FrameTable ft, const float* __restrict__ sens, LevelGeo g,
                 int chunk, const unsigned int* __restrict__ pmax, SbpDevState* st,
                 unsigned long long* __restrict__ acc_all) {
    constexpr int kGroupWarps = WIDE ? kWarpsWide : kWarpsNarrow;
    constexpr int kWindow = WIDE ? kWindowWide : kWindowNarrow;
    extern __shared__ unsigned int sacc[];  // [2][kWindow][32]: low words, then high words
    __shared__ float s_red[kGroupWarps * 7];
    __shared__ float s_box[7];
    __shared__ int s_jlo[32];
    // one-dimensional grid, chunk-major: the CTAs of one ball chunk (one per
    // group of 32 sensors) are consecutive, so live chunks come first
    const int groups = (g.M + 31) / 32;
    const int gid = (int)(blockIdx.x % (unsigned)groups);
    const int c0 = (int)(blockIdx.x / (unsigned)groups) * chunk;
    const FrameSlot fs = sbp_frame_of(ft, c0);
    if (c0 >= fs.end) return;  // uniform over the block
    const int c1 = min(fs.end, c0 + chunk);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Tk = g.Tk, M = g.M;
    unsigned long long* __restrict__ acc = acc_all + (size_t)fs.f * M * Tk;
    const int m = gid * 32 + lane;
    const bool sv = m < M;

    sbp_chunk_box(b, c0, c1, s_red, s_box);

    float sx = 0.f, sy = 0.f, sz = 0.f, nx = 0.f, ny = 0.f, nz = 0.f;
    int jlo = 0, jhi = -1;
    if (sv) {
        sx = sens[m];
        sy = sens[M + m];
        sz = sens[2 * M + m];
        nx = sens[3 * M + m];
        ny = sens[4 * M + m];
        nz = sens[5 * M + m];
        sbp_box_cells(sx, sy, sz, s_box, g, jlo, jhi);
    }
    int wmax = max(0, jhi - jlo + 1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    if (wmax == 0) return;  // no lane's sensor can be reached (uniform over the block)
    if (warp == 0) s_jlo[lane] = jlo;
    // only the cells some lane can touch are cleared (and later flushed)
    const int used = min(wmax, kWindow) * 32;
    for (int t = threadIdx.x; t < used; t += blockDim.x) {
        sacc[t] = 0u;
        sacc[kWindow * 32 + t] = 0u;
    }
    __syncthreads();

    const float scale = __int_as_float((127 + fwd_frac_bits(pmax[fs.f])) << 23);  // 2^F
    const float h = g.h_hi;
    const float d2c = -2.0f * h * h;
    unsigned int inside = 0;
    // The lane's cells jlo .. jlo + kWindow - 1 are held in shared memory;
    // impulses further out (a chunk whose window is longer than the buffer)
    // go straight to the global accumulators.
    const int base = jlo;
    const int lim = min(jhi - base, kWindow - 1);  // last shared cell that may be stored
    const int glim = Tk - 1 - base;                // last cell inside the record
    unsigned int* col = sacc + lane;
    unsigned long long* grow = acc + (size_t)m * Tk + base;
    // The warp takes its balls two at a time (i and i + 1) and evaluates
    // both pairs of its lane's sensor side by side; an odd last ball is
    // paired with an empty one. Every ball goes through the same
    // instructions, so its impulses do not depend on its partner. With the
    // ball rows 8-byte aligned and c0 even (every chunk size and frame
    // offset is), a pair of balls is read with one 8-byte load per row.
    const bool pair_ld =
        ((reinterpret_cast<uintptr_t>(b.x) | reinterpret_cast<uintptr_t>(b.y) |
          reinterpret_cast<uintptr_t>(b.z) | reinterpret_cast<uintptr_t>(b.R) |
          reinterpret_cast<uintptr_t>(b.p0) | (uintptr_t)(c0 & 1) * 4u) & 7u) == 0;
    for (int i = c0 + 2 * warp; i < c1; i += 2 * kGroupWarps) {
        const bool hasB = i + 1 < c1;
        float2 cx, cy, cz, R2, P2;
        if (pair_ld && hasB) {  // uniform over the warp
            cx = __ldg(reinterpret_cast<const float2*>(b.x + i));
            cy = __ldg(reinterpret_cast<const float2*>(b.y + i));
            cz = __ldg(reinterpret_cast<const float2*>(b.z + i));
            R2 = __ldg(reinterpret_cast<const float2*>(b.R + i));
            P2 = __ldg(reinterpret_cast<const float2*>(b.p0 + i));
        } else {
            cx = make_float2(b.x[i], hasB ? b.x[i + 1] : 0.0f);
            cy = make_float2(b.y[i], hasB ? b.y[i + 1] : 0.0f);
            cz = make_float2(b.z[i], hasB ? b.z[i + 1] : 0.0f);
            R2 = make_float2(b.R[i], hasB ? b.R[i + 1] : 0.0f);
            P2 = make_float2(b.p0[i], hasB ? b.p0[i + 1] : 0.0f);
        }
        if ((P2.x == 0.0f && P2.y == 0.0f) || !sv) continue;
        const PairDist2 pd = sbp_pair_distance2(cx, cy, cz, f2(sx), f2(sy), f2(sz));
        // inside test and window, per pair
        bool okA = P2.x != 0.0f, okB = P2.y != 0.0f;
        const float2 dd = f2add(pd.dh, pd.dl);
        if (okA && !(dd.x > R2.x)) {
            ++inside;
            okA = false;
        }
        if (okB && !(dd.y > R2.y)) {
            ++inside;
            okB = false;
        }
        PairWindow wa, wb;
        bool wA, wB;
        sbp_window2(pd.dh, pd.dl, R2, g, wa, wb, wA, wB);
        okA = okA && wA;
        okB = okB && wB;
        if (!(okA || okB)) continue;
        const float2 cosv = f2mul(
            f2fma(f2(nx), pd.dx, f2fma(f2(ny), pd.dy, f2mul(f2(nz), pd.dz))), pd.rd);
        float actA, actB;
        const float2 w = make_float2(sbp_weight(WMODE, cosv.x, actA),
                                     sbp_weight(WMODE, cosv.y, actB));
        okA = okA && w.x != 0.0f;
        okB = okB && w.y != 0.0f;
        if (!(okA || okB)) continue;
        const float2 b0 = make_float2(wa.b0, wb.b0), bL = make_float2(wa.bL, wb.bL);
        // K 2^F = p0 w 2^F / (4 d h)
        const float2 Ks = f2mul(f2mul(f2mul(P2, w), f2(g.inv_4h * scale)), pd.rd);
        const float2 ra = make_float2(fmaxf(R2.x - b0.x, 0.0f), fmaxf(R2.y - b0.y, 0.0f));
        const float2 re = make_float2(fmaxf(R2.x + bL.x, 0.0f), fmaxf(R2.y + bL.y, 0.0f));
        const float2 fa = f2mul(f2mul(Ks, ra), f2add(R2, b0));
        const float2 fe = f2neg(f2mul(f2mul(Ks, re), f2sub(R2, bL)));
        const float2 f1 = f2mul(f2mul(Ks, f2(h)), f2fma(f2(2.0f), b0, f2(-h)));
        const float2 fq = f2mul(Ks, f2(d2c));
        if (okA)
            fwd_emit<kWindow>(col, grow, wa.jL - 1 - base, wa.jH - base, wa.jH - wa.jL, lim, base, glim,
                     fa.x, fe.x, f1.x, fq.x);
        if (okB)
            fwd_emit<kWindow>(col, grow, wb.jL - 1 - base, wb.jH - base, wb.jH - wb.jL, lim, base, glim,
                     fa.y, fe.y, f1.y, fq.y);
    }
    __syncthreads();
    // Flush, one block of 32 window cells per warp at a time. The warp first
    // transposes the block's 32 x 32 low words and 32 x 32 high words in
    // place, from [cell][lane] to [lane][cell], so that it then adds each
    // sensor's 32 consecutive cells to its global row with one coalesced
    // instruction (straight from the [cell][lane] layout, every instruction
    // would scatter over 32 rows, one 32-byte sector per 8-byte sum).
    // The transpose swaps (r, r + k) with (r + k, r) for r = lane and
    // k = 1 .. 16 (at k = 16 the lower 16 lanes take the pairs): every
    // off-diagonal element moves once, and each step's 32 accesses fall in
    // 32 distinct banks. kWindow is a multiple of 32, so the blocks stay
    // inside the window; cells at or past `nrel` were never cleared and are
    // not flushed.
    static_assert(kWindow % 32 == 0, "the flush transposes whole 32-cell blocks");
    const int nrel = min(wmax, kWindow);
    for (int blk = warp; blk * 32 < nrel; blk += kGroupWarps) {
        unsigned int* const blo = sacc + blk * 32 * 32;
        unsigned int* const bhi = blo + kWindow * 32;
#pragma unroll 4
        for (int k = 1; k <= 16; ++k) {
            if (k < 16 || lane < 16) {
                const int c = (lane + k) & 31;
                const int p = lane * 32 + c, q = c * 32 + lane;
                const unsigned int l0 = blo[p], l1 = blo[q], h0 = bhi[p], h1 = bhi[q];
                blo[p] = l1;
                blo[q] = l0;
                bhi[p] = h1;
                bhi[q] = h0;
            }
        }
        __syncwarp();
        const int rel = blk * 32 + lane;
        for (int x = 0; x < 32; ++x) {
            const unsigned int wa = blo[x * 32 + lane];
            const int hi = (int)bhi[x * 32 + lane];
            if ((wa | (unsigned)hi) && rel < nrel) {
                // the low word holds the whole sum mod 2^32; the sum of the
                // low kLoBits-bit parts lies in [0, 2^32), so it is that word
                // minus hi * 2^kLoBits, mod 2^32
                const unsigned int lo = wa - ((unsigned int)hi << kLoBits);
                const long long v = (long long)hi * (1LL << kLoBits) + (long long)lo;
                atomicAdd(acc + (size_t)(gid * 32 + x) * Tk + s_jlo[x] + rel,
                          (unsigned long long)v);
            }
        }
    }
    if (inside) atomicAdd(&st->inside_pairs, (unsigned long long)inside);
}

// One CTA per sensor: S = 2^-F * P(P(D)), then clear the accumulator row.
__global__ void __launch_bounds__(kFinalizeThreads)
fwd_finalize_kernel(unsigned long long* __restrict__ acc, int Tk,
                    const unsigned int* __restrict__ pmax, float* __restrict__ S) {
    __shared__ long long warp_tot[32];
    const int m = blockIdx.y * gridDim.x + blockIdx.x;  // frame-major row
    unsigned long long* row = acc + (size_t)m * Tk;
    float* out = S + (size_t)m * Tk;
    const float inv = __int_as_float((127 - fwd_frac_bits(pmax[blockIdx.y])) << 23);  // 2^-F
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
                const long long x = v[q] + off;  // two 32-bit conversions, not one 64-bit
                out[i] = fmaf((float)(int)(x >> 32), 4294967296.0f, (float)(unsigned)x) * inv;
                row[i] = 0ull;
            }
        }
    }
}

}  // namespace

using FwdGroupKernel = void (*)(BallsDev, FrameTable, const float*, LevelGeo, int,
                                const unsigned int*, SbpDevState*, unsigned long long*);

// The accumulation kernel compiled for one orientation weight (SBP_W_*) and
// shape.
template <bool WIDE>
static FwdGroupKernel fwd_group_shape(int wmode) {
    if (wmode == SBP_W_NONE) return fwd_group_kernel<SBP_W_NONE, WIDE>;
    if (wmode == SBP_W_COS) return fwd_group_kernel<SBP_W_COS, WIDE>;
    return fwd_group_kernel<SBP_W_CLAMP, WIDE>;
}

// A tile: balls per CTA and shape, decoded from a tile value (a power of
// two in [32, SBP_FRAME_ALIGN], optionally or'ed with SBP_TILE_WIDE).
struct FwdTile {
    int chunk;
    bool wide;
    FwdGroupKernel kernel(int wmode) const {
        return wide ? fwd_group_shape<true>(wmode) : fwd_group_shape<false>(wmode);
    }
    int threads() const { return 32 * (wide ? kWarpsWide : kWarpsNarrow); }
    size_t smem() const {
        return (size_t)2 * (wide ? kWindowWide : kWindowNarrow) * 32 * sizeof(unsigned int);
    }
};

static int fwd_set_smem(const FwdTile& t, int wmode, const char* what) {
    return sbp_cuda_check(cudaFuncSetAttribute(t.kernel(wmode),
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)t.smem()),
                          what);
}

bool sbp_fwd_tile_valid(int tv) {
    const int c = tv & ~SBP_TILE_WIDE;
    return (tv & ~(SBP_TILE_WIDE | (2 * kMaxChunk - 1))) == 0 && c >= 32 && c <= kMaxChunk &&
           !(c & (c - 1));
}

// The tile of a valid tile value, else `fallback`.
static FwdTile fwd_tile_of(int tv, FwdTile fallback) {
    return sbp_fwd_tile_valid(tv) ? FwdTile{tv & ~SBP_TILE_WIDE, (tv & SBP_TILE_WIDE) != 0}
                                  : fallback;
}

int sbp_launch_forward(sbp_array_s* a, const BallsDev& b, const int* n_dev, int n_cap,
                       float* S, cudaStream_t st) {
    const LevelGeo g = sbp_level_geo(a, a->level);
    const int groups = (g.M + 31) / 32;
    // consecutive balls per CTA: the level's tuned size if sbp_autotune chose
    // one, else kChunk, fewer for small clouds so that the grid still covers
    // the GPU
    FwdTile tile{kChunk, false};
    while (tile.chunk > 32 &&
           (long long)((n_cap + tile.chunk - 1) / tile.chunk) * groups < 4LL * a->sm_count)
        tile.chunk >>= 1;
    tile = fwd_tile_of(a->fwd_chunk_lvl[a->level], tile);
    const int chunk = tile.chunk;
    if (fwd_set_smem(tile, g.wmode, "forward: smem attribute")) return SBP_ERR_CUDA;
    if (sbp_cuda_check(cudaMemsetAsync(&a->d_state->pmax_bits, 0, sizeof(unsigned int), st),
                       "forward: reset pmax"))
        return SBP_ERR_CUDA;
    const FrameTable ft{1, nullptr, n_dev, n_cap};
    fwd_pmax_kernel<<<std::max(1, std::min(4 * a->sm_count, (n_cap + 255) / 256)), 256, 0,
                      st>>>(b, ft, &a->d_state->pmax_bits, a->d_state);
    if (sbp_cuda_check(cudaGetLastError(), "forward: pmax launch")) return SBP_ERR_CUDA;
    const unsigned grid = (unsigned)(((long long)n_cap + chunk - 1) / chunk * groups);
    tile.kernel(g.wmode)<<<grid, tile.threads(), tile.smem(), st>>>(
        b, ft, a->d_sens, g, chunk, &a->d_state->pmax_bits, a->d_state, a->d_acc);
    if (sbp_cuda_check(cudaGetLastError(), "forward: accumulate launch")) return SBP_ERR_CUDA;
    fwd_finalize_kernel<<<g.M, kFinalizeThreads, 0, st>>>(a->d_acc, g.Tk,
                                                          &a->d_state->pmax_bits, S);
    if (sbp_cuda_check(cudaGetLastError(), "forward: finalize launch")) return SBP_ERR_CUDA;
    sbp_count_launches(3);
    return SBP_OK;
}

// All frames of the packed layout in one launch per kernel (sbp_forward_frames).
int sbp_launch_forward_frames(sbp_array_s* a, const BallsDev& b, const int* n_dev, float* S,
                              int chunk, cudaStream_t st) {
    const LevelGeo g = sbp_level_geo(a, a->level);
    const int F = a->frames;
    const int total = a->h_frame_off[F];
    const int groups = (g.M + 31) / 32;
    // a chunk must not straddle two frames: at most one alignment unit
    FwdTile tile = fwd_tile_of(chunk, FwdTile{kChunk, false});
    if (tile.chunk > SBP_FRAME_ALIGN) tile.chunk = SBP_FRAME_ALIGN;
    chunk = tile.chunk;
    if (fwd_set_smem(tile, g.wmode, "forward_frames: smem attribute")) return SBP_ERR_CUDA;
    // one fixed-point scale per frame, so that every frame's traces equal
    // those of a single-cloud forward of that frame
    if (sbp_cuda_check(cudaMemsetAsync(a->d_frame_pmax, 0, sizeof(unsigned int) * F, st),
                       "forward_frames: reset pmax"))
        return SBP_ERR_CUDA;
    const FrameTable ft{F, a->d_frame_off, n_dev, total};
    const int pmax_blocks = std::max(1, std::min(4 * a->sm_count / F, total / F / 256 + 1));
    fwd_pmax_kernel<<<dim3(pmax_blocks, F), 256, 0, st>>>(b, ft, a->d_frame_pmax, a->d_state);
    if (sbp_cuda_check(cudaGetLastError(), "forward_frames: pmax launch")) return SBP_ERR_CUDA;
    const unsigned grid = (unsigned)(((long long)total + chunk - 1) / chunk * groups);
    tile.kernel(g.wmode)<<<grid, tile.threads(), tile.smem(), st>>>(
        b, ft, a->d_sens, g, chunk, a->d_frame_pmax, a->d_state, a->d_acc);
    if (sbp_cuda_check(cudaGetLastError(), "forward_frames: accumulate launch"))
        return SBP_ERR_CUDA;
    fwd_finalize_kernel<<<dim3(g.M, F), kFinalizeThreads, 0, st>>>(a->d_acc, g.Tk,
                                                                   a->d_frame_pmax, S);
    if (sbp_cuda_check(cudaGetLastError(), "forward_frames: finalize launch"))
        return SBP_ERR_CUDA;
    sbp_count_launches(3);
    return SBP_OK;
}

// ---------------------------------------------------------------------------
// Forward without allocation (sbp_forward_static).
//
// Some callers cannot allocate device memory at all: a host process that
// only borrows buffers from a larger framework owning every allocation (a
// serving runtime with its own memory pool), or one held to a fixed device
// memory budget that a cudaMalloc behind its back could break.
// For them this entry point renders the same traces as sbp_forward without
// an array object: its scratch (the int64 trace accumulators and the state
// words) lives in one file-scope device array that every GPU loading this
// library holds until the process exits. The kernels are the ones
// sbp_forward launches.
// ---------------------------------------------------------------------------

namespace {

constexpr long long kStaticCells = 1LL << 21;  // largest M * T_k: 16 MiB of accumulators
constexpr int kStaticStateWords = 32;          // 256 bytes for SbpDevState (padded)

static_assert(sizeof(SbpDevState) <= kStaticStateWords * sizeof(unsigned long long),
              "state words do not fit");

// [0, kStaticStateWords): SbpDevState; then kStaticCells int64 accumulators.
static __device__ __align__(256) unsigned long long g_static_scratch[kStaticStateWords + kStaticCells];

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
unsigned long long* g_static_ptr[kMaxDevices] = {};  // device address, per device
unsigned long long g_static_ctx[kMaxDevices] = {};   // ID of the context it was taken in
int g_static_sms[kMaxDevices] = {};

// The unique ID of the calling thread's current context (0 when none is
// current), through the driver's cuCtxGetCurrent / cuCtxGetId reached from
// the runtime. A context that is destroyed and created again (cudaDeviceReset,
// or a framework that releases the primary context) gets a new ID.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

int current_ctx_id(unsigned long long* id) {
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_cur || !get_id) {
        void* p1 = nullptr;
        void* p2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p1, 12000, cudaEnableDefault,
                                             &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &p2, 12000, cudaEnableDefault,
                                             &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) {
            sbp_set_error("forward_static: the driver offers no context ID");
            return SBP_ERR_CUDA;
        }
        get_cur = reinterpret_cast<CtxGetCurrentFn>(p1);
        get_id = reinterpret_cast<CtxGetIdFn>(p2);
    }
    CUcontext ctx = nullptr;
    *id = 0;
    if (get_cur(&ctx) != CUDA_SUCCESS) {
        sbp_set_error("forward_static: cuCtxGetCurrent failed");
        return SBP_ERR_CUDA;
    }
    if (ctx && get_id(ctx, id) != CUDA_SUCCESS) {
        sbp_set_error("forward_static: cuCtxGetId failed");
        return SBP_ERR_CUDA;
    }
    return SBP_OK;
}

// Set-up per device and context (with that device current): the device
// address of the scratch array. A host-side reference to g_static_scratch is
// only a stand-in, never a usable device pointer, so kernels get this
// address. It is looked up again whenever the current context is not the one
// it was taken in, since a new context loads the module, and with it the
// array, at a new address.
int static_scratch(int dev, unsigned long long** out, int* sms) {
    if (dev < 0 || dev >= kMaxDevices) {
        sbp_set_error("forward_static: device index out of range");
        return SBP_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_static_mutex);
    unsigned long long ctx = 0;
    if (int e = current_ctx_id(&ctx)) return e;
    if (!g_static_ptr[dev] || ctx == 0 || ctx != g_static_ctx[dev]) {
        void* p = nullptr;
        if (sbp_cuda_check(cudaGetSymbolAddress(&p, g_static_scratch),
                           "forward_static: scratch address"))
            return SBP_ERR_CUDA;
        // the look-up made the device's context current if none was
        if (int e = current_ctx_id(&ctx)) return e;
        int n = 0;
        if (sbp_cuda_check(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev),
                           "forward_static: SM count"))
            return SBP_ERR_CUDA;
        g_static_sms[dev] = n > 0 ? n : 1;
        g_static_ptr[dev] = static_cast<unsigned long long*>(p);
        g_static_ctx[dev] = ctx;
    }
    *out = g_static_ptr[dev];
    *sms = g_static_sms[dev];
    return SBP_OK;
}

}  // namespace

extern "C" int sbp_forward_static(const float* sensors_dev, int M, double c_mm_per_us,
                                  double dt_us, int T_k, int weight_mode, sbp_balls balls,
                                  const int* n_dev, int n_cap, float* S_dev, sbp_stream stream) {
    if (!sensors_dev || !S_dev || !balls.x || !balls.y || !balls.z || !balls.R || !balls.p0 ||
        M < 1 || T_k < 1 || n_cap < 1 || !(c_mm_per_us > 0) || !(dt_us > 0) ||
        weight_mode < SBP_W_CLAMP || weight_mode > SBP_W_COS) {
        sbp_set_error("forward_static: invalid argument");
        return SBP_ERR_ARG;
    }
    if ((long long)M * T_k > kStaticCells) {
        sbp_set_error("forward_static: M * T_k exceeds the static scratch of 2^21 cells "
                      "(16 MiB); use sbp_forward with an array object");
        return SBP_ERR_ARG;
    }
    int dev = 0, sms = 1;
    if (sbp_cuda_check(cudaGetDevice(&dev), "forward_static: device")) return SBP_ERR_CUDA;
    unsigned long long* base = nullptr;
    if (int e = static_scratch(dev, &base, &sms)) return e;
    SbpDevState* state = reinterpret_cast<SbpDevState*>(base);
    unsigned long long* acc = base + kStaticStateWords;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    LevelGeo g;
    const double h = c_mm_per_us * dt_us;
    g.M = M;
    g.Tk = T_k;
    g.h_hi = (float)h;
    g.h_lo = (float)(h - (double)g.h_hi);
    g.inv_h = (float)(1.0 / h);
    g.inv_4h = (float)(0.25 / h);
    g.wmode = weight_mode;
    g.pad = 0;
    const BallsDev b{balls.x, balls.y, balls.z, balls.R, balls.p0};

    // the array keeps whatever the last call left: clear the state words and
    // the accumulators this call uses
    if (sbp_cuda_check(cudaMemsetAsync(base, 0,
                                       sizeof(unsigned long long) *
                                           (kStaticStateWords + (size_t)M * T_k),
                                       st),
                       "forward_static: clear scratch"))
        return SBP_ERR_CUDA;
    const int groups = (M + 31) / 32;
    FwdTile tile{kChunk, false};
    while (tile.chunk > 32 && (long long)((n_cap + tile.chunk - 1) / tile.chunk) * groups < 4LL * sms)
        tile.chunk >>= 1;
    const int chunk = tile.chunk;
    if (fwd_set_smem(tile, g.wmode, "forward_static: smem attribute")) return SBP_ERR_CUDA;
    const FrameTable ft{1, nullptr, n_dev, n_cap};
    fwd_pmax_kernel<<<std::max(1, std::min(4 * sms, (n_cap + 255) / 256)), 256, 0, st>>>(
        b, ft, &state->pmax_bits, state);
    if (sbp_cuda_check(cudaGetLastError(), "forward_static: pmax launch")) return SBP_ERR_CUDA;
    const unsigned grid = (unsigned)(((long long)n_cap + chunk - 1) / chunk * groups);
    tile.kernel(g.wmode)<<<grid, tile.threads(), tile.smem(), st>>>(
        b, ft, sensors_dev, g, chunk, &state->pmax_bits, state, acc);
    if (sbp_cuda_check(cudaGetLastError(), "forward_static: accumulate launch"))
        return SBP_ERR_CUDA;
    fwd_finalize_kernel<<<M, kFinalizeThreads, 0, st>>>(acc, T_k, &state->pmax_bits, S_dev);
    if (sbp_cuda_check(cudaGetLastError(), "forward_static: finalize launch")) return SBP_ERR_CUDA;
    sbp_count_launches(3);
    return SBP_OK;
}
