// Entry and exit of Algorithm 1 around the iteration:
//   * the envelope mesh built from the array coordinates (Section 4.1 and
//     the first step of Algorithm 1): the convex hull of the sensor
//     positions, a closed triangle mesh with outward orientation, built on
//     the host by incremental insertion in double precision;
//   * the reconstruction region inside it, pulled `inset` inward (points of
//     the mesh interior at least `inset` from its surface), and the
//     ray-casting test deciding membership (an odd number of crossings of a
//     fixed ray from the point), in double precision on the GPU;
//   * random initialisation of the point cloud inside the region: candidates
//     drawn uniformly from the sensors' bounding box by SplitMix64 at stream
//     positions 5k .. 5k+4 (x, y, z, R, p0 of candidate k), accepted in
//     candidate order, so the cloud is a function of the seed alone;
//   * the point cloud -> voxel grid conversion (the last step of
//     Algorithm 1): voxel v with centre x_v takes the sum of the values (p0
//     by default) of the balls with |x_v - c| < R, accumulated in fixed
//     point so that the grid does not depend on the order of the balls.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <unordered_set>
#include <vector>

#include "sbp_internal.cuh"
#include "sbp_scan.cuh"

struct sbp_envelope_s {
    int device = -1;
    int M = 0;
    int F = 0;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};  // bounding box of the sensors
    double volume = 0;
    std::vector<int> tri;       // [F][3] sensor indices, outward orientation
    double* d_tri = nullptr;    // [F][13]: v0, e1 = v1 - v0, e2 = v2 - v0, unit normal, offset
    float* d_ftri = nullptr;    // [F][20]: the same triangle seen along the ray (see FTri)
    double frame[6] = {0, 0, 0, 0, 0, 0};  // the two unit axes across the ray
    double lmax = 0;            // largest coordinate magnitude of the sensors
    unsigned char* d_flags = nullptr;  // sampling scratch: one flag per candidate
    long long flags_cap = 0;
    long long* d_block = nullptr;      // per-block accepted counts, then offsets; [blocks + 1]
    long long block_cap = 0;
};

namespace {

constexpr int kTriWords = 13;
constexpr int kFWords = 26;  // float record per triangle (see fast_cross)
constexpr int kEnvThreads = 256;
constexpr int kTriTile = 128;  // triangles staged in shared memory at a time
constexpr int kVoxFracHeadroom = 40;  // voxel sums kept as round(v 2^F), |v| 2^F < 2^40

// a fixed generic direction for the casting ray (not parallel to any axis or
// coordinate plane)
__device__ __constant__ double kRayDir[3] = {0.8017837257372732, 0.5345224838248488,
                                             0.2672612419124244};
constexpr double kRayDirHost[3] = {0.8017837257372732, 0.5345224838248488, 0.2672612419124244};

// ---------------------------------------------------------------------------
// host: incremental convex hull
// ---------------------------------------------------------------------------

struct HFace {
    int a, b, c;
    double n[3];
    double d;
    bool alive;
};

void face_plane(const std::vector<double>& P, HFace& f) {
    const double* A = &P[3 * f.a];
    const double* B = &P[3 * f.b];
    const double* C = &P[3 * f.c];
    const double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    const double v[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
    double n[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2],
                   u[0] * v[1] - u[1] * v[0]};
    const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int k = 0; k < 3; ++k) f.n[k] = len > 0 ? n[k] / len : 0.0;
    f.d = f.n[0] * A[0] + f.n[1] * A[1] + f.n[2] * A[2];
}

double plane_dist(const HFace& f, const double* p) {
    return f.n[0] * p[0] + f.n[1] * p[1] + f.n[2] * p[2] - f.d;
}

uint64_t edge_key(int u, int v) { return ((uint64_t)(uint32_t)u << 32) | (uint32_t)v; }

// Convex hull of n points (xyz interleaved) as outward triangles. Points
// within eps of a face count as inside. Returns false for a flat or
// degenerate set.
bool build_hull(const std::vector<double>& P, int n, std::vector<int>& tri, std::string& err) {
    double lo[3] = {P[0], P[1], P[2]}, hi[3] = {P[0], P[1], P[2]};
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], P[3 * i + k]);
            hi[k] = std::max(hi[k], P[3 * i + k]);
        }
    const double diag = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) +
                                  (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                  (hi[2] - lo[2]) * (hi[2] - lo[2]));
    const double eps = 1e-9 * diag;
    auto pt = [&](int i) { return &P[3 * i]; };
    // initial tetrahedron from extreme points
    int i0 = 0;
    for (int i = 1; i < n; ++i)
        if (pt(i)[0] < pt(i0)[0]) i0 = i;
    int i1 = -1;
    double best = 0;
    for (int i = 0; i < n; ++i) {
        const double* p = pt(i);
        const double d = std::sqrt((p[0] - pt(i0)[0]) * (p[0] - pt(i0)[0]) +
                                   (p[1] - pt(i0)[1]) * (p[1] - pt(i0)[1]) +
                                   (p[2] - pt(i0)[2]) * (p[2] - pt(i0)[2]));
        if (d > best) {
            best = d;
            i1 = i;
        }
    }
    if (i1 < 0 || best <= eps) {
        err = "envelope: the sensor positions coincide";
        return false;
    }
    const double* A = pt(i0);
    double dir[3] = {pt(i1)[0] - A[0], pt(i1)[1] - A[1], pt(i1)[2] - A[2]};
    const double dl = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    for (double& x : dir) x /= dl;
    int i2 = -1;
    best = 0;
    for (int i = 0; i < n; ++i) {
        const double w[3] = {pt(i)[0] - A[0], pt(i)[1] - A[1], pt(i)[2] - A[2]};
        const double c[3] = {w[1] * dir[2] - w[2] * dir[1], w[2] * dir[0] - w[0] * dir[2],
                             w[0] * dir[1] - w[1] * dir[0]};
        const double d = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        if (d > best) {
            best = d;
            i2 = i;
        }
    }
    if (i2 < 0 || best <= eps) {
        err = "envelope: the sensors lie on a line";
        return false;
    }
    HFace base{i0, i1, i2, {0, 0, 0}, 0, true};
    face_plane(P, base);
    int i3 = -1;
    best = 0;
    for (int i = 0; i < n; ++i) {
        const double d = std::fabs(plane_dist(base, pt(i)));
        if (d > best) {
            best = d;
            i3 = i;
        }
    }
    if (i3 < 0 || best <= eps) {
        err = "envelope: the sensors lie in a plane; a closed envelope needs a 3D array";
        return false;
    }
    double g[3];
    for (int k = 0; k < 3; ++k) g[k] = 0.25 * (pt(i0)[k] + pt(i1)[k] + pt(i2)[k] + pt(i3)[k]);
    std::vector<HFace> faces;
    auto add_oriented = [&](int a, int b, int c) {
        HFace f{a, b, c, {0, 0, 0}, 0, true};
        face_plane(P, f);
        if (plane_dist(f, g) > 0) {  // the interior must lie behind the face
            std::swap(f.b, f.c);
            face_plane(P, f);
        }
        faces.push_back(f);
    };
    add_oriented(i0, i1, i2);
    add_oriented(i0, i1, i3);
    add_oriented(i0, i2, i3);
    add_oriented(i1, i2, i3);
    std::vector<int> visible;
    std::unordered_set<uint64_t> edges;
    std::vector<std::pair<int, int>> horizon;
    for (int p = 0; p < n; ++p) {
        if (p == i0 || p == i1 || p == i2 || p == i3) continue;
        visible.clear();
        for (int f = 0; f < (int)faces.size(); ++f)
            if (faces[f].alive && plane_dist(faces[f], pt(p)) > eps) visible.push_back(f);
        if (visible.empty()) continue;
        edges.clear();
        for (int f : visible) {
            const HFace& F = faces[f];
            edges.insert(edge_key(F.a, F.b));
            edges.insert(edge_key(F.b, F.c));
            edges.insert(edge_key(F.c, F.a));
        }
        horizon.clear();
        for (int f : visible) {
            const HFace& F = faces[f];
            const int e[3][2] = {{F.a, F.b}, {F.b, F.c}, {F.c, F.a}};
            for (const auto& uv : e)
                if (!edges.count(edge_key(uv[1], uv[0]))) horizon.emplace_back(uv[0], uv[1]);
            faces[f].alive = false;
        }
        // the horizon edge u -> v of a visible face becomes the new face
        // (u, v, p), which keeps the orientation of its invisible neighbour
        for (const auto& uv : horizon) {
            HFace f{uv.first, uv.second, p, {0, 0, 0}, 0, true};
            face_plane(P, f);
            faces.push_back(f);
        }
        if (faces.size() > 64 && faces.size() > 4 * (size_t)(2 * n)) {  // drop dead faces
            std::vector<HFace> keep;
            for (const HFace& f : faces)
                if (f.alive) keep.push_back(f);
            faces.swap(keep);
        }
    }
    tri.clear();
    for (const HFace& f : faces)
        if (f.alive) {
            tri.push_back(f.a);
            tri.push_back(f.b);
            tri.push_back(f.c);
        }
    return true;
}

// ---------------------------------------------------------------------------
// device: ray casting and distance to the mesh
// ---------------------------------------------------------------------------

// Moller-Trumbore: does the ray x + t d (t > 0) cross the closed triangle?
__device__ __forceinline__ bool ray_hits(const double* T, double x, double y, double z) {
    const double dx = kRayDir[0], dy = kRayDir[1], dz = kRayDir[2];
    const double e1x = T[3], e1y = T[4], e1z = T[5], e2x = T[6], e2y = T[7], e2z = T[8];
    const double px = dy * e2z - dz * e2y, py = dz * e2x - dx * e2z, pz = dx * e2y - dy * e2x;
    const double det = e1x * px + e1y * py + e1z * pz;
    if (!(fabs(det) > 1e-300)) return false;
    const double inv = 1.0 / det;
    const double tx = x - T[0], ty = y - T[1], tz = z - T[2];
    const double u = (tx * px + ty * py + tz * pz) * inv;
    if (u < 0.0 || u > 1.0) return false;
    const double qx = ty * e1z - tz * e1y, qy = tz * e1x - tx * e1z, qz = tx * e1y - ty * e1x;
    const double v = (dx * qx + dy * qy + dz * qz) * inv;
    if (v < 0.0 || u + v > 1.0) return false;
    const double t = (e2x * qx + e2y * qy + e2z * qz) * inv;
    return t > 0.0;
}

// Squared distance from p to the closed triangle (closest point by the
// Voronoi regions of its vertices, edges and face).
template <typename R>
__device__ __forceinline__ R tri_dist2(const R* T, R px, R py, R pz) {
    const R ax = T[0], ay = T[1], az = T[2];
    const R abx = T[3], aby = T[4], abz = T[5], acx = T[6], acy = T[7], acz = T[8];
    const R apx = px - ax, apy = py - ay, apz = pz - az;
    const R d1 = abx * apx + aby * apy + abz * apz, d2 = acx * apx + acy * apy + acz * apz;
    R qx, qy, qz;
    if (d1 <= R(0) && d2 <= R(0)) {
        qx = ax, qy = ay, qz = az;
    } else {
        const R bpx = apx - abx, bpy = apy - aby, bpz = apz - abz;
        const R d3 = abx * bpx + aby * bpy + abz * bpz, d4 = acx * bpx + acy * bpy + acz * bpz;
        const R cpx = apx - acx, cpy = apy - acy, cpz = apz - acz;
        const R d5 = abx * cpx + aby * cpy + abz * cpz, d6 = acx * cpx + acy * cpy + acz * cpz;
        const R vc = d1 * d4 - d3 * d2, vb = d5 * d2 - d1 * d6, va = d3 * d6 - d5 * d4;
        if (d3 >= R(0) && d4 <= d3) {
            qx = ax + abx, qy = ay + aby, qz = az + abz;
        } else if (vc <= R(0) && d1 >= R(0) && d3 <= R(0)) {
            const R s = d1 / (d1 - d3);
            qx = ax + s * abx, qy = ay + s * aby, qz = az + s * abz;
        } else if (d6 >= R(0) && d5 <= d6) {
            qx = ax + acx, qy = ay + acy, qz = az + acz;
        } else if (vb <= R(0) && d2 >= R(0) && d6 <= R(0)) {
            const R s = d2 / (d2 - d6);
            qx = ax + s * acx, qy = ay + s * acy, qz = az + s * acz;
        } else if (va <= R(0) && (d4 - d3) >= R(0) && (d5 - d6) >= R(0)) {
            const R s = (d4 - d3) / ((d4 - d3) + (d5 - d6));
            qx = ax + abx + s * (acx - abx), qy = ay + aby + s * (acy - aby),
            qz = az + abz + s * (acz - abz);
        } else {
            const R den = R(1) / (va + vb + vc);
            const R v = vb * den, w = vc * den;
            qx = ax + abx * v + acx * w, qy = ay + aby * v + acy * w, qz = az + abz * v + acz * w;
        }
    }
    const R ex = px - qx, ey = py - qy, ez = pz - qz;
    return ex * ex + ey * ey + ez * ez;
}

// Float record of a triangle seen along the ray. With the ray direction d
// and two unit axes e_u, e_v across it, the ray from p crosses the triangle
// exactly when p's projection (p.e_u, p.e_v) lies inside the projected
// triangle and the triangle's plane lies ahead of p along d. Words:
//   0..5   projected vertices a, b, c (u, v)
//   6..11  projected edge vectors b - a, c - b, a - c (from the double vertices)
//   12..15 projected bounding box (umin, umax, vmin, vmax)
//   16..18 L1 lengths of the three edge vectors
//   19..21 unit normal n, 22..24 vertex a, 25 sign of n.d
struct RayFrame {
    double e[6];  // e_u, e_v
    double lmax;  // largest sensor coordinate magnitude
};

// One pair of projected edge functions' error bands: an edge function
// (b - a) x (p - a) evaluated in float with coordinates below L in magnitude
// is within 16 eps L |b - a|_1 of its exact value (eps = 2^-24), which
// includes the rounding of the projected coordinates themselves.
constexpr float kEps = 5.9604645e-8f;

// Ray-crossing test of one triangle: 1 = crossed, 0 = not crossed, -1 = too
// close to an edge or to the triangle's plane to decide in float.
__device__ __forceinline__ int fast_cross(const float* T, float pu, float pv, float px, float py,
                                          float pz, float kp) {
    const float m = kp * 4.0f;
    if (pu < T[12] - m || pu > T[13] + m || pv < T[14] - m || pv > T[15] + m) return 0;
    // edge functions (b - a) x (p - a); with edge vectors and vertices each
    // rounded once from double, each is within kp |edge|_1 of its exact value
    const float s0 = T[6] * (pv - T[1]) - T[7] * (pu - T[0]);
    const float s1 = T[8] * (pv - T[3]) - T[9] * (pu - T[2]);
    const float s2 = T[10] * (pv - T[5]) - T[11] * (pu - T[4]);
    const float b0 = kp * T[16], b1 = kp * T[17], b2 = kp * T[18];
    const int pos = (s0 > b0) + (s1 > b1) + (s2 > b2);
    const int neg = (s0 < -b0) + (s1 < -b1) + (s2 < -b2);
    if (pos > 0 && neg > 0) return 0;  // outside the projection
    if (pos + neg < 3) return -1;      // on an edge within the error band
    // inside the projection: crossed when the plane is ahead along d
    const float sd = T[19] * (T[22] - px) + T[20] * (T[23] - py) + T[21] * (T[24] - pz);
    if (fabsf(sd) <= kp) return -1;
    return ((sd > 0.0f) == (T[25] > 0.0f)) ? 1 : 0;
}

// Region test of the calling thread's point against every triangle, staged
// through shared memory in tiles. Each triangle is first decided in float;
// undecidable ones (a ray through an edge's error band, a point on a plane)
// and distances that may fall below the inset are evaluated in double. Every
// thread of the block must call it (it contains barriers); `active` = false
// threads only help staging.
__device__ bool env_in_region(const double* __restrict__ tri, const float* __restrict__ ftri,
                              int F, double inset, const double* frame, double lmax, bool active,
                              double x, double y, double z, float* s_tri) {
    const float pu = (float)(x * frame[0] + y * frame[1] + z * frame[2]);
    const float pv = (float)(x * frame[3] + y * frame[4] + z * frame[5]);
    const float px = (float)x, py = (float)y, pz = (float)z;
    const double L = fmax(lmax, fmax(fabs(x), fmax(fabs(y), fabs(z)))) * 1.7320508075688772;
    const float kp = (float)(16.0 * (double)kEps * L);
    // sweep 1: crossings of the ray
    int hits = 0;
    for (int t0 = 0; t0 < F; t0 += kTriTile) {
        const int cnt = min(kTriTile, F - t0);
        __syncthreads();
        for (int w = threadIdx.x; w < cnt * kFWords; w += blockDim.x)
            s_tri[w] = ftri[(size_t)t0 * kFWords + w];
        __syncthreads();
        if (!active) continue;
        for (int t = 0; t < cnt; ++t) {
            const int c = fast_cross(s_tri + t * kFWords, pu, pv, px, py, pz, kp);
            hits += c > 0 ? 1 : (c < 0 && ray_hits(tri + (size_t)(t0 + t) * kTriWords, x, y, z)
                                     ? 1 : 0);
        }
    }
    const bool inside = active && (hits & 1);
    if (!(inset > 0.0) || !__syncthreads_or(inside)) return inside;
    // sweep 2, for points inside: is any triangle closer than the inset? A
    // triangle is screened by its plane distance and its float distance
    // (each within ~1e-5 mm of exact here) before the double evaluation.
    const double best2 = inset * inset;
    const float cull = (float)(inset + 1e-3 + 16.0 * (double)kEps * L);
    const float cull2 = cull * cull;
    bool near = false;
    for (int t0 = 0; t0 < F; t0 += kTriTile) {
        const int cnt = min(kTriTile, F - t0);
        __syncthreads();
        for (int w = threadIdx.x; w < cnt * kTriWords; w += blockDim.x)
            reinterpret_cast<float*>(s_tri)[w] = (float)tri[(size_t)t0 * kTriWords + w];
        __syncthreads();
        if (!inside || near) continue;
        for (int t = 0; t < cnt && !near; ++t) {
            const float* T = s_tri + t * kTriWords;
            const float pd = T[9] * px + T[10] * py + T[11] * pz - T[12];
            if (fabsf(pd) < cull && tri_dist2<float>(T, px, py, pz) < cull2 &&
                tri_dist2<double>(tri + (size_t)(t0 + t) * kTriWords, x, y, z) < best2)
                near = true;
        }
    }
    return inside && !near;
}

__global__ void __launch_bounds__(kEnvThreads)
env_classify_kernel(const double* __restrict__ tri, const float* __restrict__ ftri, int F,
                    double inset, RayFrame fr, const float* __restrict__ px,
                    const float* __restrict__ py, const float* __restrict__ pz, long long n,
                    unsigned char* __restrict__ flags) {
    __shared__ float s_tri[kTriTile * kFWords];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < n;
    const double x = active ? (double)px[i] : 0.0;
    const double y = active ? (double)py[i] : 0.0;
    const double z = active ? (double)pz[i] : 0.0;
    const bool in = env_in_region(tri, ftri, F, inset, fr.e, fr.lmax, active, x, y, z, s_tri);
    if (active) flags[i] = in ? 1 : 0;
}

// ---------------------------------------------------------------------------
// device: seeded candidates, acceptance and compaction
// ---------------------------------------------------------------------------

constexpr uint64_t kGoldenGamma = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ uint64_t env_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// uniform in [0, 1): top 53 bits of SplitMix64 output k, times 2^-53
__device__ __forceinline__ double env_unit(uint64_t seed, long long k) {
    const uint64_t b = env_mix(seed + (uint64_t)(k + 1) * kGoldenGamma) >> 11;
    return __dmul_rn((double)b, 1.1102230246251565e-16);
}

struct Candidate {
    float x, y, z, R, p0;
};

struct SampleBox {
    double lo[3], hi[3];
    double R_lo, R_hi, p_lo, p_hi;
};

// lo + (hi - lo) u in double without contraction, rounded to float
__device__ __forceinline__ float env_lerp(double lo, double hi, double u) {
    return __double2float_rn(__dadd_rn(lo, __dmul_rn(__dsub_rn(hi, lo), u)));
}

__device__ __forceinline__ Candidate env_candidate(uint64_t seed, long long k,
                                                   const SampleBox& bx) {
    Candidate c;
    c.x = env_lerp(bx.lo[0], bx.hi[0], env_unit(seed, 5 * k));
    c.y = env_lerp(bx.lo[1], bx.hi[1], env_unit(seed, 5 * k + 1));
    c.z = env_lerp(bx.lo[2], bx.hi[2], env_unit(seed, 5 * k + 2));
    c.R = env_lerp(bx.R_lo, bx.R_hi, env_unit(seed, 5 * k + 3));
    c.p0 = env_lerp(bx.p_lo, bx.p_hi, env_unit(seed, 5 * k + 4));
    return c;
}

// flags[j] for candidate first + j, and the block's accepted count
__global__ void __launch_bounds__(kEnvThreads)
env_sample_classify_kernel(const double* __restrict__ tri, const float* __restrict__ ftri, int F,
                           double inset, RayFrame fr, uint64_t seed, long long first,
                           long long n_cand, SampleBox bx, unsigned char* __restrict__ flags,
                           long long* __restrict__ block_cnt) {
    __shared__ float s_tri[kTriTile * kFWords];
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = j < n_cand;
    Candidate c{0, 0, 0, 0, 0};
    if (active) c = env_candidate(seed, first + j, bx);
    const bool in = env_in_region(tri, ftri, F, inset, fr.e, fr.lmax, active, (double)c.x,
                                  (double)c.y, (double)c.z, s_tri);
    if (active) flags[j] = in ? 1 : 0;
    const int cnt = __syncthreads_count(in);
    if (threadIdx.x == 0) block_cnt[blockIdx.x] = cnt;
}

// exclusive offsets of the block counts (one CTA), total in block_cnt[nb]
__global__ void env_scan_kernel(long long* __restrict__ block_cnt, int nb) {
    __shared__ long long warp_tot[32];
    long long carry = 0;
    for (int b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int b = b0 + threadIdx.x;
        const long long v = b < nb ? block_cnt[b] : 0;
        long long tot;
        const long long incl = sbp_block_incl_scan(v, warp_tot, tot);
        if (b < nb) block_cnt[b] = carry + incl - v;
        carry += tot;
    }
    if (threadIdx.x == 0) block_cnt[nb] = carry;
}

// accepted candidates, in candidate order, to out[0 .. n_want)
__global__ void __launch_bounds__(kEnvThreads)
env_sample_scatter_kernel(uint64_t seed, long long first, long long n_cand, SampleBox bx,
                          const unsigned char* __restrict__ flags,
                          const long long* __restrict__ block_off, int n_want, sbp_balls out,
                          int* __restrict__ n_out) {
    __shared__ long long warp_tot[32];
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int f = j < n_cand ? flags[j] : 0;
    long long tot;
    const long long incl = sbp_block_incl_scan(f, warp_tot, tot);
    const long long pos = block_off[blockIdx.x] + incl - f;
    if (f && pos < n_want) {
        const Candidate c = env_candidate(seed, first + j, bx);
        out.x[pos] = c.x;
        out.y[pos] = c.y;
        out.z[pos] = c.z;
        out.R[pos] = c.R;
        out.p0[pos] = c.p0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const long long total = block_off[gridDim.x];
        *n_out = (int)(total < n_want ? total : n_want);
    }
}

// ---------------------------------------------------------------------------
// device: voxel grid
// ---------------------------------------------------------------------------

__global__ void vox_max_kernel(const float* __restrict__ v, const int* n_dev, int n_cap,
                               unsigned int* bits) {
    const int n = sbp_read_n(n_dev, n_cap);
    float m = 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(v[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(bits, __float_as_uint(m));
}

__device__ __forceinline__ int vox_frac_bits(unsigned int bits) {
    int e = 0;
    const float m = __uint_as_float(bits);
    if (m > 0.0f) frexpf(m, &e);  // m < 2^e
    const int F = kVoxFracHeadroom - e;
    return F < -60 ? -60 : (F > 120 ? 120 : F);
}

struct VoxGrid {
    double o[3];
    double h;
    int n[3];
    float of[3], hf;  // the origin and spacing rounded to float
    float E;          // bound on |x_f - x| of a float voxel-centre coordinate minus a ball's
};

// The exact test of reading 19, in double with explicit rounding:
// (dx^2 + dy^2) + dz^2 < R^2, dx = (o + (i + 1/2) h) - c.
__device__ __forceinline__ bool vox_inside_exact(const VoxGrid& grid, const double* c, double R2,
                                                 int ii, int j, int k) {
    const double xc = __dadd_rn(grid.o[0], __dmul_rn((double)ii + 0.5, grid.h));
    const double yc = __dadd_rn(grid.o[1], __dmul_rn((double)j + 0.5, grid.h));
    const double zc = __dadd_rn(grid.o[2], __dmul_rn((double)k + 0.5, grid.h));
    const double dx = __dsub_rn(xc, c[0]), dy = __dsub_rn(yc, c[1]), dz = __dsub_rn(zc, c[2]);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return d2 < R2;
}

// One thread per ball: every voxel of its bounding range whose centre lies
// inside the ball gets round(value 2^F) added (integer atomics, so the sum
// does not depend on the order). The test is first made in float: each float
// offset dx_f differs from the exact dx by at most E (grid.E, bounded on the
// host) plus its own rounding, so |d2_f - d2| stays below
// 2 (|dx_f| + |dy_f| + |dz_f| + 3E) E + 2^-20 (d2_f + R^2), and a voxel
// further than that from the sphere is decided in float with the exact
// test's outcome. The few voxels within that margin take the exact test.
__global__ void vox_scatter_kernel(BallsDev b, const float* __restrict__ val, const int* n_dev,
                                   int n_cap, VoxGrid grid, const unsigned int* bits,
                                   unsigned long long* __restrict__ acc) {
    const int n = sbp_read_n(n_dev, n_cap);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float Rf = b.R[i];
    const double R = (double)Rf;
    if (!(R > 0.0)) return;
    const float cf[3] = {b.x[i], b.y[i], b.z[i]};
    const double c[3] = {(double)cf[0], (double)cf[1], (double)cf[2]};
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        const double fl = floor((c[a] - R - grid.o[a]) / grid.h) - 1.0;
        const double ce = ceil((c[a] + R - grid.o[a]) / grid.h) + 1.0;
        lo[a] = (int)fmax(0.0, fmin(fl, (double)grid.n[a]));
        hi[a] = (int)fmin((double)grid.n[a] - 1.0, fmax(ce, -1.0));
        if (lo[a] > hi[a]) return;
    }
    const double v = (double)val[i];
    const double scale = ldexp(1.0, vox_frac_bits(*bits));
    const long long q = __double2ll_rn(v * scale);
    if (q == 0) return;
    const double R2 = __dmul_rn(R, R);
    const float R2f = Rf * Rf, E = grid.E;
    for (int k = lo[2]; k <= hi[2]; ++k) {
        const float dz = fmaf((float)k + 0.5f, grid.hf, grid.of[2]) - cf[2];
        for (int j = lo[1]; j <= hi[1]; ++j) {
            const float dy = fmaf((float)j + 0.5f, grid.hf, grid.of[1]) - cf[1];
            const float dyz2 = fmaf(dy, dy, dz * dz);
            const float ayz = fabsf(dy) + fabsf(dz) + 3.0f * E;
            unsigned long long* row = acc + ((size_t)k * grid.n[1] + j) * grid.n[0];
            for (int ii = lo[0]; ii <= hi[0]; ++ii) {
                const float dx = fmaf((float)ii + 0.5f, grid.hf, grid.of[0]) - cf[0];
                const float d2 = fmaf(dx, dx, dyz2);
                const float margin = fmaf(2.0f * (fabsf(dx) + ayz), E, 9.5367431640625e-7f * (d2 + R2f));
                bool in;
                if (d2 < R2f - margin) in = true;
                else if (d2 > R2f + margin) in = false;
                else in = vox_inside_exact(grid, c, R2, ii, j, k);
                if (in) atomicAdd(row + ii, (unsigned long long)q);
            }
        }
    }
}

__global__ void vox_finalize_kernel(unsigned long long* __restrict__ acc, long long total,
                                    const unsigned int* bits, float* __restrict__ out) {
    // 2^-F as a float (F in [-60, 120], so it is a normal float); the sum is
    // converted by two 32-bit conversions (|q| < 2^40), not on the FP64 pipe
    const float inv = __int_as_float((127 - vox_frac_bits(*bits)) << 23);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long q = (long long)acc[t];
        out[t] = fmaf((float)(int)(q >> 32), 4294967296.0f, (float)(unsigned int)q) * inv;
        acc[t] = 0ull;
    }
}

RayFrame env_frame(sbp_envelope env) {
    RayFrame f;
    for (int k = 0; k < 6; ++k) f.e[k] = env->frame[k];
    f.lmax = env->lmax;
    return f;
}

int env_check_device(sbp_envelope env, const char* what) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != env->device) {
        sbp_set_error(std::string(what) + ": the envelope belongs to another device");
        return SBP_ERR_ARG;
    }
    return SBP_OK;
}

}  // namespace

extern "C" {

int sbp_envelope_create(const float* pos_host, int M, sbp_envelope* out) {
    if (!pos_host || !out || M < 4) {
        sbp_set_error("envelope_create: null pointer or fewer than 4 sensors");
        return SBP_ERR_ARG;
    }
    *out = nullptr;
    std::vector<double> P(3 * (size_t)M);
    for (int i = 0; i < 3 * M; ++i) {
        P[i] = (double)pos_host[i];
        if (!std::isfinite(P[i])) {
            sbp_set_error("envelope_create: non-finite sensor coordinate");
            return SBP_ERR_NUMERIC;
        }
    }
    std::vector<int> tri;
    std::string err;
    if (!build_hull(P, M, tri, err)) {
        sbp_set_error(err);
        return SBP_ERR_ARG;
    }
    sbp_envelope e = new sbp_envelope_s();
    if (cudaGetDevice(&e->device) != cudaSuccess) {
        delete e;
        sbp_set_error("envelope_create: no CUDA device");
        return SBP_ERR_CUDA;
    }
    e->M = M;
    e->F = (int)(tri.size() / 3);
    e->tri = tri;
    for (int k = 0; k < 3; ++k) {
        e->lo[k] = P[k];
        e->hi[k] = P[k];
    }
    for (int i = 0; i < M; ++i)
        for (int k = 0; k < 3; ++k) {
            e->lo[k] = std::min(e->lo[k], P[3 * i + k]);
            e->hi[k] = std::max(e->hi[k], P[3 * i + k]);
        }
    std::vector<double> words((size_t)e->F * kTriWords);
    double vol = 0;
    for (int f = 0; f < e->F; ++f) {
        const double* a = &P[3 * tri[3 * f]];
        const double* b = &P[3 * tri[3 * f + 1]];
        const double* c = &P[3 * tri[3 * f + 2]];
        double* w = &words[(size_t)f * kTriWords];
        HFace hf{tri[3 * f], tri[3 * f + 1], tri[3 * f + 2], {0, 0, 0}, 0, true};
        face_plane(P, hf);
        for (int k = 0; k < 3; ++k) {
            w[k] = a[k];
            w[3 + k] = b[k] - a[k];
            w[6 + k] = c[k] - a[k];
            w[9 + k] = hf.n[k];
        }
        w[12] = hf.d;
        vol += (a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) +
                a[2] * (b[0] * c[1] - b[1] * c[0])) / 6.0;
    }
    e->volume = vol;
    // the frame across the ray: e_u = normalise(z x d), e_v = d x e_u
    const double* d = kRayDirHost;
    double eu[3] = {-d[1], d[0], 0.0};
    const double nu = std::sqrt(eu[0] * eu[0] + eu[1] * eu[1]);
    eu[0] /= nu;
    eu[1] /= nu;
    const double ev[3] = {d[1] * eu[2] - d[2] * eu[1], d[2] * eu[0] - d[0] * eu[2],
                          d[0] * eu[1] - d[1] * eu[0]};
    for (int k = 0; k < 3; ++k) {
        e->frame[k] = eu[k];
        e->frame[3 + k] = ev[k];
        e->lmax = std::max(e->lmax, std::max(std::fabs(e->lo[k]), std::fabs(e->hi[k])));
    }
    std::vector<float> fw((size_t)e->F * kFWords);
    for (int f = 0; f < e->F; ++f) {
        const double* w = &words[(size_t)f * kTriWords];
        double uv[3][2];
        for (int q = 0; q < 3; ++q) {
            double v[3];
            for (int k = 0; k < 3; ++k) v[k] = w[k] + (q == 1 ? w[3 + k] : q == 2 ? w[6 + k] : 0.0);
            uv[q][0] = v[0] * eu[0] + v[1] * eu[1] + v[2] * eu[2];
            uv[q][1] = v[0] * ev[0] + v[1] * ev[1] + v[2] * ev[2];
        }
        float* o = &fw[(size_t)f * kFWords];
        for (int q = 0; q < 3; ++q) {
            const int r = (q + 1) % 3;
            const double du = uv[r][0] - uv[q][0], dv = uv[r][1] - uv[q][1];
            o[2 * q] = (float)uv[q][0];
            o[2 * q + 1] = (float)uv[q][1];
            o[6 + 2 * q] = (float)du;
            o[7 + 2 * q] = (float)dv;
            o[16 + q] = (float)((std::fabs(du) + std::fabs(dv)) * (1.0 + 1e-6));
        }
        o[12] = (float)std::min({uv[0][0], uv[1][0], uv[2][0]});
        o[13] = (float)std::max({uv[0][0], uv[1][0], uv[2][0]});
        o[14] = (float)std::min({uv[0][1], uv[1][1], uv[2][1]});
        o[15] = (float)std::max({uv[0][1], uv[1][1], uv[2][1]});
        for (int k = 0; k < 3; ++k) {
            o[19 + k] = (float)w[9 + k];
            o[22 + k] = (float)w[k];
        }
        const double nd = w[9] * d[0] + w[10] * d[1] + w[11] * d[2];
        o[25] = nd > 0.0 ? 1.0f : -1.0f;
    }
    bool ok = !sbp_cuda_check(cudaMalloc(&e->d_tri, sizeof(double) * words.size()),
                              "envelope_create: alloc") &&
              !sbp_cuda_check(cudaMemcpy(e->d_tri, words.data(), sizeof(double) * words.size(),
                                         cudaMemcpyHostToDevice),
                              "envelope_create: copy") &&
              !sbp_cuda_check(cudaMalloc(&e->d_ftri, sizeof(float) * fw.size()),
                              "envelope_create: alloc") &&
              !sbp_cuda_check(cudaMemcpy(e->d_ftri, fw.data(), sizeof(float) * fw.size(),
                                         cudaMemcpyHostToDevice),
                              "envelope_create: copy");
    if (!ok) {
        cudaFree(e->d_tri);
        cudaFree(e->d_ftri);
        delete e;
        return SBP_ERR_CUDA;
    }
    *out = e;
    return SBP_OK;
}

int sbp_envelope_destroy(sbp_envelope env) {
    if (!env) return SBP_OK;
    cudaDeviceSynchronize();
    cudaFree(env->d_tri);
    cudaFree(env->d_ftri);
    cudaFree(env->d_flags);
    cudaFree(env->d_block);
    delete env;
    return SBP_OK;
}

int sbp_envelope_info(sbp_envelope env, int* n_faces, double* volume, double* bbox6) {
    if (!env) {
        sbp_set_error("envelope_info: null envelope");
        return SBP_ERR_ARG;
    }
    if (n_faces) *n_faces = env->F;
    if (volume) *volume = env->volume;
    if (bbox6)
        for (int k = 0; k < 3; ++k) {
            bbox6[k] = env->lo[k];
            bbox6[3 + k] = env->hi[k];
        }
    return SBP_OK;
}

int sbp_envelope_faces(sbp_envelope env, int* tri_host) {
    if (!env || !tri_host) {
        sbp_set_error("envelope_faces: null pointer");
        return SBP_ERR_ARG;
    }
    std::copy(env->tri.begin(), env->tri.end(), tri_host);
    return SBP_OK;
}

int sbp_envelope_classify(sbp_envelope env, const float* x_dev, const float* y_dev,
                          const float* z_dev, long long n, double inset,
                          unsigned char* inside_dev, sbp_stream stream) {
    if (!env || !x_dev || !y_dev || !z_dev || !inside_dev || n < 0 || !(inset >= 0.0)) {
        sbp_set_error("envelope_classify: invalid argument");
        return SBP_ERR_ARG;
    }
    if (int e = env_check_device(env, "envelope_classify")) return e;
    if (n == 0) return SBP_OK;
    const long long blocks = (n + kEnvThreads - 1) / kEnvThreads;
    env_classify_kernel<<<(unsigned)blocks, kEnvThreads, 0,
                          reinterpret_cast<cudaStream_t>(stream)>>>(
        env->d_tri, env->d_ftri, env->F, inset, env_frame(env), x_dev, y_dev, z_dev, n,
        inside_dev);
    sbp_count_launches(1);
    return sbp_cuda_check(cudaGetLastError(), "envelope_classify launch") ? SBP_ERR_CUDA : SBP_OK;
}

int sbp_envelope_sample(sbp_envelope env, uint64_t seed, long long first, long long n_cand,
                        double inset, double R_lo, double R_hi, double p_lo, double p_hi,
                        sbp_balls out, int n_want, int* n_dev, sbp_stream stream) {
    if (!env || !out.x || !out.y || !out.z || !out.R || !out.p0 || !n_dev || first < 0 ||
        n_cand < 1 || n_want < 0 || !(inset >= 0.0) || !(R_hi >= R_lo) || !(p_hi >= p_lo) ||
        first > (1LL << 60) / 5 || n_cand > (1LL << 31) * (long long)kEnvThreads) {
        sbp_set_error("envelope_sample: invalid argument");
        return SBP_ERR_ARG;
    }
    if (int e = env_check_device(env, "envelope_sample")) return e;
    const long long nb = (n_cand + kEnvThreads - 1) / kEnvThreads;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (env->flags_cap < n_cand || env->block_cap < nb + 1) {
        if (sbp_cuda_check(cudaStreamSynchronize(st), "envelope_sample: synchronise"))
            return SBP_ERR_CUDA;
        cudaFree(env->d_flags);
        cudaFree(env->d_block);
        env->d_flags = nullptr;
        env->d_block = nullptr;
        env->flags_cap = env->block_cap = 0;
        if (sbp_cuda_check(cudaMalloc(&env->d_flags, (size_t)n_cand), "envelope_sample: alloc") ||
            sbp_cuda_check(cudaMalloc(&env->d_block, sizeof(long long) * (size_t)(nb + 1)),
                           "envelope_sample: alloc"))
            return SBP_ERR_CUDA;
        env->flags_cap = n_cand;
        env->block_cap = nb + 1;
    }
    SampleBox bx;
    for (int k = 0; k < 3; ++k) {
        bx.lo[k] = env->lo[k];
        bx.hi[k] = env->hi[k];
    }
    bx.R_lo = R_lo;
    bx.R_hi = R_hi;
    bx.p_lo = p_lo;
    bx.p_hi = p_hi;
    env_sample_classify_kernel<<<(unsigned)nb, kEnvThreads, 0, st>>>(
        env->d_tri, env->d_ftri, env->F, inset, env_frame(env), seed, first, n_cand, bx,
        env->d_flags, env->d_block);
    env_scan_kernel<<<1, 1024, 0, st>>>(env->d_block, (int)nb);
    env_sample_scatter_kernel<<<(unsigned)nb, kEnvThreads, 0, st>>>(
        seed, first, n_cand, bx, env->d_flags, env->d_block, n_want, out, n_dev);
    sbp_count_launches(3);
    return sbp_cuda_check(cudaGetLastError(), "envelope_sample launch") ? SBP_ERR_CUDA : SBP_OK;
}

int sbp_voxelize(sbp_balls balls, const float* value_dev, const int* n_dev, int n_cap,
                 const double* origin3, double spacing, int nx, int ny, int nz,
                 unsigned long long* scratch_dev, float* vol_dev, sbp_stream stream) {
    if (!balls.x || !balls.y || !balls.z || !balls.R || !balls.p0 || n_cap < 0 || !origin3 ||
        !(spacing > 0.0) || nx < 1 || ny < 1 || nz < 1 || !scratch_dev || !vol_dev ||
        (long long)nx * ny * nz > (1LL << 40)) {
        sbp_set_error("voxelize: invalid argument");
        return SBP_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const long long total = (long long)nx * ny * nz;
    unsigned int* bits = reinterpret_cast<unsigned int*>(scratch_dev + total);
    const float* val = value_dev ? value_dev : balls.p0;
    VoxGrid grid;
    for (int k = 0; k < 3; ++k) grid.o[k] = origin3[k];
    grid.h = spacing;
    grid.n[0] = nx;
    grid.n[1] = ny;
    grid.n[2] = nz;
    // float centre x_f = fl(fl(i + 1/2) hf + of) against x = fl(fl((i + 1/2) h) + o):
    // |x_f - x| <= |o - of| + (n + 1) |h - hf| + two roundings of |x| plus one
    // of x itself, and the subtraction of the ball's coordinate (at most
    // |x| + 2 R away, bounded by the extent here with slack) one more
    grid.hf = (float)spacing;
    double E = 0.0;
    for (int k = 0; k < 3; ++k) {
        grid.of[k] = (float)origin3[k];
        const double ext = std::fabs(origin3[k]) + (grid.n[k] + 1.0) * spacing;
        const double e = std::fabs(origin3[k] - (double)grid.of[k]) +
                         (grid.n[k] + 1.0) * std::fabs(spacing - (double)grid.hf) +
                         4.0 * ext * 5.9604644775390625e-8;
        E = std::max(E, e);
    }
    grid.E = (float)(E * 2.0) + 1e-30f;  // twice the bound, rounded up
    if (sbp_cuda_check(cudaMemsetAsync(bits, 0, sizeof(unsigned int), st), "voxelize: reset"))
        return SBP_ERR_CUDA;
    int launched = 0;
    if (n_cap > 0) {
        const int blocks = std::max(1, std::min(1024, (n_cap + 255) / 256));
        vox_max_kernel<<<blocks, 256, 0, st>>>(val, n_dev, n_cap, bits);
        const BallsDev bd{balls.x, balls.y, balls.z, balls.R, balls.p0};
        vox_scatter_kernel<<<(n_cap + 127) / 128, 128, 0, st>>>(bd, val, n_dev, n_cap, grid, bits,
                                                                scratch_dev);
        launched += 2;
    }
    const int fb = (int)std::max<long long>(1, std::min<long long>(4096, (total + 255) / 256));
    vox_finalize_kernel<<<fb, 256, 0, st>>>(scratch_dev, total, bits, vol_dev);
    if (sbp_cuda_check(cudaMemsetAsync(bits, 0, sizeof(unsigned int), st), "voxelize: clear"))
        return SBP_ERR_CUDA;
    sbp_count_launches(launched + 1);
    return sbp_cuda_check(cudaGetLastError(), "voxelize launch") ? SBP_ERR_CUDA : SBP_OK;
}

}  // extern "C"
