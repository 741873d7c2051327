/*
 * FP64 CPU oracle for the SlingBAG Pro differentiable radiator and its adjoint.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call this code;
 * it exists so that tests, the smoke check and the CPU-baseline leg of the
 * benchmark can check the CUDA path against a plain, slow, obviously correct
 * evaluation. It shares no code, header or constant with the CUDA library.
 *
 * What it computes (all in double precision, inputs given as doubles):
 *
 *  Forward ("Simulate", Section 4.2 eq. for y_sim and Section 4.3 eq. for
 *  y_sim^(k); the radiator itself is SlingBAG's, Section 4.1): ball i with
 *  centre c_i, radius R_i and initial pressure p0_i, seen by sensor m at
 *  distance d = |c_i - s_m|, radiates the uniform-sphere N-shaped wave
 *      p(t) = p0 * w * (d - c t) / (2 d)     for |d - c t| < R,   0 otherwise,
 *  weighted by the sensor-orientation factor w (reading: w = max(0, n.u),
 *  u = (c_i - s_m)/d; modes "none" w = 1 and "cos" w = n.u are selectable).
 *  Sample j of level k is the average of p(t) over the cell
 *  [j dt_k, (j+1) dt_k) (cell-average reading of the unspecified sampling).
 *  With e_a = d - c j dt_k, e_b = e_a - c dt_k and E(e) = clamp(e, -R, R),
 *      S[m][j] = sum_i p0_i * w_mi * (E(e_a)^2 - E(e_b)^2) / (4 d_mi c dt_k).
 *  Pairs with d <= R (sensor inside a ball) contribute nothing and are
 *  counted in the return value.
 *
 *  Adjoint (the backpropagation of Section 4.2 and Algorithm 1; the paper
 *  prints no gradient formulas, these are derived from the forward above):
 *  given G = dL/dS, for each pair with K = w / (4 d c dt_k),
 *      A = sum_j G_j (E(e_a)^2 - E(e_b)^2)
 *      B = sum_j G_j * 2 (E(e_a) [|e_a|<R] - E(e_b) [|e_b|<R])
 *      C = sum_j G_j ([|e_a|>R] - [|e_b|>R])
 *  and
 *      dL/dp0 += K A,   dL/dR += 2 p0 K R C,
 *      dL/dc  += p0 K (B - A/d) u + p0 A / (4 d c dt_k) * grad_c(w),
 *  with grad_c(n.u) = (n - (n.u) u) / d (times [n.u > 0] in the clamped mode).
 *
 *  Downsample (Section 4.3, eq. for y_real^(k)): block mean over f samples,
 *  the record zero-padded to a multiple of f.
 *
 * Loops run over sensors (forward) and balls (adjoint) with OpenMP when the
 * caller asks for more than one thread; the arithmetic of each output element
 * is the same sequential sum either way.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { W_CLAMP = 0, W_NONE = 1, W_COS = 2 };

static double clampd(double e, double R) {
    if (e > R) return R;
    if (e < -R) return -R;
    return e;
}

/* Orientation weight of a pair and the cosine it is built from. */
static double weight(int mode, double cosv) {
    if (mode == W_NONE) return 1.0;
    if (mode == W_COS) return cosv;
    return cosv > 0.0 ? cosv : 0.0;
}

/* Cells that can be non-zero for a pair: cell j is touched when
 * e_b < R and e_a > -R, i.e. (d-R)/h - 1 < j < (d+R)/h. One extra cell on
 * each side is included; those evaluate to exactly zero. */
static void window(double d, double R, double h, long T, long* j0, long* j1) {
    long a = (long)floor((d - R) / h) - 1;
    long b = (long)floor((d + R) / h) + 1;
    if (a < 0) a = 0;
    if (b > T - 1) b = T - 1;
    *j0 = a;
    *j1 = b;
}

long oracle_forward(long n, const double* bx, const double* by, const double* bz,
                    const double* bR, const double* bp0, long M, const double* spos,
                    const double* snrm, double c, double dt, long T, int wmode,
                    double* S, int nthreads) {
    long inside = 0;
    const double h = c * dt;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1) reduction(+ : inside)
#endif
    for (long m = 0; m < M; ++m) {
        double* row = S + m * T;
        for (long j = 0; j < T; ++j) row[j] = 0.0;
        const double sx = spos[3 * m], sy = spos[3 * m + 1], sz = spos[3 * m + 2];
        const double nx = snrm[3 * m], ny = snrm[3 * m + 1], nz = snrm[3 * m + 2];
        for (long i = 0; i < n; ++i) {
            const double dx = bx[i] - sx, dy = by[i] - sy, dz = bz[i] - sz;
            const double d = sqrt(dx * dx + dy * dy + dz * dz);
            const double R = bR[i];
            if (!(d > R)) {
                inside++;
                continue;
            }
            const double cosv = (nx * dx + ny * dy + nz * dz) / d;
            const double w = weight(wmode, cosv);
            const double amp = bp0[i] * w / (4.0 * d * h);
            long j0, j1;
            window(d, R, h, T, &j0, &j1);
            for (long j = j0; j <= j1; ++j) {
                const double ea = d - (double)j * h;
                const double eb = d - (double)(j + 1) * h;
                const double qa = clampd(ea, R), qb = clampd(eb, R);
                row[j] += amp * (qa * qa - qb * qb);
            }
        }
    }
    return inside;
}

/* mask bits: 1 = p0, 2 = R, 4 = centre (x, y, z). Masked-out gradients are
 * written as zero. gp0_abs (optional, may be NULL) receives sum_m |K A| per
 * ball, the scale against which the sign of dL/dp0 is judged. */
long oracle_adjoint(long n, const double* bx, const double* by, const double* bz,
                    const double* bR, const double* bp0, long M, const double* spos,
                    const double* snrm, double c, double dt, long T, int wmode,
                    const double* G, int mask, double* gx, double* gy, double* gz,
                    double* gR, double* gp0, double* gp0_abs, int nthreads) {
    long inside = 0;
    const double h = c * dt;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 64) reduction(+ : inside)
#endif
    for (long i = 0; i < n; ++i) {
        double ax = 0, ay = 0, az = 0, aR = 0, ap = 0, apabs = 0;
        const double R = bR[i], p0 = bp0[i];
        for (long m = 0; m < M; ++m) {
            const double sx = spos[3 * m], sy = spos[3 * m + 1], sz = spos[3 * m + 2];
            const double nx = snrm[3 * m], ny = snrm[3 * m + 1], nz = snrm[3 * m + 2];
            const double dx = bx[i] - sx, dy = by[i] - sy, dz = bz[i] - sz;
            const double d = sqrt(dx * dx + dy * dy + dz * dz);
            if (!(d > R)) {
                inside++;
                continue;
            }
            const double ux = dx / d, uy = dy / d, uz = dz / d;
            const double cosv = nx * ux + ny * uy + nz * uz;
            const double w = weight(wmode, cosv);
            const double K = w / (4.0 * d * h);
            const double* g = G + m * T;
            double A = 0.0, B = 0.0, Cs = 0.0;
            long j0, j1;
            window(d, R, h, T, &j0, &j1);
            for (long j = j0; j <= j1; ++j) {
                const double ea = d - (double)j * h;
                const double eb = d - (double)(j + 1) * h;
                const double qa = clampd(ea, R), qb = clampd(eb, R);
                const double ua = fabs(ea) < R ? 1.0 : 0.0, ub = fabs(eb) < R ? 1.0 : 0.0;
                const double ca = fabs(ea) > R ? 1.0 : 0.0, cb = fabs(eb) > R ? 1.0 : 0.0;
                A += g[j] * (qa * qa - qb * qb);
                B += g[j] * 2.0 * (qa * ua - qb * ub);
                Cs += g[j] * (ca - cb);
            }
            ap += K * A;
            apabs += fabs(K * A);
            aR += 2.0 * p0 * K * R * Cs;
            const double gd = p0 * K * (B - A / d);
            /* dL/dw; grad of w wrt the centre */
            const double gw = p0 * A / (4.0 * d * h);
            double wx = 0, wy = 0, wz = 0;
            if (wmode == W_COS || (wmode == W_CLAMP && cosv > 0.0)) {
                wx = (nx - cosv * ux) / d;
                wy = (ny - cosv * uy) / d;
                wz = (nz - cosv * uz) / d;
            }
            ax += gd * ux + gw * wx;
            ay += gd * uy + gw * wy;
            az += gd * uz + gw * wz;
        }
        gp0[i] = (mask & 1) ? ap : 0.0;
        gR[i] = (mask & 2) ? aR : 0.0;
        gx[i] = (mask & 4) ? ax : 0.0;
        gy[i] = (mask & 4) ? ay : 0.0;
        gz[i] = (mask & 4) ? az : 0.0;
        if (gp0_abs) gp0_abs[i] = apabs;
    }
    return inside;
}

/*
 * Gaussian-profile radiator (the variant of Section 4.1, where a ball is a
 * Gaussian spherical source of peak p0 and standard deviation a0; stored in
 * the R slot). The initial pressure p0 exp(-r^2 / (2 a^2)) launches the
 * outgoing spherical wave p(t) = p0 w (d - c t) exp(-(d - c t)^2 / (2 a^2)) / (2 d)
 * (the incoming half of the solution is dropped, the far field d >> a;
 * pairs with d <= 6 a are skipped and counted). Its cell average is
 *     S_j = p0 w a^2 [g(e_b) - g(e_a)] / (2 d c dt),   g(e) = exp(-e^2 / (2 a^2)),
 * with e_a = d - c j dt, e_b = e_a - c dt, evaluated here on every cell of
 * the record (no truncation of the support).
 */
long oracle_forward_gauss(long n, const double* bx, const double* by, const double* bz,
                          const double* ba, const double* bp0, long M, const double* spos,
                          const double* snrm, double c, double dt, long T, int wmode,
                          double* S, int nthreads) {
    long inside = 0;
    const double h = c * dt;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1) reduction(+ : inside)
#endif
    for (long m = 0; m < M; ++m) {
        double* row = S + m * T;
        for (long j = 0; j < T; ++j) row[j] = 0.0;
        const double sx = spos[3 * m], sy = spos[3 * m + 1], sz = spos[3 * m + 2];
        const double nx = snrm[3 * m], ny = snrm[3 * m + 1], nz = snrm[3 * m + 2];
        for (long i = 0; i < n; ++i) {
            const double dx = bx[i] - sx, dy = by[i] - sy, dz = bz[i] - sz;
            const double d = sqrt(dx * dx + dy * dy + dz * dz);
            const double a = ba[i];
            if (!(d > 6.0 * a)) {
                inside++;
                continue;
            }
            const double w = weight(wmode, (nx * dx + ny * dy + nz * dz) / d);
            const double amp = bp0[i] * w * a * a / (2.0 * d * h);
            for (long j = 0; j < T; ++j) {
                const double ea = d - (double)j * h, eb = ea - h;
                row[j] += amp * (exp(-eb * eb / (2.0 * a * a)) - exp(-ea * ea / (2.0 * a * a)));
            }
        }
    }
    return inside;
}

/* Adjoint of oracle_forward_gauss, derived from it: per pair, with
 * K = w a^2 / (2 d c dt) and the cell sums over q_j = G_j,
 *   A0 = sum_j G_j [g(e_b) - g(e_a)],
 *   A1 = sum_j G_j [-(e_b / a^2) g(e_b) + (e_a / a^2) g(e_a)],     (d/dd of the bracket)
 *   A2 = sum_j G_j [(e_b^2 / a^3) g(e_b) - (e_a^2 / a^3) g(e_a)],  (d/da of the bracket)
 *   dL/dp0 += K A0,   dL/da += p0 (2 K / a A0 + K A2),
 *   dL/dc  += p0 (-K / d A0 + K A1) u + p0 a^2 A0 / (2 d c dt) grad_c(w). */
long oracle_adjoint_gauss(long n, const double* bx, const double* by, const double* bz,
                          const double* ba, const double* bp0, long M, const double* spos,
                          const double* snrm, double c, double dt, long T, int wmode,
                          const double* G, int mask, double* gx, double* gy, double* gz,
                          double* ga, double* gp0, int nthreads) {
    long inside = 0;
    const double h = c * dt;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 64) reduction(+ : inside)
#endif
    for (long i = 0; i < n; ++i) {
        double ax = 0, ay = 0, az = 0, aa = 0, ap = 0;
        const double a = ba[i], p0 = bp0[i];
        for (long m = 0; m < M; ++m) {
            const double sx = spos[3 * m], sy = spos[3 * m + 1], sz = spos[3 * m + 2];
            const double nx = snrm[3 * m], ny = snrm[3 * m + 1], nz = snrm[3 * m + 2];
            const double dx = bx[i] - sx, dy = by[i] - sy, dz = bz[i] - sz;
            const double d = sqrt(dx * dx + dy * dy + dz * dz);
            if (!(d > 6.0 * a)) {
                inside++;
                continue;
            }
            const double ux = dx / d, uy = dy / d, uz = dz / d;
            const double cosv = nx * ux + ny * uy + nz * uz;
            const double w = weight(wmode, cosv);
            const double K = w * a * a / (2.0 * d * h);
            const double* g = G + m * T;
            double A0 = 0.0, A1 = 0.0, A2 = 0.0;
            for (long j = 0; j < T; ++j) {
                const double ea = d - (double)j * h, eb = ea - h;
                const double ga_ = exp(-ea * ea / (2.0 * a * a)), gb = exp(-eb * eb / (2.0 * a * a));
                A0 += g[j] * (gb - ga_);
                A1 += g[j] * (-(eb / (a * a)) * gb + (ea / (a * a)) * ga_);
                A2 += g[j] * ((eb * eb / (a * a * a)) * gb - (ea * ea / (a * a * a)) * ga_);
            }
            ap += K * A0;
            aa += p0 * (2.0 * K / a * A0 + K * A2);
            const double gd = p0 * (-K / d * A0 + K * A1);
            const double gw = p0 * a * a * A0 / (2.0 * d * h);
            double wx = 0, wy = 0, wz = 0;
            if (wmode == W_COS || (wmode == W_CLAMP && cosv > 0.0)) {
                wx = (nx - cosv * ux) / d;
                wy = (ny - cosv * uy) / d;
                wz = (nz - cosv * uz) / d;
            }
            ax += gd * ux + gw * wx;
            ay += gd * uy + gw * wy;
            az += gd * uz + gw * wz;
        }
        gp0[i] = (mask & 1) ? ap : 0.0;
        ga[i] = (mask & 2) ? aa : 0.0;
        gx[i] = (mask & 4) ? ax : 0.0;
        gy[i] = (mask & 4) ? ay : 0.0;
        gz[i] = (mask & 4) ? az : 0.0;
    }
    return inside;
}

void oracle_downsample(long M, long T, const double* y, long f, double* yk) {
    const long Tk = (T + f - 1) / f;
    for (long m = 0; m < M; ++m) {
        for (long j = 0; j < Tk; ++j) {
            double s = 0.0;
            for (long q = 0; q < f; ++q) {
                const long t = j * f + q;
                if (t < T) s += y[m * T + t];
            }
            yk[m * Tk + j] = s / (double)f;
        }
    }
}

int oracle_num_procs(void) {
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}
