/*
 * oracle.c -- plain, slow, FP64 CPU oracle for FFT-based rigid alignment of
 * closed planar curves (Dogan, Bernal & Hagwood, arXiv 2501.17779).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * it is used by tests/, by __graft_entry__.smoke() and by bench.py's CPU
 * baseline leg.  It shares no code, header, table or helper with the CUDA
 * library; the only thing the two sides share is the seeded input generator.
 *
 * What it computes (no FFT anywhere -- the oracle is the plain definition the
 * fast method must reproduce exactly, Sec. 2 "exactly the same alignment
 * error values"):
 *
 *   O1  oracle_align_pairs: for every cyclic start point s (Eq. A-mtx), the
 *       2x2 matrix A(s), its SVD, the proper-rotation Kabsch solution of
 *       Algorithm 1, tr(R A^T); the shift with the lowest discrete energy
 *       (Eq. disc-energy) wins; the energy at the winner is evaluated
 *       directly from its definition.
 *   O2  oracle_resample: arc-length parameter of Eq. arc-length-param, a
 *       periodic C2 cubic spline through (s^l, beta^l), evaluated at uniform
 *       parameters (Sec. 2, resampling paragraph), then centring and
 *       unit-length scaling (Sec. 1, Sec. 2 first paragraph).
 *
 * Conventions (readings of the paper, each listed in the design notes):
 *   - a curve is n DISTINCT nodes, closure implicit; the paper lists N points
 *     with first = last (Sec. 2), i.e. N-1 distinct nodes.  If a caller
 *     passes the closing duplicate, it is dropped.
 *   - h = 1/N with N distinct nodes (the paper's h = 1/(N-1) counts the
 *     duplicate endpoint).
 *   - shift s in [0, N) is the paper's m = s+1, t0 = s*h; curve 2 is read at
 *     index k+s (mod N).
 *   - theta is the COUNTER-clockwise angle of the optimal rotation applied to
 *     curve 2.  The paper writes R(theta) = [[cos, sin], [-sin, cos]], a
 *     clockwise rotation, so the paper's theta is the negative of ours.
 *   - ties in energy go to the smallest shift.
 *
 * Arrays of complex numbers are interleaved (x0, y0, x1, y1, ...), which is
 * also numpy's complex128 layout.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_ERR_ARG (-1)

/* status codes written per item (same meaning as the library's) */
#define ST_OK 0
#define ST_DEGENERATE 1
#define ST_NONFINITE 2

/* flags for oracle_resample */
#define OR_CENTER 1
#define OR_UNIT_LENGTH 2

/* ------------------------------------------------------------------------ */
/* 2x2 SVD, written out from the eigen-decomposition of A^T A.               */
/*   A (row-major a11 a12 a21 a22) = U diag(s1, s2) V^T, s1 >= s2 >= 0,       */
/*   U and V orthogonal (their determinants may be +1 or -1).                 */
/* Step 1: one Jacobi rotation V0 = [[c,-s],[s,c]] diagonalises the symmetric */
/*         matrix A^T A = [[p,q],[q,r]]: tan(2w) = 2q/(p-r).                  */
/* Step 2: B = A V0 has orthogonal columns; their norms are the singular      */
/*         values and the normalised columns are U's columns.                 */
/* Step 3: order the singular values descending (swapping V's columns too).   */
/* ------------------------------------------------------------------------ */
int oracle_svd2x2(const double* A, double* U, double* S, double* V)
{
    const double a11 = A[0], a12 = A[1], a21 = A[2], a22 = A[3];
    const double p = a11 * a11 + a21 * a21;
    const double q = a11 * a12 + a21 * a22;
    const double r = a12 * a12 + a22 * a22;
    const double w = 0.5 * atan2(2.0 * q, p - r);
    const double c = cos(w), s = sin(w);
    /* V0 columns: v1 = (c, s), v2 = (-s, c) */
    double v1x = c, v1y = s, v2x = -s, v2y = c;
    /* B = A V0 */
    double b1x = a11 * v1x + a12 * v1y, b1y = a21 * v1x + a22 * v1y;
    double b2x = a11 * v2x + a12 * v2y, b2y = a21 * v2x + a22 * v2y;
    double s1 = sqrt(b1x * b1x + b1y * b1y);
    double s2 = sqrt(b2x * b2x + b2y * b2y);
    if (s2 > s1) {
        double t;
        t = s1; s1 = s2; s2 = t;
        t = b1x; b1x = b2x; b2x = t;
        t = b1y; b1y = b2y; b2y = t;
        t = v1x; v1x = v2x; v2x = t;
        t = v1y; v1y = v2y; v2y = t;
    }
    double u1x, u1y, u2x, u2y;
    if (s1 > 0.0) { u1x = b1x / s1; u1y = b1y / s1; }
    else { u1x = 1.0; u1y = 0.0; }
    /* In exact arithmetic b2 is orthogonal to b1, so u2 = +-(-u1y, u1x); the
     * sign and s2 come from projecting b2 on that direction, which keeps U
     * orthogonal even when s2 is at rounding level (rank-deficient A). */
    {
        const double t = -u1y * b2x + u1x * b2y;
        if (t >= 0.0) { u2x = -u1y; u2y = u1x; s2 = t; }
        else { u2x = u1y; u2y = -u1x; s2 = -t; }
    }
    U[0] = u1x; U[1] = u2x; U[2] = u1y; U[3] = u2y; /* columns u1, u2 */
    V[0] = v1x; V[1] = v2x; V[2] = v1y; V[3] = v2y; /* columns v1, v2 */
    S[0] = s1; S[1] = s2;
    return ORACLE_OK;
}

static double det2(const double* M) { return M[0] * M[3] - M[1] * M[2]; }

/* Algorithm 1 (Kabsch): from A = U S V^T, S~ = diag(1, sign(det U det V)),
 * R = U S~ V^T.  Writes R (row-major) and returns tr(R A^T). */
double oracle_kabsch(const double* A, double* R)
{
    double U[4], S[2], V[4];
    oracle_svd2x2(A, U, S, V);
    const double d = (det2(U) * det2(V) > 0.0) ? 1.0 : -1.0;
    /* R = U diag(1, d) V^T ;  (U D)_{ij} = U_{ij} D_j ; R_{ik} = sum_j U_{ij} D_j V_{kj} */
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 2; ++k)
            R[2 * i + k] = U[2 * i + 0] * 1.0 * V[2 * k + 0] + U[2 * i + 1] * d * V[2 * k + 1];
    /* tr(R A^T) = sum_{ij} R_ij A_ij */
    return R[0] * A[0] + R[1] * A[1] + R[2] * A[2] + R[3] * A[3];
}

/* Eq. A-mtx: A_kj(s) = sum_l beta1_k^l beta2_j^{l (+) s}, with curve 2 read
 * at index l+s (mod N). */
static void corr_matrix(const double* z1, const double* z2, int N, int s, double* A)
{
    double a11 = 0, a12 = 0, a21 = 0, a22 = 0;
    for (int l = 0; l < N; ++l) {
        const int m = (l + s) % N;
        const double x1 = z1[2 * l], y1 = z1[2 * l + 1];
        const double x2 = z2[2 * m], y2 = z2[2 * m + 1];
        a11 += x1 * x2; a12 += x1 * y2;
        a21 += y1 * x2; a22 += y1 * y2;
    }
    A[0] = a11; A[1] = a12; A[2] = a21; A[3] = a22;
}

/* Per-shift best score tr(R(s) A(s)^T) with the Kabsch rotation (the loop of
 * Algorithm 2, evaluated by the O(N) definition instead of FFTs). */
int oracle_shift_scores(const double* z1, const double* z2, int N, double* score)
{
    if (!z1 || !z2 || !score || N <= 0) return ORACLE_ERR_ARG;
    for (int s = 0; s < N; ++s) {
        double A[4], R[4];
        corr_matrix(z1, z2, N, s, A);
        score[s] = oracle_kabsch(A, R);
    }
    return ORACLE_OK;
}

static int all_finite(const double* z, int n2)
{
    for (int i = 0; i < n2; ++i)
        if (!isfinite(z[i])) return 0;
    return 1;
}

/* O1 for one pair.  Energies follow Eq. disc-energy with h = 1/N:
 *   E(s) = h (sum|z1|^2 + sum|z2|^2 - 2 tr(R(s) A(s)^T))   (Sec. 2 rewrite)
 * The winner's energy is recomputed directly as h sum ||b1 - R b2||^2.      */
static void align_one(const double* z1, const double* z2, int N, int* shift, double* theta,
                      double* energy, double* gap, signed char* status)
{
    if (!all_finite(z1, 2 * N) || !all_finite(z2, 2 * N)) {
        *shift = -1; *theta = NAN; *energy = NAN; *gap = NAN; *status = ST_NONFINITE;
        return;
    }
    const double h = 1.0 / (double)N;
    double n1 = 0, n2 = 0;
    for (int l = 0; l < N; ++l) {
        n1 += z1[2 * l] * z1[2 * l] + z1[2 * l + 1] * z1[2 * l + 1];
        n2 += z2[2 * l] * z2[2 * l] + z2[2 * l + 1] * z2[2 * l + 1];
    }
    int best = 0;
    double Ebest = INFINITY, E2 = INFINITY, Rbest[4] = {1, 0, 0, 1};
    for (int s = 0; s < N; ++s) {
        double A[4], R[4];
        corr_matrix(z1, z2, N, s, A);
        const double tr = oracle_kabsch(A, R);
        const double E = h * (n1 + n2 - 2.0 * tr);
        if (E < Ebest) {
            E2 = Ebest;
            Ebest = E;
            best = s;
            memcpy(Rbest, R, sizeof(R));
        } else if (E < E2) {
            E2 = E;
        }
    }
    /* direct energy at the winner (Eq. disc-energy) */
    double Ed = 0;
    for (int l = 0; l < N; ++l) {
        const int m = (l + best) % N;
        const double x2 = z2[2 * m], y2 = z2[2 * m + 1];
        const double rx = Rbest[0] * x2 + Rbest[1] * y2;
        const double ry = Rbest[2] * x2 + Rbest[3] * y2;
        const double dx = z1[2 * l] - rx, dy = z1[2 * l + 1] - ry;
        Ed += dx * dx + dy * dy;
    }
    *shift = best;
    *theta = atan2(Rbest[2], Rbest[0]); /* CCW angle of R = [[c,-s],[s,c]] */
    *energy = h * Ed;
    *gap = (N > 1) ? (E2 - Ebest) : INFINITY;
    *status = ST_OK;
}

int oracle_align_pairs(const double* z1, const double* z2, int64_t P, int N, int nthreads,
                       int32_t* shift, double* theta, double* energy, double* gap,
                       signed char* status)
{
    if (!z1 || !z2 || !shift || !theta || !energy || !gap || !status || P < 0 || N <= 0)
        return ORACLE_ERR_ARG;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t p = 0; p < P; ++p) {
        int sh;
        align_one(z1 + 2 * (size_t)N * p, z2 + 2 * (size_t)N * p, N, &sh, theta + p, energy + p,
                  gap + p, status + p);
        shift[p] = sh;
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* O2: arc-length resampling (Sec. 2, Eq. arc-length-param and the cubic     */
/* spline interpolation that follows it).                                   */
/* ------------------------------------------------------------------------ */

/* Cyclic tridiagonal solve for one right-hand side:
 *   a[i] x[i-1] + b[i] x[i] + c[i] x[i+1] = d[i],   indices mod n, n >= 3.
 * Thomas algorithm on the system with its corner entries removed, plus the
 * Sherman-Morrison correction for the rank-one corner term (textbook method,
 * e.g. Numerical Recipes "cyclic").  Work arrays w1..w4 have length n.      */
static void cyclic_thomas(int n, const double* a, const double* b, const double* c,
                          const double* d, double* x, double* w_bb, double* w_u, double* w_z,
                          double* w_cp)
{
    /* corner terms: alpha = c[n-1] (row n-1, col 0), beta = a[0] (row 0, col n-1) */
    const double alpha = c[n - 1], beta = a[0];
    const double gamma = -b[0];
    for (int i = 0; i < n; ++i) w_bb[i] = b[i];
    w_bb[0] = b[0] - gamma;
    w_bb[n - 1] = b[n - 1] - alpha * beta / gamma;
    /* solve T' x = d and T' z = u with u = (gamma, 0, ..., 0, alpha) */
    for (int i = 0; i < n; ++i) w_u[i] = 0.0;
    w_u[0] = gamma;
    w_u[n - 1] = alpha;
    /* Thomas (two right-hand sides, one factorisation) */
    double den = w_bb[0];
    w_cp[0] = c[0] / den;
    x[0] = d[0] / den;
    w_z[0] = w_u[0] / den;
    for (int i = 1; i < n; ++i) {
        den = w_bb[i] - a[i] * w_cp[i - 1];
        w_cp[i] = (i < n - 1) ? c[i] / den : 0.0;
        x[i] = (d[i] - a[i] * x[i - 1]) / den;
        w_z[i] = (w_u[i] - a[i] * w_z[i - 1]) / den;
    }
    for (int i = n - 2; i >= 0; --i) {
        x[i] -= w_cp[i] * x[i + 1];
        w_z[i] -= w_cp[i] * w_z[i + 1];
    }
    /* Sherman-Morrison with v = (1, 0, ..., 0, beta/gamma) */
    const double vx = x[0] + beta * x[n - 1] / gamma;
    const double vz = w_z[0] + beta * w_z[n - 1] / gamma;
    const double fact = vx / (1.0 + vz);
    for (int i = 0; i < n; ++i) x[i] -= fact * w_z[i];
}

static void resample_one(const double* pts, int64_t n_in, int N, int flags, double* out,
                         signed char* status)
{
    int64_t n = n_in;
    for (int k = 0; k < N; ++k) { out[2 * k] = NAN; out[2 * k + 1] = NAN; }
    if (!all_finite(pts, (int)(2 * n))) { *status = ST_NONFINITE; return; }
    /* first = last convention of the paper: drop an explicit closing duplicate */
    if (n >= 2 && pts[0] == pts[2 * (n - 1)] && pts[1] == pts[2 * (n - 1) + 1]) n -= 1;
    if (n < 4) { *status = ST_DEGENERATE; return; }

    double* d = (double*)malloc(sizeof(double) * (size_t)n);   /* chord lengths     */
    double* u = (double*)malloc(sizeof(double) * (size_t)(n + 1)); /* knots s^l     */
    double* hh = (double*)malloc(sizeof(double) * (size_t)n);  /* knot spacings     */
    double* A = (double*)malloc(sizeof(double) * (size_t)n);
    double* B = (double*)malloc(sizeof(double) * (size_t)n);
    double* Cc = (double*)malloc(sizeof(double) * (size_t)n);
    double* rx = (double*)malloc(sizeof(double) * (size_t)n);
    double* ry = (double*)malloc(sizeof(double) * (size_t)n);
    double* Mx = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    double* My = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    double* w = (double*)malloc(sizeof(double) * (size_t)(4 * n));

    /* Eq. arc-length-param: cumulative chord length, normalised by the total */
    double L = 0.0;
    int bad = 0;
    for (int64_t l = 0; l < n; ++l) {
        const int64_t m = (l + 1) % n;
        const double dx = pts[2 * m] - pts[2 * l], dy = pts[2 * m + 1] - pts[2 * l + 1];
        d[l] = sqrt(dx * dx + dy * dy);
        if (!(d[l] > 0.0)) bad = 1; /* a repeated node gives a zero-length knot interval */
        L += d[l];
    }
    if (bad || !(L > 0.0) || !isfinite(L)) {
        *status = ST_DEGENERATE;
        goto done;
    }
    {
        double acc = 0.0;
        u[0] = 0.0;
        for (int64_t l = 1; l < n; ++l) { acc += d[l - 1]; u[l] = acc / L; }
        u[n] = 1.0;
        for (int64_t l = 0; l < n; ++l) hh[l] = u[l + 1] - u[l];
        for (int64_t l = 0; l < n; ++l)
            if (!(hh[l] > 0.0)) { *status = ST_DEGENERATE; goto done; }

        /* Periodic cubic spline: second derivatives M_l at the knots satisfy
         *   h_{l-1} M_{l-1} + 2(h_{l-1}+h_l) M_l + h_l M_{l+1}
         *      = 6[(p_{l+1}-p_l)/h_l - (p_l-p_{l-1})/h_{l-1}],  l mod n.       */
        for (int64_t l = 0; l < n; ++l) {
            const int64_t lm = (l + n - 1) % n, lp = (l + 1) % n;
            const double hm = hh[lm], hl = hh[l];
            A[l] = hm;
            B[l] = 2.0 * (hm + hl);
            Cc[l] = hl;
            rx[l] = 6.0 * ((pts[2 * lp] - pts[2 * l]) / hl - (pts[2 * l] - pts[2 * lm]) / hm);
            ry[l] = 6.0 * ((pts[2 * lp + 1] - pts[2 * l + 1]) / hl -
                           (pts[2 * l + 1] - pts[2 * lm + 1]) / hm);
        }
        cyclic_thomas((int)n, A, B, Cc, rx, Mx, w, w + n, w + 2 * n, w + 3 * n);
        cyclic_thomas((int)n, A, B, Cc, ry, My, w, w + n, w + 2 * n, w + 3 * n);
        Mx[n] = Mx[0];
        My[n] = My[0];

        /* evaluate at t_k = k/N (textbook form of the cubic on [u_l, u_{l+1}]) */
        int64_t l = 0;
        for (int k = 0; k < N; ++k) {
            const double t = (double)k / (double)N;
            while (l < n - 1 && u[l + 1] <= t) ++l;
            const int64_t lp = (l + 1) % n;
            const double hl = hh[l];
            const double A1 = u[l + 1] - t, B1 = t - u[l];
            const double x0 = pts[2 * l], y0 = pts[2 * l + 1];
            const double x1 = pts[2 * lp], y1 = pts[2 * lp + 1];
            out[2 * k] = (Mx[l] * A1 * A1 * A1 + Mx[l + 1] * B1 * B1 * B1) / (6.0 * hl) +
                         (x0 / hl - Mx[l] * hl / 6.0) * A1 + (x1 / hl - Mx[l + 1] * hl / 6.0) * B1;
            out[2 * k + 1] = (My[l] * A1 * A1 * A1 + My[l + 1] * B1 * B1 * B1) / (6.0 * hl) +
                             (y0 / hl - My[l] * hl / 6.0) * A1 + (y1 / hl - My[l + 1] * hl / 6.0) * B1;
        }
    }
    /* centring at the node mean (reading of "centered at the origin") */
    if (flags & OR_CENTER) {
        double mx = 0, my = 0;
        for (int k = 0; k < N; ++k) { mx += out[2 * k]; my += out[2 * k + 1]; }
        mx /= (double)N;
        my /= (double)N;
        for (int k = 0; k < N; ++k) { out[2 * k] -= mx; out[2 * k + 1] -= my; }
    }
    /* unit length: closed-polygon perimeter of the N resampled nodes = 1 */
    if (flags & OR_UNIT_LENGTH) {
        double per = 0;
        for (int k = 0; k < N; ++k) {
            const int kp = (k + 1) % N;
            const double dx = out[2 * kp] - out[2 * k], dy = out[2 * kp + 1] - out[2 * k + 1];
            per += sqrt(dx * dx + dy * dy);
        }
        if (!(per > 0.0) || !isfinite(per)) {
            for (int k = 0; k < N; ++k) { out[2 * k] = NAN; out[2 * k + 1] = NAN; }
            *status = ST_DEGENERATE;
            goto done;
        }
        for (int k = 0; k < N; ++k) { out[2 * k] /= per; out[2 * k + 1] /= per; }
    }
    *status = ST_OK;
done:
    free(d); free(u); free(hh); free(A); free(B); free(Cc);
    free(rx); free(ry); free(Mx); free(My); free(w);
}

int oracle_resample(const double* pts, const int64_t* offsets, int64_t C, int N, int flags,
                    int nthreads, double* z_out, signed char* status)
{
    if (!pts || !offsets || !z_out || !status || C < 0 || N <= 0) return ORACLE_ERR_ARG;
    for (int64_t i = 0; i < C; ++i)
        if (offsets[i + 1] < offsets[i]) return ORACLE_ERR_ARG;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t i = 0; i < C; ++i)
        resample_one(pts + 2 * offsets[i], offsets[i + 1] - offsets[i], N, flags,
                     z_out + 2 * (size_t)N * i, status + i);
    return ORACLE_OK;
}

/* the number of OpenMP threads a parallel region would use (for reports) */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
