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
 *   O3  oracle_elastic_pairs: the elastic shape distance of Sec. 3: SRV
 *       functions, Eq. dist2-energy, "Approach 2" started from the FFT
 *       pre-alignment (here: O2 then O1), alternating a (t0,R)-step (O1 on
 *       SRV cell averages) with a gamma-step; the gamma-step is a lattice-path
 *       dynamic programme of the builder's own design (the paper takes its
 *       gamma-step from a reference it does not reproduce).
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
#define ST_BADSIZE 3

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

/* ------------------------------------------------------------------------ */
/* O3: elastic shape distance (Sec. 3): SRV functions, the energy of         */
/* Eq. dist2-energy and the alternation of "Approach 2" started from the    */
/* FFT pre-alignment of the arc-length-resampled curves.                     */
/*                                                                          */
/* Discretisation (readings of Sec. 3):                                     */
/*  - a curve is N nodes, node k at parameter t = k/N, scaled so that its   */
/*    closed polygon has unit length.  The SRV function                    */
/*    q = beta'/|beta'|^{1/2} is sampled at the cell midpoints              */
/*    t = (k + 1/2)/N from the chords: q_k = v_k/|v_k|^{1/2},              */
/*    v_k = N (beta[k+1] - beta[k]); (1/N) sum |q_k|^2 = 1.  Between samples */
/*    q is the periodic Catmull-Rom interpolant: in cell units u, with      */
/*    j = floor(u - 1/2), f = u - 1/2 - j, the cubic Hermite segment from   */
/*    q_j to q_{j+1} with tangents (q_{j+1} - q_{j-1})/2, (q_{j+2} - q_j)/2.*/
/*  - gamma is piecewise linear on the t-grid with node values g_k =        */
/*    N gamma(k/N), increasing, g_N = g_0 + N (gamma(t+1) = gamma(t) + 1;   */
/*    the dynamic programme fixes g_0 = 0, the refinement frees it, which   */
/*    with the grid shift s makes t0 continuous); Eq. dist2-energy by the  */
/*    midpoint rule:                                                        */
/*      E = (1/N) sum_k |q1s_k - sqrt(D_k) q2(M_k)|^2,                      */
/*      q1s_k = e^{i theta} q1[(k+s) mod N] (R q1(t + t0), t0 = s/N),       */
/*      D_k = g_{k+1} - g_k (= gamma'), M_k = (g_k + g_{k+1})/2.            */
/*  - the gamma-step (the builder's own: the paper takes its gamma-step     */
/*    from its reference [dogan] without stating it) is                     */
/*      (a) a dynamic programme over lattice paths from (0,0) to (N,N)      */
/*          with steps (a,b), 1 <= a,b <= 3, gcd(a,b) = 1 (slopes b/a in    */
/*          [1/3, 3]), optionally kept in the band |i - j| <= B, minimising */
/*          E over those paths; run on the first iteration only             */
/*          (later the refined gamma carries over: a new shift s from the   */
/*          (t0,R)-step keeps gamma and lowers E, and the refinement's free  */
/*          offset g_0 follows it);                                         */
/*      (b) a continuous refinement of all g_k (g_0 too) jointly with theta:*/
/*          damped Newton (Levenberg-Marquardt) steps on E = (1/N) sum      */
/*          |r_k|^2, r_k = q1s_k - sqrt(D_k) q2(M_k): the Hessian (the        */
/*          Gauss-Newton part, damped, plus the residual-curvature terms)   */
/*          is tridiagonal in g with a border for theta; each step shortened*/
/*          to keep every D_k above half its value and accepted only if E   */
/*          decreases; at most 64 steps, ending after an accepted step that  */
/*          lowers E by <= 1e-12 E or once the damping exceeds 1e6.          */
/*          Without theta in it the alternation converges only              */
/*          linearly (gamma partly absorbs a rotation error); without the   */
/*          curvature terms the steps converge only linearly where rotation */
/*          and the offset nearly trade off (round shapes).                 */
/*  - the (t0,R)-step is the rigid alignment of Sec. 2 (O1's criterion) of  */
/*    w_k = sqrt(D_k) q2(M_k) against q1 over all grid shifts s.            */
/* ------------------------------------------------------------------------ */

#define EL_NSTEPS 7
#define EL_LM_ITERS 64    /* Levenberg-Marquardt steps per gamma-step, at most */
#define EL_LM_TOL 1e-12   /* ... ending after an accepted step that lowers E by <= this */
                          /*     fraction of it                                      */
#define EL_LM_STALL 1e6   /* ... or once the damping exceeds this */
/* (a, b) = (cells along t, cells along gamma); this order is also the tie  */
/* order of the dynamic programme (the first best step wins).               */
static const int EL_STEP[EL_NSTEPS][2] = {{1, 1}, {1, 2}, {2, 1}, {1, 3}, {3, 1}, {2, 3},
                                          {3, 2}};

/* q(u): the periodic Catmull-Rom interpolant of the midpoint samples (the */
/* cubic Hermite curve through them with central-difference tangents, C1,   */
/* so that the energy is continuously differentiable in g); dq = dq/du.     */
static void el_interp2(const double* q, int N, double u, double* v, double* dq, double* ddq)
{
    const double x = u - 0.5;
    const double fl = floor(x);
    const double f = x - fl;
    int j = (int)fmod(fl, (double)N);
    if (j < 0) j += N;
    const int jm = (j + N - 1) % N, j1 = (j + 1) % N, j2 = (j + 2) % N;
    const double f2 = f * f, f3 = f2 * f;
    const double w[4] = {0.5 * (-f3 + 2.0 * f2 - f), 0.5 * (3.0 * f3 - 5.0 * f2 + 2.0),
                         0.5 * (-3.0 * f3 + 4.0 * f2 + f), 0.5 * (f3 - f2)};
    const double d[4] = {0.5 * (-3.0 * f2 + 4.0 * f - 1.0), 0.5 * (9.0 * f2 - 10.0 * f),
                         0.5 * (-9.0 * f2 + 8.0 * f + 1.0), 0.5 * (3.0 * f2 - 2.0 * f)};
    const double dd[4] = {-3.0 * f + 2.0, 9.0 * f - 5.0, -9.0 * f + 4.0, 3.0 * f - 1.0};
    const int id[4] = {jm, j, j1, j2};
    v[0] = v[1] = 0.0;
    for (int c = 0; c < 4; ++c) {
        v[0] += w[c] * q[2 * id[c]];
        v[1] += w[c] * q[2 * id[c] + 1];
    }
    if (dq) {
        dq[0] = dq[1] = 0.0;
        for (int c = 0; c < 4; ++c) {
            dq[0] += d[c] * q[2 * id[c]];
            dq[1] += d[c] * q[2 * id[c] + 1];
        }
    }
    if (ddq) {
        ddq[0] = ddq[1] = 0.0;
        for (int c = 0; c < 4; ++c) {
            ddq[0] += dd[c] * q[2 * id[c]];
            ddq[1] += dd[c] * q[2 * id[c] + 1];
        }
    }
}

static void el_interp(const double* q, int N, double u, double* v, double* dq)
{
    el_interp2(q, N, u, v, dq, NULL);
}

/* one cell's term |q1s_k - sqrt(D) q2(M)|^2 for gamma from x to y on it    */
static double el_term(const double* q1s, const double* q2, int N, int k, double x, double y)
{
    double v[2];
    el_interp(q2, N, 0.5 * (x + y), v, NULL);
    const double m = sqrt(y - x);
    const double dx = q1s[2 * k] - m * v[0], dy = q1s[2 * k + 1] - m * v[1];
    return dx * dx + dy * dy;
}

/* Eq. dist2-energy (midpoint rule) of node values g[0..N]                  */
static double el_energy(const double* q1s, const double* q2, int N, const double* g)
{
    double E = 0.0;
    for (int k = 0; k < N; ++k) E += el_term(q1s, q2, N, k, g[k], g[k + 1]);
    return E / (double)N;
}

/* (a) lattice-path dynamic programme over the cells' terms of the energy: */
/* V(i, j) is the least sum of |q1s_k - sqrt(D_k) q2(M_k)|^2 over the      */
/* cells k < i of a lattice path from (0, 0) to (i, j); a step (a, b)     */
/* covers cells i-a .. i-1, each with slope D = b/a and gamma running      */
/* linearly from j-b to j (the same el_term as the energy).  FP64          */
/* throughout.  Among equal sums the first step in EL_STEP order wins.     */
/* The minimising path's node values are written to g[0..N]; its energy is */
/* returned.                                                               */
static double el_dp(const double* q1s, const double* q2, int N, int band, double* g)
{
    const int M = N + 1;
    double* V = (double*)malloc(sizeof(double) * (size_t)M * M);
    signed char* arg = (signed char*)malloc((size_t)M * M);
    for (int x = 0; x < M * M; ++x) { V[x] = INFINITY; arg[x] = -1; }
    V[0] = 0.0;
    for (int i = 1; i <= N; ++i)
        for (int j = 1; j <= N; ++j) {
            if (band >= 0 && abs(i - j) > band) continue;
            double best = INFINITY;
            int bi = -1;
            for (int st = 0; st < EL_NSTEPS; ++st) {
                const int a = EL_STEP[st][0], b = EL_STEP[st][1];
                if (i - a < 0 || j - b < 0) continue;
                const double prev = V[(i - a) * M + (j - b)];
                if (prev == INFINITY) continue;
                double acc = 0.0;
                for (int p = 0; p < a; ++p) {
                    const double x = (double)(j - b) + (double)(p * b) / (double)a;
                    const double y = (double)(j - b) + (double)((p + 1) * b) / (double)a;
                    acc += el_term(q1s, q2, N, i - a + p, x, y);
                }
                const double c = prev + acc;
                if (c < best) { best = c; bi = st; }
            }
            V[i * M + j] = best;
            arg[i * M + j] = (signed char)bi;
        }
    int i = N, j = N;
    g[N] = (double)N;
    while (i > 0) {
        const int a = EL_STEP[arg[i * M + j]][0], b = EL_STEP[arg[i * M + j]][1];
        for (int p = 0; p < a; ++p) g[i - a + p] = (double)(j - b) + (double)(p * b) / (double)a;
        i -= a;
        j -= b;
    }
    free(V); free(arg);
    return el_energy(q1s, q2, N, g);
}

/* q1s_k = e^{i theta} q1[(k + s) mod N]  (the motion R q1(t + t0))        */
static void el_move(const double* q1, int N, int s, double theta, double* q1s)
{
    const double c = cos(theta), sn = sin(theta);
    for (int k = 0; k < N; ++k) {
        const double* u = q1 + 2 * ((k + s) % N);
        q1s[2 * k] = c * u[0] - sn * u[1];
        q1s[2 * k + 1] = sn * u[0] + c * u[1];
    }
}

/* (b) Levenberg-Marquardt refinement of gamma and theta for the fixed      */
/* shift s.  Unknowns: the interior node values h_1..h_{N-1} of             */
/* g_k = c + h_k (h_0 = 0, h_N = N), the offset c = g_0 (gamma extended     */
/* periodically, gamma(t+1) = gamma(t) + 1, so that together with the grid  */
/* shift s the start point t0 is continuous as in Eq. dist2-energy) and the */
/* rotation increment phi; residuals r_k = e^{i phi} q1s_k -                */
/* sqrt(D_k) q2(M_k).  Newton matrix: J^T J with its diagonal scaled by     */
/* (1 + lambda), plus sum_k <r_k, d2 r_k>; it is tridiagonal in h with a    */
/* two-column border (c, phi): Thomas algorithm on three right-hand sides,  */
/* then a 2x2 Schur complement.  Returns the energy of the refined          */
/* (theta, g).                                                              */
static double el_refine(const double* q1, const double* q2, int N, int s, double* theta,
                        double* g, int iters)
{
    const int n = N - 1;
    const size_t cz = sizeof(double) * 2 * (size_t)N;
    const size_t cn = sizeof(double) * (size_t)(N + 1);
    double* q1s = (double*)malloc(cz);
    double* qt = (double*)malloc(cz);
    el_move(q1, N, s, *theta, q1s);
    double E = el_energy(q1s, q2, N, g);
    double* Ar = (double*)malloc(cz);  /* d r_k / d g_k     */
    double* Br = (double*)malloc(cz);  /* d r_k / d g_{k+1} */
    double* R = (double*)malloc(cz);   /* r_k               */
    double* x = (double*)malloc(cn);   /* T^-1 (-grad_h)    */
    double* yc = (double*)malloc(cn);  /* T^-1 C_c          */
    double* yp = (double*)malloc(cn);  /* T^-1 C_phi        */
    double* Cc = (double*)malloc(cn);
    double* Cp = (double*)malloc(cn);
    double* gt = (double*)malloc(cn);
    double* lo = (double*)malloc(cn);
    double* di = (double*)malloc(cn);
    double* up = (double*)malloc(cn);
    double* Saa = (double*)malloc(cn);  /* <r_k, d2 r_k / d g_k^2>           */
    double* Sbb = (double*)malloc(cn);  /* <r_k, d2 r_k / d g_{k+1}^2>       */
    double* Sab = (double*)malloc(cn);  /* <r_k, d2 r_k / d g_k d g_{k+1}>   */
    double lambda = 1e-3;
    for (int it = 0; it < iters && n >= 1; ++it) {
        double Hcc = 0.0, Hcp = 0.0, Hpp = 0.0, Gc = 0.0, Gp = 0.0, Scc = 0.0, Spp = 0.0;
        for (int k = 0; k < N; ++k) {
            double v[2], dv[2], ddv[2];
            const double D = g[k + 1] - g[k];
            el_interp2(q2, N, 0.5 * (g[k] + g[k + 1]), v, dv, ddv);
            const double m = sqrt(D);
            R[2 * k] = q1s[2 * k] - m * v[0];
            R[2 * k + 1] = q1s[2 * k + 1] - m * v[1];
            /* r = q1s - sqrt(D) q2(M), with D = g_{k+1} - g_k, M = (g_k + g_{k+1})/2:
             * r_D = -q2/(2 sqrt D), r_M = -sqrt(D) q2', r_DD = q2/(4 D^{3/2}),
             * r_DM = -q2'/(2 sqrt D), r_MM = -sqrt(D) q2'';
             * d/dg_k = -d/dD + d/dM / 2, d/dg_{k+1} = d/dD + d/dM / 2              */
            double saa = 0.0, sbb = 0.0, sab = 0.0;
            for (int c = 0; c < 2; ++c) {
                const double rD = -v[c] / (2.0 * m), rM = -m * dv[c];
                const double rDD = v[c] / (4.0 * D * m), rDM = -dv[c] / (2.0 * m);
                const double rMM = -m * ddv[c];
                Ar[2 * k + c] = -rD + 0.5 * rM;
                Br[2 * k + c] = rD + 0.5 * rM;
                saa += R[2 * k + c] * (rDD - rDM + 0.25 * rMM);
                sbb += R[2 * k + c] * (rDD + rDM + 0.25 * rMM);
                sab += R[2 * k + c] * (-rDD + 0.25 * rMM);
            }
            Saa[k] = saa;
            Sbb[k] = sbb;
            Sab[k] = sab;
            const double ux = Ar[2 * k] + Br[2 * k], uy = Ar[2 * k + 1] + Br[2 * k + 1];
            const double px = -q1s[2 * k + 1], py = q1s[2 * k];  /* dr/dphi = i q1s */
            Hcc += ux * ux + uy * uy;
            Hcp += ux * px + uy * py;
            Hpp += px * px + py * py;
            Gc += R[2 * k] * ux + R[2 * k + 1] * uy;
            Gp += R[2 * k] * px + R[2 * k + 1] * py;
            Scc += saa + 2.0 * sab + sbb;
            Spp -= R[2 * k] * q1s[2 * k] + R[2 * k + 1] * q1s[2 * k + 1];  /* d2r/dphi2 = -q1s */
        }
        /* rows i = 1..n (unknown h_i) */
        for (int i = 1; i <= n; ++i) {
            const double* b0 = Br + 2 * (i - 1);
            const double* a0 = Ar + 2 * (i - 1);
            const double* a1 = Ar + 2 * i;
            const double* b1 = Br + 2 * i;
            const double* p0 = q1s + 2 * (i - 1);
            const double* p1 = q1s + 2 * i;
            di[i] = (b0[0] * b0[0] + b0[1] * b0[1] + a1[0] * a1[0] + a1[1] * a1[1]) *
                        (1.0 + lambda) +
                    Sbb[i - 1] + Saa[i];
            x[i] = -(R[2 * (i - 1)] * b0[0] + R[2 * (i - 1) + 1] * b0[1] +
                     R[2 * i] * a1[0] + R[2 * i + 1] * a1[1]);
            Cc[i] = b0[0] * (a0[0] + b0[0]) + b0[1] * (a0[1] + b0[1]) +
                    a1[0] * (a1[0] + b1[0]) + a1[1] * (a1[1] + b1[1]) +
                    Sab[i - 1] + Sbb[i - 1] + Saa[i] + Sab[i];
            Cp[i] = b0[0] * -p0[1] + b0[1] * p0[0] + a1[0] * -p1[1] + a1[1] * p1[0];
            lo[i] = i > 1 ? a0[0] * b0[0] + a0[1] * b0[1] + Sab[i - 1] : 0.0;
            up[i] = i < n ? a1[0] * b1[0] + a1[1] * b1[1] + Sab[i] : 0.0;
            yc[i] = Cc[i];
            yp[i] = Cp[i];
        }
        /* Thomas algorithm on three right-hand sides */
        for (int i = 2; i <= n; ++i) {
            const double w = lo[i] / di[i - 1];
            di[i] -= w * up[i - 1];
            x[i] -= w * x[i - 1];
            yc[i] -= w * yc[i - 1];
            yp[i] -= w * yp[i - 1];
        }
        x[n] /= di[n];
        yc[n] /= di[n];
        yp[n] /= di[n];
        for (int i = n - 1; i >= 1; --i) {
            x[i] = (x[i] - up[i] * x[i + 1]) / di[i];
            yc[i] = (yc[i] - up[i] * yc[i + 1]) / di[i];
            yp[i] = (yp[i] - up[i] * yp[i + 1]) / di[i];
        }
        /* Schur complement S (2x2) and its right-hand side */
        double S00 = Hcc * (1.0 + lambda) + Scc, S01 = Hcp, S11 = Hpp * (1.0 + lambda) + Spp;
        double r0 = -Gc, r1 = -Gp;
        for (int i = 1; i <= n; ++i) {
            S00 -= Cc[i] * yc[i];
            S01 -= Cc[i] * yp[i];
            S11 -= Cp[i] * yp[i];
            r0 -= Cc[i] * x[i];
            r1 -= Cp[i] * x[i];
        }
        const double det = S00 * S11 - S01 * S01;
        double dc = 0.0, dphi = 0.0;
        if (det > 0.0) {
            dc = (S11 * r0 - S01 * r1) / det;
            dphi = (S00 * r1 - S01 * r0) / det;
        }
        /* the step on g: dg_k = dc + dh_k, dh_0 = dh_N = 0 */
        gt[0] = 0.0;
        gt[N] = 0.0;
        for (int i = 1; i <= n; ++i) gt[i] = x[i] - yc[i] * dc - yp[i] * dphi;
        /* shorten it so that every slope keeps at least half its value */
        double alpha = 1.0;
        for (int k = 0; k < N; ++k) {
            const double D = g[k + 1] - g[k], dD = gt[k + 1] - gt[k];
            if (dD < -0.5 * D) {
                const double a = -0.5 * D / dD;
                if (a < alpha) alpha = a;
            }
        }
        for (int k = 0; k <= N; ++k) gt[k] = g[k] + alpha * (dc + gt[k]);
        const double tht = *theta + alpha * dphi;
        el_move(q1, N, s, tht, qt);
        const double Et = el_energy(qt, q2, N, gt);
        if (Et < E) {
            const double drop = E - Et;
            const double Eold = E;
            memcpy(g, gt, cn);
            memcpy(q1s, qt, cz);
            *theta = tht;
            E = Et;
            lambda = lambda * 0.25 > 1e-12 ? lambda * 0.25 : 1e-12;
            if (drop <= EL_LM_TOL * Eold) break;  /* converged */
        } else {
            lambda *= 8.0;
            if (lambda > EL_LM_STALL) break;  /* no descent left at rounding level */
        }
    }
    free(q1s); free(qt); free(Ar); free(Br); free(R); free(x); free(yc); free(yp);
    free(Cc); free(Cp); free(gt); free(lo); free(di); free(up); free(Saa); free(Sbb); free(Sab);
    return E;
}

/* SRV samples of the unit-length polygon through N nodes; sigma[k]         */
/* (k = 0..N) is the cumulative chord-length fraction at node k             */
static int el_srv(const double* beta, int N, double* q, double* sigma)
{
    if (!all_finite(beta, 2 * N)) return ST_NONFINITE;
    double per = 0.0;
    sigma[0] = 0.0;
    for (int k = 0; k < N; ++k) {
        const int k1 = (k + 1) % N;
        const double dx = beta[2 * k1] - beta[2 * k], dy = beta[2 * k1 + 1] - beta[2 * k + 1];
        per += sqrt(dx * dx + dy * dy);
        sigma[k + 1] = per;
    }
    if (!(per > 0.0) || !isfinite(per)) return ST_DEGENERATE;
    for (int k = 0; k <= N; ++k) sigma[k] /= per;
    for (int k = 0; k < N; ++k) {
        const int k1 = (k + 1) % N;
        const double vx = (double)N * (beta[2 * k1] - beta[2 * k]) / per;
        const double vy = (double)N * (beta[2 * k1 + 1] - beta[2 * k + 1]) / per;
        const double r = sqrt(vx * vx + vy * vy);
        q[2 * k] = r > 0.0 ? vx / sqrt(r) : 0.0;
        q[2 * k + 1] = r > 0.0 ? vy / sqrt(r) : 0.0;
    }
    return ST_OK;
}

/* index of beta1's node nearest to the chord-length fraction tau (the     */
/* pre-alignment's start point, found on the arc-length-resampled curve,   */
/* carried back to beta1's own parameter; linear between nodes)            */
static int el_param_index(const double* sigma, int N, double tau)
{
    int k = 0;
    while (k + 1 < N && sigma[k + 1] <= tau) ++k;
    const double d = sigma[k + 1] - sigma[k];
    const double u = (double)k + (d > 0.0 ? (tau - sigma[k]) / d : 0.0);
    return (int)floor(u + 0.5) % N;
}

/* (t0,R)-step: O1's criterion on w_k = sqrt(D_k) q2(M_k) against q1:       */
/* c(s) = sum_k w_k conj(q1[k+s]); s = argmax |c| (smallest s on ties)      */
static void el_rigid(const double* q1, const double* q2, int N, const double* g, int* s,
                     double* theta)
{
    double* w = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    for (int k = 0; k < N; ++k) {
        double v[2];
        el_interp(q2, N, 0.5 * (g[k] + g[k + 1]), v, NULL);
        const double m = sqrt(g[k + 1] - g[k]);
        w[2 * k] = m * v[0];
        w[2 * k + 1] = m * v[1];
    }
    double bestm = -1.0, cx = 0.0, cy = 0.0;
    int bs = 0;
    for (int sh = 0; sh < N; ++sh) {
        double x = 0.0, y = 0.0;
        for (int k = 0; k < N; ++k) {
            const double* u = q1 + 2 * ((k + sh) % N);
            x += w[2 * k] * u[0] + w[2 * k + 1] * u[1];
            y += w[2 * k + 1] * u[0] - w[2 * k] * u[1];
        }
        const double m2 = x * x + y * y;
        if (m2 > bestm) { bestm = m2; bs = sh; cx = x; cy = y; }
    }
    *s = bs;
    *theta = atan2(cy, cx);
    free(w);
}

typedef struct {
    int32_t shift, iters;
    double theta, energy;
    signed char status;
} el_result;

/* The alternation of Approach 2 from a starting triple (s, theta, g):     */
/*   repeat: gamma-step ((a) on the first iteration when run_dp, then (b)); */
/*           (t0,R)-step;                                                   */
/*   until an iteration lowers the energy by at most 1e-12, or max_iter.    */
/* On return (s, theta, g) is the final triple; its energy is returned and  */
/* *iters holds the iterations run.                                         */
static double el_alternate(const double* q1, const double* q2, int N, int band, int max_iter,
                           int run_dp, int* s, double* th, double* g, int* iters,
                           double* trace)
{
    double* q1s = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    double Eprev = INFINITY, E = NAN;
    *iters = 0;
    for (int it = 1; it <= max_iter; ++it) {
        if (it == 1 && run_dp) {
            el_move(q1, N, *s, *th, q1s);
            el_dp(q1s, q2, N, band, g);
        }
        el_refine(q1, q2, N, *s, th, g, EL_LM_ITERS);
        el_rigid(q1, q2, N, g, s, th);
        el_move(q1, N, *s, *th, q1s);
        E = el_energy(q1s, q2, N, g);
        if (trace) trace[it - 1] = E;
        *iters = it;
        if (Eprev - E <= 1e-12) break;
        Eprev = E;
    }
    free(q1s);
    return E;
}

/* SRV samples of both curves and the pair's status (st_out); when         */
/* pre-alignment is wanted, also the FFT pre-alignment of Sec. 3 on the     */
/* arc-length-resampled curves (O2, then O1 with the motion on curve 1),    */
/* its start point carried back to curve 1's own parameter.                 */
static int el_prepare(const double* b1, const double* b2, int N, double* q1, double* q2,
                      int prealign, int* s, double* th)
{
    const size_t cz = sizeof(double) * 2 * (size_t)N;
    double* r1 = (double*)malloc(cz);
    double* r2 = (double*)malloc(cz);
    double* sg1 = (double*)malloc(sizeof(double) * (size_t)(N + 1));
    double* sg2 = (double*)malloc(sizeof(double) * (size_t)(N + 1));
    int st1 = el_srv(b1, N, q1, sg1), st2 = el_srv(b2, N, q2, sg2);
    signed char rs1 = ST_OK, rs2 = ST_OK;
    if (st1 == ST_OK && st2 == ST_OK) {
        resample_one(b1, N, N, OR_CENTER | OR_UNIT_LENGTH, r1, &rs1);
        resample_one(b2, N, N, OR_CENTER | OR_UNIT_LENGTH, r2, &rs2);
    }
    int st = st1 == ST_NONFINITE || st2 == ST_NONFINITE ? ST_NONFINITE
             : st1 != ST_OK ? st1 : st2 != ST_OK ? st2 : rs1 != ST_OK ? rs1 : rs2;
    if (st == ST_OK && prealign) {
        double e, gap;
        signed char ast;
        /* pre-alignment with the motion on curve 1: e^{i th} r1[k+s] ~ r2[k] */
        align_one(r2, r1, N, s, th, &e, &gap, &ast);
        *s = el_param_index(sg1, N, (double)*s / (double)N);
    }
    free(r1); free(r2); free(sg1); free(sg2);
    return st;
}

/* Approach 2 for one pair: the pre-alignment, gamma = identity, then the   */
/* alternation (with the dynamic programme on its first iteration).  With   */
/* start != NULL the pre-alignment and the programme are skipped and the    */
/* alternation starts from the given triple (start->shift, start->theta,   */
/* g_start).  The energy is that of the final triple.                       */
static void elastic_one(const double* b1, const double* b2, int N, int band, int max_iter,
                        const el_result* start, const double* g_start, el_result* res,
                        double* gamma, double* trace)
{
    res->shift = -1; res->iters = 0; res->theta = NAN; res->energy = NAN;
    if (trace)
        for (int m = 0; m < max_iter; ++m) trace[m] = NAN;
    if (gamma)
        for (int m = 0; m <= N; ++m) gamma[m] = NAN;
    const size_t cz = sizeof(double) * 2 * (size_t)N;
    double* q1 = (double*)malloc(cz);
    double* q2 = (double*)malloc(cz);
    double* g = (double*)malloc(sizeof(double) * (size_t)(N + 1));
    int s = 0;
    double th = 0.0;
    const int st = el_prepare(b1, b2, N, q1, q2, start == NULL, &s, &th);
    res->status = (signed char)st;
    if (st == ST_OK) {
        if (start) {
            s = start->shift;
            th = start->theta;
            memcpy(g, g_start, sizeof(double) * (size_t)(N + 1));
        } else {
            for (int k = 0; k <= N; ++k) g[k] = (double)k;
        }
        int iters = 0;
        res->energy = el_alternate(q1, q2, N, band, max_iter, start == NULL, &s, &th, g, &iters,
                                   trace);
        res->iters = iters;
        res->shift = s;
        res->theta = th;
        if (gamma) memcpy(gamma, g, sizeof(double) * (size_t)(N + 1));
    }
    free(q1); free(q2); free(g);
}

/* O3 on P pairs of N-node curves (complex interleaved, [P, N] each).      */
/* band < 0: the full lattice.  gamma ([P, N+1], g_k = N gamma(k/N)) and   */
/* trace ([P, max_iter], the energy after each iteration) may be NULL.     */
int oracle_elastic_pairs(const double* b1, const double* b2, int64_t P, int N, int band,
                         int max_iter, int nthreads, int32_t* shift, double* theta,
                         double* energy, int32_t* iters, signed char* status, double* gamma,
                         double* trace)
{
    if (!b1 || !b2 || !shift || !theta || !energy || !iters || !status || P < 0 || N < 4 ||
        max_iter < 1)
        return ORACLE_ERR_ARG;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t p = 0; p < P; ++p) {
        el_result r;
        elastic_one(b1 + 2 * (size_t)N * p, b2 + 2 * (size_t)N * p, N, band, max_iter, NULL,
                    NULL, &r, gamma ? gamma + (size_t)(N + 1) * p : NULL,
                    trace ? trace + (size_t)max_iter * p : NULL);
        shift[p] = r.shift; theta[p] = r.theta; energy[p] = r.energy;
        iters[p] = r.iters; status[p] = r.status;
    }
    return ORACLE_OK;
}

/* The alternation alone, from a given starting triple per pair: shift0,   */
/* theta0 and g0 ([P, N+1]) -- for instance another implementation's       */
/* lattice path -- then refinement and (t0,R)-steps exactly as in           */
/* oracle_elastic_pairs.  Outputs as there (gamma may be NULL).            */
int oracle_elastic_from_start(const double* b1, const double* b2, int64_t P, int N,
                              const int32_t* shift0, const double* theta0, const double* g0,
                              int max_iter, int nthreads, int32_t* shift, double* theta,
                              double* energy, int32_t* iters, signed char* status,
                              double* gamma)
{
    if (!b1 || !b2 || !shift0 || !theta0 || !g0 || !shift || !theta || !energy || !iters ||
        !status || P < 0 || N < 4 || max_iter < 1)
        return ORACLE_ERR_ARG;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t p = 0; p < P; ++p) {
        el_result r, st;
        st.shift = shift0[p];
        st.theta = theta0[p];
        if (st.shift < 0 || st.shift >= N) {
            shift[p] = -1; theta[p] = NAN; energy[p] = NAN; iters[p] = 0;
            status[p] = ST_BADSIZE;
            continue;
        }
        elastic_one(b1 + 2 * (size_t)N * p, b2 + 2 * (size_t)N * p, N, -1, max_iter, &st,
                    g0 + (size_t)(N + 1) * p, &r, gamma ? gamma + (size_t)(N + 1) * p : NULL,
                    NULL);
        shift[p] = r.shift; theta[p] = r.theta; energy[p] = r.energy;
        iters[p] = r.iters; status[p] = r.status;
    }
    return ORACLE_OK;
}

/* the pieces, one at a time (for tests)                                    */
double oracle_elastic_dp(const double* q1s, const double* q2, int N, int band, double* g)
{
    return el_dp(q1s, q2, N, band, g);
}

double oracle_elastic_refine(const double* q1, const double* q2, int N, int s, double* theta,
                             double* g, int iters)
{
    return el_refine(q1, q2, N, s, theta, g, iters);
}

double oracle_elastic_energy(const double* q1s, const double* q2, int N, const double* g)
{
    return el_energy(q1s, q2, N, g);
}

int oracle_srv(const double* beta, int N, double* q, double* sigma)
{
    if (!beta || !q || !sigma || N < 1) return ORACLE_ERR_ARG;
    return el_srv(beta, N, q, sigma);
}
