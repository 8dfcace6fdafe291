// elastic.cu -- fa_elastic_distance: the elastic shape distance of Sec. 3,
// FP64, one CTA per curve pair (persistent grid, pairs taken from an atomic
// counter).
//
// Representation.  A curve is N nodes, node k at parameter t = k/N, scaled
// to a unit-length closed polygon.  Its SRV function q = beta'/|beta'|^{1/2}
// (Sec. 3) is sampled at the cell midpoints from the chords,
// q_k = v_k/|v_k|^{1/2}, v_k = N (beta[k+1] - beta[k]), and read between
// samples through the periodic Catmull-Rom cubic (C1).  gamma is piecewise
// linear with node values g_k = N gamma(k/N), g_N = g_0 + N.  Eq. dist2-energy
// is taken by the midpoint rule,
//     E = (1/N) sum_k |e^{i theta} q1[k+s] - sqrt(D_k) q2(M_k)|^2,
//     D_k = g_{k+1} - g_k,  M_k = (g_k + g_{k+1})/2.
//
// Method ("Approach 2" of Sec. 3, FFT-initialised).
//   prep kernel   per curve: SRV samples, chord-length fractions, status;
//                 the curves are also resampled uniformly in arc length
//                 (resample kernel) for the pre-alignment.
//   pair kernel   pre-alignment: FFT rigid alignment of the resampled curves
//                 (motion on curve 1), start point carried back to curve 1's
//                 own parameter; gamma = identity.  Then, until an iteration
//                 lowers E by at most 1e-12 (or max_iter):
//                   gamma-step (this library's own design; the paper takes
//                   its gamma-step from a reference it does not reproduce):
//                     (a) first iteration only: dynamic programme over lattice paths
//                         (0,0) -> (N,N) with steps (a,b), a,b <= 3, coprime,
//                         in the band |i - j| <= B, minimising E exactly;
//                     (b) damped Newton (Levenberg-Marquardt) steps on
//                         (g_0..g_{N-1}, theta): the Hessian (Gauss-Newton
//                         part plus the residual-curvature terms) is
//                         tridiagonal in the interior nodes with a border for
//                         the offset g_0 and the angle, solved by cyclic
//                         reduction (three right-hand sides) and
//                         a 2x2 Schur complement; at most 64 steps, ending
//                         after an accepted step gaining <= 1e-12 E;
//                   (t0,R)-step: the rigid alignment of Sec. 2 of
//                     w_k = sqrt(D_k) q2(M_k) against q1 over all grid shifts,
//                     by FFT (the correlation as in the rigid kernels), the
//                     winner's c(s) recomputed directly.
//
// Layout.  The pair CTA holds q1, q2, DFT(q1), two transform buffers, the
// node values and the solver arrays in shared memory; the dynamic programme's
// row values live in a 4-row ring (steps reach 3 rows back).  The
// Catmull-Rom values of q2 at the 8 fractional offsets the steps use, and
// the DP back-pointers, sit in shared memory when they fit and otherwise in a
// per-CTA slice of the workspace (generic pointers serve both).
#include <algorithm>
#include <cmath>

#include "cta_ops.cuh"
#include "fa_internal.cuh"
#include "fft_stages.cuh"

namespace fa {
namespace {

constexpr int kElT = 128;         // threads per pair CTA
constexpr int kNSteps = 7;
constexpr int kNFrac = 8;
constexpr int kLmIters = 64;       // Levenberg-Marquardt steps per gamma-step, at most,
constexpr double kLmTol = 1e-12;   // ending after an accepted step lowering E by <= kLmTol E
constexpr double kLmStall = 1e6;   // or once the damping exceeds this
constexpr double kStopDrop = 1e-12;

// lattice steps (a, b): a cells of q1 along t, b cells of q2 along gamma; this
// order is the tie order of the dynamic programme (the first best step wins)
__host__ __device__ constexpr int step_a(int st)
{
    return st == 0 ? 1 : st == 1 ? 1 : st == 2 ? 2 : st == 3 ? 1 : st == 4 ? 3 : st == 5 ? 2 : 3;
}
__host__ __device__ constexpr int step_b(int st)
{
    return st == 0 ? 1 : st == 1 ? 2 : st == 2 ? 1 : st == 3 ? 3 : st == 4 ? 1 : st == 5 ? 3 : 2;
}
__host__ __device__ constexpr int floor_div(int n, int d) { return n >= 0 ? n / d : -((-n + d - 1) / d); }
// cell p of a step: the midpoint of gamma on it is M = l + (2p+1) b / (2a), so the
// Catmull-Rom segment starts at sample l + jo with fraction rem / (2a)
__host__ __device__ constexpr int piece_num(int st, int p) { return (2 * p + 1) * step_b(st) - step_a(st); }
__host__ __device__ constexpr int piece_jo(int st, int p) { return floor_div(piece_num(st, p), 2 * step_a(st)); }
// the fraction in twelfths (2a divides 12 for a <= 3)
__host__ __device__ constexpr int piece_tw(int st, int p)
{
    return (piece_num(st, p) - piece_jo(st, p) * 2 * step_a(st)) * (12 / (2 * step_a(st)));
}
// the 8 fractions that occur, in twelfths: 0, 2, 3, 4, 6, 8, 9, 10
__host__ __device__ constexpr int frac_index(int tw)
{
    return tw == 0 ? 0 : tw == 2 ? 1 : tw == 3 ? 2 : tw == 4 ? 3 : tw == 6 ? 4 : tw == 8 ? 5 : tw == 9 ? 6 : 7;
}
__host__ __device__ constexpr int frac_tw(int f)
{
    return f == 0 ? 0 : f == 1 ? 2 : f == 2 ? 3 : f == 3 ? 4 : f == 4 ? 6 : f == 5 ? 8 : f == 6 ? 9 : 10;
}
static_assert(frac_tw(frac_index(piece_tw(6, 0))) == piece_tw(6, 0), "fraction table");
// sqrt(b/a) of each step, correctly rounded
__device__ __forceinline__ constexpr double step_m(int st)
{
    return st == 0 ? 1.0 : st == 1 ? 1.4142135623730951 : st == 2 ? 0.7071067811865476
         : st == 3 ? 1.7320508075688772 : st == 4 ? 0.5773502691896257
         : st == 5 ? 1.224744871391589 : 0.816496580927726;
}

// 1/sqrt(x) for x in (0, 2^100): float32 seed, two Newton steps in FP64
// (y <- y (3 - x y^2) / 2), relative error at rounding level
__device__ __forceinline__ double rsqrt_fast(double x)
{
    double y = (double)rsqrtf((float)x);
    y = y * fma(-0.5 * x, y * y, 1.5);
    y = y * fma(-0.5 * x, y * y, 1.5);
    return y;
}

struct ElasticArgs {
    const double2* q;       // SRV samples [Mtot][N]
    const double* sigma;    // chord-length fractions [Mtot][N+1]
    const double2* zr;      // arc-length resampled curves [Mtot][N]
    const int8_t* cst;      // per-curve status [Mtot]
    const int64_t* idx1;    // pair -> curve of set 1 (nullable: identity)
    const int64_t* idx2;    // pair -> curve of set 2 (nullable: identity)
    int64_t M1, M2, P;
    unsigned long long* next;  // work counter (zeroed before the launch)
    int N, logn, band, max_iter;
    double2* q2f_ws;        // per-CTA slices, used when q2f_smem == 0
    uint8_t* bp_ws;
    int64_t q2f_elems, bp_bytes;
    int q2f_smem, bp_smem;
    const double2* tf;      // FMA-form twiddles of size N
    int32_t* shift;
    double* theta;
    double* energy;
    double* gamma;          // nullable [P][N+1]
    int32_t* iters;         // nullable
    int32_t* lm_steps;      // nullable: refinement steps taken per pair
    int8_t* status;
};

// periodic Catmull-Rom value (and derivative in u) of the midpoint samples q at
// u (cell units; sample k sits at u = k + 1/2)
__device__ __forceinline__ void cr_eval(const double2* __restrict__ q, int N, double u, double2& v,
                                        double2* dv, double2* ddv = nullptr)
{
    const double x = u - 0.5;
    const double fl = floor(x);
    const double f = x - fl;
    const int j = ((int)fl) & (N - 1);
    const double2 p0 = q[(j - 1) & (N - 1)], p1 = q[j], p2 = q[(j + 1) & (N - 1)],
                  p3 = q[(j + 2) & (N - 1)];
    const double f2 = f * f, f3 = f2 * f;
    const double w0 = 0.5 * (-f3 + 2.0 * f2 - f), w1 = 0.5 * (3.0 * f3 - 5.0 * f2 + 2.0);
    const double w2 = 0.5 * (-3.0 * f3 + 4.0 * f2 + f), w3 = 0.5 * (f3 - f2);
    v.x = w0 * p0.x + w1 * p1.x + w2 * p2.x + w3 * p3.x;
    v.y = w0 * p0.y + w1 * p1.y + w2 * p2.y + w3 * p3.y;
    if (dv) {
        const double d0 = 0.5 * (-3.0 * f2 + 4.0 * f - 1.0), d1 = 0.5 * (9.0 * f2 - 10.0 * f);
        const double d2 = 0.5 * (-9.0 * f2 + 8.0 * f + 1.0), d3 = 0.5 * (3.0 * f2 - 2.0 * f);
        dv->x = d0 * p0.x + d1 * p1.x + d2 * p2.x + d3 * p3.x;
        dv->y = d0 * p0.y + d1 * p1.y + d2 * p2.y + d3 * p3.y;
    }
    if (ddv) {
        const double e0 = -3.0 * f + 2.0, e1 = 9.0 * f - 5.0, e2 = -9.0 * f + 4.0, e3 = 3.0 * f - 1.0;
        ddv->x = e0 * p0.x + e1 * p1.x + e2 * p2.x + e3 * p3.x;
        ddv->y = e0 * p0.y + e1 * p1.y + e2 * p2.y + e3 * p3.y;
    }
}

// K CTA sums of per-thread values; every thread gets the same totals
template <int T, int K>
__device__ __forceinline__ void cta_sums(double (&v)[K], double* red)
{
    constexpr int NW = T / 32;
#pragma unroll
    for (int c = 0; c < K; ++c)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], off);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int c = 0; c < K; ++c) red[w * K + c] = v[c];
    __syncthreads();
    if (threadIdx.x < K) {
        double s = red[threadIdx.x];
        for (int i = 1; i < NW; ++i) s += red[i * K + threadIdx.x];
        red[NW * K + threadIdx.x] = s;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < K; ++c) v[c] = red[NW * K + c];
    __syncthreads();
}

template <int T>
__device__ __forceinline__ double cta_min(double v, double* red)
{
    constexpr int NW = T / 32;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = red[0];
        for (int i = 1; i < NW; ++i) s = fmin(s, red[i]);
        red[NW] = s;
    }
    __syncthreads();
    v = red[NW];
    __syncthreads();
    return v;
}

__device__ __forceinline__ double2 rot(double2 c, double2 u)
{
    return make_double2(c.x * u.x - c.y * u.y, c.y * u.x + c.x * u.y);
}

// ----------------------------------------------------- dynamic programme ----
// The path costs are accumulated in float32 (the DP only chooses the
// refinement's starting path; every reported value is FP64): each cell's term
// is fmaf(dx, dx, fmaf(dy, dy, acc)) with dx = fmaf(-m, v_x, u_x), m = sqrt(b/a)
// rounded to float, and q1s, q2(M) rounded from FP64 -- the oracle performs the
// same operations in the same order.
template <int ST>
__device__ __forceinline__ void dp_steps(int i, int j, const float* __restrict__ V,
                                         int ring_stride, const float2* __restrict__ q1s,
                                         const float2* __restrict__ q2f, int fstride,
                                         float& best, int& arg)
{
    if constexpr (ST < kNSteps) {
        constexpr int a = step_a(ST), b = step_b(ST);
        if (i >= a && j >= b) {
            const float prev = V[((i - a) & 3) * ring_stride + (j - b)];
            constexpr float m = (float)step_m(ST);
            float acc = 0.0f;
#pragma unroll
            for (int p = 0; p < a; ++p) {
                const float2 u = q1s[i - a + p];
                // q2f rows hold samples -1 .. N; entry x sits at index x + 1
                const float2 v = q2f[frac_index(piece_tw(ST, p)) * fstride +
                                     (j - b + piece_jo(ST, p) + 1)];
                const float dx = fmaf(-m, v.x, u.x), dy = fmaf(-m, v.y, u.y);
                acc = fmaf(dx, dx, fmaf(dy, dy, acc));
            }
            const float c = prev + acc;
            if (c < best) { best = c; arg = ST; }
        }
        dp_steps<ST + 1>(i, j, V, ring_stride, q1s, q2f, fstride, best, arg);
    }
}

// node values g of the minimising lattice path for q1s (shared), q2f prepared
template <int T>
__device__ void elastic_dp(int N, int B, const float2* q1s, const float2* q2f, float* V,
                           uint8_t* bp, double* g)
{
    const int tid = threadIdx.x;
    const int rs = N + 1;
    const int W = B < N ? 2 * B + 1 : N;
    for (int x = tid; x <= N; x += T) V[x] = x == 0 ? 0.0f : HUGE_VALF;
    __syncthreads();
    for (int i = 1; i <= N; ++i) {
        const int jlo = max(1, i - B), jhi = min(N, i + B);
        const int base = B < N ? i - B : 1;
        float* Vi = V + (i & 3) * rs;
        for (int j = tid; j <= N; j += T) {
            float best = HUGE_VALF;
            if (j >= jlo && j <= jhi) {
                int arg = 255;
                dp_steps<0>(i, j, V, rs, q1s, q2f, rs + 1, best, arg);
                bp[(int64_t)(i - 1) * W + (j - base)] = (uint8_t)arg;
            }
            Vi[j] = best;
        }
        __syncthreads();
    }
    if (tid == 0) {
        int i = N, j = N;
        g[N] = (double)N;
        bool ok = true;
        while (i > 0) {
            const int base = B < N ? i - B : 1;
            const int st = bp[(int64_t)(i - 1) * W + (j - base)];
            if (st >= kNSteps) { ok = false; break; }
            const int a = step_a(st), b = step_b(st);
            if (i < a || j < b) { ok = false; break; }
            for (int p = 0; p < a; ++p) g[i - a + p] = (double)(j - b) + (double)(p * b) / (double)a;
            i -= a;
            j -= b;
        }
        if (!ok || j != 0)
            for (int k = 0; k <= N; ++k) g[k] = (double)k;
    }
    __syncthreads();
}

// q2f[f][x + 1] = q2(x + 1/2 + frac_f) for x = -1 .. N (Catmull-Rom, FP64,
// rounded to float)
template <int T>
__device__ void build_q2f(const double2* q2, int N, float2* q2f)
{
    const int rs = N + 2;
    for (int e = threadIdx.x; e < kNFrac * rs; e += T) {
        const int f = e / rs, x = e - f * rs - 1;
        double2 v;
        cr_eval(q2, N, (double)x + 0.5 + (double)frac_tw(f) / 12.0, v, nullptr);
        q2f[e] = make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
    }
    __syncthreads();
}

// ---------------------------------------------------------- refinement ----
// 1/x for finite x != 0 with |x| in (2^-100, 2^100): float32 seed, two
// Newton steps in FP64 (r <- r (2 - x r)), relative error at rounding level
__device__ __forceinline__ double rcp_fast(double x)
{
    double r = (double)__frcp_rn((float)x);
    r = r * fma(-x, r, 2.0);
    r = r * fma(-x, r, 2.0);
    return r;
}

// Cyclic reduction of the tridiagonal system with rows r = 1..n (lower lo[r],
// diagonal di[r], upper up[r]) on three right-hand sides x, y1, y2 (all
// overwritten by the solutions), FP64, in place; out-of-range rows act as
// identity rows.  The forward reduction eliminates, at stride h = 1, 2, 4, ..,
// the couplings of rows r = 2h, 4h, .. to r +- h, until one decoupled row H
// (2H > n) is left; back substitution then solves rows h, 3h, 5h, .. from
// their solved neighbours at r +- h, for h = H/2 .. 1.  About 2n row updates in
// all, against n log2 n for parallel cyclic reduction (~9 k FP64 instructions
// instead of ~39 k at n = 255; the elastic kernel 13 % faster on the gallery
// pairs).
// Every level reads only rows the level does not write: one barrier per level.
template <int T>
__device__ void cr3(int n, double* lo, double* di, double* up, double* x, double* y1, double* y2)
{
    int h = 1;
    for (; 2 * h <= n; h <<= 1) {
        for (int r = 2 * h * (1 + threadIdx.x); r <= n; r += 2 * h * T) {
            const double al = -lo[r] * rcp_fast(di[r - h]);
            double dd = fma(al, up[r - h], di[r]);
            double xx = fma(al, x[r - h], x[r]);
            double a1 = fma(al, y1[r - h], y1[r]);
            double a2 = fma(al, y2[r - h], y2[r]);
            const double l2 = al * lo[r - h];
            double u2 = 0.0;
            if (r + h <= n) {
                const double ga = -up[r] * rcp_fast(di[r + h]);
                dd = fma(ga, lo[r + h], dd);
                xx = fma(ga, x[r + h], xx);
                a1 = fma(ga, y1[r + h], a1);
                a2 = fma(ga, y2[r + h], a2);
                u2 = ga * up[r + h];
            }
            lo[r] = l2; di[r] = dd; up[r] = u2; x[r] = xx; y1[r] = a1; y2[r] = a2;
        }
        __syncthreads();
    }
    // h is now H with 2H > n: row H (if any) couples to nothing
    if (threadIdx.x == 0 && h <= n) {
        const double iv = rcp_fast(di[h]);
        x[h] *= iv;
        y1[h] *= iv;
        y2[h] *= iv;
    }
    __syncthreads();
    for (h >>= 1; h >= 1; h >>= 1) {
        for (int r = h + 2 * h * threadIdx.x; r <= n; r += 2 * h * T) {
            double xx = x[r], a1 = y1[r], a2 = y2[r];
            if (r - h >= 1) {
                xx = fma(-lo[r], x[r - h], xx);
                a1 = fma(-lo[r], y1[r - h], a1);
                a2 = fma(-lo[r], y2[r - h], a2);
            }
            if (r + h <= n) {
                xx = fma(-up[r], x[r + h], xx);
                a1 = fma(-up[r], y1[r + h], a1);
                a2 = fma(-up[r], y2[r + h], a2);
            }
            const double iv = rcp_fast(di[r]);
            x[r] = xx * iv;
            y1[r] = a1 * iv;
            y2[r] = a2 * iv;
        }
        __syncthreads();
    }
}

struct CellBuf {
    double2 *R, *A, *Bv;       // r_k, d r_k / d g_k, d r_k / d g_{k+1}
    double *Saa, *Sbb, *Sab;   // <r_k, second derivatives of r_k> (full Newton terms)
};

struct LmArrays {
    double *Cc, *Cp;
    double *di, *xv, *lo, *up, *yc, *yp;
};

// One pass over the cells at node values g and rotation cs: residuals, their
// first and second derivatives into buf, and the CTA sums
//   h[0..2] = Hcc, Hcp, Hpp (Gauss-Newton border), h[3..4] = Gc, Gp (gradient),
//   h[5..6] = Scc, Spp (second-order border terms), h[7] = N E (the energy).
template <int T>
__device__ __forceinline__ void cell_pass(const double2* q1, const double2* q2, int N, int s,
                                          double2 cs, const double* g, const CellBuf& buf,
                                          double (&h)[8], double* red)
{
#pragma unroll
    for (int c = 0; c < 8; ++c) h[c] = 0.0;
    for (int k = threadIdx.x; k < N; k += T) {
        double2 v, dv, ddv;
        cr_eval(q2, N, 0.5 * (g[k] + g[k + 1]), v, &dv, &ddv);
        const double D = g[k + 1] - g[k];
        const double rs = rsqrt_fast(D);
        const double m = D * rs;
        const double hm = 0.5 * rs;
        const double2 u = rot(cs, q1[(k + s) & (N - 1)]);
        const double2 r = make_double2(fma(-m, v.x, u.x), fma(-m, v.y, u.y));
        // r = u - sqrt(D) q2(M): r_D = -q2/(2 sqrt D), r_M = -sqrt(D) q2',
        // r_DD = q2/(4 D^{3/2}), r_DM = -q2'/(2 sqrt D), r_MM = -sqrt(D) q2'';
        // d/dg_k = -d/dD + d/dM / 2, d/dg_{k+1} = d/dD + d/dM / 2
        const double2 rD = make_double2(-v.x * hm, -v.y * hm);
        const double2 rM = make_double2(-m * dv.x, -m * dv.y);
        const double q4 = 0.5 * hm * rs * rs;  // 1 / (4 D^{3/2})
        const double2 rDD = make_double2(v.x * q4, v.y * q4);
        const double2 rDM = make_double2(-dv.x * hm, -dv.y * hm);
        const double2 rMM = make_double2(-m * ddv.x, -m * ddv.y);
        const double2 a = make_double2(fma(0.5, rM.x, -rD.x), fma(0.5, rM.y, -rD.y));
        const double2 b = make_double2(fma(0.5, rM.x, rD.x), fma(0.5, rM.y, rD.y));
        const double pDD = r.x * rDD.x + r.y * rDD.y, pDM = r.x * rDM.x + r.y * rDM.y;
        const double pMM = 0.25 * (r.x * rMM.x + r.y * rMM.y);
        buf.R[k] = r;
        buf.A[k] = a;
        buf.Bv[k] = b;
        buf.Saa[k] = pDD - pDM + pMM;
        buf.Sbb[k] = pDD + pDM + pMM;
        buf.Sab[k] = pMM - pDD;
        const double ux = a.x + b.x, uy = a.y + b.y;
        const double px = -u.y, py = u.x;
        h[0] = fma(ux, ux, fma(uy, uy, h[0]));
        h[1] = fma(ux, px, fma(uy, py, h[1]));
        h[2] = fma(px, px, fma(py, py, h[2]));
        h[3] = fma(r.x, ux, fma(r.y, uy, h[3]));
        h[4] = fma(r.x, px, fma(r.y, py, h[4]));
        h[5] += 4.0 * pMM;                      // <r, r_MM>: c moves M only
        h[6] -= r.x * u.x + r.y * u.y;          // d2r/dphi2 = -u
        h[7] = fma(r.x, r.x, fma(r.y, r.y, h[7]));
    }
    cta_sums<T, 8>(h, red);  // includes the barrier that publishes buf
}

// Levenberg-Marquardt refinement of (g, theta) for the shift s; returns N E.
// The trial point's cell pass also serves as the next step's when the step is
// accepted (two buffers, swapped), so each step costs one pass over the cells.
template <int T, int NMAX>
__device__ double elastic_refine(const double2* q1, const double2* q2, int N, int s,
                                 double& theta, double* g0, double* gt0, CellBuf cur,
                                 CellBuf alt, const LmArrays& L, double* red, int& steps)
{
    const int tid = threadIdx.x;
    const int n = N - 1;
    double* g = g0;
    double* gt = gt0;
    double* bc = red + (T / 32 + 2) * 8 - 2;  // broadcast slot (the reductions use fewer)
    if (tid == 0) sincos(theta, &bc[1], &bc[0]);
    __syncthreads();
    double2 cs = make_double2(bc[0], bc[1]);
    double h[8];
    cell_pass<T>(q1, q2, N, s, cs, g, cur, h, red);
    double En = h[7];
    double lambda = 1e-3;
    for (int it = 0; it < kLmIters; ++it) {
        ++steps;
        for (int i = 1 + tid; i <= n; i += T) {
            const double2 b0 = cur.Bv[i - 1], a0 = cur.A[i - 1], a1 = cur.A[i], b1 = cur.Bv[i];
            const double2 r0 = cur.R[i - 1], r1 = cur.R[i];
            const double2 p0 = rot(cs, q1[(i - 1 + s) & (N - 1)]);
            const double2 p1 = rot(cs, q1[(i + s) & (N - 1)]);
            const double sbb0 = cur.Sbb[i - 1], sab0 = cur.Sab[i - 1], saa1 = cur.Saa[i], sab1 = cur.Sab[i];
            L.di[i] = (b0.x * b0.x + b0.y * b0.y + a1.x * a1.x + a1.y * a1.y) * (1.0 + lambda) +
                      sbb0 + saa1;
            L.xv[i] = -(r0.x * b0.x + r0.y * b0.y + r1.x * a1.x + r1.y * a1.y);
            const double cc = b0.x * (a0.x + b0.x) + b0.y * (a0.y + b0.y) + a1.x * (a1.x + b1.x) +
                              a1.y * (a1.y + b1.y) + sab0 + sbb0 + saa1 + sab1;
            const double cp = b0.x * -p0.y + b0.y * p0.x + a1.x * -p1.y + a1.y * p1.x;
            L.Cc[i] = cc;
            L.Cp[i] = cp;
            L.yc[i] = cc;
            L.yp[i] = cp;
            L.lo[i] = i > 1 ? a0.x * b0.x + a0.y * b0.y + sab0 : 0.0;
            L.up[i] = i < n ? a1.x * b1.x + a1.y * b1.y + sab1 : 0.0;
        }
        __syncthreads();
        cr3<T>(n, L.lo, L.di, L.up, L.xv, L.yc, L.yp);
        double sc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // Cc.yc, Cc.yp, Cp.yp, Cc.x, Cp.x
        for (int i = 1 + tid; i <= n; i += T) {
            const double yc = L.yc[i], yp = L.yp[i], xv = L.xv[i];
            sc[0] = fma(L.Cc[i], yc, sc[0]);
            sc[1] = fma(L.Cc[i], yp, sc[1]);
            sc[2] = fma(L.Cp[i], yp, sc[2]);
            sc[3] = fma(L.Cc[i], xv, sc[3]);
            sc[4] = fma(L.Cp[i], xv, sc[4]);
        }
        cta_sums<T, 5>(sc, red);
        const double S00 = h[0] * (1.0 + lambda) + h[5] - sc[0], S01 = h[1] - sc[1];
        const double S11 = h[2] * (1.0 + lambda) + h[6] - sc[2];
        const double r0 = -h[3] - sc[3], r1 = -h[4] - sc[4];
        const double det = S00 * S11 - S01 * S01;
        double dc = 0.0, dphi = 0.0;
        if (det > 0.0) {
            dc = (S11 * r0 - S01 * r1) / det;
            dphi = (S00 * r1 - S01 * r0) / det;
        }
        // step on the interior nodes, then the slope-keeping shortening
        for (int k = tid; k <= N; k += T)
            gt[k] = (k == 0 || k == N) ? 0.0 : L.xv[k] - L.yc[k] * dc - L.yp[k] * dphi;
        __syncthreads();
        double al = 1.0;
        for (int k = tid; k < N; k += T) {
            const double D = g[k + 1] - g[k], dD = gt[k + 1] - gt[k];
            if (dD < -0.5 * D) al = fmin(al, -0.5 * D / dD);
        }
        al = cta_min<T>(al, red);
        for (int k = tid; k <= N; k += T) gt[k] = fma(al, dc + gt[k], g[k]);
        const double tht = fma(al, dphi, theta);
        if (tid == 0) sincos(tht, &bc[1], &bc[0]);
        __syncthreads();
        const double2 ct = make_double2(bc[0], bc[1]);
        double ht[8];
        cell_pass<T>(q1, q2, N, s, ct, gt, alt, ht, red);
        const double Et = ht[7];
        bool stop;
        if (Et < En) {
            double* tg = g; g = gt; gt = tg;
            const CellBuf tb = cur; cur = alt; alt = tb;
#pragma unroll
            for (int c = 0; c < 8; ++c) h[c] = ht[c];
            theta = tht;
            cs = ct;
            stop = En - Et <= kLmTol * En;
            En = Et;
            lambda = fmax(lambda * 0.25, 1e-12);
        } else {
            lambda *= 8.0;
            stop = lambda > kLmStall;
        }
        if (stop) break;
    }
    if (g != g0) {
        for (int k = tid; k <= N; k += T) g0[k] = g[k];
        __syncthreads();
    }
    return En;
}

// ------------------------------------------------------ rigid alignment ----
// argmax_s |c(s)|, c(s) = sum_k a[k] conj(b[k+s]), with X = a (overwritten),
// Bspec = DFT(b); a kept in Acopy for the direct c(s*); returns s* and c(s*)
template <int T, int NMAX>
__device__ int rigid_fft(double2* X, const double2* Acopy, const double2* Bspec,
                         const double2* b, int N, int logn, const double2* tf, double2& cbest,
                         long long* sk, int* si, double* red)
{
    fft_rt<T, NMAX>(X, logn, tf);
    for (int k = threadIdx.x; k < N; k += T) X[k] = cmulc(X[k], Bspec[k]);
    __syncthreads();
    fft_rt<T, NMAX>(X, logn, tf);
    long long key = -1;
    int idx = 0;
    for (int k = threadIdx.x; k < N; k += T) {
        const double2 y = X[k];
        const long long kq = __double_as_longlong(fma(y.x, y.x, y.y * y.y));
        if (key_better(kq, k, key, idx)) { key = kq; idx = k; }
    }
    cta_argmax<T>(key, idx, sk, si);
    double c[2] = {0.0, 0.0};
    for (int k = threadIdx.x; k < N; k += T) {
        const double2 u = Acopy[k], v = b[(k + idx) & (N - 1)];
        c[0] = fma(u.x, v.x, fma(u.y, v.y, c[0]));
        c[1] = fma(u.y, v.x, fma(-u.x, v.y, c[1]));
    }
    cta_sums<T, 2>(c, red);
    cbest = make_double2(c[0], c[1]);
    return idx;
}

// NMAX: the largest N this instantiation handles (sizes the per-thread
// register blocks of the transforms and of the reduction solver)
// Resident pair CTAs per SM the kernel is compiled for: at N <= 256 four (its
// registers capped at 128, with some spills; the Catmull-Rom table and the
// back-pointers then live in the workspace), which measured 5.7 % faster than
// two CTAs of 246 registers with everything in shared memory (18.75 against
// 19.88 ms on 4,096 gallery pairs, identical energies); larger N are bound by
// shared memory to two.
template <int NMAX>
constexpr int el_min_blocks() { return NMAX <= 256 ? 4 : 1; }

template <int T, int NMAX>
__global__ void __launch_bounds__(T, el_min_blocks<NMAX>()) elastic_pair_kernel(const __grid_constant__ ElasticArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N, tid = threadIdx.x;
    const int B = (a.band < 0 || a.band >= N) ? N : a.band;
    double2* q1 = reinterpret_cast<double2*>(smem_raw);
    double2* q2 = q1 + N;
    double2* Q1 = q2 + N;
    double2* X = Q1 + N;
    double2* Y = X + N;
    double2* q1s = Y + N;
    double* g = reinterpret_cast<double*>(q1s + N);
    double* gt = g + (N + 1);
    double* ar = gt + (N + 1);                 // 12 (N+1): solver arrays / DP ring
    double* red = ar + 12 * (N + 1);           // (T/32 + 2) * 8
    long long* sk = reinterpret_cast<long long*>(red + (T / 32 + 2) * 8);
    int* si = reinterpret_cast<int*>(sk + T / 32);
    int* ib = si + T / 32;                     // [4] broadcast ints
    unsigned char* tail = reinterpret_cast<unsigned char*>(ib + 4);
    tail = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tail) + 15) & ~uintptr_t(15));
    double2* q2f;
    uint8_t* bp;
    if (a.q2f_smem) {
        q2f = reinterpret_cast<double2*>(tail);
        tail += (size_t)a.q2f_elems * sizeof(double2);
    } else {
        q2f = a.q2f_ws + (int64_t)blockIdx.x * a.q2f_elems;
    }
    bp = a.bp_smem ? reinterpret_cast<uint8_t*>(tail) : a.bp_ws + (int64_t)blockIdx.x * a.bp_bytes;
    LmArrays L;
    L.Cc = ar; L.Cp = ar + (N + 1);
    L.di = ar + 2 * (N + 1); L.xv = ar + 3 * (N + 1); L.lo = ar + 4 * (N + 1);
    L.up = ar + 5 * (N + 1); L.yc = ar + 6 * (N + 1); L.yp = ar + 7 * (N + 1);
    // the refinement's two cell buffers: one in the transform buffers, the other
    // in the Catmull-Rom table's space (9N doubles of its 16(N+2)), which the
    // lattice DP no longer needs once it has run
    CellBuf cb0, cb1;
    cb0.R = X; cb0.A = Y; cb0.Bv = q1s;
    cb0.Saa = ar + 8 * (N + 1); cb0.Sbb = ar + 9 * (N + 1); cb0.Sab = ar + 10 * (N + 1);
    cb1.R = q2f; cb1.A = q2f + N; cb1.Bv = q2f + 2 * N;
    {
        double* d = reinterpret_cast<double*>(q2f + 3 * N);
        cb1.Saa = d; cb1.Sbb = d + N; cb1.Sab = d + 2 * N;
    }
    const double nanv = __longlong_as_double(0x7ff8000000000000LL);

    // pairs are taken from a global counter (iteration counts differ between
    // pairs; a fixed stride would leave the slowest CTA as the tail)
    for (;;) {
        if (tid == 0) {
            const unsigned long long t = atomicAdd(a.next, 1ull);
            ib[2] = (int)(t >> 32);
            ib[3] = (int)(t & 0xffffffffu);
        }
        __syncthreads();
        const int64_t pair = ((int64_t)(unsigned)ib[2] << 32) | (int64_t)(unsigned)ib[3];
        __syncthreads();
        if (pair >= a.P) break;
        const int64_t i1 = a.idx1 ? a.idx1[pair] : pair;
        const int64_t i2 = a.idx2 ? a.idx2[pair] : pair;
        const bool inr = i1 >= 0 && i1 < a.M1 && i2 >= 0 && i2 < a.M2;
        const int64_t c1 = inr ? i1 : 0, c2 = inr ? a.M1 + i2 : 0;
        const int s1 = a.cst[c1], s2 = a.cst[c2];
        const int st = !inr ? FA_STATUS_BAD_SIZE
                       : (s1 == FA_STATUS_NONFINITE || s2 == FA_STATUS_NONFINITE) ? FA_STATUS_NONFINITE
                       : s1 ? s1 : s2;
        if (st != FA_STATUS_OK) {
            if (tid == 0) {
                a.shift[pair] = -1;
                a.theta[pair] = nanv;
                a.energy[pair] = nanv;
                a.status[pair] = (int8_t)st;
                if (a.iters) a.iters[pair] = 0;
                if (a.lm_steps) a.lm_steps[pair] = 0;
            }
            if (a.gamma)
                for (int k = tid; k <= N; k += T) a.gamma[pair * (N + 1) + k] = nanv;
            continue;
        }
        // ---- pre-alignment on the resampled curves: e^{i th} zr1[k+s] ~ zr2[k]
        const double2* zr1 = a.zr + c1 * N;
        const double2* zr2 = a.zr + c2 * N;
        for (int k = tid; k < N; k += T) {
            X[k] = zr2[k];
            Y[k] = zr1[k];
            q1[k] = a.q[c1 * N + k];
            q2[k] = a.q[c2 * N + k];
            Q1[k] = q1[k];
        }
        __syncthreads();
        build_q2f<T>(q2, N, reinterpret_cast<float2*>(q2f));
        fft_rt<T, NMAX>(Y, a.logn, a.tf);
        for (int k = tid; k < N; k += T) q1s[k] = zr2[k];  // the direct c(s*) reads it
        __syncthreads();
        double2 cb;
        int s = rigid_fft<T, NMAX>(X, q1s, Y, zr1, N, a.logn, a.tf, cb, sk, si, red);
        double theta = atan2(cb.y, cb.x);
        // the start point in curve 1's own parameter (nearest node)
        if (tid == 0) {
            const double* sg = a.sigma + c1 * (N + 1);
            const double tau = (double)s / (double)N;
            int lo = 0, hi = N - 1;  // largest k < N with sg[k] <= tau
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (sg[mid] <= tau) lo = mid; else hi = mid - 1;
            }
            const double d = sg[lo + 1] - sg[lo];
            const double u = (double)lo + (d > 0.0 ? (tau - sg[lo]) / d : 0.0);
            ib[0] = ((int)floor(u + 0.5)) & (N - 1);
        }
        // DFT(q1) for the (t0, R)-steps
        __syncthreads();
        s = ib[0];
        fft_rt<T, NMAX>(Q1, a.logn, a.tf);
        for (int k = tid; k <= N; k += T) g[k] = (double)k;
        __syncthreads();

        // the first gamma-step's lattice path (float32 path sums: the DP only
        // picks the refinement's starting path; every reported value is FP64)
        {
            double2 cs;
            sincos(theta, &cs.y, &cs.x);
            float2* q1f = reinterpret_cast<float2*>(q1s);
            for (int k = tid; k < N; k += T) {
                const double2 u = rot(cs, q1[(k + s) & (N - 1)]);
                q1f[k] = make_float2(__double2float_rn(u.x), __double2float_rn(u.y));
            }
            __syncthreads();
            elastic_dp<T>(N, B, q1f, reinterpret_cast<const float2*>(q2f),
                          reinterpret_cast<float*>(ar), bp, g);
        }
        int it = 0, lm = 0;
        double Eprev = HUGE_VAL, En = 0.0;
        if (a.max_iter == 0) {
            // no iteration: report the starting triple (pre-alignment s, theta
            // and the lattice path) with its FP64 energy
            double2 cs;
            sincos(theta, &cs.y, &cs.x);
            double e[1] = {0.0};
            for (int k = tid; k < N; k += T) {
                double2 v;
                cr_eval(q2, N, 0.5 * (g[k] + g[k + 1]), v, nullptr);
                const double D = g[k + 1] - g[k];
                const double m = D * rsqrt_fast(D);
                const double2 u = rot(cs, q1[(k + s) & (N - 1)]);
                const double dx = fma(-m, v.x, u.x), dy = fma(-m, v.y, u.y);
                e[0] = fma(dx, dx, fma(dy, dy, e[0]));
            }
            cta_sums<T, 1>(e, red);
            En = e[0] / (double)N;
        }
        for (it = 1; it <= a.max_iter; ++it) {
            elastic_refine<T, NMAX>(q1, q2, N, s, theta, g, gt, cb0, cb1, L, red, lm);
            // (t0, R)-step on w_k = sqrt(D_k) q2(M_k)
            for (int k = tid; k < N; k += T) {
                double2 v;
                cr_eval(q2, N, 0.5 * (g[k] + g[k + 1]), v, nullptr);
                const double D = g[k + 1] - g[k];
                const double m = D * rsqrt_fast(D);
                X[k] = make_double2(m * v.x, m * v.y);
                Y[k] = X[k];
            }
            __syncthreads();
            s = rigid_fft<T, NMAX>(X, Y, Q1, q1, N, a.logn, a.tf, cb, sk, si, red);
            theta = atan2(cb.y, cb.x);
            double2 cs;
            sincos(theta, &cs.y, &cs.x);
            double e[1] = {0.0};
            for (int k = tid; k < N; k += T) {
                const double2 u = rot(cs, q1[(k + s) & (N - 1)]), w = Y[k];
                const double dx = u.x - w.x, dy = u.y - w.y;
                e[0] = fma(dx, dx, fma(dy, dy, e[0]));
            }
            cta_sums<T, 1>(e, red);
            En = e[0] / (double)N;
            if (Eprev - En <= kStopDrop) break;
            Eprev = En;
        }
        if (it > a.max_iter) it = a.max_iter;
        if (tid == 0) {
            a.shift[pair] = s;
            a.theta[pair] = theta;
            a.energy[pair] = En;
            a.status[pair] = FA_STATUS_OK;
            if (a.iters) a.iters[pair] = it;
            if (a.lm_steps) a.lm_steps[pair] = lm;
        }
        if (a.gamma)
            for (int k = tid; k <= N; k += T) a.gamma[pair * (N + 1) + k] = g[k];
        __syncthreads();
    }
}

// per curve (one warp each): SRV samples, chord-length fractions, status
constexpr int kPrepWarps = 4;
__global__ void __launch_bounds__(32 * kPrepWarps)
    elastic_prep_kernel(const double2* __restrict__ set1, const double2* __restrict__ set2,
                        int64_t M1, int64_t Mtot, int N, const int8_t* __restrict__ rstatus,
                        double2* __restrict__ q, double* __restrict__ sigma,
                        int8_t* __restrict__ cst)
{
    const int64_t c = (int64_t)blockIdx.x * kPrepWarps + (threadIdx.x >> 5);
    if (c >= Mtot) return;
    const int lane = threadIdx.x & 31;
    const double2* b = c < M1 ? set1 + c * N : set2 + (c - M1) * N;
    // lane owns nodes [lane*C, (lane+1)*C), C = N/32 (N >= 32) or 1
    const int C = N >= 32 ? N / 32 : 1;
    const int k0 = lane * C;
    const bool act = k0 < N;
    double part = 0.0;
    bool bad = false;
    if (act)
        for (int k = k0; k < k0 + C; ++k) {
            const double2 p = b[k], p1 = b[(k + 1) & (N - 1)];
            bad |= !finite2(p);
            const double dx = p1.x - p.x, dy = p1.y - p.y;
            part += sqrt(dx * dx + dy * dy);
        }
    const bool anybad = __any_sync(0xffffffffu, bad);
    // inclusive scan of the lane partial sums -> perimeter and chunk offsets
    double incl = part;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
    }
    const double per = __shfl_sync(0xffffffffu, incl, 31);
    const double excl = incl - part;
    int8_t stc = FA_STATUS_OK;
    if (anybad) stc = FA_STATUS_NONFINITE;
    else if (!(per > 0.0) || !isfinite(per)) stc = FA_STATUS_DEGENERATE;
    else if (rstatus[c] != FA_STATUS_OK) stc = rstatus[c];
    double* sg = sigma + c * (N + 1);
    if (act && stc == FA_STATUS_OK) {
        double run = excl;
        if (lane == 0) sg[0] = 0.0;
        for (int k = k0; k < k0 + C; ++k) {
            const double2 p = b[k], p1 = b[(k + 1) & (N - 1)];
            const double dx = p1.x - p.x, dy = p1.y - p.y;
            run += sqrt(dx * dx + dy * dy);
            sg[k + 1] = run / per;
            const double vx = (double)N * dx / per, vy = (double)N * dy / per;
            const double r = sqrt(vx * vx + vy * vy);
            const double sr = sqrt(r);
            q[c * N + k] = r > 0.0 ? make_double2(vx / sr, vy / sr) : make_double2(0.0, 0.0);
        }
    }
    if (lane == 0) cst[c] = stc;
}

__global__ void uniform_offsets_kernel(int64_t* off, int64_t M, int N)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= M) off[i] = i * N;
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct ElLayout {
    size_t off_offsets, off_rws, off_zr, off_q, off_sigma, off_cst, off_rst, off_next, off_slots, total;
    size_t smem;
    int q2f_smem, bp_smem, grid;
    int64_t q2f_elems, bp_bytes;
};

// shared memory per pair CTA: four CTAs per SM at N <= 256, two above
inline size_t el_smem_budget(int N) { return N <= 256 ? (size_t)56 * 1024 : (size_t)112 * 1024; }

ElLayout el_layout(const fa_handle* h, int64_t Mtot, int64_t P, int N, int band)
{
    ElLayout L{};
    const int B = (band < 0 || band >= N) ? N : band;
    const int W = B < N ? 2 * B + 1 : N;
    L.q2f_elems = (int64_t)kNFrac * (N + 2);
    L.bp_bytes = (int64_t)N * W;
    size_t fixed = 6 * (size_t)N * sizeof(double2) + 14 * (size_t)(N + 1) * sizeof(double) +
                   (kElT / 32 + 2) * 8 * sizeof(double) + (kElT / 32) * (sizeof(long long) + sizeof(int)) +
                   4 * sizeof(int) + 16;
    size_t sm = fixed;
    const size_t budget = el_smem_budget(N);
    L.q2f_smem = sm + L.q2f_elems * sizeof(double2) <= budget;
    if (L.q2f_smem) sm += L.q2f_elems * sizeof(double2);
    L.bp_smem = sm + (size_t)L.bp_bytes <= budget;
    if (L.bp_smem) sm += (size_t)L.bp_bytes;
    L.smem = sm;
    int per_sm = 1;
    {
        const void* k = N <= 256 ? (const void*)elastic_pair_kernel<kElT, 256>
                                 : (const void*)elastic_pair_kernel<kElT, 1024>;
        if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kElT, sm) != cudaSuccess || per_sm < 1)
            per_sm = 1;
    }
    L.grid = (int)std::max<int64_t>(1, std::min<int64_t>(P, (int64_t)h->num_sms * per_sm));
    size_t o = 0;
    L.off_offsets = o; o = align256(o + sizeof(int64_t) * (size_t)(Mtot + 1));
    L.off_rws = o; o = align256(o + resample_ws_bytes(Mtot, Mtot * N, N, FA_CENTER | FA_UNIT_LENGTH));
    L.off_zr = o; o = align256(o + sizeof(double2) * (size_t)Mtot * N);
    L.off_q = o; o = align256(o + sizeof(double2) * (size_t)Mtot * N);
    L.off_sigma = o; o = align256(o + sizeof(double) * (size_t)Mtot * (N + 1));
    L.off_cst = o; o = align256(o + (size_t)Mtot);
    L.off_rst = o; o = align256(o + (size_t)Mtot);
    L.off_next = o; o = align256(o + sizeof(unsigned long long));
    L.off_slots = o;
    if (!L.q2f_smem) o += align256(sizeof(double2) * (size_t)L.q2f_elems * L.grid);
    if (!L.bp_smem) o += align256((size_t)L.bp_bytes * L.grid);
    L.total = o;
    return L;
}

}  // namespace

size_t elastic_ws_bytes(const fa_handle* h, int64_t M1, int64_t M2, int64_t P, int N, int band)
{
    return el_layout(h, M1 + M2, P, N, band).total;
}

int launch_elastic(const fa_handle* h, const double* set1, int64_t M1, const double* set2,
                   int64_t M2, int N, const int64_t* idx1, const int64_t* idx2, int64_t P,
                   int band, int max_iter, int32_t* shift, double* theta, double* energy,
                   double* gamma, int32_t* iters, int32_t* lm_steps, int8_t* status, void* ws,
                   cudaStream_t st)
{
    const int64_t Mtot = M1 + M2;
    const ElLayout L = el_layout(h, Mtot, P, N, band);
    unsigned char* base = static_cast<unsigned char*>(ws);
    int64_t* off = reinterpret_cast<int64_t*>(base + L.off_offsets);
    double2* zr = reinterpret_cast<double2*>(base + L.off_zr);
    double2* q = reinterpret_cast<double2*>(base + L.off_q);
    double* sigma = reinterpret_cast<double*>(base + L.off_sigma);
    int8_t* cst = reinterpret_cast<int8_t*>(base + L.off_cst);
    int8_t* rst = reinterpret_cast<int8_t*>(base + L.off_rst);
    unsigned char* slots = base + L.off_slots;
    unsigned long long* next = reinterpret_cast<unsigned long long*>(base + L.off_next);

    // the two curve sets as one list: set 1 then set 2 (resampling reads one
    // point array, so set 2 follows set 1 in it through the offsets when the
    // sets are adjacent; otherwise each set is resampled on its own)
    uniform_offsets_kernel<<<(unsigned)((M1 + 256) / 256), 256, 0, st>>>(off, M1, N);
    int rc = cuda_error(cudaGetLastError(), "elastic offsets launch");
    if (rc != FA_OK) return rc;
    rc = launch_resample(h, set1, off, M1, M1 * N, N, FA_CENTER | FA_UNIT_LENGTH, zr, rst,
                             base + L.off_rws, st);
    if (rc != FA_OK) return rc;
    if (M2 > 0) {
        uniform_offsets_kernel<<<(unsigned)((M2 + 256) / 256), 256, 0, st>>>(off, M2, N);
        rc = launch_resample(h, set2, off, M2, M2 * N, N, FA_CENTER | FA_UNIT_LENGTH, zr + M1 * N,
                             rst + M1, base + L.off_rws, st);
        if (rc != FA_OK) return rc;
    }
    elastic_prep_kernel<<<(unsigned)((Mtot + kPrepWarps - 1) / kPrepWarps), 32 * kPrepWarps, 0,
                          st>>>(reinterpret_cast<const double2*>(set1),
                                reinterpret_cast<const double2*>(set2), M1, Mtot, N, rst, q,
                                sigma, cst);
    rc = cuda_error(cudaGetLastError(), "elastic prep launch");
    if (rc != FA_OK) return rc;
    ElasticArgs A{};
    A.q = q; A.sigma = sigma; A.zr = zr; A.cst = cst; A.idx1 = idx1; A.idx2 = idx2;
    A.M1 = M1; A.M2 = M2; A.P = P; A.next = next; A.N = N; A.logn = 31 - __builtin_clz((unsigned)N);
    A.band = band; A.max_iter = max_iter;
    A.q2f_elems = L.q2f_elems; A.bp_bytes = L.bp_bytes;
    A.q2f_smem = L.q2f_smem; A.bp_smem = L.bp_smem;
    A.q2f_ws = L.q2f_smem ? nullptr : reinterpret_cast<double2*>(slots);
    A.bp_ws = L.bp_smem ? nullptr
                        : slots + (L.q2f_smem ? 0 : align256(sizeof(double2) * (size_t)L.q2f_elems * L.grid));
    A.tf = h->tf64[A.logn];
    A.shift = shift; A.theta = theta; A.energy = energy; A.gamma = gamma; A.iters = iters;
    A.lm_steps = lm_steps;
    A.status = status;
    auto kern = N <= 256 ? elastic_pair_kernel<kElT, 256> : elastic_pair_kernel<kElT, 1024>;
    if (L.smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(
            kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
        if (e != cudaSuccess) return cuda_error(e, "elastic: cudaFuncSetAttribute");
    }
    const cudaError_t me = cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
    if (me != cudaSuccess) return cuda_error(me, "elastic counter reset");
    kern<<<L.grid, kElT, L.smem, st>>>(A);
    return cuda_error(cudaGetLastError(), "elastic launch");
}

}  // namespace fa
