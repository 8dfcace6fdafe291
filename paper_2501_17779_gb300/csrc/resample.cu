// resample.cu -- arc-length resampling (Sec. 2: Eq. arc-length-param, then a
// cubic spline through (s^l, beta^l) evaluated at uniform parameters), FP64.
//
// One warp per curve.  Lane j owns a contiguous chunk of nodes
// [s_j, s_{j+1}) (P chunks, P = 32 for n >= 64).  Steps:
//   A. chord lengths d_l = |p_{l+1} - p_l| (node-parallel, with the check for
//      non-finite nodes), their sum per chunk; a warp scan gives each chunk's
//      starting arc length and the perimeter L.
//   B. forward sweep over each chunk's interior nodes (all but its last):
//      cumulative arc lengths S_l = L u_l, the periodic-spline equations
//          h_{l-1} M_{l-1} + 2(h_{l-1}+h_l) M_l + h_l M_{l+1}
//              = 6[(p_{l+1}-p_l)/h_l - (p_l-p_{l-1})/h_{l-1}],   h_l = d_l / L,
//      multiplied through by L and solved for M' = M / (6 L^2), so that they read
//          d_{l-1} M'_{l-1} + 2(d_{l-1}+d_l) M'_l + d_l M'_{l+1} = tau_l - tau_{l-1}
//      with the unit chord directions tau_l = (p_{l+1}-p_l)/d_l (fewer FP64
//      instructions; the evaluation's h_l^2 M / 6 is d_l^2 M'), and the Thomas
//      elimination of the interior with the chunk's two
//      neighbouring interface nodes (the last node of the previous chunk and
//      of this chunk) kept as unknowns: M_i = y_i - I_{j-1} g_i - I_j k_i.
//   C. the same sweep accumulates the first interior node's back-substitution
//      coefficients (y, g, k); eliminating the interiors leaves a cyclic
//      tridiagonal system in the P interface values, solved by parallel
//      cyclic reduction with warp shuffles.
//   D. a backward sweep writes M for every node.
//   E. the spline is evaluated at t_k = k/N_out, then the outputs are centred
//      at their mean and divided by the closed-polygon perimeter of the
//      outputs (both summed in the same loop).  For N_out <= 1024 the
//      interval of every output comes from a per-warp table in shared memory:
//      B counts each knot S_l at the first output whose target reaches it,
//      a prefix sum turns the counts into intervals, and 32 consecutive
//      outputs are evaluated at a time (coalesced stores, independent loads).
//      Larger N_out: each lane a contiguous block of outputs, its intervals
//      by bisection and stepping over the knots.
// Per-node intermediates (arc lengths, chord lengths, the forward sweep's
// records, M: 48 B per node) live in a caller- or handle-provided workspace
// (global memory, L1/L2 resident while a warp works on its curve).  The chord
// vectors and reciprocal chord lengths are recomputed where B and E need them
// (two FP64 subtractions from the input, one Newton reciprocal) instead of
// being stored: the workspace's latency, not the FP64 pipe, bounds the kernel.
#include <algorithm>

#include "df.cuh"
#include "fa_internal.cuh"

namespace fa {
namespace {

constexpr int kWarps = 4;  // curves per CTA

// Resident CTAs per SM requested from the compiler (it also sizes the grid): 4
// caps the kernel at 128 registers (no spills, 16 warps per SM).  Measured
// against it: 2 CTAs +17 %, 3 +3.4 % (less workspace in flight does not make
// up for fewer warps), 5 +0.9 % and 6 +4.5 % (96 / 80 registers, spills).
#ifndef FA_RESAMPLE_MIN_BLOCKS
#define FA_RESAMPLE_MIN_BLOCKS 4
#endif

struct Ws {
    double* U;     // cumulative arc length S_l = L u_l [n_pts]
    double* D;     // chord lengths d_l                 [n_pts]
    double2* F0;   // forward sweep (c'_l, g'_l)        [n_pts]
    double2* F1;   // forward sweep y'_l (x, y)         [n_pts]
    double2* M;    // spline second derivatives M_l     [n_pts] (stored over F1)
    double2* Z;    // raw outputs before normalisation  [C*N_out] (FP32 output only)
};

// ---- reciprocal square root, reciprocal and square root by one Newton step ---
// The FP32 seed is built from the double's bits with integer instructions, the
// FP32 hardware approximation (rsqrtf / __frcp_rn / __fsqrt_rn) refines it to
// ~2^-22, and one Newton-Raphson step (Newton's method on f(y) = 1/y^2 - q,
// f(r) = 1/r - x, f(s) = s^2 - q) squares the relative error to below 1e-13.
// FP64 is the scarce unit on this part (1/64 of the FP32 rate), so the steps
// keep their FP64 instructions to one or two, doing the rest with float-float
// and integer arithmetic (see each function).  The chord lengths, their
// reciprocals, the pivots and the perimeter need no more: their errors move
// the resampled nodes by < 2e-13 of the curve length, inside the 1e-12 parity
// bound.  Valid for positive normal inputs of moderate exponent, which
// chords, perimeters and pivots of curves of reasonable size are; other
// inputs take the CUDA call.
__device__ __forceinline__ bool f32_range(double x)
{
    const int e = (int)((__double_as_longlong(x) >> 52) & 0x7ff) - 1023;
    return e > -120 && e < 120;
}
__device__ __forceinline__ float seed_f32(double x)  // x truncated to a float (x > 0)
{
    const long long b = __double_as_longlong(x);
    const unsigned e = (unsigned)(((b >> 52) & 0x7ff) - 1023 + 127);
    return __uint_as_float((e << 23) | (unsigned)((b >> 29) & 0x7fffff));
}
__device__ __forceinline__ double widen_f32(float f)  // exact float -> double by bits (f > 0)
{
    const unsigned u = __float_as_uint(f);
    const unsigned long long e = ((u >> 23) & 0xff) - 127 + 1023;
    return __longlong_as_double((long long)((e << 52) | ((unsigned long long)(u & 0x7fffff) << 29)));
}
// float -> double by bits for any finite sign (zero and subnormal floats give 0)
__device__ __forceinline__ double widen_any(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned ef = (u >> 23) & 0xff;
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned long long mag =
        ef == 0 ? 0ull
                : ((unsigned long long)(ef - 127 + 1023) << 52) | ((unsigned long long)(u & 0x7fffff) << 29);
    return __longlong_as_double((long long)(sign | mag));
}
// exponent range in which a double splits into two normal floats (see split_pos)
__device__ __forceinline__ bool split_range(double x)
{
    const int e = (int)((__double_as_longlong(x) >> 52) & 0x7ff) - 1023;
    return e > -70 && e < 120;
}
// x = xh + xl to 2^-47 relative: xh the top 24 significand bits (truncated),
// xl the next 24 bits (rounded), both from the bits with integer instructions
// (x > 0 inside split_range, where both parts are normal floats).
__device__ __forceinline__ void split_pos(double x, float& xh, float& xl)
{
    xh = seed_f32(x);
    const long long b = __double_as_longlong(x);
    const int fe = (int)((b >> 52) & 0x7ff) - 1023 + 127;  // float exponent field of x
    const int m = (int)(b & 0x1fffffff);                    // the 29 bits below xh
    xl = fe > 52 ? __fmul_rn(__int2float_rn(m), __uint_as_float((unsigned)(fe - 52) << 23)) : 0.0f;
}
// The residual 1 - x y^2 (y a float near x^{-1/2}) or 1 - x y (y near 1/x),
// evaluated in float-float arithmetic (Dekker's exact product by FMA, then
// float sums whose operands nearly cancel): the residual is about 2^-22 and
// comes out with an absolute error near 2^-47, i.e. to about 2^-25 of itself,
// which is all one Newton-Raphson step needs.
__device__ __forceinline__ float resid_rsqrt(float xh, float xl, float y)
{
    const float yy = __fmul_rn(y, y), yye = __fmaf_rn(y, y, -yy);  // y^2 = yy + yye exactly
    const float p = __fmul_rn(xh, yy), pe = __fmaf_rn(xh, yy, -p);  // xh yy = p + pe exactly
    const float t = __fmaf_rn(xh, yye, __fmaf_rn(xl, yy, pe));      // the small products
    return __fsub_rn(__fsub_rn(1.0f, p), t);                        // 1 - p is exact (p ~ 1)
}
__device__ __forceinline__ float resid_rcp(float xh, float xl, float y)
{
    const float p = __fmul_rn(xh, y), pe = __fmaf_rn(xh, y, -p);
    return __fsub_rn(__fsub_rn(1.0f, p), __fmaf_rn(xl, y, pe));
}
// 1/sqrt(q) and 1/x by one Newton-Raphson step from an FP32 seed, the step's
// residual in float-float and its single FP64 instruction the final add:
// y0 + (y0/2) e with e = 1 - q y0^2 (rsqrt), r0 + r0 e with e = 1 - x r0 (rcp).
// The seed's relative error e0 <= 2^-22 leaves 1.5 e0^2 < 9e-14 (rsqrt) and
// e0^2 < 6e-14 (rcp) after the step, plus about 2^-46 from the residual.
__device__ __forceinline__ double rsqrt_nr(double q)
{
    if (!split_range(q)) return rsqrt(q);
    float qh, ql;
    split_pos(q, qh, ql);
    const float y0f = rsqrtf(qh);
    const float e = resid_rsqrt(qh, ql, y0f);
    return widen_f32(y0f) + widen_any(__fmul_rn(__fmul_rn(0.5f, y0f), e));
}
__device__ __forceinline__ double rcp_nr(double x)
{
    if (__double_as_longlong(x) <= 0 || !split_range(x)) return __drcp_rn(x);
    float xh, xl;
    split_pos(x, xh, xl);
    const float r0 = __frcp_rn(xh);
    const float e = resid_rcp(xh, xl, r0);
    return widen_f32(r0) + widen_any(__fmul_rn(r0, e));
}
// sqrt(q) from the correctly rounded FP32 square root of q's leading float
// (relative error <= 2^-23) and one Newton-Raphson step s0 + (q - s0^2)/(2 s0)
// whose divisor is taken in FP32: relative error below 2^-45.  Two FP64
// instructions.  Valid for q > 0 inside f32_range.
__device__ __forceinline__ double sqrt_nr(double q)
{
    if (!f32_range(q)) return sqrt(q);
    const float s0f = __fsqrt_rn(seed_f32(q));
    const double s0 = widen_f32(s0f);
    return fma(fma(-s0, s0, q), widen_f32(__fdiv_rn(0.5f, s0f)), s0);
}
// |(dx, dy)| in float-float: the FP64 components split exactly enough (2^-47),
// the squared length by exact products, and the square root from the FP32
// root of the leading part with one Newton step whose residual q - s0^2 is
// formed exactly (s0^2 = p + pe by FMA, q.h - p exact by Sterbenz) -- about
// 2^-46 relative.  FP32 and integer instructions only.
__device__ __forceinline__ dfl df_chord(double2 d)
{
    const cdf c = split_c(d);
    const dfl q = df_dot2<+1>(c.re, c.re, c.im, c.im);
    if (!(q.h > 0.0f)) return {0.0f, 0.0f};
    const float s0 = __fsqrt_rn(q.h);
    const float pp = __fmul_rn(s0, s0), pe = __fmaf_rn(s0, s0, -pp);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(q.h, pp), pe), q.l);
    return fast_two_sum(s0, __fmul_rn(r, __fdiv_rn(0.5f, s0)));
}
// 2x for x >= 0 with integer instructions only (exact; subnormals shift,
// normals step the exponent, the largest binade goes to +Inf, Inf/NaN stay)
__device__ __forceinline__ double twice_pos(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned e = (unsigned)(b >> 52);
    const unsigned long long r = e == 0 ? b << 1
                                 : e < 0x7feu ? b + (1ull << 52)
                                 : e == 0x7feu ? 0x7ff0000000000000ull : b;
    return __longlong_as_double((long long)r);
}

// ---- the spline solve in float-float, in units scaled by 2^k ~ 1/L --------
// v 2^k as a double-float, from the bits (split_d with the exponent moved by
// k): exact to 2^-47 relative; magnitudes that land below 2^-126 give 0 (only
// a chord vector's near-zero component can), and the caller keeps every
// scaled magnitude below 2^120.
__device__ __forceinline__ dfl split_scaled(double v, int k)
{
    const long long b = __double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff);
    const int fe = e - 1023 + 127 + k;  // float exponent field of v 2^k
    if (e == 0 || fe <= 0) return {0.f, 0.f};
    const unsigned sign = (unsigned)((unsigned long long)b >> 32) & 0x80000000u;
    const float hi = __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)((b >> 29) & 0x7fffff));
    if (fe < 53) return {hi, 0.f};
    const int m = (int)(b & 0x1fffffff);
    const float lo = __fmul_rn(__int2float_rn(m), __uint_as_float((unsigned)(fe - 52) << 23));
    return {hi, sign ? -lo : lo};
}
// f 2^k as a double, from the bits (zero and subnormal floats give 0; the
// caller keeps |k| < 800, so the exponent stays in range)
__device__ __forceinline__ double widen_scaled(float f, int k)
{
    const unsigned u = __float_as_uint(f);
    const unsigned ef = (u >> 23) & 0xff;
    if (ef == 0) return 0.0;
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    return __longlong_as_double((long long)(sign | ((unsigned long long)(ef - 127 + 1023 + k) << 52) |
                                            ((unsigned long long)(u & 0x7fffff) << 29)));
}
// (x.h + x.l) 2^k in FP64: one FP64 instruction
__device__ __forceinline__ double to_d(dfl x, int k) { return widen_scaled(x.h, k) + widen_scaled(x.l, k); }
// unit chord direction (p_{l+1} - p_l) / d_l from the chord vector scaled by
// 2^k and its scaled length h = d_l 2^k (1/h by a float-float Newton step)
__device__ __forceinline__ cdf tau_dfh(double2 cv, dfl h, int k)
{
    const dfl r = df_rcp(h);
    return {df_mul(split_scaled(cv.x, k), r), df_mul(split_scaled(cv.y, k), r)};
}
__device__ __forceinline__ cdf cscale(cdf a, dfl s) { return {df_mul(a.re, s), df_mul(a.im, s)}; }

__device__ __forceinline__ double2 d2(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ double2 add2(double2 a, double2 b) { return d2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 sub2(double2 a, double2 b) { return d2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 scl2(double2 a, double s) { return d2(a.x * s, a.y * s); }
// chord vector p_{l+1} - p_l of a closed curve of n nodes (the same FP64
// subtraction as the chord pass, so the same bits); recomputed from the input
// where it is needed instead of being kept in the workspace
__device__ __forceinline__ double2 chord_vec(const double2* __restrict__ p, int l, int n)
{
    const double2 a = __ldg(p + l), b = __ldg(p + (l + 1 == n ? 0 : l + 1));
    return d2(b.x - a.x, b.y - a.y);
}

// arc-length target L t_k of output k (t_k = k / N_out); (double)k from the
// exact float of k < 2^20 by bits (no FP64 conversion)
__device__ __forceinline__ double arc_target(int k, bool pow2, double LN, double L, int Nout)
{
    const double kd = k > 0 ? widen_f32(__int2float_rn(k)) : 0.0;
    return pow2 ? kd * LN : L * (kd / (double)Nout);
}

// the spline on interval l (knots S_l <= st < S_{l+1}) at arc length st
__device__ __forceinline__ double2 eval_interval(const double2* __restrict__ p,
                                                 const double* U, const double* D,
                                                 const double2* M, int l, int n, double st)
{
    const int ln = (l + 1 == n) ? 0 : l + 1;
    const double2 pl = __ldg(p + l), pn = __ldg(p + ln);
    const double2 cv = d2(pn.x - pl.x, pn.y - pl.y);  // p_{l+1} - p_l
    const double2 Ml = M[l], Mn = M[ln];
    const double d = D[l];
    const double u = st - U[l];      // arc length into the interval
    const double b = u * rcp_nr(d);  // (t - u_l) / h_l
    // cubic weights a(a^2 - 1) h6 and b(b^2 - 1) h6 (a = 1 - b, h6 =
    // h^2 M / 6 / M' = d^2 with M' = M / (6 L^2)) from
    // w = b(b - 1) h6 = -ab h6 = u (u - d): the second is w(1 + b), the
    // first w(2 - b) = 3w - w(1 + b)  (4 FP64 instructions instead of 8)
    const double w = u * (u - d);
    const double cb = fma(w, b, w);
    const double ca = fma(w, 3.0, -cb);
    return d2(fma(ca, Ml.x, fma(cb, Mn.x, fma(b, cv.x, pl.x))),
              fma(ca, Ml.y, fma(cb, Mn.y, fma(b, cv.y, pl.y))));
}

// Output counts of up to kEvalCap outputs per warp in shared memory, one
// padding word per 32 so that a lane walking its own block of 32 consecutive
// entries hits a bank of its own.
constexpr int kEvalCap = 1024;
constexpr int kCntStride = kEvalCap + kEvalCap / 32;
__device__ __forceinline__ int pidx(int k) { return k + (k >> 5); }

__device__ __forceinline__ double shfl_d(double v, int src, int width)
{
    return __shfl_sync(0xffffffffu, v, src, width);
}
__device__ __forceinline__ double2 shfl_d2(double2 v, int src, int width)
{
    return d2(__shfl_sync(0xffffffffu, v.x, src, width), __shfl_sync(0xffffffffu, v.y, src, width));
}

template <bool F32OUT>
__device__ __forceinline__ void store_out(void* zout, int64_t i, double2 v)
{
    if constexpr (F32OUT)
        static_cast<float2*>(zout)[i] = make_float2((float)v.x, (float)v.y);
    else
        static_cast<double2*>(zout)[i] = v;
}

template <bool F32OUT>
__device__ void fill_nan(void* zout, int64_t base, int Nout, int lane)
{
    const double q = __longlong_as_double(0x7ff8000000000000LL);
    for (int k = lane; k < Nout; k += 32) store_out<F32OUT>(zout, base + k, d2(q, q));
}

// one curve by one warp (every branch below is warp-uniform)
template <bool F32OUT>
__device__ __forceinline__ void resample_curve(int64_t curve, int lane,
                                               const double2* __restrict__ pts,
                                               const int64_t* __restrict__ offsets,
                                               int64_t n_pts, int Nout, int flags,
                                               void* __restrict__ zout,
                                               int8_t* __restrict__ status, const Ws& ws,
                                               int* __restrict__ cnt)
{
    const int64_t o = offsets[curve];
    const int64_t o1 = offsets[curve + 1];
    const int64_t zbase = curve * (int64_t)Nout;
    // The CSR offsets come from device memory the host has not seen: a curve
    // whose range is not inside [0, n_pts], runs backwards or holds more than
    // 2^30 nodes is flagged and skipped, so that no index below leaves the
    // input or the workspace (both sized by n_pts).
    if (o < 0 || o1 < o || o1 > n_pts || o1 - o > ((int64_t)1 << 30)) {
        fill_nan<F32OUT>(zout, zbase, Nout, lane);
        if (lane == 0) status[curve] = FA_STATUS_BAD_SIZE;
        return;
    }
    int n = (int)(o1 - o);
    const double2* p = pts + o;

    // ---- input checks (whole warp) ----------------------------------------
    // Non-finite nodes take precedence over every other status.  For curves
    // of 4 or more nodes they are caught in step A, which loads every node
    // anyway (a dropped closing duplicate equals node 0, which A checks).
    const int n_in = n;
    if (n >= 2) {
        const double2 a = __ldg(p), b = __ldg(p + n - 1);
        if (a.x == b.x && a.y == b.y) n -= 1;  // explicit closing duplicate (first = last)
    }
    if (n < 4) {
        bool nf = false;
        for (int l = lane; l < n_in; l += 32) nf |= !finite2(__ldg(p + l));
        nf = __any_sync(0xffffffffu, nf);
        fill_nan<F32OUT>(zout, zbase, Nout, lane);
        if (lane == 0) status[curve] = nf ? FA_STATUS_NONFINITE : FA_STATUS_DEGENERATE;
        return;
    }

    // ---- chunking -----------------------------------------------------------
    int P = 32;
    while (2 * P > n) P >>= 1;  // every chunk has >= 2 nodes (>= 1 interior)
    const bool act = lane < P;
    const int sj = (int)((int64_t)lane * n / P);
    const int sj1 = (int)((int64_t)(lane + 1) * n / P);
    const int ej = sj1 - 1;  // this chunk's interface node

    double* U = ws.U + o;
    double* D = ws.D + o;
    double2* F0 = ws.F0 + o;
    double2* F1 = ws.F1 + o;
    double2* M = ws.M + o;

    // ---- A: chords (node-parallel, coalesced), chunk sums, warp scan --------
    // d = q * rsqrt(q) and 1/d = rsqrt(q) from one reciprocal square root
    // (q = |p_{l+1} - p_l|^2 >= 0, so its bit pattern tests > 0 as an integer)
    bool zero = false, nf = false;
    unsigned emax = 0;      // largest biased exponent of a coordinate
    unsigned dmin = 2047u;  // smallest biased exponent of a chord length
    for (int l = lane; l < n; l += 32) {
        const double2 pl = __ldg(p + l);
        const double2 pn = __ldg(p + ((l + 1 == n) ? 0 : l + 1));
        nf |= !finite2(pl);
        emax = max(emax, max((unsigned)(__double_as_longlong(pl.x) >> 52) & 0x7ffu,
                             (unsigned)(__double_as_longlong(pl.y) >> 52) & 0x7ffu));
        const double dx = pn.x - pl.x, dy = pn.y - pl.y;
        const double q = fma(dx, dx, dy * dy);
        const bool pos = __double_as_longlong(q) > 0;
        const double rs = rsqrt_nr(q);
        zero |= !pos;
        const double dl = pos ? q * rs : 0.0;
        dmin = min(dmin, (unsigned)(__double_as_longlong(dl) >> 52) & 0x7ffu);
        D[l] = dl;
    }
    if (__any_sync(0xffffffffu, nf)) {
        fill_nan<F32OUT>(zout, zbase, Nout, lane);
        if (lane == 0) status[curve] = FA_STATUS_NONFINITE;
        return;
    }
    __syncwarp();
    double csum = 0.0;
    if (act)
        for (int l = sj; l < sj1; ++l) csum += D[l];
    if (__any_sync(0xffffffffu, zero)) {
        fill_nan<F32OUT>(zout, zbase, Nout, lane);
        if (lane == 0) status[curve] = FA_STATUS_DEGENERATE;
        return;
    }
    double incl = csum;  // inclusive scan over lanes (lanes >= P hold 0)
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    const double L = __shfl_sync(0xffffffffu, incl, 31);
    const double base = incl - csum;  // arc length before node s_j
    __syncwarp();

    // The spline solve (steps B-D) runs in float-float, in units scaled by
    // 2^ks (2^-ks <= L < 2^(1-ks)): scaled chords are in (2^-100, 2), their
    // reciprocals below 2^100, every quantity of the solve in float range.
    // Curves whose chords span more than 2^100 below L, or whose perimeter
    // is beyond 2^+-800, solve in FP64.  The solve needs ~1e-8 relative on M
    // (M enters the outputs through terms of order d^2 |M|, a 1e-4..1e-6 part
    // of the curve for these samplings); float-float gives ~1e-13.
    const int eLb = (int)((__double_as_longlong(L) >> 52) & 0x7ff);  // biased exponent of L
    const int dminw = (int)__reduce_min_sync(0xffffffffu, dmin);
    const bool dfsolve = eLb > 1023 - 800 && eLb < 1023 + 800 && eLb - dminw < 100;
    const int ks = 1023 - eLb;

    // ---- output-interval counts (taken in B, used by E) ----------------------
    // For N_out <= kEvalCap each knot S_l is counted at kf(l), the first output
    // k with L t_k >= S_l (none when kf = N_out); the prefix sums of the counts
    // give, for every output, the number of knots at or below its target, so
    // E reads each output's interval from the table instead of searching.
    const bool pow2 = (Nout & (Nout - 1)) == 0;
    const double invN = 1.0 / (double)Nout;
    const double LN = L * invN;  // arc length per output step
    const bool table = Nout <= kEvalCap;
    if (table)
        for (int k = lane; k < Nout; k += 32) cnt[pidx(k)] = 0;
    __syncwarp();
    // kf = ceil(S_l N / L) from an FP32 estimate x (two truncations to 24
    // bits and two roundings: relative error below 3 * 2^-23, so
    // |x - S_l N / L| < 4e-4 for N_out <= 1024) whenever x is at least 1e-3
    // away from an integer; otherwise from the targets themselves
    // (the bit patterns of nonnegative doubles order like their values):
    // checks around the estimate, bisection over [0, N_out] if it is off
    const int eLx = (int)((__double_as_longlong(L) >> 52) & 0x7ff) - 1023;
    const bool est = eLx > -100 && eLx < 120;
    const float nl = est ? __fdiv_rn(__int2float_rn(Nout), seed_f32(L)) : 0.0f;
    auto count_knot = [&](double Sl) {
        const long long sb = __double_as_longlong(Sl);
        int e = 0;
        bool exact = false;
        if (est && sb > 0 && f32_range(Sl)) {
            const float x = __fmul_rn(seed_f32(Sl), nl);
            const float xf = floorf(x);
            const float fr = __fsub_rn(x, xf);
            e = min(__float2int_rz(xf), Nout - 1) + 1;
            exact = fr > 1e-3f && fr < 0.999f;
            if (!exact) e = min(max(__float2int_ru(x), 0), Nout);
        }
        if (!exact) {
            const bool lo_ok =
                e == 0 || __double_as_longlong(arc_target(e - 1, pow2, LN, L, Nout)) < sb;
            const bool hi_ok =
                e == Nout || __double_as_longlong(arc_target(e, pow2, LN, L, Nout)) >= sb;
            if (!(lo_ok && hi_ok)) {
                int lo = 0, hi = Nout;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (__double_as_longlong(arc_target(mid, pow2, LN, L, Nout)) >= sb) hi = mid;
                    else lo = mid + 1;
                }
                e = lo;
            }
        }
        if (e < Nout) atomicAdd(cnt + pidx(e), 1);
    };

    // ---- B: forward sweep over the interior ---------------------------------
    // The system is solved for M' = M / (6 L^2) (right-hand sides tau_l -
    // tau_{l-1}); the evaluation uses h^2 M' = h^2 M / (6 L^2).  The first
    // row needs no special case: with c' = 0, y' = 0, g' = -1 the general
    // recurrence gives exactly den = B, y' = R / B, g' = h_{l-1} / B.
    // Back substitution M_i = y'_i - c'_i M_{i+1} - g'_i I_{j-1} (M_{e_j} = I_j)
    // gives the first interior node as
    //   M_{s_j} = sum_i pi_i (y'_i - g'_i I_{j-1}) + pi_{e_j} I_j,
    //   pi_i = prod_{m = s_j}^{i-1} (-c'_m),
    // so the sweep also accumulates yF = sum pi_i y'_i, gF = sum pi_i g'_i and
    // kF = -pi_{e_j}: M_{s_j} = yF - gF I_{j-1} - kF I_j (no second pass).
    // interface-node equation data kept for the reduced system
    double Ae = 0, Be = 0, Ce = 0;
    double2 Re = d2(0, 0), yL = d2(0, 0);
    double gL = 0, kL = 0;
    double2 yF = d2(0, 0);
    double gF = 0, kF = 0;
    cdf yLd{{0.f, 0.f}, {0.f, 0.f}};  // the float-float solve's last interior values
    dfl gLd{0.f, 0.f}, kLd{0.f, 0.f};
    if (act && !dfsolve) {
        const double* __restrict__ Dr = D;
        double* __restrict__ Ur = U;
        double2* __restrict__ F0r = F0;
        double2* __restrict__ F1r = F1;
        const int lp = (sj == 0) ? n - 1 : sj - 1;
        double hprev = Dr[lp];
        double2 tprev = scl2(chord_vec(p, lp, n), rcp_nr(Dr[lp]));
        double S = base;
        double cp = 0, gp = -1.0;
        double2 yp = d2(0, 0);
        double pi = 1.0;
        // operands of the next row, loaded one row ahead
        double h = Dr[sj], ih = rcp_nr(h);
        double2 cv = chord_vec(p, sj, n);
        for (int i = sj; i < ej; ++i) {
            const double hn = Dr[i + 1], ihn = rcp_nr(hn);  // i + 1 <= ej < n
            const double2 cvn = chord_vec(p, i + 1, n);
            Ur[i] = S;
            if (table) count_knot(S);
            S += h;
            const double2 tau = scl2(cv, ih);
            const double2 R = sub2(tau, tprev);
            const double B = twice_pos(hprev + h);
            const double den = fma(-hprev, cp, B);
            const double r = rcp_nr(den);
            const double ncp = h * r;
            const double2 nyp = d2((R.x - hprev * yp.x) * r, (R.y - hprev * yp.y) * r);
            const double ngp = -hprev * gp * r;
            F0r[i] = d2(ncp, ngp);
            F1r[i] = nyp;
            yF = d2(fma(pi, nyp.x, yF.x), fma(pi, nyp.y, yF.y));
            gF = fma(pi, ngp, gF);
            pi *= -ncp;
            cp = ncp; gp = ngp; yp = nyp;
            hprev = h; tprev = tau;
            h = hn; ih = ihn; cv = cvn;
        }
        kF = -pi;
        // last interior node's values: M_L = y'_L - I_{j-1} g'_L - I_j c'_L
        yL = yp; gL = gp; kL = cp;
        // interface node e_j (the loop, which runs at least once, leaves h,
        // ih and cv holding chord e_j's values)
        Ur[ej] = S;
        if (table) count_knot(S);
        const double2 tau = scl2(cv, ih);
        Re = sub2(tau, tprev);
        Ae = hprev;
        Ce = h;
        Be = twice_pos(hprev + Ce);
    } else if (act) {
        // the same sweep in float-float (scaled units; FP64 only for the arc
        // lengths S and the conversions of the interface data below)
        const double* __restrict__ Dr = D;
        double* __restrict__ Ur = U;
        float4* __restrict__ F0r = reinterpret_cast<float4*>(F0);
        float4* __restrict__ F1r = reinterpret_cast<float4*>(F1);
        const int lp = (sj == 0) ? n - 1 : sj - 1;
        dfl hprev = split_scaled(Dr[lp], ks);
        cdf tprev = tau_dfh(chord_vec(p, lp, n), hprev, ks);
        double S = base;
        dfl cp{0.f, 0.f}, gp{-1.f, 0.f}, pi{1.f, 0.f}, gFd{0.f, 0.f};
        cdf yp{{0.f, 0.f}, {0.f, 0.f}}, yFd{{0.f, 0.f}, {0.f, 0.f}};
        double h64 = Dr[sj];
        double2 cv = chord_vec(p, sj, n);
        for (int i = sj; i < ej; ++i) {
            const double hn64 = Dr[i + 1];  // i + 1 <= ej < n
            const double2 cvn = chord_vec(p, i + 1, n);
            Ur[i] = S;
            if (table) count_knot(S);
            S += h64;
            const dfl h = split_scaled(h64, ks);
            const cdf tau = tau_dfh(cv, h, ks);
            const cdf R = csub(tau, tprev);
            const dfl den = df_sub(df_twice(df_add(hprev, h)), df_mul(hprev, cp));
            const dfl r = df_rcp(den);
            const dfl ncp = df_mul(h, r);
            const cdf nyp{df_mul(df_sub(R.re, df_mul(hprev, yp.re)), r),
                          df_mul(df_sub(R.im, df_mul(hprev, yp.im)), r)};
            const dfl ngp = df_neg(df_mul(df_mul(hprev, gp), r));
            F0r[i] = make_float4(ncp.h, ncp.l, ngp.h, ngp.l);
            F1r[i] = st4(nyp);
            yFd = cadd(yFd, cscale(nyp, pi));
            gFd = df_add(gFd, df_mul(pi, ngp));
            pi = df_neg(df_mul(pi, ncp));
            cp = ncp; gp = ngp; yp = nyp;
            hprev = h; tprev = tau;
            h64 = hn64; cv = cvn;
        }
        yLd = yp; gLd = gp; kLd = cp;
        Ur[ej] = S;
        if (table) count_knot(S);
        const dfl Ced = split_scaled(h64, ks);
        const cdf Red = csub(tau_dfh(cv, Ced, ks), tprev);
        // the interface data in FP64 for the reduced system (scaled units)
        Ae = to_d(hprev, 0);
        Ce = to_d(Ced, 0);
        Be = to_d(df_twice(df_add(hprev, Ced)), 0);
        Re = d2(to_d(Red.re, 0), to_d(Red.im, 0));
        yL = d2(to_d(yp.re, 0), to_d(yp.im, 0));
        gL = to_d(gp, 0);
        kL = to_d(cp, 0);
        yF = d2(to_d(yFd.re, 0), to_d(yFd.im, 0));
        gF = to_d(gFd, 0);
        kF = -to_d(pi, 0);
    }

    // reduced cyclic system over the P interfaces:
    //   al I_{j-1} + be I_j + ga I_{j+1} = de
    const int nxt = (lane + 1) & (P - 1);
    const int prv = (lane + P - 1) & (P - 1);
    const double2 yFn = shfl_d2(yF, nxt, P);
    const double gFn = shfl_d(gF, nxt, P);
    const double kFn = shfl_d(kF, nxt, P);
    double al = -Ae * gL;
    double be = Be - Ae * kL - Ce * gFn;
    double ga = -Ce * kFn;
    double2 de = d2(Re.x - Ae * yL.x - Ce * yFn.x, Re.y - Ae * yL.y - Ce * yFn.y);
    // parallel cyclic reduction: strides 1, 2, .., P/4 leave each equation
    // coupled only to the one at distance P/2
    for (int s = 1; 2 * s < P; s <<= 1) {
        const int lm = (lane + P - s) & (P - 1), lq = (lane + s) & (P - 1);
        const double al_m = shfl_d(al, lm, P), be_m = shfl_d(be, lm, P), ga_m = shfl_d(ga, lm, P);
        const double2 de_m = shfl_d2(de, lm, P);
        const double al_p = shfl_d(al, lq, P), be_p = shfl_d(be, lq, P), ga_p = shfl_d(ga, lq, P);
        const double2 de_p = shfl_d2(de, lq, P);
        // the diagonals stay positive (diagonally dominant system), and M
        // enters the output only through d^2-scaled terms: the reciprocals'
        // 1e-13 relative error is far below what the output resolves
        const double k1 = al * rcp_nr(be_m), k2 = ga * rcp_nr(be_p);
        be = be - ga_m * k1 - al_p * k2;
        de = d2(de.x - de_m.x * k1 - de_p.x * k2, de.y - de_m.y * k1 - de_p.y * k2);
        al = -al_m * k1;
        ga = -ga_p * k2;
    }
    double2 I;
    {
        const int pm = (lane + P / 2) & (P - 1);
        const double off_j = al + ga;
        const double off_m = shfl_d(al, pm, P) + shfl_d(ga, pm, P);
        const double be_m = shfl_d(be, pm, P);
        const double2 de_m = shfl_d2(de, pm, P);
        const double rdet = rcp_nr(be * be_m - off_j * off_m);
        I = d2((de.x * be_m - off_j * de_m.x) * rdet, (de.y * be_m - off_j * de_m.y) * rdet);
    }
    const double2 Iprev = shfl_d2(I, prv, P);

    // ---- D: second backward sweep writes M ----------------------------------
    if (act && dfsolve) {
        // float-float, scaled units; M' = M_scaled 2^ks stored in FP64
        const double sc = __longlong_as_double((long long)(1023 + ks) << 52);  // 2^ks
        M[ej] = scl2(I, sc);
        const cdf Id = split_c(I), Ipd = split_c(Iprev);
        cdf Mi{df_sub(df_sub(yLd.re, df_mul(Ipd.re, gLd)), df_mul(Id.re, kLd)),
               df_sub(df_sub(yLd.im, df_mul(Ipd.im, gLd)), df_mul(Id.im, kLd))};
        M[ej - 1] = d2(to_d(Mi.re, ks), to_d(Mi.im, ks));
        const float4* __restrict__ F0r = reinterpret_cast<const float4*>(F0);
        const float4* __restrict__ F1r = reinterpret_cast<const float4*>(F1);
        for (int i = ej - 2; i >= sj; --i) {
            const float4 f0 = F0r[i];
            const cdf y = ld4(F1r[i]);
            const dfl c{f0.x, f0.y}, g{f0.z, f0.w};
            Mi = {df_sub(df_sub(y.re, df_mul(c, Mi.re)), df_mul(g, Ipd.re)),
                  df_sub(df_sub(y.im, df_mul(c, Mi.im)), df_mul(g, Ipd.im))};
            M[i] = d2(to_d(Mi.re, ks), to_d(Mi.im, ks));
        }
    } else if (act) {
        M[ej] = I;
        double2 Mi = d2(yL.x - Iprev.x * gL - I.x * kL, yL.y - Iprev.y * gL - I.y * kL);
        M[ej - 1] = Mi;
        for (int i = ej - 2; i >= sj; --i) {
            const double2 f0 = F0[i];
            const double2 f1 = F1[i];
            Mi = d2(fma(-f0.x, Mi.x, fma(-Iprev.x, f0.y, f1.x)),
                    fma(-f0.x, Mi.y, fma(-Iprev.y, f0.y, f1.y)));
            M[i] = Mi;
        }
    }
    __syncwarp();

    // ---- E: evaluation at t_k = k / N_out ------------------------------------
    double2* raw = F32OUT ? (ws.Z + zbase) : (static_cast<double2*>(zout) + zbase);
    double2 ssum = d2(0, 0);
    const bool unit = (flags & FA_UNIT_LENGTH) != 0;
    double per_len = 0.0;
    // The node sum (for the mean) and the perimeter of the outputs are
    // accumulated in float-float (about 48 significant bits; FP64 is the
    // scarce unit) when every coordinate and the perimeter lie in a range
    // where the float parts stay normal: coordinates below 2^60 in magnitude,
    // perimeter in [2^-40, 2^40].  Their errors (2^-47 of each summand, the
    // chord lengths to 2^-46 of themselves) move the normalised nodes by
    // < 1e-14.  Other curves sum in FP64.
    const int eL = (int)((__double_as_longlong(L) >> 52) & 0x7ff) - 1023;
    const bool dfsum = __reduce_max_sync(0xffffffffu, emax) < 1023u + 60u && eL > -40 && eL < 40;
    dfl sx{0.f, 0.f}, sy{0.f, 0.f}, per_df{0.f, 0.f};
    // one output into the mean's sum; one chord |a - b| into the perimeter
    // (the chord's components in FP64, exact differences of nearby values;
    // its length and both sums in float-float when dfsum)
    auto add_node = [&](double2 S) {
        if (dfsum) {
            const cdf Sd = split_c(S);
            sx = df_add(sx, Sd.re);
            sy = df_add(sy, Sd.im);
        } else {
            ssum = add2(ssum, S);
        }
    };
    auto add_chord = [&](double2 a, double2 b) {
        if (dfsum) {
            per_df = df_add(per_df, df_chord(sub2(a, b)));
        } else {
            const double dx = a.x - b.x, dy = a.y - b.y;
            const double q = fma(dx, dx, dy * dy);
            per_len += __double_as_longlong(q) > 0 ? sqrt_nr(q) : 0.0;
        }
    };
    int k0 = 0, k1 = 0;
    double2 Sfirst = d2(0, 0), Sprev = d2(0, 0);
    if (table) {
        // the interval of every output from the counts taken in B: l_k =
        // (number of knots S_l <= L t_k) - 1, the last knot at or below the
        // target (the knots are nondecreasing); then 32 consecutive outputs at
        // a time are evaluated with independent, nearly coalesced loads
        // inclusive prefix sums: lane i sums its block of consecutive k, a
        // warp scan gives the block's offset, the block is rewritten as l_k
        const int per = (Nout + 31) >> 5;
        const int q0 = min(lane * per, Nout), q1 = min(q0 + per, Nout);
        int run = 0;
        for (int k = q0; k < q1; ++k) run += cnt[pidx(k)];
        int incl = run;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        int acc = incl - run - 1;
        for (int k = q0; k < q1; ++k) {
            acc += cnt[pidx(k)];
            cnt[pidx(k)] = acc;
        }
        __syncwarp();
        // outputs g + lane; the chord to output k - 1 comes from the lane
        // below, or for lane 0 from the previous group's last output
        double2 S = d2(0, 0), Sc = d2(0, 0), S0 = d2(0, 0);
        for (int g = 0; g < Nout; g += 32) {
            const int k = g + lane;
            if (k < Nout) {
                S = eval_interval(p, U, D, M, cnt[pidx(k)], n, arc_target(k, pow2, LN, L, Nout));
                raw[k] = S;
                add_node(S);
            }
            const double2 Sb = d2(__shfl_up_sync(0xffffffffu, S.x, 1),
                                  __shfl_up_sync(0xffffffffu, S.y, 1));
            if (unit && k < Nout && k > 0) add_chord(S, lane == 0 ? Sc : Sb);
            Sc = shfl_d2(S, 31, 32);
            if (g == 0) S0 = S;
        }
        if (unit) {  // the closing chord, output N_out - 1 to output 0 (lane 0)
            const double2 Sl = shfl_d2(S, (Nout - 1) & 31, 32);
            if (lane == 0) add_chord(S0, Sl);
        }
    } else {
        // each lane a contiguous block of outputs, its first interval by
        // bisection over the knots, the following ones by stepping
        const int per = (Nout + 31) / 32;
        k0 = lane * per;
        k1 = min(k0 + per, Nout);
        if (k0 < k1) {
            const long long sb0 = __double_as_longlong(arc_target(k0, pow2, LN, L, Nout));
            // last l with S_l <= L t (S_0 = 0)
            int lo = 0, hi = n - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__double_as_longlong(U[mid]) <= sb0) lo = mid; else hi = mid - 1;
            }
            int l = lo;
            for (int k = k0; k < k1; ++k) {
                const double st = arc_target(k, pow2, LN, L, Nout);
                const long long sb = __double_as_longlong(st);
                while (l + 1 < n && __double_as_longlong(U[l + 1]) <= sb) ++l;
                const double2 S = eval_interval(p, U, D, M, l, n, st);
                raw[k] = S;
                add_node(S);
                if (unit) {
                    if (k > k0) add_chord(S, Sprev);
                    else Sfirst = S;
                    Sprev = S;
                }
            }
        }
    }
    if (dfsum) {  // the lane's float-float partial sums to FP64 (exact: h + l)
        ssum = d2(widen_any(sx.h) + widen_any(sx.l), widen_any(sy.h) + widen_any(sy.l));
        per_len = widen_any(per_df.h) + widen_any(per_df.l);
    }
    if (!table && unit) {
        // the chord from this lane's last output to the next one: the next
        // lane's first (output k1), or output 0 after the last output
        const double2 Snext = shfl_d2(Sfirst, k1 < Nout ? lane + 1 : 0, 32);
        if (k0 < k1) {
            const double dx = Snext.x - Sprev.x, dy = Snext.y - Sprev.y;
            const double q = fma(dx, dx, dy * dy);
            per_len += __double_as_longlong(q) > 0 ? sqrt_nr(q) : 0.0;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        ssum.x += __shfl_xor_sync(0xffffffffu, ssum.x, off);
        ssum.y += __shfl_xor_sync(0xffffffffu, ssum.y, off);
    }
    __syncwarp();
    const double2 mean = (flags & FA_CENTER) ? d2(ssum.x * invN, ssum.y * invN) : d2(0, 0);
    double scale = 1.0;
    if (flags & FA_UNIT_LENGTH) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) per_len += __shfl_xor_sync(0xffffffffu, per_len, off);
        if (!(per_len > 0.0)) {
            __syncwarp();
            fill_nan<F32OUT>(zout, zbase, Nout, lane);
            if (lane == 0) status[curve] = FA_STATUS_DEGENERATE;
            return;
        }
        scale = 1.0 / per_len;
    }
    const double2 off = d2(-mean.x * scale, -mean.y * scale);
    for (int k = lane; k < Nout; k += 32) {
        const double2 S = raw[k];
        store_out<F32OUT>(zout, zbase + k, d2(fma(S.x, scale, off.x), fma(S.y, scale, off.y)));
    }
    if (lane == 0) status[curve] = FA_STATUS_OK;
}

// Persistent grid: each warp takes the next curve from a counter until none is
// left (curve sizes differ, so a fixed assignment would leave the last wave of
// CTAs as a tail).  The curves are taken in input order: handing out long
// curves first measured slower (more workspace in flight at once).
template <bool F32OUT>
__global__ void __launch_bounds__(kWarps * 32, FA_RESAMPLE_MIN_BLOCKS)
    resample_kernel(const double2* __restrict__ pts, const int64_t* __restrict__ offsets,
                    int64_t C, int64_t n_pts, int Nout, int flags, void* __restrict__ zout,
                    int8_t* __restrict__ status, Ws ws, unsigned long long* __restrict__ next)
{
    __shared__ int s_cnt[kWarps * kCntStride];  // each warp's output-interval table
    const int lane = threadIdx.x & 31;
    int* cnt = s_cnt + (threadIdx.x >> 5) * kCntStride;
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(next, 1ull);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= (unsigned long long)C) break;
        resample_curve<F32OUT>((int64_t)c, lane, pts, offsets, n_pts, Nout, flags, zout, status,
                               ws, cnt);
        __syncwarp();
    }
}

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

size_t resample_ws_bytes(int64_t C, int64_t n_pts, int N_out, int flags)
{
    // sizes beyond 2^40 nodes or curves saturate (no caller can hold them, and a
    // wrapped product would make an impossible batch look small)
    constexpr int64_t kMax = (int64_t)1 << 40;
    if (C > kMax || n_pts > kMax || N_out > (1 << 20)) return SIZE_MAX;
    const size_t np = (size_t)(n_pts > 0 ? n_pts : 0);
    size_t b = 2 * align256(np * sizeof(double)) + 2 * align256(np * sizeof(double2));
    const size_t c = (size_t)(C > 0 ? C : 0);
    if (flags & FA_STORE_FP32) b += align256(c * (size_t)N_out * sizeof(double2));
    return b + 256;  // the work counter
}

int launch_resample(const fa_handle* h, const double* pts, const int64_t* offsets, int64_t C,
                    int64_t n_pts, int N_out, int flags, void* z_out, int8_t* status, void* wsp,
                    cudaStream_t st, unsigned long long* counter, int64_t stage_curve0)
{
    if (C == 0) return FA_OK;
    const size_t np = (size_t)(n_pts > 0 ? n_pts : 0);
    char* b = static_cast<char*>(wsp);
    Ws ws;
    ws.U = reinterpret_cast<double*>(b); b += align256(np * sizeof(double));
    ws.D = reinterpret_cast<double*>(b); b += align256(np * sizeof(double));
    ws.F0 = reinterpret_cast<double2*>(b); b += align256(np * sizeof(double2));
    ws.F1 = reinterpret_cast<double2*>(b); b += align256(np * sizeof(double2));
    ws.M = ws.F1;  // M_i overwrites y'_i: step D reads each y'_i just before it writes M_i
    ws.Z = (flags & FA_STORE_FP32) ? reinterpret_cast<double2*>(b) + stage_curve0 * N_out : nullptr;
    if (flags & FA_STORE_FP32) b += align256((size_t)C * (size_t)N_out * sizeof(double2));
    unsigned long long* next = counter ? counter : reinterpret_cast<unsigned long long*>(b);
    int sms = h ? h->num_sms : 0;
    if (sms <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 1;
    }
    const int64_t blocks = std::min<int64_t>((C + kWarps - 1) / kWarps,
                                             (int64_t)sms * FA_RESAMPLE_MIN_BLOCKS);
    const double2* p = reinterpret_cast<const double2*>(pts);
    const cudaError_t me = cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
    if (me != cudaSuccess) return cuda_error(me, "resample counter reset");
    if (flags & FA_STORE_FP32)
        resample_kernel<true><<<(unsigned)blocks, kWarps * 32, 0, st>>>(
            p, offsets, C, (int64_t)np, N_out, flags, z_out, status, ws, next);
    else
        resample_kernel<false><<<(unsigned)blocks, kWarps * 32, 0, st>>>(
            p, offsets, C, (int64_t)np, N_out, flags, z_out, status, ws, next);
    return cuda_error(cudaGetLastError(), "resample launch");
}

}  // namespace fa
