// fa_internal.cuh -- shared declarations of the CUDA side of libfftalign.so.
// Device helpers here are used only by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "fftalign.h"

struct fa_handle {
    int device = 0;
    int num_sms = 0;
    // twiddle tables W_N[k] = exp(-2 pi i k / N), k = 0..N-1, for N = 2^logn,
    // logn in [2, 14] for tw64 (the ragged path's long transforms), [2, 12] otherwise
    double2* tw64[15] = {};
    float2* tw32[13] = {};
    // FMA-form twiddles for e in [0, N/2): (m, rho) with W_N^e = m (1 + i rho) when
    // |cos| >= |sin| (e <= N/8 or e >= 3N/8), else W_N^e = m (rho + i); |rho| <= 1
    double2* tf64[13] = {};
    float4* tdf[13] = {};   // W_N[k] in double-float (re.h, re.l, im.h, im.l), FA_PREC_MIXED
    // fa_align_pairs_ragged: the plan (index into the compiled (CTA size, pairs
    // per CTA) set) of each transform-length bucket log2 L, and the time per
    // bucket of the last autotuning (ms, 0 when untuned)
    int ragged_plan[16] = {};
    float ragged_plan_ms[16] = {};
    // handle-owned scratch, used when the caller passes no workspace
    void* ws = nullptr;
    size_t ws_bytes = 0;
    // streams and events of the pipelined host entry point (created on first use)
    cudaStream_t pipe[4] = {};
    cudaEvent_t pipe_ev[5] = {};
};

namespace fa {

constexpr int kMinLogN = 2;
constexpr int kMaxLogN = 12;
constexpr int kMaxDirectN = 4096;
constexpr int kMaxElasticN = 1024;
// below 32 nodes the elastic alternation is not stable under rounding (an input
// perturbation of 1e-15 moves the energy by 1e-2 at N = 8 and 16)
constexpr int kMinElasticN = 32;
constexpr int kMaxRaggedN = 8192;      // largest node count of fa_align_pairs_ragged
constexpr int kMaxRaggedLogL = 14;     // its longest transform, 2^14

// error reporting (thread-local message for fa_last_error)
int set_error(int code, const std::string& msg);
int cuda_error(cudaError_t e, const char* where);

// Makes the handle's device current for the lifetime of the object and
// restores the caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    int rc = FA_OK;
    explicit DeviceGuard(int dev)
    {
        cudaError_t e = cudaGetDevice(&prev);
        if (e == cudaSuccess && prev != dev) e = cudaSetDevice(dev);
        if (e != cudaSuccess) rc = cuda_error(e, "cudaSetDevice");
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};


// ---------------------------------------------------------------- device ----
__device__ __forceinline__ bool finite2(double2 v)
{
    // exponent field all ones <=> Inf or NaN; integer test, no FP64 instruction
    const unsigned long long ex = 0x7ff0000000000000ULL;
    return ((__double_as_longlong(v.x) & ex) != ex) && ((__double_as_longlong(v.y) & ex) != ex);
}

__device__ __forceinline__ double2 ld_z(const double2* __restrict__ p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ double2 ld_z(const float2* __restrict__ p, int64_t i)
{
    const float2 v = __ldg(p + i);
    return make_double2((double)v.x, (double)v.y);
}

// (a.x + i a.y)(b.x + i b.y): 2 DMUL + 2 DFMA
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ double2 cmulc(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}

// Which form a FMA twiddle W_N^e (0 <= e < N/2) is stored in (see fa_handle::tf64).
__host__ __device__ __forceinline__ bool tw_form_b(int e, int N) { return 8 * e > N && 8 * e < 3 * N; }

// argmax key order: larger |c|^2 first, then the smaller shift.  |c|^2 >= 0,
// so its IEEE bit pattern orders like the value (integer compare).
__device__ __forceinline__ bool key_better(long long ka, int ia, long long kb, int ib)
{
    return ka > kb || (ka == kb && ia < ib);
}

// ------------------------------------------------------------- launchers ----
int launch_align_fft(const fa_handle* h, const void* z1, const void* z2, int64_t P, int logn,
                     int ztype, int32_t* shift, double* theta, double* energy, int8_t* status,
                     cudaStream_t st);
int launch_align_df(const fa_handle* h, const void* z1, const void* z2, int64_t P, int logn,
                    int ztype, int32_t* shift, double* theta, double* energy, int8_t* status,
                    cudaStream_t st);
int launch_align_all_df(const fa_handle* h, const void* z, int64_t M, int logn, int ztype,
                        void* ws, int8_t* status, int32_t* shift, double* theta, double* energy,
                        cudaStream_t st);
int launch_align_direct(const fa_handle* h, const void* z1, const void* z2, int64_t P, int N,
                        int ztype, int32_t* shift, double* theta, double* energy, int8_t* status,
                        cudaStream_t st);
size_t align_all_ws_bytes(int64_t M, int N);
// spectra of M curves (FP64) into spec [M][N]; statuses and the diagonal of the
// all-pairs outputs
int launch_spectra(const fa_handle* h, const void* z, int64_t M, int logn, int ztype,
                   double2* spec, int8_t* status, int32_t* shift, double* theta, double* energy,
                   cudaStream_t st);
// the tensor-core all-pairs search (prec = FA_PREC_TC_*), N = 256 or 512
size_t align_all_tc_ws_bytes(int64_t M, int logn, int prec);
int launch_align_all_tc(const fa_handle* h, const void* z, int64_t M, int logn, int ztype, int prec,
                        void* ws, int8_t* status, int32_t* shift, double* theta, double* energy,
                        cudaStream_t st);
int launch_align_all(const fa_handle* h, const void* z, int64_t M, int logn, int ztype, void* ws,
                     int8_t* status, int32_t* shift, double* theta, double* energy,
                     cudaStream_t st);
int ragged_set_attributes();
size_t ragged_ws_bytes(const fa_handle* h, int64_t P, int max_n);
int ragged_num_plans();
int ragged_plan_threads(int plan);
int ragged_plan_group(int plan);
bool ragged_plan_fits(int plan, int bucket);
int ragged_default_plan(int bucket);
int ragged_max_bucket(int max_n);
int ragged_prepare(const int64_t* off, int64_t P, int max_n, void* ws, int32_t* shift,
                   double* theta, double* energy, int8_t* status, cudaStream_t st);
int ragged_hist(void* ws, int* hist, cudaStream_t st);
int ragged_run_bucket(const fa_handle* h, const void* z1, const void* z2, const int64_t* off,
                      int64_t P, int max_n, int ztype, int bucket, int plan, int32_t* shift,
                      double* theta, double* energy, int8_t* status, void* ws, bool reset,
                      cudaStream_t st);
int launch_align_ragged(const fa_handle* h, const void* z1, const void* z2, const int64_t* off,
                        int64_t P, int max_n, int ztype, int32_t* shift, double* theta,
                        double* energy, int8_t* status, void* ws, cudaStream_t st);
// counter: the kernel's 8-byte work counter, or nullptr for the one at the end
// of ws; stage_curve0: the first curve's row in ws's complex128 staging area
// (FA_STORE_FP32).  Launches that share one workspace concurrently (disjoint
// curves of one CSR array, offsets absolute) pass their own counter and row.
int launch_resample(const fa_handle* h, const double* pts, const int64_t* offsets, int64_t C,
                    int64_t n_pts, int N_out, int flags, void* z_out, int8_t* status, void* ws,
                    cudaStream_t st, unsigned long long* counter = nullptr,
                    int64_t stage_curve0 = 0);
size_t resample_ws_bytes(int64_t C, int64_t n_pts, int N_out, int flags);
int build_twiddles(fa_handle* h);
size_t elastic_ws_bytes(const fa_handle* h, int64_t M1, int64_t M2, int64_t P, int N, int band);
int launch_elastic(const fa_handle* h, const double* set1, int64_t M1, const double* set2,
                   int64_t M2, int N, const int64_t* idx1, const int64_t* idx2, int64_t P,
                   int band, int max_iter, int32_t* shift, double* theta, double* energy,
                   double* gamma, int32_t* iters, int32_t* lm_steps, int8_t* status, void* ws,
                   cudaStream_t st);

}  // namespace fa
