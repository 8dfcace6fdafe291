// api.cu -- the extern "C" entry points of libfftalign.so (declared, with
// their contracts, in include/fftalign.h): argument validation, device
// selection, twiddle tables and workspace management.  All arithmetic of the
// method runs in the kernels of align_fft.cu, align_direct.cu and resample.cu.
#include <cuda_runtime.h>

#include <new>
#include <string>

#include "fa_internal.cuh"

namespace fa {

static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

int cuda_error(cudaError_t e, const char* where)
{
    if (e == cudaSuccess) return FA_OK;
    return set_error(FA_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// W_N[k] = exp(-2 pi i k / N) = cospi(2k/N) - i sinpi(2k/N); 2k/N is exact in binary.
__global__ void twiddle_kernel(double2* w64, float2* w32, int N)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    double s, c;
    sincospi(2.0 * (double)k / (double)N, &s, &c);
    w64[k] = make_double2(c, -s);
    w32[k] = make_float2((float)c, (float)-s);
}

// FMA-form twiddles (m, rho) for e in [0, N/2): W = m (1 + i rho) or m (rho + i).
__global__ void fma_twiddle_kernel(double2* tf, int N)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N / 2) return;
    double s, c;
    sincospi(2.0 * (double)e / (double)N, &s, &c);
    const double wr = c, wi = -s;
    tf[e] = tw_form_b(e, N) ? make_double2(wi, wr / wi) : make_double2(wr, wi / wr);
}

// W_N[k] as double-float pairs: hi = nearest float, lo = nearest float to the rest
__global__ void df_twiddle_kernel(const double2* w64, float4* tdf, int N)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const double2 w = w64[k];
    const float rh = __double2float_rn(w.x), ih = __double2float_rn(w.y);
    tdf[k] = make_float4(rh, __double2float_rn(w.x - (double)rh), ih,
                         __double2float_rn(w.y - (double)ih));
}

int build_twiddles(fa_handle* h)
{
    for (int L = kMaxLogN + 1; L <= kMaxRaggedLogL; ++L) {
        const int N = 1 << L;
        float2* tmp32 = nullptr;
        cudaError_t e = cudaMalloc(&h->tw64[L], N * sizeof(double2));
        if (e == cudaSuccess) e = cudaMalloc(&tmp32, N * sizeof(float2));
        if (e != cudaSuccess) return cuda_error(e, "fa_create: cudaMalloc twiddles");
        twiddle_kernel<<<(N + 255) / 256, 256>>>(h->tw64[L], tmp32, N);
        e = cudaDeviceSynchronize();
        cudaFree(tmp32);
        if (e != cudaSuccess) return cuda_error(e, "fa_create: twiddle kernel");
    }
    for (int L = kMinLogN; L <= kMaxLogN; ++L) {
        const int N = 1 << L;
        cudaError_t e = cudaMalloc(&h->tw64[L], N * sizeof(double2));
        if (e != cudaSuccess) return cuda_error(e, "fa_create: cudaMalloc twiddles");
        e = cudaMalloc(&h->tw32[L], N * sizeof(float2));
        if (e != cudaSuccess) return cuda_error(e, "fa_create: cudaMalloc twiddles");
        e = cudaMalloc(&h->tf64[L], (N / 2) * sizeof(double2));
        if (e != cudaSuccess) return cuda_error(e, "fa_create: cudaMalloc twiddles");
        e = cudaMalloc(&h->tdf[L], N * sizeof(float4));
        if (e != cudaSuccess) return cuda_error(e, "fa_create: cudaMalloc twiddles");
        fma_twiddle_kernel<<<(N / 2 + 255) / 256, 256>>>(h->tf64[L], N);
        twiddle_kernel<<<(N + 255) / 256, 256>>>(h->tw64[L], h->tw32[L], N);
        df_twiddle_kernel<<<(N + 255) / 256, 256>>>(h->tw64[L], h->tdf[L], N);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_error(e, "fa_create: twiddle kernel");
    }
    return cuda_error(cudaDeviceSynchronize(), "fa_create: twiddle build");
}

static int ensure_ws(fa_handle* h, size_t bytes)
{
    if (h->ws_bytes >= bytes) return FA_OK;
    if (h->ws) {
        cudaError_t e = cudaFree(h->ws);  // implicit device synchronisation
        h->ws = nullptr;
        h->ws_bytes = 0;
        if (e != cudaSuccess) return cuda_error(e, "workspace cudaFree");
    }
    cudaError_t e = cudaMalloc(&h->ws, bytes);
    if (e != cudaSuccess) {
        h->ws = nullptr;
        return cuda_error(e, "workspace cudaMalloc");
    }
    h->ws_bytes = bytes;
    return FA_OK;
}

// A pair inherits the resampling status of its curves: a curve that could not
// be resampled makes the pair's outputs NaN with that status.
// pairs p < count: curve statuses rst[p] and rst[p + second] (the pair's two
// curves) override the alignment's outputs
__global__ void merge_status_kernel(const int8_t* __restrict__ rst, int64_t count, int64_t second,
                                    int32_t* __restrict__ shift, double* __restrict__ theta,
                                    double* __restrict__ energy, int8_t* __restrict__ status)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= count) return;
    const int8_t s = rst[p] != FA_STATUS_OK ? rst[p] : rst[second + p];
    if (s != FA_STATUS_OK) {
        shift[p] = -1;
        theta[p] = __longlong_as_double(0x7ff8000000000000LL);
        energy[p] = __longlong_as_double(0x7ff8000000000000LL);
        status[p] = s;
    }
}

}  // namespace fa

using namespace fa;

extern "C" {

const char* fa_last_error(void) { return g_last_error.c_str(); }

int fa_version(void) { return 10000; }

int fa_create(fa_handle** out, int device)
{
    if (!out) return set_error(FA_ERR_INVALID_ARG, "fa_create: null handle pointer");
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return cuda_error(e, "fa_create: cudaGetDeviceCount");
    if (device < 0 || device >= count)
        return set_error(FA_ERR_INVALID_ARG, "fa_create: no such device");
    fa_handle* h = new (std::nothrow) fa_handle();
    if (!h) return set_error(FA_ERR_INVALID_ARG, "fa_create: out of host memory");
    h->device = device;
    for (int b = 0; b < 16; ++b) h->ragged_plan[b] = ragged_default_plan(b);
    DeviceGuard g(device);
    if (g.rc != FA_OK) { delete h; return g.rc; }
    e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) { delete h; return cuda_error(e, "fa_create: attributes"); }
    int rc = build_twiddles(h);
    if (rc == FA_OK) rc = ragged_set_attributes();
    if (rc != FA_OK) { fa_destroy(h); return rc; }
    *out = h;
    return FA_OK;
}

int fa_destroy(fa_handle* h)
{
    if (!h) return set_error(FA_ERR_INVALID_ARG, "fa_destroy: null handle");
    DeviceGuard g(h->device);
    for (int L = kMaxLogN + 1; L <= kMaxRaggedLogL; ++L)
        if (h->tw64[L]) cudaFree(h->tw64[L]);
    for (int L = 0; L <= kMaxLogN; ++L) {
        if (h->tw64[L]) cudaFree(h->tw64[L]);
        if (h->tw32[L]) cudaFree(h->tw32[L]);
        if (h->tf64[L]) cudaFree(h->tf64[L]);
        if (h->tdf[L]) cudaFree(h->tdf[L]);
    }
    if (h->ws) cudaFree(h->ws);
    for (int k = 0; k < 4; ++k)
        if (h->pipe[k]) cudaStreamDestroy(h->pipe[k]);
    for (int k = 0; k < 5; ++k)
        if (h->pipe_ev[k]) cudaEventDestroy(h->pipe_ev[k]);
    delete h;
    return FA_OK;
}

size_t fa_resample_workspace_size(int64_t C, int64_t n_pts, int32_t N_out, int32_t flags)
{
    if (C < 0 || n_pts < 0 || N_out <= 0) return 0;
    return resample_ws_bytes(C, n_pts, N_out, flags);
}

int fa_resample_arclength(fa_handle* h, const double* pts, const int64_t* offsets, int64_t C,
                          int64_t n_pts, int32_t N_out, int32_t flags, void* z_out,
                          int8_t* status, void* workspace, size_t workspace_bytes, void* stream)
{
    if (!h) return set_error(FA_ERR_INVALID_ARG, "fa_resample_arclength: null handle");
    if (C < 0 || n_pts < 0)
        return set_error(FA_ERR_INVALID_ARG, "fa_resample_arclength: negative size");
    if (N_out < 4 || N_out > (1 << 20))
        return set_error(FA_ERR_UNSUPPORTED, "fa_resample_arclength: N_out outside [4, 2^20]");
    if (flags & ~(FA_CENTER | FA_UNIT_LENGTH | FA_STORE_FP32))
        return set_error(FA_ERR_INVALID_ARG, "fa_resample_arclength: unknown flag");
    if (C == 0) return FA_OK;
    if (!offsets || !z_out || !status || (n_pts > 0 && !pts))
        return set_error(FA_ERR_INVALID_ARG, "fa_resample_arclength: null pointer");
    if (C > (int64_t)1 << 40 || n_pts > (int64_t)1 << 40)
        return set_error(FA_ERR_UNSUPPORTED, "fa_resample_arclength: size too large");
    DeviceGuard g(h->device);
    if (g.rc != FA_OK) return g.rc;
    const size_t need = resample_ws_bytes(C, n_pts, N_out, flags);
    void* ws = workspace;
    if (ws) {
        if (workspace_bytes < need)
            return set_error(FA_ERR_WORKSPACE, "fa_resample_arclength: workspace too small");
        if (reinterpret_cast<uintptr_t>(ws) & 255)
            return set_error(FA_ERR_INVALID_ARG, "fa_resample_arclength: workspace not 256-aligned");
    } else {
        const int rc = ensure_ws(h, need);
        if (rc != FA_OK) return rc;
        ws = h->ws;
    }
    return launch_resample(h, pts, offsets, C, n_pts, N_out, flags, z_out, status, ws,
                           static_cast<cudaStream_t>(stream));
}

int fa_align_pairs(fa_handle* h, const void* z1, const void* z2, int64_t P, int32_t N,
                   int32_t ztype, int32_t method, int32_t prec, int32_t* shift, double* theta,
                   double* energy, int8_t* status, void* stream)
{
    if (!h) return set_error(FA_ERR_INVALID_ARG, "fa_align_pairs: null handle");
    if (P < 0) return set_error(FA_ERR_INVALID_ARG, "fa_align_pairs: negative pair count");
    if (ztype != FA_Z_F64 && ztype != FA_Z_F32)
        return set_error(FA_ERR_INVALID_ARG, "fa_align_pairs: unknown ztype");
    if (method != FA_FFT && method != FA_DIRECT)
        return set_error(FA_ERR_INVALID_ARG, "fa_align_pairs: unknown method");
    if (prec != FA_PREC_FP64 && prec != FA_PREC_MIXED)
        return set_error(FA_ERR_INVALID_ARG, "fa_align_pairs: unknown precision");
    if (prec == FA_PREC_MIXED && method != FA_FFT)
        return set_error(FA_ERR_INVALID_ARG, "fa_align_pairs: FA_PREC_MIXED needs FA_FFT");
    int logn = -1;
    if (method == FA_FFT) {
        for (int L = kMinLogN; L <= kMaxLogN; ++L)
            if (N == (1 << L)) logn = L;
        if (logn < 0)
            return set_error(FA_ERR_UNSUPPORTED,
                             "fa_align_pairs: FA_FFT needs N a power of two in [4, 4096]");
    } else if (N < 1 || N > kMaxDirectN) {
        return set_error(FA_ERR_UNSUPPORTED, "fa_align_pairs: FA_DIRECT needs N in [1, 4096]");
    }
    if (P == 0) return FA_OK;
    if (P > (int64_t)1 << 31)
        return set_error(FA_ERR_UNSUPPORTED, "fa_align_pairs: more than 2^31 pairs");
    if (!z1 || !z2 || !shift || !theta || !energy || !status)
        return set_error(FA_ERR_INVALID_ARG, "fa_align_pairs: null pointer");
    DeviceGuard g(h->device);
    if (g.rc != FA_OK) return g.rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (method == FA_FFT && prec == FA_PREC_MIXED)
        return launch_align_df(h, z1, z2, P, logn, ztype, shift, theta, energy, status, st);
    if (method == FA_FFT)
        return launch_align_fft(h, z1, z2, P, logn, ztype, shift, theta, energy, status, st);
    return launch_align_direct(h, z1, z2, P, N, ztype, shift, theta, energy, status, st);
}

size_t fa_align_pairs_ragged_workspace_size(fa_handle* h, int64_t P, int32_t max_n)
{
    if (!h || P < 0 || max_n < 4 || max_n > kMaxRaggedN) return 0;
    DeviceGuard g(h->device);
    return ragged_ws_bytes(h, P, max_n);
}

static int ragged_check(fa_handle* h, const void* z1, const void* z2, const int64_t* offsets,
                        int64_t P, int32_t max_n, int32_t ztype, int32_t* shift, double* theta,
                        double* energy, int8_t* status, void* workspace, size_t workspace_bytes,
                        void** ws_out)
{
    if (!h) return set_error(FA_ERR_INVALID_ARG, "fa_align_pairs_ragged: null handle");
    if (P < 0 || P > ((int64_t)1 << 31) - 1)
        return set_error(FA_ERR_INVALID_ARG, "fa_align_pairs_ragged: bad pair count");
    if (max_n < 4 || max_n > kMaxRaggedN)
        return set_error(FA_ERR_UNSUPPORTED, "fa_align_pairs_ragged: max_n outside [4, 8192]");
    if (ztype != FA_Z_F64 && ztype != FA_Z_F32)
        return set_error(FA_ERR_INVALID_ARG, "fa_align_pairs_ragged: unknown ztype");
    if (P == 0) return FA_OK;
    if (!z1 || !z2 || !offsets || !shift || !theta || !energy || !status)
        return set_error(FA_ERR_INVALID_ARG, "fa_align_pairs_ragged: null pointer");
    const size_t need = ragged_ws_bytes(h, P, max_n);
    void* ws = workspace;
    if (ws) {
        if (workspace_bytes < need)
            return set_error(FA_ERR_WORKSPACE, "fa_align_pairs_ragged: workspace too small");
        if (reinterpret_cast<uintptr_t>(ws) & 255)
            return set_error(FA_ERR_INVALID_ARG, "fa_align_pairs_ragged: workspace not 256-aligned");
    } else {
        const int rc = ensure_ws(h, need);
        if (rc != FA_OK) return rc;
        ws = h->ws;
    }
    *ws_out = ws;
    return FA_OK;
}

int fa_align_pairs_ragged(fa_handle* h, const void* z1, const void* z2, const int64_t* offsets,
                          int64_t P, int32_t max_n, int32_t ztype, int32_t* shift, double* theta,
                          double* energy, int8_t* status, void* workspace, size_t workspace_bytes,
                          void* stream)
{
    if (h) {
        DeviceGuard g(h->device);
        if (g.rc != FA_OK) return g.rc;
        void* ws = nullptr;
        int rc = ragged_check(h, z1, z2, offsets, P, max_n, ztype, shift, theta, energy, status,
                              workspace, workspace_bytes, &ws);
        if (rc != FA_OK || P == 0) return rc;
        return launch_align_ragged(h, z1, z2, offsets, P, max_n, ztype, shift, theta, energy,
                                   status, ws, static_cast<cudaStream_t>(stream));
    }
    return set_error(FA_ERR_INVALID_ARG, "fa_align_pairs_ragged: null handle");
}

int fa_align_pairs_ragged_autotune(fa_handle* h, const void* z1, const void* z2,
                                   const int64_t* offsets, int64_t P, int32_t max_n,
                                   int32_t ztype, int32_t* shift, double* theta, double* energy,
                                   int8_t* status, void* workspace, size_t workspace_bytes,
                                   void* stream, int32_t* chosen_threads)
{
    if (!h) return set_error(FA_ERR_INVALID_ARG, "fa_align_pairs_ragged_autotune: null handle");
    DeviceGuard g(h->device);
    if (g.rc != FA_OK) return g.rc;
    void* ws = nullptr;
    int rc = ragged_check(h, z1, z2, offsets, P, max_n, ztype, shift, theta, energy, status,
                          workspace, workspace_bytes, &ws);
    if (rc != FA_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (P == 0) {
        if (chosen_threads) *chosen_threads = ragged_plan_threads(h->ragged_plan[ragged_max_bucket(max_n)]);
        return FA_OK;
    }
    // which buckets the batch fills
    rc = ragged_prepare(offsets, P, max_n, ws, shift, theta, energy, status, st);
    int hist[16] = {};
    if (rc == FA_OK) rc = ragged_hist(ws, hist, st);
    if (rc != FA_OK) return rc;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return cuda_error(e, "autotune: events");
    int top = -1;
    for (int b = ragged_max_bucket(max_n); b >= kMinLogN && rc == FA_OK; --b) {
        h->ragged_plan_ms[b] = 0.f;
        if (hist[b] == 0) continue;
        if (top < 0) top = b;
        // every compiled plan that fits this length: one warm-up, three timed runs
        float best_ms = -1.f;
        int best = h->ragged_plan[b];
        for (int pl = 0; pl < ragged_num_plans() && rc == FA_OK; ++pl) {
            if (!ragged_plan_fits(pl, b)) continue;
            rc = ragged_run_bucket(h, z1, z2, offsets, P, max_n, ztype, b, pl, shift, theta, energy,
                                   status, ws, true, st);
            if (rc != FA_OK) break;
            e = cudaEventRecord(e0, st);
            for (int r = 0; r < 3 && rc == FA_OK && e == cudaSuccess; ++r)
                rc = ragged_run_bucket(h, z1, z2, offsets, P, max_n, ztype, b, pl, shift, theta,
                                       energy, status, ws, true, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (rc == FA_OK && e != cudaSuccess) rc = cuda_error(e, "autotune");
            if (rc != FA_OK) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= 3.f;
            if (best_ms < 0.f || ms < best_ms) { best_ms = ms; best = pl; }
        }
        h->ragged_plan[b] = best;
        h->ragged_plan_ms[b] = best_ms > 0.f ? best_ms : 0.f;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != FA_OK) return rc;
    // leave the outputs of the chosen plans (sums run in a plan-dependent
    // order, so other plans can differ in the last bit)
    rc = launch_align_ragged(h, z1, z2, offsets, P, max_n, ztype, shift, theta, energy, status, ws, st);
    if (rc != FA_OK) return rc;
    if (chosen_threads) *chosen_threads = ragged_plan_threads(h->ragged_plan[top >= 0 ? top : ragged_max_bucket(max_n)]);
    return FA_OK;
}

int fa_align_pairs_ragged_set_plan(fa_handle* h, int32_t bucket, int32_t threads,
                                   int32_t pairs_per_cta)
{
    if (!h) return set_error(FA_ERR_INVALID_ARG, "fa_align_pairs_ragged_set_plan: null handle");
    if (bucket < kMinLogN || bucket > kMaxRaggedLogL)
        return set_error(FA_ERR_INVALID_ARG, "fa_align_pairs_ragged_set_plan: bucket outside [2, 14]");
    for (int pl = 0; pl < ragged_num_plans(); ++pl)
        if (ragged_plan_threads(pl) == threads && ragged_plan_group(pl) == pairs_per_cta) {
            if (!ragged_plan_fits(pl, bucket))
                return set_error(FA_ERR_UNSUPPORTED,
                                 "fa_align_pairs_ragged_set_plan: plan does not fit this length");
            h->ragged_plan[bucket] = pl;
            h->ragged_plan_ms[bucket] = 0.f;
            return FA_OK;
        }
    return set_error(FA_ERR_UNSUPPORTED, "fa_align_pairs_ragged_set_plan: no such compiled plan");
}

int fa_align_pairs_ragged_plan(fa_handle* h, int32_t* threads, int32_t* pairs_per_cta, float* ms)
{
    if (!h) return set_error(FA_ERR_INVALID_ARG, "fa_align_pairs_ragged_plan: null handle");
    for (int b = 0; b < 16; ++b) {
        const int pl = h->ragged_plan[b];
        if (threads) threads[b] = b >= kMinLogN && b <= kMaxRaggedLogL ? ragged_plan_threads(pl) : 0;
        if (pairs_per_cta) pairs_per_cta[b] = b >= kMinLogN && b <= kMaxRaggedLogL ? ragged_plan_group(pl) : 0;
        if (ms) ms[b] = h->ragged_plan_ms[b];
    }
    return FA_OK;
}

size_t fa_align_all_pairs_workspace_size(int64_t M, int32_t N)
{
    if (M < 0 || N <= 0) return 0;
    return align_all_ws_bytes(M, N);
}

static bool is_tc_prec(int32_t prec) { return prec >= FA_PREC_TC_BF16X3 && prec <= FA_PREC_TC_TF32X3; }

size_t fa_align_all_pairs_workspace_size_prec(int64_t M, int32_t N, int32_t prec)
{
    if (M < 0 || M > (1 << 16) || N <= 0) return 0;
    if (prec == FA_PREC_FP64 || prec == FA_PREC_MIXED) return align_all_ws_bytes(M, N);
    if (!is_tc_prec(prec) || (N != 256 && N != 512)) return 0;
    return align_all_tc_ws_bytes(M, N == 256 ? 8 : 9, prec);
}

int fa_align_all_pairs(fa_handle* h, const void* z, int64_t M, int32_t N, int32_t ztype,
                       int32_t prec, int32_t* shift, double* theta, double* energy,
                       int8_t* status, void* workspace, size_t workspace_bytes, void* stream)
{
    if (!h) return set_error(FA_ERR_INVALID_ARG, "fa_align_all_pairs: null handle");
    if (M < 0) return set_error(FA_ERR_INVALID_ARG, "fa_align_all_pairs: negative curve count");
    if (ztype != FA_Z_F64 && ztype != FA_Z_F32)
        return set_error(FA_ERR_INVALID_ARG, "fa_align_all_pairs: unknown ztype");
    if (prec != FA_PREC_FP64 && prec != FA_PREC_MIXED && !is_tc_prec(prec))
        return set_error(FA_ERR_INVALID_ARG, "fa_align_all_pairs: unknown precision");
    int logn = -1;
    for (int L = kMinLogN; L <= kMaxLogN; ++L)
        if (N == (1 << L)) logn = L;
    if (logn < 0)
        return set_error(FA_ERR_UNSUPPORTED,
                         "fa_align_all_pairs: N must be a power of two in [4, 4096]");
    if (is_tc_prec(prec) && N != 256 && N != 512)
        return set_error(FA_ERR_UNSUPPORTED,
                         "fa_align_all_pairs: the tensor-core search needs N = 256 or 512");
    if (M == 0) return FA_OK;
    if (M > (1 << 16))
        return set_error(FA_ERR_UNSUPPORTED, "fa_align_all_pairs: more than 65536 curves");
    if (!z || !shift || !theta || !energy || !status)
        return set_error(FA_ERR_INVALID_ARG, "fa_align_all_pairs: null pointer");
    const size_t need = is_tc_prec(prec) ? align_all_tc_ws_bytes(M, logn, prec)
                                         : align_all_ws_bytes(M, N);
    DeviceGuard g(h->device);
    if (g.rc != FA_OK) return g.rc;
    void* ws = workspace;
    if (ws) {
        if (workspace_bytes < need)
            return set_error(FA_ERR_WORKSPACE, "fa_align_all_pairs: workspace too small");
        if (reinterpret_cast<uintptr_t>(ws) & 255)
            return set_error(FA_ERR_INVALID_ARG, "fa_align_all_pairs: workspace not 256-aligned");
    } else {
        const int rc = ensure_ws(h, need);
        if (rc != FA_OK) return rc;
        ws = h->ws;
    }
    if (prec == FA_PREC_MIXED)
        return launch_align_all_df(h, z, M, logn, ztype, ws, status, shift, theta, energy,
                                   static_cast<cudaStream_t>(stream));
    if (is_tc_prec(prec))
        return launch_align_all_tc(h, z, M, logn, ztype, prec, ws, status, shift, theta, energy,
                                   static_cast<cudaStream_t>(stream));
    return launch_align_all(h, z, M, logn, ztype, ws, status, shift, theta, energy,
                            static_cast<cudaStream_t>(stream));
}

size_t fa_elastic_workspace_size(fa_handle* h, int64_t M1, int64_t M2, int64_t P, int32_t N,
                                  int32_t band)
{
    if (!h || M1 < 0 || M2 < 0 || P < 0 || N < kMinElasticN || N > kMaxElasticN || (N & (N - 1)))
        return 0;
    return elastic_ws_bytes(h, M1, M2, P, N, band);
}

int fa_elastic_distance(fa_handle* h, const double* curves1, int64_t M1, const double* curves2,
                        int64_t M2, int32_t N, const int64_t* idx1, const int64_t* idx2,
                        int64_t P, int32_t band, int32_t max_iter, int32_t* shift,
                        double* theta, double* energy, double* gamma, int32_t* iters,
                        int32_t* lm_steps, int8_t* status, void* workspace,
                        size_t workspace_bytes, void* stream)
{
    if (!h) return set_error(FA_ERR_INVALID_ARG, "fa_elastic_distance: null handle");
    if (M1 < 0 || M2 < 0 || P < 0)
        return set_error(FA_ERR_INVALID_ARG, "fa_elastic_distance: negative size");
    if (N < kMinElasticN || N > kMaxElasticN || (N & (N - 1)))
        return set_error(FA_ERR_UNSUPPORTED,
                         "fa_elastic_distance: N must be a power of two in [32, 1024]");
    if (max_iter < 0 || max_iter > 1000)
        return set_error(FA_ERR_INVALID_ARG, "fa_elastic_distance: max_iter outside [0, 1000]");
    if (band < -1) return set_error(FA_ERR_INVALID_ARG, "fa_elastic_distance: band < -1");
    if ((!idx1 && M1 < P) || (!idx2 && M2 < P))
        return set_error(FA_ERR_INVALID_ARG,
                         "fa_elastic_distance: without index arrays each set needs P curves");
    if (M1 > ((int64_t)1 << 32) || M2 > ((int64_t)1 << 32) || P > ((int64_t)1 << 40))
        return set_error(FA_ERR_UNSUPPORTED, "fa_elastic_distance: size too large");
    if (P == 0) return FA_OK;
    if (!curves1 || !curves2 || !shift || !theta || !energy || !status || M1 == 0 || M2 == 0)
        return set_error(FA_ERR_INVALID_ARG, "fa_elastic_distance: null pointer or empty set");
    DeviceGuard g(h->device);
    if (g.rc != FA_OK) return g.rc;
    const size_t need = elastic_ws_bytes(h, M1, M2, P, N, band);
    void* ws = workspace;
    if (ws) {
        if (workspace_bytes < need)
            return set_error(FA_ERR_WORKSPACE, "fa_elastic_distance: workspace too small");
        if (reinterpret_cast<uintptr_t>(ws) & 255)
            return set_error(FA_ERR_INVALID_ARG, "fa_elastic_distance: workspace not 256-aligned");
    } else {
        const int rc = ensure_ws(h, need);
        if (rc != FA_OK) return rc;
        ws = h->ws;
    }
    return launch_elastic(h, curves1, M1, curves2, M2, N, idx1, idx2, P, band, max_iter, shift,
                          theta, energy, gamma, iters, lm_steps, status, ws,
                          static_cast<cudaStream_t>(stream));
}

}  // extern "C"

extern "C" int fa_align_curves_host(fa_handle* h, const double* pts, const int64_t* offsets,
                                    int64_t P, int32_t N, int32_t flags, int32_t method,
                                    int32_t prec, int32_t* shift, double* theta, double* energy,
                                    int8_t* status, void* stream)
{
    if (!h) return set_error(FA_ERR_INVALID_ARG, "fa_align_curves_host: null handle");
    if (P < 0) return set_error(FA_ERR_INVALID_ARG, "fa_align_curves_host: negative pair count");
    if (flags & ~FA_STORE_FP32)
        return set_error(FA_ERR_INVALID_ARG, "fa_align_curves_host: unknown flag");
    if (P == 0) return FA_OK;
    if (!pts && offsets && offsets[2 * P] > 0)
        return set_error(FA_ERR_INVALID_ARG, "fa_align_curves_host: null pointer");
    if (!offsets || !shift || !theta || !energy || !status)
        return set_error(FA_ERR_INVALID_ARG, "fa_align_curves_host: null pointer");
    const int64_t C = 2 * P;
    if (offsets[0] != 0)
        return set_error(FA_ERR_INVALID_ARG, "fa_align_curves_host: offsets[0] must be 0");
    for (int64_t i = 0; i < C; ++i)
        if (offsets[i + 1] < offsets[i])
            return set_error(FA_ERR_INVALID_ARG, "fa_align_curves_host: decreasing offsets");
    const int64_t n_pts = offsets[C];
    if (C > (int64_t)1 << 40 || n_pts > (int64_t)1 << 40)
        return set_error(FA_ERR_UNSUPPORTED, "fa_align_curves_host: size too large");
    const int ztype = (flags & FA_STORE_FP32) ? FA_Z_F32 : FA_Z_F64;
    const size_t zb = (flags & FA_STORE_FP32) ? sizeof(float2) : sizeof(double2);
    auto a256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const int rflags = FA_CENTER | FA_UNIT_LENGTH | (flags & FA_STORE_FP32);
    const size_t b_off = a256((size_t)(C + 1) * sizeof(int64_t));
    const size_t b_pts = a256((size_t)n_pts * sizeof(double2));
    const size_t b_z = a256((size_t)C * (size_t)N * zb);
    const size_t b_rst = a256((size_t)C);
    const size_t b_sh = a256((size_t)P * sizeof(int32_t));
    const size_t b_th = a256((size_t)P * sizeof(double));
    const size_t b_st = a256((size_t)P);
    const size_t b_ws = a256(resample_ws_bytes(C, n_pts, N, rflags));
    const size_t b_cnt = 256;  // the resampling launches' work counters
    if (N < 4 || N > (1 << 20))
        return set_error(FA_ERR_UNSUPPORTED, "fa_align_curves_host: N outside [4, 2^20]");
    DeviceGuard g(h->device);
    if (g.rc != FA_OK) return g.rc;
    int rc = ensure_ws(h, b_off + b_pts + b_z + b_rst + b_sh + 2 * b_th + b_st + b_cnt + b_ws);
    if (rc != FA_OK) return rc;
    char* w = static_cast<char*>(h->ws);
    int64_t* d_off = reinterpret_cast<int64_t*>(w); w += b_off;
    double* d_pts = reinterpret_cast<double*>(w); w += b_pts;
    char* d_z = w; w += b_z;
    int8_t* d_rst = reinterpret_cast<int8_t*>(w); w += b_rst;
    int32_t* d_sh = reinterpret_cast<int32_t*>(w); w += b_sh;
    double* d_th = reinterpret_cast<double*>(w); w += b_th;
    double* d_en = reinterpret_cast<double*>(w); w += b_th;
    int8_t* d_st = reinterpret_cast<int8_t*>(w); w += b_st;
    unsigned long long* d_cnt = reinterpret_cast<unsigned long long*>(w); w += b_cnt;
    void* d_ws = w;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // Pipeline: the pairs in up to four chunks, each on its own stream (upload
    // of its curves, resampling, alignment, download), so that the copy engine
    // uploads chunk k+1 while the SMs work on chunk k.  The chunks touch
    // disjoint parts of every buffer, the resampling workspace included (it is
    // addressed by absolute node index); each launch has its own counter.
    const int nchunk = P >= 2048 ? 4 : (P >= 1024 ? 2 : 1);
    if (nchunk > 1 && !h->pipe[0]) {
        for (int k = 0; k < 4; ++k) {
            cudaError_t e1 = cudaStreamCreateWithFlags(&h->pipe[k], cudaStreamNonBlocking);
            if (e1 != cudaSuccess) return cuda_error(e1, "fa_align_curves_host: stream");
        }
        for (int k = 0; k < 5; ++k) {
            cudaError_t e1 = cudaEventCreateWithFlags(&h->pipe_ev[k], cudaEventDisableTiming);
            if (e1 != cudaSuccess) return cuda_error(e1, "fa_align_curves_host: event");
        }
    }
    cudaError_t e = cudaMemcpyAsync(d_off, offsets, (size_t)(C + 1) * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nchunk > 1) e = cudaEventRecord(h->pipe_ev[4], st);
    if (e != cudaSuccess) return cuda_error(e, "fa_align_curves_host: upload");
    const size_t zrow = (size_t)N * zb;
    for (int k = 0; k < nchunk; ++k) {
        const int64_t a = P * k / nchunk, b = P * (k + 1) / nchunk, m = b - a;
        cudaStream_t cs = nchunk > 1 ? h->pipe[k] : st;
        if (nchunk > 1) {
            e = cudaStreamWaitEvent(cs, h->pipe_ev[4], 0);
            if (e != cudaSuccess) return cuda_error(e, "fa_align_curves_host: wait");
        }
        // this chunk's curves: [a, b) and [P + a, P + b)
        for (int half = 0; half < 2; ++half) {
            const int64_t c0 = half * P + a, c1 = half * P + b;
            const int64_t o0 = offsets[c0], o1 = offsets[c1];
            if (o1 > o0) {
                e = cudaMemcpyAsync(d_pts + 2 * o0, pts + 2 * o0, (size_t)(o1 - o0) * sizeof(double2),
                                    cudaMemcpyHostToDevice, cs);
                if (e != cudaSuccess) return cuda_error(e, "fa_align_curves_host: upload");
            }
            rc = launch_resample(h, d_pts, d_off + c0, m, n_pts, N, rflags, d_z + (size_t)c0 * zrow,
                                 d_rst + c0, d_ws, cs, d_cnt + 2 * k + half, c0);
            if (rc != FA_OK) return rc;
        }
        rc = fa_align_pairs(h, d_z + (size_t)a * zrow, d_z + (size_t)(P + a) * zrow, m, N, ztype,
                            method, prec, d_sh + a, d_th + a, d_en + a, d_st + a, cs);
        if (rc != FA_OK) return rc;
        merge_status_kernel<<<(unsigned)((m + 255) / 256), 256, 0, cs>>>(
            d_rst + a, m, P, d_sh + a, d_th + a, d_en + a, d_st + a);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(shift + a, d_sh + a, (size_t)m * sizeof(int32_t), cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(theta + a, d_th + a, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(energy + a, d_en + a, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(status + a, d_st + a, (size_t)m, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess && nchunk > 1) e = cudaEventRecord(h->pipe_ev[k], cs);
        if (e == cudaSuccess && nchunk > 1) e = cudaStreamWaitEvent(st, h->pipe_ev[k], 0);
        if (e != cudaSuccess) return cuda_error(e, "fa_align_curves_host");
    }
    e = cudaStreamSynchronize(st);
    return cuda_error(e, "fa_align_curves_host");
}
