// noalloc.cu -- fa_resample_arclength_noalloc: arc-length resampling that
// allocates no device memory at all.
//
// Some callers cannot call cudaMalloc: host applications that reserve the
// whole device memory budget up front and forbid libraries from allocating
// on their own, and latency-critical loops in which the implicit device
// synchronisation of an allocation is unacceptable.  Such callers also cannot
// create a handle (fa_create allocates twiddle tables), so this entry point
// takes none.  Its per-node scratch lives in the fixed file-scope array below,
// which every GPU that loads the library holds until the process exits.
//
// The array's name is only a host-side stand-in in host code, not a device
// address: the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and handed to the kernel.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "fa_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FA_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on `dev` (the current device).
int scratch_address(int dev, void** out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return fa::cuda_error(e, "fa_resample_arclength_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return FA_OK;
}

}  // namespace

extern "C" int fa_resample_arclength_noalloc(const double* pts, const int64_t* offsets,
                                             int64_t C, int64_t n_pts, int32_t N_out,
                                             int32_t flags, void* z_out, int8_t* status,
                                             void* stream)
{
    using fa::set_error;
    if (C < 0 || n_pts < 0)
        return set_error(FA_ERR_INVALID_ARG, "fa_resample_arclength_noalloc: negative size");
    if (N_out < 4 || N_out > (1 << 20))
        return set_error(FA_ERR_UNSUPPORTED,
                         "fa_resample_arclength_noalloc: N_out outside [4, 2^20]");
    if (flags & ~(FA_CENTER | FA_UNIT_LENGTH | FA_STORE_FP32))
        return set_error(FA_ERR_INVALID_ARG, "fa_resample_arclength_noalloc: unknown flag");
    if (C == 0) return FA_OK;
    if (!offsets || !z_out || !status || (n_pts > 0 && !pts))
        return set_error(FA_ERR_INVALID_ARG, "fa_resample_arclength_noalloc: null pointer");
    if (C > (int64_t)1 << 40 || n_pts > (int64_t)1 << 40)
        return set_error(FA_ERR_UNSUPPORTED, "fa_resample_arclength_noalloc: size too large");
    const size_t need = fa::resample_ws_bytes(C, n_pts, N_out, flags);
    if (need > (size_t)FA_NOALLOC_SCRATCH_BYTES)
        return set_error(FA_ERR_UNSUPPORTED,
                         "fa_resample_arclength_noalloc: this batch needs " + std::to_string(need) +
                             " bytes of scratch but the fixed buffer holds " +
                             std::to_string((size_t)FA_NOALLOC_SCRATCH_BYTES) +
                             " bytes; split it into smaller batches");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fa::cuda_error(e, "fa_resample_arclength_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(FA_ERR_UNSUPPORTED, "fa_resample_arclength_noalloc: device ordinal too large");
    void* ws = nullptr;
    const int rc = scratch_address(dev, &ws);
    if (rc != FA_OK) return rc;
    return fa::launch_resample(nullptr, pts, offsets, C, n_pts, N_out, flags, z_out, status, ws,
                               static_cast<cudaStream_t>(stream));
}
