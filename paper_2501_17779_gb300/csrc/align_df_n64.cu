// align_df_n64.cu -- FA_PREC_MIXED kernels for N = 64 (one translation unit per
// size range; the kernels are in align_df_impl.cuh).
#include "align_df_impl.cuh"

namespace fa {

int align_df_pairs_6(const fa_handle* h, const void* z1, const void* z2, int64_t P, int logn, int ztype,
                      int32_t* shift, double* theta, double* energy, int8_t* status, cudaStream_t st)
{
    const bool f64 = ztype == FA_Z_F64;
    switch (logn) {
        FA_DF_PAIRS_CASE(6)
    }
    return FA_ERR_UNSUPPORTED;
}

int align_df_all_6(const fa_handle* h, const void* z, int64_t M, int logn, int ztype, float4* spec,
                    int8_t* status, int32_t* shift, double* theta, double* energy, cudaStream_t st)
{
    const bool f64 = ztype == FA_Z_F64;
    switch (logn) {
        FA_DF_ALL_CASE(6)
    }
    return FA_ERR_UNSUPPORTED;
}

}  // namespace fa
