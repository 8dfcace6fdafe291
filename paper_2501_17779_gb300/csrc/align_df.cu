// align_df.cu -- FA_PREC_MIXED entry: dispatch by transform size to the
// translation units that instantiate the double-float kernels.
#include "fa_internal.cuh"

namespace fa {

#define FA_DF_PAIRS_ARGS                                                                      \
    const fa_handle *h, const void *z1, const void *z2, int64_t P, int logn, int ztype,      \
        int32_t *shift, double *theta, double *energy, int8_t *status, cudaStream_t st
#define FA_DF_ALL_ARGS                                                                        \
    const fa_handle *h, const void *z, int64_t M, int logn, int ztype, float4 *spec,         \
        int8_t *status, int32_t *shift, double *theta, double *energy, cudaStream_t st
int align_df_pairs_2_5(FA_DF_PAIRS_ARGS);
int align_df_pairs_6(FA_DF_PAIRS_ARGS);
int align_df_pairs_7(FA_DF_PAIRS_ARGS);
int align_df_pairs_8(FA_DF_PAIRS_ARGS);
int align_df_pairs_9(FA_DF_PAIRS_ARGS);
int align_df_pairs_10(FA_DF_PAIRS_ARGS);
int align_df_pairs_11(FA_DF_PAIRS_ARGS);
int align_df_pairs_12(FA_DF_PAIRS_ARGS);
int align_df_all_2_5(FA_DF_ALL_ARGS);
int align_df_all_6(FA_DF_ALL_ARGS);
int align_df_all_7(FA_DF_ALL_ARGS);
int align_df_all_8(FA_DF_ALL_ARGS);
int align_df_all_9(FA_DF_ALL_ARGS);
int align_df_all_10(FA_DF_ALL_ARGS);
int align_df_all_11(FA_DF_ALL_ARGS);
int align_df_all_12(FA_DF_ALL_ARGS);
#undef FA_DF_PAIRS_ARGS
#undef FA_DF_ALL_ARGS
#define FA_DF_PAIRS_SIG                                                                       \
    const fa_handle*, const void*, const void*, int64_t, int, int, int32_t*, double*,       \
        double*, int8_t*, cudaStream_t
#define FA_DF_ALL_SIG                                                                         \
    const fa_handle*, const void*, int64_t, int, int, float4*, int8_t*, int32_t*, double*,  \
        double*, cudaStream_t

int launch_align_df(const fa_handle* h, const void* z1, const void* z2, int64_t P, int logn,
                    int ztype, int32_t* shift, double* theta, double* energy, int8_t* status,
                    cudaStream_t st)
{
    if (P == 0) return FA_OK;
    static int (*const part[])(FA_DF_PAIRS_SIG) = {
        align_df_pairs_6, align_df_pairs_7, align_df_pairs_8, align_df_pairs_9,
        align_df_pairs_10, align_df_pairs_11, align_df_pairs_12};
    auto f = logn <= 5 ? align_df_pairs_2_5 : part[logn < 6 ? 0 : logn > 12 ? 6 : logn - 6];
    const int rc = f(h, z1, z2, P, logn, ztype, shift, theta, energy, status, st);
    if (rc == FA_ERR_UNSUPPORTED) return set_error(FA_ERR_UNSUPPORTED, "align_df: unsupported N");
    return rc;
}

int launch_align_all_df(const fa_handle* h, const void* z, int64_t M, int logn, int ztype,
                        void* ws, int8_t* status, int32_t* shift, double* theta, double* energy,
                        cudaStream_t st)
{
    if (M == 0) return FA_OK;
    float4* spec = static_cast<float4*>(ws);
    static int (*const part[])(FA_DF_ALL_SIG) = {
        align_df_all_6, align_df_all_7, align_df_all_8, align_df_all_9,
        align_df_all_10, align_df_all_11, align_df_all_12};
    auto f = logn <= 5 ? align_df_all_2_5 : part[logn < 6 ? 0 : logn > 12 ? 6 : logn - 6];
    const int rc = f(h, z, M, logn, ztype, spec, status, shift, theta, energy, st);
    if (rc == FA_ERR_UNSUPPORTED)
        return set_error(FA_ERR_UNSUPPORTED, "align_all_pairs: unsupported N");
    return rc;
}

}  // namespace fa
