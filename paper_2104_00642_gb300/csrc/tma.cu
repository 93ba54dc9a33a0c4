// tma.cu -- host side of the TMA copies: tensor maps of the field array.
#include <cstdint>

#include "tma.cuh"

namespace pic {

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn()
{
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

}  // namespace

bool tma_encode_field_map(CUtensorMap *map, const float *base, int ext0, int ext1, long long pitch, long long vol,
                          int ncomp, const int *box)
{
    EncodeTiled fn = encode_fn();
    if (!fn) return false;
    // the copy engine's rules: 16-byte aligned base and strides, a tile row of
    // a multiple of 16 bytes, at most 256 elements per tile dimension
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (pitch * 4) % 16 || (vol * 4) % 16 || (box[0] * 4) % 16)
        return false;
    for (int d = 0; d < 3; d++)
        if (box[d] < 1 || box[d] > 256) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)ext0, (cuuint64_t)ext1, (cuuint64_t)ncomp};
    const cuuint64_t strides[2] = {(cuuint64_t)(pitch * 4), (cuuint64_t)(vol * 4)};
    const cuuint32_t bdim[3] = {(cuuint32_t)box[0], (cuuint32_t)box[1], (cuuint32_t)box[2]};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, bdim, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tma_encode_field_map3(CUtensorMap *map, const float *base, const int *ext, long long sy, long long sz,
                           long long vol, int ncomp, const int *box)
{
    EncodeTiled fn = encode_fn();
    if (!fn) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (sy * 4) % 16 || (sz * 4) % 16 || (vol * 4) % 16 ||
        (box[0] * 4) % 16)
        return false;
    for (int d = 0; d < 4; d++)
        if (box[d] < 1 || box[d] > 256) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)ext[0], (cuuint64_t)ext[1], (cuuint64_t)ext[2], (cuuint64_t)ncomp};
    const cuuint64_t strides[3] = {(cuuint64_t)(sy * 4), (cuuint64_t)(sz * 4), (cuuint64_t)(vol * 4)};
    const cuuint32_t bdim[4] = {(cuuint32_t)box[0], (cuuint32_t)box[1], (cuuint32_t)box[2], (cuuint32_t)box[3]};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(base), dims, strides, bdim, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace pic
