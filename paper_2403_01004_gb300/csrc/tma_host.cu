// Host-side tensor-map encoding for the TMA march kernels.  cuTensorMapEncodeTiled is taken from
// the driver through the runtime's entry-point query, so the library does not link libcuda.
#include <cudaTypedefs.h>

#include <mutex>

#include "tma.cuh"

namespace pb {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_once;

void resolve() {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    else
        cudaGetLastError();
}

CUtensorMapDataType dtype_of(int elem_bytes) {
    switch (elem_bytes) {
        case 8: return CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
        case 4: return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
        default: return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    }
}

}  // namespace

bool tma_available() {
    std::call_once(g_once, resolve);
    return g_encode != nullptr;
}

bool tma_state_map(CUtensorMap* m, const void* base, int elem, int nr, int nt, int np, int box_x, int box_y) {
    if (!tma_available()) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
    if (((long long)nr * elem) % 16 != 0) return false;
    if ((box_x * elem) % 16 != 0 || box_x > 256 || box_y > 256) return false;
    cuuint64_t dims[3] = {(cuuint64_t)nr, (cuuint64_t)nt, (cuuint64_t)np};
    cuuint64_t strides[2] = {(cuuint64_t)nr * elem, (cuuint64_t)nr * nt * elem};
    cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(m, dtype_of(elem), 3, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool tma_coef_map(CUtensorMap* m, const void* base, int elem, int nr, int nt, int np, int box_x, int box_y) {
    if (!tma_available()) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
    if (box_x > 256 || box_y > 256) return false;
    if (elem == 2) {
        // one 8-byte element per 4-word bfloat16 record (a raw copy: the type only sets the size)
        if (((long long)nr * 8) % 16 != 0 || (box_x * 8) % 16 != 0) return false;
        cuuint64_t d3[3] = {(cuuint64_t)nr, (cuuint64_t)nt, (cuuint64_t)np};
        cuuint64_t s3[2] = {(cuuint64_t)8 * nr, (cuuint64_t)8 * nr * nt};
        cuuint32_t b3[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
        cuuint32_t e3[3] = {1, 1, 1};
        return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void*>(base), d3, s3, b3, e3,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    cuuint64_t dims[4] = {4, (cuuint64_t)nr, (cuuint64_t)nt, (cuuint64_t)np};
    cuuint64_t strides[3] = {(cuuint64_t)4 * elem, (cuuint64_t)4 * elem * nr, (cuuint64_t)4 * elem * nr * nt};
    cuuint32_t box[4] = {4, (cuuint32_t)box_x, (cuuint32_t)box_y, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = g_encode(m, elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                          const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace pb
