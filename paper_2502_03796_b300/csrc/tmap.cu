// tmap.cu - TMA tensor map over a packed trace buffer.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "magus_internal.h"

namespace magus {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// The packed buffer as a [rows][32] uint32 tensor; a copy moves box_rows x 32 deltas into
// shared memory with the 128-byte swizzle (chunk c of row R at position c ^ (R & 7)).
// Rows past the end of the buffer read as zeros.
int make_trace_tmap(const uint32_t *traces, uint64_t total_elems, int box_rows, CUtensorMap *out,
                    std::string *err) {
    auto fn = encode_fn();
    if (!fn) {
        *err = "cuTensorMapEncodeTiled is not available from the driver";
        return MAGUS_ECUDA;
    }
    const uint64_t rows = total_elems / kTraceAlign > 0 ? total_elems / kTraceAlign : 1;
    cuuint64_t dims[2] = {(cuuint64_t)kTraceAlign, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kTraceAlign * sizeof(uint32_t)};
    cuuint32_t box[2] = {(cuuint32_t)kTraceAlign, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, (void *)traces, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
        return MAGUS_ECUDA;
    }
    return MAGUS_OK;
}

}  // namespace magus
