// ns_dense.cuh -- dense-tile (tensor-core) work item of the persistent kernel.
#pragma once
#include "ns_internal.cuh"

namespace ns {

template <bool BF16, bool HINT>
__device__ void dense_item(const ExecDesc& D, int32_t d, unsigned char* smem, uint64_t pol_first,
                           uint64_t pol_last)
{
}

inline size_t dense_smem_bytes(int K, int TM, int TK, bool bf16) { return 0; }
inline ns_status_t dense_prepare(const void* kern, size_t smem) { return NS_OK; }

}  // namespace ns
