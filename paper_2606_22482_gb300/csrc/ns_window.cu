// ns_window.cu -- the window pass of the planner (row/column extraction, windows, compaction,
// density binning, residual CSR).
#include "ns_internal.cuh"

namespace ns {

ns_status_t window_pass(Plan* P, WindowResult* W, cudaStream_t s)
{
    set_error("dense tiles are not available in this build");
    return NS_ERR_UNSUPPORTED;
}

}  // namespace ns
