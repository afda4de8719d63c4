// ns_pending.cu -- entry points whose implementation is not in this build yet.  Each returns
// NS_ERR_UNSUPPORTED with a message; none launches a kernel.
#include "ns_internal.cuh"

using namespace ns;

extern "C" {
ns_status_t ns_serve_create(const ns_serve_cfg_t*, ns_server_t* out)
{
    if (out) *out = nullptr;
    set_error("serving not built yet");
    return NS_ERR_UNSUPPORTED;
}
ns_status_t ns_serve_register_graph(ns_server_t, const ns_csr_t*, int32_t*)
{
    set_error("serving not built yet");
    return NS_ERR_UNSUPPORTED;
}
ns_status_t ns_serve_submit(ns_server_t, const ns_request_t*, uint64_t*)
{
    set_error("serving not built yet");
    return NS_ERR_UNSUPPORTED;
}
ns_status_t ns_serve_poll(ns_server_t, uint64_t, int*, ns_req_stats_t*)
{
    set_error("serving not built yet");
    return NS_ERR_UNSUPPORTED;
}
double ns_serve_now(void) { return 0.0; }
ns_status_t ns_serve_destroy(ns_server_t) { return NS_OK; }
}
