// Continuous-batching server for gradient queries (see gradsim.h).
#include "gs_runtime.h"

using namespace gs;

extern "C" gs_status gs_server_create(gs_ctx*, const gs_server_opts*, gs_server** out) {
    if (out) *out = nullptr;
    return set_error(GS_EUNSUPPORTED, "server not built yet");
}
extern "C" void gs_server_destroy(gs_server*) {}
extern "C" gs_status gs_query_submit(gs_server*, const gs_query*, uint64_t*) { return set_error(GS_EUNSUPPORTED, "server"); }
extern "C" gs_status gs_query_poll(gs_server*, uint64_t, gs_result*, int) { return set_error(GS_EUNSUPPORTED, "server"); }
extern "C" gs_status gs_query_cancel(gs_server*, uint64_t) { return set_error(GS_EUNSUPPORTED, "server"); }
extern "C" gs_status gs_server_stats_get(gs_server*, gs_server_stats*) { return set_error(GS_EUNSUPPORTED, "server"); }
extern "C" void gs_result_free(gs_result*) {}
