// Continuous-batching request server (placeholder until the serving loop lands).
#include "api_internal.hpp"

using namespace rsaprng;

extern "C" {

int rsaprng_server_create(rsaprng_ctx *, uint64_t, int, rsaprng_server **out)
{
    if (out)
        *out = nullptr;
    return fail(RSAPRNG_ERR_ARG, "server not built yet");
}
int rsaprng_server_submit(rsaprng_server *, rsaprng_id, uint64_t, uint64_t *) { return RSAPRNG_ERR_ARG; }
int rsaprng_server_poll(rsaprng_server *, uint64_t, int *) { return RSAPRNG_ERR_ARG; }
int rsaprng_server_wait(rsaprng_server *, uint64_t, uint64_t) { return RSAPRNG_ERR_ARG; }
int rsaprng_server_result(rsaprng_server *, uint64_t, const double **, uint64_t *) { return RSAPRNG_ERR_ARG; }
int rsaprng_server_copy(rsaprng_server *, uint64_t, double *, void *) { return RSAPRNG_ERR_ARG; }
int rsaprng_server_release(rsaprng_server *, uint64_t) { return RSAPRNG_ERR_ARG; }
int rsaprng_server_cancel(rsaprng_server *, uint64_t) { return RSAPRNG_ERR_ARG; }
int rsaprng_server_stats(rsaprng_server *, rsaprng_stats *) { return RSAPRNG_ERR_ARG; }
void rsaprng_server_destroy(rsaprng_server *) {}

}
