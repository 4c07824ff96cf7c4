// Serving runtime: placeholder entry points until the continuous-batching
// server is in place.
#include "host_common.h"

using namespace air;

extern "C" air_status air_server_create(size_t, int, air_server **out) {
    if (out) *out = nullptr;
    return fail(AIR_ERR_INVALID_ARG, "the server is not available in this build");
}
extern "C" air_status air_server_submit(air_server *, const air_geometry *, const float *, float, float, int,
                                        int, uint64_t *) {
    return fail(AIR_ERR_INVALID_ARG, "the server is not available in this build");
}
extern "C" air_status air_server_poll(air_server *, uint64_t, float *) {
    return fail(AIR_ERR_INVALID_ARG, "the server is not available in this build");
}
extern "C" air_status air_server_wait(air_server *, uint64_t, float *) {
    return fail(AIR_ERR_INVALID_ARG, "the server is not available in this build");
}
extern "C" air_status air_server_times(air_server *, uint64_t, double *) {
    return fail(AIR_ERR_INVALID_ARG, "the server is not available in this build");
}
extern "C" air_status air_server_destroy(air_server *) { return AIR_OK; }
