// server.cu -- continuous-batching server over the persistent batch launch.
#include "server.h"

using namespace scl;

extern "C" int scl_server_stop(scl_ctx* ctx) {
    if (!ctx) return SCL_OK;
    ctx->server.reset();
    return SCL_OK;
}
