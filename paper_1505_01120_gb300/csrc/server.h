// server.h -- continuous-batching server state (filled in by server.cu).
#pragma once

#include "runtime.h"

namespace scl {

struct Server {
    virtual ~Server() = default;
};

}  // namespace scl
