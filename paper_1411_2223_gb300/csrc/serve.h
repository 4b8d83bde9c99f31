// Continuous-batching serving engine (host scheduler thread).
#pragma once

struct sq_ctx;

namespace sq {

struct ServeEngine;
void serve_shutdown(ServeEngine *e);
bool serve_uses_gauge(ServeEngine *e, int gauge_id);

}  // namespace sq
