// Serving engine: placeholder until the scheduler lands.
#include "serve.h"
#include "sq_host.h"

namespace sq {

struct ServeEngine {};
void serve_shutdown(ServeEngine *e) { delete e; }
bool serve_uses_gauge(ServeEngine *, int) { return false; }

}  // namespace sq

extern "C" int serve_submit(sq_ctx *, int, const double *, double, double, uint64_t *) {
  return SQ_ERR_UNSUPPORTED;
}
extern "C" int serve_poll(sq_ctx *, uint64_t, double *, sq_cg_stats *, int) {
  return SQ_ERR_UNSUPPORTED;
}
extern "C" int serve_cancel(sq_ctx *, uint64_t) { return SQ_ERR_UNSUPPORTED; }
extern "C" int serve_stats(sq_ctx *, sq_serve_stats *, int) { return SQ_ERR_UNSUPPORTED; }
extern "C" int serve_configure(sq_ctx *, int, int) { return SQ_ERR_UNSUPPORTED; }
