// Serving loop: placeholder entry points until the continuous-batching scheduler lands.
#include "lnr_internal.h"

namespace lnr {
struct Server {};
}  // namespace lnr

using namespace lnr;

extern "C" {

lnr_status lnr_serve_start(lnr_ctx* c, int, int) { return c ? fail(c, LNR_E_STATE, "serving not built") : LNR_E_ARG; }
lnr_status lnr_serve_stop(lnr_ctx* c) { return c ? LNR_OK : LNR_E_ARG; }
lnr_status lnr_set_memory_budget(lnr_ctx* c, size_t bytes) {
    if (!c) return LNR_E_ARG;
    c->mem_budget = bytes;
    return LNR_OK;
}
lnr_status lnr_submit(lnr_ctx* c, const lnr_view*, const lnr_intrinsics*, int, int, int, float, uint64_t*) {
    return c ? fail(c, LNR_E_STATE, "serving not started") : LNR_E_ARG;
}
lnr_status lnr_poll(lnr_ctx* c, uint64_t, float*, double*) { return c ? fail(c, LNR_E_STATE, "serving not started") : LNR_E_ARG; }
lnr_status lnr_serve_stats(lnr_ctx* c, uint64_t out[4]) {
    if (!c || !out) return LNR_E_ARG;
    for (int i = 0; i < 4; ++i) out[i] = 0;
    return LNR_OK;
}

}  // extern "C"
