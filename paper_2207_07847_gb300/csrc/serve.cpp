// Serving: continuous batching of solve requests.
#include <cstring>

#include "lap.h"

extern "C" {
void lap_server_options_default(lap_server_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->hbm_budget_bytes = int64_t(8) << 30;
    o->max_slots = 256;
    o->check_every = 8;
}
lap_status lap_server_create(const lap_server_options *, lap_server *out)
{
    if (out) *out = nullptr;
    return LAP_ERR_UNSUPPORTED;
}
lap_status lap_serve_submit(lap_server, lap_handle, int32_t, const double *, double *, lap_done_cb,
                            void *, uint64_t *)
{
    return LAP_ERR_UNSUPPORTED;
}
lap_status lap_serve_wait(lap_server, uint64_t, double, lap_solve_info *) { return LAP_ERR_UNSUPPORTED; }
lap_status lap_serve_cancel(lap_server, uint64_t) { return LAP_ERR_UNSUPPORTED; }
void lap_server_destroy(lap_server) {}
}
