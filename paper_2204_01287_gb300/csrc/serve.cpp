// serve.cpp — serving loop (pc_submit / pc_poll).
#include "pc_api_internal.h"

namespace pcr {
void serve_shutdown(Ctx&) {}
}  // namespace pcr

extern "C" {
pc_status pc_submit(pc_ctx*, pc_cloud, const pc_view*, uint32_t, pc_ticket*) { return PC_ENOTSUP; }
pc_status pc_poll(pc_ctx*, pc_ticket, int32_t, pc_result*) { return PC_ENOTSUP; }
pc_status pc_release_ticket(pc_ctx*, pc_ticket) { return PC_ENOTSUP; }
pc_status pc_build_lod(pc_ctx*, pc_cloud, const pc_lod_opts*, pc_cloud*) { return PC_ENOTSUP; }
}
