// Entry points not implemented yet.
#include "pn_internal.cuh"
extern "C" int pn_server_create(const pn_server_cfg*, pn_server_t*) { pn_set_error("not implemented"); return PN_EINVAL; }
extern "C" int pn_server_destroy(pn_server_t) { return PN_OK; }
extern "C" int pn_submit(pn_server_t, pn_system_t, const pn_job*, uint64_t*) { pn_set_error("not implemented"); return PN_EINVAL; }
extern "C" int pn_poll(pn_server_t, uint64_t, pn_result*, int64_t) { pn_set_error("not implemented"); return PN_EINVAL; }
extern "C" int pn_cancel(pn_server_t, uint64_t) { return PN_EINVAL; }
extern "C" size_t pn_job_footprint(pn_system_t, int, int) { return 0; }
