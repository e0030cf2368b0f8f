// server.cpp -- continuous-batching serving loop (perm_submit / perm_poll).
#include <cstring>

#include "plan.hpp"

using namespace perm;

struct perm_server_s { int dummy; };

extern "C" {
perm_status_t perm_server_create(const perm_server_opts_t *, perm_server_t *out) {
    if (out) *out = nullptr;
    return fail(PERM_ERR_INTERNAL, "serving not built yet");
}
perm_status_t perm_submit(perm_server_t, const perm_matrix_t *, uint64_t *) { return fail(PERM_ERR_ARG, "no server"); }
perm_status_t perm_poll(perm_server_t, uint64_t, int32_t, perm_result_t *) { return fail(PERM_ERR_ARG, "no server"); }
perm_status_t perm_server_stats(perm_server_t, perm_server_stats_t *) { return fail(PERM_ERR_ARG, "no server"); }
void perm_server_destroy(perm_server_t) {}
}
