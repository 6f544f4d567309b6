// Serving loop (placeholder).
#include "pnp_internal.h"

extern "C" {
int pnp_server_create(const pnp_server_opts *, pnp_server **out) { if (out) *out = nullptr; return PNP_ERR_INVALID; }
void pnp_server_destroy(pnp_server *) {}
int pnp_submit(pnp_server *, const pnp_problem_desc *, const double *, const double *, uint64_t *) { return PNP_ERR_INVALID; }
int pnp_poll(pnp_server *, uint64_t, double *, double *, pnp_stats *) { return PNP_ERR_UNKNOWN_TICKET; }
int pnp_server_get_stats(pnp_server *, pnp_server_stats *) { return PNP_ERR_INVALID; }
}
