// Entry points whose implementation is being written: they validate nothing
// and report MRHS_ERR_INVALID.
#include "internal.cuh"
namespace mrhs { mrhs_status api_record(mrhs_status code, const std::string &msg); }
#define PENDING return mrhs::api_record(MRHS_ERR_INVALID, "not available yet")
extern "C" {
void mrhs_mg_default_params(mrhs_mg_params *p) { if (p) { *p = mrhs_mg_params{}; p->n_levels = 2; p->n_vec[0] = 8; p->outer_m = 4; p->max_rhs = 64; } }
mrhs_status mrhs_setup_mg(mrhs_lattice *, const mrhs_mg_params *, mrhs_mg **) { PENDING; }
void mrhs_destroy_mg(mrhs_mg *) {}
mrhs_status mrhs_mg_level_info(mrhs_mg *, int, int *, int *) { PENDING; }
mrhs_status mrhs_mg_get_prolongator(mrhs_mg *, int, double *) { PENDING; }
mrhs_status mrhs_mg_get_coarse_links(mrhs_mg *, int, double *) { PENDING; }
mrhs_status mrhs_restrict(mrhs_mg *, int, const void *, void *, int, void *) { PENDING; }
mrhs_status mrhs_prolong(mrhs_mg *, int, const void *, void *, int, void *) { PENDING; }
mrhs_status mrhs_coarse_apply(mrhs_mg *, int, const void *, void *, int, mrhs_precision, void *) { PENDING; }
mrhs_status mrhs_vcycle(mrhs_mg *, const void *, void *, int, void *) { PENDING; }
mrhs_status mrhs_solve(mrhs_mg *, const void *, void *, int, double, double *, mrhs_solve_stats *, void *) { PENDING; }
mrhs_status mrhs_server_create(const mrhs_server_params *, mrhs_server **) { PENDING; }
mrhs_status mrhs_server_add_config(mrhs_server *, mrhs_mg *, int, int *) { PENDING; }
mrhs_status mrhs_submit(mrhs_server *, int, const double *, double *, int, double, uint64_t *) { PENDING; }
mrhs_status mrhs_poll(mrhs_server *, uint64_t, mrhs_request_stats *) { PENDING; }
mrhs_status mrhs_server_drain(mrhs_server *) { PENDING; }
void mrhs_server_destroy(mrhs_server *) {}
}
