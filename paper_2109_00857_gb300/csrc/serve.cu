// serve.cu -- batched build+solve and the replanning server (see include/mdp.h).
#include "mdp_internal.cuh"

using namespace mdpgb;

static mdp_status not_built(const char *what) {
  set_error(std::string(what) + ": not available in this build");
  return MDP_ERR_ARG;
}

extern "C" mdp_status mdp_batch_create(const mdp_batch_item *, int32_t, double, mdp_batch *out) {
  if (out) *out = nullptr;
  return not_built("mdp_batch_create");
}
extern "C" mdp_status mdp_batch_run(mdp_batch, void *, int32_t *, double *) { return not_built("mdp_batch_run"); }
extern "C" void mdp_batch_free(mdp_batch) {}
extern "C" mdp_status mdp_serve_create(size_t, int32_t, mdp_server *out) {
  if (out) *out = nullptr;
  return not_built("mdp_serve_create");
}
extern "C" mdp_status mdp_env_register(mdp_server, const mdp_env *, const mdp_grid *, const mdp_actions *,
                                       int32_t, int32_t *) { return not_built("mdp_env_register"); }
extern "C" mdp_status mdp_serve_submit(mdp_server, const mdp_request *, uint64_t *) { return not_built("mdp_serve_submit"); }
extern "C" mdp_status mdp_serve_poll(mdp_server, uint64_t, int32_t, mdp_result *, float *, int16_t *) {
  return not_built("mdp_serve_poll");
}
extern "C" mdp_status mdp_serve_stats(mdp_server, int64_t *, int64_t *, int64_t *) { return not_built("mdp_serve_stats"); }
extern "C" mdp_status mdp_serve_destroy(mdp_server) { return not_built("mdp_serve_destroy"); }
