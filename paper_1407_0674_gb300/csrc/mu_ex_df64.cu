// mu_ex pipeline instantiated in dd FFT arithmetic (compiled on its own so
// the precisions build in parallel).
#include "mu_ex_core.cuh"

namespace pnp {
int run_pipeline_df64(Problem *p, DeviceBuffers *db, const double *d_rho, double *d_mu, cudaStream_t st) {
    return run_pipeline<dd>(p, db, d_rho, d_mu, st);
}
}  // namespace pnp
