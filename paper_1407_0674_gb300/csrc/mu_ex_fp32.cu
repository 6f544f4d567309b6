// mu_ex pipeline instantiated in float FFT arithmetic (compiled on its own so
// the precisions build in parallel).
#include "mu_ex_core.cuh"

namespace pnp {
int run_pipeline_fp32(Problem *p, DeviceBuffers *db, const double *d_rho, double *d_mu, cudaStream_t st, bool tc) {
    return run_pipeline<float>(p, db, d_rho, d_mu, st, tc);
}
}  // namespace pnp
