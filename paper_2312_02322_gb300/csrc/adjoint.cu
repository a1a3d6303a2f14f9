// Discrete adjoint of the RK4 trajectory map (cross-section gradients).
#include <cuda_runtime.h>

#include "internal.h"

using namespace mqct;

extern "C" mqct_status mqct_adjoint(mqct_system sys, const mqct_traj *trajs, int32_t n, const double *weight,
                                    const int32_t *group, int32_t n_groups, const double *dL_dsigma, int32_t ckpt,
                                    double *dL_dparam, void *cuda_stream)
{
    (void)trajs; (void)weight; (void)group; (void)n_groups; (void)dL_dsigma; (void)ckpt; (void)dL_dparam;
    (void)cuda_stream;
    if (!sys || n < 0) return fail(MQCT_ERR_INVALID_ARG, "mqct_adjoint: bad argument");
    return fail(MQCT_ERR_UNSUPPORTED, "mqct_adjoint: not available in this build");
}
