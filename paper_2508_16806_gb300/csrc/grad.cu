// Adjoint of unrolled fixed-step PDHG (placeholder until the kernels land).
#include "common.cuh"

namespace pdhg {

lp_status run_grad(Handle*, const lp_opts*, int, int, const double*, double*, double*, double*,
                   double*, int, double*)
{
    return LP_NOT_SUPPORTED;
}

}  // namespace pdhg
