// Element-apply instances for order 1, float arithmetic.
#include "fe_dispatch.cuh"

namespace etp {
ETP_DEFINE_LAUNCH_ELEM_APPLY(1, float)
}  // namespace etp
