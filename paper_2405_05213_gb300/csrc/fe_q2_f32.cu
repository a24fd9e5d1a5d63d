// Element-apply instances for order 2, float arithmetic.
#include "fe_dispatch.cuh"

namespace etp {
ETP_DEFINE_LAUNCH_ELEM_APPLY(2, float)
}  // namespace etp
