// Element-apply instances for order 1, double arithmetic.
#include "fe_dispatch.cuh"

namespace etp {
ETP_DEFINE_LAUNCH_ELEM_APPLY(1, double)
}  // namespace etp
