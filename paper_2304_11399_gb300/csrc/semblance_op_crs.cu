// Instantiations of the semblance kernels for the ZO-CRS operator.
#include "semblance_kernels.cuh"

namespace tt {
namespace sk {
template KFn pick_kernel<TT_OP_CRS>(int, int, int, bool);
template SFn pick_stack<TT_OP_CRS>(int, bool);
template OFn pick_order<TT_OP_CRS>(bool);
}  // namespace sk
}  // namespace tt
