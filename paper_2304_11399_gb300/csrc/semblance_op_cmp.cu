// Instantiations of the semblance kernels for the CMP operator.
#include "semblance_kernels.cuh"

namespace tt {
namespace sk {
template KFn pick_kernel<TT_OP_CMP>(int, int, int, bool);
template SFn pick_stack<TT_OP_CMP>(int, bool);
template OFn pick_order<TT_OP_CMP>(bool);
}  // namespace sk
}  // namespace tt
