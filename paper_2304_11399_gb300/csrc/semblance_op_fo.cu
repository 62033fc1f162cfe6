// Instantiations of the semblance kernels for the FO-CRS operator.
#include "semblance_kernels.cuh"

namespace tt {
namespace sk {
template KFn pick_kernel<TT_OP_FOCRS>(int, int, int, bool);
template SFn pick_stack<TT_OP_FOCRS>(int, bool);
template OFn pick_order<TT_OP_FOCRS>(bool);
}  // namespace sk
}  // namespace tt
