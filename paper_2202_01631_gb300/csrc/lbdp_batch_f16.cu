// Batched kernels and launchers of the CfgF16 precision mode.
#include "lbdp_ops.cuh"

namespace lbdp {
const BatchOps kBatchF16 = BOps<CfgF16>::table();
}  // namespace lbdp
