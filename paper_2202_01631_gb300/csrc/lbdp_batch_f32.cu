// Batched kernels and launchers of the CfgF32 precision mode.
#include "lbdp_ops.cuh"

namespace lbdp {
const BatchOps kBatchF32 = BOps<CfgF32>::table();
}  // namespace lbdp
