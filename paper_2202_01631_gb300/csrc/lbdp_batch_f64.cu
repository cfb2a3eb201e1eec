// Batched kernels and launchers of the CfgF64 precision mode.
#include "lbdp_ops.cuh"

namespace lbdp {
const BatchOps kBatchF64 = BOps<CfgF64>::table();
}  // namespace lbdp
