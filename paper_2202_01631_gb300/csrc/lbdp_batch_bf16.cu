// Batched kernels and launchers of the CfgBF16 precision mode.
#include "lbdp_ops.cuh"

namespace lbdp {
const BatchOps kBatchBF16 = BOps<CfgBF16>::table();
}  // namespace lbdp
