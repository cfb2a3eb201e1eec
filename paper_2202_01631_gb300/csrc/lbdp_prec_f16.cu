// Single-box kernels and launchers of the CfgF16 precision mode.
#include "lbdp_ops.cuh"

namespace lbdp {
const PrecOps kOpsF16 = Ops<CfgF16>::table();
}  // namespace lbdp
