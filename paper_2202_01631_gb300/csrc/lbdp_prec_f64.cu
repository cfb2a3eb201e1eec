// Single-box kernels and launchers of the CfgF64 precision mode.
#include "lbdp_ops.cuh"

namespace lbdp {
const PrecOps kOpsF64 = Ops<CfgF64>::table();
}  // namespace lbdp
