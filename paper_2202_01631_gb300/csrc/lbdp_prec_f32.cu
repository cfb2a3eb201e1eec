// Single-box kernels and launchers of the CfgF32 precision mode.
#include "lbdp_ops.cuh"

namespace lbdp {
const PrecOps kOpsF32 = Ops<CfgF32>::table();
}  // namespace lbdp
