// Single-box kernels and launchers of the CfgBF16 precision mode.
#include "lbdp_ops.cuh"

namespace lbdp {
const PrecOps kOpsBF16 = Ops<CfgBF16>::table();
}  // namespace lbdp
