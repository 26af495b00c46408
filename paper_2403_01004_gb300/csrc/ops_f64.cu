// Kernel instantiations for the PolF64 precision policy.
#include "ops_impl.cuh"

namespace pb {
Ops* ops_f64() {
    static OpsImpl<PolF64> ops;
    return &ops;
}
}  // namespace pb
