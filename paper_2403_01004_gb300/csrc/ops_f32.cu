// Kernel instantiations for the PolF32 precision policy.
#include "ops_impl.cuh"

namespace pb {
Ops* ops_f32() {
    static OpsImpl<PolF32> ops;
    return &ops;
}
}  // namespace pb
