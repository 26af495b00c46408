// Kernel instantiations for the PolB16 precision policy.
#include "ops_impl.cuh"

namespace pb {
Ops* ops_b16() {
    static OpsImpl<PolB16> ops;
    return &ops;
}
}  // namespace pb
