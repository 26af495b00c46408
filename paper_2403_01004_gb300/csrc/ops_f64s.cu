// Kernel instantiations for the PolF64S precision policy (float64 storage and stage recurrence,
// float32 records and stencil arithmetic).
#include "ops_impl.cuh"

namespace pb {
Ops* ops_f64s() {
    static OpsImpl<PolF64S> ops;
    return &ops;
}
}  // namespace pb
