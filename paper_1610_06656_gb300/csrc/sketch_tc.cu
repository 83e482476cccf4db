// Tensor-core (tcgen05) sketch engine: placeholder until the sm_103a kernel lands; AUTO falls back to nothing
// here because tc_supported() reports false, so the SIMT engine runs.
#include "internal.h"

namespace smp {

bool tc_supported(const smp_ctx*) { return false; }

cudaError_t launch_sketch_tc(smp_ctx*, const void*, int64_t, const void*, int64_t, int64_t, int64_t) {
    return cudaErrorNotSupported;
}

}  // namespace smp
