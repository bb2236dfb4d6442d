// Allocation entry points of the library.  Every device and pinned-host
// allocation the library makes for a context, an adjoint, a thermal model or
// a batch goes through these two functions, so that
// brahms_fail_next_allocations (tests of the error paths) can make the next
// ones report cudaErrorMemoryAllocation without calling the allocator.
#pragma once

#include <cuda_runtime.h>

namespace brahms {

cudaError_t dev_alloc(void** p, size_t bytes);
cudaError_t pinned_alloc(void** p, size_t bytes);

}  // namespace brahms
