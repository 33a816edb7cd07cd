// Programmatic dependent launch helper shared by the chain's kernels.
#pragma once

namespace lst {

// Programmatic dependent launch: the chain's kernels are launched so that the
// next one may start while this one drains. Every kernel first waits for its
// predecessor grid to complete (and its writes to be visible); the successor
// is scheduled as this grid's blocks retire. A no-op for a kernel launched
// without the attribute.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

}  // namespace lst
