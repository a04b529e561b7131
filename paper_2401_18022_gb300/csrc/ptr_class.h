// Where a caller's buffer lives, decided from what cudaPointerGetAttributes
// reports (its memory type and device) and the device the call runs on.
// Kept free of CUDA headers so that a host-only test can compile it.
#pragma once

namespace isrs {

// cudaMemoryType values: 0 unregistered host, 1 registered (pinned) host,
// 2 device, 3 managed.
enum PtrClass {
    kPtrHost = 0,          // host memory: the library copies through it
    kPtrDevice = 1,        // device memory the current device can use directly
    kPtrOtherDevice = 2    // device memory of another GPU: rejected
};

inline int ptr_class(int memory_type, int owner_device, int current_device)
{
    if (memory_type == 2) return owner_device == current_device ? kPtrDevice : kPtrOtherDevice;
    if (memory_type == 3) return kPtrDevice;   // managed memory migrates to whichever device uses it
    return kPtrHost;
}

}  // namespace isrs
