// Device-side constants and helpers shared by the kernel translation units.
#pragma once

#include <cuda_runtime.h>

namespace ppk {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// SMs of the current device (cached per process).
inline int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 132;
    }
    return sms;
}

}  // namespace ppk
