// Device allocations owned by the library all go through dev_malloc.
//
// Failure injection for tests: while the environment variable
// REX_FAIL_DEVICE_ALLOC holds a number n >= 1, the n-th allocation counted from
// the moment the variable took that value, and every later one while it keeps
// it, fails with cudaErrorMemoryAllocation without touching the device.  Unset,
// empty or not a positive number: every allocation goes to cudaMalloc.  This
// lets a test drive each allocation-failure path of the C ABI (the caller sees
// REX_ENOMEM and every buffer allocated before the failure is released) on any
// machine, GPU or not.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace rex {

cudaError_t dev_malloc(void** p, size_t bytes);

template <typename T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  void* q = nullptr;
  const cudaError_t e = dev_malloc(&q, bytes);
  *p = static_cast<T*>(q);
  return e;
}

}  // namespace rex
