// The CUDA device of a context made current for the extent of one C-ABI
// call, and the caller's current device given back when the call returns:
// a call never leaves another device current behind the caller's back.
#pragma once

#include <cuda_runtime.h>

struct DeviceScope {
  int prev = -1;                  // the caller's device to give back (-1: none)
  cudaError_t err = cudaSuccess;  // of the switch; the call fails with it
  explicit DeviceScope(int dev) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) cur = -1;
    if (cur != dev) {
      err = cudaSetDevice(dev);
      if (err == cudaSuccess) prev = cur;
    }
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DeviceScope(const DeviceScope &) = delete;
  DeviceScope &operator=(const DeviceScope &) = delete;
};
