// Which CUDA device a call may run on: the decision of the device check that
// every GPU entry point makes before it launches (api.cpp, check_device).
// A context's tables live on the device that was current when they were
// uploaded; a kernel launched on another device would read them through a
// foreign address (an illegal-address fault, or silent peer reads).  Kept free
// of CUDA calls so that the host tests can exercise the refusal paths.
#pragma once

namespace ed {

enum DeviceVerdict {
  kDeviceOk = 0,
  kDeviceWrongCurrent = 1,   // the current device is not the context's device
  kDeviceForeignBuffer = 2,  // a caller's buffer is device memory of another device
};

// ctx_dev: the context's device; cur_dev: the current device; buf_dev: the
// device that owns a caller's buffer, or -1 for host or managed memory (the
// library copies host buffers itself; managed memory is reachable anywhere).
inline DeviceVerdict device_verdict(int ctx_dev, int cur_dev, int buf_dev) {
  if (cur_dev != ctx_dev) return kDeviceWrongCurrent;
  if (buf_dev >= 0 && buf_dev != ctx_dev) return kDeviceForeignBuffer;
  return kDeviceOk;
}

}  // namespace ed
