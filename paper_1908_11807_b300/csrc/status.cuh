// Host-side mapping of CUDA launch errors and the device error word onto the
// library's status codes, shared by every entry point that reports them.
#pragma once

#include <cuda_runtime.h>

#include "../../include/arborx_b300.h"
#include "common.cuh"

namespace abx {

// Status of the launches just enqueued on this host thread (reads and clears
// the runtime's last-error slot).
inline int launch_status() {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ARBORX_OK : ARBORX_ECUDA;
}

// Status carried by a device error word (ERR_* bits).
inline int err_bits_to_status(uint32_t bits) {
  if (bits & ERR_NONFINITE) return ARBORX_EINVAL;
  if (bits & ERR_TIMEOUT) return ARBORX_ETIMEOUT;
  if (bits & (ERR_STACK | ERR_CSR)) return ARBORX_EOVERFLOW;
  return ARBORX_OK;
}

}  // namespace abx
