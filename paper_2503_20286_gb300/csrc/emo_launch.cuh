// Host launchers whose shapes the C ABI tunes, and the sticky device status.
#pragma once

#include <cuda_runtime.h>

#include "emo_internal.cuh"

namespace emo {

// The association kernels of every problem; grid = sms x blocks_per_sm.
cudaError_t launch_assoc(Plan* plan, int nprob, const int* m_of, int sms, int blocks_per_sm, cudaStream_t s);
// Sticky device status: the first failure any call on this device reported
// since the last read (k_finish sets it); read after the stream's prior work.
cudaError_t sticky_status(cudaStream_t s, int32_t* out, bool clear);

}  // namespace emo
