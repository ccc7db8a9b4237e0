// fb_host.h -- host-side plan operations shared between the planner
// (fb_fft.cu) and the request server (fb_serve.cu).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include "fb_fft.h"

namespace fbfft {
namespace host {

// A regular (non-batched-uneven) plan; ext_scratch: allocate no scratch,
// every exec passes one of plan_scratch_bytes bytes.
int plan_create(fb_fft_plan_t* out, int rank, const long long* dims, long long batch, unsigned flags,
                cudaStream_t build_stream, bool ext_scratch);
long long plan_scratch_bytes(fb_fft_plan_t p);  // four-step intermediate (0 if none)
long long plan_table_bytes(fb_fft_plan_t p);    // device bytes the plan itself holds
long long plan_io_bytes(fb_fft_plan_t p);       // bytes of one input (= one output)
// Launch the plan's passes on `stream`; scratch: plan_scratch_bytes of
// device memory (may be null when that is 0); err: device-visible int[16]
// for bounded-wait errors (null: the plan's own).
int plan_exec_on(fb_fft_plan_t p, const void* in, void* out, int direction, cudaStream_t stream, void* scratch,
                 int* err);
void plan_free(fb_fft_plan_t p);
// Record a failed CUDA call for fb_fft_last_error and map it to a status.
int fail(cudaError_t e, const char* what);

}  // namespace host
}  // namespace fbfft
