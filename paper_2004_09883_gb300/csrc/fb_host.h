// fb_host.h -- host-side plan operations shared between the planner
// (fb_fft.cu) and the request server (fb_serve.cu).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "fb_fft.h"
#include "fb_internal.h"

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

// One job of a request shape on the one-kernel engine (k_fft_uneven): its
// descriptor with the twiddle pointers bound, and where it reads and writes.
struct BatchJob {
    PassDesc d;       // in / out: element offsets into the buffers src / dst name
    int phase;        // launch it runs in: jobs of phase k + 1 read what phase k wrote
    int src, dst;     // 0 the request's input, 1 its output, 2 its scratch
    bool last;        // the job that finishes the transform (takes the 1/N scale)
    int land, work;   // landing / work buffer elements its tiles need
};
// Every job of one request shape (rank, dims, batch): up to three phases
// (one per axis of a 2-D / 3-D shape; columns then rows of a 1-D four-step
// length), twiddle tables in a device buffer of its own.
struct BatchRecipe {
    std::vector<BatchJob> jobs;
    int phases = 0;
    long long scratch_bytes = 0;  // four-step intermediate of one request
    long long table_bytes = 0;    // device bytes the recipe holds
    long long tiles = 0;          // tiles of all its jobs
    float scale = 1.f;            // 1 / (elements of one transform)
    float2* tw = nullptr;
};
// UNSUPPORTED_SIZE when some axis (or four-step factor) exceeds one job's
// 2048 points, or the tensor-core flag is set: such shapes run per request.
int recipe_create(BatchRecipe** out, int rank, const long long* dims, long long batch, unsigned flags,
                  cudaStream_t stream);
void recipe_free(BatchRecipe* r);
// One launch of k_fft_uneven over the job and tile-prefix tables in device
// memory (njobs jobs, `tiles` tiles in all); the launch counter counts it.
int batch_launch(bool forward, const PassDesc* jobs, const int* tile_start, int njobs, long long tiles,
                 int land_max, int work_max, cudaStream_t stream);
// The same launch with the tables (host memory, at most 16 jobs) copied
// into the kernel parameter: nothing to copy to the device beforehand.
int batch_launch_inline(bool forward, const PassDesc* jobs, const int* tile_start, int njobs, long long tiles,
                        int land_max, int work_max, cudaStream_t stream);
// Record a failed CUDA call for fb_fft_last_error and map it to a status.
int fail(cudaError_t e, const char* what);

}  // namespace host
}  // namespace fbfft
