// twiddle.cu -- the twiddle-table kernel: exp(-2*pi*i*m/D) evaluated in FP64
// on the GPU (CUDA's sincospi after exact integer reduction of m modulo D) and
// rounded to nearest FP32.  The tables only ever hold the forward sign; the
// inverse uses their conjugates, which is exact.
#include "fb_internal.h"

namespace fbfft {

__global__ void k_twiddles(float2* __restrict__ tw, TwiddleJob job)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= job.count) return;
    long long m, D;
    if (job.kind == 0) {
        D = job.D;
        m = (long long)((unsigned long long)(i % D) * (unsigned long long)(job.mult % D) % (unsigned long long)D);
    } else {
        const long long r = i / job.Ns + 1;
        const long long k = i % job.Ns;
        D = job.D > 0 ? job.D : (long long)job.Ns * job.R;  // D set: w_D^{r k} (a split factor table)
        m = (r * k) % D;
    }
    double s, c;
    sincospi(-2.0 * (double)m / (double)D, &s, &c);
    tw[job.offset + i] = make_float2((float)c, (float)s);
}

cudaError_t launch_twiddles(float2* tw, const TwiddleJob& job, cudaStream_t stream)
{
    if (job.count <= 0) return cudaSuccess;
    const int threads = 256;
    const long long blocks = (job.count + threads - 1) / threads;
    k_twiddles<<<(unsigned)blocks, threads, 0, stream>>>(tw, job);
    return cudaGetLastError();
}

}  // namespace fbfft
