// fb_fft_noalloc.cu -- fb_fft_exec_1d_noalloc: a batched 1-D transform that
// allocates no device memory.
//
// Who needs it: callers that cannot call cudaMalloc -- a plug-in or embedded
// library whose host application owns all device memory through its own
// allocator (and may forbid driver allocations outright), real-time code that
// must not enter an allocator that can block, or code that has to run in a
// device-memory budget fixed before it starts.  The plan API (fb_fft_plan)
// allocates twiddle tables and a four-step intermediate on the device; this
// entry point uses a workspace that lives in this file instead:
//
//   g_fb_noalloc_ws: a file-scope static __device__ array, 256-byte aligned,
//   of kWsScratch + kWsTwiddle complex64 values plus an error word
//   (32 MiB + 256 KiB + 256 B).  Every GPU that loads the library holds it
//   until the process exits.
//
// The passes are built by the same pass builder as the plan API's
// (fb_plan.h: kernels, tiles, shared memory, TMA), with the twiddle jobs
// collected in a fixed-capacity table on the stack.  The first launch of each
// kernel in the process sets its shared-memory limit (a fixed table, no heap);
// the CUDA runtime itself may allocate host memory inside its calls.
// In host code the array's name is only a stand-in for the device object, so
// the first call on each device resolves its device address with
// cudaGetSymbolAddress (with that device current) and caches it.  Every call
// shares the one array and overwrites it (twiddles, intermediate, error word,
// which is cleared at the start of each call): calls that overlap on the GPU
// -- on different streams, or from different host threads -- race and must be
// serialised by the caller.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "fb_fft.h"
#include "fb_internal.h"
#include "fb_plan.h"

using namespace fbfft;
using namespace fbfft::plan;

namespace {

constexpr long long kWsScratch = 4LL << 20;  // complex64 values: 32 MiB four-step intermediate
constexpr long long kWsTwiddle = 32LL << 10; // complex64 values: 256 KiB of twiddle tables
constexpr long long kWsErr = 32;             // 256 bytes holding the device error words
static __device__ __align__(256) float2 g_fb_noalloc_ws[kWsScratch + kWsTwiddle + kWsErr];

struct DevSlot {
    float2* base;
    bool ready;
};
DevSlot g_slot[64];
std::mutex g_slot_mu;

// Device address of the workspace on the current device (resolved once).
cudaError_t workspace(float2** base)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_slot_mu);
    if (!g_slot[dev].ready) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_fb_noalloc_ws);
        if (e != cudaSuccess) return e;
        g_slot[dev].base = static_cast<float2*>(p);
        g_slot[dev].ready = true;
    }
    *base = g_slot[dev].base;
    return cudaSuccess;
}

// Twiddle jobs in a fixed-capacity table: the stage tables of the lengths
// used and the four-step split tables.  Offsets count complex64 values from
// the table base.  A full table (or one past kWsTwiddle) refuses more.
struct StackTwiddles {
    static constexpr int kMaxJobs = 24;
    TwiddleJob jobs[kMaxJobs];
    int njobs = 0;
    long long total = 0;
    long long cached_L[2] = {0, 0};
    int cached_off[2][kMaxStages + 1] = {};
    int ncached = 0;

    bool stages(long long L, const int* radix, int nst, int* off)
    {
        for (int c = 0; c < ncached; ++c)
            if (cached_L[c] == L) {
                std::memcpy(off, cached_off[c], sizeof(int) * (nst + 1));
                return true;
            }
        TwiddleJob js[kMaxStages + 1];
        int nj = 0;
        const long long used = stage_tables(L, radix, nst, total, js, &nj, off);
        if (njobs + nj > kMaxJobs || total + used > kWsTwiddle) return false;
        for (int j = 0; j < nj; ++j) jobs[njobs++] = js[j];
        total += used;
        if (ncached < 2) {
            cached_L[ncached] = L;
            std::memcpy(cached_off[ncached], off, sizeof(int) * (nst + 1));
            ++ncached;
        }
        return true;
    }
    // exp(-2 pi i (m * mult) / D), m < count; returns its offset or -1 when full
    long long add_linear(long long count, long long D, long long mult)
    {
        if (njobs == kMaxJobs || total + count > kWsTwiddle) return -1;
        jobs[njobs++] = TwiddleJob{total, count, D, mult, 0, 0, 0};
        const long long off = total;
        total += (count + 1) & ~1LL;
        return off;
    }
};

// Launch pass q on `s`: grid capped to the CTAs resident at once, twiddles
// and error word in the workspace, the four-step tables bound to `tw`.
int launch(const PassPlan& q, const float2* in, float2* out, float2* tw, int* err, bool fwd, bool evict_first,
           bool debug_timeout, float scale, bool apply_scale, int sms, cudaStream_t s)
{
    PassPlan b = q;
    b.d.tw = tw;
    if (b.d.ptw) {
        b.d.ptw_lo = tw + reinterpret_cast<long long>(q.d.ptw_lo);
        b.d.ptw_hi = tw + reinterpret_cast<long long>(q.d.ptw_hi);
    }
    LineArgs a;
    const size_t smem = line_args(a, b, in, out, err);
    a.d.evict_first = evict_first ? 1 : 0;
    if (debug_timeout && a.d.async_io) a.d.debug_extra_tx = 16;
    if (apply_scale) {
        a.d.apply_scale = 1;
        a.d.scale = scale;
    }
    const LineKernel k = pass_kernel(q, fwd);
    int occ = 0;
    if (line_occupancy(k, smem, &occ) != cudaSuccess || occ < 1) return FB_FFT_ERR_CUDA;
    const long long grid = q.grid < (long long)sms * occ ? q.grid : (long long)sms * occ;
    return line_launch(k, a, grid, smem, s) == cudaSuccess ? FB_FFT_OK : FB_FFT_ERR_CUDA;
}

bool env_is(const char* name, char v)
{
    const char* s = std::getenv(name);
    return s && s[0] == v;
}

// The transform itself (no argument checks beyond sizes; see the caller).
int run(const float2* src, float2* dst, long long n, long long batch, bool fwd, bool apply_scale, cudaStream_t s,
        float2* ws, int* err)
{
    float2* scratch = ws;
    float2* tw = ws + kWsScratch;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FB_FFT_ERR_CUDA;
    const float scale = (float)(1.0 / (double)n);
    const bool evict = src != dst && !env_is("FB_FFT_EVICT_FIRST", '0');
    const bool debug = env_is("FB_FFT_NOALLOC_DEBUG_TIMEOUT", '1');
    StackTwiddles twj;
    if (n <= FB_FFT_MAX_SMEM_LEN) {  // one pass over contiguous lines, no intermediate
        PassPlan p;
        int rc = make_line_pass(p, twj, n, 1, batch, 1, n, 0, 1, n, 0, false, false, false);
        if (rc != FB_FFT_OK) return rc;
        for (int j = 0; j < twj.njobs; ++j)
            if (launch_twiddles(tw, twj.jobs[j], s) != cudaSuccess) return FB_FFT_ERR_CUDA;
        return launch(p, src, dst, tw, err, fwd, evict, debug, scale, apply_scale, sms, s);
    }
    // four-step, as the plan API schedules it: columns (length n1, times
    // exp(s 2 pi i n2 k1 / n)) into the workspace, rows (length n2) written
    // transposed to out, one chunk of the batch at a time.
    long long n1 = 0, n2 = 0;
    int rc = split_fourstep(n, &n1, &n2);
    if (rc != FB_FFT_OK) return rc;
    const int plog = (ilog2ll(n) + 1) / 2;
    const long long lo_cnt = 1LL << plog, hi_cnt = (n + lo_cnt - 1) >> plog;
    const long long chunk = std::min(batch, kWsScratch / n);
    PassPlan col, row;
    rc = make_line_pass(col, twj, n1, chunk, n2, n2, 1, n, n2, 1, n, true, true, true);
    if (rc != FB_FFT_OK) return rc;
    rc = make_line_pass(row, twj, n2, chunk, n1, 1, n2, n, n1, 1, n, false, true, false);
    if (rc != FB_FFT_OK) return rc;
    const long long lo_off = twj.add_linear(lo_cnt, n, 1);
    const long long hi_off = twj.add_linear(hi_cnt, n, lo_cnt);
    if (lo_off < 0 || hi_off < 0) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    col.d.ptw_log = plog;
    ptw_to_smem(col, hi_cnt);
    col.d.ptw_lo = reinterpret_cast<const float2*>(lo_off);  // offsets until launch binds them
    col.d.ptw_hi = reinterpret_cast<const float2*>(hi_off);
    for (int j = 0; j < twj.njobs; ++j)
        if (launch_twiddles(tw, twj.jobs[j], s) != cudaSuccess) return FB_FFT_ERR_CUDA;
    for (long long b0 = 0; b0 < batch; b0 += chunk) {
        const long long nb = std::min(chunk, batch - b0);
        PassPlan pc = col, pr = row;  // the last chunk may hold fewer transforms
        pc.d.ntiles = nb * pc.d.tiles_per_o;
        pr.d.ntiles = nb * pr.d.tiles_per_o;
        pc.grid = pc.d.ntiles;
        pr.grid = pr.d.ntiles;
        rc = launch(pc, src + b0 * n, scratch, tw, err, fwd, evict, debug, scale, false, sms, s);
        if (rc != FB_FFT_OK) return rc;
        rc = launch(pr, scratch, dst + b0 * n, tw, err, fwd, false, debug, scale, apply_scale, sms, s);
        if (rc != FB_FFT_OK) return rc;
    }
    return FB_FFT_OK;
}

}  // namespace

extern "C" int fb_fft_exec_1d_noalloc(const void* in, void* out, long long n, long long batch, int direction,
                                      unsigned flags, void* stream)
{
    if (n < 1 || batch < 0 || (direction != FB_FFT_FORWARD && direction != FB_FFT_INVERSE) ||
        (flags & ~(FB_FFT_SCALE_INV_N | FB_FFT_NOALLOC_CHECK)))
        return FB_FFT_ERR_INVALID_ARG;
    long long n1 = 0, n2 = 0;
    int rc = split_fourstep(n, &n1, &n2);
    if (rc != FB_FFT_OK) return rc;
    if (n > kWsScratch) return FB_FFT_ERR_UNSUPPORTED_SIZE;  // one transform must fit the workspace
    if (batch == 0) return FB_FFT_OK;
    if (!in || !out || (((uintptr_t)in | (uintptr_t)out) & 7)) return FB_FFT_ERR_INVALID_ARG;
    if (batch > kWsScratch * 4096) return FB_FFT_ERR_UNSUPPORTED_SIZE;  // keeps n * batch * 8 far from overflow
    const uintptr_t bytes = (uintptr_t)(n * batch) * 8u;
    const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out;
    if (a != b && a < b + bytes && b < a + bytes) return FB_FFT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float2* ws = nullptr;
    if (workspace(&ws) != cudaSuccess) return FB_FFT_ERR_CUDA;
    int* err = reinterpret_cast<int*>(ws + kWsScratch + kWsTwiddle);
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return FB_FFT_ERR_CUDA;

    const bool fwd = direction == FB_FFT_FORWARD;
    const bool apply_scale = !fwd && (flags & FB_FFT_SCALE_INV_N);
    if (n == 1) {  // X[0] = x[0] (the 1/N scale is 1): a copy, or nothing in place
        if (a != b && cudaMemcpyAsync(out, in, (size_t)bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return FB_FFT_ERR_CUDA;
    } else {
        rc = run(static_cast<const float2*>(in), static_cast<float2*>(out), n, batch, fwd, apply_scale, s, ws, err);
        if (rc != FB_FFT_OK) return rc;
    }
    if (flags & FB_FFT_NOALLOC_CHECK) {  // wait, then report a device wait that gave up
        int word = 0;
        if (cudaMemcpyAsync(&word, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return FB_FFT_ERR_CUDA;
        if (word) return FB_FFT_ERR_TIMEOUT;
    }
    return FB_FFT_OK;
}
