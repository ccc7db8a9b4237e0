// fb_fft_noalloc.cu -- fb_fft_exec_1d_noalloc: a batched 1-D transform that
// allocates nothing.
//
// Who needs it: callers that cannot call cudaMalloc -- code running while a
// CUDA graph is being captured elsewhere in the process, real-time or
// signal-context code that must not enter the allocator, and embedders whose
// memory is owned by another allocator and who cannot hand us a plan-sized
// scratch buffer.  The plan API (fb_fft_plan) allocates twiddle tables and a
// four-step intermediate on the device; this entry point uses a workspace
// that lives in this file instead:
//
//   g_fb_noalloc_ws: a file-scope static __device__ array, 256-byte aligned,
//   of kWsScratch + kWsTwiddle complex64 values plus an error word
//   (32 MiB + 256 KiB + 256 B).  Every GPU that loads the library holds it
//   until the process exits.
//
// The kernels are the library's line-pass kernels; only where their scratch,
// twiddle tables and error word live differs.  Host-side planning uses the
// stack only (no heap, no device allocation, no allocating library call).
// In host code the array's name is only a stand-in for the device object, so
// the first call on each device resolves its device address with
// cudaGetSymbolAddress (with that device current) and caches it; make that
// first call before any stream capture.  Every call shares the one array and
// overwrites it (twiddles, intermediate, error word, which is cleared at the
// start of each call): calls that overlap on the GPU -- on different streams,
// or from different host threads -- race and must be serialised by the caller.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "fb_fft.h"
#include "fb_internal.h"
#include "fft_p2.cuh"

using namespace fbfft;

namespace {

constexpr long long kWsScratch = 4LL << 20;  // complex64 values: 32 MiB four-step intermediate
constexpr long long kWsTwiddle = 32LL << 10; // complex64 values: 256 KiB of twiddle tables
constexpr long long kWsErr = 32;             // 256 bytes holding the device error word
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

// Twiddle jobs on the stack: stage tables of the lengths used, and the
// four-step split tables.  Offsets count complex64 values from the table base.
struct StackTwiddles {
    TwiddleJob jobs[24];
    int njobs = 0;
    long long total = 0;
    bool add(const TwiddleJob& j)
    {
        if (njobs == 24 || total + j.count > kWsTwiddle) return false;
        jobs[njobs++] = j;
        total += (j.count + 1) & ~1LL;
        return true;
    }
};

struct Pass {
    PassDesc d;
    LineKernel k[2];  // inverse, forward
    long long grid;
    size_t smem;
    bool async_ok;
};

// One line pass, the same kernel choice, tile shape and TMA eligibility as
// the plan builder makes for these modes.
int fill_pass(Pass& p, StackTwiddles& tw, long long L, long long O, long long C, long long in_sn, long long in_sc,
              long long in_so, long long out_sk, long long out_sc, long long out_so, bool in_t, bool out_t, bool ptw)
{
    p = Pass{};  // every field zero (no offset tables, no post-twiddle, no scale)
    PassDesc& d = p.d;
    int nst = 0;
    int rc = fb_fft_factorize(L, d.radix, kMaxStages, &nst);
    if (rc != FB_FFT_OK) return rc;
    d.nst = nst;
    long long Ns = 1;
    for (int s = 0; s < nst; ++s) {
        d.ns[s] = (int)Ns;
        if (Ns > 1) {
            d.twoff[s] = (int)tw.total;
            if (!tw.add(TwiddleJob{tw.total, Ns * (d.radix[s] - 1), 0, 0, 1, d.radix[s], (int)Ns}))
                return FB_FFT_ERR_UNSUPPORTED_SIZE;
        }
        Ns *= d.radix[s];
    }
    if ((L & (L - 1)) == 0) {
        int lg = 0;
        while ((1LL << lg) < L) ++lg;
        if (p2_tw_split(lg)) {  // the 16 x 15 factor table of the split last stage
            d.twoff[nst] = (int)tw.total;
            if (!tw.add(TwiddleJob{tw.total, 16 * 15, L, 0, 1, 16, 16})) return FB_FFT_ERR_UNSUPPORTED_SIZE;
        }
    }
    set_stage_products(d);
    const bool pow2 = (L & (L - 1)) == 0;
    const bool cfast = in_t || out_t;
    long long T, land;
    int threads;
    if (pow2) {
        int lg = 0;
        while ((1LL << lg) < L) ++lg;
        const int io = ptw ? kIoCCP : (in_t ? kIoCC : (out_t ? kIoNC : kIoNN));
        threads = (cfast && L >= 512) ? 512 : 256;
        p.k[1] = line_kernel_p2(threads, true, lg, io);
        p.k[0] = line_kernel_p2(threads, false, lg, io);
        T = p2_tile_lines(threads, lg, io);
        land = p2_land_elems(threads, lg, io);
        d.tws = p2_smem_twiddles(lg);
    } else {
        const bool mixed = L <= kMixedMaxLen;
        int a2 = 0;
        while (((L >> a2) & 1) == 0) ++a2;
        threads = mixed ? kMixedThreads : kGenericThreads;
        p.k[1] = mixed ? line_kernel_mixed(true, a2) : line_kernel_generic(true);
        p.k[0] = mixed ? line_kernel_mixed(false, a2) : line_kernel_generic(false);
        const long long cap = (long long)threads * (mixed ? kMixedElems : kGenericElems);
        T = 1;
        while (T * 2 * L <= cap && T * 2 <= (cfast ? 16 : threads)) T *= 2;
        long long cpow = 1;
        while (cpow < C) cpow *= 2;
        if (T > cpow) T = cpow;
        land = (L * T + 15) & ~15LL;
    }
    if (!p.k[0].fn || !p.k[1].fn) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    int logT = 0;
    while ((1LL << logT) < T) ++logT;
    d.L = (int)L;
    d.LS = (int)(L + (L >> 4) + 1);
    d.logT = logT;
    d.in_sn = in_sn, d.in_sc = in_sc, d.in_so = in_so;
    d.out_sk = out_sk, d.out_sc = out_sc, d.out_so = out_so;
    d.C = C;
    d.tiles_per_o = (C + T - 1) / T;
    d.ntiles = O * d.tiles_per_o;
    d.in_tfast = in_t ? 1 : 0;
    d.out_tfast = out_t ? 1 : 0;
    d.ptw = ptw ? 1 : 0;
    d.scale = 1.0f;
    const bool in_ok = in_t ? (T % 2 == 0 && in_sn % 2 == 0 && (O == 1 || in_so % 2 == 0))
                            : (in_sc == L && in_sn == 1 && L % 2 == 0 && (O == 1 || in_so % 2 == 0));
    const bool out_ok = out_t ? (T % 2 == 0 && out_sk % 2 == 0 && (O == 1 || out_so % 2 == 0))
                              : (out_sc == L && out_sk == 1 && L % 2 == 0 && (O == 1 || out_so % 2 == 0));
    int br = 0;
    if (L <= 256)
        br = (int)L;
    else
        for (int b = 256; b >= 1 && !br; --b)
            if (L % b == 0 && (b * T * 8) % 128 == 0) br = b;
    p.async_ok = in_ok && out_ok && br > 0;
    d.box_rows = br > 0 ? br : 1;
    d.land_stride = (int)land;
    p.smem = line_smem_bytes(land, (int)L, (int)T, nst, p.async_ok, d.tws);
    if (p.smem > 227 * 1024) {
        p.async_ok = false;
        p.smem = line_smem_bytes(land, (int)L, (int)T, nst, false, d.tws);
    }
    if (p.smem > 227 * 1024) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    p.grid = d.ntiles;
    return FB_FFT_OK;
}

int encode(CUtensorMap* tm, const float2* base, const PassDesc& d, long long O, long long sn, long long so)
{
    static PFN_cuTensorMapEncodeTiled_v12000 enc = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    if (!enc) return -1;
    if (O == 1) so = (long long)d.L * sn;
    cuuint64_t dims[3] = {(cuuint64_t)d.C, (cuuint64_t)d.L, (cuuint64_t)O};
    cuuint64_t strides[2] = {(cuuint64_t)sn * 8, (cuuint64_t)so * 8};
    cuuint32_t box[3] = {(cuuint32_t)(1 << d.logT), (cuuint32_t)d.box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<float2*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS
               ? 0
               : -1;
}

int launch(const Pass& p, const float2* in, float2* out, const float2* tw, int* err, bool fwd, float scale,
           bool apply_scale, int sms, cudaStream_t s)
{
    LineArgs a;
    std::memset(&a, 0, sizeof(a));
    a.d = p.d;
    a.d.in = in;
    a.d.out = out;
    a.d.tw = tw;
    a.d.err = err;
    if (p.d.ptw) {
        a.d.ptw_lo = tw + reinterpret_cast<long long>(p.d.ptw_lo);
        a.d.ptw_hi = tw + reinterpret_cast<long long>(p.d.ptw_hi);
    }
    if (apply_scale) {
        a.d.apply_scale = 1;
        a.d.scale = scale;
    }
    const long long O = p.d.ntiles / p.d.tiles_per_o;
    a.d.async_io = 0;
    if (p.async_ok && (((uintptr_t)in | (uintptr_t)out) & 15) == 0) {
        a.d.async_io = 1;
        if (p.d.in_tfast && encode(&a.tm_in, in, p.d, O, p.d.in_sn, p.d.in_so) != 0) a.d.async_io = 0;
        if (p.d.out_tfast && encode(&a.tm_out, out, p.d, O, p.d.out_sk, p.d.out_so) != 0) a.d.async_io = 0;
    }
    const size_t smem = line_smem_bytes(p.d.land_stride, p.d.L, 1 << p.d.logT, p.d.nst, a.d.async_io != 0, p.d.tws);
    const LineKernel& k = p.k[fwd ? 1 : 0];
    int occ = 0;
    if (line_occupancy(k, smem, &occ) != cudaSuccess || occ < 1) return FB_FFT_ERR_CUDA;
    long long grid = p.grid < (long long)sms * occ ? p.grid : (long long)sms * occ;
    return line_launch(k, a, grid, smem, s) == cudaSuccess ? FB_FFT_OK : FB_FFT_ERR_CUDA;
}

}  // namespace

extern "C" int fb_fft_exec_1d_noalloc(const void* in, void* out, long long n, long long batch, int direction,
                                      unsigned flags, void* stream)
{
    if (n < 1 || batch < 0 || (direction != FB_FFT_FORWARD && direction != FB_FFT_INVERSE) ||
        (flags & ~FB_FFT_SCALE_INV_N))
        return FB_FFT_ERR_INVALID_ARG;
    long long n1 = 0, n2 = 0;
    int rc = fb_fft_split(n, &n1, &n2);
    if (rc != FB_FFT_OK) return rc;
    if (n > kWsScratch) return FB_FFT_ERR_UNSUPPORTED_SIZE;  // one transform must fit the workspace
    if (batch == 0) return FB_FFT_OK;
    if (!in || !out || (((uintptr_t)in | (uintptr_t)out) & 7)) return FB_FFT_ERR_INVALID_ARG;
    const uintptr_t bytes = (uintptr_t)(n * batch) * 8u;
    const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out;
    if (a != b && a < b + bytes && b < a + bytes) return FB_FFT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float2* ws = nullptr;
    if (workspace(&ws) != cudaSuccess) return FB_FFT_ERR_CUDA;
    float2* scratch = ws;
    float2* tw = ws + kWsScratch;
    int* err = reinterpret_cast<int*>(ws + kWsScratch + kWsTwiddle);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FB_FFT_ERR_CUDA;

    const bool fwd = direction == FB_FFT_FORWARD;
    const bool apply_scale = !fwd && (flags & FB_FFT_SCALE_INV_N);
    const float scale = (float)(1.0 / (double)n);
    const float2* src = static_cast<const float2*>(in);
    float2* dst = static_cast<float2*>(out);
    StackTwiddles twj;
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return FB_FFT_ERR_CUDA;

    if (n2 == 1) {  // one pass, no intermediate
        Pass p;
        rc = fill_pass(p, twj, n, 1, batch, 1, n, 0, 1, n, 0, false, false, false);
        if (rc != FB_FFT_OK) return rc;
        for (int j = 0; j < twj.njobs; ++j)
            if (launch_twiddles(tw, twj.jobs[j], s) != cudaSuccess) return FB_FFT_ERR_CUDA;
        rc = launch(p, src, dst, tw, err, fwd, scale, apply_scale, sms, s);
        return rc;
    }
    // four-step: columns (length n1, times the split twiddle) into the
    // workspace, rows (length n2) written transposed to out, one chunk of
    // the batch at a time.
    int plog = 0;
    while ((1LL << plog) * (1LL << plog) < n) ++plog;
    const long long lo_cnt = 1LL << plog, hi_cnt = (n + lo_cnt - 1) >> plog;
    const long long chunk_max = kWsScratch / n;
    const long long c1 = batch < chunk_max ? batch : chunk_max;
    Pass col, row;
    rc = fill_pass(col, twj, n1, c1, n2, n2, 1, n, n2, 1, n, true, true, true);
    if (rc != FB_FFT_OK) return rc;
    rc = fill_pass(row, twj, n2, c1, n1, 1, n2, n, n1, 1, n, false, true, false);
    if (rc != FB_FFT_OK) return rc;
    const long long lo_off = twj.total;
    if (!twj.add(TwiddleJob{lo_off, lo_cnt, n, 1, 0, 0, 0})) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    const long long hi_off = twj.total;
    if (!twj.add(TwiddleJob{hi_off, hi_cnt, n, lo_cnt, 0, 0, 0})) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    col.d.ptw_log = plog;
    col.d.ptw_lo = reinterpret_cast<const float2*>(lo_off);
    col.d.ptw_hi = reinterpret_cast<const float2*>(hi_off);
    for (int j = 0; j < twj.njobs; ++j)
        if (launch_twiddles(tw, twj.jobs[j], s) != cudaSuccess) return FB_FFT_ERR_CUDA;
    for (long long b0 = 0; b0 < batch; b0 += c1) {
        const long long nb = batch - b0 < c1 ? batch - b0 : c1;
        Pass pc = col, pr = row;  // the last chunk may hold fewer transforms
        pc.d.ntiles = nb * pc.d.tiles_per_o;
        pr.d.ntiles = nb * pr.d.tiles_per_o;
        pc.grid = pc.d.ntiles;
        pr.grid = pr.d.ntiles;
        rc = launch(pc, src + b0 * n, scratch, tw, err, fwd, scale, false, sms, s);
        if (rc != FB_FFT_OK) return rc;
        rc = launch(pr, scratch, dst + b0 * n, tw, err, fwd, scale, apply_scale, sms, s);
        if (rc != FB_FFT_OK) return rc;
    }
    return FB_FFT_OK;
}
