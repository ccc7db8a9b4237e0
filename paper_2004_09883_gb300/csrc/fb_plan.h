// fb_plan.h -- the pass builder shared by the plan API (fb_fft.cu) and the
// no-allocation entry point (fb_fft_noalloc.cu): radix schedules, four-step
// splits, the line-pass descriptor with its kernel, tile, shared-memory and
// TMA choices, and the kernel arguments of one launch.  Both entry points
// build their passes here, so they run the same kernels the same way.  Host
// code only; not part of the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "fb_fft.h"
#include "fb_internal.h"
#include "fft_p2.cuh"

namespace fbfft {
namespace plan {

// CTA size of passes over short contiguous lines of length L: 64 compute
// threads up to 128 points, 128 for 256 points (small CTAs, several per SM,
// three tiles in flight each; on the 3-D bench's L = 128 pass 64 measured 4 %
// faster than 128 and 12 % faster than 256).  FB_FFT_NN_SMALL_THREADS = 64,
// 128 or 256 forces one size.
inline int nn_small_threads(long long L)
{
    static int v = [] {
        const char* s = std::getenv("FB_FFT_NN_SMALL_THREADS");
        const int n = s ? std::atoi(s) : 0;
        return (n == 64 || n == 128 || n == 256) ? n : 0;
    }();
    return v ? v : (L <= 128 ? 64 : 128);
}

enum BufKind { kBufIn = 0, kBufOut = 1, kBufScratch = 2 };
constexpr size_t kMaxSmemBytes = 227 * 1024;

struct PassPlan {
    PassDesc d;
    int threads;  // CTA size of the chosen kernel
    int lg;       // log2(L) for a compile-time power-of-two kernel, 0 = generic kernel
    int io;       // IoMode of the power-of-two kernel
    int kind;     // 0 power-of-two kernel, 1 generic kernel, 2 mixed kernel (lg = log2 of the 2-factor),
                  // 3 plane pass (two trailing axes, lg1 = log2 rows, lg = log2 row length),
                  // 4 job of the batched-uneven kernel
    int lg1 = 0;
    long long grid;
    size_t smem;
    bool async_ok;  // tiles can move by TMA (given 16-byte aligned buffer bases)
    int src, dst;
    long long src_off, dst_off;  // element offsets into the source / destination buffer
    int group;                   // profiling group (the pass's role in the schedule)
    bool last;                   // last pass of its data: gets the 1/N scale
    long long scale_n = 0;       // transform length the 1/N scale refers to (0: the plan's N)
    int slot = 0;                // batched-uneven plans: side stream the pass runs on
    long long off_in_idx = -1;   // batched-uneven plans: index of the pass's offset
    long long off_out_idx = -1;  // tables in the plan's device offset buffer
    bool tc = false;             // radix-16 stages on the tensor cores
    int multi = -1;              // batched-uneven plans: the merged launch this pass belongs to
};

inline bool is_smooth(long long n)
{
    if (n < 1) return false;
    for (long long p : {2LL, 3LL, 5LL})
        while (n % p == 0) n /= p;
    return n == 1;
}

inline long long pow2floor(long long x)
{
    long long p = 1;
    while (p * 2 <= x) p *= 2;
    return p;
}
inline long long pow2ceil(long long x)
{
    long long p = 1;
    while (p < x) p *= 2;
    return p;
}
inline int ilog2ll(long long x)
{
    int l = 0;
    while ((1LL << l) < x) ++l;
    return l;
}

// Radix schedule of an in-shared-memory line: the power-of-two part as the
// compile-time kernels order it (pow2_radix: 16s, with the leftover 8/4/2
// last when that makes two stages, first otherwise), then 5s, then 3s.
inline int factorize(long long n, int* r, int cap, bool odd_first = false)
{
    if (n < 1) return FB_FFT_ERR_INVALID_ARG;
    if (!is_smooth(n) || n > FB_FFT_MAX_SMEM_LEN) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    int c = 0;
    auto push = [&](int v) {
        if (c < cap) r[c] = v;
        ++c;
    };
    int a = 0;
    while (n % 2 == 0) n /= 2, ++a;
    if (odd_first && n > 1) {  // only ever asked for lengths with a factor 3 or 5
        while (n % 5 == 0) n /= 5, push(5);
        while (n % 3 == 0) n /= 3, push(3);
        for (int s = 0; s < pow2_nst(a); ++s) push(pow2_radix(a, s));
        return c;
    }
    for (int s = 0; s < pow2_nst(a); ++s) push(pow2_radix(a, s));
    while (n % 5 == 0) n /= 5, push(5);
    while (n % 3 == 0) n /= 3, push(3);
    return c;
}

// n = n1 * n2 with n1 the divisor of n closest to sqrt(n) from below and
// both factors fitting one line pass.
inline int split_square(long long n, long long* n1, long long* n2)
{
    long long best = 0;
    for (long long d = 1; d * d <= n; ++d)
        if (n % d == 0 && n / d <= FB_FFT_MAX_SMEM_LEN) best = d;
    if (best == 0) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    *n1 = best, *n2 = n / best;
    return FB_FFT_OK;
}

inline int split_fourstep(long long n, long long* n1, long long* n2)
{
    if (n < 1) return FB_FFT_ERR_INVALID_ARG;
    if (!is_smooth(n) || n > FB_FFT_MAX_1D_LEN) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    if (n <= FB_FFT_MAX_SMEM_LEN) {
        *n1 = n, *n2 = 1;
        return FB_FFT_OK;
    }
    // N1 = the divisor of n closest to sqrt(n) from below with both factors fitting.
    long long best = 0;
    for (long long d = 1; d * d <= n; ++d)
        if (n % d == 0 && n / d <= FB_FFT_MAX_SMEM_LEN) best = d;
    if (best == 0) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    *n1 = best, *n2 = n / best;
    return FB_FFT_OK;
}

// Twiddle tables one line length reads: a table per stage s with Ns > 1
// (entries w_{Ns R}^{r k} at [(r-1) Ns + k]) and, for a power-of-two length
// whose last stage is split (p2_tw_split), the 16 x 15 factor table w_L^{r k},
// k < 16.  Lays them out from element `base` (each table 16-byte aligned),
// writes their jobs to jobs[0..*njobs) (at most kMaxStages + 1), the offsets
// to off[0..nst] (off[nst]: the factor table; 0 where none) and returns the
// elements used.
inline long long stage_tables(long long L, const int* radix, int nst, long long base, TwiddleJob* jobs, int* njobs,
                              int* off)
{
    long long total = base, Ns = 1;
    *njobs = 0;
    for (int s = 0; s <= nst; ++s) off[s] = 0;
    for (int s = 0; s < nst; ++s) {
        const long long cnt = Ns * (radix[s] - 1);
        if (Ns > 1 && cnt > 0) {
            jobs[(*njobs)++] = TwiddleJob{total, cnt, 0, 0, 1, radix[s], (int)Ns};
            off[s] = (int)total;
            total += (cnt + 1) & ~1LL;
        }
        Ns *= radix[s];
    }
    if ((L & (L - 1)) == 0 && p2_tw_split(ilog2ll(L))) {
        jobs[(*njobs)++] = TwiddleJob{total, 16 * 15, L, 0, 1, 16, 16};
        off[nst] = (int)total;
        total += 16 * 15;
    }
    return total - base;
}

// The compiled kernel a pass runs in one direction.
inline LineKernel pass_kernel(const PassPlan& q, bool fwd)
{
    if (q.kind == 4) {  // a job of the batched-uneven kernel: launched per phase, not per pass
        LineKernel k{nullptr, q.threads, fwd, 0, -1};
        k.kind = 4;
        return k;
    }
    if (q.tc) return line_kernel_p2tc(q.threads, fwd, q.lg, q.io);
    if (q.kind == 3) return line_kernel_plane(fwd, q.lg1, q.lg, q.threads);
    if (q.kind == 2) return line_kernel_mixed(fwd, q.lg);
    if (q.kind == 1) return line_kernel_generic(fwd);
    return line_kernel_p2(q.threads, fwd, q.lg, q.io);
}

// Dynamic shared memory of a pass's kernel (exact for the compile-time
// power-of-two kernels, a bound for the others).
inline size_t pass_smem(const PassPlan& q, bool async)
{
    const size_t ptw = q.d.ptw_smem ? (size_t)(ptw_pad((int)((1LL << q.d.ptw_log) + q.d.ptw_hi_cnt - 1)) + 1) * sizeof(float2) : 0;
    if (q.kind == 0) return (size_t)p2_smem_bytes(q.threads, q.lg, q.io, async, q.tc) + ptw;
    if (q.kind == 3) return (size_t)plane_smem_bytes(q.lg1, q.lg, q.threads);
    if (q.kind == 4) return q.smem;
    return line_smem_bytes(q.d.land_stride, q.d.L, 1 << q.d.logT, q.d.nst, async, q.d.tws);
}

// Resident CTAs per SM of a pass (shared memory and the 96-register cap).
inline int pass_ctas_per_sm(const PassPlan& q, size_t smem)
{
    if (q.kind == 3) return 1;  // plane pass: one CTA per SM
    const int by_smem = (int)(233472 / (smem + 1024));  // 228 KB per SM, 1 KB reserved per CTA
    const int by_regs = q.kind == 0 ? 65536 / ((q.threads + p2_producer_threads(q.lg)) * p2_launch_regs(q.threads, q.lg))
                                    : 65536 / ((q.threads + 32) * 96);
    const int by_tmem = q.tc ? 512 / tc_tmem_cols(q.threads) : by_smem;  // 512 TMEM columns per SM
    return std::min(std::min(by_smem, by_regs), by_tmem);
}

// Four-step column pass (ptw_log set): keep the post-twiddle tables in shared
// memory when that costs the compile-time kernel no resident CTA.
inline void ptw_to_smem(PassPlan& a, long long hi_cnt)
{
    if (a.kind != 0 || a.tc || !a.d.ptw) return;
    const int before = pass_ctas_per_sm(a, a.smem);
    PassPlan b = a;
    b.d.ptw_smem = 1;
    b.d.ptw_hi_cnt = (int)hi_cnt;
    const size_t smem = pass_smem(b, b.async_ok);
    if (smem > kMaxSmemBytes || pass_ctas_per_sm(b, smem) < before) return;
    a = b;
    a.smem = smem;
}

// Fill a line pass: L-point DFTs over lines (o, c); strides in elements.
// `twb` receives the stage twiddle tables the pass reads: it provides
// bool stages(L, radix, nst, off) writing the table offsets of the nst
// stages, then (off[nst]) that of a split last stage's factor table, and
// returns false when it has no room for them.
template <class Twiddles>
int make_line_pass(PassPlan& p, Twiddles& twb, long long L, long long O, long long C,
                   long long in_sn, long long in_sc, long long in_so, long long out_sk, long long out_sc,
                   long long out_so, bool in_tfast, bool out_tfast, bool ptw, bool odd_first = false,
                   int max_lines = 0, bool tc = false)
{
    p = PassPlan{};  // zero descriptor, default member values (no offset tables)
    PassDesc& d = p.d;
    const bool pow2_len = (L & (L - 1)) == 0;
    const bool mixed_len = !pow2_len && L <= kMixedMaxLen;  // mixed kernels fix the radix order
    int nst = factorize(L, d.radix, kMaxStages, odd_first && !pow2_len && !mixed_len);
    if (nst < 0) return nst;
    if (nst > kMaxStages) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    d.nst = nst;
    set_stage_products(d);
    int off[kMaxStages + 1] = {};
    if (!twb.stages(L, d.radix, nst, off)) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    for (int s = 0; s <= nst && s < kMaxStages; ++s) d.twoff[s] = off[s];

    const bool cfast = in_tfast || out_tfast;
    const bool pow2 = (L & (L - 1)) == 0;
    p.lg = pow2 ? ilog2ll(L) : 0;
    long long T = 1, land = 0;
    if (pow2) {
        // Compile-time kernels: strided tiles want 16 lines for 128-byte rows,
        // so long lines on a strided side take the 512-thread kernel.
        if (in_tfast && !out_tfast) return FB_FFT_ERR_UNSUPPORTED_SIZE;  // never planned
        p.io = ptw ? kIoCCP : (in_tfast ? kIoCC : (out_tfast ? kIoNC : kIoNN));
        // radix-16 stages on the tensor cores for L >= 256: 256-thread CTAs, two per
        // SM, so one CTA's butterflies overlap the other's matrix products
        p.tc = tc && line_kernel_p2tc(256, true, p.lg, p.io).fn != nullptr;
        p.threads = (!p.tc && cfast && L >= 512) ? 512 : 256;
        // short contiguous lines: 128-thread CTAs, three per SM, three tiles in flight each
        if (!p.tc && !cfast && L >= 32 && L <= 256) p.threads = nn_small_threads(L);
        if (!line_kernel_p2(p.threads, true, p.lg, p.io).fn) return FB_FFT_ERR_UNSUPPORTED_SIZE;
        T = p2_tile_lines(p.threads, p.lg, p.io);
        land = p2_land_elems(p.threads, p.lg, p.io);
        d.tws = p.tc ? 0 : p2_smem_twiddles(p.lg);
    } else {
        p.io = -1;
        int a2 = 0;
        while (((L >> a2) & 1) == 0) ++a2;
        p.kind = mixed_len ? 2 : 1;
        p.lg = mixed_len ? a2 : 0;
        p.threads = mixed_len ? kMixedThreads : kGenericThreads;
        const long long cap = (long long)p.threads * (mixed_len ? kMixedElems : kGenericElems);
        if (L > cap) return FB_FFT_ERR_UNSUPPORTED_SIZE;
        T = pow2floor(cap / L);
        T = std::min<long long>(T, cfast ? 16 : p.threads);
        if (max_lines > 0) T = std::min<long long>(T, pow2floor(max_lines));
        T = std::max<long long>(1, std::min(T, pow2ceil(C)));
        land = land_stride_elems((int)L, (int)T);
        if (!pass_kernel(p, true).fn) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    }

    d.L = (int)L;
    d.LS = (int)(L + (L >> 4) + 1);
    d.logT = ilog2ll(T);
    d.in_sn = in_sn, d.in_sc = in_sc, d.in_so = in_so;
    d.out_sk = out_sk, d.out_sc = out_sc, d.out_so = out_so;
    d.C = C;
    d.tiles_per_o = (C + T - 1) / T;
    d.ntiles = O * d.tiles_per_o;
    d.in_tfast = in_tfast ? 1 : 0;
    d.out_tfast = out_tfast ? 1 : 0;
    d.scale = 1.0f;
    // TMA needs 16-byte aligned addresses and 16-byte multiples: n-fast tiles
    // must be contiguous (line stride L, L even), c-fast views need even strides
    // and an even tile width.
    const bool in_ok = in_tfast ? (T % 2 == 0 && in_sn % 2 == 0 && (O == 1 || in_so % 2 == 0))
                                : (in_sc == L && in_sn == 1 && L % 2 == 0 && (O == 1 || in_so % 2 == 0));
    const bool out_ok = out_tfast ? (T % 2 == 0 && out_sk % 2 == 0 && (O == 1 || out_so % 2 == 0))
                                  : (out_sc == L && out_sk == 1 && L % 2 == 0 && (O == 1 || out_so % 2 == 0));
    p.async_ok = in_ok && out_ok && C < (1LL << 31) && O < (1LL << 31);
    // 3-D boxes of T x br rows: every box must start 128-byte aligned in
    // shared memory (one box when L <= 256), br <= 256 and a divisor of L.
    int br = 0;
    if (L <= 256)
        br = (int)L;
    else
        for (int b = 256; b >= 1 && !br; --b)
            if (L % b == 0 && (b * T * 8) % 128 == 0) br = b;
    if (br == 0 && (in_tfast || out_tfast)) p.async_ok = false;
    d.box_rows = br > 0 ? br : 1;
    d.land_stride = (int)land;
    d.ptw = ptw ? 1 : 0;
    p.smem = pass_smem(p, p.async_ok);
    if (p.smem > kMaxSmemBytes) {
        p.async_ok = false;
        p.smem = pass_smem(p, false);
    }
    if (p.smem > kMaxSmemBytes) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    p.grid = d.ntiles;  // capped to the resident CTA count when the plan is built
    return FB_FFT_OK;
}

// cuTensorMapEncodeTiled, fetched from the driver once (no libcuda link needed).
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
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
    return fn;
}

// 3-D view {C (contiguous), L (stride sn), O (stride so)} of complex64
// values, moved in boxes of T x box_rows x 1.  Returns 0 on success.
inline int encode_view(CUtensorMap* tm, const float2* base, long long C, long long L, long long O, long long sn,
                long long so, int T, int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return -1;
    if (O == 1) so = L * sn;
    cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)L, (cuuint64_t)O};
    cuuint64_t strides[2] = {(cuuint64_t)sn * 8, (cuuint64_t)so * 8};
    cuuint32_t box[3] = {(cuuint32_t)T, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<float2*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

// Kernel arguments of one launch of pass q reading `in` and writing `out`
// (offsets already applied); err (if not null) replaces the descriptor's
// error word.  Tiles move by TMA when the pass allows it and both bases are
// 16-byte aligned (tensor maps encoded here, they hold the addresses).
// Returns the launch's dynamic shared memory in bytes.
inline size_t line_args(LineArgs& args, const PassPlan& q, const float2* in, float2* out, int* err)
{
    std::memset(&args, 0, sizeof(args));
    args.d = q.d;
    PassDesc& d = args.d;
    if (err) d.err = err;
    d.in = in;
    d.out = out;
    d.async_io = 0;
    if (q.kind == 3) {
        // plane pass: bulk row loads, one tensor store of each CTA's column block
        // (view {L2, L1, planes}, box {L2 / cluster, L1, 1})
        const LineKernel pk = pass_kernel(q, true);
        const int L1 = 1 << q.lg1;
        if (q.async_ok && (((uintptr_t)d.in | (uintptr_t)d.out) & 15) == 0 &&
            encode_view(&args.tm_out, d.out, d.C, L1, d.ntiles, d.out_sk, d.out_so, d.L / std::max(1, pk.cluster),
                        L1) == 0)
            d.async_io = 1;
    } else if (q.async_ok && (((uintptr_t)d.in | (uintptr_t)d.out) & 15) == 0) {
        d.async_io = 1;
        const long long O = d.ntiles / d.tiles_per_o;
        if (d.in_tfast && !d.off_in &&
            encode_view(&args.tm_in, d.in, d.C, d.L, O, d.in_sn, d.in_so, 1 << d.logT, d.box_rows) != 0)
            d.async_io = 0;
        if (d.out_tfast && !d.off_out &&
            encode_view(&args.tm_out, d.out, d.C, d.L, O, d.out_sk, d.out_so, 1 << d.logT, d.box_rows) != 0)
            d.async_io = 0;
    }
    return pass_smem(q, d.async_io != 0);
}

}  // namespace plan
}  // namespace fbfft
