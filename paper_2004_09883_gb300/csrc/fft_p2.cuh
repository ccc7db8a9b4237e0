// fft_p2.cuh -- the line pass for power-of-two lines, specialised at compile
// time on the line length (L = 2^LG), the CTA size and the in/out layout.
//
// Everything that shapes the index arithmetic is a template constant: the
// radix schedule (16, 16, ..., then one of 8/4/2), Ns of every stage, lines per
// tile T, the shared-memory strides and which side is strided.  What remains
// at run time is the tile walk (pointers, strides, counts), the twiddle table
// base and the optional 1/N scale.
#pragma once

#include "fft_device.cuh"
#include "fft_tc.cuh"

namespace fbfft {

// In/out layouts of a pass.  N = lines contiguous in memory (a tile is T whole
// lines), C = lines adjacent in memory (a tile is T columns x L rows).
enum IoMode {
    kIoNN = 0,   // contiguous in and out: 1-D lines, last axis of multi-D
    kIoCC = 1,   // strided in and out: the other axes of multi-D
    kIoNC = 2,   // contiguous in, strided out: four-step rows (transposed store)
    kIoCCP = 3,  // strided in and out, output times exp(s 2 pi i c k / N): four-step columns
};

__host__ __device__ constexpr int p2_min(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int p2_max(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr bool io_in_strided(int io) { return io == kIoCC || io == kIoCCP; }
__host__ __device__ constexpr bool io_out_strided(int io) { return io != kIoNN; }
// Lines per tile: 16 (128-byte rows) when a side is strided, else as many
// whole lines as the tile holds (at most one per thread).
__host__ __device__ constexpr int p2_tile_lines(int threads, int lg, int io)
{
    return (io_in_strided(io) || io_out_strided(io)) ? p2_min(16, threads * kElemsPerThread >> lg)
                                                     : p2_min(threads, threads * kElemsPerThread >> lg);
}
// Row padding of contiguous landing layouts: with G < 16 threads per line a
// half-warp touches 16/G lines at G consecutive values each; rows G values
// apart (mod 16) put those lines on disjoint banks.  (Even, so every row stays
// 16-byte aligned for its bulk copy.)
__host__ __device__ constexpr int p2_row_pad(int threads, int lg, int io, bool out_side)
{
    const int T = p2_tile_lines(threads, lg, io);
    const int G = threads / T;
    const bool strided = out_side ? io_out_strided(io) : io_in_strided(io);
    return (!strided && G < 16) ? (G >= 2 ? G : 2) : 0;
}
// Three-stage schedules whose last two radices are 16 (L = 2048, 4096) have
// a last-stage table of L - L/16 entries, too many for shared memory.  With
// k = 16 kh + kl (kh < Ns of the middle stage), that stage's twiddle factors:
//   w_L^{k r} = w_{L/16}^{kh r} * w_L^{kl r},
// the first factor an entry of the middle stage's table, the second of a
// 16 x 15 table of its own (offset twoff[NST]).
__host__ __device__ constexpr bool p2_tw_split(int lg)
{
    return pow2_nst(lg) == 3 && pow2_radix(lg, 1) == 16 && pow2_radix(lg, 2) == 16 &&
           pow2_ns(lg, 1) * 15 + pow2_ns(lg, 2) * 15 > 1024;
}
// Stage twiddle tables (stages 1..NST-1) small enough to copy into shared
// memory once per CTA: their total entry count, or 0 when they stay in global.
__host__ __device__ constexpr int p2_smem_twiddles(int lg)
{
    if (p2_tw_split(lg)) return pow2_ns(lg, 1) * 15 + 16 * 15;
    int total = 0;
    for (int s = 1; s < pow2_nst(lg); ++s) total += pow2_ns(lg, s) * (pow2_radix(lg, s) - 1);
    return total <= 1024 ? total : 0;
}
// Elements of one landing buffer (input layout, then reused for the output layout).
__host__ __device__ constexpr int p2_land_elems(int threads, int lg, int io)
{
    const int T = p2_tile_lines(threads, lg, io);
    const int L = 1 << lg;
    const int in_e = io_in_strided(io) ? L * T : (L + p2_row_pad(threads, lg, io, false)) * T;
    const int out_e = io_out_strided(io) ? L * T : (L + p2_row_pad(threads, lg, io, true)) * T;
    return (p2_max(in_e, out_e) + 15) & ~15;
}

// Padded work-buffer line stride.  Strided modes read/write it across lines
// (consecutive threads on consecutive lines): a half-warp holds H = 16/T
// positions of each of its T lines (T < 16), so rows must start H * (odd)
// banks apart: stride mod 2H == H (T >= 16: an odd stride).  On the 1024-
// and 2048-point strided passes this halved the last stage's bank conflicts.
// The contiguous mode with G < 16 threads per line puts 16/G lines in one
// half-warp: a stride of G (mod 16) values puts them on disjoint banks.
__host__ __device__ constexpr int p2_strided_stride(int ls0, int h)
{
    return ls0 % (2 * h) == h ? ls0 : p2_strided_stride(ls0 + 1, h);
}
__host__ __device__ constexpr int p2_work_stride(int threads, int lg, int io)
{
    const int L = 1 << lg;
    const int LS0 = L + L / 16;
    const int T = p2_tile_lines(threads, lg, io);
    const int G = threads / T;
    if (io == kIoNN) return G < 16 ? LS0 + ((G - LS0 % 16) % 16 + 16) % 16 : LS0 + 1;
    return p2_strided_stride(LS0, T < 16 ? 16 / T : 1);
}
// First work-buffer generation of strided tiles with fewer than 16 lines:
// the first stage writes radix-R groups (positions R j + r) of T lines, and
// a half-warp holds 16/T groups side by side, R positions apart, which the
// row stride alone cannot spread (same banks for j and j + 1).  XOR-ing the
// low two index bits with the next two moves group j + 1 by an odd amount
// (then the usual i + i/16 padding); the next stage reads it back with one
// per-thread XOR, its offsets r * L/16 keeping the low four bits.  On the
// 1024- and 2048-point strided passes this removed the first stage's store
// conflicts.
__host__ __device__ constexpr bool p2_swz0(int threads, int lg, int io)
{
    return io_in_strided(io) && p2_tile_lines(threads, lg, io) < 16 && pow2_nst(lg) >= 2 &&
           pow2_radix(lg, 0) < 16 && pow2_radix(lg, 1) == 16;
}
__host__ __device__ __forceinline__ int spad_x(int i) { return spad(i ^ ((i >> 2) & 3)); }
// Index of entry e of the four-step tables kept in shared memory (lo, then
// hi): one pad entry every 32 spreads the gathers of a half-warp's lines.
__host__ __device__ constexpr int ptw_pad(int e) { return e + (e >> 5); }

// Dynamic shared memory of a power-of-two line pass: alignment slack and
// mbarriers (256 B), landing buffer(s), the work buffer (when there is more
// than one stage), stage twiddles, and for tensor-core kernels B^T + alignment.
// Landing buffers in flight per CTA: 128-thread CTAs (short contiguous lines,
// three CTAs per SM) keep three, so two tile loads stay in flight while one
// tile is transformed.
__host__ __device__ constexpr int p2_nbuf(int threads) { return threads <= 128 ? 3 : 2; }
__host__ __device__ constexpr long long p2_smem_bytes(int threads, int lg, int io, bool async, bool tc)
{
    return 256 + 8LL * (p2_land_elems(threads, lg, io) * (async ? p2_nbuf(threads) : 1) +
                        (pow2_nst(lg) > 1 ? (long long)p2_work_stride(threads, lg, io) * p2_tile_lines(threads, lg, io) : 0) +
                        (tc ? 0 : p2_smem_twiddles(lg))) +
           (tc ? (long long)kTcExtraSmem : 0);
}

template <int THREADS, int LG, int IO>
struct P2 {
    static constexpr int L = 1 << LG;
    static constexpr bool IN_T = io_in_strided(IO);
    static constexpr bool OUT_T = io_out_strided(IO);
    static constexpr bool PTW = IO == kIoCCP;
    static constexpr int T = p2_tile_lines(THREADS, LG, IO);
    static constexpr int LOGT = ilog2(T);
    static constexpr int G = THREADS / T;
    static constexpr int NST = pow2_nst(LG);
    static constexpr int LS = p2_work_stride(THREADS, LG, IO);  // padded work-buffer line stride
    static constexpr int LLS = L + p2_row_pad(THREADS, LG, IO, false);  // landing line stride (contiguous in)
    static constexpr int OLS = L + p2_row_pad(THREADS, LG, IO, true);   // landing line stride (contiguous out)
    static constexpr int LAND = p2_land_elems(THREADS, LG, IO);
    static constexpr int NBUF = p2_nbuf(THREADS);  // landing buffers
    static constexpr int BR = L < 256 ? L : 256;  // rows per 3-D TMA box
    static constexpr int TWS = p2_smem_twiddles(LG);  // twiddle entries kept in shared memory (0: global)
    static constexpr bool SWZ0 = p2_swz0(THREADS, LG, IO);  // first work-buffer generation XOR-swizzled
    static_assert(T * L <= THREADS * kElemsPerThread, "tile exceeds the CTA's registers");
    static_assert(T >= 1 && G >= 1, "bad tile shape");
};

// Barrier among the compute warps only (named barrier 1; the producer warp
// never joins it).
template <int THREADS>
__device__ __forceinline__ void compute_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(THREADS) : "memory");
}
// Same, returning whether any compute thread passed `pred`.
template <int THREADS>
__device__ __forceinline__ bool compute_sync_or(bool pred)
{
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((unsigned)pred), "n"(THREADS)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Offset of stage s's table inside the shared-memory twiddle copy.
__host__ __device__ constexpr int p2_tws_off(int lg, int s)
{
    return s <= 1 ? 0 : p2_tws_off(lg, s - 1) + pow2_ns(lg, s - 1) * (pow2_radix(lg, s - 1) - 1);
}

// One Stockham stage (stage S of the compile-time schedule) over the tile.
template <int THREADS, bool FWD, int LG, int IO, int S>
__device__ __forceinline__ void p2_stage(const PassDesc& d, float2* land, float2* work, int Tv, int c0,
                                         const float2* tws)
{
    using C = P2<THREADS, LG, IO>;
    constexpr int L = C::L, T = C::T, G = C::G;
    constexpr int R = pow2_radix(LG, S);
    constexpr int NS = pow2_ns(LG, S);
    constexpr int LR = L / R;
    constexpr int Q = (kElemsPerThread + R - 1) / R;
    constexpr bool first = S == 0;
    constexpr bool last = S == C::NST - 1;
    constexpr bool tfast = (first && C::IN_T) || (last && C::OUT_T);
    const int tid = threadIdx.x;
    const int t = tfast ? (tid & (T - 1)) : (tid / G);
    const int jb = tfast ? (tid >> C::LOGT) : (tid & (G - 1));
    const bool tok = t < Tv;
    float2 v[Q][R];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (q * G >= LR) break;  // compile-time: no butterflies left for this slot
        const int j = jb + q * G;
        if (tok && ((q + 1) * G <= LR || j < LR)) {
            if constexpr (first) {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    v[q][r] = C::IN_T ? land[(j + r * LR) * T + t] : land[t * C::LLS + j + r * LR];
            } else if constexpr (S == 1 && C::SWZ0) {
                static_assert(LR % 16 == 0, "second-stage offsets keep the low four index bits");
                const float2* p = work + t * C::LS;
                const int jx = j ^ ((j >> 2) & 3);
#pragma unroll
                for (int r = 0; r < R; ++r) v[q][r] = p[spad(jx + r * LR)];
            } else {
                const float2* p = work + t * C::LS;
#pragma unroll
                for (int r = 0; r < R; ++r) v[q][r] = p[spad(j + r * LR)];
            }
        } else if constexpr (C::NST >= 3) {
            // defined on every path: loaded and used under the same condition,
            // which the register allocator cannot prove, the values of every
            // stage would otherwise stay live around the tile loop (three-stage
            // schedules spilled; two-stage ones measured faster without this)
#pragma unroll
            for (int r = 0; r < R; ++r) v[q][r] = make_float2(0.f, 0.f);
        }
    }
    if constexpr (first == last) compute_sync<THREADS>();  // reads and writes share the landing buffer
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (q * G >= LR) break;
        const int j = jb + q * G;
        if (tok && ((q + 1) * G <= LR || j < LR)) {
            const int k = j & (NS - 1);
            if constexpr (NS > 1) {
                if constexpr (p2_tw_split(LG) && S == 2) {
                    // w_L^{k r} = w_{L/16}^{kh r} w_L^{kl r} from the two tables for r = 1
                    // and r = 8 only; the others by one complex multiply each from
                    // those (w^r = w^{r-1} w: at most seven products in a row, as
                    // for the four-step twiddle), 4 shared loads per butterfly
                    // instead of 30
                    static_assert(R == 16, "the split stage is radix 16");
                    constexpr int NS1 = pow2_ns(LG, 1);
                    const float2* th = tws + p2_tws_off(LG, 1) + (k >> 4);  // w_{L/16}^{kh r}
                    const float2* tl = tws + p2_tws_off(LG, 2) + (k & 15);  // w_L^{kl r}
                    const float2 w1 = cmul(th[0], tl[0]);
                    const float2 w8 = cmul(th[7 * NS1], tl[7 * 16]);
                    float2 w = w1;
                    v[q][1] = twmul<FWD>(v[q][1], w1);
#pragma unroll
                    for (int r = 2; r < 8; ++r) {
                        w = cmul(w, w1);
                        v[q][r] = twmul<FWD>(v[q][r], w);
                    }
                    w = w8;
                    v[q][8] = twmul<FWD>(v[q][8], w8);
#pragma unroll
                    for (int r = 9; r < 16; ++r) {
                        w = cmul(w, w1);
                        v[q][r] = twmul<FWD>(v[q][r], w);
                    }
                } else if constexpr (C::TWS > 0) {
                    const float2* tw = tws + p2_tws_off(LG, S) + k;
#pragma unroll
                    for (int r = 1; r < R; ++r) v[q][r] = twmul<FWD>(v[q][r], tw[(r - 1) * NS]);
                } else {
                    const float2* tw = d.tw + d.twoff[S] + k;
#pragma unroll
                    for (int r = 1; r < R; ++r) v[q][r] = twmul<FWD>(v[q][r], __ldg(tw + (r - 1) * NS));
                }
            }
            dft<R, FWD>(v[q]);
            if constexpr (!last) {
                float2* p = work + t * C::LS;
                const int base = (j - k) * R + k;
                if constexpr (S == 0 && C::SWZ0) {
#pragma unroll
                    for (int r = 0; r < R; ++r) p[spad_x(base + r * NS)] = v[q][r];
                } else {
#pragma unroll
                    for (int r = 0; r < R; ++r) p[spad(base + r * NS)] = v[q][r];
                }
            } else {
                // last stage: NS = L / R, so k == j and output index kk = j + r * LR
                // Four-step twiddle exp(-2 pi i c kk / N) of output kk of line c:
                // read from the split tables for r = 0 and r = 8, and stepped by
                // exp(-2 pi i c LR / N) for the r between (at most 7 products in a
                // row: a few ulp).  The table reads are gathers over the 16
                // lines of a half-warp at stride kk, which land on few banks:
                // three per butterfly instead of one per value.
                float2 w = make_float2(1.f, 0.f), wstep = make_float2(1.f, 0.f);
                const unsigned c = (unsigned)(c0 + t);
                auto ptw_at = [&](unsigned m) {  // m = c kk < N < 2^31
                    const unsigned mlo = m & ((1u << d.ptw_log) - 1), mhi = m >> d.ptw_log;
                    if (d.ptw_smem) {  // tables copied behind the stage twiddles
                        const float2* pt = tws + C::TWS;
                        return cmul(pt[ptw_pad((1 << d.ptw_log) + (int)mhi)], pt[ptw_pad((int)mlo)]);
                    }
                    return cmul(__ldg(d.ptw_hi + mhi), __ldg(d.ptw_lo + mlo));
                };
                if constexpr (C::PTW) {
                    if constexpr (R > 1) wstep = ptw_at(c * (unsigned)LR);
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int kk = j + r * LR;
                    float2 y = v[q][r];
                    if constexpr (C::PTW) {
                        w = (r % 8 == 0) ? ptw_at(c * (unsigned)kk) : cmul(w, wstep);
                        y = twmul<FWD>(y, w);
                    }
                    if (d.apply_scale) y = d.scale * y;
                    if constexpr (C::OUT_T)
                        land[kk * T + t] = y;
                    else
                        land[t * C::OLS + kk] = y;
                }
            }
        }
    }
}

// A radix-16 stage on the tensor cores (fft_tc.cuh): same gather, twiddles
// and scatter as p2_stage, the 16-point DFT as one FP16 hi/lo matrix product
// per 128 butterflies.  Needs exactly one butterfly per compute thread and at
// least two stages (the A tiles live in the work buffer).
template <int THREADS, bool FWD, int LG, int IO, int S>
__device__ __forceinline__ void p2_stage_tc(const PassDesc& d, float2* land, float2* work, int Tv, int c0,
                                            const float2* tws, TcState& tc)
{
    using C = P2<THREADS, LG, IO>;
    constexpr int L = C::L, T = C::T, G = C::G;
    constexpr int R = 16;
    constexpr int NS = pow2_ns(LG, S);
    constexpr int LR = L / R;
    constexpr bool first = S == 0;
    constexpr bool last = S == C::NST - 1;
    constexpr bool tfast = (first && C::IN_T) || (last && C::OUT_T);
    static_assert(pow2_radix(LG, S) == 16 && C::NST >= 2, "tensor-core stage: radix 16, not the only stage");
    static_assert(T * LR == THREADS && THREADS % 128 == 0, "tensor-core stage: one butterfly per thread");
    static_assert(T * L * 8 <= T * C::LS * 8, "A tiles fit the work buffer");
    static_assert(!(S == 0 && C::SWZ0), "the swizzled first generation is written by an FP32 stage");
    const int tid = threadIdx.x;
    const int t = tfast ? (tid & (T - 1)) : (tid / G);
    const int j = tfast ? (tid >> C::LOGT) : (tid & (G - 1));
    const bool tok = t < Tv;
    float2 v[R];
    if (tok) {
        if constexpr (first) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = C::IN_T ? land[(j + r * LR) * T + t] : land[t * C::LLS + j + r * LR];
        } else if constexpr (S == 1 && C::SWZ0) {
            static_assert(LR % 16 == 0, "second-stage offsets keep the low four index bits");
            const float2* p = work + t * C::LS;
            const int jx = j ^ ((j >> 2) & 3);
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = p[spad(jx + r * LR)];
        } else {
            const float2* p = work + t * C::LS;
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = p[spad(j + r * LR)];
        }
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = make_float2(0.f, 0.f);
    }
    if constexpr (!first && !kTcATmem) compute_sync<THREADS>();  // A rows overwrite the work buffer just read
    const int k = j & (NS - 1);
    if constexpr (NS > 1) {  // tensor-core kernels keep the stage twiddles in global memory (L1-cached)
        const float2* tw = d.tw + d.twoff[S] + k;
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = twmul<FWD>(v[r], __ldg(tw + (r - 1) * NS));
    }
    const unsigned abase = smem_u32(work);
    int e;
    if constexpr (kTcATmem) {
        e = tc_put_row_tmem(v, tc);
        tc_fence_before();  // the TMEM stores, before the barrier the issuing thread waits at
    } else {
        e = tc_put_row(v, abase, tid >> 7, tid & 127);
        fence_proxy_async();  // the A rows -> visible to the tensor cores
    }
    // (also: every thread's gather is done before any thread scatters below)
    compute_sync<THREADS>();
    if (tid == 0) {
        if constexpr (kTcATmem)
            tc_issue_tmem<THREADS / 128>(tc);
        else
            tc_issue<THREADS / 128>(tc, abase);
    }
    const bool ok = mbar_wait_bounded(tc.bar, tc.uses & 1u);
    tc.uses++;
    if (!ok && (tid & 31) == 0) atomicExch(d.err, 1);
    tc_fence_after();
    tc_get_row(tc, e, v);  // every product has landed: the A tiles are dead, the work buffer is free
    if (!tok) return;
    if constexpr (!last) {
        float2* p = work + t * C::LS;
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) p[spad(base + r * NS)] = v[r];
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int kk = j + r * LR;
            float2 y = v[r];
            if constexpr (C::PTW) {
                const unsigned m = (unsigned)(c0 + t) * (unsigned)kk;  // < N < 2^31
                const float2 w = cmul(__ldg(d.ptw_hi + (m >> d.ptw_log)),
                                      __ldg(d.ptw_lo + (m & ((1u << d.ptw_log) - 1))));
                y = twmul<FWD>(y, w);
            }
            if (d.apply_scale) y = d.scale * y;
            if constexpr (C::OUT_T)
                land[kk * T + t] = y;
            else
                land[t * C::OLS + kk] = y;
        }
    }
}

// Stage S, on the tensor cores when TC and the stage is radix 16.
template <int THREADS, bool FWD, int LG, int IO, int S, bool TC>
__device__ __forceinline__ void p2_run_stage(const PassDesc& d, float2* land, float2* work, int Tv, int c0,
                                             const float2* tws, TcState& tc)
{
    if constexpr (TC && pow2_radix(LG, S) == 16) {
        p2_stage_tc<THREADS, FWD, LG, IO, S>(d, land, work, Tv, c0, tws, tc);
    } else {
        // tensor-core kernels copy no stage twiddles: their FP32 stage is the first (no twiddles)
        static_assert(!TC || pow2_ns(LG, S) == 1, "FP32 stage with twiddles in a tensor-core kernel");
        p2_stage<THREADS, FWD, LG, IO, S>(d, land, work, Tv, c0, tws);
    }
}

template <int THREADS, bool FWD, int LG, int IO, int S, bool TC>
__device__ __forceinline__ void p2_stages_from(const PassDesc& d, float2* land, float2* work, int Tv, int c0,
                                               bool async, const float2* tws, TcState& tc)
{
    using C = P2<THREADS, LG, IO>;
    if constexpr (S < C::NST) {
        p2_run_stage<THREADS, FWD, LG, IO, S, TC>(d, land, work, Tv, c0, tws, tc);
        if constexpr (S == C::NST - 1)
            if (async) fence_proxy_async();  // output tile -> visible to the TMA store
        compute_sync<THREADS>();              // (last stage: the work buffer is free again)
        p2_stages_from<THREADS, FWD, LG, IO, S + 1, TC>(d, land, work, Tv, c0, async, tws, tc);
    }
}

// Compute threads: copy the stage twiddle tables into shared memory.
template <int THREADS, int LG, int S>
__device__ __forceinline__ void p2_copy_twiddles(const PassDesc& d, float2* tws)
{
    if constexpr (S < pow2_nst(LG)) {
        constexpr bool lo = p2_tw_split(LG) && S == 2;  // the 16 x 15 factor table instead
        constexpr int n = lo ? 16 * 15 : pow2_ns(LG, S) * (pow2_radix(LG, S) - 1);
        const float2* src = d.tw + d.twoff[lo ? 3 : S];
        for (int e = threadIdx.x; e < n; e += THREADS) tws[p2_tws_off(LG, S) + e] = __ldg(src + e);
        p2_copy_twiddles<THREADS, LG, S + 1>(d, tws);
    }
}

__device__ __forceinline__ TileIdx p2_tile_index(const PassDesc& d, long long tile, int logT, int T)
{
    TileIdx ti;
    ti.o = tile / d.tiles_per_o;
    ti.c0 = (tile - ti.o * d.tiles_per_o) << logT;
    const long long rem = d.C - ti.c0;
    ti.Tv = rem < T ? (int)rem : T;
    return ti;
}

// Producer warp (all lanes): start the TMA loads of one tile.
template <int THREADS, int LG, int IO>
__device__ __forceinline__ void p2_issue_load(const PassDesc& d, const CUtensorMap* tm, long long tile,
                                              float2* land, unsigned long long* bar, int lane)
{
    using C = P2<THREADS, LG, IO>;
    const TileIdx ti = p2_tile_index(d, tile, C::LOGT, C::T);
    const float2* src = tile_in_base(d, ti, C::IN_T);
    // the caller's input is read once per exec: let its lines leave L2 first,
    // so the pass's output stays there for the next pass
    const bool ef = d.evict_first != 0;
    const unsigned long long pol = ef ? l2_evict_first_policy() : 0ull;
    if constexpr (!C::IN_T) {
        const unsigned bytes = (unsigned)(ti.Tv * C::L) * 8u;
        if (lane == 0) mbar_arrive_expect_tx(bar, bytes + d.debug_extra_tx);
        __syncwarp();
        if (C::LLS == C::L && !d.off_in) {
            if (lane == 0) bulk_load_1d(land, src, bytes, bar, d.err, ef, pol);
        } else {
            for (int t = lane; t < ti.Tv; t += 32)
                bulk_load_1d(land + t * C::LLS, line_in(d, ti, src, t), C::L * 8u, bar, d.err, ef, pol);
        }
    } else if (!d.off_in) {
        if (lane == 0) {
            mbar_arrive_expect_tx(bar, (unsigned)(C::T * C::L) * 8u + d.debug_extra_tx);
            for (int n0 = 0; n0 < C::L; n0 += C::BR)
                tma_load_3d(land + n0 * C::T, tm, (int)ti.c0, n0, (int)ti.o, bar, d.err, ef, pol);
        }
    } else {
        // irregular transform bases: one bulk copy per row of Tv columns
        if (lane == 0) mbar_arrive_expect_tx(bar, (unsigned)(ti.Tv * C::L) * 8u + d.debug_extra_tx);
        __syncwarp();
        for (int n = lane; n < C::L; n += 32)
            bulk_load_1d(land + n * C::T, src + (long long)n * d.in_sn, (unsigned)ti.Tv * 8u, bar, d.err, ef, pol);
    }
}
// Producer warp (all lanes): start the TMA stores of one finished tile.
template <int THREADS, int LG, int IO>
__device__ __forceinline__ void p2_issue_store(const PassDesc& d, const CUtensorMap* tm, long long tile,
                                               const float2* land, int lane)
{
    using C = P2<THREADS, LG, IO>;
    const TileIdx ti = p2_tile_index(d, tile, C::LOGT, C::T);
    float2* dst = tile_out_base(d, ti, C::OUT_T);
    // output the next pass of this exec reads again, small enough to stay in L2
    const bool el = d.evict_last != 0;
    const unsigned long long pol = el ? l2_evict_last_policy() : 0ull;
    if constexpr (!C::OUT_T) {
        if (C::OLS == C::L && !d.off_out) {
            if (lane == 0) bulk_store_1d(dst, land, (unsigned)(ti.Tv * C::L) * 8u, d.err, el, pol);
        } else {
            for (int t = lane; t < ti.Tv; t += 32)
                bulk_store_1d(line_out(d, ti, dst, t), land + t * C::OLS, C::L * 8u, d.err, el, pol);
        }
    } else if (!d.off_out) {
        if (lane == 0)
            for (int k0 = 0; k0 < C::L; k0 += C::BR)
                tma_store_3d(tm, (int)ti.c0, k0, (int)ti.o, land + k0 * C::T, d.err, el, pol);
    } else {
        for (int k = lane; k < C::L; k += 32)
            bulk_store_1d(dst + (long long)k * d.out_sk, land + k * C::T, (unsigned)ti.Tv * 8u, d.err, el, pol);
    }
    bulk_commit();
}

// Plain-copy fallback (misaligned bases, odd strides).
template <int THREADS, int LG, int IO>
__device__ __forceinline__ void p2_plain_load(const PassDesc& d, const TileIdx& ti, float2* land)
{
    using C = P2<THREADS, LG, IO>;
    const float2* gin = tile_in_base(d, ti, C::IN_T);
    if constexpr (!C::IN_T) {
        for (int e = threadIdx.x; e < ti.Tv * C::L; e += THREADS) {
            const int t = e >> LG, n = e & (C::L - 1);
            land[t * C::LLS + n] = line_in(d, ti, gin, t)[(long long)n * d.in_sn];
        }
    } else {
        for (int e = threadIdx.x; e < C::T * C::L; e += THREADS) {
            const int n = e >> C::LOGT, t = e & (C::T - 1);
            if (t < ti.Tv) land[e] = gin[(long long)n * d.in_sn + t];
        }
    }
}
template <int THREADS, int LG, int IO>
__device__ __forceinline__ void p2_plain_store(const PassDesc& d, const TileIdx& ti, const float2* land)
{
    using C = P2<THREADS, LG, IO>;
    float2* gout = tile_out_base(d, ti, C::OUT_T);
    if constexpr (!C::OUT_T) {
        for (int e = threadIdx.x; e < ti.Tv * C::L; e += THREADS) {
            const int t = e >> LG, k = e & (C::L - 1);
            line_out(d, ti, gout, t)[(long long)k * d.out_sk] = land[t * C::OLS + k];
        }
    } else {
        for (int e = threadIdx.x; e < C::T * C::L; e += THREADS) {
            const int k = e >> C::LOGT, t = e & (C::T - 1);
            if (t < ti.Tv) gout[(long long)k * d.out_sk + t] = land[e];
        }
    }
}

// Register split.  Three-stage schedules (L >= 512) need ~124 registers per
// compute thread, but with one producer warp beside 8 or 16 compute warps one
// SM sub-partition holds 5 warps and the cap is 96 (16384 registers each).
// Those kernels get a whole producer warpgroup instead: it lowers its
// registers to 24 (setmaxnreg.dec) and the compute warps raise theirs from
// the launch count to what the released registers allow (setmaxnreg.inc),
// per sub-partition: 4 x 112 + 24 <= 5 x 96 (512 threads, 1 CTA per SM),
// 2 x (2 x 104 + 24) <= 2 x 3 x 80 (256 threads, 2 CTAs per SM).
__host__ __device__ constexpr bool p2_split(int lg) { return pow2_nst(lg) >= 3; }
__host__ __device__ constexpr int p2_producer_threads(int lg) { return p2_split(lg) ? 128 : 32; }
__host__ __device__ constexpr int p2_launch_regs(int threads, int lg)
{
    return p2_split(lg) ? (threads == 512 ? 96 : 80) : 96;
}
template <int THREADS, int LG>
struct P2Regs {
    static constexpr bool SPLIT = p2_split(LG);
    static constexpr int PRODUCER_THREADS = p2_producer_threads(LG);
    static constexpr int LAUNCH = p2_launch_regs(THREADS, LG);
    static constexpr int PRODUCER = 24;
    static constexpr int COMPUTE =
        SPLIT ? ((THREADS + PRODUCER_THREADS) * LAUNCH - PRODUCER_THREADS * PRODUCER) / THREADS / 8 * 8 : LAUNCH;
    static_assert(THREADS * COMPUTE + PRODUCER_THREADS * PRODUCER <= (THREADS + PRODUCER_THREADS) * LAUNCH,
                  "register split exceeds the CTA's launch allocation");
    static_assert(!SPLIT || (THREADS == 256 || THREADS == 512), "register split sized for 256 or 512 threads");
};

// The power-of-two line pass.  THREADS compute threads plus one producer warp
// (or warpgroup, see the register split).  Persistent CTAs walk tiles
// blockIdx.x, +gridDim.x, ...  With TMA on (d.async_io) the producer warp owns
// every copy: it loads tile i into landing buffer i % NBUF (mbarrier full[b],
// counted in bytes), and once the compute warps release a buffer (mbarrier
// empty[b]) it stores the finished tile and reloads the buffer with tile
// i + NBUF.  Compute warps only wait for `full` and synchronise among
// themselves on a named barrier, so copy bookkeeping never stalls them.
// Every wait is bounded.  TC: radix-16 stages on the tensor cores
// (fft_tc.cuh); the CTA then also holds B^T (4 KB after the work buffer;
// its stage twiddles stay in global memory)
// and tc_tmem_cols(THREADS) TMEM columns, allocated by compute warp 0 and
// freed before it exits.
template <int THREADS, bool FWD, int LG, int IO, bool TC = false>
__global__ void __maxnreg__((P2Regs<THREADS, LG>::LAUNCH)) k_fft_p2(const __grid_constant__ LineArgs a)
{
    using C = P2<THREADS, LG, IO>;
    const PassDesc& d = a.d;
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    constexpr int NBUF = C::NBUF;
    unsigned long long* full = reinterpret_cast<unsigned long long*>(smem_raw);            // [NBUF]
    unsigned long long* empty = reinterpret_cast<unsigned long long*>(smem_raw) + NBUF;    // [NBUF]
    unsigned long long* mma_bar = reinterpret_cast<unsigned long long*>(smem_raw) + 2 * NBUF;
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(mma_bar + 1);
    static_assert(8 * (2 * NBUF + 1) + 4 <= 128, "barriers fit the 128-byte header");
    float2* land0 = reinterpret_cast<float2*>(smem_raw + 128);
    const bool async = d.async_io != 0;
    float2* work = land0 + (async ? NBUF : 1) * C::LAND;
    // stage twiddles (when small) follow the work buffer
    float2* tws = work + (C::NST > 1 ? C::T * C::LS : 0);
    const long long step = gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kProducer = THREADS / 32;
    if (async && threadIdx.x == 0) {
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], THREADS);
        }
    }
    if (TC && threadIdx.x == 0) mbar_init(mma_bar, 1);
    if ((async || TC) && threadIdx.x == 0) fence_mbar_init();
    __syncthreads();
    pdl_start();

    using RG = P2Regs<THREADS, LG>;
    if (warp >= kProducer) {
        if constexpr (RG::SPLIT) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(RG::PRODUCER));
        if (warp != kProducer || !async) return;  // the rest of a producer warpgroup has nothing to do
        // ---- producer warp ----
        bool ok = true;
        int i = 0;
        long long tile = blockIdx.x;
        for (; tile < d.ntiles; tile += step, ++i) {
            const int b = i % NBUF;
            if (i >= NBUF) {  // buffer b still holds tile i-NBUF: wait until it is computed, store it
                ok = mbar_wait_bounded(&empty[b], (unsigned)((i - NBUF) / NBUF) & 1u);
                if (!ok) break;
                p2_issue_store<THREADS, LG, IO>(d, &a.tm_out, tile - NBUF * step, land0 + b * C::LAND, lane);
                bulk_wait_read_all();  // the store has read the buffer
                __syncwarp();
            }
            p2_issue_load<THREADS, LG, IO>(d, &a.tm_in, tile, land0 + b * C::LAND, &full[b], lane);
        }
        // drain: store the last (up to NBUF) tiles once computed
        for (int k = (i >= NBUF ? i - NBUF : 0); ok && k < i; ++k) {
            const int b = k % NBUF;
            ok = mbar_wait_bounded(&empty[b], (unsigned)(k / NBUF) & 1u);
            if (ok) p2_issue_store<THREADS, LG, IO>(d, &a.tm_out, blockIdx.x + (long long)k * step,
                                                    land0 + b * C::LAND, lane);
        }
        if (!ok && lane == 0) atomicExch(d.err, 1);
        bulk_wait_all();
        return;
    }

    // ---- compute warps ----
    if constexpr (RG::SPLIT) asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(RG::COMPUTE));
    TcState tc{0u, mma_bar, 0u, 0u, 0u};
    if constexpr (TC) {
        unsigned char* bmat = reinterpret_cast<unsigned char*>(
            (reinterpret_cast<uintptr_t>(tws) + 127) & ~static_cast<uintptr_t>(127));
        if (warp == 0) tc_alloc<tc_tmem_cols(THREADS)>(tmem_slot);
        tc_build_b<THREADS, FWD>(bmat);
        fence_proxy_async();  // B^T -> visible to the tensor cores
        tc_fence_before();
        compute_sync<THREADS>();
        tc_fence_after();
        tc.tmem = *tmem_slot;
        tc.bsm = smem_u32(bmat);
        tc.a = tc.tmem + 32u * (THREADS / 128);  // A rows after the accumulators
    }
    if constexpr (C::TWS > 0 && !TC) {
        p2_copy_twiddles<THREADS, LG, 1>(d, tws);
        compute_sync<THREADS>();
    }
    if constexpr (C::PTW && !TC) {
        if (d.ptw_smem) {  // four-step tables: lo then hi, behind the stage twiddles
            float2* pt = tws + C::TWS;
            const int lo = 1 << d.ptw_log;
            for (int e = threadIdx.x; e < lo; e += THREADS) pt[ptw_pad(e)] = __ldg(d.ptw_lo + e);
            for (int e = threadIdx.x; e < d.ptw_hi_cnt; e += THREADS) pt[ptw_pad(lo + e)] = __ldg(d.ptw_hi + e);
            compute_sync<THREADS>();
        }
    }
    int i = 0;
    for (long long tile = blockIdx.x; tile < d.ntiles; tile += step, ++i) {
        const TileIdx ti = p2_tile_index(d, tile, C::LOGT, C::T);
        const int buf = async ? (i % NBUF) : 0;
        float2* land = land0 + buf * C::LAND;
        const int c0 = (int)ti.c0;
        if (async) {
            const bool bad = !mbar_wait_bounded(&full[buf], (unsigned)(i / NBUF) & 1u);
            if (compute_sync_or<THREADS>(bad)) {
                if (threadIdx.x == 0) atomicExch(d.err, 1);
                break;  // the producer's own bounded waits end it
            }
        } else {
            p2_plain_load<THREADS, LG, IO>(d, ti, land);
            compute_sync<THREADS>();
        }
        p2_run_stage<THREADS, FWD, LG, IO, 0, TC>(d, land, work, ti.Tv, c0, tws, tc);
        if constexpr (C::NST == 1) {
            if (async) fence_proxy_async();
        } else {
            compute_sync<THREADS>();
        }
        p2_stages_from<THREADS, FWD, LG, IO, 1, TC>(d, land, work, ti.Tv, c0, async, tws, tc);
        if (async) {
            mbar_arrive(&empty[buf]);  // after this thread's proxy fence
        } else {
            compute_sync<THREADS>();
            p2_plain_store<THREADS, LG, IO>(d, ti, land);
            compute_sync<THREADS>();
        }
    }
    if constexpr (TC) {
        tc_fence_before();
        compute_sync<THREADS>();
        if (warp == 0) {
            tc_fence_after();
            tc_dealloc<tc_tmem_cols(THREADS)>(tc.tmem);
        }
    }
}

template <int THREADS, bool FWD, int LG, int IO, bool TC = false>
LineKernel p2_entry()
{
    LineKernel k = make_entry<THREADS>(k_fft_p2<THREADS, FWD, LG, IO, TC>, FWD, LG, IO);
    k.threads = THREADS + P2Regs<THREADS, LG>::PRODUCER_THREADS;  // compute warps + producer warp(s)
    k.producers = P2Regs<THREADS, LG>::PRODUCER_THREADS;
    k.split_regs = P2Regs<THREADS, LG>::SPLIT ? P2Regs<THREADS, LG>::LAUNCH : 0;
    k.tc = TC;
    return k;
}

}  // namespace fbfft
